"""GPU parity of the fine operators and integer maps against the oracle."""
import numpy as np
import pytest

import sw_inputs as si
from oracle import lattice, operators
from tests.gpu_helpers import relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    import paper_1801_07823_gb300 as m
    return m


@pytest.fixture(scope="module")
def ctx(sw):
    c = sw.sw_context_create(0)
    yield c
    c.free()


SHAPES = [(16, 16), (12, 20), (64, 32), (256, 256)]


@pytest.mark.parametrize("L0,L1", SHAPES)
def test_fine_operators_fp64(sw, ctx, L0, L1):
    """Eq. staggeredD, Eq. defA and the Schur operator, <= 1e-13 relative."""
    m = 0.07
    th = np.random.default_rng(L0 + L1).uniform(-np.pi, np.pi, (2, L1, L0))
    g = sw.sw_gauge_load(ctx, th)
    F = operators.FineOperators(th, m)
    v = si.gaussian_complex(17, L0 * L1)
    refs = {sw.SW_OP_D: F.D @ v, sw.SW_OP_DDAG: F.D.conj().T @ v, sw.SW_OP_A: F.A @ v,
            sw.SW_OP_ADAG: F.Adag @ v}
    s = np.zeros_like(v)
    s[F.even] = F.schur(v[F.even])
    refs[sw.SW_OP_S] = s
    for op, ref in refs.items():
        out = np.full_like(v, np.nan)
        sw.sw_dslash(g, m, op, sw.SW_PREC_FP64, v, out)
        assert relerr(out, ref) < 1e-13, (op, relerr(out, ref))
    g.free()


def test_dslash_fp32(sw, ctx):
    L0, L1, m = 64, 48, 0.1
    th = np.random.default_rng(3).uniform(-np.pi, np.pi, (2, L1, L0))
    g = sw.sw_gauge_load(ctx, th)
    v = si.gaussian_complex(4, L0 * L1)
    ref = operators.dirac(th, m) @ v
    out = np.zeros(L0 * L1, dtype=np.complex64)
    sw.sw_dslash(g, m, sw.SW_OP_D, sw.SW_PREC_FP32, v.astype(np.complex64), out)
    assert relerr(out.astype(complex), ref) < 2e-6
    g.free()


def test_device_buffers_and_large_lattice(sw, ctx):
    """The device-pointer path at 1024^2, on torch CUDA tensors."""
    import torch
    L = 1024
    th = np.random.default_rng(5).uniform(-np.pi, np.pi, (2, L, L))
    g = sw.sw_gauge_load(ctx, torch.from_numpy(th).cuda())
    v = si.gaussian_complex(6, L * L)
    vin = torch.from_numpy(v).cuda()
    out = torch.empty_like(vin)
    for op, mat in ((sw.SW_OP_D, operators.dirac(th, 0.01)),):
        sw.sw_dslash(g, 0.01, op, sw.SW_PREC_FP64, vin, out)
        torch.cuda.synchronize()
        assert relerr(out.cpu().numpy(), mat @ v) < 1e-13
    g.free()


def test_maps_bit_exact(sw, ctx):
    L0, L1 = 24, 16
    g = sw.sw_gauge_load(ctx, np.zeros((2, L1, L0)))
    mp = sw.sw_debug_maps(g, 2, 2)
    assert np.array_equal(mp["eta"], lattice.eta(L0, L1))
    assert np.array_equal(mp["eps"], lattice.epsilon(L0, L1))
    assert np.array_equal(mp["kd_block"], lattice.kd_block(L0, L1))
    assert np.array_equal(mp["kd_parity"], lattice.kd_parity(L0, L1))
    assert np.array_equal(mp["agg"], lattice.fine_aggregate(L0, L1, 2, 2))
    g.free()


def test_argument_errors(sw, ctx):
    th = np.zeros((2, 16, 16))
    g = sw.sw_gauge_load(ctx, th)
    v = np.zeros(256, dtype=complex)
    with pytest.raises(sw.SwError) as e:
        sw.sw_dslash(g, 0.0, sw.SW_OP_A, sw.SW_PREC_FP64, v, v.copy())
    assert e.value.code == -1
    with pytest.raises(sw.SwError) as e:
        sw.sw_mg_setup(g, -0.1, 2, [(2, 2)], [4])
    assert e.value.code == -1
    with pytest.raises(sw.SwError) as e:
        sw.sw_mg_setup(g, 0.1, 2, [(3, 3)], [4])
    assert e.value.code == -2
    with pytest.raises(sw.SwError) as e:
        sw.sw_gauge_load(ctx, np.zeros((2, 10, 12)))
    assert e.value.code == -2
    g.free()


def test_cg_even_odd_parity(sw, ctx):
    """The comparison CG on the GPU against the oracle's: same stopping rule,
    iterations within 3 %, solution within the solve tolerance."""
    L, m = 64, 0.02
    th = si.heatbath_u1(L, L, 6.0, 50, seed=9, device="cuda")
    g = sw.sw_gauge_load(ctx, th)
    b = si.gaussian_complex(88, L * L)
    x = np.zeros_like(b)
    st = sw.sw_cg_eo_solve(g, m, b, x, 1e-10)
    xo, k = operators.cg_eo_solve(th, m, b, 1e-10, 100000)
    D = operators.dirac(th, m)
    assert st["converged"] and np.linalg.norm(b - D @ x) / np.linalg.norm(b) <= 1e-10
    assert abs(st["outer_iters"] - k) <= max(3, 0.03 * k), (st["outer_iters"], k)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-7
    g.free()


@pytest.mark.parametrize("L0,L1", [(16, 16), (12, 20), (64, 32)])
def test_naik_operators(sw, ctx, L0, L1):
    """Naik-improved D (Eq. freehisq, gauged with the path's links) and its KD
    form D_Naik B_Naik^-1 against the oracle, <= 1e-13 relative."""
    m = 0.05
    th = np.random.default_rng(L0 * L1).uniform(-np.pi, np.pi, (2, L1, L0))
    g = sw.sw_gauge_load(ctx, th)
    Dn, Bn, An = operators.naik_kd_operator(th, m)
    v = si.gaussian_complex(23, L0 * L1)
    for op, mat in ((sw.SW_OP_DNAIK, Dn), (sw.SW_OP_ANAIK, An)):
        out = np.zeros_like(v)
        sw.sw_dslash(g, m, op, sw.SW_PREC_FP64, v, out)
        assert relerr(out, mat @ v) < 1e-13, (op, relerr(out, mat @ v))
    g.free()
