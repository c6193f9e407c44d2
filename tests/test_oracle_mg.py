"""Pins of the oracle's Krylov solvers and multigrid setup/solve."""
import numpy as np
import pytest
import scipy.sparse as sp

import sw_inputs as si
from oracle import krylov, lattice, mg, operators


def rand_theta(L, seed):
    return np.random.default_rng(seed).uniform(-np.pi, np.pi, (2, L, L))


def psi0_for(L, nvec, levels, seed=5, blocks=((4, 4), (2, 2))):
    out = [[si.gaussian_complex(si.stream_seed(seed, 0, i), L * L) for i in range(nvec[0])]]
    if levels >= 3:
        E = L // (2 * blocks[0][0])
        out.append([si.gaussian_complex(si.stream_seed(seed, 1, i), E * E * 2 * nvec[0])
                     for i in range(nvec[1])])
    return out


# ---------------------------------------------------------------- Krylov
def test_krylov_methods_on_small_systems():
    rng = np.random.default_rng(0)
    n = 40
    M = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    M = np.eye(n) * 12 + M
    b = rng.normal(size=n) + 1j * rng.normal(size=n)
    xs = np.linalg.solve(M, b)
    H = M.conj().T @ M
    x, k = krylov.cg(lambda v: H @ v, M.conj().T @ b, 1e-12, 500)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-9
    x, k = krylov.cgne(lambda v: M @ v, lambda v: M.conj().T @ v, b, 1e-12, 500)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-9
    x, it, rs, conv = krylov.fgcr(lambda v: M @ v, lambda r: r, b, 1e-12 * np.linalg.norm(b), 8, 500)
    assert conv and np.linalg.norm(b - M @ x) <= 1e-12 * np.linalg.norm(b)
    # one MR step is the exact minimiser of ||b - alpha M b||, relaxed by omega
    x, r = krylov.mr(lambda v: M @ v, b, 1, 1.0)
    q = M @ b
    alpha = np.vdot(q, b) / np.vdot(q, q)
    assert np.allclose(x, alpha * b) and np.allclose(r, b - M @ x)
    a2 = np.linspace(-2, 2, 41)
    best = min(np.linalg.norm(b - (alpha.real + t) * q) for t in a2 * 1e-3)
    assert np.linalg.norm(r) <= best + 1e-12
    # CG stops at the requested tolerance
    x, k = krylov.cg(lambda v: H @ v, M.conj().T @ b, 1e-4, 500)
    rr = np.linalg.norm(M.conj().T @ b - H @ x) / np.linalg.norm(M.conj().T @ b)
    assert rr <= 1e-4 and k < 500


# ---------------------------------------------------------------- setup
@pytest.fixture(scope="module")
def hier16():
    L = 16
    th = si.heatbath_u1(L, L, 3.0, 30, seed=21)
    H = mg.Hierarchy(th, 0.05, 2, [(4, 4)], [6], psi0_for(L, [6], 2))
    return th, H


def test_prolongator_orthonormal_and_chiral(hier16):
    th, H = hier16
    P = H.levels[0].P.toarray()
    assert np.max(np.abs(P.conj().T @ P - np.eye(P.shape[1]))) < 1e-14
    eps = H.F.eps.astype(float)
    nv = 6
    sigma3 = np.tile(np.concatenate([np.ones(nv), -np.ones(nv)]), P.shape[1] // (2 * nv))
    assert np.max(np.abs(eps[:, None] * P - P * sigma3[None, :])) < 1e-15   # eps P = P sigma3
    # support: column (X, c, i) lives on aggregate X
    agg = lattice.fine_aggregate(16, 16, 4, 4)
    cols_agg = np.arange(P.shape[1]) // (2 * nv)
    assert np.all(np.abs(P[agg[:, None] != cols_agg[None, :]]) == 0)


def test_null_vectors_in_range_and_near_null():
    L = 16
    th = si.heatbath_u1(L, L, 3.0, 30, seed=22)
    p0 = psi0_for(L, [4], 2, seed=9)
    F = operators.FineOperators(th, 0.05)
    vecs, its = mg.near_null_vectors(lambda v: F.A @ v, lambda v: F.Adag @ v, p0[0], mg.Params())
    H = mg.Hierarchy(th, 0.05, 2, [(4, 4)], [4], p0)
    P = H.levels[0].P.toarray()
    for v in vecs:
        assert np.linalg.norm(v - P @ (P.conj().T @ v)) / np.linalg.norm(v) < 1e-13
    # the relaxation lowers the Rayleigh quotient of A A^dag by a large factor
    AAd = lambda v: F.A @ (F.Adag @ v)
    for v, v0 in zip(vecs, p0[0]):
        q0 = np.vdot(v0, AAd(v0)).real / np.vdot(v0, v0).real
        q = np.vdot(v, AAd(v)).real / np.vdot(v, v).real
        assert q < 0.05 * q0


def test_coarse_operator_is_dense_galerkin(hier16):
    """Sec. III: A_hat = P^dag A P, checked column by column with dense matrices."""
    th, H = hier16
    P = H.levels[0].P.toarray()
    A = H.F.A.toarray()
    Ah = H.levels[1].op.toarray()
    for j in range(0, P.shape[1], 5):
        col = P.conj().T @ (A @ P[:, j])
        assert np.max(np.abs(Ah[:, j] - col)) < 1e-13
    # the stencil is nearest neighbour on the coarse lattice (2x2 coarse sites here,
    # so every pair of coarse sites is a neighbour) and the coarse dof follow sigma3
    assert H.levels[1].extent == (2, 2)


def test_gauge_invariance_of_the_hierarchy():
    """Setup on (U^g, G psi0) gives P' = G P and the same A_hat, because CG,
    the chiral projectors and Gram-Schmidt commute with the diagonal unitary G."""
    L = 16
    th = si.heatbath_u1(L, L, 6.0, 20, seed=23)
    alpha = np.random.default_rng(3).uniform(-np.pi, np.pi, (L, L))
    g = np.exp(1j * alpha.ravel())
    p0 = psi0_for(L, [4, 6], 3, seed=4, blocks=((2, 2), (2, 2)))
    # a fixed number of CG steps, so both setups stop at the same iteration
    prm = mg.Params(setup_tol=0.0, setup_maxiter=12)
    H1 = mg.Hierarchy(th, 0.1, 3, [(2, 2), (2, 2)], [4, 6], p0, prm)
    p0g = [[g * v for v in p0[0]], p0[1]]
    H2 = mg.Hierarchy(si.gauge_transform(th, alpha), 0.1, 3, [(2, 2), (2, 2)], [4, 6], p0g, prm)
    P1, P2 = H1.levels[0].P.toarray(), H2.levels[0].P.toarray()
    assert np.max(np.abs(P2 - g[:, None] * P1)) < 1e-11
    for l in (1, 2):
        a, b = H1.levels[l].op.toarray(), H2.levels[l].op.toarray()
        assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(a))


# ---------------------------------------------------------------- solve
def test_two_level_solve_matches_dense():
    L = 16
    th = si.heatbath_u1(L, L, 3.0, 30, seed=24)
    H = mg.Hierarchy(th, 0.02, 2, [(2, 2)], [6], psi0_for(L, [6], 2, blocks=((2, 2),)))
    b = si.gaussian_complex(1001, L * L)
    x, st = H.solve(b, 1e-10)
    D = operators.dirac(th, 0.02).toarray()
    xd = np.linalg.solve(D, b)
    assert st["converged"] and st["true_resid"] <= 1e-10
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
    assert np.linalg.norm(b - D @ x) / np.linalg.norm(b) <= 1e-10


@pytest.mark.slow
def test_three_level_solve_converges():
    L = 32
    th = si.heatbath_u1(L, L, 6.0, 40, seed=25)
    H = mg.Hierarchy(th, 0.01, 3, [(4, 4), (2, 2)], [8, 12], psi0_for(L, [8, 12], 3))
    b = si.gaussian_complex(1002, L * L)
    x, st = H.solve(b, 1e-10)
    assert st["converged"] and st["true_resid"] <= 1e-10
    assert st["inter_solves"] == st["outer_iters"] and st["coarsest_solves"] == st["inter_iters"]
    # six Schur applications per outer iteration (MR 2 + 1 + MR 2 + GCR 1)
    assert st["fine_applies"] >= 6 * st["outer_iters"]


def test_galerkin_mg_of_D_stalls():
    """Sec. III.B, Fig. residstag: the same recipe applied to D itself (P^dag D P)
    stalls, while coarsening the KD-preconditioned A converges (oracle)."""
    L = 32
    th = si.heatbath_u1(L, L, 6.0, 100, seed=26)
    p0 = psi0_for(L, [8, 12], 3)
    b = si.gaussian_complex(1003, L * L)
    prm = mg.Params(outer_maxiter=30)
    HA = mg.Hierarchy(th, 0.01, 3, [(4, 4), (2, 2)], [8, 12], p0, prm)
    HD = mg.Hierarchy(th, 0.01, 3, [(4, 4), (2, 2)], [8, 12], p0, prm, fine_op="D")
    _, sa = HA.solve(b, 1e-10)
    _, sd = HD.solve(b, 1e-10)
    assert sa["converged"] and sa["outer_iters"] < 30
    assert not sd["converged"] and sd["true_resid"] > 0.1
    # the D hierarchy is the literal Galerkin product of D
    P = HD.levels[0].P.toarray()
    Dd = HD.F.D.toarray()
    Ah = HD.levels[1].op.toarray()
    assert np.max(np.abs(Ah - P.conj().T @ Dd @ P)) < 1e-13
