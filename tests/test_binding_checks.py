"""Argument checks of the Python binding, on CPU: a buffer of the wrong element
type or size, or a tensor on another GPU than the context's, is rejected
before its pointer reaches the library (whose kernels would otherwise read or
write outside it).  No library call is made: the handles are stand-ins."""
import types

import numpy as np
import pytest

import paper_1801_07823_gb300 as sw


def _gauge(L0=8, L1=4, device=0):
    return types.SimpleNamespace(ptr=None, ctx_ptr=None, shape=(L1, L0), device=device)


def test_wrong_dtype_is_rejected():
    g = _gauge()
    ok = np.zeros(32, dtype=np.complex128)
    with pytest.raises(ValueError, match="complex128"):
        sw.sw_dslash(g, 0.1, sw.SW_OP_D, sw.SW_PREC_FP64, np.zeros(32, dtype=np.complex64), ok)
    with pytest.raises(ValueError, match="complex64"):
        sw.sw_dslash(g, 0.1, sw.SW_OP_D, sw.SW_PREC_FP32, ok, ok.copy())


def test_wrong_size_is_rejected():
    g = _gauge()
    with pytest.raises(ValueError, match="elements"):
        sw.sw_dslash(g, 0.1, sw.SW_OP_D, sw.SW_PREC_FP64, np.zeros(31, dtype=np.complex128),
                     np.zeros(32, dtype=np.complex128))
    mg = types.SimpleNamespace(ptr=None, ctx_ptr=None, shape=(4, 8), device=0)
    with pytest.raises(ValueError, match="elements"):
        sw.sw_mg_solve(mg, np.zeros(32, dtype=np.complex128), np.zeros(16, dtype=np.complex128), 1e-10)
    with pytest.raises(ValueError, match="elements"):
        sw.sw_mg_solve_batch(mg, np.zeros((3, 32), dtype=np.complex128),
                             np.zeros((2, 32), dtype=np.complex128), 1e-10)
    with pytest.raises(ValueError):
        sw.sw_dslash_schur_noalloc(g, 0.1, np.zeros(32, dtype=np.complex128),
                                   np.zeros(32, dtype=np.complex128))


def test_tensor_on_another_device_is_rejected():
    h = types.SimpleNamespace(device=0)
    fake = types.SimpleNamespace(dtype="torch.complex128", numel=lambda: 32, is_cuda=True,
                                 device=types.SimpleNamespace(index=1))
    with pytest.raises(ValueError, match="cuda:1"):
        sw._check_buf(h, fake, 32, "complex128", "in")
    same = types.SimpleNamespace(dtype="torch.complex128", numel=lambda: 32, is_cuda=True,
                                 device=types.SimpleNamespace(index=0))
    sw._check_buf(h, same, 32, "complex128", "in")


def test_psi0_shapes_are_checked():
    g = types.SimpleNamespace(ptr=None, ctx_ptr=None, shape=(16, 16), device=0)
    good0 = np.zeros((2, 256), dtype=np.complex128)
    bad1 = np.zeros((3, 5), dtype=np.complex128)
    with pytest.raises(ValueError, match="psi0"):
        sw.sw_mg_setup(g, 0.1, 3, [(2, 2), (2, 2)], [2, 3], psi0=[good0, bad1])
