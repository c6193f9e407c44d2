"""Python binding of libsw (include/sw.h): ctypes argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays may be
numpy arrays (host memory, on_device = 0) or torch CUDA tensors (device
memory, on_device = 1); complex fields are complex128 (complex64 for the FP32
Dslash).  All compute runs in the CUDA library; there is no fallback: if
libsw.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = [
    "SwError", "lib", "SW_OP_D", "SW_OP_DDAG", "SW_OP_A", "SW_OP_ADAG", "SW_OP_S", "SW_OP_DNAIK",
    "SW_OP_ANAIK",
    "SW_PREC_FP64", "SW_PREC_FP32", "SW_PREC_FP16S", "SW_PREC_DF64", "SW_MG_FP64", "SW_MG_MIXED", "SW_MG_COARSEN_A", "SW_MG_COARSEN_D",
    "sw_context_create", "sw_context_free", "sw_last_error",
    "sw_gauge_load", "sw_gauge_free", "sw_dslash", "sw_mg_params_default", "sw_mg_setup",
    "sw_mg_free", "sw_mg_solve", "sw_mg_solve_batch", "sw_debug_maps", "sw_mg_level_info",
    "sw_mg_export_P", "sw_mg_export_Y", "sw_mg_apply_level", "sw_mg_transfer",
    "sw_stream_seed", "sw_set_timing", "sw_kernel_times", "sw_launch_count",
    "sw_dslash_schur_noalloc", "sw_debug_cgne_stall", "sw_cg_eo_solve", "sw_debug_batch_stall",
    "sw_autotune_entries", "sw_mg_level_maps", "sw_context_set_sm_share", "sw_fp64_peak",
]

SW_OP_D, SW_OP_DDAG, SW_OP_A, SW_OP_ADAG, SW_OP_S, SW_OP_DNAIK, SW_OP_ANAIK = 0, 1, 2, 3, 4, 5, 6
SW_PREC_FP64, SW_PREC_FP32, SW_PREC_FP16S, SW_PREC_DF64 = 0, 1, 2, 3
SW_MG_FP64, SW_MG_MIXED = 0, 1
SW_MG_COARSEN_A, SW_MG_COARSEN_D = 0, 1
ERRORS = {0: "SW_OK", -1: "SW_ERR_ARG", -2: "SW_ERR_SHAPE", -3: "SW_ERR_OOM", -4: "SW_ERR_NOCONV",
          -5: "SW_ERR_BREAKDOWN", -6: "SW_ERR_NAN", -7: "SW_ERR_CUDA", -8: "SW_ERR_TIMEOUT"}
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsw.so")


class SwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class sw_mg_params(ctypes.Structure):
    _fields_ = [("setup_maxiter", ctypes.c_int), ("setup_tol", ctypes.c_double),
                ("setup_passes", ctypes.c_int), ("outer_restart", ctypes.c_int),
                ("outer_maxiter", ctypes.c_int), ("smoother_iters", ctypes.c_int),
                ("omega", ctypes.c_double), ("inter_restart", ctypes.c_int),
                ("inter_maxiter", ctypes.c_int), ("inter_tol", ctypes.c_double),
                ("coarsest_maxiter", ctypes.c_int), ("coarsest_tol", ctypes.c_double),
                ("precision", ctypes.c_int), ("fine_operator", ctypes.c_int),
                ("batch_iterates", ctypes.c_int)]


class sw_solve_stats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("restarts", ctypes.c_int), ("fine_applies", ctypes.c_longlong),
                ("inter_iters", ctypes.c_longlong), ("inter_solves", ctypes.c_longlong),
                ("coarsest_iters", ctypes.c_longlong), ("coarsest_solves", ctypes.c_longlong),
                ("true_resid", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None
_VP, _I, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double


def lib():
    """The loaded libsw.so (raises if it is not built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "sw_context_create": (_I, [_I, _VP, ctypes.POINTER(_VP)]),
            "sw_context_free": (None, [_VP]),
            "sw_last_error": (ctypes.c_char_p, [_VP]),
            "sw_gauge_load": (_I, [_VP, _I, _I, _VP, _I, ctypes.POINTER(_VP)]),
            "sw_gauge_free": (None, [_VP]),
            "sw_dslash": (_I, [_VP, _D, _I, _I, _VP, _VP, _I]),
            "sw_mg_params_default": (None, [ctypes.POINTER(sw_mg_params)]),
            "sw_mg_setup": (_I, [_VP, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(sw_mg_params), ctypes.c_uint64,
                                 ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
            "sw_mg_free": (None, [_VP]),
            "sw_mg_solve": (_I, [_VP, _VP, _VP, _D, _I, ctypes.POINTER(sw_solve_stats)]),
            "sw_mg_solve_batch": (_I, [_VP, _I, _VP, _VP, _D, _I, ctypes.POINTER(sw_solve_stats)]),
            "sw_debug_maps": (_I, [_VP, _I, _I, _VP, _VP, _VP, _VP, _VP]),
            "sw_mg_level_info": (_I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I),
                                      ctypes.POINTER(_I)]),
            "sw_mg_export_P": (_I, [_VP, _I, _VP]),
            "sw_mg_export_Y": (_I, [_VP, _I, _VP]),
            "sw_mg_apply_level": (_I, [_VP, _I, _I, _I, _VP, _VP, _I]),
            "sw_mg_transfer": (_I, [_VP, _I, _I, _VP, _VP, _I]),
            "sw_stream_seed": (ctypes.c_uint64, [ctypes.c_uint64, _I, _I]),
            "sw_set_timing": (_I, [_VP, _I]),
            "sw_kernel_times": (_I, [_VP, _I, _VP, _VP]),
            "sw_launch_count": (ctypes.c_longlong, []),
            "sw_dslash_schur_noalloc": (_I, [_VP, _D, _VP, _VP]),
            "sw_debug_cgne_stall": (_I, [_VP]),
            "sw_cg_eo_solve": (_I, [_VP, _D, _VP, _VP, _D, _I, _I, ctypes.POINTER(sw_solve_stats)]),
            "sw_debug_batch_stall": (_I, [_VP, _I]),
            "sw_autotune_entries": (_I, [_I, _VP, _VP, _VP, _VP, _VP]),
            "sw_mg_level_maps": (_I, [_VP, _I, _VP, _VP]),
            "sw_context_set_sm_share": (_I, [_VP, _I, _I]),
            "sw_fp64_peak": (_I, [_VP, ctypes.POINTER(_D)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class _Handle:
    """An object returned by the library, with the context it reports errors to."""

    def __init__(self, ptr, ctx_ptr, free):
        self.ptr, self.ctx_ptr, self._free = ptr, ctx_ptr, free

    def free(self):
        if self.ptr:
            self._free(self.ptr)
            self.ptr = None


def _check(rc, ctx_ptr, allow=()):
    if rc != 0 and rc not in allow:
        msg = lib().sw_last_error(ctx_ptr)
        raise SwError(rc, msg.decode() if msg else "")
    return rc


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError("expected a numpy array or a torch tensor")


def _same_place(*arrs):
    places = {_ptr(a)[1] for a in arrs}
    if len(places) != 1:
        raise ValueError("all buffers of one call must be on the host or all on the device")
    return places.pop()


def _dtype_name(a) -> str:
    if isinstance(a, np.ndarray):
        return a.dtype.name
    return str(a.dtype).replace("torch.", "")


def _check_buf(h, a, numel: int, dtype: str = "complex128", what: str = "buffer"):
    """Rejects, before the library sees its pointer, a buffer of the wrong
    element type or size, or a device tensor on another GPU than the one the
    handle's context uses: the kernels would otherwise read or write outside it."""
    if _dtype_name(a) != dtype:
        raise ValueError(f"{what}: expected {dtype}, got {_dtype_name(a)}")
    n = int(a.size) if isinstance(a, np.ndarray) else int(a.numel())
    if n != numel:
        raise ValueError(f"{what}: expected {numel} elements, got {n}")
    if not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False):
        dev = getattr(h, "device", None)
        if dev is not None and a.device.index != dev:
            raise ValueError(f"{what}: tensor is on cuda:{a.device.index}, the context on cuda:{dev}")


def sw_context_create(device: int = 0, stream=None) -> _Handle:
    """stream: a raw cudaStream_t value (e.g. torch.cuda.current_stream().cuda_stream) or None."""
    out = _VP()
    rc = lib().sw_context_create(device, stream or None, ctypes.byref(out))
    if rc != 0:
        raise SwError(rc, "sw_context_create failed")
    h = _Handle(out, out, lib().sw_context_free)
    h.device = int(device)
    return h


def sw_context_free(ctx: _Handle):
    ctx.free()


def sw_last_error(ctx: _Handle) -> str:
    return lib().sw_last_error(ctx.ptr).decode()


def sw_gauge_load(ctx: _Handle, theta) -> _Handle:
    """theta: float64 [2, L1, L0] link angles (numpy or torch CUDA tensor)."""
    if len(theta.shape) != 3 or int(theta.shape[0]) != 2:
        raise ValueError("theta must have shape [2, L1, L0]")
    L1, L0 = int(theta.shape[1]), int(theta.shape[2])
    _check_buf(ctx, theta, 2 * L0 * L1, "float64", "theta")
    p, dev = _ptr(theta)
    out = _VP()
    _check(lib().sw_gauge_load(ctx.ptr, L0, L1, p, dev, ctypes.byref(out)), ctx.ptr)
    h = _Handle(out, ctx.ptr, lib().sw_gauge_free)
    h.shape = (L1, L0)
    h.device = getattr(ctx, "device", None)
    return h


def sw_gauge_free(g: _Handle):
    g.free()


def sw_dslash(g: _Handle, mass: float, op: int, precision: int, inp, out):
    dev = _same_place(inp, out)
    dt = "complex64" if precision == SW_PREC_FP32 else "complex128"
    N = g.shape[0] * g.shape[1]
    _check_buf(g, inp, N, dt, "in")
    _check_buf(g, out, N, dt, "out")
    _check(lib().sw_dslash(g.ptr, float(mass), op, precision, _ptr(inp)[0], _ptr(out)[0], dev),
           g.ctx_ptr)
    return out


def sw_mg_params_default() -> sw_mg_params:
    p = sw_mg_params()
    lib().sw_mg_params_default(ctypes.byref(p))
    return p


def sw_mg_setup(g: _Handle, mass: float, levels: int, block, nvec, params=None, seed: int = 0,
                psi0=None) -> _Handle:
    """block: [(b0, b1)] * (levels-1); nvec: [nv] * (levels-1); psi0: None or a list
    of numpy complex128 arrays [nvec[l], ndof_l] (vector-major)."""
    if len(block) != levels - 1 or len(nvec) != levels - 1:
        raise ValueError("block and nvec need one entry per level below the fine one")
    blk = (_I * (2 * (levels - 1)))(*[int(v) for b in block for v in b])
    nv = (_I * (levels - 1))(*[int(v) for v in nvec])
    keep = []
    ps = None
    if psi0 is not None:
        if len(psi0) != levels - 1:
            raise ValueError("psi0 needs one array per level below the coarsest")
        ps = (_VP * (levels - 1))()
        L1, L0 = g.shape
        E0, E1, ndof = L0, L1, L0 * L1
        for l, arr in enumerate(psi0):
            a = np.ascontiguousarray(arr, dtype=np.complex128)
            if a.size != int(nvec[l]) * ndof:
                raise ValueError(f"psi0[{l}]: expected {int(nvec[l])} x {ndof} elements, got {a.size}")
            keep.append(a)
            ps[l] = a.ctypes.data
            b0, b1 = block[l]
            E0, E1 = (E0 // (2 * b0), E1 // (2 * b1)) if l == 0 else (E0 // b0, E1 // b1)
            ndof = E0 * E1 * 2 * int(nvec[l])
    out = _VP()
    prm = ctypes.byref(params) if params is not None else None
    _check(lib().sw_mg_setup(g.ptr, float(mass), levels, blk, nv, prm, seed, ps,
                             ctypes.byref(out)), g.ctx_ptr)
    h = _Handle(out, g.ctx_ptr, lib().sw_mg_free)
    h.shape = g.shape
    h.device = getattr(g, "device", None)
    return h


def sw_mg_free(mg: _Handle):
    mg.free()


def sw_mg_solve(mg: _Handle, b, x, tol: float, allow_noconv: bool = False) -> dict:
    dev = _same_place(b, x)
    N = mg.shape[0] * mg.shape[1]
    _check_buf(mg, b, N, what="b")
    _check_buf(mg, x, N, what="x")
    st = sw_solve_stats()
    rc = _check(lib().sw_mg_solve(mg.ptr, _ptr(b)[0], _ptr(x)[0], float(tol), dev,
                                  ctypes.byref(st)), mg.ctx_ptr,
                allow=(-4,) if allow_noconv else ())
    d = st.as_dict()
    d["rc"] = rc
    return d


def sw_mg_solve_batch(mg: _Handle, B, X, tol: float, allow_noconv: bool = False):
    dev = _same_place(B, X)
    nrhs = int(B.shape[0])
    N = mg.shape[0] * mg.shape[1]
    _check_buf(mg, B, nrhs * N, what="B")
    _check_buf(mg, X, nrhs * N, what="X")
    st = (sw_solve_stats * max(nrhs, 1))()
    _check(lib().sw_mg_solve_batch(mg.ptr, nrhs, _ptr(B)[0], _ptr(X)[0], float(tol), dev, st),
           mg.ctx_ptr, allow=(-4,) if allow_noconv else ())
    return [st[k].as_dict() for k in range(nrhs)]


def sw_debug_maps(g: _Handle, a0: int, a1: int) -> dict:
    L1, L0 = g.shape
    N = L0 * L1
    out = {k: np.zeros(n, dtype=np.int32) for k, n in
           (("eta", 2 * N), ("eps", N), ("kd_block", N), ("kd_parity", N), ("agg", N))}
    _check(lib().sw_debug_maps(g.ptr, a0, a1, *[out[k].ctypes.data for k in
                                                ("eta", "eps", "kd_block", "kd_parity", "agg")]),
           g.ctx_ptr)
    out["eta"] = out["eta"].reshape(2, N)
    return out


def sw_mg_level_info(mg: _Handle, level: int):
    e0, e1, nc = _I(), _I(), _I()
    _check(lib().sw_mg_level_info(mg.ptr, level, ctypes.byref(e0), ctypes.byref(e1),
                                  ctypes.byref(nc)), mg.ctx_ptr)
    return e0.value, e1.value, nc.value


def sw_mg_export_P(mg: _Handle, level: int, nv: int) -> np.ndarray:
    e0, e1, nc = sw_mg_level_info(mg, level)
    P = np.zeros((e0 * e1 * nc, nv), dtype=np.complex128)
    _check(lib().sw_mg_export_P(mg.ptr, level, P.ctypes.data), mg.ctx_ptr)
    return P


def sw_mg_export_Y(mg: _Handle, level: int) -> np.ndarray:
    e0, e1, nc = sw_mg_level_info(mg, level)
    Y = np.zeros((e0 * e1, 5, nc, nc), dtype=np.complex128)
    _check(lib().sw_mg_export_Y(mg.ptr, level, Y.ctypes.data), mg.ctx_ptr)
    return Y


def _level_len(mg: _Handle, level: int) -> int:
    e0, e1, nc = sw_mg_level_info(mg, level)
    return e0 * e1 * nc


def sw_mg_apply_level(mg: _Handle, level: int, precision: int, dagger: int, inp, out):
    dev = _same_place(inp, out)
    n = _level_len(mg, level)
    _check_buf(mg, inp, n, what="in")
    _check_buf(mg, out, n, what="out")
    _check(lib().sw_mg_apply_level(mg.ptr, level, precision, dagger, _ptr(inp)[0], _ptr(out)[0],
                                   dev), mg.ctx_ptr)
    return out


def sw_mg_transfer(mg: _Handle, level: int, direction: int, inp, out):
    dev = _same_place(inp, out)
    nf, nc = _level_len(mg, level), _level_len(mg, level + 1)
    _check_buf(mg, inp, nf if direction == 0 else nc, what="in")
    _check_buf(mg, out, nc if direction == 0 else nf, what="out")
    _check(lib().sw_mg_transfer(mg.ptr, level, direction, _ptr(inp)[0], _ptr(out)[0], dev),
           mg.ctx_ptr)
    return out


def sw_stream_seed(seed: int, level: int, index: int) -> int:
    return int(lib().sw_stream_seed(seed, level, index))


def sw_set_timing(ctx: _Handle, enable: bool):
    _check(lib().sw_set_timing(ctx.ptr, 1 if enable else 0), ctx.ptr)


def sw_kernel_times(ctx: _Handle, n: int = 7):
    """[(launches, total ms)] per timing category (0: fine S, l: coarse level l+1,
    5: persistent coarsest CGNE kernel, 6: its iteration count)."""
    cnt = np.zeros(n, dtype=np.int64)
    ms = np.zeros(n, dtype=np.float64)
    _check(lib().sw_kernel_times(ctx.ptr, n, cnt.ctypes.data, ms.ctypes.data), ctx.ptr)
    return [(int(a), float(b)) for a, b in zip(cnt, ms)]


def sw_launch_count() -> int:
    return int(lib().sw_launch_count())


def sw_fp64_peak(ctx: _Handle) -> float:
    """Measured FP64 FMA throughput of the context's device, TFLOP/s."""
    v = _D(0.0)
    _check(lib().sw_fp64_peak(ctx.ptr, ctypes.byref(v)), ctx.ptr)
    return float(v.value)


def sw_dslash_schur_noalloc(g: _Handle, mass: float, inp, out):
    """Schur operator with the library's fixed scratch (device tensors only)."""
    p_in, d_in = _ptr(inp)
    p_out, d_out = _ptr(out)
    if not (d_in and d_out):
        raise ValueError("sw_dslash_schur_noalloc takes device buffers only")
    N = g.shape[0] * g.shape[1]
    _check_buf(g, inp, N, what="in")
    _check_buf(g, out, N, what="out")
    _check(lib().sw_dslash_schur_noalloc(g.ptr, float(mass), p_in, p_out), g.ctx_ptr)
    return out


def sw_debug_cgne_stall(mg: _Handle) -> int:
    """Return code of the persistent CGNE run with a withheld barrier arrival."""
    return int(lib().sw_debug_cgne_stall(mg.ptr))


def sw_cg_eo_solve(g: _Handle, mass: float, b, x, tol: float, maxiter: int = 1000000,
                   allow_noconv: bool = False) -> dict:
    """CG on the even/odd normal system (the paper's comparison solver)."""
    dev = _same_place(b, x)
    N = g.shape[0] * g.shape[1]
    _check_buf(g, b, N, what="b")
    _check_buf(g, x, N, what="x")
    st = sw_solve_stats()
    rc = _check(lib().sw_cg_eo_solve(g.ptr, float(mass), _ptr(b)[0], _ptr(x)[0], float(tol),
                                     int(maxiter), dev, ctypes.byref(st)), g.ctx_ptr,
                allow=(-4,) if allow_noconv else ())
    d = st.as_dict()
    d["rc"] = rc
    return d


def sw_debug_batch_stall(mg: _Handle, nrhs: int = 16) -> int:
    """Return code of the batched coarsest kernel run with a withheld barrier arrival."""
    return int(lib().sw_debug_batch_stall(mg.ptr, int(nrhs)))


def sw_autotune_entries() -> list:
    """[(nc, K, coarse sites, stages, us per iteration)] chosen by the autotuner so far."""
    n = int(lib().sw_autotune_entries(0, None, None, None, None, None))
    if n <= 0:
        return []
    nc, K, sites, st = (np.zeros(n, dtype=np.int32) for _ in range(4))
    us = np.zeros(n, dtype=np.float64)
    lib().sw_autotune_entries(n, nc.ctypes.data, K.ctypes.data, sites.ctypes.data,
                              st.ctypes.data, us.ctypes.data)
    return [(int(a), int(b), int(c), int(d), float(e)) for a, b, c, d, e in zip(nc, K, sites, st, us)]


def sw_mg_level_maps(mg: _Handle, level: int):
    """(agg, chir) int32 maps of a level's dofs as the transfer kernels use them."""
    n = mg.shape[0] * mg.shape[1] if level == 1 else _level_len(mg, level)
    agg = np.zeros(n, dtype=np.int32)
    chir = np.zeros(n, dtype=np.int32)
    _check(lib().sw_mg_level_maps(mg.ptr, int(level), agg.ctypes.data, chir.ctypes.data),
           mg.ctx_ptr)
    return agg, chir


def sw_context_set_sm_share(ctx: _Handle, num: int, den: int):
    """Persistent coarsest kernels of this context hold num/den of the SMs."""
    _check(lib().sw_context_set_sm_share(ctx.ptr, int(num), int(den)), ctx.ptr)
