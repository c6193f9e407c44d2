"""Coarsest-level CGNE with reduced-precision operands, emulated on the CPU
(test infrastructure).

The coarsest solve of the K-cycle only has to reduce its residual to 0.2
(Table kcycle), so its stencil may run in less than FP64.  This module
emulates a stencil application whose operands (the stencil entries and the
vector) are rounded to p explicit mantissa bits before the products, with the
products and sums in FP32 (complex64), as a tensor-core contraction with FP32
accumulation does (p = 23: FP32, p = 10: TF32, p = 7: BF16).  The "3xTF32"
form splits each operand into a TF32 head and a TF32 tail and adds the three
leading products.  CGNE itself (Sec. IV) runs in FP64 around the emulated
operator, as the library's batched coarsest solve does.

    python -m oracle.precision L [nrhs]   # iterations to 0.2 per precision
"""
from __future__ import annotations

import json
import sys

import numpy as np

import sw_inputs as si
from oracle import krylov
from oracle import mg as omg

FORMS = {"fp64": None, "fp32": (23, False), "3xtf32": (10, True), "tf32": (10, False),
         "bf16": (7, False)}


def round_mantissa(x: np.ndarray, bits: int) -> np.ndarray:
    """float32 values rounded to `bits` explicit mantissa bits, to nearest even
    (exponent range of float32, as TF32 and BF16 keep it)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    if bits >= 23:
        return u.astype(np.uint32).view(np.float32)
    drop = np.uint64(23 - bits)
    lsb = (u >> drop) & np.uint64(1)
    u = ((u + (np.uint64(1) << (drop - np.uint64(1))) - np.uint64(1) + lsb) >> drop) << drop
    return u.astype(np.uint32).view(np.float32)


def round_complex(z: np.ndarray, bits: int) -> np.ndarray:
    z = np.asarray(z, dtype=np.complex64)
    return (round_mantissa(z.real, bits) + 1j * round_mantissa(z.imag, bits)).astype(np.complex64)


def reduced_operator(M, bits: int, split: bool):
    """v -> M v with operands rounded to `bits` mantissa bits, FP32 products and
    sums; split: head/tail operands, three leading products."""
    head = M.astype(np.complex64)
    head.data = round_complex(M.data, bits)
    tail = None
    if split:
        tail = M.astype(np.complex64)
        tail.data = round_complex(M.data - head.data.astype(np.complex128), bits)

    def apply(v):
        vh = round_complex(v, bits)
        y = head @ vh
        if split:
            vt = round_complex(v - vh.astype(np.complex128), bits)
            y = y + head @ vt + tail @ vh
        return y.astype(np.complex128)
    return apply


def cgne_iterations(A, Adag, form: str, b: np.ndarray, tol: float = 0.2, maxit: int = 2048):
    """Iterations CGNE takes to tol with the operator in the given form, and the
    true FP64 residual it reached."""
    if FORMS[form] is None:
        op, opd = (lambda v: A @ v), (lambda v: Adag @ v)
    else:
        bits, split = FORMS[form]
        op, opd = reduced_operator(A, bits, split), reduced_operator(Adag, bits, split)
    x, k = krylov.cgne(op, opd, b, tol, maxit)
    return k, float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


def coarsest_operator(L: int, m: float = 1e-3, beta: float = 6.0, sweeps: int = 300,
                      blocks=((4, 4), (2, 2)), nvec=(24, 32)):
    """The coarsest operator of a 3-level oracle hierarchy (paper setup)."""
    th = si.heatbath_u1(L, L, beta, sweeps, seed=1, device="cpu")
    psi0 = si.null_vector_guesses(L, L, list(nvec), 3, [tuple(b) for b in blocks])
    H = omg.Hierarchy(th, m, 3, [tuple(b) for b in blocks], list(nvec),
                      [list(a) for a in psi0], omg.Params(coarsest_maxiter=2048))
    return H.levels[-1].op.tocsr(), H.levels[-1].opdag.tocsr()


def main():
    L = int(sys.argv[1])
    nrhs = int(sys.argv[2]) if len(sys.argv) > 2 else 2
    A, Ad = coarsest_operator(L, sweeps=2000 if L >= 256 else 300)
    res = {}
    for form in FORMS:
        runs = [cgne_iterations(A, Ad, form, si.gaussian_complex(9000 + s, A.shape[0]))
                for s in range(nrhs)]
        res[form] = {"iters": [k for k, _ in runs], "true_resid": [r for _, r in runs]}
    print(json.dumps({"L": L, "n": A.shape[0], "res": res}))


if __name__ == "__main__":
    main()
