"""Shared helpers of the GPU parity tests (no oracle arithmetic here)."""
import numpy as np

import sw_inputs as si


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def psi0_arrays(L0, L1, nvec, levels, blocks, seed=5):
    """Initial null-vector guesses per level, vector-major numpy arrays."""
    return si.null_vector_guesses(L0, L1, nvec, levels, blocks, seed)


def compact_P(Psp, chir, agg, nv):
    """Oracle's sparse P -> [ndof][nv]: entry i of row r is column
    (agg[r], chirality of r, i)."""
    P = Psp.toarray()
    rows = np.arange(P.shape[0])
    c = np.where(chir > 0, 0, 1)
    base = agg * 2 * nv + c * nv
    return np.stack([P[rows, base + i] for i in range(nv)], axis=1)


def assemble_stencil(Y, E0, E1):
    """Dense coarse operator from stencil blocks Y[X][d] (d: self, +0, -0, +1, -1)."""
    ns, _, nc, _ = Y.shape
    M = np.zeros((ns * nc, ns * nc), dtype=complex)
    for X in range(ns):
        X0, X1 = X % E0, X // E0
        nb = [X, (X0 + 1) % E0 + E0 * X1, (X0 - 1) % E0 + E0 * X1,
              X0 + E0 * ((X1 + 1) % E1), X0 + E0 * ((X1 - 1) % E1)]
        for d in range(5):
            M[X * nc:(X + 1) * nc, nb[d] * nc:(nb[d] + 1) * nc] += Y[X, d]
    return M
