"""Operator-application counts of the oracle's own full solve of the 256^2
multigrid workload, with the wall time it took (test infrastructure).

A full oracle solve of that workload (3 levels, Nv 24/32, m = 1e-3, 1e-10)
takes tens of minutes on one core, so the CPU baseline and the reference arm
of the bench time single applications of the oracle's operators on the machine
at hand and scale them by what this script records once: how many times the
solve applied S (fine), A_hat on level 2 and A_hat (or its adjoint) on level 3,
and the ratio of the solve's wall time to the time those applications alone
take here (the rest: BLAS-1, Gram-Schmidt, transfers, interpreter overhead).

The hierarchy is set up as the paper prescribes (Table kcycle: CG on A A^dag
to 1e-4 or 250 iterations per null vector; coarsest CGNE cap 2048 as the
workload's preset).  The gauge field comes from the CPU heatbath, which differs
from the CUDA heatbath's field only by rounding in the draws (same seed and
algorithm), so the counts are those of a statistically equivalent field.

    python -m oracle.solve_counts      # writes oracle/solve_counts_256.json
"""
from __future__ import annotations

import json
import os
import platform
import time

import numpy as np

import sw_inputs as si
from oracle import mg as omg

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "solve_counts_256.json")
L, BETA, SWEEPS, MASS = 256, 6.0, 2000, 1e-3
BLOCKS, NVEC = [(4, 4), (2, 2)], [24, 32]
TOL, COARSEST_CAP = 1e-10, 2048
RHS_SEED = 1003  # Gaussian right-hand side, stream 1000 + 3


class _Counted:
    """A sparse operator that counts its applications."""

    def __init__(self, M):
        self.M, self.n, self.shape = M, 0, M.shape

    def __matmul__(self, v):
        self.n += 1
        return self.M @ v


def apply_times(H, reps: int) -> dict:
    """Seconds per application of S, A_hat (level 2) and A_hat (level 3)."""
    out = {}
    ve = np.ones(H.F.even.size, dtype=complex)
    t = time.perf_counter()
    for _ in range(reps):
        H.F.schur(ve)
    out["S"] = (time.perf_counter() - t) / reps
    for lvl in (1, 2):
        op = H.levels[lvl].op
        M = op.M if isinstance(op, _Counted) else op
        v = np.ones(M.shape[0], dtype=complex)
        t = time.perf_counter()
        for _ in range(reps):
            M @ v
        out[f"A{lvl + 1}"] = (time.perf_counter() - t) / reps
    return out


def main():
    t0 = time.perf_counter()
    th = si.heatbath_u1(L, L, BETA, SWEEPS, seed=1, device="cpu")
    psi0 = si.null_vector_guesses(L, L, NVEC, 3, BLOCKS)
    t1 = time.perf_counter()
    H = omg.Hierarchy(th, MASS, 3, BLOCKS, NVEC, [list(a) for a in psi0],
                      omg.Params(coarsest_maxiter=COARSEST_CAP))
    t2 = time.perf_counter()
    for lvl in (1, 2):
        lev = H.levels[lvl]
        lev.op, lev.opdag = _Counted(lev.op), _Counted(lev.opdag)
    b = si.gaussian_complex(RHS_SEED, L * L)
    t3 = time.perf_counter()
    x, st = H.solve(b, TOL)
    wall = time.perf_counter() - t3
    counts = {"S": int(st["fine_applies"]),
              "A2": int(H.levels[1].op.n + H.levels[1].opdag.n),
              "A3": int(H.levels[2].op.n + H.levels[2].opdag.n)}
    per = apply_times(H, reps=20)
    modelled = sum(counts[k] * per[k] for k in counts)
    rec = {
        "workload": {"L": L, "beta": BETA, "sweeps": SWEEPS, "mass": MASS, "blocks": BLOCKS,
                     "nvec": NVEC, "tol": TOL, "coarsest_maxiter": COARSEST_CAP,
                     "rhs": f"gaussian_complex({RHS_SEED})", "gauge": "CPU heatbath, seed 1"},
        "counts": counts,
        "stats": {k: (float(v) if isinstance(v, (float, np.floating)) else int(v))
                  for k, v in st.items()},
        "solve_wall_s": wall,
        "apply_s": per,
        "overhead_ratio": wall / modelled,
        "heatbath_s": t1 - t0,
        "setup_s": t2 - t1,
        "machine": {"processor": platform.processor() or platform.machine(),
                    "python": platform.python_version(), "numpy": np.__version__},
    }
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


if __name__ == "__main__":
    main()
