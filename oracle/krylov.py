"""Krylov methods of the oracle, written out step by step in FP64.

Inner products are <a, b> = sum conj(a) b (numpy.vdot).  Every solver starts
from a zero initial guess.  Each returns the iterate and the iteration count.
"""
from __future__ import annotations

import numpy as np


def cg(op, b: np.ndarray, tol: float, maxiter: int):
    """Conjugate gradient on a Hermitian positive (semi)definite ``op`` (Hestenes and
    Stiefel).  Stops when ||r_k|| <= tol ||b|| or after ``maxiter`` iterations.
    Used for the null-vector setup on A A^dag (Sec. IV, Table kcycle)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    stop = tol * np.sqrt(rr)
    k = 0
    while k < maxiter and np.sqrt(rr) > stop:
        q = op(p)
        alpha = rr / np.vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
        k += 1
    return x, k


def cgne(op, opdag, b: np.ndarray, tol: float, maxiter: int):
    """CG on the normal error (Craig's method): CG on op op^dag y = b with
    x = op^dag y, iterating on x and r = b - op x directly.  Stops when
    ||r|| <= tol ||b|| or after ``maxiter`` iterations (coarsest level,
    Sec. IV and Table kcycle)."""
    x = np.zeros_like(b)
    r = b.copy()
    rr = np.vdot(r, r).real
    stop = tol * np.sqrt(rr)
    p = opdag(r)
    k = 0
    while k < maxiter and np.sqrt(rr) > stop:
        alpha = rr / np.vdot(p, p).real
        x = x + alpha * p
        r = r - alpha * op(p)
        rr_new = np.vdot(r, r).real
        p = opdag(r) + (rr_new / rr) * p
        rr = rr_new
        k += 1
    return x, k


def mr(op, b: np.ndarray, niter: int, omega: float):
    """Global minimal-residual smoother with relaxation omega (Sec. IV, Table kcycle):
    x = 0, r = b; repeat: q = op r, alpha = <q, r>/<q, q>, x += omega alpha r,
    r -= omega alpha q.  Returns (x, r) with r = b - op x."""
    x = np.zeros_like(b)
    r = b.copy()
    for _ in range(niter):
        q = op(r)
        alpha = np.vdot(q, r) / np.vdot(q, q).real
        x = x + omega * alpha * r
        r = r - omega * alpha * q
    return x, r


def fgcr(op, precond, b: np.ndarray, tol_abs: float, restart: int, maxiter: int,
         confirm: bool = True, on_iter=None):
    """Flexible restarted GCR (Axelsson 1987), the outer solver of the K-cycle.

    Iteration k: p_k = M(r); q_k = op p_k; modified Gram-Schmidt of q_k against
    q_0..q_{k-1} (same combination applied to p_k); normalise by ||q_k||;
    alpha = <q_k, r>; x += alpha p_k; r -= alpha q_k.  After ``restart``
    directions the true residual b - op x is recomputed and the basis dropped.
    Stops when ||r|| <= tol_abs on the recurrence residual (with ``confirm``, only
    once the recomputed true residual agrees; otherwise it restarts from it) or
    after ``maxiter`` iterations.
    Returns (x, iterations, restarts, converged)."""
    x = np.zeros_like(b)
    r = b.copy()
    P, Q = [], []
    it = restarts = 0
    while True:
        rn = np.sqrt(np.vdot(r, r).real)
        if rn <= tol_abs:
            if not confirm:
                return x, it, restarts, True
            rt = b - op(x)
            if np.sqrt(np.vdot(rt, rt).real) <= tol_abs:
                return x, it, restarts, True
            r = rt
            P, Q = [], []
            restarts += 1
            continue
        if it >= maxiter:
            return x, it, restarts, False
        p = precond(r)
        q = op(p)
        for pj, qj in zip(P, Q):
            beta = np.vdot(qj, q)
            q = q - beta * qj
            p = p - beta * pj
        g = np.sqrt(np.vdot(q, q).real)
        q = q / g
        p = p / g
        alpha = np.vdot(q, r)
        x = x + alpha * p
        r = r - alpha * q
        P.append(p); Q.append(q)
        it += 1
        if on_iter is not None:
            on_iter(it, r)
        if len(P) == restart and it < maxiter:
            r = b - op(x)
            P, Q = [], []
            restarts += 1
