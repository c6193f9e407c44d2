"""Kaehler-Dirac preconditioned adaptive multigrid of the oracle (FP64).

Setup (Sec. IV, bullet list and Table kcycle):
  near-null vectors psi = psi0 + e with CG on A A^dag e = -A A^dag psi0;
  global orthonormalisation of the set; chiral doubling with (1 +- eps)/2 on
  level 1 and (1 +- sigma3)/2 on coarser levels (Sec. III.C, Sec. IV);
  orthonormalisation per aggregate and chirality (the columns of P, P^dag P = I);
  coarse operator A_hat = P^dag A P (Sec. III, R = P^dag), recursively.
Solve (Sec. IV, Table kcycle): flexible GCR(32) on the Schur operator I - A_eo A_oe,
preconditioned by a K-cycle: MR pre-smoother, restriction of (r_e, 0), a GCR(8)
solve of A_hat (max 16 iterations, tolerance 0.2) preconditioned by the next
level's K-cycle, or CGNE on the coarsest level (tolerance 0.2, max 256),
prolongation keeping the even part, MR post-smoother.

The coarse operators are plain sparse matrices: P^dag A P is one sparse product.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import krylov, lattice
from .operators import FineOperators


@dataclass
class Params:
    """Table kcycle defaults."""
    setup_maxiter: int = 250
    setup_tol: float = 1e-4
    setup_passes: int = 1
    outer_restart: int = 32
    outer_maxiter: int = 2000
    smoother_iters: int = 2
    omega: float = 0.85
    inter_restart: int = 8
    inter_maxiter: int = 16
    inter_tol: float = 0.2
    coarsest_maxiter: int = 256
    coarsest_tol: float = 0.2


def norm(v):
    return np.sqrt(np.vdot(v, v).real)


def near_null_vectors(op, opdag, psi0s, p: Params):
    """One near-null vector per initial guess psi0 (Sec. IV): r = -A A^dag psi0,
    CG on A A^dag e = r to tolerance setup_tol or setup_maxiter iterations,
    psi = psi0 + e.  With setup_passes > 1 the recipe repeats from psi/||psi||."""
    normal = lambda v: op(opdag(v))
    out, iters = [], []
    for psi0 in psi0s:
        start = psi0.astype(complex)
        for ps in range(p.setup_passes):
            if ps > 0:
                start = psi / norm(psi)
            r = -normal(start)
            e, k = krylov.cg(normal, r, p.setup_tol, p.setup_maxiter)
            psi = start + e
            iters.append(k)
        out.append(psi)
    return out, iters


def gram_schmidt(vecs):
    """Modified Gram-Schmidt in index order, one pass (global orthonormalisation)."""
    out = []
    for v in vecs:
        w = v.copy()
        for u in out:
            w = w - np.vdot(u, w) * u
        n = norm(w)
        if not n > 0:
            raise FloatingPointError("Gram-Schmidt breakdown")
        out.append(w / n)
    return out


def prolongator(vecs, chir: np.ndarray, agg: np.ndarray, nagg: int) -> sp.csr_matrix:
    """Chirally doubled, block-orthonormalised prolongator P.

    Column (X, c, i) -> X * 2Nv + c * Nv + i holds (1 + s_c chi)/2 psi_i restricted
    to aggregate X (s_0 = +1, s_1 = -1), orthonormalised against columns (X, c, j < i)
    by modified Gram-Schmidt in index order.  The aggregates are independent, so
    the loop over i runs on all (X, c) pairs at once."""
    nv = len(vecs)
    V = np.stack(vecs, axis=1)                          # [ndof, Nv]
    rows_all, cols_all, vals_all = [], [], []
    for c, sgn in enumerate((1, -1)):
        sel = np.nonzero(chir == sgn)[0]
        order = sel[np.argsort(agg[sel], kind="stable")]
        per = order.size // nagg
        idx = order.reshape(nagg, per)                  # dofs of (X, c), increasing
        W = V[idx]                                      # [nagg, per, Nv]
        Q = np.empty_like(W)
        for i in range(nv):
            w = W[:, :, i].copy()
            for j in range(i):
                coef = np.einsum("ap,ap->a", Q[:, :, j].conj(), w)
                w = w - coef[:, None] * Q[:, :, j]
            n = np.sqrt(np.einsum("ap,ap->a", w.conj(), w).real)
            if not np.all(n > 0):
                raise FloatingPointError("block orthonormalisation breakdown")
            Q[:, :, i] = w / n[:, None]
        col = (np.arange(nagg)[:, None, None] * 2 * nv + c * nv + np.arange(nv)[None, None, :])
        rows_all.append(np.broadcast_to(idx[:, :, None], Q.shape).ravel())
        cols_all.append(np.broadcast_to(col, Q.shape).ravel())
        vals_all.append(Q.ravel())
    ndof = chir.size
    return sp.coo_matrix((np.concatenate(vals_all), (np.concatenate(rows_all), np.concatenate(cols_all))),
                         shape=(ndof, nagg * 2 * nv)).tocsr()


@dataclass
class Level:
    op: sp.csr_matrix            # operator on this level (A on level 1, A_hat below)
    opdag: sp.csr_matrix
    chir: np.ndarray             # chirality of each dof (eps or sigma3)
    extent: tuple                # lattice extents of this level (sites)
    nc: int                      # dof per site
    P: sp.csr_matrix = None      # prolongator to this level from the next coarser one
    setup_iters: list = field(default_factory=list)


class Hierarchy:
    """Setup of the multigrid hierarchy (Sec. IV, Table kcycle).

    theta: [2, L1, L0] link angles.  blocks[0] = level-1 aggregate in KD blocks,
    blocks[l] = level-(l+1) aggregate in coarse sites.  nvec[l] = null vectors
    computed on level l+1.  psi0[l] = list of initial vectors on level l+1 (from
    sw_inputs), each of length ndof(l+1)."""

    def __init__(self, theta, m, levels, blocks, nvec, psi0, params: Params = None,
                 fine_op: str = "A"):
        """fine_op = "A": the paper's method (coarsen A = D B^-1, Schur outer
        solve).  fine_op = "D": the Galerkin MG of D itself (Sec. III.B, the
        variant the paper shows to stall), same recipe with D in place of A and
        the outer solve on the full D."""
        self.p = params or Params()
        self.F = FineOperators(theta, m)
        self.fine_op = fine_op
        F = self.F
        self.levels = []
        ext = (F.L0, F.L1)
        fop = F.A if fine_op == "A" else F.D
        lev = Level(op=fop, opdag=fop.conj().T.tocsr(), chir=F.eps, extent=ext, nc=1)
        self.levels.append(lev)
        for l in range(levels - 1):
            nv = nvec[l]
            b0, b1 = blocks[l]
            if l == 0:
                agg = lattice.fine_aggregate(F.L0, F.L1, b0, b1)
                cext = (F.L0 // (2 * b0), F.L1 // (2 * b1))
            else:
                site_agg = lattice.coarse_aggregate(ext[0], ext[1], b0, b1)
                agg = np.repeat(site_agg, lev.nc)
                cext = (ext[0] // b0, ext[1] // b1)
            nagg = cext[0] * cext[1]
            op, opdag = lev.op, lev.opdag
            vecs, its = near_null_vectors(lambda v: op @ v, lambda v: opdag @ v, psi0[l], self.p)
            vecs = gram_schmidt(vecs)
            lev.P = prolongator(vecs, lev.chir, agg, nagg)
            lev.setup_iters = its
            Ahat = (lev.P.conj().T @ (lev.op @ lev.P)).tocsr()
            chir = np.tile(np.concatenate([np.ones(nv, int), -np.ones(nv, int)]), nagg)
            lev = Level(op=Ahat, opdag=Ahat.conj().T.tocsr(), chir=chir, extent=cext, nc=2 * nv)
            self.levels.append(lev)
            ext = cext

    # ---- solve -------------------------------------------------------------
    # The steps of the solve are methods, in the paper's order, so that each
    # can be read (and a test can swap one for a deliberately wrong variant).
    def fine_schur(self, v):
        """The level-1 operator of the solve, I - A_eo A_oe (one fine mat-vec)."""
        self.st["fine_applies"] += 1
        return self.F.schur(v)

    def solve_level(self, l, rhs):
        """Approximate solve on level l >= 1 (Sec. IV, Table kcycle): GCR on A_hat
        preconditioned by the next K-cycle on intermediate levels, CGNE on the
        coarsest level."""
        p, lev = self.p, self.levels[l]
        op = lambda v: lev.op @ v
        if l == len(self.levels) - 1:
            e, k = krylov.cgne(op, lambda v: lev.opdag @ v, rhs, p.coarsest_tol, p.coarsest_maxiter)
            self.st["coarsest_iters"] += k
            self.st["coarsest_solves"] += 1
            return e
        e, k, _, _ = krylov.fgcr(op, lambda r: self.kcycle(l, r), rhs, p.inter_tol * norm(rhs),
                                 p.inter_restart, p.inter_maxiter, confirm=False)
        self.st["inter_iters"] += k
        self.st["inter_solves"] += 1
        return e

    def kcycle(self, l, r):
        """K-cycle of an intermediate level l: (1) MR pre-smoother, (2) coarse
        correction P A_hat^-1 P^dag on the smoothed residual, (3) MR post-smoother
        on the residual left after steps 1 and 2."""
        p, lev = self.p, self.levels[l]
        op = lambda v: lev.op @ v
        x1, r1 = krylov.mr(op, r, p.smoother_iters, p.omega)
        ehat = self.solve_level(l + 1, lev.P.conj().T @ r1)
        e = lev.P @ ehat
        r2 = r1 - op(e)
        x3, _ = krylov.mr(op, r2, p.smoother_iters, p.omega)
        return x1 + e + x3

    def kcycle_fine(self, r):
        """K-cycle of the fine level on the even half (Sec. IV): the same three
        steps with S, restricting (r1, 0) (odd contributions set to zero) and
        keeping the even part of the prolonged error."""
        F, p = self.F, self.p
        S = self.fine_schur
        x1, r1 = krylov.mr(S, r, p.smoother_iters, p.omega)
        full = np.zeros(F.N, dtype=complex)
        full[F.even] = r1
        ehat = self.solve_level(1, self.levels[0].P.conj().T @ full)
        e = (self.levels[0].P @ ehat)[F.even]
        r2 = r1 - S(e)
        x3, _ = krylov.mr(S, r2, p.smoother_iters, p.omega)
        return x1 + e + x3

    def solve(self, b: np.ndarray, tol: float, on_outer=None):
        """Solve D x = b (b as [N] complex, site order x0 + L0 x1) to
        ||b - D x|| <= tol ||b||.  Returns (x, stats dict)."""
        F, p = self.F, self.p
        self.st = st = dict(fine_applies=0, inter_iters=0, inter_solves=0, coarsest_iters=0,
                            coarsest_solves=0)
        nlev = len(self.levels)
        bn = norm(b)
        if self.fine_op == "D":
            def Dop(v):
                st["fine_applies"] += 1
                return F.D @ v

            def kcycle_D(r):
                x1, r1 = krylov.mr(Dop, r, p.smoother_iters, p.omega)
                ehat = self.solve_level(1, self.levels[0].P.conj().T @ r1)
                e = self.levels[0].P @ ehat
                r2 = r1 - Dop(e)
                x3, _ = krylov.mr(Dop, r2, p.smoother_iters, p.omega)
                return x1 + e + x3
            x, it, rs, conv = krylov.fgcr(Dop, kcycle_D, b.astype(complex), tol * bn,
                                          p.outer_restart, p.outer_maxiter, confirm=True,
                                          on_iter=on_outer)
            st.update(outer_iters=it, restarts=rs, converged=conv,
                      true_resid=norm(b - F.D @ x) / bn)
            return x, st
        bt = F.schur_rhs(b)
        precond = self.kcycle_fine if nlev > 1 else (lambda r: r)
        ze, it, rs, conv = krylov.fgcr(self.fine_schur, precond, bt, tol * bn, p.outer_restart,
                                       p.outer_maxiter, confirm=True, on_iter=on_outer)
        x = F.reconstruct(b, ze)
        st.update(outer_iters=it, restarts=rs, converged=conv,
                  true_resid=norm(b - F.D @ x) / bn)
        return x, st
