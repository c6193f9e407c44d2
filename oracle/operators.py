"""Fine-level operators of the oracle as explicit scipy sparse matrices (FP64).

Each matrix is assembled entry by entry from its definition; applying an
operator is one sparse mat-vec.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import lattice


def links(theta: np.ndarray) -> np.ndarray:
    """U_mu(x) = exp(i theta_mu(x)) as complex [2, N], theta given as [2, L1, L0]
    (the U(1) links of the lattice Schwinger model, Sec. I)."""
    return np.exp(1j * theta.reshape(2, -1))


def dirac(theta: np.ndarray, m: float) -> sp.csr_matrix:
    """Staggered operator of Eq. staggeredD with a = 1, written out literally:

        D_{x,y} = 1/2 sum_mu eta_mu(x) [U_mu(x) delta_{x+mu,y} - U_mu(x-mu)^* delta_{x-mu,y}]
                  + m delta_{x,y},

    periodic in both directions.  Duplicate (x, y) entries (extent 2) add up.
    """
    _, L1, L0 = theta.shape
    N = L0 * L1
    U = links(theta)
    et = lattice.eta(L0, L1)
    x0, x1 = lattice.coords(L0, L1)
    s = np.arange(N)
    rows, cols, vals = [s], [s], [np.full(N, m, dtype=complex)]
    for mu in range(2):
        d0, d1 = (1, 0) if mu == 0 else (0, 1)
        fwd = lattice.site(x0 + d0, x1 + d1, L0, L1)
        bwd = lattice.site(x0 - d0, x1 - d1, L0, L1)
        rows += [s, s]
        cols += [fwd, bwd]
        vals += [0.5 * et[mu] * U[mu], -0.5 * et[mu] * np.conj(U[mu][bwd])]
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N)).tocsr()


NAIK_C1, NAIK_C3 = 9.0 / 8.0, -1.0 / 24.0


def dirac_naik(theta: np.ndarray, m: float) -> sp.csr_matrix:
    """Naik-improved staggered operator (Sec. II.A, Eq. freehisq), in the sign and
    1/2 normalisation of Eq. staggeredD: one-link hops weighted c1 = 9/8 and
    three-link hops weighted c3 = -1/24 (so 1/2 c1 = 9/16, 1/2 c3 = -1/48 as
    printed; free symbol sin p (1 + sin^2 p / 6)).  The paper gives the free
    operator only; the three-link hop here carries the product of the three
    links along its path, U_mu(x) U_mu(x+mu) U_mu(x+2mu)."""
    _, L1, L0 = theta.shape
    N = L0 * L1
    U = links(theta)
    et = lattice.eta(L0, L1)
    x0, x1 = lattice.coords(L0, L1)
    s = np.arange(N)
    rows, cols, vals = [s], [s], [np.full(N, m, dtype=complex)]
    for mu in range(2):
        d0, d1 = (1, 0) if mu == 0 else (0, 1)
        nb = [lattice.site(x0 + k * d0, x1 + k * d1, L0, L1) for k in range(-3, 4)]
        f1, b1, f3, b3 = nb[4], nb[2], nb[6], nb[0]
        long_f = U[mu] * U[mu][f1] * U[mu][nb[5]]          # U(x) U(x+mu) U(x+2mu)
        long_b = U[mu][b3] * U[mu][nb[1]] * U[mu][b1]      # U(x-3mu) U(x-2mu) U(x-mu)
        rows += [s, s, s, s]
        cols += [f1, b1, f3, b3]
        vals += [0.5 * NAIK_C1 * et[mu] * U[mu], -0.5 * NAIK_C1 * et[mu] * np.conj(U[mu][b1]),
                 0.5 * NAIK_C3 * et[mu] * long_f, -0.5 * NAIK_C3 * et[mu] * np.conj(long_b)]
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N)).tocsr()


def naik_kd_operator(theta: np.ndarray, m: float):
    """(D_Naik, B_Naik, A_Naik = D_Naik B_Naik^-1): the KD split of the Naik operator
    (Sec. II.A): three-link hops always leave the 2x2 block, so B_Naik is B with
    its hops scaled by c1 = 9/8."""
    _, L1, L0 = theta.shape
    Dn = dirac_naik(theta, m)
    Bn, _ = block_split(Dn, L0, L1)
    An = (Dn @ block_inverse(Bn, L0, L1)).tocsr()
    return Dn, Bn, An


def block_split(Dm: sp.csr_matrix, L0: int, L1: int):
    """D = B + C (Sec. II.A): B keeps the entries of D that couple two sites of
    the same 2x2 Kaehler-Dirac block (the mass term included), C the rest."""
    blk = lattice.kd_block(L0, L1)
    coo = Dm.tocoo()
    inside = blk[coo.row] == blk[coo.col]
    N = Dm.shape[0]
    B = sp.coo_matrix((coo.data[inside], (coo.row[inside], coo.col[inside])), shape=(N, N)).tocsr()
    C = sp.coo_matrix((coo.data[~inside], (coo.row[~inside], coo.col[~inside])), shape=(N, N)).tocsr()
    return B, C


def block_inverse(B: sp.csr_matrix, L0: int, L1: int) -> sp.csr_matrix:
    """B^-1, block by block: the 4x4 matrix of every block is gathered from B and
    inverted with numpy.linalg.inv (LU with partial pivoting).  Requires every
    block to be non-singular (m > 0)."""
    blk = lattice.kd_block(L0, L1)
    N = B.shape[0]
    members = np.argsort(blk, kind="stable").reshape(-1, 4)   # the 4 sites of each block
    local = np.empty(N, dtype=np.int64)
    local[members] = np.arange(4)[None, :]
    coo = B.tocoo()
    dense = np.zeros((members.shape[0], 4, 4), dtype=complex)
    np.add.at(dense, (blk[coo.row], local[coo.row], local[coo.col]), coo.data)
    inv = np.linalg.inv(dense)
    rows = np.repeat(members, 4, axis=1).ravel()
    cols = np.tile(members, (1, 4)).ravel()
    return sp.coo_matrix((inv.ravel(), (rows, cols)), shape=(N, N)).tocsr()


class FineOperators:
    """D, B, C, B^-1 and A = D B^-1 (Eq. defA) for one gauge field and mass, plus
    the block-parity index sets used by the Schur system (Table kcycle)."""

    def __init__(self, theta: np.ndarray, m: float):
        _, L1, L0 = theta.shape
        self.L0, self.L1, self.m = L0, L1, m
        self.N = L0 * L1
        self.D = dirac(theta, m)
        self.B, self.C = block_split(self.D, L0, L1)
        self.Binv = block_inverse(self.B, L0, L1)
        self.A = (self.D @ self.Binv).tocsr()
        self.Adag = self.A.conj().T.tocsr()
        par = lattice.kd_parity(L0, L1)
        self.even = np.nonzero(par == 0)[0]
        self.odd = np.nonzero(par == 1)[0]
        self.A_eo = self.A[self.even][:, self.odd].tocsr()
        self.A_oe = self.A[self.odd][:, self.even].tocsr()
        self.eps = lattice.epsilon(L0, L1)

    def schur(self, xe: np.ndarray) -> np.ndarray:
        """S x_e = x_e - A_eo A_oe x_e (Table kcycle, level-1 operator)."""
        return xe - self.A_eo @ (self.A_oe @ xe)

    def schur_rhs(self, b: np.ndarray) -> np.ndarray:
        """b_e - A_eo b_o: right-hand side of the Schur system for A z = b."""
        return b[self.even] - self.A_eo @ b[self.odd]

    def reconstruct(self, b: np.ndarray, ze: np.ndarray) -> np.ndarray:
        """Full solution of D x = b from z_e: z_o = b_o - A_oe z_e, x = B^-1 z."""
        z = np.zeros(self.N, dtype=complex)
        z[self.even] = ze
        z[self.odd] = b[self.odd] - self.A_oe @ ze
        return self.Binv @ z


def cg_eo_solve(theta: np.ndarray, m: float, b: np.ndarray, tol: float, maxiter: int):
    """The comparison solver of Sec. II (Eq. normal) and Sec. IV (Fig. iterworst):
    CG on (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o over the site parity eps,
    then x_o = (b_o - D_oe x_e) / m.  The full residual is the CG residual / m on
    the even sites, so CG runs to ||r|| <= tol m ||b||, restarting from the true
    residual if the recurrence has drifted from it.  Returns (x, iterations)."""
    from . import krylov
    _, L1, L0 = theta.shape
    D = dirac(theta, m)
    eps = lattice.epsilon(L0, L1)
    e, o = np.nonzero(eps > 0)[0], np.nonzero(eps < 0)[0]
    Deo = D[e][:, o].tocsr()
    Doe = D[o][:, e].tocsr()
    rhs = m * b[e] - Deo @ b[o]
    op = lambda v: m * m * v - Deo @ (Doe @ v)
    target = tol * m * np.linalg.norm(b)
    xe = np.zeros_like(rhs)
    k = 0
    # restart from the true residual when the recurrence residual has drifted
    for _ in range(8):
        r = rhs - op(xe)
        rn = np.linalg.norm(r)
        if rn <= target or k >= maxiter:
            break
        dx, kk = krylov.cg(op, r, target / rn, maxiter - k)
        xe = xe + dx
        k += kk
    x = np.zeros(L0 * L1, dtype=complex)
    x[e] = xe
    x[o] = (b[o] - Doe @ xe) / m
    return x, k
