"""Pins of the oracle's fine operators against what the paper and mathematics fix.

Each test names the passage it checks.  Conventions of the oracle (and of the
library): D of Eq. staggeredD with the factor 1/2, site s = x0 + L0 x1.
"""
import os

import numpy as np
import pytest

import sw_inputs as si
from oracle import lattice, operators

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_theta(L, seed):
    return np.random.default_rng(seed).uniform(-np.pi, np.pi, (2, L, L))


def dense_D(theta, m):
    return operators.dirac(theta, m).toarray()


# ---------------------------------------------------------------- spectra
@pytest.mark.parametrize("L,m", [(8, 0.0), (8, 0.3), (16, 0.05)])
def test_free_staggered_spectrum(L, m):
    """Sec. II: at U = 1, lambda = m +- i sqrt(sum_mu sin^2 p_mu), p_mu = 2 pi n/L,
    n in [-L/4 + 1, L/4]; each value twice (two tastes in 2D)."""
    ev = np.linalg.eigvals(dense_D(np.zeros((2, L, L)), m))
    n = np.arange(-L // 4 + 1, L // 4 + 1)
    p = 2 * np.pi * n / L
    s = np.sqrt(np.sin(p)[:, None] ** 2 + np.sin(p)[None, :] ** 2).ravel()
    expect = np.concatenate([m + 1j * s, m - 1j * s, m + 1j * s, m - 1j * s])
    key = lambda z: np.lexsort((np.round(z.real, 9), np.round(z.imag, 9)))
    a, b = ev[key(ev)], expect[key(expect)]
    assert np.max(np.abs(a - b)) < 1e-12


def kd_free_eigs(L, m):
    """Sec. II.A, free spectrum after KD preconditioning, massive form, in the
    normalisation of Eq. staggeredD (hopping 1/2): the paper's formula with m
    replaced by 2m, rho = sqrt(d / (d + 4 m^2)); momenta of the 2a blocked
    lattice p = 2 pi n / (L/2), n = 0 .. L/2 - 1; each value twice."""
    d = 2
    rho = np.sqrt(d / (d + 4 * m * m))
    n = np.arange(L // 2)
    p = 2 * np.pi * n / (L // 2)
    cs = (np.cos(p)[:, None] + np.cos(p)[None, :]).ravel()
    c = rho * cs / d
    lam_p = 1 - rho * (c + 1j * np.sqrt(1 - c * c + 0j))
    lam_m = 1 - rho * (c - 1j * np.sqrt(1 - c * c + 0j))
    return np.concatenate([lam_p, lam_m, lam_p, lam_m])


@pytest.mark.parametrize("L,m", [(8, 0.0), (8, 0.1), (16, 0.5)])
def test_free_kd_spectrum(L, m):
    F = operators.FineOperators(np.zeros((2, L, L)), m)
    ev = np.linalg.eigvals(F.A.toarray())
    exp = kd_free_eigs(L, m)
    key = lambda z: np.lexsort((np.round(z.real, 9), np.round(z.imag, 9)))
    assert np.max(np.abs(ev[key(ev)] - exp[key(exp)])) < 1e-12
    # all on the circle 1 - rho e^{i theta} (Sec. II.A)
    rho = np.sqrt(2 / (2 + 4 * m * m))
    assert np.max(np.abs(np.abs(ev - 1) - rho)) < 1e-12


def test_free_block_and_hop_unitary():
    """Sec. II.A: at U = 1, B_hat = B eps / sqrt(d/4 + m^2) and C_hat = C eps / sqrt(d/4)
    (1/2-normalised operator) square to the identity."""
    L, m = 8, 0.3
    F = operators.FineOperators(np.zeros((2, L, L)), m)
    E = np.diag(F.eps.astype(float))
    Bh = F.B.toarray() @ E / np.sqrt(0.5 + m * m)
    Ch = F.C.toarray() @ E / np.sqrt(0.5)
    I = np.eye(L * L)
    assert np.max(np.abs(Bh @ Bh - I)) < 1e-13
    assert np.max(np.abs(Ch @ Ch - I)) < 1e-13
    assert np.max(np.abs(Bh - Bh.conj().T)) < 1e-14


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("seed", [1, 2])
def test_staggered_invariants(seed):
    L, m = 8, 0.37
    th = rand_theta(L, seed)
    D = dense_D(th, m)
    D0 = dense_D(th, 0.0)
    eps = np.diag(lattice.epsilon(L, L).astype(float))
    I = np.eye(L * L)
    assert np.max(np.abs(D0 + D0.conj().T)) < 1e-15                 # anti-Hermitian at m = 0
    assert np.max(np.abs(eps @ D @ eps - D.conj().T)) < 1e-15       # eps-Hermiticity
    assert np.max(np.abs(eps @ D + D @ eps - 2 * m * eps)) < 1e-15  # eps D + D eps = 2 m eps
    assert np.max(np.abs(D @ D.conj().T - D.conj().T @ D)) < 1e-14  # normality
    # even/odd block form: D_ee = D_oo = m (Sec. II, eq. before Eq. normal)
    ev = np.diag(eps) > 0
    assert np.max(np.abs(D[np.ix_(ev, ev)] - m * np.eye(ev.sum()))) < 1e-15


def test_gauge_covariance():
    """D[U^g] = G D[U] G^dag for U^g_mu(x) = g(x) U_mu(x) g(x + mu)^*."""
    L, m = 8, 0.2
    th = rand_theta(L, 3)
    alpha = np.random.default_rng(4).uniform(-np.pi, np.pi, (L, L))
    G = np.diag(np.exp(1j * alpha.ravel()))
    Dg = dense_D(si.gauge_transform(th, alpha), m)
    assert np.max(np.abs(Dg - G @ dense_D(th, m) @ G.conj().T)) < 1e-14


def test_frustration_and_corner_cancellation():
    """Eq. frustration: eta_mu(x) eta_nu(x+mu) eta_mu(x+nu) eta_nu(x) = -1; at U = 1
    the corner terms of D^dag D cancel (Fig. 2Dlattice)."""
    L = 8
    et = lattice.eta(L, L)
    x0, x1 = lattice.coords(L, L)
    s = np.arange(L * L)
    sp0 = lattice.site(x0 + 1, x1, L, L)
    sp1 = lattice.site(x0, x1 + 1, L, L)
    prod = et[0][s] * et[1][sp0] * et[0][sp1] * et[1][s]
    assert np.all(prod == -1)
    D = dense_D(np.zeros((2, L, L)), 0.2)
    N = D.conj().T @ D
    diag = lattice.site(x0 + 1, x1 + 1, L, L)
    assert np.max(np.abs(N[s, diag])) < 1e-15
    # with a generic field the corner terms are present
    Dg = dense_D(rand_theta(L, 9), 0.2)
    Ng = Dg.conj().T @ Dg
    assert np.max(np.abs(Ng[s, diag])) > 1e-3


def test_block_partition_halves_links():
    """Fig. BC_partition: B and C each hold half of the d N links; B has the
    2x2 blocks with corners at even coordinates."""
    L = 8
    F = operators.FineOperators(rand_theta(L, 5), 0.1)
    Bo = F.B.tocoo()
    off = Bo.row != Bo.col
    assert off.sum() == 2 * (L * L)          # N links, each as two entries
    assert F.C.nnz == 2 * (L * L)
    blk = lattice.kd_block(L, L)
    assert np.all(blk[Bo.row] == blk[Bo.col])
    Cc = F.C.tocoo()
    assert np.all(blk[Cc.row] != blk[Cc.col])


def load_localblock():
    entries = []
    with open(os.path.join(GOLDEN, "localblock.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line:
                entries.append(line)
    return entries


@pytest.mark.parametrize("seed", [6, 7])
def test_local_block_matches_paper(seed):
    """Eq. localblock.  The printed block equals eps B eps of Eq. staggeredD's B
    (the printed hopping has the opposite sign of Eq. staggeredD; eps B eps =
    2m - B flips exactly the hops): Eq. staggeredD's sign is the normative one."""
    L, m = 8, 0.23
    th = rand_theta(L, seed)
    U = operators.links(th)
    F = operators.FineOperators(th, m)
    n0, n1 = 2, 4                                   # block with corner 2n = (2, 4)
    off = {"0": (0, 0), "x": (1, 0), "y": (0, 1)}
    order = [(0, 0), (1, 1), (1, 0), (0, 1)]        # printed row order
    sites = [lattice.site(n0 + a, n1 + b, L, L) for a, b in order]
    paper = np.zeros((4, 4), dtype=complex)
    for row, col, coef, kind, *rest in load_localblock():
        if kind == "mass":
            v = float(coef) * m
        else:
            mu = 0 if rest[0] == "x" else 1
            dx, dy = off[rest[1]]
            u = U[mu][lattice.site(n0 + dx, n1 + dy, L, L)]
            v = float(coef) * (np.conj(u) if rest[2] == "1" else u)
        paper[int(row) - 1, int(col) - 1] += v
    B = F.B.toarray()[np.ix_(sites, sites)]
    e = np.diag(F.eps[sites].astype(float))
    assert np.max(np.abs(paper - e @ B @ e)) < 1e-15
    assert np.max(np.abs(paper - (2 * m * np.eye(4) - B))) < 1e-15


# ---------------------------------------------------------------- A and S
def test_gamma5_LR_hermiticity_and_pairs():
    """Eqs. gamma5L, gamma5R: eps B^-1 A = A^dag eps B^-1 and A B eps = B eps A^dag;
    eigenvalues of A come in complex-conjugate pairs."""
    L, m = 8, 0.1
    F = operators.FineOperators(rand_theta(L, 8), m)
    A, B, Bi = F.A.toarray(), F.B.toarray(), F.Binv.toarray()
    E = np.diag(F.eps.astype(float))
    g5L, g5R = E @ Bi, B @ E
    assert np.max(np.abs(g5L @ A - A.conj().T @ g5L)) < 1e-12
    assert np.max(np.abs(A @ g5R - g5R @ A.conj().T)) < 1e-12
    assert np.max(np.abs(g5L @ g5R - np.eye(L * L))) < 1e-13
    ev = np.linalg.eigvals(A)
    d = np.abs(ev[:, None] - np.conj(ev)[None, :]).min(axis=1)
    assert d.max() < 1e-9


def test_A_definition_and_block_parity():
    """Eq. defA: A = D B^-1 = I + C B^-1; A_ee = A_oo = I on KD-block parity."""
    L, m = 8, 0.15
    F = operators.FineOperators(rand_theta(L, 10), m)
    A = F.A.toarray()
    I = np.eye(L * L)
    assert np.max(np.abs(A - (I + F.C.toarray() @ F.Binv.toarray()))) < 1e-13
    assert np.max(np.abs(F.B.toarray() @ F.Binv.toarray() - I)) < 1e-13
    e, o = F.even, F.odd
    assert np.max(np.abs(A[np.ix_(e, e)] - np.eye(e.size))) < 1e-14
    assert np.max(np.abs(A[np.ix_(o, o)] - np.eye(o.size))) < 1e-14


def test_schur_solve_reproduces_dense_solve():
    """Table kcycle, level 1: solving (I - A_eo A_oe) z_e = b_e - A_eo b_o, then
    z_o = b_o - A_oe z_e and x = B^-1 z solves D x = b."""
    L, m = 8, 0.05
    th = rand_theta(L, 12)
    F = operators.FineOperators(th, m)
    b = si.gaussian_complex(99, L * L)
    e = F.even
    S = np.eye(e.size) - (F.A_eo @ F.A_oe).toarray()
    ze = np.linalg.solve(S, F.schur_rhs(b))
    x = F.reconstruct(b, ze)
    xd = np.linalg.solve(dense_D(th, m), b)
    assert np.max(np.abs(x - xd)) / np.max(np.abs(xd)) < 1e-12
    # S applied through the oracle's sparse route equals the dense Schur matrix
    v = si.gaussian_complex(5, e.size)
    assert np.max(np.abs(F.schur(v) - S @ v)) < 1e-13


def test_maps_of_the_paper():
    L = 16
    et = lattice.eta(L, L)
    x0, x1 = lattice.coords(L, L)
    assert np.all(et[0] == 1) and np.all(et[1] == (-1) ** x0)
    assert np.all(lattice.epsilon(L, L) == (-1) ** (x0 + x1))
    agg = lattice.fine_aggregate(L, L, 4, 4)
    assert np.bincount(agg).tolist() == [64] * 4
    # each aggregate holds 32 sites of each chirality, 16 KD blocks
    eps = lattice.epsilon(L, L)
    for a in range(4):
        assert np.sum(eps[agg == a] == 1) == 32
        assert np.unique(lattice.kd_block(L, L)[agg == a]).size == 16


def test_cg_even_odd_solves_the_system():
    """Sec. II, Eq. normal: D^dag D is block diagonal over the site parity, and
    CG on m^2 - D_eo D_oe followed by the odd reconstruction solves D x = b."""
    L, m = 16, 0.05
    th = rand_theta(L, 31)
    D = dense_D(th, m)
    N = D.conj().T @ D
    eps = lattice.epsilon(L, L)
    e, o = eps > 0, eps < 0
    assert np.max(np.abs(N[np.ix_(e, o)])) < 1e-14
    b = si.gaussian_complex(77, L * L)
    x, k = operators.cg_eo_solve(th, m, b, 1e-10, 10000)
    assert np.linalg.norm(b - D @ x) / np.linalg.norm(b) <= 1e-10
    assert np.max(np.abs(x - np.linalg.solve(D, b))) / np.max(np.abs(x)) < 1e-8


@pytest.mark.parametrize("m", [0.0, 0.2])
def test_naik_free_spectrum(m):
    """Eq. freehisq: lambda = m +- i sqrt(sum_mu sin^2 p (1 + sin^2 p / 6)^2), each twice."""
    L = 16
    ev = np.linalg.eigvals(operators.dirac_naik(np.zeros((2, L, L)), m).toarray())
    n = np.arange(-L // 4 + 1, L // 4 + 1)
    p = 2 * np.pi * n / L
    f = (np.sin(p) * (1 + np.sin(p) ** 2 / 6)) ** 2
    s = np.sqrt(f[:, None] + f[None, :]).ravel()
    exp = np.concatenate([m + 1j * s, m - 1j * s, m + 1j * s, m - 1j * s])
    key = lambda z: np.lexsort((np.round(z.real, 9), np.round(z.imag, 9)))
    assert np.max(np.abs(ev[key(ev)] - exp[key(exp)])) < 1e-12


def test_naik_kd_free_spectrum_and_block():
    """Sec. II.A, Naik paragraph: B_Naik is the unimproved block with its hops
    rescaled (9/8 here, 9/16 in the printed normalisation), and the massless
    free KD spectrum is 1 - [(1-x) S1 + x S2] +- i sqrt(1 - [(1-x) S1 + x S2]^2
    - 2x [S2 - S1 + x (S3 - 1)]), S_n = (1/2) sum_mu cos(n p_mu), x = -1/27."""
    L = 16
    th = np.zeros((2, L, L))
    Dn, Bn, An = operators.naik_kd_operator(th, 0.0)
    B = operators.FineOperators(th, 0.3).B.toarray() - 0.3 * np.eye(L * L)
    assert np.max(np.abs(Bn.toarray() - 9.0 / 8.0 * B)) < 1e-15
    ev = np.linalg.eigvals(An.toarray())
    x = (-1.0 / 48.0) / (9.0 / 16.0)
    p = 2 * np.pi * np.arange(L // 2) / (L // 2)
    P0, P1 = np.meshgrid(p, p, indexing="ij")
    S = lambda k: 0.5 * (np.cos(k * P0) + np.cos(k * P1)).ravel()
    c = (1 - x) * S(1) + x * S(2)
    im = np.sqrt((1 - c * c - 2 * x * (S(2) - S(1) + x * (S(3) - 1))).astype(complex))
    exp = np.concatenate([1 - c + 1j * im, 1 - c - 1j * im] * 2)
    assert spectra_distance(ev, exp) < 1e-7  # square-root branch points cost precision


def spectra_distance(a, b):
    """Largest distance of the optimal one-to-one matching of two spectra."""
    from scipy.optimize import linear_sum_assignment
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return float(cost[r, c].max())


def test_naik_invariants():
    """The gauged Naik operator keeps eps-Hermiticity and gauge covariance."""
    L, m = 12, 0.1
    th = rand_theta(L, 40)
    Dn = operators.dirac_naik(th, m).toarray()
    eps = np.diag(lattice.epsilon(L, L).astype(float))
    assert np.max(np.abs(eps @ Dn @ eps - Dn.conj().T)) < 1e-15
    alpha = np.random.default_rng(41).uniform(-np.pi, np.pi, (L, L))
    G = np.diag(np.exp(1j * alpha.ravel()))
    Dg = operators.dirac_naik(si.gauge_transform(th, alpha), m).toarray()
    assert np.max(np.abs(Dg - G @ Dn @ G.conj().T)) < 1e-14
