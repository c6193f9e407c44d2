"""Index maps of the 2D staggered lattice and its multigrid hierarchy (oracle).

Site order: s = x0 + L0 * x1 (x0 fastest), periodic in both directions.
"""
from __future__ import annotations

import numpy as np


def coords(L0: int, L1: int):
    """Arrays x0[s], x1[s] for s = x0 + L0 * x1."""
    s = np.arange(L0 * L1)
    return s % L0, s // L0


def site(x0, x1, L0: int, L1: int):
    """Lexicographic index of (x0, x1) with periodic wrap."""
    return (np.asarray(x0) % L0) + L0 * (np.asarray(x1) % L1)


def eta(L0: int, L1: int) -> np.ndarray:
    """Staggered phases eta_mu(x) = (-1)^(sum_{nu<mu} x_nu) (Sec. II, definition after Eq. staggeredD).

    In 2D: eta_0 = 1 and eta_1 = (-1)^x0.  Returns int array [2, N].
    """
    x0, x1 = coords(L0, L1)
    return np.stack([np.ones_like(x0), np.where(x0 % 2 == 0, 1, -1)])


def epsilon(L0: int, L1: int) -> np.ndarray:
    """Chirality epsilon(x) = (-1)^(x0 + x1) (Eq. epsilon)."""
    x0, x1 = coords(L0, L1)
    return np.where((x0 + x1) % 2 == 0, 1, -1)


def kd_block(L0: int, L1: int) -> np.ndarray:
    """Kaehler-Dirac block index of each site: 2x2 blocks with corners at even
    coordinates (Sec. II.A, Fig. BC_partition; corner at 2n as in Eq. localblock).  Block
    (X0, X1) = (x0 // 2, x1 // 2) gets index X0 + (L0 / 2) X1."""
    x0, x1 = coords(L0, L1)
    return (x0 // 2) + (L0 // 2) * (x1 // 2)


def kd_parity(L0: int, L1: int) -> np.ndarray:
    """Parity (X0 + X1) mod 2 of the Kaehler-Dirac block holding each site.

    Reading of the paper's fine-level "even/odd" (Sec. IV, Table kcycle): the parity of
    the 2x2 blocks, the only site partition on which A_ee = A_oo = I."""
    x0, x1 = coords(L0, L1)
    return ((x0 // 2) + (x1 // 2)) % 2


def fine_aggregate(L0: int, L1: int, a0: int, a1: int) -> np.ndarray:
    """Level-1 aggregate of each site: a0 x a1 KD blocks = 2a0 x 2a1 sites
    (Table kcycle: 4^2 KD blocks, 8^2 fine sites).  Coarse site index
    X0 + E0 X1 with E0 = L0 / (2 a0)."""
    x0, x1 = coords(L0, L1)
    E0 = L0 // (2 * a0)
    return (x0 // (2 * a0)) + E0 * (x1 // (2 * a1))


def coarse_aggregate(E0: int, E1: int, b0: int, b1: int) -> np.ndarray:
    """Aggregate of each coarse site of an E0 x E1 coarse lattice with b0 x b1
    coarse sites per aggregate (Table kcycle: 2^2 on levels > 1)."""
    X = np.arange(E0 * E1)
    X0, X1 = X % E0, X // E0
    return (X0 // b0) + (E0 // b0) * (X1 // b1)
