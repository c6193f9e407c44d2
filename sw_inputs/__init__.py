"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module generates inputs only: U(1) gauge fields from a heatbath of the
Wilson plaquette action and complex Gaussian vectors.  It holds none of the
multigrid method's arithmetic (no Dirac operator, no transfer, no solver).

Random numbers come from one counter-based generator, SplitMix64
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014): the n-th 64-bit output of stream ``seed`` is
``mix(seed + (n + 1) * 0x9E3779B97F4A7C15)`` with the SplitMix64 finaliser
``mix``.  Gaussians use the Box-Muller transform of two such uniforms.
Vectors are plain numpy; the gauge heatbath runs with torch float64 on the CPU
or a CUDA device (same algorithm and counters; the field is a deterministic
function of the seed and the device type).
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wraps modulo 2**64)."""
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Outputs number ``counters`` (uint64 array) of the SplitMix64 stream ``seed``."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * GOLDEN
    return _mix(state)


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Doubles in (0, 1]: the top 53 bits of the SplitMix64 output, plus one ulp."""
    u = splitmix64(seed, counters)
    return ((u >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def stream_seed(seed: int, *keys: int) -> int:
    """Derives an independent stream seed from ``seed`` and integer keys."""
    s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    for k in keys:
        with np.errstate(over="ignore"):
            s = _mix(s ^ np.uint64(k & 0xFFFFFFFFFFFFFFFF)) + GOLDEN
    return int(s[0])


def gaussian_complex(seed: int, n: int) -> np.ndarray:
    """n complex numbers with independent N(0,1) real and imaginary parts.

    Element j takes uniforms 2j and 2j+1 of stream ``seed``;
    Box-Muller: re = r cos(2 pi u2), im = r sin(2 pi u2), r = sqrt(-2 ln u1).
    """
    j = np.arange(n, dtype=np.uint64)
    u1 = uniform01(seed, 2 * j)
    u2 = uniform01(seed, 2 * j + np.uint64(1))
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * np.pi * u2
    return r * np.cos(t) + 1j * r * np.sin(t)


def gaussian_source(seed: int, L0: int, L1: int) -> np.ndarray:
    """A complex Gaussian fermion source as a [L1, L0] complex128 array."""
    return gaussian_complex(seed, L0 * L1).reshape(L1, L0)


_MASK = {k: (1 << (64 - k)) - 1 for k in (11, 27, 30, 31)}


def _tmix(z):
    """SplitMix64 finaliser on an int64 torch tensor (two's-complement wrap,
    logical right shifts by masking)."""
    z = (z ^ ((z >> 30) & _MASK[30])) * _as_i64(0xBF58476D1CE4E5B9)
    z = (z ^ ((z >> 27) & _MASK[27])) * _as_i64(0x94D049BB133111EB)
    return z ^ ((z >> 31) & _MASK[31])


def _as_i64(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def torch_uniform01(seed: int, counters):
    """Same values as ``uniform01`` for int64 torch counters (any device)."""
    state = _as_i64(seed) + (counters + 1) * _as_i64(0x9E3779B97F4A7C15)
    u = _tmix(state)
    return (((u >> 11) & _MASK[11]).double() + 1.0) * (2.0 ** -53)


def _von_mises(seed: int, ctr0: int, kappa, max_attempts: int = 64):
    """Samples angles with density proportional to exp(kappa cos t), t in (-pi, pi].

    Best and Fisher (1979), "Efficient simulation of the von Mises distribution",
    Appl. Statist. 28, 152: rejection from a wrapped Cauchy envelope.  Element i,
    attempt a uses uniforms ctr0 + (a * n + i) * 3 + {0, 1, 2}.  A sample that is
    still rejected after ``max_attempts`` is drawn uniformly (probability far below
    1e-30 at the couplings used here).  kappa: float64 torch tensor.
    """
    import torch
    n = kappa.numel()
    dev = kappa.device
    out = torch.zeros(n, dtype=torch.float64, device=dev)
    small = kappa < 1e-8
    kap = torch.where(small, torch.ones_like(kappa), kappa)
    tau = 1.0 + torch.sqrt(1.0 + 4.0 * kap * kap)
    rho = (tau - torch.sqrt(2.0 * tau)) / (2.0 * kap)
    r = (1.0 + rho * rho) / (2.0 * rho)
    idx = torch.arange(n, device=dev)

    def attempt(a, sel):
        base = ctr0 + (a * n + sel) * 3
        u1 = torch_uniform01(seed, base)
        u2 = torch_uniform01(seed, base + 1)
        u3 = torch_uniform01(seed, base + 2)
        rr = r[sel]
        z = torch.cos(torch.pi * u1)
        f = (1.0 + rr * z) / (rr + z)
        c = kap[sel] * (rr - f)
        ok = (c * (2.0 - c) - u2 > 0.0) | (torch.log(c / u2) + 1.0 - c >= 0.0)
        sm = small[sel]
        ok = ok | sm
        ang = torch.where(u3 > 0.5, 1.0, -1.0) * torch.arccos(torch.clamp(f, -1.0, 1.0))
        ang = torch.where(sm, torch.pi * (2.0 * u3 - 1.0), ang)
        return ok, ang

    # The first attempts run on every element without compaction (no host
    # synchronisation); an element keeps the angle of its first accepted attempt,
    # which is what the one-at-a-time rejection loop gives.
    accepted = torch.zeros(n, dtype=torch.bool, device=dev)
    first = min(8, max_attempts)
    for a in range(first):
        ok, ang = attempt(a, idx)
        take = ok & ~accepted
        out = torch.where(take, ang, out)
        accepted |= ok
    todo = idx[~accepted]
    for a in range(first, max_attempts):
        if todo.numel() == 0:
            break
        ok, ang = attempt(a, todo)
        out[todo[ok]] = ang[ok]
        todo = todo[~ok]
    if todo.numel():
        base = ctr0 + max_attempts * n * 3 + todo
        out[todo] = torch.pi * (2.0 * torch_uniform01(seed, base) - 1.0)
    return out


def heatbath_u1(L0: int, L1: int, beta: float, sweeps: int, seed: int,
                device: str = "cpu") -> np.ndarray:
    """Quenched compact U(1) gauge field theta[mu, x1, x0] after ``sweeps`` heatbath sweeps.

    Action S = beta * sum_plaquettes (1 - cos theta_p) with
    theta_p(x) = theta_0(x) + theta_1(x + 0hat) - theta_0(x + 1hat) - theta_1(x).
    Each link is redrawn from its exact conditional (von Mises) distribution
    given its two staples.  A sweep visits theta_0 on rows x1 even, then x1 odd,
    then theta_1 on columns x0 even, then x0 odd: links inside one such set share
    no plaquette, so they update together.  Cold start (theta = 0).  Periodic.
    Runs with torch float64 on ``device`` ("cpu" or "cuda"); the field is a
    deterministic function of (seed, device type).
    """
    import torch
    if L0 % 2 or L1 % 2:
        raise ValueError("heatbath needs even extents")
    th = torch.zeros((2, L1, L0), dtype=torch.float64, device=device)
    nl = (L0 * L1) // 2
    for sw in range(sweeps):
        for ps in range(4):
            mu, par = ps // 2, ps % 2
            t0, t1 = th[0], th[1]
            if mu == 0:
                # plaquette at x:      theta + [t1(x+0) - t0(x+1) - t1(x)]          = theta + a
                # plaquette at x-1hat: [t0(x-1) + t1(x-1+0) - t1(x-1)] - theta     = b - theta
                a = torch.roll(t1, -1, 1) - torch.roll(t0, -1, 0) - t1
                t0m = torch.roll(t0, 1, 0)
                t1m = torch.roll(t1, 1, 0)
                b = t0m + torch.roll(t1m, -1, 1) - t1m
                a, b = a[par::2, :], b[par::2, :]
                k = torch.exp(1j * a) + torch.exp(-1j * b)
            else:
                # plaquette at x:      [t0(x) + t1(x+0) - t0(x+1)] - theta          = a - theta
                # plaquette at x-0hat: theta + [t0(x-0) - t0(x-0+1) - t1(x-0)]     = theta + b
                a = t0 + torch.roll(t1, -1, 1) - torch.roll(t0, -1, 0)
                t0m = torch.roll(t0, 1, 1)
                b = t0m - torch.roll(t0m, -1, 0) - torch.roll(t1, 1, 1)
                a, b = a[:, par::2], b[:, par::2]
                k = torch.exp(-1j * a) + torch.exp(1j * b)
            # weight exp(beta |k| cos(theta + arg k)): theta = t - arg k, t ~ von Mises(beta |k|)
            kap = (beta * torch.abs(k)).reshape(-1)
            psi = torch.angle(k).reshape(-1)
            ctr0 = (sw * 4 + ps) * (nl * 3 * 65)
            t = _von_mises(seed, ctr0, kap)
            newv = torch.angle(torch.exp(1j * (t - psi))).reshape(a.shape)
            if mu == 0:
                th[0][par::2, :] = newv
            else:
                th[1][:, par::2] = newv
    return th.cpu().numpy()


def null_vector_guesses(L0: int, L1: int, nvec, levels: int, blocks, seed: int = 5):
    """Initial guesses of the null vectors, one [nvec[l], ndof] array per
    level l = 0 .. levels-2: Gaussian vectors from streams stream_seed(seed, l, i).
    Level 0 has one dof per fine site; level 1 has 2 nvec[0] dof per aggregate
    of blocks[0] KD blocks (2 blocks[0] fine sites per direction), and each
    further level 2 nvec[l-1] dof per aggregate of blocks[l-1] sites."""
    out = [np.stack([gaussian_complex(stream_seed(seed, 0, i), L0 * L1) for i in range(nvec[0])])]
    E0, E1 = L0 // (2 * blocks[0][0]), L1 // (2 * blocks[0][1])
    nc = 2 * nvec[0]
    for lv in range(1, levels - 1):
        out.append(np.stack([gaussian_complex(stream_seed(seed, lv, i), E0 * E1 * nc)
                             for i in range(nvec[lv])]))
        E0, E1, nc = E0 // blocks[lv][0], E1 // blocks[lv][1], 2 * nvec[lv]
    return out


def plaquette_mean(theta: np.ndarray) -> float:
    """Average cos(theta_p) over all plaquettes (input-quality diagnostic)."""
    t0, t1 = theta[0], theta[1]
    tp = t0 + np.roll(t1, -1, axis=1) - np.roll(t0, -1, axis=0) - t1
    return float(np.mean(np.cos(tp)))


def gauge_transform(theta: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """Links of the gauge-rotated field U^g_mu(x) = g(x) U_mu(x) g(x+mu)^*, g = exp(i alpha)."""
    t = theta.copy()
    t[0] = theta[0] + alpha - np.roll(alpha, -1, axis=1)
    t[1] = theta[1] + alpha - np.roll(alpha, -1, axis=0)
    return t
