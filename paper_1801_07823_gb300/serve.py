"""Serving loop: a stream of single-RHS solve requests over resident gauge fields.

Requests (gauge field, mass, right-hand side) arrive at any time.  Each worker
owns one CUDA stream and one libsw context and keeps the multigrid
hierarchies it has built resident on the device (an LRU cache keyed by gauge
field and mass).  A request is admitted when a worker is free and its
hierarchy is cached or fits into the HBM budget (least recently used
hierarchies of idle workers are evicted to make room); otherwise it waits.
Admitted requests run concurrently on the workers' streams, so the solves of
different requests overlap on the GPU while new requests keep arriving
(continuous admission).  Every kernel of the library sums in a fixed order
and each context has its own scratch, so a request's result is bitwise the
same whether it runs alone or in the mix.

Masses are served from a fixed grid (hierarchies are per mass): a request's
mass is rounded to the nearest grid value on a log scale.

With batch_max > 1 a worker that takes a request also takes the other queued
requests on the same hierarchy (same gauge field and mass, hence the same
level shapes), up to batch_max in all, and solves them in one
sw_mg_solve_batch call (on a mixed hierarchy: one lockstep K-cycle and one
batched coarsest solve per visit).  Every request then goes through
sw_mg_solve_batch, whose result for a right-hand side does not depend on its
batch-mates, so a request's result is still the same whatever it was grouped
with.  The admission model then also counts the batch workspace.
"""
from __future__ import annotations

import heapq
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import SW_MG_MIXED, sw_context_create, sw_gauge_load, sw_mg_params_default, sw_mg_setup
from . import sw_context_set_sm_share, sw_mg_solve, sw_mg_solve_batch


def hierarchy_bytes(L: int, blocks, nvec, mixed: bool, outer_restart: int = 32,
                    inter_restart: int = 8) -> int:
    """Device bytes of a 3-level (or 2-level) hierarchy and its solve workspace
    (complex128 = 16 B), from the sizes of its arrays."""
    N = L * L
    b = N * 64                                     # B^-1 table
    b += N * 16 * (4 + 3)                          # fine scratch, lexicographic/parity-split copies
    b += (N // 2) * 16 * (2 * outer_restart + 13)  # FGCR basis and K-cycle vectors (even half)
    sites, nc = N, 1
    E = L
    for l, (blk, nv) in enumerate(zip(blocks, nvec)):
        b += sites * nc * nv * 16                  # P
        E = E // (2 * blk[0]) if l == 0 else E // blk[0]
        sites, nc = E * E, 2 * nv
        last = l == len(nvec) - 1
        ysz = sites * 5 * nc * nc
        b += ysz * 16                              # Y (FP64)
        if last:
            b += ysz * 8 + sites * nc * 64         # sum plane and vector forms of its FP64 CGNE
        if mixed:
            b += ysz * (16 if last else 4) + sites * 5 * 4
        nb = 0 if last else inter_restart
        b += sites * nc * 16 * (2 * nb + 13)       # solver vectors of this level
    if mixed:
        b += N * 32 + N * 8                        # FP32 B^-1 and scratch
    return int(b)


def batch_workspace_bytes(L: int, blocks, nvec, outer_restart: int = 32,
                          inter_restart: int = 8, width: int = 16) -> int:
    """Device bytes of the workspace of batched solves, from the sizes of its
    arrays: per-right-hand-side work vectors for `width` right-hand sides
    (grown on demand), plus the arrays every batch shares, which are sized for
    the widest batch (64): the coarsest iterates, the stacked TF32 stencil tiles
    of A and A^dag, the TF32 right-hand-side tiles and the fine staging
    buffers."""
    N = L * L
    lens = [N // 2]                                 # level 1: even half of the fine lattice
    E, nc = L, 1
    for l, (blk, nv) in enumerate(zip(blocks, nvec)):
        E = E // (2 * blk[0]) if l == 0 else E // blk[0]
        nc = 2 * nv
        lens.append(E * E * nc)
    b = 0
    for l, n in enumerate(lens):
        last = l == len(lens) - 1
        nbas = 0 if last else (outer_restart if l == 0 else inter_restart)
        per_rhs = 2 if last else 2 + 2 + 2 * nbas + 6
        b += width * per_rhs * n * 16
    wmax = 64
    n_last = lens[-1]
    sites = n_last // nc
    b += 3 * n_last * wmax * 16                     # iterates X, R, P
    b += 2 * sites * 5 * 128 * nc * 4               # stacked TF32 tiles of A and A^dag
    b += 2 * sites * 2 * wmax * nc * 4              # TF32 right-hand-side tiles of r and p
    b += 3 * N * wmax * 16                          # fine staging buffers
    return int(b)


@dataclass(order=True)
class Request:
    arrival: float
    rid: int = field(compare=False)
    gauge: int = field(compare=False)
    mass: float = field(compare=False)
    b: np.ndarray = field(compare=False, repr=False)
    x: np.ndarray = field(default=None, compare=False, repr=False)
    start: float = field(default=0.0, compare=False)
    finish: float = field(default=0.0, compare=False)
    worker: int = field(default=-1, compare=False)
    stats: dict = field(default=None, compare=False)
    batch: int = field(default=1, compare=False)     # requests solved in the same call


class Server:
    """Multi-worker solve server on one GPU.

    gauges: list of (theta [2, L, L], label).  masses: the mass grid.
    psi0_fn: optional function (L, blocks, nvec) -> initial null-vector guesses.
    workers: number of concurrent streams.  hbm_budget: bytes that resident
    hierarchies may use in total.  sm_share: (num, den) share of the SMs each
    worker's persistent coarsest kernels hold (default 1/workers, so that the
    coarsest solves of all workers can run at the same time); a request's
    result depends on the share, not on the other requests in flight.
    affinity: every hierarchy (gauge field, mass) belongs to one worker (dealt
    round-robin in order of first use), which serves all of its requests, so
    each hierarchy is set up once and its queued requests meet in one queue
    for batching; without it any free worker takes any request and builds the
    hierarchies it needs itself.  hier_cfg: optional function L -> (blocks,
    nvec) giving the hierarchy of a lattice size (default: blocks and nvec for
    every size), e.g. one more level for the largest lattices."""

    def __init__(self, gauges, masses, workers=2, hbm_budget=40 << 30, tol=1e-10, mixed=True,
                 blocks=((4, 4), (2, 2)), nvec=(24, 32), params=None, device=0, psi0_fn=None,
                 batch_max=1, sm_share=None, affinity=False, hier_cfg=None):
        import torch
        if int(batch_max) > 1 and not mixed:
            raise ValueError("batch_max > 1 needs mixed=True: sw_mg_solve_batch batches the "
                             "coarsest solves of mixed-precision hierarchies only")
        self.torch = torch
        self.gauges = gauges
        self.masses = np.array(sorted(masses))
        self.tol = tol
        self.mixed = mixed
        self.blocks = [tuple(b) for b in blocks]
        self.nvec = list(nvec)
        self.hier_cfg = hier_cfg
        self.params = params or {}
        self.budget = hbm_budget
        self.psi0_fn = psi0_fn
        self.batch_max = max(1, min(64, int(batch_max)))
        self.affinity = affinity
        self.owner = {}
        self.lock = threading.Condition()
        self.queue: list[Request] = []
        self.done: list[Request] = []
        self.closed = False
        self.used = 0
        self.workers = []
        for w in range(workers):
            with torch.cuda.device(device):
                stream = torch.cuda.Stream()
            ctx = sw_context_create(device, stream.cuda_stream)
            share = sm_share or (1, workers)
            sw_context_set_sm_share(ctx, share[0], share[1])
            gh = [sw_gauge_load(ctx, th) for th, _ in gauges]
            self.workers.append(dict(id=w, stream=stream, ctx=ctx, gauges=gh, cache={},
                                     busy=False, thread=None))
        for wk in self.workers:
            t = threading.Thread(target=self._run, args=(wk,), daemon=True)
            wk["thread"] = t
            t.start()

    # ------------------------------------------------------------------ API
    def snap_mass(self, m: float) -> float:
        return float(self.masses[np.argmin(np.abs(np.log(self.masses) - np.log(m)))])

    def _own(self, key):
        """Worker that owns hierarchy `key` under affinity (lock held)."""
        if key not in self.owner:
            self.owner[key] = len(self.owner) % len(self.workers)
        return self.owner[key]

    def prewarm(self, keys):
        """Builds the hierarchies of (gauge, mass) keys before requests arrive
        (on their owners under affinity, else on every worker) and returns the
        wall time it took."""
        t0 = time.perf_counter()
        jobs = []
        for wk in self.workers:
            mine = [k for k in keys if not self.affinity or self._own(k) == wk["id"]]
            jobs.append(threading.Thread(target=lambda w=wk, ks=mine: [self._hierarchy(w, k)
                                                                        for k in ks]))
        for j in jobs:
            j.start()
        for j in jobs:
            j.join()
        return time.perf_counter() - t0

    def submit(self, rid: int, gauge: int, mass: float, b: np.ndarray) -> Request:
        r = Request(time.perf_counter(), rid, gauge, self.snap_mass(mass), b)
        with self.lock:
            if self.affinity:
                self._own((r.gauge, r.mass))
            heapq.heappush(self.queue, r)
            self.lock.notify_all()
        return r

    def drain(self):
        with self.lock:
            while self.queue or any(w["busy"] for w in self.workers):
                self.lock.wait(timeout=0.1)

    def close(self):
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        for wk in self.workers:
            wk["thread"].join()
        for wk in self.workers:
            for h in wk["cache"].values():
                h["mg"].free()
            for g in wk["gauges"]:
                g.free()
            wk["ctx"].free()

    # ------------------------------------------------------------------ workers
    def _cfg(self, L: int):
        if self.hier_cfg is None:
            return self.blocks, self.nvec
        blocks, nvec = self.hier_cfg(L)
        return [tuple(b) for b in blocks], list(nvec)

    def _footprint(self, gauge: int) -> int:
        L = self.gauges[gauge][0].shape[-1]
        blocks, nvec = self._cfg(L)
        b = hierarchy_bytes(L, blocks, nvec, self.mixed)
        if self.batch_max > 1 and self.mixed:
            b += batch_workspace_bytes(L, blocks, nvec, width=min(64, 2 * self.batch_max))
        return b

    def _companions(self, r):
        """Queued requests on r's hierarchy, earliest first, that join r's batch
        (lock held)."""
        if self.batch_max <= 1:
            return []
        same = sorted(q for q in self.queue if q is not r and (q.gauge, q.mass) == (r.gauge, r.mass))
        return same[:self.batch_max - 1]

    def _pick(self, wk):
        """Request this worker serves next (lock held): the earliest one whose
        hierarchy it already holds, else the earliest one whose hierarchy fits
        the HBM budget after evicting this worker's least recently used ones."""
        order = sorted(self.queue)
        if self.affinity:
            order = [r for r in order if self.owner[(r.gauge, r.mass)] == wk["id"]]
        for r in order:
            if (r.gauge, r.mass) in wk["cache"]:
                return r, 0
        for r in order:
            need = self._footprint(r.gauge)
            while self.used + need > self.budget and wk["cache"]:
                k = min(wk["cache"], key=lambda kk: wk["cache"][kk]["last"])
                h = wk["cache"].pop(k)
                h["mg"].free()
                self.used -= h["bytes"]
            if self.used + need <= self.budget:
                return r, need
        return None, 0

    def _hierarchy(self, wk, key, need=None):
        """Sets up (once) the hierarchy `key` on worker wk's stream and context."""
        if key in wk["cache"]:
            return wk["cache"][key]
        if need is None:  # prewarm: account for it here
            need = self._footprint(key[0])
            with self.lock:
                self.used += need
        gauge, mass = key
        p = sw_mg_params_default()
        for k, v in self.params.items():
            setattr(p, k, v)
        if self.mixed:
            p.precision = SW_MG_MIXED
        L = self.gauges[gauge][0].shape[-1]
        blocks, nvec = self._cfg(L)
        psi0 = self.psi0_fn(L, blocks, nvec) if self.psi0_fn else None
        with self.torch.cuda.stream(wk["stream"]):
            mg = sw_mg_setup(wk["gauges"][gauge], mass, len(nvec) + 1, blocks, nvec, params=p,
                             psi0=psi0)
        wk["cache"][key] = dict(mg=mg, bytes=need, last=time.perf_counter())
        return wk["cache"][key]

    def _run(self, wk):
        torch = self.torch
        while True:
            with self.lock:
                while True:
                    if self.closed and not self.queue:
                        return
                    r, need = self._pick(wk) if self.queue else (None, 0)
                    if r is not None:
                        batch = [r] + self._companions(r)
                        taken = {id(q) for q in batch}
                        self.queue = [q for q in self.queue if id(q) not in taken]
                        heapq.heapify(self.queue)
                        self.used += need
                        wk["busy"] = True
                        break
                    self.lock.wait(timeout=0.05)
            t_start = time.perf_counter()
            for q in batch:
                q.start = t_start
                q.worker = wk["id"]
            try:
                with torch.cuda.stream(wk["stream"]):
                    key = (r.gauge, r.mass)
                    if key not in wk["cache"]:
                        try:
                            self._hierarchy(wk, key, need)
                        except Exception:
                            with self.lock:
                                self.used -= need
                            raise
                    h = wk["cache"][key]
                    h["last"] = time.perf_counter()
                    if self.batch_max > 1:
                        B = np.stack([q.b for q in batch])
                        X = np.zeros_like(B)
                        sts = sw_mg_solve_batch(h["mg"], B, X, self.tol, allow_noconv=True)
                        for q, xq, sq in zip(batch, X, sts):
                            q.x, q.stats = xq, sq
                    else:
                        x = np.zeros_like(r.b)
                        r.stats = sw_mg_solve(h["mg"], r.b, x, self.tol, allow_noconv=True)
                        r.x = x
            except Exception as exc:  # failed requests are reported, the worker goes on
                for q in batch:
                    q.stats = {"converged": 0, "error": f"{type(exc).__name__}: {exc}"}
            t_end = time.perf_counter()
            for q in batch:
                q.finish = t_end
                q.batch = len(batch)
            with self.lock:
                wk["busy"] = False
                self.done.extend(batch)
                self.lock.notify_all()


def latency_summary(done) -> dict:
    lat = np.array([r.finish - r.arrival for r in done])
    if lat.size == 0:
        return {}
    span = max(r.finish for r in done) - min(r.arrival for r in done)
    return {"requests": int(lat.size), "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "solves_per_s": float(lat.size / span), "makespan_s": float(span),
            "all_converged": bool(all(r.stats.get("converged") for r in done)),
            "failed": int(sum(1 for r in done if not r.stats.get("converged"))),
            "mean_batch": float(np.mean([r.batch for r in done]))}


def poisson_stream(server, requests, rate, seed=0):
    """Submits (gauge, mass, b) requests at Poisson arrival times with the given
    rate (1/s) and waits until all are done; returns the finished requests.
    Bound the time of each solve with the server's solver parameters
    (outer_maxiter)."""
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    t = 0.0
    for i, (gauge, mass, b) in enumerate(requests):
        t += rng.exponential(1.0 / rate)
        delay = t0 + t - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        server.submit(i, gauge, mass, b)
    server.drain()
    return sorted(server.done, key=lambda r: r.rid)
