"""Host logic of the serving loop on CPU, with the library calls and CUDA
streams replaced by fakes: admission under the HBM budget with LRU eviction,
reuse of resident hierarchies, mass snapping, failure isolation, batching of
requests on one hierarchy and the latency summary."""
import contextlib
import threading
import time
import types

import numpy as np
import pytest

from paper_1801_07823_gb300 import serve


class _Fake:
    def __init__(self):
        self.lock = threading.Lock()
        self.live = 0          # hierarchies alive now
        self.max_live = 0
        self.setups = 0
        self.fail_mass = None  # a setup at this mass raises
        self.setup_delay = 0.0
        self.batches = []      # (mass, request ids) per batched call

    def context_create(self, device, stream):
        return types.SimpleNamespace(free=lambda: None)

    def gauge_load(self, ctx, th):
        return types.SimpleNamespace(free=lambda: None, L=th.shape[-1])

    def params_default(self):
        return types.SimpleNamespace(precision=0)

    def mg_setup(self, g, mass, levels, blocks, nvec, params=None, psi0=None):
        if mass == self.fail_mass:
            raise RuntimeError("setup failed")
        time.sleep(self.setup_delay)
        fake = self

        class _MG:
            def __init__(self):
                self.mass = mass
                self.freed = False

            def free(self):
                assert not self.freed
                self.freed = True
                with fake.lock:
                    fake.live -= 1

        with self.lock:
            self.setups += 1
            self.live += 1
            self.max_live = max(self.max_live, self.live)
        return _MG()

    def mg_solve(self, mg, b, x, tol, allow_noconv=False):
        assert not mg.freed
        x[:] = b / mg.mass
        return {"converged": 1, "outer_iters": 1, "true_resid": 0.0}

    def mg_solve_batch(self, mg, B, X, tol, allow_noconv=False):
        assert not mg.freed and B.ndim == 2 and X.shape == B.shape
        with self.lock:
            self.batches.append((mg.mass, B[:, 0].real.astype(int).tolist()))
        time.sleep(0.02)
        X[:] = B / mg.mass
        return [{"converged": 1, "outer_iters": 1, "true_resid": 0.0} for _ in range(len(B))]


@pytest.fixture()
def fake(monkeypatch):
    f = _Fake()
    monkeypatch.setattr(serve, "sw_context_create", f.context_create)
    monkeypatch.setattr(serve, "sw_gauge_load", f.gauge_load)
    monkeypatch.setattr(serve, "sw_mg_params_default", f.params_default)
    monkeypatch.setattr(serve, "sw_mg_setup", f.mg_setup)
    monkeypatch.setattr(serve, "sw_mg_solve", f.mg_solve)
    monkeypatch.setattr(serve, "sw_mg_solve_batch", f.mg_solve_batch)
    monkeypatch.setattr(serve, "sw_context_set_sm_share", lambda ctx, n, d: None)
    import torch
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "device", lambda *a, **k: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "stream", lambda *a, **k: contextlib.nullcontext())
    return f


def _gauges(L=16, n=2):
    return [(np.zeros((2, L, L)), f"g{i}") for i in range(n)]


def test_budget_admission_and_lru_eviction(fake):
    gauges = _gauges()
    one = serve.hierarchy_bytes(16, [(4, 4), (2, 2)], [24, 32], True)
    # room for two resident hierarchies, four (gauge, mass) keys in the stream
    srv = serve.Server(gauges, [1e-2, 1e-1], workers=2, hbm_budget=int(2.5 * one))
    try:
        rng = np.random.default_rng(0)
        reqs = []
        for i in range(24):
            gi, m = i % 2, (1e-2, 1e-1)[(i // 2) % 2]
            b = rng.standard_normal(256) + 1j * rng.standard_normal(256)
            reqs.append(srv.submit(i, gi, m, b))
        srv.drain()
        assert fake.max_live <= 2 and srv.used <= srv.budget
        assert len(srv.done) == 24
        for r in srv.done:
            assert r.stats["converged"] and np.allclose(r.x, r.b / r.mass)
            assert r.finish >= r.start >= r.arrival
    finally:
        srv.close()
    assert fake.live == 0


def test_resident_hierarchy_is_reused(fake):
    srv = serve.Server(_gauges(n=1), [1e-2], workers=1)
    try:
        for i in range(5):
            srv.submit(i, 0, 1e-2, np.ones(256, dtype=complex))
        srv.drain()
        assert fake.setups == 1 and len(srv.done) == 5
    finally:
        srv.close()


def test_mass_snapping_on_log_grid(fake):
    srv = serve.Server(_gauges(n=1), [1e-3, 1e-2, 1e-1], workers=1)
    try:
        assert srv.snap_mass(2e-3) == 1e-3
        assert srv.snap_mass(4e-3) == 1e-2  # log-midpoint of 1e-3 and 1e-2 is 3.16e-3
        assert srv.snap_mass(1.0) == 1e-1
    finally:
        srv.close()


def test_failed_setup_is_reported_and_worker_goes_on(fake):
    fake.fail_mass = 1e-1
    srv = serve.Server(_gauges(n=1), [1e-2, 1e-1], workers=1)
    try:
        srv.submit(0, 0, 1e-1, np.ones(256, dtype=complex))
        srv.submit(1, 0, 1e-2, np.ones(256, dtype=complex))
        srv.drain()
        by = {r.rid: r for r in srv.done}
        assert not by[0].stats["converged"] and "setup failed" in by[0].stats["error"]
        assert by[1].stats["converged"]
        assert srv.used == serve.hierarchy_bytes(16, [(4, 4), (2, 2)], [24, 32], True)
        s = serve.latency_summary(srv.done)
        assert s["requests"] == 2 and s["failed"] == 1 and not s["all_converged"]
        assert 0 <= s["p50_s"] <= s["p99_s"]
    finally:
        srv.close()


def test_requests_on_one_hierarchy_are_batched(fake):
    """batch_max > 1: requests queued on the same (gauge, mass) share one
    batched call, never with another hierarchy's; results and accounting per
    request are unchanged."""
    fake.setup_delay = 0.2          # the first setup lets the queue fill
    gauges = _gauges(n=2)
    srv = serve.Server(gauges, [1e-2, 1e-1], workers=1, batch_max=4)
    key = {}
    try:
        for i in range(14):
            gi, m = (0, 1e-2) if i < 10 else (1, 1e-1)
            key[i] = (gi, m)
            srv.submit(i, gi, m, np.full(256, float(i), dtype=complex))
        srv.drain()
        assert sorted(r.rid for r in srv.done) == list(range(14))
        for r in srv.done:
            assert r.stats["converged"] and np.allclose(r.x, r.b / r.mass)
        assert all(len(ids) <= 4 for _, ids in fake.batches)
        for mass, ids in fake.batches:      # one hierarchy per call
            assert len({key[i] for i in ids}) == 1 and key[ids[0]][1] == mass
        s = serve.latency_summary(srv.done)
        assert s["mean_batch"] > 1.0
        one = serve.hierarchy_bytes(16, [(4, 4), (2, 2)], [24, 32], True)
        assert srv._footprint(0) == one + serve.batch_workspace_bytes(16, [(4, 4), (2, 2)], [24, 32],
                                                                      width=8)
    finally:
        srv.close()


def test_batching_on_fp64_hierarchies_is_rejected(fake):
    """sw_mg_solve_batch batches mixed-precision hierarchies only, so a server
    that would batch FP64 hierarchies is refused when it is built, instead of
    failing every request later."""
    with pytest.raises(ValueError):
        serve.Server(_gauges(n=1), [1e-2], workers=1, mixed=False, batch_max=4)
    srv = serve.Server(_gauges(n=1), [1e-2], workers=1, mixed=False, batch_max=1)
    srv.close()


def test_affinity_sets_up_each_hierarchy_once(fake):
    """With affinity every (gauge, mass) hierarchy is built by one worker only,
    all of its requests run there, and prewarm builds them before requests
    arrive."""
    gauges = _gauges(n=3)
    srv = serve.Server(gauges, [1e-2, 1e-1], workers=2, affinity=True, batch_max=4)
    try:
        keys = [(g, m) for g in range(3) for m in (1e-2, 1e-1)]
        srv.prewarm(keys)
        assert fake.setups == len(keys)
        rng = np.random.default_rng(3)
        for i in range(30):
            gi, m = keys[int(rng.integers(len(keys)))]
            srv.submit(i, gi, m, np.full(256, float(i + 1), dtype=complex))
        srv.drain()
        assert fake.setups == len(keys) and len(srv.done) == 30
        by_key = {}
        for r in srv.done:
            by_key.setdefault((r.gauge, r.mass), set()).add(r.worker)
            assert np.allclose(r.x, r.b / r.mass)
        assert all(len(w) == 1 for w in by_key.values())
        assert len({w for ws in by_key.values() for w in ws}) == 2
    finally:
        srv.close()
