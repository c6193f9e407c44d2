"""Host logic of the serving loop on CPU, with the library calls and CUDA
streams replaced by fakes: admission under the HBM budget with LRU eviction,
reuse of resident hierarchies, mass snapping, failure isolation and the
latency summary."""
import contextlib
import threading
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

    def context_create(self, device, stream):
        return types.SimpleNamespace(free=lambda: None)

    def gauge_load(self, ctx, th):
        return types.SimpleNamespace(free=lambda: None, L=th.shape[-1])

    def params_default(self):
        return types.SimpleNamespace(precision=0)

    def mg_setup(self, g, mass, levels, blocks, nvec, params=None, psi0=None):
        if mass == self.fail_mass:
            raise RuntimeError("setup failed")
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


@pytest.fixture()
def fake(monkeypatch):
    f = _Fake()
    monkeypatch.setattr(serve, "sw_context_create", f.context_create)
    monkeypatch.setattr(serve, "sw_gauge_load", f.gauge_load)
    monkeypatch.setattr(serve, "sw_mg_params_default", f.params_default)
    monkeypatch.setattr(serve, "sw_mg_setup", f.mg_setup)
    monkeypatch.setattr(serve, "sw_mg_solve", f.mg_solve)
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
