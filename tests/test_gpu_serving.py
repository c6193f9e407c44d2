"""Serving loop: concurrent solves on several streams give, request by
request, bitwise the same results as solving each request alone."""
import numpy as np
import pytest

import sw_inputs as si
from tests.gpu_helpers import psi0_arrays

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("batch_max", [1, 4])
def test_serving_results_alone_equal_mixed(batch_max):
    """Each request's solution is bitwise the same when it is served alone and
    when it is served among concurrent requests on three workers, with and
    without batching of queued requests on one hierarchy (mixed precision, so
    batches use the tensor-core coarsest kernel); every worker holds a third of
    the SMs for its coarsest kernels in both runs.  With batching, some
    requests must have been solved in a batch."""
    from paper_1801_07823_gb300 import serve
    from oracle import operators
    gauges = [(si.heatbath_u1(L, L, beta, 200, seed=s, device="cuda"), f"L{L} b{beta}")
              for s, (L, beta) in enumerate([(32, 6.0), (64, 6.0), (32, 10.0), (64, 10.0)])]
    masses = [0.01, 0.1]
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(14):
        gid = int(rng.integers(2)) if batch_max > 1 else int(rng.integers(len(gauges)))
        L = gauges[gid][0].shape[-1]
        m = float(np.exp(rng.uniform(np.log(1e-2), np.log(1e-1))))
        reqs.append((gid, m, si.gaussian_complex(500 + i, L * L)))
    psi0 = lambda L, blocks, nvec: psi0_arrays(L, L, nvec, len(nvec) + 1, blocks)
    kw = dict(nvec=(8, 12), psi0_fn=psi0, hbm_budget=8 << 30, params=dict(outer_maxiter=300),
              batch_max=batch_max, sm_share=(1, 3))
    alone = serve.Server(gauges, masses, workers=1, **kw)
    for i, (gid, m, b) in enumerate(reqs):
        alone.submit(i, gid, m, b)
        alone.drain()
    ref = sorted(alone.done, key=lambda r: r.rid)
    alone.close()
    mix = serve.Server(gauges, masses, workers=3, **kw)
    got = serve.poisson_stream(mix, reqs, rate=400.0)
    summary = serve.latency_summary(got)
    workers_used = {r.worker for r in got}
    mix.close()
    assert summary["all_converged"] and len(got) == len(reqs)
    assert len(workers_used) > 1
    if batch_max > 1:
        assert max(r.batch for r in got) > 1
    for a, b in zip(ref, got):
        assert a.rid == b.rid and a.mass == b.mass
        assert np.array_equal(a.x, b.x), a.rid
        th = gauges[a.gauge][0]
        D = operators.dirac(th, a.mass)
        r = np.linalg.norm(reqs[a.rid][2] - D @ b.x) / np.linalg.norm(reqs[a.rid][2])
        assert r <= 1e-10


def test_hierarchy_footprint_model():
    """The admission model's byte count against the device memory a setup takes."""
    import torch
    import paper_1801_07823_gb300 as sw
    from paper_1801_07823_gb300 import serve
    L = 128
    th = si.heatbath_u1(L, L, 6.0, 10, seed=3, device="cuda")
    ctx = sw.sw_context_create(0)
    g = sw.sw_gauge_load(ctx, th)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    p = sw.sw_mg_params_default()
    p.precision = sw.SW_MG_MIXED
    h = sw.sw_mg_setup(g, 0.01, 3, [(4, 4), (2, 2)], [24, 32], params=p,
                       psi0=psi0_arrays(L, L, [24, 32], 3, [(4, 4), (2, 2)]))
    x = np.zeros(L * L, dtype=complex)
    sw.sw_mg_solve(h, si.gaussian_complex(1, L * L), x, 1e-8)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    model = serve.hierarchy_bytes(L, [(4, 4), (2, 2)], [24, 32], True)
    h.free()
    g.free()
    ctx.free()
    assert 0.6 * used <= model <= 1.6 * used + (8 << 20), (model, used)
