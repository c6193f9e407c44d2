"""The allocation-free Schur operator against sw_dslash(SW_OP_S).

sw_dslash_schur_noalloc serves callers that cannot call cudaMalloc
(applications or frameworks that own every device allocation of the process,
loops that must not enter the allocator); it keeps its scratch in a fixed
device array.  This file is collected last so a
run that stops at the first failure has run every other test first.
"""
import numpy as np
import pytest

import sw_inputs as si
from tests.gpu_helpers import relerr

pytestmark = pytest.mark.gpu


def test_noalloc_schur_matches_dslash_twice():
    import torch
    import paper_1801_07823_gb300 as sw
    ctx = sw.sw_context_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        L0, L1 = 64, 48
        th = np.random.default_rng(11).uniform(-np.pi, np.pi, (2, L1, L0))
        g = sw.sw_gauge_load(ctx, th)
        # two calls in a row with different inputs and masses: the shared scratch
        # keeps the first call's contents, which must not leak into the second
        for seed, m in ((21, 0.07), (22, 0.013)):
            v = torch.from_numpy(si.gaussian_complex(seed, L0 * L1)).cuda()
            ref = torch.empty_like(v)
            out = torch.full_like(v, float("nan"))
            sw.sw_dslash(g, m, sw.SW_OP_S, sw.SW_PREC_FP64, v, ref)
            sw.sw_dslash_schur_noalloc(g, m, v, out)
            torch.cuda.synchronize()
            assert relerr(out.cpu().numpy(), ref.cpu().numpy()) < 1e-13
        big = sw.sw_gauge_load(ctx, np.zeros((2, 512, 512)))
        v = torch.zeros(512 * 512, dtype=torch.complex128, device="cuda")
        with pytest.raises(sw.SwError) as e:
            sw.sw_dslash_schur_noalloc(big, 0.1, v, v.clone())
        assert e.value.code == -2
        big.free()
        g.free()
    finally:
        ctx.free()
