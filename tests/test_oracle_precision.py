"""Reduced-precision coarsest operands (oracle/precision.py): the rounding
emulation against torch's bfloat16 conversion and exact ties, and CGNE to
0.2 on a coarsest operator of the paper's hierarchy with FP32, TF32, BF16
and 3xTF32 operands."""
import numpy as np
import pytest

import sw_inputs as si
from oracle import precision


def test_round_mantissa_matches_bfloat16_and_ties():
    torch = pytest.importorskip("torch")
    x = (si.gaussian_complex(77, 4096).real * 10.0 ** np.arange(-4, 4).repeat(512)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(precision.round_mantissa(x, 7), ref)
    one = np.float32(1.0)
    ulp10 = np.float32(2.0 ** -10)
    assert precision.round_mantissa(np.array([one + ulp10 / 2]), 10)[0] == one          # tie to even
    assert precision.round_mantissa(np.array([one + 3 * ulp10 / 2]), 10)[0] == one + 2 * ulp10
    assert precision.round_mantissa(np.array([-(one + 3 * ulp10 / 4)]), 10)[0] == -(one + ulp10)
    assert np.array_equal(precision.round_mantissa(x, 23), x)


def test_reduced_precision_cgne_reaches_the_coarsest_tolerance():
    A, Ad = precision.coarsest_operator(64)
    b = si.gaussian_complex(9000, A.shape[0])
    k64, r64 = precision.cgne_iterations(A, Ad, "fp64", b)
    assert r64 <= 0.2
    growth = {"fp32": 1.1, "3xtf32": 1.1, "tf32": 1.2, "bf16": 1.25}
    for form, g in growth.items():
        k, r = precision.cgne_iterations(A, Ad, form, b)
        # the recursive residual of the emulated operator drifts slightly from the true one
        assert r <= 0.21, (form, r)
        assert k64 <= k * 1.02 and k <= g * k64, (form, k, k64)
