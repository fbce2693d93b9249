"""The skip-Cholesky's FP64 inverse square root (an FP32 estimate and one
third-order refinement step) against CUDA's 1.0 / sqrt on the device and
against the host's correctly rounded sqrt and division."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def ulps(a, b):
    return np.abs(a.view(np.int64) - b.view(np.int64))


def test_rsqrt_within_two_ulp():
    from paper_1710_03608_gb300 import ctd as m
    rng = np.random.default_rng(3)
    d = np.concatenate([
        np.logspace(-300, 300, 20001),          # both branches (the FP32 range and beyond)
        rng.uniform(0.5, 2.0, 200_000),          # one binade around 1, densely
        rng.lognormal(0.0, 15.0, 200_000),       # pivots of every size
        np.array([1e-30, 1e30, 1.0000000000000002e-30, 9.999999999999999e29, 1.0, 4.0,
                  2.0 ** -1022, 2.0 ** 1000, 3.0, 0.25]),
    ])
    d = d[(d > 0) & np.isfinite(d)]
    out, ref = m.selftest_rsqrt(d)
    assert ulps(out, ref).max() <= 2
    host = 1.0 / np.sqrt(d)
    assert ulps(out, host).max() <= 2
    # powers of 4: within one ulp of the exact power of 2
    p = 4.0 ** np.arange(-20, 21)
    out, _ = m.selftest_rsqrt(p)
    assert ulps(out, 2.0 ** -np.arange(-20, 21).astype(np.float64)).max() <= 1
