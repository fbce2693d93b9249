"""The allocation-free sampling entry point, ctd_sample_noalloc.

Callers inside another allocator's arena, under a hard device-memory cap, or
on latency-critical paths cannot (or must not) call cudaMalloc.  For them the
library offers the front of CTD-S (column distribution, draws, unique draws)
with its scratch in fixed device arrays instead of fresh allocations.  These
tests call it through the C ABI and compare it with ctd_static's own draws;
integer results must match exactly.  The file is named so pytest runs it last.
"""
import numpy as np
import pytest

from paper_1710_03608_gb300 import synth

pytestmark = pytest.mark.gpu


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


def noalloc(m, X, s, seed, alpha=1):
    import torch
    draws = torch.full((s,), -7, dtype=torch.int64, device="cuda")
    uniq = torch.full((s,), -7, dtype=torch.int64, device="cuda")
    n = m.sample_noalloc(X, alpha, s, seed, draws, uniq)
    return draws.cpu().numpy(), uniq.cpu().numpy()[:n]


@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_two_calls_match_ctd_static(alpha):
    import torch
    m = ctd()
    coo = synth.small_uniform()
    X = m.Coo.from_synth(coo)
    F = m.ctd_static(X, alpha, 50, 1e-6, 3, m.CTD_FP64)
    I_ref, Iu_ref = F.samples()
    first = noalloc(m, X, 50, 3, alpha)
    free_before = torch.cuda.mem_get_info()[0]
    second = noalloc(m, X, 50, 3, alpha)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before  # nothing allocated
    for draws, uniq in (first, second):
        assert np.array_equal(draws, I_ref)
        assert np.array_equal(uniq, Iu_ref)


def test_previous_contents_do_not_leak():
    """A larger tensor first, then a smaller one: the shared arrays keep the
    last call's contents, so the entry point must clear them itself."""
    m = ctd()
    big = synth.traffic_10m(scale=0.3)
    small = synth.small_uniform()
    Xb, Xs = m.Coo.from_synth(big), m.Coo.from_synth(small)
    ref_b = m.ctd_static(Xb, 1, 500, 1e-6, 1, m.CTD_FP32_BULK, m.CTD_SKIP_C).samples()
    ref_s = m.ctd_static(Xs, 1, 50, 1e-6, 2, m.CTD_FP64, m.CTD_SKIP_C).samples()
    for X, s, seed, ref in ((Xb, 500, 1, ref_b), (Xs, 50, 2, ref_s)):
        draws, uniq = noalloc(m, X, s, seed)
        assert np.array_equal(draws, ref[0])
        assert np.array_equal(uniq, ref[1])


def test_all_zero_input_draws_nothing():
    """||X|| = 0: no column can be drawn.  ctd_static reports zero draws;
    this entry point marks every draw -1 and reports no unique draw."""
    m = ctd()
    coo = synth.tiny((5, 4, 3), 10, seed=1)
    coo.val[:] = 0
    X = m.Coo.from_synth(coo)
    assert m.ctd_static(X, 1, 10, 1e-6, 0, m.CTD_FP64).sizes().s_draws == 0
    draws, uniq = noalloc(m, X, 10, 0)
    assert np.all(draws == -1) and uniq.size == 0


def test_fiber_sum_overflow_is_reported():
    """Five values of 2^31 - 1 in one fiber: the column's sum of squares
    wraps a 64-bit accumulator; the call must still report CTD_EOVERFLOW."""
    m = ctd()
    big = 2 ** 31 - 1
    coo = synth.Coo3((8, 3, 2), np.arange(5), np.ones(5, np.int64), np.zeros(5, np.int64),
                     np.full(5, big, np.int64))
    with pytest.raises(m.CtdError) as e:
        noalloc(m, m.Coo.from_synth(coo), 5, 0)
    assert e.value.status == "CTD_EOVERFLOW"


def test_limits_are_reported():
    m = ctd()
    # N_alpha = 2048 * 1024 > CTD_NOALLOC_MAX_COLS: rejected before any kernel runs
    wide = synth.tiny((4, 2048, 1024), 10, seed=1)
    with pytest.raises(m.CtdError) as e:
        noalloc(m, m.Coo.from_synth(wide), 5, 0)
    assert e.value.status == "CTD_EINVAL"
    # host memory would need a staging buffer: rejected
    import torch
    Xh = m.Coo.from_synth(synth.small_uniform(), device=False)
    d = torch.empty(5, dtype=torch.int64, device="cuda")
    with pytest.raises(m.CtdError):
        m.sample_noalloc(Xh, 1, 5, 0, d, d)
