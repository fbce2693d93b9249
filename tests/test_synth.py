"""The seeded synthetic workloads follow their stated recipe (CPU): shapes,
distinct in-range coordinates, value laws, Zipf-skewed ids, the planted
block, the 256-tensor law and the Poisson arrival process."""
import numpy as np
import pytest

from paper_1710_03608_gb300 import synth


def _distinct_in_range(x):
    I, J, K = x.dims
    assert x.i.dtype == np.int32 and x.val.dtype == np.int32
    assert (x.i >= 0).all() and (x.i < I).all()
    assert (x.j >= 0).all() and (x.j < J).all()
    assert (x.k >= 0).all() and (x.k < K).all()
    lin = x.i.astype(np.int64) + I * (x.j.astype(np.int64) + J * x.k.astype(np.int64))
    assert np.unique(lin).shape[0] == x.nnz


def _zipf_slope(ids, top=30):
    """Least-squares slope of log frequency against log rank over the most
    frequent ids."""
    f = np.sort(np.bincount(ids))[::-1][:top].astype(float)
    r = np.arange(1, f.shape[0] + 1, dtype=float)
    return np.polyfit(np.log(r), np.log(f), 1)[0]


def test_small_uniform():
    x = synth.small_uniform()
    assert x.dims == (100, 100, 50) and x.nnz == 5000
    _distinct_in_range(x)
    assert x.val.min() >= 1
    assert x.val.mean() == pytest.approx(4.0, abs=0.15)        # Poisson(3) + 1


def test_traffic_tensor_recipe():
    x = synth.traffic_10m(scale=0.2)
    assert x.dims == (2000, 2000, 200) and x.nnz == 80_000
    _distinct_in_range(x)
    assert x.val.min() >= 1
    assert x.val.mean() == pytest.approx(1 / 0.3, rel=0.05)   # Geometric(0.3) on {1, 2, ...}
    assert _zipf_slope(x.i) == pytest.approx(-1.2, abs=0.25)  # Zipf(1.2) sources
    assert _zipf_slope(x.j) == pytest.approx(-1.2, abs=0.25)  # and destinations
    # time is uniform: every step's share within 25% of 1/K
    share = np.bincount(x.k, minlength=200) / x.nnz
    assert np.abs(share * 200 - 1).max() < 0.25
    # the same seed gives the same tensor
    y = synth.traffic_10m(scale=0.2)
    assert all(np.array_equal(a, b) for a, b in ((x.i, y.i), (x.j, y.j), (x.k, y.k),
                                                 (x.val, y.val)))


def test_slice_stream_and_planted_block():
    S = synth.traffic_stream_20k(scale=0.05, steps=42)
    I, J = S.dims2
    assert (I, J) == (1000, 1000)
    plain, planted = S.slice(39), S.slice(40)
    for sl in (plain, planted):
        assert sl.dims == (I, J, 1)
        _distinct_in_range(sl)
        assert sl.val.min() >= 1
    assert plain.nnz == 1250
    assert plain.val.mean() == pytest.approx(3.0, abs=0.3)    # Poisson(2) + 1
    # at a planted step every source x destination cell of the block is
    # present, with the Poisson(40) counts added to any background count
    cells = {(a, b): v for a, b, v in zip(planted.i.tolist(), planted.j.tolist(),
                                         planted.val.tolist())}
    block = [(a, b) for a in S.planted_src.tolist() for b in S.planted_dst.tolist()]
    assert len(block) == S.planted_src.shape[0] * S.planted_dst.shape[0] == 10 * 2
    vals = np.array([cells.get(c, 0) for c in block])
    assert (vals > 0).all() and vals.mean() == pytest.approx(40, abs=6)


def test_batch_law():
    B = synth.batch_256()
    assert len(B) == 256
    for b in B:
        I, J, K = b.dims
        assert 500 <= I <= 20000 and 500 <= J <= 20000 and 10 <= K <= 500
        assert 1 <= b.nnz <= 2_000_000 and b.nnz <= I * J * K // 4
        assert b.s == max(1, min(I, J) // 20)
    nnz = np.array([b.nnz for b in B], dtype=float)
    assert 1e4 <= np.exp(np.log(nnz).mean()) <= 2e6


def test_poisson_arrivals():
    R = synth.serving_requests(duration_s=2.0)
    t = np.array([r.arrival_s for r in R])
    assert (np.diff(t) > 0).all() and t[-1] < 2.0
    assert len(R) == pytest.approx(4000, rel=0.05)             # 2 kHz for 2 s
    gaps = np.diff(t)
    assert gaps.std() / gaps.mean() == pytest.approx(1.0, abs=0.1)   # exponential gaps
    streams = np.array([r.stream for r in R])
    assert set(streams.tolist()) == set(range(64))
    for s in range(64):                                        # steps numbered in order
        steps = [r.step for r in R if r.stream == s]
        assert steps == list(range(len(steps)))
    assert all(1e4 <= r.nnz <= 1e6 for r in R)


@pytest.mark.parametrize("values, vparam, mean", [("geometric", 0.3, 1 / 0.3), ("poisson1", 3.0, 4.0)])
def test_device_generator_follows_the_traffic_law(values, vparam, mean):
    """The on-device generator (here on the CPU device) draws the same law as
    `traffic`: distinct in-range coordinates, the value law, Zipf(1.2) ids,
    uniform time, and the same tensor for the same seed."""
    import torch
    dims = (2000, 2000, 200)
    out = synth.traffic_device(dims, 80_000, 1.2, 1.2, values, vparam, 11, device="cpu")
    i, j, k, v = (t.numpy() for t in out)
    x = synth.Coo3(dims, i, j, k, v)
    assert all(t.dtype == torch.int32 for t in out) and x.nnz == 80_000
    _distinct_in_range(x)
    assert x.val.min() >= 1
    assert x.val.mean() == pytest.approx(mean, rel=0.05)
    assert _zipf_slope(x.i) == pytest.approx(-1.2, abs=0.25)
    assert _zipf_slope(x.j) == pytest.approx(-1.2, abs=0.25)
    share = np.bincount(x.k, minlength=200) / x.nnz
    assert np.abs(share * 200 - 1).max() < 0.25
    again = synth.traffic_device(dims, 80_000, 1.2, 1.2, values, vparam, 11, device="cpu")
    assert all(torch.equal(a, b) for a, b in zip(out, again))


def test_device_generator_saturating_law():
    """A Zipf law that needs many draws per distinct coordinate (one of the
    256-tensor specs with 1.7*10^6 nonzeros) still yields nnz distinct
    coordinates."""
    sp = synth.batch_256()[3]
    out = synth.traffic_device(sp.dims, sp.nnz, 1.2, 1.2, "poisson1", 3.0, sp.seed, device="cpu")
    x = synth.Coo3(sp.dims, *(t.numpy() for t in out))
    assert x.nnz == sp.nnz
    _distinct_in_range(x)


def test_nway_uniform():
    dims = (9, 8, 7, 6)
    idx, val = synth.nway_uniform(dims, 500, seed=3, vmax=7, signed=True)
    assert len(idx) == 4 and all(a.dtype == np.int32 for a in idx) and val.dtype == np.int32
    for a, d in zip(idx, dims):
        assert (a >= 0).all() and (a < d).all()
    lin = sum(a.astype(np.int64) * int(np.prod(dims[:n])) for n, a in enumerate(idx))
    assert np.unique(lin).shape[0] == 500
    assert 1 <= np.abs(val).min() and np.abs(val).max() <= 7 and (val < 0).any()
