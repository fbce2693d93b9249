"""Section 5's online DDoS detector on R: the CUDA path (through the C ABI)
against the oracle's rule on the oracle's own factors.  The candidates are
integers and the average norm is an exactly rounded sum divided by a count,
so both must agree bit for bit."""
import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth
from tests.parity import tie_margin

pytestmark = pytest.mark.gpu


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


def planted_stream(steps=9, dims2=(300, 200), nnz=1500, seed=77):
    """A small source x destination stream with a block of heavy counts from
    24 sources to 6 destinations added at steps 4-6."""
    rng = np.random.default_rng(seed)
    src = np.sort(rng.choice(dims2[0], 24, replace=False)).astype(np.int64)
    dst = np.sort(rng.choice(dims2[1], 6, replace=False)).astype(np.int64)
    return synth.SliceStream(dims2, steps, nnz, 1.1, 2.0, seed, [4, 5, 6], src, dst, 40.0)


@pytest.mark.parametrize("d,eps", [(10, 0.15), (40, 1e-6)])
def test_dynamic_detector_matches_oracle(d, eps):
    m = ctd()
    S = planted_stream()
    G = m.Dynamic(S.dims2, 1, m.CTD_FP32_BULK, 3)
    st = O.DynamicState(*S.dims2)
    for t in range(S.steps):
        sl = S.slice(t)
        G.step_slice(m.Coo.from_synth(sl), d, eps)
        step = O.ctd_d_step(st, S.dims2, sl.i, sl.j, sl.val, d, eps, 3)
        assert tie_margin(step.ratios, eps) > 1e-7, "near-tie in the independence test"
        got, mean = G.ddos_candidates()
        want, want_mean = O.ddos_candidates(st.fibers, st.R_cols, with_mean=True)
        assert [int(x) for x in got] == want, t
        assert mean == want_mean, (t, mean, want_mean)
    # the planted destinations are found once their block has arrived
    assert set(S.planted_dst.tolist()) & set(int(x) for x in got)


def test_static_detector_matches_oracle():
    """CTD-S factors (alpha = 1): the destination of fiber f = j + J*k is j."""
    m = ctd()
    coo = synth.traffic_10m(scale=0.1)
    F = m.ctd_static(m.Coo.from_synth(coo), 1, 400, 1e-6, 2, m.CTD_FP32_BULK)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 400, 1e-6, 2)
    J = coo.dims[1]
    fibers = [(int(f) // J, int(f) % J) for f in ref.fibers]
    cols = [ref.R[:, c] for c in range(ref.R.shape[1])]
    want, want_mean = O.ddos_candidates(fibers, cols, with_mean=True)
    got, mean = F.ddos_candidates()
    assert [int(x) for x in got] == want
    assert mean == want_mean
    assert len(want) > 0


def test_detector_edge_cases():
    m = ctd()
    # an all-zero stream: R stays empty, nothing flagged, average 0
    G = m.Dynamic((20, 10), 1, m.CTD_FP64, 0)
    z = synth.tiny((20, 10, 1), 30, seed=3)
    z.val[:] = 0
    G.step_slice(m.Coo.from_synth(z), 5, 1e-6)
    got, mean = G.ddos_candidates()
    assert got.size == 0 and mean == 0.0
    # a single kept fiber: its norm equals the average, so it is not flagged
    one = synth.tiny((20, 10, 1), 1, seed=4)
    G.step_slice(m.Coo.from_synth(one), 5, 1e-6)
    got, mean = G.ddos_candidates()
    assert got.size == 0 and mean == float(abs(int(one.val[0])))
    # alpha = 2 factors have no destination mode
    G2 = m.Dynamic((20, 10), 2, m.CTD_FP64, 0)
    G2.step_slice(m.Coo.from_synth(synth.tiny((20, 10, 1), 30, seed=5)), 5, 1e-6)
    with pytest.raises(m.CtdError) as e:
        G2.ddos_candidates()
    assert e.value.status == "CTD_EINVAL"
