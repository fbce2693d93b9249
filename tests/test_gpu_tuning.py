"""The launch-shape knobs (ctd_set_tuning) change how the hot kernels are
laid out on the GPU, never what they compute; the autotuner over them
returns a setting from its grid."""
import numpy as np
import pytest

from paper_1710_03608_gb300 import synth

pytestmark = pytest.mark.gpu


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


@pytest.fixture
def defaults_after():
    yield
    m = ctd()
    for k in m.TUNING_KEYS:
        m.set_tuning(k, -1)


def test_knobs_do_not_change_results(defaults_after):
    """Q-form rows staged or not, more or fewer dense rows of R in the C
    fill, any copy grid: R, U and C bit for bit, the error to the last bit
    (CTD_DETERMINISTIC fixes each column's entry order)."""
    m = ctd()
    coo = synth.traffic((2000, 2000, 200), 400_000, 1.2, 1.2, "poisson1", 13, 3.0)
    X = m.Coo.from_synth(coo)

    def run():
        F = m.ctd_static(X, 1, 300, 1e-6, 5, m.CTD_FP32_BULK, m.CTD_DETERMINISTIC)
        out = (F.R_dense(), F.U(), F.C(), F.error())
        F.free()
        return out

    ref = run()
    for knobs in ({"qform_hot_kb": 0}, {"qform_hot_kb": 100, "cfill_dense_kb": 64},
                  {"cfill_dense_kb": 128, "copy_blocks_per_sm": 1},
                  {"copy_blocks_per_sm": 32, "qform_hot_kb": 150}):
        for k in m.TUNING_KEYS:
            m.set_tuning(k, -1)
        for k, v in knobs.items():
            m.set_tuning(k, v)
        assert {k: m.get_tuning(k) for k in knobs} == knobs
        R, U, C, e = run()
        assert np.array_equal(R, ref[0]), knobs
        assert np.array_equal(U, ref[1]), knobs
        assert all(np.array_equal(a, b) for a, b in zip(C, ref[2])), knobs
        assert e == ref[3], knobs


def test_autotuner_picks_from_its_grid(defaults_after):
    from paper_1710_03608_gb300 import measure
    m = ctd()
    coo = synth.traffic((1000, 1000, 100), 100_000, 1.2, 1.2, "poisson1", 14, 3.0)
    X = m.Coo.from_synth(coo)
    r = measure.autotune_kernels(X, 200, 1, calls=2, save=False)
    for k, v in r["best"].items():
        assert v in measure.KNOB_GRID[k]
        assert m.get_tuning(k) == v
    assert r["class"] == "nnz_1e5" and r["tuned_ms"] > 0 and r["default_ms"] > 0
