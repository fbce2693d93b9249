"""The launch-shape tuning file (CPU): size classes by decade of nonzeros,
per-class settings applied through ctd_set_tuning (no GPU work), defaults
for a class the file does not hold, and the batched worker count kept
beside them."""
import json

import pytest


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1710_03608_gb300 import _build
    _build.build()  # the knobs are host state: no GPU needed


@pytest.fixture
def tune_file(tmp_path, monkeypatch):
    from paper_1710_03608_gb300 import ctd, measure
    path = tmp_path / "autotune.json"
    monkeypatch.setattr(measure, "TUNE_FILE", str(path))
    yield path
    ctd.load()
    for k in ctd.TUNING_KEYS:
        ctd.set_tuning(k, -1)


def test_size_classes():
    from paper_1710_03608_gb300 import measure
    assert measure.size_class(0) == "nnz_1e0"
    assert measure.size_class(12_000) == "nnz_1e4"
    assert measure.size_class(40_000) == "nnz_1e5"
    assert measure.size_class(10_000_000) == "nnz_1e7"


def test_apply_and_defaults(tune_file):
    from paper_1710_03608_gb300 import ctd, measure
    ctd.load()
    measure._tune_save({"kernels": {"nnz_1e7": {"qform_hot_kb": 0, "cfill_dense_kb": 176,
                                                 "copy_blocks_per_sm": 2}}})
    measure._tune_save({"batched_workers": 12})   # merged, not overwritten
    d = json.loads(tune_file.read_text())
    assert d["batched_workers"] == 12 and "nnz_1e7" in d["kernels"]
    assert measure.tuned_workers() == 12
    got = measure.apply_tuning(9_000_000)
    assert got == {"qform_hot_kb": 0, "cfill_dense_kb": 176, "copy_blocks_per_sm": 2}
    assert ctd.get_tuning() == got
    # a class the file does not hold: the defaults
    assert measure.apply_tuning(5_000) == {"qform_hot_kb": 200, "cfill_dense_kb": 220,
                                           "copy_blocks_per_sm": 8}


def test_knob_ranges_rejected():
    from paper_1710_03608_gb300 import ctd
    ctd.load()
    for key, bad in (("qform_hot_kb", 201), ("cfill_dense_kb", 63), ("copy_blocks_per_sm", 33)):
        with pytest.raises(ctd.CtdError):
            ctd.set_tuning(key, bad)
    with pytest.raises(ctd.CtdError):
        ctd.set_tuning("no_such_knob", 1)
