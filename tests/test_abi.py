"""The C ABI library loads and exports every symbol include/ctd.h declares (CPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "ctd.h")).read()
    return sorted(set(re.findall(r"^CTD_API\s+[a-z_ ]+\*?\s*(ctd_[A-Za-z_0-9]+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_03608_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared()
    for n in ("ctd_static", "ctd_dynamic_step", "ctd_error"):
        assert n in names


def test_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (ctd_[A-Za-z_0-9]+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_binding_names_match_header(lib):
    from paper_1710_03608_gb300 import ctd
    assert sorted(ctd.EXPORTED) == declared()
    L = ctd.load()
    assert ctd.version().startswith("ctd-gb300")
    for n in declared():
        assert hasattr(L, n)


def test_no_compute_without_gpu_raises_cleanly(lib):
    """Without a GPU a call fails with a status, not a crash or a CPU fallback."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_1710_03608_gb300 import ctd, synth
    x = synth.tiny()
    X = ctd.Coo.from_synth(x, device=False)
    with pytest.raises(ctd.CtdError):
        ctd.ctd_static(X, 1, 5, 1e-6, 0, 0, stream=0)
