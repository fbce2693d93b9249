"""Stored expected values (tests/golden/, written by make_golden.py from the
oracle): the oracle must still produce them (CPU), and the CUDA path must
match them (GPU)."""
import json
import os

import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_oracle_reproduces_static_fixture():
    g = load("static_small_uniform.json")
    coo = synth.small_uniform()
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 50, 1e-6, 0)
    assert int(ref.T) == g["T"]
    assert [int(v) for v in ref.I] == g["draws"]
    assert [int(v) for v in ref.I_unique] == g["unique"]
    assert [int(v) for v in ref.fibers] == g["fibers"]
    C = O.c_full(ref.X, ref.R)
    assert int(C.nnz) == g["nnz_C"]
    assert int((C.data.astype("int64") * (C.indices.astype("int64") + 1)).sum()) == g["C_checksum"]
    assert abs(O.projection_error(ref.X, ref.R) - g["error_lemma32"]) <= 1e-13


def test_oracle_reproduces_dynamic_fixture():
    g = load("dynamic_three_steps.json")
    state = O.DynamicState(60, 40)
    for t, want in enumerate(g["steps"]):
        sl = synth.tiny((60, 40, 1), 1200, seed=50 + t, vmax=5)
        res = O.ctd_d_step(state, (60, 40), sl.i, sl.j, sl.val, 30, 1e-6, 4)
        assert [int(v) for v in res.I] == want["draws"]
        assert [int(v) for v in res.new_fibers] == want["new_fibers"]
        assert len(state.R_cols) == want["kept_total"]
        assert abs(state.err_num / state.err_den - want["error"]) <= 1e-13
        # the per-step increments equal the literal dense error (pin P9)
        assert abs(want["error"] - want["error_dense"]) <= 1e-12


@pytest.mark.gpu
def test_cuda_matches_static_fixture():
    from paper_1710_03608_gb300 import ctd
    g = load("static_small_uniform.json")
    coo = synth.small_uniform()
    F = ctd.ctd_static(ctd.Coo.from_synth(coo), 1, 50, 1e-6, 0, ctd.CTD_FP64)
    sz = F.sizes()
    assert sz.sqnorm_X == g["T"]
    I, Iu = F.samples()
    assert I.tolist() == g["draws"] and Iu.tolist() == g["unique"]
    assert F.fibers()[0].tolist() == g["fibers"]
    assert sz.nnz_C == g["nnz_C"]
    p, r, v = F.C()
    assert int((v.astype(np.int64) * (r.astype(np.int64) + 1)).sum()) == g["C_checksum"]
    assert abs(F.error() - g["error_lemma32"]) <= 1e-10 * g["error_lemma32"]


@pytest.mark.gpu
def test_cuda_matches_dynamic_fixture():
    from paper_1710_03608_gb300 import ctd
    g = load("dynamic_three_steps.json")
    G = ctd.Dynamic((60, 40), 1, ctd.CTD_FP64, 4, 0)
    for t, want in enumerate(g["steps"]):
        sl = synth.tiny((60, 40, 1), 1200, seed=50 + t, vmax=5)
        G.step_slice(ctd.Coo.from_synth(sl), 30, 1e-6)
        assert G.samples()[0].tolist() == want["draws"]
        assert G.sizes().s_kept == want["kept_total"]
        assert abs(G.error() - want["error"]) <= 1e-10 * want["error"]
