"""Batched CTD-S: each tensor's result equals its own ctd_static call, and
the oracle's, on a batch of uneven traffic tensors."""
import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth
from tests.parity import error_tol, rel_fro, u_tol

pytestmark = pytest.mark.gpu


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


def small_batch(count=12):
    """The 256-tensor workload's law (log-uniform I, J, K, nnz; Zipf(1.2);
    Poisson(3)+1; s = min(I, J) / 20) with nnz capped for the oracle."""
    return synth.batch_256(count=count, nnz_cap=20_000)


@pytest.mark.parametrize("workers", [1, 4])
def test_batched_equals_single_calls(workers):
    m = ctd()
    specs = small_batch()
    tensors = [sp.tensor() for sp in specs]
    Xs = [m.Coo.from_synth(x) for x in tensors]
    s = [sp.s for sp in specs]
    seeds = list(range(len(specs)))
    Fb = m.ctd_static_batched(Xs, 1, s, seeds, 1e-6, m.CTD_FP32_BULK, 0, workers)
    for t, (X, F) in enumerate(zip(Xs, Fb)):
        G = m.ctd_static(X, 1, s[t], 1e-6, seeds[t], m.CTD_FP32_BULK)
        assert np.array_equal(F.samples()[0], G.samples()[0])
        assert np.array_equal(F.R_dense(), G.R_dense())
        assert np.array_equal(F.U(), G.U())
        pf, rf, vf = F.C()
        pg, rg, vg = G.C()
        assert np.array_equal(pf, pg) and np.array_equal(rf, rg) and np.array_equal(vf, vg)
        # integer stages are bit-exact; the error sums in FP32 in the order the
        # counting sort left each column's entries, so it agrees to rounding
        assert abs(F.error() - G.error()) <= 1e-6 * max(G.error(), 1e-6)


def test_batched_matches_oracle():
    m = ctd()
    specs = small_batch(6)
    tensors = [sp.tensor() for sp in specs]
    Xs = [m.Coo.from_synth(x) for x in tensors]
    Fb = m.ctd_static_batched(Xs, 1, [sp.s for sp in specs], [7] * len(specs), 1e-6,
                              m.CTD_FP32_BULK)
    for x, sp, F in zip(tensors, specs, Fb):
        ref = O.ctd_s(x.dims, x.i, x.j, x.k, x.val, 1, sp.s, 1e-6, 7)
        assert np.array_equal(F.samples()[1], ref.I_unique)
        assert np.array_equal(F.R_dense(), ref.R)
        assert rel_fro(F.U(), ref.U) <= u_tol(ref.R)
        e_ref = O.projection_error(ref.X, ref.R)
        assert abs(F.error() - e_ref) <= error_tol(1, e_ref)
