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


def _R_from_coo(dims, raw, kept):
    """R's columns (rows ascending, counts) read straight from the COO
    entries: mode-1 column j + J*k of X."""
    i, j, k, v = (a.cpu().numpy().astype(np.int64) for a in raw)
    col = j + int(dims[1]) * k
    pos = {int(c): q for q, c in enumerate(kept)}
    sel = np.flatnonzero(np.isin(col, kept))
    cq = np.array([pos[int(c)] for c in col[sel]], np.int64)
    o = np.lexsort((i[sel], cq))
    cq, ii, vv = cq[o], i[sel][o], v[sel][o]
    b = np.searchsorted(cq, np.arange(len(kept) + 1))
    return [(ii[b[q]:b[q + 1]], vv[b[q]:b[q + 1]]) for q in range(len(kept))]


def _bad_columns(R, truth):
    p, r, v = R
    return [q for q, (ti, tv) in enumerate(truth)
            if not (np.array_equal(r[p[q]:p[q + 1]], ti) and np.array_equal(v[p[q]:p[q + 1]], tv))]


def test_batched_full_256_law():
    """All 256 tensors of the workload's law at full size (1.1*10^8 nonzeros,
    drawn on the device): one ctd_static_batched call gives every tensor the
    result of its own ctd_static call (draws, kept fibers, R and U bit for
    bit, C on sampled columns, the error to FP32 rounding), and the oracle's
    on 8 tensors spread over the size range."""
    import torch
    m = ctd()
    specs = synth.batch_256()
    raw = [synth.traffic_device(sp.dims, sp.nnz, 1.2, 1.2, "poisson1", 3.0, sp.seed)
           for sp in specs]
    Xs = [m.Coo(sp.dims, *t) for sp, t in zip(specs, raw)]
    s = [sp.s for sp in specs]
    seeds = list(range(len(specs)))
    Fb = m.ctd_static_batched(Xs, 1, s, seeds, 1e-6, m.CTD_FP32_BULK, 0, 8)
    rng = np.random.default_rng(5)
    for t, (X, F) in enumerate(zip(Xs, Fb)):
        G = m.ctd_static(X, 1, s[t], 1e-6, seeds[t], m.CTD_FP32_BULK)
        assert np.array_equal(F.samples()[0], G.samples()[0])
        assert np.array_equal(F.fibers()[0], G.fibers()[0])
        RF, RG = F.R(), G.R()
        if not all(np.array_equal(a, b) for a, b in zip(RF, RG)):
            kept = F.fibers()[0]
            truth = _R_from_coo(specs[t].dims, raw[t], kept)
            pytest.fail(f"tensor {t} ({specs[t].dims}, nnz {specs[t].nnz}, s {s[t]}): R differs; "
                        f"columns wrong in the batched result {_bad_columns(RF, truth)[:8]}, "
                        f"in the single call {_bad_columns(RG, truth)[:8]}")
        assert np.array_equal(F.U(), G.U())
        cols = rng.integers(0, F.sizes().n_cols, 40)
        assert np.array_equal(F.C_columns(cols), G.C_columns(cols))
        assert abs(F.error() - G.error()) <= 1e-6 * max(G.error(), 1e-6)
        G.free()
    # the oracle on tensors with s <= 150, spread over nnz
    small = sorted((sp.nnz, t) for t, sp in enumerate(specs) if sp.s <= 150)
    pick = [small[q][1] for q in np.linspace(0, len(small) - 1, 8).astype(int)]
    for t in pick:
        sp = specs[t]
        i, j, k, v = (a.cpu().numpy() for a in raw[t])
        ref = O.ctd_s(sp.dims, i, j, k, v, 1, sp.s, 1e-6, seeds[t])
        F = Fb[t]
        assert np.array_equal(F.samples()[0], ref.I)
        assert np.array_equal(F.R_dense(), ref.R)
        assert rel_fro(F.U(), ref.U) <= u_tol(ref.R)
        e_ref = O.projection_error(ref.X, ref.R)
        assert abs(F.error() - e_ref) <= error_tol(1, e_ref)
    del raw
    torch.cuda.empty_cache()
