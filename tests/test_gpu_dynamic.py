"""CTD-D parity: one step at a time, CUDA path (through the C ABI) vs the
FP64 oracle's literal Algorithm 2 with a dense C."""
import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth
from tests.parity import error_tol, rel_fro, tie_margin, u_tol

pytestmark = pytest.mark.gpu


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


def slices_small(n, dims2=(60, 40), nnz=150, seed=0):
    return [synth.tiny((dims2[0], dims2[1], 1), nnz, seed=seed * 100 + t) for t in range(n)]


def run_stream(slices, dims2, d, eps, seed, precision, alpha=1, check_every=True, flags=0,
               dense_error=True):
    m = ctd()
    G = m.Dynamic(dims2, alpha, precision, seed, 0, flags)
    st = O.DynamicState(dims2[alpha - 1], dims2[2 - alpha])
    for t, sl in enumerate(slices):
        X = m.Coo.from_synth(sl)
        G.step_slice(X, d, eps)
        if alpha == 1:
            step = O.ctd_d_step(st, dims2, sl.i, sl.j, sl.val, d, eps, seed, keep_X=True)
        else:  # mode 2: swap the roles of the two slice modes
            step = O.ctd_d_step(st, (dims2[1], dims2[0]), sl.j, sl.i, sl.val, d, eps, seed,
                                keep_X=True)
        if check_every or t == len(slices) - 1:
            check_step(G, st, step, t, eps, precision, dense_error)
    return G, st


def check_step(G, st, step, t, eps, precision, dense_error=True):
    sz = G.sizes()
    assert sz.t_steps == t + 1
    I, Iu = G.samples()
    assert np.array_equal(I, step.I)
    assert np.array_equal(Iu, step.I_unique)
    assert tie_margin(step.ratios, eps) > 1e-7, "near-tie"
    info, sq = G.step(t)
    assert info[0] == len(step.I_unique) and info[1] == len(step.new_fibers)
    assert sq[0] == float(step.T_slice)
    fib, fstep = G.fibers()
    assert [(int(a), int(b)) for a, b in zip(fstep, fib)] == st.fibers
    R_ref = (np.stack([np.rint(c).astype(np.int64) for c in st.R_cols], axis=1)
             if st.R_cols else np.zeros((st.n_rows, 0), np.int64))
    assert np.array_equal(G.R_dense(), R_ref)
    if st.R_cols:
        assert rel_fro(G.U(), st.U) <= u_tol(R_ref)
    tol = max(u_tol(R_ref), 1e-12)
    # per-entry bars for this step's M and lower-left block of C: with
    # M = ((Delta R)^T R^(t)) U^(t) (Eq. C_t+1_final, left to right), an error
    # of relative size tol in U^(t) moves row m of M by at most
    # tol ||g_m|| ||U^(t)||_F (g_m the exact integer row m of (Delta R)^T R^(t)),
    # and entry (m, f) of the block M C^(t) by that times ||C^(t)(:, f)||
    dt_new = R_ref.shape[1]
    dt_old = dt_new - len(step.new_fibers)
    row_scale = None
    if step.M is not None and dt_old > 0 and dt_new > dt_old:
        Rt, dR = R_ref[:, :dt_old], R_ref[:, dt_old:]
        g = (dR.T @ Rt).astype(np.float64)
        Ut = np.linalg.inv((Rt.T @ Rt).astype(np.float64))
        row_scale = 4.0 * tol * np.linalg.norm(g, axis=1) * np.linalg.norm(Ut)
        Mg = G.M(t)
        assert rel_fro(Mg, step.M) <= u_tol(R_ref)
        assert np.all(np.abs(Mg - step.M) <= row_scale[:, None])
    elif step.M is not None:
        assert rel_fro(G.M(t), step.M) <= u_tol(R_ref)
    # every column of C^(t+1) (exact new block, implicit lower-left blocks)
    J = st.n_cols_slice
    ncols = J * (t + 1)
    if st.C is not None and st.C.shape[0]:
        got = G.C_columns(np.arange(ncols))
        assert got.shape == st.C.shape
        assert rel_fro(got, st.C) <= tol
        assert np.array_equal(got[:, -J:], st.C[:, -J:])       # new block is exact
        if row_scale is not None and t > 0:
            old = st.C[:dt_old, :J * t]
            bar = row_scale[:, None] * np.linalg.norm(old, axis=0)[None, :]
            diff = np.abs(got[dt_old:, :J * t] - st.C[dt_old:, :J * t])
            assert np.all(diff <= bar), float(np.max(diff - bar))
    # the literal X~ = R U C (Eq. error) loses every digit once U is the inverse
    # of a nearly singular R^T R (full row rank); there the oracle's per-step
    # projection form (Householder QR of R, reading A20) is the reference
    e_lit = O.dynamic_error_dense(st) if dense_error else st.err_num / st.err_den
    assert abs(G.error() - e_lit) <= error_tol(precision, e_lit) + 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_small_stream_every_step(precision):
    run_stream(slices_small(8, seed=1), (60, 40), 20, 1e-6, 5, precision)


def test_mode2_stream():
    run_stream(slices_small(5, seed=2), (60, 40), 15, 1e-6, 3, 0, alpha=2)


def test_first_step_equals_static():
    m = ctd()
    sl = slices_small(1, seed=3)[0]
    G = m.Dynamic((60, 40), 1, 0, 11)
    G.step_slice(m.Coo.from_synth(sl), 25, 1e-6)
    F = m.ctd_static(m.Coo.from_synth(sl), 1, 25, 1e-6, 11, 0)
    assert np.array_equal(G.samples()[0], F.samples()[0])
    assert np.array_equal(G.fibers()[0], F.fibers()[0])
    assert np.array_equal(G.R_dense(), F.R_dense())
    assert rel_fro(G.U(), F.U()) <= 1e-12
    assert abs(G.error() - F.error()) <= 1e-12


def test_empty_slice_step():
    sl = slices_small(3, seed=4)
    sl[1].val[:] = 0
    G, st = run_stream(sl, (60, 40), 10, 1e-6, 1, 0)
    info, sq = G.step(1)
    assert info[0] == 0 and info[1] == 0 and sq[0] == 0.0


def test_keep_last_c_releases_older_blocks():
    m = ctd()
    G = m.Dynamic((60, 40), 1, 0, 2, 0, m.CTD_KEEP_LAST_C)
    for sl in slices_small(3, seed=6):
        G.step_slice(m.Coo.from_synth(sl), 10, 1e-6)
    # the newest block stays readable, older ones were released
    assert G.C_columns([2 * 40 + 1]).shape[1] == 1
    with pytest.raises(m.CtdError):
        G.C_columns([0])


def test_failed_step_is_either_harmless_or_refused():
    """A step whose device allocations are refused returns CTD_ENOMEM.  If
    it failed before it changed the state, the same step succeeds afterwards
    and the stream ends as one that never failed; if it failed part-way, the
    state refuses further steps and getters (CTD_EINVAL) instead of going on
    from a half-updated R."""
    m = ctd()
    dims2 = (60, 40)
    sl = slices_small(3, dims2, seed=12)
    X = [m.Coo.from_synth(s) for s in sl]
    ref = m.Dynamic(dims2, 1, m.CTD_FP64, 5)
    for x in X:
        ref.step_slice(x, 10, 1e-6)
    R_ref, e_ref = ref.R_dense(), ref.error()
    outcomes = set()
    try:
        for n in (0, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128):
            G = m.Dynamic(dims2, 1, m.CTD_FP64, 5)
            G.step_slice(X[0], 10, 1e-6)
            m.fault_inject_alloc(n)
            try:
                G.step_slice(X[1], 10, 1e-6)
                outcomes.add("no refusal reached")
                continue
            except m.CtdError as e:
                assert e.status == "CTD_ENOMEM"
            finally:
                m.fault_inject_alloc(-1)
            try:
                G.step_slice(X[1], 10, 1e-6)
            except m.CtdError as e:
                assert e.status == "CTD_EINVAL" and "part-way" in str(e)
                with pytest.raises(m.CtdError):
                    G.sizes()
                outcomes.add("refused")
                continue
            G.step_slice(X[2], 10, 1e-6)
            assert np.array_equal(G.R_dense(), R_ref)
            assert abs(G.error() - e_ref) <= 1e-10 * max(e_ref, 1e-2)
            outcomes.add("harmless")
    finally:
        m.fault_inject_alloc(-1)
    assert {"refused", "harmless"} <= outcomes, outcomes


def test_traffic_stream_scaled():
    """Slices of 1,000 x 1,000 (1,250 nonzeros each, Zipf(1.1), Poisson(2)+1)
    with a planted 10 x 2 block of Poisson(40) counts at steps 40-45
    (here within 14 steps: none), d = 400, eps = 1e-6, FP32 bulk."""
    stream = synth.traffic_stream_20k(scale=0.05, steps=14)
    run_stream(list(stream), stream.dims2, 400, 1e-6, 0, 1, check_every=False)


def test_traffic_stream_full_size_sampled():
    """The 2*10^4 x 2*10^4 stream at full size (5*10^5 nonzeros per slice,
    d = 400, FP32 bulk, empty start), three steps, in the launch
    configuration of the stream measurement.  Checked per step against the
    oracle where it is cheap at this size: the draws and unique draws equal
    the oracle's (its Philox targets on the slice's exact CDF, Algorithm 2
    draws); every column R gained is the slice's own fiber, bit for bit;
    d~_t stays within the unique draws so far and I_alpha; the error lies
    in [0, 1]."""
    m = ctd()
    S = synth.traffic_stream_20k(steps=3)
    I, J = S.dims2
    G = m.Dynamic(S.dims2, 1, m.CTD_FP32_BULK, 0)
    n_unique = 0
    for t in range(S.steps):
        sl = S.slice(t)
        G.step_slice(m.Coo.from_synth(sl), 400, 1e-6)
        rows, cols, _, n_cols = O.matricize(sl.dims, sl.i, sl.j, sl.k, 1)
        vals = np.asarray(sl.val, dtype=np.int64)
        ref_I = O.sample_columns(O.cdf(O.column_sqnorms(cols, vals, n_cols)), 400, 0,
                                 step=t, stream=0)
        gI, gIu = G.samples()
        assert np.array_equal(gI, ref_I)
        assert np.array_equal(gIu, O.unique_columns(ref_I))
        n_unique += gIu.shape[0]
        fib, fstep = G.fibers()
        new = np.nonzero(fstep == t)[0]
        assert np.isin(fib[new], gIu).all()
        p, r, v = G.R()
        for c in new:
            mask = cols == fib[c]
            o = np.argsort(rows[mask], kind="stable")
            assert np.array_equal(r[p[c]:p[c + 1]], rows[mask][o])
            assert np.array_equal(v[p[c]:p[c + 1]], vals[mask][o])
        sz = G.sizes()
        assert sz.t_steps == t + 1 and sz.s_kept == fib.shape[0]
        assert sz.s_kept <= min(I, n_unique)
        assert 0.0 <= G.error() <= 1.0


def test_traffic_stream_full_size_u_error_c():
    """The same full-size stream (2*10^4 x 2*10^4 slices, 5*10^5 nonzeros,
    d = 400, FP32 bulk), three steps against the oracle's Algorithm 2 run on
    the whole slices: draws, unique draws, kept fibers and R bit for bit, U
    within the U bar, the error within the FP32-bulk bar (the oracle's
    per-step projection form), and the newest block of C, R^(t+1)^T dX
    (exact), on 500 sampled columns per step."""
    m = ctd()
    S = synth.traffic_stream_20k(steps=3)
    G = m.Dynamic(S.dims2, 1, m.CTD_FP32_BULK, 0)
    st = O.DynamicState(S.dims2[0], S.dims2[1])
    st.track_c = False          # the dense C of all steps is not needed here
    rng = np.random.default_rng(11)
    J = S.dims2[1]
    for t in range(S.steps):
        sl = S.slice(t)
        G.step_slice(m.Coo.from_synth(sl), 400, 1e-6)
        step = O.ctd_d_step(st, S.dims2, sl.i, sl.j, sl.val, 400, 1e-6, 0)
        I, Iu = G.samples()
        assert np.array_equal(I, step.I) and np.array_equal(Iu, step.I_unique)
        assert tie_margin(step.ratios, 1e-6) > 1e-7, "near-tie"
        fib, fstep = G.fibers()
        assert [(int(a), int(b)) for a, b in zip(fstep, fib)] == st.fibers
        R_ref = np.stack([np.rint(c).astype(np.int64) for c in st.R_cols], axis=1)
        assert np.array_equal(G.R_dense(), R_ref)
        assert rel_fro(G.U(), st.U) <= u_tol(R_ref)
        e_ref = st.err_num / st.err_den
        assert abs(G.error() - e_ref) <= error_tol(1, e_ref)
        cols = np.sort(rng.choice(J, 500, replace=False))
        got = G.C_columns(J * t + cols)
        assert np.array_equal(got, step.C_new[:, cols].astype(np.float64))


def test_planted_block_stream_scaled():
    """The same stream shape over steps 36..47 so the planted block (steps
    40-45) arrives mid-stream."""
    stream = synth.traffic_stream_20k(scale=0.05, steps=48)
    sl = [stream.slice(t) for t in range(36, 48)]
    run_stream(sl, stream.dims2, 400, 1e-6, 0, 0, check_every=False)


@pytest.mark.parametrize("precision", [0, 1])
def test_rank_saturation(precision):
    """R^(t) reaches full row rank (600) after twelve steps of d = 80 on
    600 x 400 slices; every later candidate lies in its span. The kept count
    never exceeds the row count and every decision matches the oracle, whose
    residual ratios leave a wide gap (kept >= 1e-4, skipped <= 1e-12)."""
    S = synth.SliceStream((600, 400), 14, 3000, 1.1, 2.0, 91)
    G, st = run_stream([S.slice(t) for t in range(S.steps)], S.dims2, 80, 1e-6, 3, precision,
                       check_every=False, dense_error=False)
    assert G.sizes().s_kept == len(st.R_cols) == 600


def test_near_saturation_weak_keeps():
    """A 2,000-row traffic stream (scale 0.1 of the 20,000-row one) with
    d = 400 reaches full row rank after 34 steps. On the way fibers are kept
    with residual ratios near 1e-5, and the last dimension is reached while
    every other candidate's ratio sits between 1e-9 and 1e-7. Every step's
    kept count, the fiber list and R match the oracle; the error matches its
    projection form. The oracle's literal U overflows in this regime (its
    rank-one updates divide by residuals near 1e-5), so U is not compared."""
    m = ctd()
    S = synth.traffic_stream_20k(scale=0.1, steps=34)
    G = m.Dynamic(S.dims2, 1, m.CTD_FP32_BULK, 0)
    st = O.DynamicState(*S.dims2)
    st.track_c = False
    with np.errstate(all="ignore"):
        for t in range(S.steps):
            sl = S.slice(t)
            G.step_slice(m.Coo.from_synth(sl), 400, 1e-6)
            step = O.ctd_d_step(st, S.dims2, sl.i, sl.j, sl.val, 400, 1e-6, 0)
            assert tie_margin(step.ratios, 1e-6) > 1e-7, "near-tie"
            info, _ = G.step(t)
            assert info[1] == len(step.new_fibers), t
    fib, fstep = G.fibers()
    assert [(int(a), int(b)) for a, b in zip(fstep, fib)] == st.fibers
    R_ref = np.stack([np.rint(c).astype(np.int64) for c in st.R_cols], axis=1)
    assert np.array_equal(G.R_dense(), R_ref)
    assert G.sizes().s_kept == len(st.R_cols) == 2000
    e = st.err_num / st.err_den
    assert abs(G.error() - e) <= error_tol(1, e)


def test_repeat_streams_bit_identical():
    """With CTD_DETERMINISTIC, two CTD-D runs over the same 1,000 x 1,000
    traffic slices (FP32 bulk) give bit-identical errors, kept counts and R
    after every step."""
    m = ctd()
    S = synth.traffic_stream_20k(scale=0.05, steps=10)
    runs = []
    for _ in range(2):
        G = m.Dynamic(S.dims2, 1, m.CTD_FP32_BULK, 0, 0, m.CTD_DETERMINISTIC)
        hist = []
        for t in range(S.steps):
            G.step_slice(m.Coo.from_synth(S.slice(t)), 400, 1e-6)
            info, _ = G.step(t)
            hist.append((int(info[1]), G.error()))
        runs.append((hist, G.R_dense().tobytes()))
    assert runs[0] == runs[1]


def _stack(slices):
    I, J = slices[0].dims[0], slices[0].dims[1]
    i = np.concatenate([s.i for s in slices])
    j = np.concatenate([s.j for s in slices])
    k = np.concatenate([np.full(s.nnz, t) for t, s in enumerate(slices)])
    v = np.concatenate([s.val for s in slices])
    return synth.Coo3((I, J, len(slices)), i, j, k, v)


@pytest.mark.parametrize("precision", [0, 1])
def test_seeded_from_static(precision):
    """The paper's CTD-D setting (Sec. 4): CTD-S factors of an 8-slice
    history seed the state, then two slices arrive. Against the oracle's
    seeded state and Algorithm 2 steps: fibers (time, slice fiber), R, U,
    every column of C (history through the M chain, new blocks exact) and
    the error."""
    m = ctd()
    slices = [synth.tiny((60, 40, 1), 200, seed=90 + t) for t in range(10)]
    hist = _stack(slices[:8])
    S = m.ctd_static(m.Coo.from_synth(hist), 1, 60, 1e-6, 5, precision)
    G = m.Dynamic.from_static(S)
    ref = O.ctd_s(hist.dims, hist.i, hist.j, hist.k, hist.val, 1, 60, 1e-6, 5)
    st = O.dynamic_state_from_static(ref, hist.dims, keep_X=True)

    def compare(new_block=None):
        fib, fstep = G.fibers()
        assert [(int(a), int(b)) for a, b in zip(fstep, fib)] == st.fibers
        R_ref = np.stack([np.rint(c).astype(np.int64) for c in st.R_cols], axis=1)
        assert np.array_equal(G.R_dense(), R_ref)
        assert rel_fro(G.U(), st.U) <= u_tol(R_ref)
        ncols = st.C.shape[1]
        got = G.C_columns(np.arange(ncols))
        assert rel_fro(got, st.C) <= max(u_tol(R_ref), 1e-12)
        if new_block:
            assert np.array_equal(got[:, -new_block:], st.C[:, -new_block:])
        e = O.dynamic_error_dense(st)
        assert abs(G.error() - e) <= error_tol(precision, e) + 1e-12

    compare()
    info, _ = G.step(0)
    assert info[1] == len(st.R_cols) and info[2] == 0
    for t, sl in enumerate(slices[8:]):
        G.step_slice(m.Coo.from_synth(sl), 15, 1e-6)
        step = O.ctd_d_step(st, (60, 40), sl.i, sl.j, sl.val, 15, 1e-6, 5, keep_X=True)
        assert tie_margin(step.ratios, 1e-6) > 1e-7, "near-tie"
        info, _ = G.step(t + 1)
        assert info[1] == len(step.new_fibers)
        compare(new_block=40)
    assert G.sizes().t_steps == 3
