"""CTD-S parity: CUDA path (through the C ABI) vs the FP64 oracle."""
import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth
from tests.parity import error_tol, rel_fro, tie_margin, u_residual, u_tol

pytestmark = pytest.mark.gpu


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


def run(coo, alpha, s, eps, seed, precision, host=False, flags=0):
    m = ctd()
    X = m.Coo.from_synth(coo, device=not host)
    return m.ctd_static(X, alpha, s, eps, seed, precision, flags)


def check(F, ref, eps, precision, full_c=True, c_cols=None, err_ref=None):
    sz = F.sizes()
    assert sz.sqnorm_X == float(ref.T)
    I, Iu = F.samples()
    assert np.array_equal(I, ref.I)
    assert np.array_equal(Iu, ref.I_unique)
    assert tie_margin(ref.ratios, eps) > 1e-7, "near-tie in the independence test"
    fib, _ = F.fibers()
    assert np.array_equal(fib, ref.fibers)
    assert np.array_equal(F.R_dense(), ref.R)
    if ref.R.shape[1]:
        U = F.U()
        assert rel_fro(U, ref.U) <= u_tol(ref.R)
        # the GPU's U is at least as good an inverse as the oracle's
        assert u_residual(U, ref.R) <= 2.0 * u_residual(ref.U, ref.R) + 1e-9
    if full_c:
        p, r, v = F.C()
        Cref = O.c_full(ref.X, ref.R)
        assert np.array_equal(p, Cref.indptr)
        assert np.array_equal(r, Cref.indices)
        assert np.array_equal(v, Cref.data.astype(np.float64))
        assert sz.nnz_C == Cref.nnz
    if c_cols is not None:
        got = F.C_columns(c_cols)
        want = O.c_columns(ref.X, ref.R, c_cols)
        assert np.array_equal(got, want.astype(np.float64))
    if err_ref is not None:
        e = F.error()
        assert abs(e - err_ref) <= error_tol(precision, err_ref), (e, err_ref)


@pytest.mark.parametrize("alpha", [1, 2, 3])
@pytest.mark.parametrize("precision", [0, 1])
def test_small_uniform_full(alpha, precision):
    coo = synth.small_uniform()
    s, eps, seed = 50, 1e-6, 0
    F = run(coo, alpha, s, eps, seed, precision)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, alpha, s, eps, seed)
    e_ref = O.relative_error_dense(ref.X, ref.R, ref.U, O.c_full(ref.X, ref.R))
    check(F, ref, eps, precision, err_ref=e_ref)


def check_dist(F, ref):
    """Rows 1-2 element by element: every squared column norm and every CDF
    entry equal to the oracle's exact integers."""
    n2, c = F.column_dist()
    assert np.array_equal(n2.astype(np.int64), ref.sqnorms)
    assert np.array_equal(c.astype(np.int64), ref.cdf)


@pytest.mark.parametrize("alpha", [1, 2, 3])
@pytest.mark.parametrize("host", [False, True])
def test_column_dist_small(alpha, host):
    m = ctd()
    coo = synth.small_uniform()
    F = run(coo, alpha, 50, 1e-6, 0, 0, host=host, flags=m.CTD_KEEP_DIST)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, alpha, 50, 1e-6, 0)
    check_dist(F, ref)


@pytest.mark.parametrize("nnz", [1, 3, 4097, 20_001])
def test_column_dist_ragged(nnz):
    """Signed values, nnz around the 4-entry vector width, column counts
    that are not multiples of the 4096-column scan tile."""
    m = ctd()
    coo = synth.tiny((37, 53, 29), nnz, seed=nnz, vmax=9, signed=True)
    for alpha in (1, 3):
        F = run(coo, alpha, 64, 1e-6, 1, 0, flags=m.CTD_KEEP_DIST)
        ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, alpha, 64, 1e-6, 1)
        check_dist(F, ref)
        assert np.array_equal(F.samples()[0], ref.I)


def bucket_case(kind):
    """A 40 x 5000 x 1000 tensor: 5*10^6 columns of X_(1), enough for the
    bucketed matricization (611 buckets of 8192 columns).  "balanced": 3*10^5
    uniform entries (about 500 per bucket).  "over_capacity": 15,000 more
    entries in the first bucket's columns, more than a place block stages
    (10,240), so that bucket writes straight to global memory.  "skewed":
    40,000 more, past twice that, so the plain passes run instead."""
    dims = (40, 5000, 1000)
    base = synth.tiny(dims, 300_000, seed=51, vmax=6, signed=True)
    if kind == "balanced":
        return base
    extra = 15_000 if kind == "over_capacity" else 40_000
    rng = np.random.default_rng(52)
    lin = rng.choice(40 * 8192, size=extra, replace=False)
    col = lin // 40
    i = np.concatenate([base.i, lin % 40])
    j = np.concatenate([base.j, col % 5000])
    k = np.concatenate([base.k, col // 5000])
    v = np.concatenate([base.val, rng.integers(1, 7, size=extra)])
    key = i + 40 * (j + 5000 * k)
    _, first = np.unique(key, return_index=True)
    first = np.sort(first)
    return synth.Coo3(dims, i[first], j[first], k[first], v[first])


@pytest.mark.parametrize("kind", ["balanced", "over_capacity", "skewed"])
def test_bucketed_matricize(kind):
    m = ctd()
    coo = bucket_case(kind)
    F = run(coo, 1, 200, 1e-6, 4, 0, flags=m.CTD_KEEP_DIST)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 200, 1e-6, 4)
    check_dist(F, ref)
    check(F, ref, 1e-6, 0, err_ref=O.projection_error(ref.X, ref.R))


def test_memory_usage_matches_oracle():
    """Eq. (memoryEff) from the library's factors equals the oracle's count."""
    from paper_1710_03608_gb300 import measure
    coo = synth.small_uniform()
    F = run(coo, 1, 50, 1e-6, 0, 0)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 50, 1e-6, 0)
    want = O.memory_usage(ref.X, ref.R, ref.U, O.c_full(ref.X, ref.R))
    assert measure.memory_usage(F) == want


def test_host_input_matches_device_input():
    coo = synth.small_uniform()
    Fd = run(coo, 1, 50, 1e-6, 3, 0)
    Fh = run(coo, 1, 50, 1e-6, 3, 0, host=True)
    assert np.array_equal(Fd.samples()[0], Fh.samples()[0])
    assert np.array_equal(Fd.R_dense(), Fh.R_dense())
    assert np.array_equal(Fd.U(), Fh.U())
    assert abs(Fd.error() - Fh.error()) <= 1e-12 * Fh.error()


@pytest.mark.parametrize("seed", [0, 1])
def test_signed_values(seed):
    coo = synth.tiny((40, 30, 20), 2000, seed=seed + 20, vmax=7, signed=True)
    F = run(coo, 1, 200, 1e-6, seed, 0)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 200, 1e-6, seed)
    e_ref = O.relative_error_dense(ref.X, ref.R, ref.U, O.c_full(ref.X, ref.R))
    check(F, ref, 1e-6, 0, err_ref=e_ref)


def test_sample_every_fiber_exact():
    coo = synth.tiny((30, 12, 6), 400, seed=4)
    F = run(coo, 1, 8192, 1e-6, 1, 0)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 8192, 1e-6, 1)
    check(F, ref, 1e-6, 0, err_ref=0.0)
    assert abs(F.error()) <= 1e-12


@pytest.mark.parametrize("precision", [0, 1])
def test_traffic_scaled_full(precision):
    """A 2,000 x 2,000 x 200 traffic tensor (8*10^4 nonzeros, Zipf(1.2),
    Geometric(0.3)) with s = 500: many tiles, ragged tails, full C."""
    coo = synth.traffic_10m(scale=0.2)
    F = run(coo, 1, 500, 1e-6, 0, precision)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 500, 1e-6, 0)
    check(F, ref, 1e-6, precision, err_ref=O.projection_error(ref.X, ref.R))


def test_deterministic_flag_parity():
    """The sorted-column path (CTD_DETERMINISTIC) against the oracle on the
    2,000 x 2,000 x 200 traffic tensor, FP32 bulk."""
    m = ctd()
    coo = synth.traffic_10m(scale=0.2)
    F = run(coo, 1, 500, 1e-6, 0, 1, flags=m.CTD_DETERMINISTIC)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 500, 1e-6, 0)
    check(F, ref, 1e-6, 1, err_ref=O.projection_error(ref.X, ref.R))


@pytest.mark.parametrize("case", ["int64_sums", "wide_registers", "wider_than_registers",
                                  "int16_rows", "int32_rows", "int8_rows_wide_x"])
def test_c_fill_paths(case):
    """Each C = R^T X path against the oracle: partial sums beyond int32
    (||X||_F^2 >= 2^31), s~ in (512, 1024] (the widest register layout),
    s~ > 1024 (shared-memory accumulators only), the dense rows of R
    stored as int16 (max |R| in (127, 32767]) or int32 (larger), and int8
    rows while X has a value outside int8 (so the four-products-per-
    instruction form is off); the int8 layout with X in int8 is the default
    of the small-count cases."""
    if case == "int8_rows_wide_x":
        # fiber 0 = 100 e_0 is kept first; fiber 1 = 200 e_0 is parallel to it and
        # skipped, so R stays within int8 while X holds 200
        base = synth.tiny((60, 40, 10), 3000, seed=37, vmax=5)
        keep = ~((base.k == 0) & (base.j <= 1))
        coo = synth.Coo3(base.dims, np.concatenate([base.i[keep], [0, 0]]),
                         np.concatenate([base.j[keep], [0, 1]]),
                         np.concatenate([base.k[keep], [0, 0]]),
                         np.concatenate([base.val[keep], [100, 200]]))
        s = 2000
    elif case == "int64_sums":
        coo, s = synth.tiny((60, 40, 10), 3000, seed=31, vmax=100_000), 300
    elif case == "int16_rows":
        coo, s = synth.tiny((60, 40, 10), 3000, seed=34, vmax=300), 300
    elif case == "int32_rows":
        coo, s = synth.tiny((40, 30, 4), 3000, seed=36, vmax=300), 2000
        coo.val[7] = 33_000  # ||X||^2 stays below 2^31; this fiber is kept
    elif case == "wide_registers":
        coo, s = synth.tiny((900, 600, 2), 15_000, seed=32, vmax=5), 2000
    else:
        coo, s = synth.tiny((1200, 800, 2), 20_000, seed=33, vmax=5), 4000
    F = run(coo, 1, s, 1e-6, 5, 0)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, s, 1e-6, 5)
    kept = ref.R.shape[1]
    if case == "int64_sums":
        assert F.sizes().sqnorm_X >= 2 ** 31
    elif case in ("int16_rows", "int32_rows"):
        assert F.sizes().sqnorm_X < 2 ** 31
        top = np.abs(ref.R).max()
        assert (127 < top <= 32767) if case == "int16_rows" else top > 32767
    elif case == "wide_registers":
        assert 512 < kept <= 1024
    elif case == "int8_rows_wide_x":
        assert np.abs(ref.R).max() <= 127 < np.abs(coo.val).max()
        assert 1 not in ref.fibers
    else:
        assert kept > 1024
    check(F, ref, 1e-6, 0, err_ref=O.projection_error(ref.X, ref.R))


def test_edge_all_zero():
    coo = synth.tiny((5, 4, 3), 10, seed=1)
    coo.val[:] = 0
    F = run(coo, 1, 10, 1e-6, 0, 0)
    sz = F.sizes()
    assert sz.s_unique == 0 and sz.s_kept == 0 and sz.nnz_C == 0
    assert F.error() == 0.0


def test_edge_single_nonzero_and_s1():
    coo = synth.tiny((5, 4, 3), 1, seed=2)
    F = run(coo, 1, 1, 0.5, 7, 0)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 1, 0.5, 7)
    check(F, ref, 0.5, 0, err_ref=0.0)


def test_errors_are_reported():
    m = ctd()
    coo = synth.small_uniform()
    with pytest.raises(m.CtdError) as e:
        run(coo, 4, 50, 1e-6, 0, 0)
    assert e.value.status == "CTD_EINVAL"
    with pytest.raises(m.CtdError):
        run(coo, 1, 0, 1e-6, 0, 0)
    bad = synth.Coo3(coo.dims, coo.i.copy(), coo.j.copy(), coo.k.copy(), coo.val.copy())
    bad.i[17] = 100  # outside I = 100: the kernels skip it and flag it
    with pytest.raises(m.CtdError) as e:
        run(bad, 1, 50, 1e-6, 0, 0)
    assert e.value.status == "CTD_EINVAL"


@pytest.fixture(scope="module")
def traffic_full():
    coo = synth.traffic_10m()
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 500, 1e-6, 0)
    return coo, ref


def test_traffic_10m_full_size(traffic_full):
    """The 10^4 x 10^4 x 10^3, 10^7-nonzero workload at full size, FP32 bulk:
    integer stages and U element by element, C on sampled columns, the
    error against Lemma 3.2's projection form."""
    coo, ref = traffic_full
    F = run(coo, 1, 500, 1e-6, 0, 1)
    rng = np.random.default_rng(0)
    nz = np.flatnonzero(np.diff(ref.X.ptr))
    cols = np.concatenate([rng.choice(nz, 200, replace=False),
                           nz[np.argsort(np.diff(ref.X.ptr)[nz])[-20:]], [0, ref.X.n_cols - 1]])
    check(F, ref, 1e-6, 1, full_c=False, c_cols=cols, err_ref=O.projection_error(ref.X, ref.R))


def test_traffic_10m_dist_and_full_c(traffic_full):
    """The 10^7-nonzero workload in the bench's launch configuration (FP32
    bulk): all 10^7 squared column norms and CDF entries bit-exact, and the
    whole of C = R^T X_(alpha) (6.6*10^8 entries) equal to the oracle's exact
    product, compared in blocks of 10^6 columns."""
    m = ctd()
    coo, ref = traffic_full
    F = run(coo, 1, 500, 1e-6, 0, 1, flags=m.CTD_KEEP_DIST)
    check_dist(F, ref)
    assert np.array_equal(F.R_dense(), ref.R)
    p, r, v = F.C()
    assert p[0] == 0 and p[-1] == F.sizes().nnz_C
    Xs = ref.X.scipy()
    import scipy.sparse as sp
    Rt = sp.csr_matrix(ref.R.T.astype(np.int64))
    step = 1_000_000
    for a in range(0, ref.X.n_cols, step):
        b = min(a + step, ref.X.n_cols)
        want = (Rt @ Xs[:, a:b]).tocsc()
        want.eliminate_zeros()
        want.sort_indices()
        lo, hi = int(p[a]), int(p[b])
        assert np.array_equal(p[a:b + 1] - lo, want.indptr), a
        assert np.array_equal(r[lo:hi], want.indices), a
        assert np.array_equal(v[lo:hi], want.data.astype(np.float32).astype(np.float64)), a


def test_repeat_calls_bit_identical(traffic_full):
    """With CTD_DETERMINISTIC, three calls on the 10^7-nonzero workload (FP32
    bulk, then FP64) give bit-identical U, C and error: each column's
    entries are put in one order after the matricization, so no
    floating-point sum depends on the order the scatter's atomics took."""
    m = ctd()
    coo, _ = traffic_full
    X = m.Coo.from_synth(coo)
    for precision in (1, 0):
        seen = []
        for _ in range(3):
            F = m.ctd_static(X, 1, 500, 1e-6, 0, precision, m.CTD_DETERMINISTIC)
            p, r, v = F.C()
            seen.append((F.error(), F.U().tobytes(), hash(p.tobytes()), hash(r.tobytes()),
                         hash(v.tobytes())))
            F.free()
        assert all(x == seen[0] for x in seen[1:])


def test_sqnorm_range():
    """||X||_F^2 must stay below 2^63 (the int64 CDF, reading A12): three
    values of 2^31 - 1 pass it and the call reports CTD_EOVERFLOW; two stay
    below it and the call succeeds with the exact total."""
    m = ctd()
    big = 2 ** 31 - 1
    i, j, k = np.array([0, 1, 2]), np.array([0, 1, 2]), np.array([0, 0, 1])
    coo = synth.Coo3((4, 3, 2), i, j, k, np.full(3, big, np.int64))
    with pytest.raises(m.CtdError) as e:
        run(coo, 1, 5, 1e-6, 0, 0)
    assert e.value.status == "CTD_EOVERFLOW"
    coo2 = synth.Coo3((4, 3, 2), i[:2], j[:2], k[:2], np.full(2, big, np.int64))
    F = run(coo2, 1, 64, 1e-6, 0, 0)
    assert F.sizes().sqnorm_X == float(2 * big * big)
    assert F.sizes().s_kept == 2


@pytest.mark.parametrize("n", [3, 5])
def test_fiber_sum_overflow(n):
    """n values of 2^31 - 1 in one fiber: the column's exact sum passes 2^63
    (n = 5 would also wrap a 64-bit accumulator to a value below 2^63), so
    the call reports CTD_EOVERFLOW (reading A12), as the oracle raises."""
    m = ctd()
    big = 2 ** 31 - 1
    i = np.arange(n)
    coo = synth.Coo3((8, 3, 2), i, np.ones(n, np.int64), np.zeros(n, np.int64),
                     np.full(n, big, np.int64))
    with pytest.raises(OverflowError):
        O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 5, 1e-6, 0)
    with pytest.raises(m.CtdError) as e:
        run(coo, 1, 5, 1e-6, 0, 0)
    assert e.value.status == "CTD_EOVERFLOW"


def test_bounded_wait_gives_up_and_context_survives():
    """The grid barrier's bounded wait, on a word nothing changes, gives up
    with CTD_ETIMEOUT (no trap, no hang); the next call works."""
    m = ctd()
    with pytest.raises(m.CtdError) as e:
        m.selftest_bounded_wait(1 << 12)
    assert e.value.status == "CTD_ETIMEOUT"
    coo = synth.small_uniform()
    F = run(coo, 1, 50, 1e-6, 0, 0)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 50, 1e-6, 0)
    assert F.sizes().s_kept == ref.R.shape[1]


def test_allocation_failure_is_reported():
    """With device allocations refused after n more, a call returns
    CTD_ENOMEM and releases what it held; with the hook off the same call
    gives the oracle's result."""
    m = ctd()
    coo = synth.small_uniform()
    X = m.Coo.from_synth(coo)
    try:
        for n in (0, 3, 10, 20):
            m.fault_inject_alloc(n)
            with pytest.raises(m.CtdError) as e:
                m.ctd_static(X, 1, 50, 1e-6, 0, m.CTD_FP64)
            assert e.value.status == "CTD_ENOMEM"
    finally:
        m.fault_inject_alloc(-1)
    F = m.ctd_static(X, 1, 50, 1e-6, 0, m.CTD_FP64)
    ref = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 50, 1e-6, 0)
    assert np.array_equal(F.R_dense(), ref.R)
