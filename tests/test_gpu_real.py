"""CTD-S on real-valued tensors (FP32 values): ctd_static_nway through the C
ABI against the oracle.  The draws follow reading A28 (squares on a
fixed-point grid) and match bit for bit; R holds the sampled FP32 values
exactly; U, C and the error come from FP64 arithmetic whose additions run in
another order than the oracle's, so they are compared within bars derived
from the arithmetic."""
import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth
from tests.parity import error_tol, error_tol_real, rel_fro, tie_margin, u_residual, u_tol

pytestmark = pytest.mark.gpu


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


def check_real(F, ref, eps, precision, cols=None):
    sz = F.sizes()
    T_ref = ref.X.sqnorm()
    assert abs(sz.sqnorm_X - T_ref) <= 1e-13 * T_ref
    I, Iu = F.samples()
    assert np.array_equal(I, ref.I) and np.array_equal(Iu, ref.I_unique)
    assert tie_margin(ref.ratios, eps) > 1e-7, "near-tie in the independence test"
    assert np.array_equal(F.fibers()[0], ref.fibers)
    assert np.array_equal(F.R_dense(), ref.R)
    if ref.R.shape[1]:
        U = F.U()
        assert rel_fro(U, ref.U) <= u_tol(ref.R)
        assert u_residual(U, ref.R) <= 2.0 * u_residual(ref.U, ref.R) + 1e-9
    # C: each entry within the FP64 accumulation bar (1e-12 of sum |r_m||x_f|),
    # plus the rounding to FP32 when C is stored as float
    if cols is None:
        cols = np.arange(ref.X.n_cols)
    got = F.C_columns(cols)
    want = O.c_columns(ref.X, ref.R, cols)
    Xa = O.Matricized(ref.X.n_rows, ref.X.n_cols, ref.X.ptr, ref.X.rows, np.abs(ref.X.vals))
    scale = O.c_columns(Xa, np.abs(ref.R), cols)
    bar = 1e-12 * scale + (2.0 ** -24 * np.abs(want) if precision == 1 else 0.0)
    assert np.all(np.abs(got - want) <= bar)
    e_ref = O.projection_error(ref.X, ref.R)
    assert abs(F.error() - e_ref) <= error_tol_real(e_ref, ref.R)


@pytest.mark.parametrize("dims", [(12, 10, 9), (7, 6, 5, 4)])
@pytest.mark.parametrize("precision", [0, 1])
def test_real_every_mode(dims, precision):
    m = ctd()
    idx, val = synth.nway_real(dims, int(np.prod(dims)) // 2, seed=len(dims) + 30)
    X = m.CooN.from_arrays(dims, idx, val)
    for alpha in range(1, len(dims) + 1):
        F = m.ctd_static_nway(X, alpha, 80, 1e-6, alpha, precision, m.CTD_KEEP_DIST)
        ref = O.ctd_s_nway(dims, idx, val, alpha, 80, 1e-6, alpha)
        n2, c = F.column_dist()
        assert np.array_equal(n2.astype(np.int64), ref.sqnorms)   # the A28 weights
        assert np.array_equal(c.astype(np.int64), ref.cdf)
        check_real(F, ref, 1e-6, precision)


def test_real_traffic_shape():
    """A 2000 x 2000 x 200 traffic tensor (8*10^4 nonzeros) with real values
    (the counts times 1 + 0.1 N(0, 1), random signs), FP32 bulk, C on
    sampled columns.  (Noise over several octaves makes the kept fibers so
    ill-conditioned that U is not resolved in FP64 on either side: reading
    A17.)"""
    m = ctd()
    coo = synth.traffic_10m(scale=0.2)
    rng = np.random.default_rng(3)
    val = (coo.val * (1 + 0.1 * rng.normal(0, 1, coo.nnz)) * rng.choice([-1, 1], coo.nnz))
    val = val.astype(np.float32)
    idx = [coo.i, coo.j, coo.k]
    F = m.ctd_static_nway(m.CooN.from_arrays(coo.dims, idx, val), 1, 500, 1e-6, 0, 1)
    ref = O.ctd_s_nway(coo.dims, idx, val, 1, 500, 1e-6, 0)
    nz = np.flatnonzero(np.diff(ref.X.ptr))
    cols = np.random.default_rng(4).choice(nz, 300, replace=False)
    check_real(F, ref, 1e-6, 1, cols=cols)


def test_real_values_holding_integers_match_counts():
    """FP32 values that are small integers give the integer path's draws,
    kept fibers, R, U and C (the weights are the integer squares times a
    power of two, and the Gram of integers is exact in FP64), and its error
    within the stated bar of the precision."""
    m = ctd()
    coo = synth.small_uniform()
    idx = [coo.i, coo.j, coo.k]
    for precision in (0, 1):
        Fr = m.ctd_static_nway(m.CooN.from_arrays(coo.dims, idx, coo.val.astype(np.float32)), 1,
                               50, 1e-6, 0, precision)
        Fi = m.ctd_static(m.Coo.from_synth(coo), 1, 50, 1e-6, 0, precision)
        assert np.array_equal(Fr.samples()[0], Fi.samples()[0])
        assert np.array_equal(Fr.fibers()[0], Fi.fibers()[0])
        assert np.array_equal(Fr.R_dense(), Fi.R_dense().astype(np.float64))
        assert rel_fro(Fr.U(), Fi.U()) <= 1e-12
        cols = np.arange(Fi.sizes().n_cols)
        assert np.array_equal(Fr.C_columns(cols), Fi.C_columns(cols))
        # the integer path's FP32-bulk error runs in FP32 (its stated bar);
        # the real path's is FP64 in both modes
        assert abs(Fr.error() - Fi.error()) <= error_tol(precision, Fi.error())


def test_real_nonfinite_is_rejected():
    m = ctd()
    dims = (5, 4, 3)
    idx, val = synth.nway_real(dims, 20, seed=5)
    for bad in (np.nan, np.inf):
        v = val.copy()
        v[7] = bad
        with pytest.raises(m.CtdError) as e:
            m.ctd_static_nway(m.CooN.from_arrays(dims, idx, v), 1, 5, 1e-6, 0)
        assert e.value.status == "CTD_EINVAL"
