"""CTD-S on N-way tensors (Section 2.1's matricization of any order):
ctd_static_nway through the C ABI against the oracle's ctd_s_nway."""
import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth
from tests.parity import error_tol, rel_fro, tie_margin, u_residual, u_tol

pytestmark = pytest.mark.gpu


def ctd():
    from paper_1710_03608_gb300 import ctd as m
    return m


def check(F, ref, eps, precision, full_c=True, c_cols=None):
    sz = F.sizes()
    assert sz.sqnorm_X == float(ref.T)
    I, Iu = F.samples()
    assert np.array_equal(I, ref.I) and np.array_equal(Iu, ref.I_unique)
    assert tie_margin(ref.ratios, eps) > 1e-7, "near-tie in the independence test"
    fib, _ = F.fibers()
    assert np.array_equal(fib, ref.fibers)
    assert np.array_equal(F.R_dense(), ref.R)
    if ref.R.shape[1]:
        U = F.U()
        assert rel_fro(U, ref.U) <= u_tol(ref.R)
        assert u_residual(U, ref.R) <= 2.0 * u_residual(ref.U, ref.R) + 1e-9
    if full_c:
        p, r, v = F.C()
        Cref = O.c_full(ref.X, ref.R)
        assert np.array_equal(p, Cref.indptr) and np.array_equal(r, Cref.indices)
        assert np.array_equal(v, Cref.data.astype(np.float64))
    if c_cols is not None:
        assert np.array_equal(F.C_columns(c_cols), O.c_columns(ref.X, ref.R, c_cols))
    e_ref = O.projection_error(ref.X, ref.R)
    assert abs(F.error() - e_ref) <= error_tol(precision, e_ref)


@pytest.mark.parametrize("dims", [(40, 30), (9, 8, 7, 6), (6, 5, 4, 3, 7)])
@pytest.mark.parametrize("precision", [0, 1])
def test_every_mode(dims, precision):
    m = ctd()
    idx, val = synth.nway_uniform(dims, 600, seed=len(dims) + 10, signed=True)
    X = m.CooN.from_arrays(dims, idx, val)
    for alpha in range(1, len(dims) + 1):
        F = m.ctd_static_nway(X, alpha, 80, 1e-6, alpha, precision, m.CTD_KEEP_DIST)
        ref = O.ctd_s_nway(dims, idx, val, alpha, 80, 1e-6, alpha)
        n2, c = F.column_dist()
        assert np.array_equal(n2.astype(np.int64), ref.sqnorms)
        assert np.array_equal(c.astype(np.int64), ref.cdf)
        check(F, ref, 1e-6, precision)


@pytest.mark.parametrize("alpha", [1, 4])
def test_four_way_traffic_size(alpha):
    """A 2000 x 2000 x 16 x 50 tensor (source x destination x port x time),
    2*10^5 nonzeros: the source mode and the time mode, FP32 bulk; C on
    sampled columns."""
    m = ctd()
    dims = (2000, 2000, 16, 50)
    idx, val = synth.nway_uniform(dims, 200_000, seed=77)
    F = m.ctd_static_nway(m.CooN.from_arrays(dims, idx, val), alpha, 300, 1e-6, 3,
                          m.CTD_FP32_BULK)
    ref = O.ctd_s_nway(dims, idx, val, alpha, 300, 1e-6, 3)
    rng = np.random.default_rng(1)
    nz = np.flatnonzero(np.diff(ref.X.ptr))
    check(F, ref, 1e-6, 1, full_c=False, c_cols=rng.choice(nz, 100, replace=False))


def test_host_input_and_three_way_agree():
    """Host input gives the device input's result, and a 3-way tensor through
    ctd_static_nway gives ctd_static's result (same draws, R, U)."""
    m = ctd()
    coo = synth.small_uniform()
    idx = [coo.i, coo.j, coo.k]
    for alpha in (1, 3):
        Fd = m.ctd_static_nway(m.CooN.from_arrays(coo.dims, idx, coo.val), alpha, 50, 1e-6, 0)
        Fh = m.ctd_static_nway(m.CooN.from_arrays(coo.dims, idx, coo.val, device=False), alpha,
                               50, 1e-6, 0)
        F3 = m.ctd_static(m.Coo.from_synth(coo), alpha, 50, 1e-6, 0)
        for F in (Fh, F3):
            assert np.array_equal(F.samples()[0], Fd.samples()[0])
            assert np.array_equal(F.fibers()[0], Fd.fibers()[0])
            assert np.array_equal(F.R_dense(), Fd.R_dense())
            assert np.array_equal(F.U(), Fd.U())


def test_errors_are_reported():
    m = ctd()
    dims = (5, 4, 3, 2)
    idx, val = synth.nway_uniform(dims, 20, seed=3)
    X = m.CooN.from_arrays(dims, idx, val)
    for alpha in (0, 5):
        with pytest.raises(m.CtdError) as e:
            m.ctd_static_nway(X, alpha, 5, 1e-6, 0)
        assert e.value.status == "CTD_EINVAL"
    bad = [a.copy() for a in idx]
    bad[2][4] = 3                      # mode 3 has extent 3
    with pytest.raises(m.CtdError) as e:
        m.ctd_static_nway(m.CooN.from_arrays(dims, bad, val), 1, 5, 1e-6, 0)
    assert e.value.status == "CTD_EINVAL"
    wide = (2, 70000, 70000)           # N_1 = 4.9 * 10^9 columns
    X = m.CooN.from_arrays(wide, [np.zeros(1), np.zeros(1), np.zeros(1)], np.ones(1))
    with pytest.raises(m.CtdError) as e:
        m.ctd_static_nway(X, 1, 5, 1e-6, 0)
    assert e.value.status == "CTD_EINVAL"
