"""Pins of the FP64 oracle against things other than itself: brute force on
dense arrays, numpy/scipy library routines, closed forms, invariants and a
chi-square test of the sampling law.  CPU only."""
import math

import numpy as np
import pytest

from oracle import ctd_oracle as O
from paper_1710_03608_gb300 import synth


def dense(coo):
    X = np.zeros(coo.dims, dtype=np.int64)
    X[coo.i, coo.j, coo.k] = coo.val
    return X


def unfold(X, alpha):
    """Kolda-Bader mode-n unfolding: move mode n first, then Fortran-order reshape."""
    Xm = np.moveaxis(X, alpha - 1, 0)
    return Xm.reshape(Xm.shape[0], -1, order="F")


# --- P1: matricization, squared norms, CDF ---------------------------------

@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_norms_and_cdf_match_dense_unfolding(alpha):
    coo = synth.tiny((7, 5, 4), 60, seed=3, signed=True)
    Xa = unfold(dense(coo), alpha)
    rows, cols, n_rows, n_cols = O.matricize(coo.dims, coo.i, coo.j, coo.k, alpha)
    assert (n_rows, n_cols) == Xa.shape
    # every nonzero lands at the unfolding's (row, col)
    assert np.array_equal(Xa[rows, cols], coo.val.astype(np.int64))
    sq = O.column_sqnorms(cols, coo.val, n_cols)
    assert np.array_equal(sq, np.sum(Xa * Xa, axis=0))
    c = O.cdf(sq)
    assert int(c[-1]) == int(np.sum(Xa * Xa))
    assert np.array_equal(np.diff(np.concatenate([[0], c])), sq)


def test_sqnorms_exact_past_int64_or_raise():
    """Column sums are exact integers: two values of 2^31 - 1 in one fiber sum
    to 2^63 - 2^33 + 2 (Python-int arithmetic) and are returned exactly;
    three reach past 2^63 and raise (reading A12), and so do five, whose sum
    would also wrap an unsigned 64-bit accumulator back to a small value."""
    big = 2 ** 31 - 1
    assert 2 * big * big == 2 ** 63 - 2 ** 33 + 2
    sq = O.column_sqnorms(np.array([3, 3, 0]), np.array([big, big, 2]), 5)
    assert int(sq[3]) == 2 ** 63 - 2 ** 33 + 2 and int(sq[0]) == 4
    for n in (3, 5):
        with pytest.raises(OverflowError):
            O.column_sqnorms(np.array([1] * n), np.array([big] * n), 2)
    assert (5 * big * big) % 2 ** 64 < 2 ** 63  # the wrapped sum looks valid


def test_matricized_columns_match_dense():
    coo = synth.tiny((6, 5, 4), 40, seed=5)
    Xa = unfold(dense(coo), 1)
    M = O.Matricized.from_coo(coo.dims, coo.i, coo.j, coo.k, coo.val, 1)
    for f in range(Xa.shape[1]):
        assert np.array_equal(M.column(f), Xa[:, f])


# --- P2: Philox4x64-10 against numpy's independent implementation ----------

@pytest.mark.parametrize("key", [(0, 0), (5, 0), (2**64 - 1, 12345)])
@pytest.mark.parametrize("ctr", [(0, 0, 0, 0), (7, 3, 1, 0), (2**63, 2**40, 9, 77)])
def test_philox_matches_numpy(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(ctr, dtype=np.uint64))
    want = [int(v) for v in bg.random_raw(4)]
    # numpy increments the counter before it generates a block
    c = list(ctr)
    c[0] += 1
    for w in range(4):
        if c[w] >= 2**64:
            c[w] -= 2**64
            if w + 1 < 4:
                c[w + 1] += 1
        else:
            break
    assert O.philox4x64_10(c, key) == want


# --- P3: sampling law --------------------------------------------------------

def test_sampling_chi_square():
    scipy_stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(11)
    sq = rng.integers(0, 50, size=64).astype(np.int64)
    sq[[3, 17, 40]] = 0
    c = O.cdf(sq)
    n = 200_000
    draws = O.sample_columns(c, n, seed=1234)
    counts = np.bincount(draws, minlength=64)
    assert counts[[3, 17, 40]].sum() == 0          # P(f) = 0 => never drawn
    p = sq / sq.sum()
    nz = p > 0
    stat, pval = scipy_stats.chisquare(counts[nz], n * p[nz])
    assert pval > 1e-3, (stat, pval)


def test_single_nonzero_column_is_always_drawn():
    sq = np.zeros(100, dtype=np.int64)
    sq[42] = 9
    draws = O.sample_columns(O.cdf(sq), 500, seed=0)
    assert np.all(draws == 42)


def test_empty_tensor_draws_nothing():
    assert O.sample_columns(O.cdf(np.zeros(10, np.int64)), 50, seed=0).size == 0


def test_draw_target_is_floor_of_scaled_u():
    # target = floor(u * T / 2^64) is always < T and monotone in u
    for T in (1, 2, 3, 10**12, 2**62 + 7):
        for k in range(20):
            t = O.draw_target(k, T, seed=9)
            assert 0 <= t < T


def test_draw_maps_target_to_smallest_column_past_it():
    """Algorithm 1's draw with reading A2: on a CDF with T = 4 every target
    t in {0..3} lands on a step, so a search that took cdf[f] >= t (or
    dropped the zero-norm columns differently) picks another column."""
    sq = np.array([0, 1, 0, 1, 1, 0, 1], dtype=np.int64)   # cdf 0 1 1 2 3 3 4
    want = {0: 1, 1: 3, 2: 4, 3: 6}
    draws = O.sample_columns(O.cdf(sq), 64, seed=5, step=2, stream=1)
    seen = set()
    for k, f in enumerate(draws):
        t = O.draw_target(k, 4, seed=5, step=2, stream=1)
        assert f == want[t]
        seen.add(t)
    assert seen == {0, 1, 2, 3}


# --- P4: unique ---------------------------------------------------------------

def test_unique_is_the_distinct_sorted_draws():
    sq = np.arange(1, 30, dtype=np.int64) ** 2
    I = O.sample_columns(O.cdf(sq), 200, seed=3)
    Iu = O.unique_columns(I)
    assert list(Iu) == sorted(set(int(x) for x in I))


# --- P5, P6: the independence filter and U ----------------------------------

def _planted():
    """Columns with planted dependencies: a scaled duplicate, a sum of two
    kept columns, and parallel single-nonzero columns on the same row."""
    I = 8
    base = np.array([[3, 0, 1, 0, 0, 2, 0, 0],
                     [0, 2, 0, 0, 1, 0, 0, 4],
                     [1, 1, 1, 1, 0, 0, 0, 0]], dtype=np.int64).T
    cols = [base[:, 0], base[:, 1], 2 * base[:, 0], base[:, 0] + base[:, 1], base[:, 2]]
    e3 = np.zeros(I, np.int64); e3[3] = 5
    e3b = np.zeros(I, np.int64); e3b[3] = 2
    cols += [e3, e3b]
    return np.stack(cols, axis=1)


def test_filter_skips_planted_dependencies():
    R0 = _planted()
    kept, R_cols, U, ratios = O._filter(lambda f: R0[:, f], list(range(R0.shape[1])), [], None, 1e-6)
    assert kept == [0, 1, 4, 5]
    R = np.stack(R_cols, axis=1)
    assert np.linalg.matrix_rank(R) == np.linalg.matrix_rank(R0.astype(float)) == len(kept)
    # P6: U = (R^T R)^{-1}
    G = R.T @ R
    Ui = np.linalg.inv(G)
    assert np.linalg.norm(U - Ui) <= 1e-12 * np.linalg.norm(Ui)
    assert np.linalg.norm(U @ G - np.eye(len(kept))) < 1e-10


def test_filter_tie_counts_as_dependent():
    # eps = 1 makes ||res|| <= ||x|| always true after the first column
    R0 = _planted()
    kept, *_ = O._filter(lambda f: R0[:, f], list(range(R0.shape[1])), [], None, 1.0)
    assert kept == [0]


def test_filter_compares_norms_against_eps():
    """Algorithm 1's independence test compares ||res|| with eps ||x|| (reading A5), not
    squared norms with eps or eps^2: at eps = 0.1 a fiber with residual
    ratio 0.050 is dependent and one with 0.206 is kept.  Comparing
    ||res||^2 with eps ||x||^2 would drop both; comparing ||res|| with
    eps^2 ||x|| would keep both."""
    X = np.array([[100, 0, 0], [100, 5, 0], [100, 0, 21]], dtype=np.int64).T
    kept, R_cols, _, ratios = O._filter(lambda f: X[:, f], [0, 1, 2], [], None, 0.1)
    assert kept == [0, 2]
    assert np.array_equal(np.stack(R_cols, axis=1), X[:, [0, 2]])


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_ctd_s_rank_and_U(seed):
    coo = synth.tiny((12, 6, 5), 90, seed=seed)
    res = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 40, 1e-6, seed)
    Xa = unfold(dense(coo), 1)
    R0 = Xa[:, res.I_unique].astype(float)
    assert np.array_equal(res.R, Xa[:, res.fibers])
    assert res.R.shape[1] == np.linalg.matrix_rank(R0)
    G = res.R.T.astype(float) @ res.R.astype(float)
    Ui = np.linalg.inv(G)
    assert np.linalg.norm(res.U - Ui) <= 1e-10 * np.linalg.norm(Ui)


# --- P7: C, the error, optimality (Lemma 3.2) --------------------------------

@pytest.mark.parametrize("alpha", [1, 2, 3])
def test_c_is_r_transpose_x(alpha):
    coo = synth.tiny((6, 7, 5), 80, seed=4, signed=True)
    res = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, alpha, 30, 1e-6, 0)
    Xa = unfold(dense(coo), alpha)
    C = O.c_full(res.X, res.R)
    assert np.array_equal(C.toarray(), res.R.T @ Xa)
    cols = [0, 3, Xa.shape[1] - 1]
    assert np.array_equal(O.c_columns(res.X, res.R, cols), (res.R.T @ Xa)[:, cols])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_error_forms_agree_with_lstsq(seed):
    coo = synth.tiny((10, 8, 6), 120, seed=seed + 10)
    res = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 25, 1e-6, seed)
    Xa = unfold(dense(coo), 1).astype(float)
    C = O.c_full(res.X, res.R)
    e_lit = O.relative_error_dense(res.X, res.R, res.U, C)
    e_proj = O.projection_error(res.X, res.R)
    # least squares against ALL sampled columns, duplicates and dependents included
    R0 = Xa[:, res.I]
    L, *_ = np.linalg.lstsq(R0, Xa, rcond=None)
    e_ls = np.sum((R0 @ L - Xa) ** 2) / np.sum(Xa ** 2)
    assert abs(e_lit - e_ls) <= 1e-10 * max(e_ls, 1e-3)
    assert abs(e_proj - e_ls) <= 1e-10 * max(e_ls, 1e-3)
    assert 0.0 <= e_ls <= 1.0


def test_error_hand_computed():
    """Eq. (error) by hand on X_(1) = [[1, 1], [0, 1]] (||X||^2 = 3):
    R = x_0 = (1, 0): U = 1, C = [1, 1], residual [[0, 0], [0, 1]], e = 1/3;
    R = x_1 = (1, 1): U = 1/2, C = [1, 2], residual [[1/2, 0], [-1/2, 0]],
    e = 1/6; both fibers: e = 0.  The squared ratio (reading A6): its root
    would give 0.577 and 0.408."""
    X = O.Matricized.from_coo((2, 2, 1), [0, 0, 1], [0, 1, 1], [0, 0, 0], [1, 1, 1], 1)
    for R, U, e in ((np.array([[1], [0]]), np.array([[1.0]]), 1 / 3),
                    (np.array([[1], [1]]), np.array([[0.5]]), 1 / 6),
                    (np.array([[1, 1], [0, 1]]), None, 0.0)):
        C = O.c_full(X, R)
        if R.shape[1] == 1:
            assert np.array_equal(C.toarray(), R.T @ np.array([[1, 1], [0, 1]]))
        else:
            U = np.linalg.inv((R.T @ R).astype(float))
        assert O.relative_error_dense(X, R, U, C) == pytest.approx(e, abs=1e-15)
        assert O.projection_error(X, R) == pytest.approx(e, abs=1e-15)


def test_sampling_every_fiber_gives_exact_reconstruction():
    coo = synth.tiny((6, 4, 3), 30, seed=2)
    res = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 4000, 1e-6, 5)
    nonempty = np.flatnonzero(res.sqnorms)
    assert np.array_equal(res.I_unique, nonempty)
    C = O.c_full(res.X, res.R)
    assert abs(O.relative_error_dense(res.X, res.R, res.U, C)) <= 1e-12


def test_error_identity_with_u_and_cct():
    # Eq. (7): ||X - R U C||^2 = T - <U, C C^T> when U = (R^T R)^{-1}, C = R^T X
    coo = synth.tiny((9, 7, 5), 100, seed=8)
    res = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 20, 1e-6, 8)
    C = O.c_full(res.X, res.R).toarray().astype(float)
    e_lit = O.relative_error_dense(res.X, res.R, res.U, O.c_full(res.X, res.R))
    e_gram = (res.T - float(np.sum(res.U * (C @ C.T)))) / res.T
    assert abs(e_lit - e_gram) < 1e-12


# --- P8, P9, P10: CTD-D ---------------------------------------------------------

def _slices(n, dims2=(9, 7), nnz=25, seed=0):
    out = []
    for t in range(n):
        c = synth.tiny((dims2[0], dims2[1], 1), nnz, seed=seed * 100 + t)
        out.append(c)
    return out


def test_first_dynamic_step_equals_static():
    sl = _slices(1, seed=3)[0]
    st = O.DynamicState(9, 7)
    step = O.ctd_d_step(st, (9, 7), sl.i, sl.j, sl.val, 20, 1e-6, seed=4)
    ref = O.ctd_s((9, 7, 1), sl.i, sl.j, sl.k, sl.val, 1, 20, 1e-6, 4)
    assert np.array_equal(step.I, ref.I)
    assert np.array_equal(step.new_fibers, ref.fibers)
    assert np.linalg.norm(st.U - ref.U) <= 1e-13 * np.linalg.norm(ref.U)
    assert np.array_equal(step.C_new, ref.R.T @ unfold(dense(sl), 1))


def test_dynamic_error_increment_matches_literal_c():
    st = O.DynamicState(9, 7)
    for t, sl in enumerate(_slices(6, seed=1)):
        O.ctd_d_step(st, (9, 7), sl.i, sl.j, sl.val, 4, 1e-6, seed=2, keep_X=True)
        e_inc = st.err_num / st.err_den
        e_lit = O.dynamic_error_dense(st)
        assert abs(e_inc - e_lit) <= 1e-10 * max(e_lit, 1e-6), (t, e_inc, e_lit)


def test_dynamic_c_exact_when_history_is_spanned():
    # if R^(t) spans every column of X^(t), C^(t+1) equals R^(t+1)^T X^(t+1)
    st = O.DynamicState(6, 5)
    sls = _slices(4, dims2=(6, 5), nnz=20, seed=2)
    for sl in sls:
        O.ctd_d_step(st, (6, 5), sl.i, sl.j, sl.val, 500, 1e-6, seed=1, keep_X=True)
    Xd = np.concatenate([b.scipy().toarray() for b in st.X_blocks], axis=1).astype(float)
    R = np.stack(st.R_cols, axis=1)
    assert np.linalg.matrix_rank(R) == np.linalg.matrix_rank(Xd)
    assert np.allclose(st.C, R.T @ Xd, rtol=1e-9, atol=1e-7)


def test_dynamic_c_hand_computed():
    """Algorithm 2 and Eq. (C_t+1_final) by hand, I = 3, two slices of two
    columns, eps = 0.5.  Slice 0: a = (1, 0, 0) and a' = (2, 1, 0); a' has
    residual ratio 1/sqrt(5) = 0.447 <= 0.5 against a, so R^(1) = [a] (its
    history is not spanned) and C^(1) = a^T [a, a'] = [1, 2].  Slice 1:
    b = (1, 1, 1) and an empty column; b's residual ratio against a is
    sqrt(2/3) > 0.5, so it is kept: R^(2) = [a, b].  The lower-left block
    ((b^T a) U^(1)) C^(1) = [1, 2] -- not b^T [a, a'] = [1, 3], since a' is
    outside range R^(1) -- the upper-right a^T [b, 0] = [1, 0] and the new
    block b^T [b, 0] = [3, 0], so C^(2) = [[1, 2, 1, 0], [1, 2, 3, 0]].
    The error: a' keeps its reconstruction a * 2 and residual (0, 1, 0) of
    squared norm 1; b is exact; e = 1 / (1 + 5 + 3) = 1/9 (reading A20)."""
    st = O.DynamicState(3, 2)
    r0 = O.ctd_d_step(st, (3, 2), [0, 0, 1], [0, 1, 1], [1, 2, 1], 50, 0.5, seed=3,
                      keep_X=True)
    assert list(r0.I_unique) == [0, 1] and list(r0.new_fibers) == [0]
    assert np.array_equal(st.C, [[1.0, 2.0]])
    r1 = O.ctd_d_step(st, (3, 2), [0, 1, 2], [0, 0, 0], [1, 1, 1], 50, 0.5, seed=3, keep_X=True)
    assert list(r1.new_fibers) == [0]
    assert np.array_equal(np.stack(st.R_cols, axis=1), [[1, 1], [0, 1], [0, 1]])
    assert np.allclose(r1.M, [[1.0]], rtol=0, atol=1e-15)
    assert np.allclose(st.C, [[1, 2, 1, 0], [1, 2, 3, 0]], rtol=0, atol=1e-14)
    assert st.err_num / st.err_den == pytest.approx(1 / 9, abs=1e-15)
    assert O.dynamic_error_dense(st) == pytest.approx(1 / 9, abs=1e-14)


def test_reordering_parenthesizations_agree():
    rng = np.random.default_rng(0)
    dR = rng.integers(0, 4, size=(30, 3)).astype(float)
    Rt = rng.integers(0, 4, size=(30, 6)).astype(float)
    U = np.linalg.inv(Rt.T @ Rt + np.eye(6))
    C = rng.integers(0, 9, size=(6, 40)).astype(float)
    forms = [((dR.T @ Rt) @ U) @ C, (dR.T @ (Rt @ U)) @ C, dR.T @ ((Rt @ U) @ C),
             dR.T @ (Rt @ (U @ C)), (dR.T @ Rt) @ (U @ C)]
    for f in forms[1:]:
        assert np.allclose(f, forms[0], rtol=1e-12, atol=1e-12)


# --- Section 5: DDoS rule on a planted block ---------------------------------

def test_ddos_rule_flags_planted_destinations():
    # background traffic uses destinations 0..29; two victims (33, 37) first
    # appear at steps 3-4, each hit by 12 sources with heavy counts
    I, J = 60, 40
    rng = np.random.default_rng(5)
    victims = [33, 37]
    st = O.DynamicState(I, J)
    for t in range(6):
        bg = synth.tiny((I, 30, 1), 150, seed=50 + t)
        i, j, v = list(bg.i), list(bg.j), list(bg.val)
        if t in (3, 4):
            for dst in victims:
                for s_ in rng.choice(I, size=12, replace=False):
                    i.append(s_); j.append(dst); v.append(40)
        O.ctd_d_step(st, (I, J), np.array(i), np.array(j), np.array(v), 10, 0.15, seed=3)
    flagged = O.ddos_candidates(st.fibers, st.R_cols)
    assert set(victims) <= set(flagged)
    assert len(flagged) < 10


def test_ddos_rule_hand_computed():
    """Section 5's rule on a hand-made R: fibers (t, destination) in column
    order; destination 7 appears twice and only its first fiber (norm 3)
    counts. Representatives' norms 3, 4, 5, 12 -> average 6 -> only 9 flagged;
    a representative equal to the average is not flagged (strict)."""
    fibers = [(0, 7), (0, 2), (1, 7), (1, 4), (2, 9)]
    cols = [np.array([3, 0, 0]), np.array([0, 4, 0]), np.array([100, 0, 0]),
            np.array([3, 0, 4]), np.array([12, 0, 0])]
    got, mean = O.ddos_candidates(fibers, cols, with_mean=True)
    assert mean == 6.0 and got == [9]
    # norms 2, 4, 6: the average equals the middle one, which is not flagged
    got, mean = O.ddos_candidates([(0, 1), (0, 2), (0, 3)],
                                  [np.array([2]), np.array([4]), np.array([6])], with_mean=True)
    assert mean == 4.0 and got == [3]
    # the average has no summation order: a thousand norms of sqrt(2) and one of
    # 1000 sqrt(2), exactly rounded once
    fib = [(0, d) for d in range(1001)]
    cols = [np.array([1, 1])] * 1000 + [np.array([1000, 1000])]
    got, mean = O.ddos_candidates(fib, cols, with_mean=True)
    assert mean == math.fsum([math.sqrt(2.0)] * 1000 + [math.sqrt(2e6)]) / 1001
    assert got == [1000]
    assert O.ddos_candidates([], []) == []


# --- A10 / A12 edge cases ----------------------------------------------------------

def test_all_zero_tensor():
    coo = synth.tiny((4, 3, 2), 5, seed=1)
    coo.val[:] = 0
    res = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 1, 10, 1e-6, 0)
    assert res.T == 0 and res.I.size == 0 and res.R.shape[1] == 0


def test_negative_values_allowed():
    coo = synth.tiny((8, 6, 4), 70, seed=9, signed=True)
    res = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, 2, 30, 1e-6, 1)
    Xa = unfold(dense(coo), 2).astype(float)
    R0 = Xa[:, res.I]
    L, *_ = np.linalg.lstsq(R0, Xa, rcond=None)
    e_ls = np.sum((R0 @ L - Xa) ** 2) / np.sum(Xa ** 2)
    assert abs(O.projection_error(res.X, res.R) - e_ls) < 1e-10


# --- Section 4's CTD-D setting: a state seeded with CTD-S factors of the history ---

def _stream_tensor(slices):
    """Stack slices (I x J x 1 each) along time: slice k becomes k = k."""
    I, J = slices[0].dims[0], slices[0].dims[1]
    i = np.concatenate([s.i for s in slices])
    j = np.concatenate([s.j for s in slices])
    k = np.concatenate([np.full(s.nnz, t) for t, s in enumerate(slices)])
    v = np.concatenate([s.val for s in slices])
    return (I, J, len(slices)), i, j, k, v


def test_seeded_state_one_slice_equals_one_step():
    """Seeding with CTD-S of a one-slice history equals one Algorithm 2 step
    from the empty state on that slice (same draws: counter step 0)."""
    sl = synth.tiny((30, 20, 1), 120, seed=61)
    dims3, i, j, k, v = _stream_tensor([sl])
    ref = O.ctd_s(dims3, i, j, k, v, 1, 25, 1e-6, 4)
    seeded = O.dynamic_state_from_static(ref, dims3)
    st = O.DynamicState(30, 20)
    O.ctd_d_step(st, (30, 20), sl.i, sl.j, sl.val, 25, 1e-6, 4)
    assert seeded.fibers == st.fibers and seeded.t == st.t == 1
    assert np.array_equal(np.stack(seeded.R_cols, 1), np.stack(st.R_cols, 1))
    assert np.allclose(seeded.U, st.U, rtol=1e-10, atol=0)
    assert np.array_equal(seeded.C, st.C)
    assert abs(seeded.err_num / seeded.err_den - st.err_num / st.err_den) <= 1e-12


def test_seeded_state_error_two_routes():
    """After seeding with a 6-slice history and three more steps, the literal
    Eq. (error) with the dense C (R U C over all columns) equals the per-step
    projection bookkeeping; the history's fibers are its slices' columns."""
    slices = [synth.tiny((40, 25, 1), 150, seed=70 + t) for t in range(9)]
    dims3, i, j, k, v = _stream_tensor(slices[:6])
    ref = O.ctd_s(dims3, i, j, k, v, 1, 40, 1e-6, 2)
    st = O.dynamic_state_from_static(ref, dims3, keep_X=True)
    assert abs(O.dynamic_error_dense(st) - st.err_num / st.err_den) <= 1e-10
    for (t, jj), col in zip(st.fibers, st.R_cols):
        s_ = slices[t]
        dense = np.zeros(40)
        m = s_.j == jj
        dense[s_.i[m]] = s_.val[m]
        assert np.array_equal(dense, col)
    for sl in slices[6:]:
        O.ctd_d_step(st, (40, 25), sl.i, sl.j, sl.val, 12, 1e-6, 2, keep_X=True)
    assert st.t == 9
    assert abs(O.dynamic_error_dense(st) - st.err_num / st.err_den) <= 1e-9


def test_memory_usage_by_hand():
    """Eq. (memoryEff) on a 2 x 2 x 1 tensor with X(0,0) = 1 and X(1,1) = 2,
    every fiber sampled: R = diag(1, 2) (2 nonzeros), U = (R^T R)^{-1} =
    diag(1, 1/4) (2), C = R^T X_(1) = diag(1, 4) (2), nnz(X) = 2, so the
    memory usage is (2 + 2 + 2) / 2 = 3."""
    res = O.ctd_s((2, 2, 1), np.array([0, 1]), np.array([0, 1]), np.array([0, 0]),
                  np.array([1, 2]), 1, 64, 1e-6, 0)
    assert np.array_equal(res.R, np.array([[1, 0], [0, 2]]))
    assert np.allclose(res.U, np.diag([1.0, 0.25]))
    C = O.c_full(res.X, res.R)
    assert np.array_equal(C.toarray(), np.array([[1, 0], [0, 4]]))
    assert O.memory_usage(res.X, res.R, res.U, C) == 3.0


# --- N-way tensors (Section 2.1 of any order) ------------------------------

def _random_nway(dims, nnz, seed):
    rng = np.random.default_rng(seed)
    lin = rng.choice(int(np.prod(dims)), size=nnz, replace=False)
    idx, rest = [], lin
    for d in dims:
        idx.append(rest % d)
        rest = rest // d
    val = rng.integers(1, 6, size=nnz) * rng.choice([-1, 1], size=nnz)
    return idx, val


@pytest.mark.parametrize("dims", [(5, 7), (3, 4, 2, 5), (2, 3, 2, 3, 2)])
def test_nway_matricization_matches_dense_unfolding(dims):
    """Every nonzero lands at its (row, column) of numpy's mode-n unfolding
    (mode n first, then Fortran order), for every mode."""
    idx, val = _random_nway(dims, 25, seed=len(dims))
    X = np.zeros(dims, dtype=np.int64)
    X[tuple(idx)] = val
    for alpha in range(1, len(dims) + 1):
        Xa = unfold(X, alpha)
        rows, cols, n_rows, n_cols = O.matricize_nway(dims, idx, alpha)
        assert (n_rows, n_cols) == Xa.shape
        assert np.array_equal(Xa[rows, cols], val)
        assert np.array_equal(O.column_sqnorms(cols, val, n_cols), np.sum(Xa * Xa, axis=0))


def test_nway_matricization_by_hand():
    """dims (2, 3, 2, 2), the entry at (1, 2, 0, 1), mode 3: its row is i3 = 0
    and its column i1 + 2 i2 + (2 * 3) i4 = 1 + 4 + 6 = 11 of 12."""
    rows, cols, n_rows, n_cols = O.matricize_nway((2, 3, 2, 2), [[1], [2], [0], [1]], 3)
    assert (int(rows[0]), int(cols[0]), n_rows, n_cols) == (0, 11, 2, 12)


def test_nway_reduces_to_three_way():
    """For N = 3 the N-way matricization is the 3-way one, and a 4-way tensor
    whose last mode has extent 1 gives CTD-S's result on the 3-way tensor."""
    coo = synth.tiny((6, 5, 4), 40, seed=21, signed=True)
    for alpha in (1, 2, 3):
        a = O.matricize(coo.dims, coo.i, coo.j, coo.k, alpha)
        b = O.matricize_nway(coo.dims, [coo.i, coo.j, coo.k], alpha)
        assert all(np.array_equal(x, y) for x, y in zip(a[:2], b[:2])) and a[2:] == b[2:]
        r3 = O.ctd_s(coo.dims, coo.i, coo.j, coo.k, coo.val, alpha, 30, 1e-6, 2)
        r4 = O.ctd_s_nway(coo.dims + (1,), [coo.i, coo.j, coo.k, np.zeros_like(coo.i)],
                          coo.val, alpha, 30, 1e-6, 2)
        assert np.array_equal(r3.I, r4.I) and np.array_equal(r3.fibers, r4.fibers)
        assert np.array_equal(r3.R, r4.R) and np.array_equal(r3.U, r4.U)


# --- real values (reading A28) ---------------------------------------------

def test_sampling_weights_by_hand():
    """Values 1.5, -0.5, 3: squares 2.25, 0.25, 9; the largest is 9 = 0.5625 * 2^4,
    so the grid is 2^(32 - 4) and the weights are 2.25 * 2^28, 0.25 * 2^28 and
    9 * 2^28 exactly; all zeros give zero weights."""
    w = O.sampling_weights(np.array([1.5, -0.5, 3.0], dtype=np.float32))
    assert list(w) == [603979776, 67108864, 2415919104]
    assert list(O.sampling_weights(np.zeros(3, np.float32))) == [0, 0, 0]


def test_real_values_holding_integers_draw_as_counts():
    """A real tensor whose values are small integers has weights proportional
    to the integer squares (a power of two apart), and floor(u T / 2^64)
    compared with a CDF scaled by a power of two picks the same column, so
    the draws, the kept fibers, R and U equal the integer oracle's."""
    coo = synth.tiny((8, 7, 6), 120, seed=41, vmax=9, signed=True)
    idx = [coo.i, coo.j, coo.k]
    for alpha in (1, 2, 3):
        ri = O.ctd_s_nway(coo.dims, idx, coo.val, alpha, 60, 1e-6, 5)
        rr = O.ctd_s_nway(coo.dims, idx, coo.val.astype(np.float32), alpha, 60, 1e-6, 5)
        assert np.array_equal(ri.I, rr.I) and np.array_equal(ri.fibers, rr.fibers)
        assert np.array_equal(ri.R.astype(np.float64), rr.R)
        assert np.allclose(ri.U, rr.U, rtol=1e-12, atol=0)
        assert rr.X.sqnorm() == float(ri.X.sqnorm())


def test_real_sampling_law():
    """The draws of a real tensor follow P(f) = ||x_f||^2 / ||X||^2 up to the
    grid: chi-square of 20,000 draws on 6 columns against the exact law."""
    vals = np.array([0.3, 1.7, -2.2, 0.05, 3.1, 1.0], dtype=np.float32)
    w = O.column_weights(np.arange(6), vals, 6)
    p_exact = vals.astype(np.float64) ** 2 / np.sum(vals.astype(np.float64) ** 2)
    assert np.allclose(w / w.sum(), p_exact, rtol=1e-8, atol=1e-9)
    I = O.sample_columns(O.cdf(w), 20000, 7)
    obs = np.bincount(I, minlength=6)
    chi2 = float(np.sum((obs - 20000 * p_exact) ** 2 / (20000 * p_exact)))
    assert chi2 < 20.5   # 5 degrees of freedom, p = 0.001
