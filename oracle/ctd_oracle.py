"""FP64 CPU oracle for CTD (Lee, Choi, Sael: "CTD: Fast, Accurate, and
Interpretable Method for Static and Dynamic Tensor Decompositions").

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke entry point and the
benchmark's CPU-baseline leg may import this module.  It is a plain, slow,
step-by-step restatement of the paper's method and shares no code with the
CUDA library: no kernels, helpers, tables or constants are common to both.
Inputs are plain arrays (the seeded generators produce them); nothing here
reads a value computed by the GPU path.

What each function follows:
  matricize              Section 2.1 (mode-alpha matricization), reading A1
  matricize_nway         Section 2.1 for an N-way tensor, reading A1
  column_sqnorms, cdf    Algorithm 1 (squared norms), Eq. (1)
  sampling_weights, column_weights   Eq. (1) for real (FP32) values, reading A28
  philox4x64_10          Salmon et al., SC'11 (counter-based RNG), reading A2
  sample_columns         Algorithm 1 (draws with replacement), reading A2
  unique_columns         Algorithm 1 (unique draws), reading A3
  ctd_s                  Algorithm 1, step by step, FP64
  ctd_s_nway             Algorithm 1 on an N-way tensor (Section 2.1's
                         matricization of any order, Algorithm 1 unchanged)
  ctd_d_step             Algorithm 2, step by step, FP64
  c_columns              Algorithm 1's C / Eq. (3), exact int64
  relative_error_dense   Eq. (error), brute force on small inputs
  memory_usage           Eq. (memoryEff): (nnz(C) + nnz(U) + nnz(R)) / nnz(X)
  projection_error       Lemma 3.2 (Eqs. 4-7): error = ||X - R R^+ X||^2/||X||^2
  ddos_candidates        Section 5, detection rule on R's fibers
  dynamic_state_from_static   Section 4's CTD-D setting: CTD-S factors of the
                         history as the starting state of Algorithm 2

Readings of points the paper leaves open (same letters everywhere):
  A1 column order of X_(alpha): little-endian over the other modes
     (alpha=1: f = j + J*k; alpha=2: f = i + I*k; alpha=3: f = i + I*j).
  A2 draws: Philox4x64-10 with key (seed, 0) and counter (k, step, stream, 0);
     u = first output word; target = floor(u * T / 2^64); the drawn column is
     the smallest f with cdf[f] > target.
  A3 I' is ascending.
  A4 equality in the independence test counts as dependent (skip).
  A5 Euclidean norms.
  A6 the relative error is the squared ratio.
  A9 a dynamic state may start empty; the first kept fiber then gives
     U = 1/(x^T x), as for Algorithm 1's first kept fiber.
  A10 an all-zero input yields no draws and an empty factor.
  A12 zero and negative values are allowed; squares are summed exactly, and
      ||X||^2 (or one column's sum) at or past 2^63 is an overflow error.
  A14 a residual ratio within 1e-7 of eps is a near-tie; parity cases are
      checked to have none (the decision there depends on rounding).
  A17 U is compared within max(1e-10, 1e-15 kappa(R^T R)) relative (both
      sides carry errors of order kappa u), and the GPU's ||U R^T R - I||
      may be at most twice this oracle's.
  A20 CTD-D's error: the reconstruction of earlier columns does not change
      when R grows, so each step adds ||dX||^2 - ||P dX||^2, P the
      projector onto range(R) after the step.
  A21 the test's residual is evaluated as x minus its orthogonal projection
      onto range(R), by Gram-Schmidt with reorthogonalization (equal to
      x - R U R^T x in exact arithmetic; stable in floating point).
  A23 Section 5's average norm is the exact sum of the representatives'
     norms rounded once, divided by their count (no summation order).
  A27 an entry of U counts as a nonzero of Eq. (memoryEff) when its
      magnitude exceeds 1e-12 of U's largest (rounding noise is not fill).
  A28 real values: each square on a fixed-point grid, floor(v^2 2^(32-E))
     with 2^E the smallest power of two above the largest square; the draws
     use those exact integers.
  A29 real values: the error's bar is the FP64 bar widened to
      4 n u kappa(R^T R) (n rows of R, u = 2^-53), since the Gram matrix of
      real values is rounded.

Parity pinned by tests/test_oracle_pins.py (brute force, numpy/scipy
library routines, invariants, chi-square).  The DDoS rule is pinned by a
hand-computed case and semantically (planted block), not against the
paper's Table 4 numbers (parity unpinned for Table 4: the CAIDA data are
not available).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

try:  # scipy is only used for sparse products (a library matmul)
    import scipy.sparse as _sp
except Exception:  # pragma: no cover
    _sp = None

_MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# Section 2.1: mode-alpha matricization (reading A1)
# ---------------------------------------------------------------------------

def matricize(dims, i, j, k, alpha: int):
    """Row index (the alpha index) and column index of each nonzero of X_(alpha).

    Returns (rows int64, cols int64, I_alpha, N_alpha)."""
    I, J, K = (int(d) for d in dims)
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    if alpha == 1:
        return i, j + J * k, I, J * K
    if alpha == 2:
        return j, i + I * k, J, I * K
    if alpha == 3:
        return k, i + I * j, K, I * J
    raise ValueError("alpha must be 1, 2 or 3")


def matricize_nway(dims, idx, alpha: int):
    """Section 2.1 for an N-way tensor: the row of a nonzero is its mode-alpha
    index and its column is the little-endian index of the other modes,
    col = sum over n != alpha of i_n * prod over m < n, m != alpha of I_m
    (reading A1; for N = 3 this is `matricize`).

    Returns (rows int64, cols int64, I_alpha, N_alpha)."""
    dims = [int(d) for d in dims]
    N = len(dims)
    if not 1 <= alpha <= N:
        raise ValueError("alpha must be in 1..N")
    idx = [np.asarray(x, dtype=np.int64) for x in idx]
    rows = idx[alpha - 1]
    cols = np.zeros_like(rows)
    stride = 1
    for n in range(N):
        if n == alpha - 1:
            continue
        cols = cols + idx[n] * stride
        stride *= dims[n]
    return rows, cols, dims[alpha - 1], stride


# ---------------------------------------------------------------------------
# Algorithm 1 / Eq. (1): squared column norms and their prefix sums
# ---------------------------------------------------------------------------

def column_sqnorms(cols, vals, n_cols: int) -> np.ndarray:
    """|X_(alpha)(:, f)|^2 for every column f, exact.

    Each square is below 2^63 (|v| <= 2^31).  When the column sums could
    leave the int64 range they are formed in Python integers, and a column
    sum at or past 2^63 raises OverflowError (reading A12: the
    distribution's integers are int64)."""
    v = np.asarray(vals, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    sq = v * v
    if sq.size == 0 or int(sq.max()) * int(np.bincount(cols).max()) < (1 << 63):
        out = np.zeros(n_cols, dtype=np.int64)
        np.add.at(out, cols, sq)
        return out
    exact = np.zeros(n_cols, dtype=object)
    np.add.at(exact, cols, sq.astype(object))
    if any(int(x) >= (1 << 63) for x in exact):
        raise OverflowError("a squared column norm does not fit in int64")
    return exact.astype(np.int64)


def sampling_weights(vals) -> np.ndarray:
    """Eq. (1)'s summands for real values (reading A28): the FP32 values'
    squares (exact in FP64) on a fixed-point grid, floor(v^2 * 2^(32 - E))
    with M = f * 2^E (f in [1/2, 1)) the largest square, so every weight is
    an exact integer below 2^32 (all zero when every value is zero)."""
    v = np.asarray(vals, dtype=np.float32).astype(np.float64)
    sq = v * v
    M = float(sq.max()) if sq.size else 0.0
    if M == 0.0:
        return np.zeros(sq.shape[0], dtype=np.int64)
    E = math.frexp(M)[1]
    return np.floor(np.ldexp(sq, 32 - E)).astype(np.int64)


def column_weights(cols, vals, n_cols: int) -> np.ndarray:
    """Per column of X_(alpha), the sum of its values' sampling weights
    (real values, reading A28); exact int64 (each weight < 2^32)."""
    out = np.zeros(n_cols, dtype=np.int64)
    np.add.at(out, np.asarray(cols, dtype=np.int64), sampling_weights(vals))
    return out


def cdf(sqnorms: np.ndarray) -> np.ndarray:
    """Inclusive prefix sum of the squared norms; the last entry is ||X||_F^2."""
    out = np.cumsum(np.asarray(sqnorms, dtype=np.int64))
    if out.size and (np.any(out < 0)):
        raise OverflowError("||X||_F^2 does not fit in int64")
    return out


# ---------------------------------------------------------------------------
# Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), reading A2
# ---------------------------------------------------------------------------

_PHILOX_M = (0xD2E7470EE14C6C93, 0xCA5A826395121157)
_PHILOX_W = (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B)


def philox4x64_10(counter: Sequence[int], key: Sequence[int]) -> List[int]:
    """Ten rounds of the Philox S-P network on a 4x64-bit counter.

    Each round multiplies words 0 and 2 by the two round multipliers, keeps
    the 128-bit products' halves, XORs the high halves with the odd words and
    the round key, and permutes; the key is bumped by the Weyl constants
    before every round after the first."""
    x = [int(c) & _MASK64 for c in counter]
    kk = [int(c) & _MASK64 for c in key]
    for r in range(10):
        if r:
            kk = [(kk[0] + _PHILOX_W[0]) & _MASK64, (kk[1] + _PHILOX_W[1]) & _MASK64]
        p0 = _PHILOX_M[0] * x[0]
        p1 = _PHILOX_M[1] * x[2]
        hi0, lo0 = p0 >> 64, p0 & _MASK64
        hi1, lo1 = p1 >> 64, p1 & _MASK64
        x = [hi1 ^ x[1] ^ kk[0], lo1, hi0 ^ x[3] ^ kk[1], lo0]
    return x


# ---------------------------------------------------------------------------
# Algorithm 1: sampling with replacement, then unique
# ---------------------------------------------------------------------------

def draw_target(k: int, total: int, seed: int, step: int = 0, stream: int = 0) -> int:
    """Draw k's integer target in [0, total): floor(u * total / 2^64)."""
    u = philox4x64_10((k, step, stream, 0), (seed, 0))[0]
    return (u * int(total)) >> 64


def sample_columns(cdf_arr: np.ndarray, s: int, seed: int, step: int = 0,
                   stream: int = 0) -> np.ndarray:
    """s column indices drawn with P(f) = |x_f|^2 / ||X||_F^2 (Algorithm 1)."""
    if cdf_arr.size == 0 or int(cdf_arr[-1]) == 0:
        return np.zeros(0, dtype=np.int64)  # reading A10
    total = int(cdf_arr[-1])
    out = np.empty(s, dtype=np.int64)
    for k in range(s):
        t = draw_target(k, total, seed, step, stream)
        # smallest f with cdf[f] > t
        out[k] = int(np.searchsorted(cdf_arr, t, side="right"))
    return out


def unique_columns(I: np.ndarray) -> np.ndarray:
    """I' = the distinct elements of I, ascending (Algorithm 1, reading A3)."""
    return np.unique(np.asarray(I, dtype=np.int64))


# ---------------------------------------------------------------------------
# Column access (CSC view of X_(alpha))
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Matricized:
    """X_(alpha) as CSC: column f holds rows[ptr[f]:ptr[f+1]]; values exact
    int64 for counts, float64 (from FP32) for real values."""

    n_rows: int
    n_cols: int
    ptr: np.ndarray
    rows: np.ndarray
    vals: np.ndarray

    @staticmethod
    def from_coo(dims, i, j, k, val, alpha: int) -> "Matricized":
        return Matricized.from_rows_cols(*matricize(dims, i, j, k, alpha), val)

    @staticmethod
    def from_rows_cols(rows, cols, n_rows: int, n_cols: int, val) -> "Matricized":
        order = np.lexsort((rows, cols))
        rows = rows[order]
        cols = cols[order]
        vals = np.asarray(val)
        vals = vals.astype(np.float64 if np.issubdtype(vals.dtype, np.floating) else np.int64)
        vals = vals[order]
        ptr = np.zeros(n_cols + 1, dtype=np.int64)
        np.add.at(ptr, cols + 1, 1)
        ptr = np.cumsum(ptr)
        return Matricized(n_rows, n_cols, ptr, rows, vals)

    def column(self, f: int) -> np.ndarray:
        """Dense column X_(alpha)(:, f) (int64, or float64 for real values)."""
        x = np.zeros(self.n_rows, dtype=self.vals.dtype)
        a, b = int(self.ptr[f]), int(self.ptr[f + 1])
        x[self.rows[a:b]] = self.vals[a:b]
        return x

    @property
    def real(self) -> bool:
        return bool(np.issubdtype(self.vals.dtype, np.floating))

    def sqnorm(self):
        """||X||_F^2: exact int for counts, FP64 for real values."""
        if self.real:
            return float(np.sum(self.vals * self.vals))
        return int(np.sum(self.vals * self.vals))

    def scipy(self):
        return _sp.csc_matrix((self.vals, self.rows, self.ptr), shape=(self.n_rows, self.n_cols))


# ---------------------------------------------------------------------------
# Algorithm 1 / Algorithm 2: the independence filter
# ---------------------------------------------------------------------------

def _filter(x_of, candidates, R_cols: List[np.ndarray], U: Optional[np.ndarray],
            eps: float):
    """Run the sequential independence test over `candidates` in order.

    R_cols holds the current columns (dense float64, length I_alpha); U is
    their (R^T R)^{-1} (None when R is empty).  For each candidate x
    (Algorithm 1 / Algorithm 2), step by step:
      residual: res = x - R U R^T x.  Because U = (R^T R)^{-1} (Colibri's
        Theorem 1, used in Lemma 3.2), R U R^T is the orthogonal projector
        onto range(R), so res is x minus its projection.  It is evaluated
        as res = x - Q (Q^T x) with an orthonormal basis Q of range(R),
        applied twice (Gram-Schmidt with reorthogonalization), which keeps
        ||res|| accurate to rounding however ill-conditioned R gets; the
        product R (U (R^T x)) with the incrementally updated U loses that
        accuracy once kappa(R^T R) grows large (reading A21).
      test: skip when ||res|| <= eps ||x|| (reading A4);
      update: delta = ||res||^2, y = U R^T x;
      U grows by the block update;
      x is appended to R (and res / ||res|| to Q).
    Returns (kept candidate positions, R_cols, U, ratios) where ratios[k] =
    ||res|| / ||x|| for every candidate (for tie margins).
    """
    kept: List[int] = []
    ratios: List[float] = []
    n0 = len(R_cols)
    cap = n0 + len(candidates)
    Rbuf = Qbuf = None
    for pos, f in enumerate(candidates):
        x = x_of(f).astype(np.float64)
        if Rbuf is None:
            Rbuf = np.zeros((x.shape[0], max(cap, 1)))
            Qbuf = np.zeros((x.shape[0], max(cap, 1)))
            for c, col in enumerate(R_cols):
                Rbuf[:, c] = col
            if n0:  # orthonormal basis of the warm-start columns
                Qbuf[:, :n0] = _orthonormal_basis(Rbuf[:, :n0])
        n = n0 + len(kept)
        xn = float(np.sqrt(x @ x))
        if n == 0:
            # Algorithm 1's first kept fiber (and reading A9): R <- [x], U <- 1/(x^T x)
            if xn == 0.0:
                ratios.append(0.0)
                continue
            Rbuf[:, 0] = x
            Qbuf[:, 0] = x / xn
            U = np.array([[1.0 / (x @ x)]])
            kept.append(pos)
            ratios.append(1.0)
            continue
        R = Rbuf[:, :n]
        Q = Qbuf[:, :n]
        res = x - Q @ (Q.T @ x)
        res = res - Q @ (Q.T @ res)
        rn = float(np.sqrt(res @ res))
        ratios.append(rn / xn if xn > 0 else 0.0)
        if rn <= eps * xn:
            continue
        delta = rn * rn
        y = U @ (R.T @ x)
        Un = np.empty((n + 1, n + 1))
        Un[:n, :n] = U + np.outer(y, y) / delta
        Un[:n, n] = -y / delta
        Un[n, :n] = -y / delta
        Un[n, n] = 1.0 / delta
        U = Un
        Rbuf[:, n] = x
        Qbuf[:, n] = res / rn
        kept.append(pos)
    if Rbuf is not None:
        R_cols = [Rbuf[:, c].copy() for c in range(n0 + len(kept))]
    return kept, R_cols, U, ratios


def _orthonormal_basis(R: np.ndarray) -> np.ndarray:
    """Orthonormal basis of range(R) for full-column-rank R (numpy QR)."""
    Q, _ = np.linalg.qr(R)
    return Q


@dataclasses.dataclass
class StaticResult:
    T: int                   # ||X||_F^2, exact
    sqnorms: np.ndarray      # |x_f|^2 for every column
    cdf: np.ndarray
    I: np.ndarray            # the s draws (Algorithm 1)
    I_unique: np.ndarray     # I' (Algorithm 1)
    kept: np.ndarray         # positions in I' of the columns of R
    fibers: np.ndarray       # column ids of R's fibers (= I_unique[kept])
    R: np.ndarray            # dense int64 I_alpha x s~
    U: np.ndarray            # float64 s~ x s~
    ratios: np.ndarray       # ||res|| / ||x|| per candidate in I' order
    X: Matricized


def ctd_s(dims, i, j, k, val, alpha: int, s: int, eps: float, seed: int,
          step: int = 0, stream: int = 0) -> StaticResult:
    """Algorithm 1 (CTD-S) up to U.  C is available through
    `c_full` or `c_columns` because it can be far larger than R and U."""
    return _ctd_s(matricize(dims, i, j, k, alpha), val, s, eps, seed, step, stream)


def ctd_s_nway(dims, idx, val, alpha: int, s: int, eps: float, seed: int) -> StaticResult:
    """Algorithm 1 on an N-way tensor (idx: the N index arrays): the same
    steps on the mode-alpha matricization of `matricize_nway`."""
    return _ctd_s(matricize_nway(dims, idx, alpha), val, s, eps, seed, 0, 0)


def _ctd_s(mat, val, s: int, eps: float, seed: int, step: int, stream: int) -> StaticResult:
    """Algorithm 1's steps on a matricization (rows, cols, I_alpha, N_alpha)."""
    rows, cols, n_rows, n_cols = mat
    X = Matricized.from_rows_cols(rows, cols, n_rows, n_cols, val)  # matricize
    if X.real:                                                      # squared norms
        sq = column_weights(cols, val, n_cols)                      # (A28 for reals)
    else:
        sq = column_sqnorms(cols, val, n_cols)
    c = cdf(sq)
    T = int(c[-1]) if c.size else 0
    I = sample_columns(c, s, seed, step, stream)                    # draws
    Iu = unique_columns(I)                                          # unique
    kept, R_cols, U, ratios = _filter(X.column, list(Iu), [], None, eps)  # 5-15
    fibers = Iu[np.asarray(kept, dtype=np.int64)] if kept else np.zeros(0, np.int64)
    if R_cols:
        R = np.stack([X.column(int(f)) for f in fibers], axis=1)
    else:
        R = np.zeros((X.n_rows, 0), dtype=X.vals.dtype)
        U = np.zeros((0, 0))
    return StaticResult(T, sq, c, I, Iu, np.asarray(kept, dtype=np.int64), fibers,
                        R, U, np.asarray(ratios), X)


# ---------------------------------------------------------------------------
# Algorithm 1 / Eq. (3): C_(alpha) = R^T X_(alpha), exact
# ---------------------------------------------------------------------------

def c_columns(X: Matricized, R: np.ndarray, cols) -> np.ndarray:
    """Dense columns C_(alpha)(:, cols) = R^T X_(alpha)(:, cols): exact int64
    for counts, float64 for real values."""
    R = np.asarray(R, dtype=X.vals.dtype)
    out = np.zeros((R.shape[1], len(cols)), dtype=X.vals.dtype)
    for n, f in enumerate(cols):
        a, b = int(X.ptr[f]), int(X.ptr[f + 1])
        if b > a:
            out[:, n] = R[X.rows[a:b], :].T @ X.vals[a:b]
    return out


def c_full(X: Matricized, R: np.ndarray):
    """C_(alpha) = R^T X_(alpha) as a scipy CSC matrix (exact int64 for
    counts, float64 for real values)."""
    Rs = _sp.csc_matrix(np.asarray(R, dtype=X.vals.dtype))
    C = (Rs.T @ X.scipy()).tocsc()
    C.eliminate_zeros()
    C.sort_indices()
    return C


# ---------------------------------------------------------------------------
# Eq. (error) and Lemma 3.2
# ---------------------------------------------------------------------------

def relative_error_dense(X: Matricized, R: np.ndarray, U: np.ndarray, C) -> float:
    """||X~ - X||_F^2 / ||X||_F^2 with X~_(alpha) = R U C_(alpha) (Eq. error,
    Eq. 3), computed densely.  Small inputs only."""
    Xd = X.scipy().toarray().astype(np.float64)
    Cd = C.toarray().astype(np.float64) if hasattr(C, "toarray") else np.asarray(C, np.float64)
    Xt = np.asarray(R, np.float64) @ (U @ Cd) if R.shape[1] else np.zeros_like(Xd)
    den = float(np.sum(Xd * Xd))
    if den == 0.0:
        return 0.0
    return float(np.sum((Xt - Xd) ** 2)) / den


def memory_usage(X: Matricized, R: np.ndarray, U: np.ndarray, C) -> float:
    """Eq. (memoryEff), Section 4 (Experimental Settings): the memory of the
    factors relative to the tensor's, counted in nonzero entries,
    (nnz(C) + nnz(U) + nnz(R)) / nnz(X).  C, R and X are exact integers; an
    entry of the floating-point U counts when its magnitude exceeds 1e-12 of
    U's largest (reading A27: a zero of the exact inverse may carry rounding
    noise)."""
    nnz_x = int(np.count_nonzero(X.vals))
    nnz_c = int(C.count_nonzero()) if hasattr(C, "count_nonzero") else int(np.count_nonzero(C))
    U = np.asarray(U, dtype=np.float64)
    nnz_u = int(np.count_nonzero(np.abs(U) > 1e-12 * np.abs(U).max())) if U.size else 0
    return (nnz_c + nnz_u + int(np.count_nonzero(R))) / nnz_x


def projection_error(X: Matricized, R: np.ndarray, chunk: int = 1 << 17) -> float:
    """Lemma 3.2: the CTD-S error equals ||X - R R^+ X||_F^2 / ||X||_F^2.

    Computed as 1 - ||Q^T X||_F^2 / ||X||_F^2 with Q an orthonormal basis of
    range(R) from numpy's QR (a library routine), streaming over columns."""
    T = X.sqnorm()
    if T == 0:
        return 0.0
    if R.shape[1] == 0:
        return 1.0
    Q, _ = np.linalg.qr(np.asarray(R, np.float64))
    Xs = X.scipy().astype(np.float64)
    acc = 0.0
    for a in range(0, X.n_cols, chunk):
        blk = Xs[:, a:a + chunk]
        if blk.nnz == 0:
            continue
        P = (blk.T @ Q)   # (cols x s~) dense
        acc += float(np.sum(P * P))
    return (T - acc) / T


# ---------------------------------------------------------------------------
# Algorithm 2 (CTD-D): one time step
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class DynamicState:
    """Factors after t steps: R^(t) (dense columns), U^(t), C^(t) (dense,
    d~_t x N^(t), optional), plus bookkeeping for the error."""

    n_rows: int
    n_cols_slice: int
    R_cols: List[np.ndarray] = dataclasses.field(default_factory=list)
    fibers: List[tuple] = dataclasses.field(default_factory=list)   # (t, f)
    U: Optional[np.ndarray] = None
    C: Optional[np.ndarray] = None          # dense float64, kept when track_c
    t: int = 0
    track_c: bool = True
    X_blocks: List = dataclasses.field(default_factory=list)   # for brute force
    err_num: float = 0.0
    err_den: int = 0


@dataclasses.dataclass
class StepResult:
    I: np.ndarray
    I_unique: np.ndarray
    kept: np.ndarray            # positions in I' of the new columns (Delta R)
    new_fibers: np.ndarray      # their fiber ids within the slice
    M: Optional[np.ndarray]     # ((Delta R)^T R^(t)) U^(t), Delta d~ x d~_t
    C_new: Optional[np.ndarray] # R^(t+1)^T Delta X, exact int64 (d~_{t+1} x J)
    T_slice: int
    ratios: np.ndarray


def ctd_d_step(state: DynamicState, dims2, i, j, val, d: int, eps: float,
               seed: int, stream: int = 0, keep_X: bool = False) -> StepResult:
    """Algorithm 2 for one incoming slice Delta X (I x J x 1) with alpha = 1.

    It samples d columns of Delta X_(alpha) exactly as Algorithm 1 does,
    warm-starts from R^(t), U^(t), runs the same sequential test against
    the growing R^(t+1), and updates C_(alpha) with the
    block form of Eq. (C_t+1_final), whose lower-left block is evaluated
    left to right as (((Delta R)^T R^(t)) U^(t)) C^(t) (the reordering)."""
    I_, J_ = (int(dims2[0]), int(dims2[1]))
    k = np.zeros_like(np.asarray(i))
    dX = Matricized.from_coo((I_, J_, 1), i, j, k, val, 1)          # matricize
    sq = column_sqnorms(matricize((I_, J_, 1), i, j, k, 1)[1], val, J_)  # squared norms
    c = cdf(sq)
    Ts = int(c[-1]) if c.size else 0
    Id = sample_columns(c, d, seed, state.t, stream)                 # draws
    Iu = unique_columns(Id)                                          # unique
    R_old = [col.copy() for col in state.R_cols]                     # warm start
    U_old = None if state.U is None else state.U.copy()
    d_t = len(R_old)
    kept, R_cols, U, ratios = _filter(dX.column, list(Iu), list(R_old), U_old, eps)  # 6-16
    new_f = Iu[np.asarray(kept, dtype=np.int64)] if kept else np.zeros(0, np.int64)
    # C update, Eq. (C_t+1_final)
    R_new_int = (np.stack([dX.column(int(f)) for f in new_f], axis=1)
                 if len(new_f) else np.zeros((I_, 0), np.int64))
    R_old_int = (np.stack([np.rint(col).astype(np.int64) for col in R_old], axis=1)
                 if d_t else np.zeros((I_, 0), np.int64))
    R_all_int = np.concatenate([R_old_int, R_new_int], axis=1)
    C_new = c_columns(dX, R_all_int, range(J_))                      # [R^(t)T dX; dR^T dX]
    M = None
    if len(new_f) and d_t:
        M = ((R_new_int.T.astype(np.float64) @ R_old_int.astype(np.float64)) @ U_old)
    if state.track_c:
        # C^(t) is d~_t x N^(t); before the first step it has no columns
        top = state.C if state.C is not None else np.zeros((d_t, 0))
        if len(new_f):
            # lower-left block, parenthesized from the left
            lower = M @ top if M is not None else np.zeros((len(new_f), top.shape[1]))
            left = np.concatenate([top, lower], axis=0)
        else:
            left = top                                                # no fiber kept: the block above only
        state.C = np.concatenate([left, C_new.astype(np.float64)], axis=1)
    state.R_cols = R_cols
    state.U = U if R_cols else None
    state.fibers += [(state.t, int(f)) for f in new_f]
    if keep_X:
        state.X_blocks.append(dX)
    # per-step error increment (the old columns' reconstruction is unchanged)
    if Ts:
        if R_cols:
            R = R_all_int.astype(np.float64)
            Q, _ = np.linalg.qr(R)
            P = dX.scipy().astype(np.float64).T @ Q
            state.err_num += Ts - float(np.sum(P * P))
        else:
            state.err_num += Ts
    state.err_den += Ts
    state.t += 1
    return StepResult(Id, Iu, np.asarray(kept, np.int64), new_f, M, C_new, Ts, np.asarray(ratios))


def dynamic_state_from_static(res: StaticResult, dims3, track_c: bool = True,
                              keep_X: bool = False) -> DynamicState:
    """The starting state of the paper's CTD-D experiments (Section 4,
    performance of CTD-D): the history, the first time slices of a tensor
    whose third mode is time, decomposed by Algorithm 1 (alpha = 1), then
    extended slice by slice by Algorithm 2.  A column f = j + J k of the
    history (reading A1) is fiber j of time step k; C^(t) of the history is
    Eq. (3)'s C = R^T X_(1); the error bookkeeping starts from the
    history's ||X - R R^+ X||^2 (Lemma 3.2) over ||X||^2.  The next step is
    time step K (its draws use that counter)."""
    I, J, K = (int(d) for d in dims3)
    st = DynamicState(I, J)
    st.track_c = track_c
    st.R_cols = [res.R[:, c].astype(np.float64) for c in range(res.R.shape[1])]
    st.fibers = [(int(f) // J, int(f) % J) for f in res.fibers]
    st.U = res.U.copy() if st.R_cols else None
    if track_c:
        st.C = (c_full(res.X, res.R).toarray().astype(np.float64) if st.R_cols
                else np.zeros((0, res.X.n_cols)))
    if keep_X:
        st.X_blocks.append(res.X)
    st.t = K
    st.err_num = projection_error(res.X, res.R) * float(res.T) if res.T else 0.0
    st.err_den = int(res.T)
    return st


def dynamic_error_dense(state: DynamicState) -> float:
    """Eq. (error) for X^(t) = [dX_0, ..., dX_{t-1}] with the literal dense C^(t)."""
    if not state.X_blocks or state.C is None:
        raise ValueError("needs keep_X=True and track_c=True")
    Xd = np.concatenate([b.scipy().toarray().astype(np.float64) for b in state.X_blocks], axis=1)
    den = float(np.sum(Xd * Xd))
    if den == 0.0:
        return 0.0
    if not state.R_cols:
        return 1.0
    R = np.stack(state.R_cols, axis=1)
    Xt = R @ (state.U @ state.C)
    return float(np.sum((Xt - Xd) ** 2)) / den


# ---------------------------------------------------------------------------
# Section 5: DDoS candidates from CTD-D's R
# ---------------------------------------------------------------------------

def ddos_candidates(fibers: Sequence[tuple], R_cols: Sequence[np.ndarray],
                    with_mean: bool = False):
    """Section 5's detector on R (reading A23): group R's fibers (t, destination) by
    destination; the first fiber of each group (in R's column order)
    represents it; report, ascending, the destinations whose representative's
    2-norm exceeds the average 2-norm over all representatives.

    Each norm is the square root (rounded once) of the column's exact integer
    sum of squares; the average is the exact sum of those norms rounded once
    (math.fsum), divided by their count, so it has no summation order."""
    first = {}
    for (t, dst), col in zip(fibers, R_cols):
        if dst not in first:
            c = np.asarray(col, dtype=np.int64)
            first[dst] = math.sqrt(float(int(np.dot(c, c))))
    mean = math.fsum(first.values()) / len(first) if first else 0.0
    out = sorted(dst for dst, nrm in first.items() if nrm > mean)
    return (out, mean) if with_mean else out
