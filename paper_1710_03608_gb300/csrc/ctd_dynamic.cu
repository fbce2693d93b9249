// CTD-D (Algorithm 2): one time step on a new slice dX.
//
// The first steps (matricize, draw, unique) are those of Algorithm 1 on dX
// alone (counter (k, t, stream)).  The step warm-starts from R^(t), U^(t) and tests the d' candidates
// in order against the growing R^(t+1).  For a block of candidates X_c the
// squared residual of candidate k against R^(t) and the candidates kept
// before it is the pivot of an in-order Cholesky (with skip) of the Schur
// complement
//     S = X_c^T X_c - W^T W,   W = L^{-1} B,   B = R^(t)^T X_c,
// where L L^T = R^(t)^T R^(t) is kept across steps (L^(t+1) =
// [[L, 0], [W_K^T, L_S]]).  W comes from forward substitution, so the pivots
// are backward stable (errors ~ n u ||x||^2); forming S as X_c^T X_c -
// B^T U B with the explicit inverse would amplify them by kappa and keep
// dependent fibers.  The block form takes the same decisions as the
// sequential loop.  With Y_K = U^(t) B_K and S_K = L_S L_S^T, the rank-|K|
// update of U is Algorithm 1's bordered update applied |K| times, in block form:
//     U^(t+1) = [[U + Y_K S_K^{-1} Y_K^T, -Y_K S_K^{-1}], [., S_K^{-1}]].
// C update: the new columns R^(t+1)^T dX are computed exactly; the
// lower-left block ((dR)^T R^(t)) U^(t) C^(t) of Eq. (C_t+1_final) is kept
// as M_{t+1} = ((dR)^T R^(t)) U^(t) = Y_K^T (the paper's left-to-right
// order) and applied to old columns when they are read.
// The error of the old columns does not change (their reconstruction
// R^(t+1) U^(t+1) [C; M C] equals R^(t) U^(t) C), so the relative error
// accumulates ||dX||^2 - ||P_{t+1} dX||^2 per step, with
// ||P_{t+1} dX||^2 = ||Q^T dX||_F^2 with an orthonormal basis Q of
// range(R^(t+1)) kept across steps (the same as sum_f c_f^T U^(t+1) c_f).
#include <algorithm>
#include <cstring>
#include <numeric>

#include "ctd_internal.cuh"

using namespace ctd;

namespace {

// a keep whose pivot is below this fraction of ||x||^2 (residual ratio below
// 1e-4) ends a filter round (see ctd_dynamic_step)
constexpr double WEAK_KEEP = 1e-8;

struct StepRec {
  int64_t d_draws = 0, d_unique = 0, d_kept = 0, d_before = 0, nnz = 0;
  int64_t ncols = 0;               // columns of X_(alpha) this record covers (a slice: J;
                                   // a seeded history: J times its time slices)
  double sq = 0.0, err = 0.0;      // ||dX||^2 and ||dX - P dX||^2
  double* WK = nullptr;            // W_K = L^(t)^{-1} R^(t)^T dR: d_before x d_kept
  double* M = nullptr;             // Y_K = L^(t)^{-T} W_K = U^(t) R^(t)^T dR, computed on
                                   // first request (column-major = M_{t+1} row-major)
  uint64_t* Coff = nullptr;        // new-column block, height d_before + d_kept
  uint32_t* Ccnt = nullptr;
  uint16_t* Crow = nullptr;
  void* Cval = nullptr;
  int64_t nnzC = 0;
};

__global__ void k_gather_cols_f64(const double* __restrict__ A, int64_t lda, int64_t m,
                                  const int* __restrict__ idx, int n, double* __restrict__ out,
                                  int64_t ldo) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % m, c = e / m;
    out[r + c * ldo] = A[r + (int64_t)idx[c] * lda];
  }
}

// out (n x m) = A^T for A (m x n)
__global__ void k_transpose_f64(const double* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                double* __restrict__ out, int64_t ldo) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % m, c = e / m;
    out[c + r * ldo] = A[r + c * lda];
  }
}

// V(:, c) = candidate column idx[c] (dense n_rows x n, V zeroed beforehand)
__global__ void k_densify_cols(const unsigned long long* __restrict__ cptr,
                               const int32_t* __restrict__ crow, const int32_t* __restrict__ cval,
                               const int* __restrict__ idx, int n, double* __restrict__ V,
                               int64_t ldv) {
  for (int c = blockIdx.x; c < n; c += gridDim.x) {
    const int k = idx[c];
    for (unsigned long long p = cptr[k] + threadIdx.x; p < cptr[k + 1]; p += blockDim.x)
      V[crow[p] + (int64_t)c * ldv] = (double)cval[p];
  }
}

// qn[i] += sum_c Qt(d0 + c, i)^2 for the n new rows of Q^T
__global__ void k_qn_add(const double* __restrict__ Qt, int64_t ld, int64_t d0, int n,
                         int64_t n_rows, double* __restrict__ qn) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = qn[i];
    for (int c = 0; c < n; ++c) {
      const double q = Qt[d0 + c + i * ld];
      s = fma(q, q, s);
    }
    qn[i] = s;
  }
}

__global__ void k_add_offset(const unsigned long long* __restrict__ in, int64_t n,
                             unsigned long long off, unsigned long long* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = in[e] + off;
}

}  // namespace

struct ctd_factors::Dyn {
  int64_t I = 0, J = 0;
  unsigned flags = 0;
  int64_t t = 0;                     // records so far (a seeded history is record 0)
  int64_t hist_k = 0;                // time slices of a seeded history (0: none)
  int64_t cap_d = 0;                 // leading dimension of U
  int64_t cap_cols = 0, cap_nnz = 0, cap_fib = 0;
  std::vector<StepRec> steps;
  std::vector<int64_t> fiber_id, fiber_step;
  double err_num = 0.0, err_den = 0.0;
  double sq_total = 0.0;
  int64_t nnz_total = 0, nnzC_total = 0;
  int64_t last_d = 0, last_du = 0;
  bool all_positive = true;          // every value seen so far > 0
  double max_T = 0.0;                // largest ||dX||^2 so far
  bool incomplete = false;           // a step failed after it began to change the state
  int64_t* lastI = nullptr;          // device [8192]
  int64_t* lastIu = nullptr;
};

// time index of the next incoming slice (the Philox counter's step and the
// step recorded with the fibers it contributes)
static inline int64_t next_time(const ctd_factors::Dyn& D) {
  return D.hist_k > 0 ? D.hist_k + (D.t - 1) : D.t;
}

ctd_factors::~ctd_factors() {
  if (dyn) {
    cudaStreamSynchronize(stream);
    for (auto& s : dyn->steps) {
      dfree(s.M, stream);
      dfree(s.WK, stream);
      dfree(s.Coff, stream);
      dfree(s.Ccnt, stream);
      dfree(s.Crow, stream);
      dfree(s.Cval, stream);
    }
    dfree(dyn->lastI, stream);
    dfree(dyn->lastIu, stream);
    dfree(U, stream);
    dfree(L, stream);
    dfree(Qt, stream);
    dfree(qn, stream);
    L = nullptr;
    Qt = nullptr;
    qn = nullptr;
    dfree(fibers, stream);
    fibers = nullptr;
    dfree(Rcolptr, stream);
    dfree(Rrow, stream);
    dfree(Rval, stream);
    dfree(Rrowptr, stream);
    dfree(Rcol, stream);
    dfree(Rcval, stream);
    U = nullptr;
    delete dyn;
    dyn = nullptr;
  }
}

extern "C" ctd_status ctd_dynamic_create(const int64_t dims2[2], int alpha, int precision,
                                         uint64_t seed, uint64_t stream_id, unsigned flags,
                                         ctd_factors** state) {
  if (!dims2 || !state) return fail(CTD_EINVAL, "NULL argument");
  if (alpha != 1 && alpha != 2) return fail(CTD_EINVAL, "alpha must be 1 or 2 (time is mode 3)");
  if (dims2[0] < 1 || dims2[1] < 1 || dims2[0] > INT32_MAX || dims2[1] > INT32_MAX)
    return fail(CTD_EINVAL, "slice dimensions must be in [1, 2^31)");
  if (precision != CTD_FP64 && precision != CTD_FP32_BULK)
    return fail(CTD_EINVAL, "unknown precision");
  if (flags & ~(unsigned)(CTD_KEEP_LAST_C | CTD_DETERMINISTIC))
    return fail(CTD_EINVAL, "unknown flag");
  ctd_factors* F = new ctd_factors();
  F->kind = 1;
  F->alpha = alpha;
  F->precision = precision;
  F->seed = seed;
  F->stream_id = stream_id;
  F->dims[0] = dims2[0];
  F->dims[1] = dims2[1];
  F->dims[2] = 1;
  mode_extents(F->dims, alpha, &F->n_rows, &F->n_cols);
  F->dyn = new ctd_factors::Dyn();
  F->dyn->I = dims2[0];
  F->dyn->J = dims2[1];
  F->dyn->flags = flags;
  ctd_status rc = dalloc_n(&F->dyn->lastI, 8192, nullptr);
  if (rc == CTD_OK) rc = dalloc_n(&F->dyn->lastIu, 8192, nullptr);
  if (rc == CTD_OK) rc = dalloc_n(&F->Rcolptr, 1, nullptr);
  if (rc == CTD_OK) rc = dalloc_n(&F->qn, F->n_rows, nullptr);
  if (rc == CTD_OK && cudaMemsetAsync(F->qn, 0, F->n_rows * 8, nullptr) != cudaSuccess)
    rc = fail(CTD_ECUDA, "memset failed");
  if (rc == CTD_OK && cudaMemsetAsync(F->Rcolptr, 0, 8, nullptr) != cudaSuccess)
    rc = fail(CTD_ECUDA, "memset failed");
  if (rc == CTD_OK && cudaStreamSynchronize(nullptr) != cudaSuccess)
    rc = fail(CTD_ECUDA, "synchronize failed");
  if (rc != CTD_OK) {
    delete F;
    return rc;
  }
  *state = F;
  return CTD_OK;
}

// grow L and Q^T (ld cap, a multiple of 512) to hold n kept fibers,
// keeping the first d
static ctd_status grow_U(ctd_factors* F, int64_t d, int64_t n, cudaStream_t st) {
  auto& D = *F->dyn;
  if (n <= D.cap_d) return CTD_OK;
  int64_t cap = std::max<int64_t>(std::max<int64_t>(2 * D.cap_d, n), 512);
  // d~ never exceeds I_alpha: up to 8192 rows, take that size at once (no
  // regrowth copies; at most 0.5 GB each for L and Q^T)
  if (F->n_rows <= 8192) cap = std::max<int64_t>(cap, F->n_rows);
  cap = (cap + 511) / 512 * 512;
  const int64_t rows = F->n_rows;
  double *L2, *Q2;
  CTD_TRY(dalloc_n(&L2, (size_t)cap * cap, st));
  if (ctd_status rc = dalloc_n(&Q2, (size_t)cap * rows, st); rc != CTD_OK) {
    dfree(L2, st);
    return rc;
  }
  CTD_CUDA(cudaMemsetAsync(L2, 0, (size_t)cap * cap * 8, st));
  CTD_CUDA(cudaMemsetAsync(Q2, 0, (size_t)cap * rows * 8, st));
  if (d > 0) {
    CTD_CUDA(cudaMemcpy2DAsync(L2, cap * 8, F->L, D.cap_d * 8, d * 8, d,
                               cudaMemcpyDeviceToDevice, st));
    CTD_CUDA(cudaMemcpy2DAsync(Q2, cap * 8, F->Qt, D.cap_d * 8, d * 8, rows,
                               cudaMemcpyDeviceToDevice, st));
  }
  dfree(F->L, st);
  dfree(F->Qt, st);
  F->L = L2;
  F->Qt = Q2;
  D.cap_d = cap;
  return CTD_OK;
}

// W(:, c) = Q^T x_c for sparse columns x_c (CSC) and Q given by rows (row i of
// Q at Qt + i * ld, first d entries used): a block per column, threads over
// the d entries, the column's nonzeros in order (deterministic); columns with
// more than skip_above nonzeros are left to the split kernels.
__global__ void k_qt_times_sparse(const unsigned long long* __restrict__ cptr,
                                  const int32_t* __restrict__ crow,
                                  const int32_t* __restrict__ cval, int n,
                                  const double* __restrict__ Qt, int64_t ld, int64_t d,
                                  unsigned long long skip_above, double* __restrict__ W) {
  for (int c = blockIdx.x; c < n; c += gridDim.x) {
    const unsigned long long a = cptr[c], b = cptr[c + 1];
    if (b - a > skip_above) continue;  // a heavy column: split over blocks elsewhere
    for (int64_t r0 = 0; r0 < d; r0 += 4 * (int64_t)blockDim.x) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      for (unsigned long long p = a; p < b; ++p) {
        const double v = (double)cval[p];
        const double* q = Qt + (int64_t)crow[p] * ld;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t r = r0 + threadIdx.x + (int64_t)u * blockDim.x;
          if (r < d) acc[u] = fma(v, q[r], acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t r = r0 + threadIdx.x + (int64_t)u * blockDim.x;
        if (r < d) W[r + (int64_t)c * d] = acc[u];
      }
    }
  }
}

__global__ void k_i32_to_i64(const int* __restrict__ in, int n, int64_t* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    out[e] = in[e];
}

// y += x (n entries)
// Y(:, idx[c]) += X(:, c) (or = when add is 0), m rows, for c < n
__global__ void k_scatter_cols_f64(const double* __restrict__ X, int64_t ldx, int64_t m,
                                   const int* __restrict__ idx, int n, int add,
                                   double* __restrict__ Y, int64_t ldy) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % m, c = e / m;
    double* y = Y + r + (int64_t)idx[c] * ldy;
    *y = add ? *y + X[r + c * ldx] : X[r + c * ldx];
  }
}

__global__ void k_axpy_f64(int64_t n, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] += x[e];
}

// out (lower, n x n, ld ldo) = transpose of the upper triangle of A (ld lda);
// out's strict upper triangle is left alone
__global__ void k_lower_from_upper_T(const double* __restrict__ A, int64_t lda, int64_t n,
                                     double* __restrict__ out, int64_t ldo) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % n, c = e / n;
    if (r >= c) out[r + c * ldo] = A[c + r * lda];
  }
}

// column c of V (m x n, ld m) scaled to unit norm (zero columns stay zero)
__global__ void k_unit_columns(double* __restrict__ V, int64_t m, int n) {
  __shared__ double part[32];
  __shared__ double scale;
  for (int c = blockIdx.x; c < n; c += gridDim.x) {
    double* v = V + (int64_t)c * m;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) acc = fma(v[i], v[i], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
      scale = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
    }
    __syncthreads();
    const double sc = scale;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) v[i] *= sc;
    __syncthreads();
  }
}

__global__ void k_add_diag(double* __restrict__ A, int64_t lda, int n, double x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    A[i + (int64_t)i * lda] += x;
}

// One Cholesky-QR pass: L L^T = V^T V + shift I, out = V L^{-T}.  *ok is
// false if a pivot was not positive (V numerically rank deficient).
static ctd_status cholqr_pass(const double* V, int64_t m, int n, double shift, double* out,
                              Arena& scratch, cudaStream_t st, bool* ok) {
  double *G, *L, *Li, *thr;
  int *keep, *idx;
  unsigned* status;
  CTD_TRY(scratch.get(&G, (size_t)n * n));
  CTD_TRY(scratch.get(&L, (size_t)n * n));
  CTD_TRY(scratch.get(&Li, (size_t)n * n));
  CTD_TRY(scratch.get(&thr, n));
  CTD_TRY(scratch.get(&keep, n));
  CTD_TRY(scratch.get(&idx, n + 1));
  CTD_TRY(scratch.get(&status, 4));
  dgemm(true, false, n, n, m, 1.0, V, m, V, m, 0.0, G, n, st);
  if (shift > 0.0) CTD_LAUNCH(k_add_diag, (grid_for(n, 256, 64)), (256), 0, st, G, n, n, shift);
  CTD_CUDA(cudaMemsetAsync(thr, 0, (size_t)n * 8, st));
  CTD_CUDA(cudaMemsetAsync(status, 0, 4 * sizeof(unsigned), st));
  CTD_TRY(launch_chol_skip(G, n, n, thr, keep, st, nullptr, nullptr, status));
  launch_compact_flags(keep, n, idx, idx + n, st);
  int nk = 0;
  unsigned h_status = 0;
  CTD_TRY(d2h(&nk, idx + n, 1, st));
  CTD_TRY(d2h(&h_status, status, 1, st));
  CTD_CUDA(cudaGetLastError());
  CTD_TRY(sync(st));
  if (h_status & DEV_TIMEOUT) return fail(CTD_ETIMEOUT, "skip-Cholesky grid barrier gave up");
  *ok = nk == n;
  if (!*ok) return CTD_OK;
  launch_gather_lower(G, n, idx, idx + n, n, L, n, st);
  CTD_TRY(tri_inverse(L, n, n, Li, n, st));
  dgemm(false, true, m, n, n, 1.0, V, m, Li, n, 0.0, out, m, st);
  return CTD_OK;
}

template <typename T>
static ctd_status grow_array(T** p, int64_t used, int64_t need, int64_t* cap, cudaStream_t st) {
  if (need <= *cap) return CTD_OK;
  int64_t c = std::max<int64_t>(std::max<int64_t>(2 * *cap, need), 1024);
  T* q;
  CTD_TRY(dalloc_n(&q, c, st));
  if (used > 0) CTD_CUDA(cudaMemcpyAsync(q, *p, used * sizeof(T), cudaMemcpyDeviceToDevice, st));
  dfree(*p, st);
  *p = q;
  *cap = c;
  return CTD_OK;
}

// The new columns' residuals V (nr x kr, orthogonal to range(Q) already)
// become kr new basis vectors: V2 = V L_S^{-T} (L_S the filter's factor of
// their Schur complement, Li its inverse) is orthonormal up to the filter's
// rounding and one Cholesky-QR pass makes it so to working precision.  If
// that pass meets a non-positive pivot (V2 too far from orthonormal), the
// residuals are orthonormalized from scratch: unit columns, one shifted
// Cholesky-QR pass, then two plain ones (Fukaya et al., SIAM J. Sci. Comput.
// 42(1), 2020).  Lam^T = Q_new^T V (upper triangular up to rounding) gives
// L's new diagonal block; Q_new^T goes into Qt after the first dtc rows and
// the row norms of Q grow by those of Q_new.  V2 and Vq are nr x kr scratch.
static ctd_status finish_basis(ctd_factors* F, int64_t dtc, int kr, double* V, double* V2,
                               double* Vq, const double* Li, int64_t ldli, Arena& scratch,
                               cudaStream_t st) {
  const int64_t nr = F->n_rows, ld = F->dyn->cap_d;
  dgemm(false, true, nr, kr, kr, 1.0, V, nr, Li, ldli, 0.0, V2, nr, st);
  bool ok = false;
  CTD_TRY(cholqr_pass(V2, nr, kr, 0.0, Vq, scratch, st, &ok));
  if (!ok) {
    double* V0;  // the residuals themselves, for Lam below
    CTD_TRY(scratch.get(&V0, (size_t)nr * kr));
    CTD_CUDA(cudaMemcpyAsync(V0, V, (size_t)nr * kr * 8, cudaMemcpyDeviceToDevice, st));
    CTD_LAUNCH(k_unit_columns, ((unsigned)std::min(kr, 4096)), (256), 0, st, V, nr, kr);
    const double u = 1.1102230246251565e-16;
    const double shift = 11.0 * ((double)nr * kr + (double)kr * (kr + 1)) * u * kr;
    CTD_TRY(cholqr_pass(V, nr, kr, shift, V2, scratch, st, &ok));
    if (ok) CTD_TRY(cholqr_pass(V2, nr, kr, 0.0, V, scratch, st, &ok));
    if (ok) CTD_TRY(cholqr_pass(V, nr, kr, 0.0, Vq, scratch, st, &ok));
    if (!ok) return fail(CTD_ENOTSUP, "new basis vectors are numerically dependent");
    V = V0;
  }
  double* Lam;
  CTD_TRY(scratch.get(&Lam, (size_t)kr * kr));
  dgemm(true, false, kr, kr, nr, 1.0, Vq, nr, V, nr, 0.0, Lam, kr, st);
  CTD_LAUNCH(k_lower_from_upper_T, (grid_for((int64_t)kr * kr, 256, (int64_t)num_sms() * 4)),
             (256), 0, st, Lam, kr, kr, F->L + dtc + dtc * ld, ld);
  CTD_LAUNCH(k_transpose_f64, (grid_for(nr * kr, 256, (int64_t)num_sms() * 8)), (256), 0, st, Vq,
             nr, nr, kr, F->Qt + dtc, ld);
  CTD_LAUNCH(k_qn_add, (grid_for(nr, 256, (int64_t)num_sms() * 4)), (256), 0, st, F->Qt, ld, dtc,
             kr, nr, F->qn);
  return CTD_OK;
}

extern "C" ctd_status ctd_dynamic_step(ctd_factors* F, const ctd_coo3* dXd, int64_t d, double eps,
                                       void* stream) {
  if (!F || !dXd) return fail(CTD_EINVAL, "NULL argument");
  if (F->kind != 1 || !F->dyn) return fail(CTD_EINVAL, "not a CTD-D state");
  if (d < 1 || d > 8192) return fail(CTD_EINVAL, "d must be in [1, 8192]");
  if (!(eps >= 0.0 && eps < 1.0)) return fail(CTD_EINVAL, "eps must be in [0, 1)");
  auto& D = *F->dyn;
  if (D.incomplete)
    return fail(CTD_EINVAL, "an earlier step on this state failed part-way; create a new state");
  if (dXd->dims[0] != D.I || dXd->dims[1] != D.J || dXd->dims[2] != 1)
    return fail(CTD_EINVAL, "slice dimensions differ from the state's");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  F->stream = st;
  Arena scratch;
  scratch.st = st;
  CooDev X;
  CTD_TRY(stage_coo(dXd, F->alpha, scratch, st, &X));
  const int64_t dt = F->s_kept;
  const bool fp32 = F->precision == CTD_FP32_BULK;
  StepRec rec;
  // a step that fails returns the device buffers of its own record
  bool recorded = false;
  struct RecRelease {
    StepRec& r;
    bool& done;
    cudaStream_t st;
    ~RecRelease() {
      if (done) return;
      dfree(r.WK, st);
      dfree(r.M, st);
      dfree(r.Coff, st);
      dfree(r.Ccnt, st);
      dfree(r.Crow, st);
      dfree(r.Cval, st);
    }
  } rec_release{rec, recorded, st};
  rec.d_draws = d;
  rec.d_before = dt;
  rec.nnz = X.nnz;
  rec.ncols = F->n_cols;

  // matricize, draw, unique
  Matricized M;
  {
    PhaseScope ph("d_matricize", st);
    CTD_TRY(matricize(X, scratch, st, &M, (D.flags & CTD_DETERMINISTIC) != 0));
  }
  int* d_count;
  CTD_TRY(scratch.get(&d_count, 4));
  {
    PhaseScope ph("d_sample_unique", st);
    launch_sample(M.cdf, M.n_cols, d, F->seed, (uint64_t)next_time(D), F->stream_id, D.lastI, st);
    launch_sort_unique(D.lastI, d, D.lastIu, d_count, st);
  }
  unsigned status = 0;
  int du = 0;
  unsigned minkey[2] = {0, 0};
  uint64_t T = 0;
  CTD_TRY(d2h(minkey, M.minval, 2, st));
  const int minval = decode_min(minkey[0]);
  const bool x_int8 = minval >= -128 && decode_max(minkey[1]) <= 127;
  CTD_TRY(d2h(&status, M.status, 1, st));
  CTD_TRY(d2h(&du, d_count, 1, st));
  if (M.n_cols > 0) CTD_TRY(d2h(&T, M.cdf + (M.n_cols - 1), 1, st));
  CTD_CUDA(cudaGetLastError());
  CTD_TRY(sync(st));
  CTD_TRY(status_from_device(status));
  rec.sq = (double)T;
  rec.d_unique = du;
  // from here on the step changes the state; a failure below leaves it
  // incomplete, and later steps refuse it
  D.incomplete = true;
  if (X.nnz > 0 && minval <= 0) D.all_positive = false;
  D.max_T = std::max(D.max_T, (double)T);
  D.last_d = T ? d : 0;
  D.last_du = du;

  // the independence test, in rounds.  The block filter takes the sequential loop's
  // decisions while the kept block of the Schur complement stays well
  // conditioned.  A candidate kept with a tiny residual (ratio below 1e-4)
  // would make it ill-conditioned for every later candidate of the block (its
  // pivots and explicit re-tests would carry errors of order u * kappa), so a
  // round ends at such a keep: the round's kept candidates join R and the
  // orthonormal basis Q (explicit Gram-Schmidt, accurate for small residuals),
  // and the next round tests the remaining candidates against the grown basis.
  int kept_total = 0;
  // R^(t) already spans every mode-alpha vector (d~_t = I_alpha independent
  // columns): every candidate's residual is exactly zero, so none is kept.
  if (du > 0 && dt < M.n_rows) {
    // candidates X_c (CSC and by row)
    uint64_t *rc_sizes, *rc_ptr, *rcr_ptr;
    CTD_TRY(scratch.get(&rc_sizes, du + 1));
    CTD_TRY(scratch.get(&rc_ptr, du + 1));
    launch_column_sizes(M.colptr, D.lastIu, d_count, du, rc_sizes, st);
    launch_scan_u64(rc_sizes, rc_ptr, du, false, M.tmp, M.status, st);
    uint64_t nnz_cand = 0;
    CTD_TRY(d2h(&nnz_cand, rc_ptr + du, 1, st));
    CTD_TRY(sync(st));
    int32_t *rc_row, *rc_val, *rcr_col, *rcr_val;
    CTD_TRY(scratch.get(&rc_row, nnz_cand));
    CTD_TRY(scratch.get(&rc_val, nnz_cand));
    CTD_TRY(scratch.get(&rcr_col, nnz_cand));
    CTD_TRY(scratch.get(&rcr_val, nnz_cand));
    CTD_TRY(scratch.get(&rcr_ptr, M.n_rows + 1));
    launch_gather_columns(M.colptr, M.csc_row, M.csc_val, D.lastIu, d_count, du, rc_ptr, rc_row,
                          rc_val, st);
    // rows of each gathered column in ascending order, so every floating-point
    // sum over a candidate's entries is reproducible
    launch_sort_segments(rc_ptr, du, rc_row, rc_val, rcr_col, rcr_val, M.n_rows, st);
    CTD_TRY(build_csr_from_csc(rc_ptr, rc_row, rc_val, du, (int64_t)nnz_cand, M.n_rows, 0,
                               rcr_ptr, rcr_col, rcr_val, scratch, st));
    // exact Gram of the candidates (once) and their squared norms
    double *G0, *xn2;
    CTD_TRY(scratch.get(&G0, (size_t)du * du));
    CTD_TRY(scratch.get(&xn2, du));
    {
      PhaseScope ph("d_gram", st);
      CTD_TRY(launch_spmm_dense(M.csc(), D.lastIu, d_count, du,
                                CsrDev{rcr_ptr, rcr_col, rcr_val, du}, G0, du, st, &scratch));
      launch_thresholds(G0, du, du, 1.0, xn2, st);  // ||x_k||^2
    }
    const int64_t dt0 = dt;  // W_K of the whole step, against Q^(t), for the M chain
    if (dt0 > 0) CTD_TRY(dalloc_n(&rec.WK, (size_t)dt0 * du, st));
    uint64_t* rr_ptr = nullptr;  // by-row layout of a later round's candidates
    int32_t *rr_col = nullptr, *rr_val = nullptr;
    int* d_kr;
    CTD_TRY(scratch.get(&d_kr, 1));
    int start = 0;
    while (start < du && F->s_kept < M.n_rows) {
      const int dur = du - start;
      const int64_t dtc = F->s_kept;
      const uint64_t* rptr = rc_ptr + start;  // this round's candidates (absolute offsets)
      const uint64_t* cr_ptr = rcr_ptr;
      const int32_t *cr_col = rcr_col, *cr_val = rcr_val;
      if (start > 0) {
        if (!rr_ptr) {
          CTD_TRY(scratch.get(&rr_ptr, M.n_rows + 1));
          CTD_TRY(scratch.get(&rr_col, nnz_cand));
          CTD_TRY(scratch.get(&rr_val, nnz_cand));
        }
        CTD_TRY(build_csr_from_csc(rptr, rc_row, rc_val, dur, (int64_t)nnz_cand, M.n_rows, 0,
                                   rr_ptr, rr_col, rr_val, scratch, st));
        cr_ptr = rr_ptr;
        cr_col = rr_col;
        cr_val = rr_val;
      }
      // the Schur complement of the round's candidates against R:
      // S = X_r^T X_r - W^T W with W = Q^T X_r (= L^{-1} R^T X_r, R = Q L^T)
      double *S, *W = nullptr;
      CTD_TRY(scratch.get(&S, (size_t)dur * dur));
      CTD_CUDA(cudaMemcpy2DAsync(S, (size_t)dur * 8, G0 + start + (size_t)start * du,
                                 (size_t)du * 8, (size_t)dur * 8, dur, cudaMemcpyDeviceToDevice,
                                 st));
      if (dtc > 0) {
        PhaseScope ph("d_gram", st);
        CTD_TRY(scratch.get(&W, (size_t)dtc * dur));
        // candidates with more than 256 nonzeros: split over blocks
        const int64_t max_heavy = std::min<int64_t>(dur, (int64_t)nnz_cand / 257);
        CTD_LAUNCH(k_qt_times_sparse, ((unsigned)std::min(dur, 65535)), (256), 0, st,
                   reinterpret_cast<const unsigned long long*>(rptr), rc_row, rc_val, dur, F->Qt,
                   D.cap_d, dtc, max_heavy > 0 ? 256ull : ~0ull, W);
        if (max_heavy > 0) {
          int64_t* hl;
          unsigned* nh;
          CTD_TRY(scratch.get(&hl, max_heavy));
          CTD_TRY(scratch.get(&nh, 1));
          CTD_CUDA(cudaMemsetAsync(nh, 0, sizeof(unsigned), st));
          launch_list_columns_nnz(rptr, dur, 257, hl, nh, st);
          CTD_TRY(launch_heavy_columns(hl, nh, max_heavy, rptr, rc_row, rc_val, F->Qt, D.cap_d,
                                       dtc, W, nullptr, scratch, st));
        }
        dgemm(true, false, dur, dur, dtc, -1.0, W, dtc, W, dtc, 1.0, S, dur, st);
      }
      FilterIn fi;
      fi.du = dur;
      fi.S = S;
      fi.xnorm2 = xn2 + start;
      fi.eps = eps;
      fi.cptr = rptr;
      fi.crow = rc_row;
      fi.cval = rc_val;
      fi.c_rowptr = cr_ptr;
      fi.c_col = cr_col;
      fi.c_val = cr_val;
      fi.n_rows = M.n_rows;
      if (dtc > 0) {
        fi.dt = dtc;
        fi.Qt = F->Qt;
        fi.ldq = D.cap_d;
        fi.W = W;
      }
      FilterOut fo;
      CTD_TRY(run_filter(fi, fo, scratch, st));
      // the round ends at its first keep with a residual ratio below 1e-4
      int kr = fo.kept, next = du;
      for (int c = 0, seen = 0; c < dur; ++c) {
        if (!fo.keep_h[c]) continue;
        ++seen;
        if (fo.piv_h[c] < WEAK_KEEP * fo.xn_h[c]) {
          kr = seen;
          next = start + c + 1;
          break;
        }
      }
      const int* idx = fo.idx;  // round-relative positions of the kept candidates
      if (kr > 0) {
        CTD_CUDA(cudaMemcpyAsync(d_kr, &kr, sizeof(int), cudaMemcpyHostToDevice, st));
        const int64_t dn = dtc + kr;
        const double* Li = fo.Li;  // inverse of the filter's factor (leading kr x kr used)
        const int64_t ldli = fo.kept;
        F->U_valid = false;
        CTD_TRY(grow_U(F, dtc, dn, st));
        const int64_t ld = D.cap_d;
        // Gram-Schmidt of the kept candidates against Q: X_K = Q W_K + V
        // with V orthogonal to range(Q); then V = Q_new Lam^T (Lam lower
        // triangular) with Q_new orthonormal.  So R_new = Q_new' L_new^T with
        // L_new = [[L, 0], [W_K^T, Lam]], a Cholesky factor of R^T R; the
        // first d_before rows of W_K are kept for the M chain
        // (M_{t+1} = W_K^T L^(t)^{-1} = ((dR)^T R^(t)) U^(t), formed on request).
        PhaseScope ph("d_update_u", st);
        {
          PhaseScope phq("d_q_basis", st);
          const int64_t nr = M.n_rows;
          double *V, *V2, *Vq;
          CTD_TRY(scratch.get(&V, (size_t)nr * kr));
          CTD_TRY(scratch.get(&V2, (size_t)nr * kr));
          CTD_TRY(scratch.get(&Vq, (size_t)nr * kr));
          CTD_CUDA(cudaMemsetAsync(V, 0, (size_t)nr * kr * 8, st));
          CTD_LAUNCH(k_densify_cols, ((unsigned)std::min(kr, 4096)), (128), 0, st,
                     reinterpret_cast<const unsigned long long*>(rptr), rc_row, rc_val, idx, kr,
                     V, nr);
          if (dtc > 0) {
            double* WKs;
            CTD_TRY(scratch.get(&WKs, (size_t)dtc * kr));
            const unsigned gk = grid_for(dtc * kr, 256, (int64_t)num_sms() * 8);
            CTD_LAUNCH(k_gather_cols_f64, (gk), (256), 0, st, W, dtc, dtc, idx, kr, WKs, dtc);
            dgemm(true, false, nr, kr, dtc, -1.0, F->Qt, ld, WKs, dtc, 1.0, V, nr, st);
            // a second pass holds the new vectors orthogonal to ~u / rho for a
            // residual ratio rho >= eps (and adds its coefficients to W_K):
            // every later decision is taken against this basis.  A vector
            // whose first pass kept at least 1/sqrt(2) of its norm is
            // orthogonal to working accuracy after that pass (Kahan's
            // criterion, as given in Parlett, The Symmetric Eigenvalue
            // Problem), so in FP32 bulk mode only the weaker vectors take the
            // second pass; FP64 mode (error bar 1e-10) takes it for all.
            std::vector<int> weak;
            for (int c = 0, seen = 0; c < dur && seen < kr; ++c) {
              if (!fo.keep_h[c]) continue;
              if (!fp32 || fo.piv_h[c] < 0.5 * fo.xn_h[c]) weak.push_back(seen);
              ++seen;
            }
            const int nwk = (int)weak.size();
            if (nwk == kr) {
              double* Hm;
              CTD_TRY(scratch.get(&Hm, (size_t)dtc * kr));
              dgemm(false, false, dtc, kr, nr, 1.0, F->Qt, ld, V, nr, 0.0, Hm, dtc, st);
              dgemm(true, false, nr, kr, dtc, -1.0, F->Qt, ld, Hm, dtc, 1.0, V, nr, st);
              CTD_LAUNCH(k_axpy_f64, (gk), (256), 0, st, dtc * kr, Hm, WKs);
            } else if (nwk > 0) {
              int* d_weak;
              double *Vw, *Hm;
              CTD_TRY(scratch.get(&d_weak, nwk));
              CTD_TRY(scratch.get(&Vw, (size_t)nr * nwk));
              CTD_TRY(scratch.get(&Hm, (size_t)dtc * nwk));
              CTD_CUDA(cudaMemcpyAsync(d_weak, weak.data(), nwk * sizeof(int),
                                       cudaMemcpyHostToDevice, st));
              const unsigned gv = grid_for(nr * nwk, 256, (int64_t)num_sms() * 8);
              const unsigned gh = grid_for(dtc * nwk, 256, (int64_t)num_sms() * 8);
              CTD_LAUNCH(k_gather_cols_f64, (gv), (256), 0, st, V, nr, nr, d_weak, nwk, Vw, nr);
              dgemm(false, false, dtc, nwk, nr, 1.0, F->Qt, ld, Vw, nr, 0.0, Hm, dtc, st);
              dgemm(true, false, nr, nwk, dtc, -1.0, F->Qt, ld, Hm, dtc, 1.0, Vw, nr, st);
              CTD_LAUNCH(k_scatter_cols_f64, (gv), (256), 0, st, Vw, nr, nr, d_weak, nwk, 0, V, nr);
              CTD_LAUNCH(k_scatter_cols_f64, (gh), (256), 0, st, Hm, dtc, dtc, d_weak, nwk, 1, WKs,
                         dtc);
            }
            CTD_LAUNCH(k_transpose_f64, (gk), (256), 0, st, WKs, dtc, dtc, kr, F->L + dtc, ld);
            if (dt0 > 0)
              CTD_CUDA(cudaMemcpy2DAsync(rec.WK + (size_t)kept_total * dt0, (size_t)dt0 * 8, WKs,
                                         (size_t)dtc * 8, (size_t)dt0 * 8, kr,
                                         cudaMemcpyDeviceToDevice, st));
          }
          CTD_TRY(finish_basis(F, dtc, kr, V, V2, Vq, Li, ldli, scratch, st));
        }
        // append the kept columns to R (CSC)
        int64_t* newf;
        uint64_t *nsz, *nptr;
        CTD_TRY(scratch.get(&newf, kr));
        CTD_TRY(scratch.get(&nsz, kr + 1));
        CTD_TRY(scratch.get(&nptr, kr + 1));
        launch_gather_i64(D.lastIu + start, idx, d_kr, kr, newf, st);
        // the new columns come from the candidates' (row-sorted) CSC, by kept
        // position, so R's columns keep a reproducible row order
        int64_t* kp64;
        CTD_TRY(scratch.get(&kp64, kr));
        CTD_LAUNCH(k_i32_to_i64, (grid_for(kr, 256, 64)), (256), 0, st, idx, kr, kp64);
        launch_column_sizes(rptr, kp64, d_kr, kr, nsz, st);
        launch_scan_u64(nsz, nptr, kr, false, M.tmp, M.status, st);
        uint64_t nnz_new = 0;
        std::vector<int64_t> hf(kr);
        CTD_TRY(d2h(&nnz_new, nptr + kr, 1, st));
        CTD_TRY(d2h(hf.data(), newf, kr, st));
        CTD_TRY(sync(st));
        const int64_t nnzR = F->nnz_R;
        int64_t cap_cols = D.cap_cols + 1;
        CTD_TRY(grow_array(&F->Rcolptr, dtc + 1, dn + 1, &cap_cols, st));
        D.cap_cols = cap_cols - 1;
        int64_t cap_nnz_r = D.cap_nnz, cap_nnz_v = D.cap_nnz;
        CTD_TRY(grow_array(&F->Rrow, nnzR, nnzR + (int64_t)nnz_new, &cap_nnz_r, st));
        CTD_TRY(grow_array(&F->Rval, nnzR, nnzR + (int64_t)nnz_new, &cap_nnz_v, st));
        D.cap_nnz = cap_nnz_r;
        launch_gather_columns(rptr, rc_row, rc_val, kp64, d_kr, kr, nptr, F->Rrow + nnzR,
                              F->Rval + nnzR, st);
        CTD_LAUNCH(k_add_offset, (grid_for(kr + 1, 256, 64)), (256), 0, st,
                   reinterpret_cast<const unsigned long long*>(nptr), kr + 1,
                   (unsigned long long)nnzR,
                   reinterpret_cast<unsigned long long*>(F->Rcolptr + dtc));
        // the fiber ids on the device too (the detector of Section 5 reads them)
        CTD_TRY(grow_array(&F->fibers, dtc, dn, &D.cap_fib, st));
        CTD_CUDA(cudaMemcpyAsync(F->fibers + dtc, newf, (size_t)kr * sizeof(int64_t),
                                 cudaMemcpyDeviceToDevice, st));
        F->nnz_R = nnzR + (int64_t)nnz_new;
        F->s_kept = dn;
        for (int q = 0; q < kr; ++q) {
          D.fiber_id.push_back(hf[q]);
          D.fiber_step.push_back(next_time(D));
        }
        kept_total += kr;
      }
      start = next;
    }
    if (kept_total > 0) {
      // R by row (rows sorted by column), for the C fill
      dfree(F->Rrowptr, st);
      dfree(F->Rcol, st);
      dfree(F->Rcval, st);
      CTD_TRY(dalloc_n(&F->Rrowptr, M.n_rows + 1, st));
      CTD_TRY(dalloc_n(&F->Rcol, std::max<int64_t>(F->nnz_R, 1), st));
      CTD_TRY(dalloc_n(&F->Rcval, std::max<int64_t>(F->nnz_R, 1), st));
      CTD_TRY(build_csr_from_csc(F->Rcolptr, F->Rrow, F->Rval, F->s_kept, F->nnz_R, M.n_rows, 0,
                                 F->Rrowptr, F->Rcol, F->Rcval, scratch, st));
    }
  }
  rec.d_kept = kept_total;

  // C update: the new columns R^(t+1)^T dX (exact), and the error increment
  const int64_t dn = F->s_kept;
  double pu = 0.0;
  if (dn > 0 && X.nnz > 0) {
    CsrDev R{F->Rrowptr, F->Rcol, F->Rcval, (int)dn};
    R.nnz = F->nnz_R;
    uint32_t* ub;
    CTD_TRY(scratch.get(&ub, M.n_cols));
    CTD_TRY(dalloc_n(&rec.Coff, M.n_cols + 1, st));
    CTD_TRY(dalloc_n(&rec.Ccnt, M.n_cols, st));
    {
      PhaseScope ph("d_c_bounds", st);
      launch_c_bounds(M.csc(), M.n_cols, R, ub, st);
      launch_scan_u32(ub, rec.Coff, M.n_cols, false, M.tmp, M.status, st);
    }
    // the capacity is read back while the error kernels (which do not need
    // C) run
    uint64_t cap = 0;
    Readback rbc(st);
    CTD_TRY(rbc.add(&cap, rec.Coff + M.n_cols, 1));
    CTD_TRY(rbc.mark());
    double* d_pu;
    uint64_t* d_nnzc;
    CTD_TRY(scratch.get(&d_pu, 1));
    CTD_TRY(scratch.get(&d_nnzc, 1));
    {
      // ||P_{t+1} dX||^2 = ||Q^(t+1)^T dX||_F^2 with the maintained basis Q
      PhaseScope ph("d_error", st);
      CTD_TRY(launch_qform_rows(M.csc(), M.n_cols, M.nnz, F->Qt, D.cap_d, dn, F->qn, M.n_rows, d_pu,
                                scratch, st));
    }
    CTD_TRY(rbc.wait_mark());
    CTD_TRY(dalloc_n(&rec.Crow, std::max<uint64_t>(cap, 1), st));
    CTD_TRY(dalloc(&rec.Cval, std::max<uint64_t>(cap, 1) * (fp32 ? 4 : 8), st));
    {
      PhaseScope ph("d_c_fill", st);
      CTD_TRY(launch_c_fill(M.csc(), M.n_cols, M.n_rows, M.nnz, R, rec.Coff, rec.Ccnt, rec.Crow, rec.Cval, fp32,
                            D.all_positive, x_int8, (uint64_t)D.max_T, st));
    }
    launch_sum_u32(rec.Ccnt, M.n_cols, d_nnzc, st, C_COUNT);
    uint64_t nnzc = 0;
    CTD_TRY(d2h(&pu, d_pu, 1, st));
    CTD_TRY(d2h(&nnzc, d_nnzc, 1, st));
    CTD_TRY(d2h(&status, M.status, 1, st));
    CTD_CUDA(cudaGetLastError());
    CTD_TRY(sync(st));
    CTD_TRY(status_from_device(status));
    rec.nnzC = (int64_t)nnzc;
  }
  rec.err = (double)T - pu;
  if (rec.err < 0.0) rec.err = 0.0;
  D.err_num += rec.err;
  D.err_den += (double)T;
  D.sq_total += (double)T;
  D.nnz_total += X.nnz;
  D.nnzC_total += rec.nnzC;
  if ((D.flags & CTD_KEEP_LAST_C) && !D.steps.empty()) {
    auto& prev = D.steps.back();
    dfree(prev.Coff, st);
    dfree(prev.Ccnt, st);
    dfree(prev.Crow, st);
    dfree(prev.Cval, st);
    prev.Coff = nullptr;
    prev.Ccnt = nullptr;
    prev.Crow = nullptr;
    prev.Cval = nullptr;
  }
  D.steps.push_back(rec);
  recorded = true;
  D.t += 1;
  F->nnz_X = D.nnz_total;
  F->T = (uint64_t)D.sq_total;
  F->nnz_C = D.nnzC_total;
  F->have_err = true;
  F->err = D.err_den > 0 ? D.err_num / D.err_den : 0.0;
  D.incomplete = false;
  return CTD_OK;
}

__global__ void k_fiber_mod(const int64_t* __restrict__ f, int64_t n, int64_t w,
                            int64_t* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = f[e] % w;
}

__global__ void k_iota(int n, int* __restrict__ a32, int64_t* __restrict__ a64) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    a32[e] = e;
    a64[e] = e;
  }
}

// A CTD-D state that starts from CTD-S factors of the history (the setting of
// the paper's CTD-D experiments): R, its fibers (f = w + W k becomes time k,
// slice fiber w), the basis Q and the Cholesky factor L of R^T R (from the
// exact Gram of R, then the same orthonormalization as a step), and C of
// the history as record 0.
extern "C" ctd_status ctd_dynamic_from_static(const ctd_factors* S, uint64_t stream_id,
                                              unsigned flags, void* stream,
                                              ctd_factors** state) {
  if (!S || !state) return fail(CTD_EINVAL, "NULL argument");
  if (S->kind != 0) return fail(CTD_EINVAL, "not CTD-S factors");
  if (S->real) return fail(CTD_ENOTSUP, "CTD-D takes integer counts");
  if (S->alpha != 1 && S->alpha != 2) return fail(CTD_EINVAL, "alpha must be 1 or 2 (time is mode 3)");
  if (!S->Coff || !S->have_err)
    return fail(CTD_EINVAL, "the CTD-S factors need C and the error (no skip flags)");
  CTD_TRY(sync(S->stream));
  const int64_t dims2[2] = {S->dims[0], S->dims[1]};
  ctd_factors* F = nullptr;
  CTD_TRY(ctd_dynamic_create(dims2, S->alpha, S->precision, S->seed, stream_id, flags, &F));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  F->stream = st;
  auto& D = *F->dyn;
  const int64_t n = S->s_kept, nr = F->n_rows, W = F->n_cols, N = S->n_cols;
  const int64_t nnzR = S->nnz_R;
  const bool fp32 = S->precision == CTD_FP32_BULK;
  auto bail = [&](ctd_status rc) {
    cudaStreamSynchronize(st);
    ctd_free(F);
    return rc;
  };
#define SEED(expr)                     \
  do {                                 \
    ctd_status _r = (expr);            \
    if (_r != CTD_OK) return bail(_r); \
  } while (0)
#define SEEDC(call)                                                              \
  do {                                                                           \
    if ((call) != cudaSuccess) return bail(fail(CTD_ECUDA, std::string(#call))); \
  } while (0)
  Arena scratch;
  scratch.st = st;
  if (n > 0) {
    // R (CSC), its fibers, R by row
    dfree(F->Rcolptr, st);
    SEED(dalloc_n(&F->Rcolptr, n + 1, st));
    SEED(dalloc_n(&F->Rrow, std::max<int64_t>(nnzR, 1), st));
    SEED(dalloc_n(&F->Rval, std::max<int64_t>(nnzR, 1), st));
    SEED(dalloc_n(&F->fibers, n, st));
    SEEDC(cudaMemcpyAsync(F->Rcolptr, S->Rcolptr, (n + 1) * 8, cudaMemcpyDeviceToDevice, st));
    SEEDC(cudaMemcpyAsync(F->Rrow, S->Rrow, nnzR * 4, cudaMemcpyDeviceToDevice, st));
    SEEDC(cudaMemcpyAsync(F->Rval, S->Rval, nnzR * 4, cudaMemcpyDeviceToDevice, st));
    CTD_LAUNCH(k_fiber_mod, (grid_for(n, 256, 256)), (256), 0, st, S->fibers, n, W, F->fibers);
    D.cap_cols = n;
    D.cap_nnz = std::max<int64_t>(nnzR, 1);
    D.cap_fib = n;
    F->s_kept = n;
    F->nnz_R = nnzR;
    std::vector<int64_t> hf(n);
    SEED(d2h(hf.data(), S->fibers, n, st));
    SEED(sync(st));
    for (int64_t c = 0; c < n; ++c) {
      D.fiber_id.push_back(hf[c] % W);
      D.fiber_step.push_back(hf[c] / W);
    }
    SEED(dalloc_n(&F->Rrowptr, nr + 1, st));
    SEED(dalloc_n(&F->Rcol, std::max<int64_t>(nnzR, 1), st));
    SEED(dalloc_n(&F->Rcval, std::max<int64_t>(nnzR, 1), st));
    SEED(build_csr_from_csc(F->Rcolptr, F->Rrow, F->Rval, n, nnzR, nr, 0, F->Rrowptr, F->Rcol,
                            F->Rcval, scratch, st));
    // L: Cholesky factor of the exact Gram of R (all columns independent)
    int *i32, *keep, *idx, *cnt, *force;
    int64_t* i64;
    double *G, *thr, *piv, *Lk, *Li, *V, *V2, *Vq;
    unsigned* status;
    SEED(scratch.get(&i32, n));
    SEED(scratch.get(&i64, n));
    SEED(scratch.get(&keep, n));
    SEED(scratch.get(&idx, n));
    SEED(scratch.get(&cnt, 1));
    SEED(scratch.get(&force, n));
    SEED(scratch.get(&G, (size_t)n * n));
    SEED(scratch.get(&thr, n));
    SEED(scratch.get(&piv, n));
    SEED(scratch.get(&Lk, (size_t)n * n));
    SEED(scratch.get(&Li, (size_t)n * n));
    SEED(scratch.get(&status, 4));
    CTD_LAUNCH(k_iota, (grid_for(n, 256, 256)), (256), 0, st, (int)n, i32, i64);
    SEEDC(cudaMemcpyAsync(cnt, &n, sizeof(int), cudaMemcpyHostToDevice, st));
    SEED(launch_spmm_dense(CscDev{F->Rcolptr, F->Rrow, F->Rval}, i64, cnt, (int)n,
                           CsrDev{F->Rrowptr, F->Rcol, F->Rcval, (int)n}, G, n, st));
    SEEDC(cudaMemsetAsync(thr, 0, n * 8, st));
    SEEDC(cudaMemsetAsync(force, 0xff, n * sizeof(int), st));
    SEEDC(cudaMemsetAsync(status, 0, 4 * sizeof(unsigned), st));
    SEED(launch_chol_skip(G, n, n, thr, keep, st, force, piv, status));
    launch_compact_flags(keep, (int)n, idx, cnt, st);
    int kept = 0;
    unsigned h_status = 0;
    SEED(d2h(&kept, cnt, 1, st));
    SEED(d2h(&h_status, status, 1, st));
    SEED(sync(st));
    if (h_status & DEV_TIMEOUT) return bail(fail(CTD_ETIMEOUT, "skip-Cholesky grid barrier gave up"));
    if (kept != n)
      return bail(fail(CTD_ENOTSUP, "the history's fibers are numerically dependent"));
    launch_gather_lower(G, n, idx, cnt, (int)n, Lk, n, st);
    SEED(tri_inverse(Lk, n, n, Li, n, st));
    // Q and L through the same orthonormalization as a step's new columns
    SEED(grow_U(F, 0, n, st));
    SEED(scratch.get(&V, (size_t)nr * n));
    SEED(scratch.get(&V2, (size_t)nr * n));
    SEED(scratch.get(&Vq, (size_t)nr * n));
    SEEDC(cudaMemsetAsync(V, 0, (size_t)nr * n * 8, st));
    CTD_LAUNCH(k_densify_cols, ((unsigned)std::min<int64_t>(n, 4096)), (128), 0, st,
               reinterpret_cast<const unsigned long long*>(F->Rcolptr), F->Rrow, F->Rval, i32,
               (int)n, V, nr);
    SEED(finish_basis(F, 0, (int)n, V, V2, Vq, Li, n, scratch, st));
    F->U_valid = false;
  }
  // record 0: the history, whose C is CTD-S's C
  StepRec rec;
  rec.d_draws = S->s;
  rec.d_unique = S->s_unique;
  rec.d_kept = n;
  rec.d_before = 0;
  rec.nnz = S->nnz_X;
  rec.ncols = N;
  rec.sq = (double)S->T;
  rec.err = S->err * (double)S->T;
  rec.nnzC = S->nnz_C;
  const size_t vsz = fp32 ? 4 : 8;
  SEED(dalloc_n(&rec.Coff, N + 1, st));
  SEED(dalloc_n(&rec.Ccnt, std::max<int64_t>(N, 1), st));
  SEED(dalloc_n(&rec.Crow, std::max<uint64_t>(S->C_cap, 1), st));
  SEED(dalloc(&rec.Cval, std::max<uint64_t>(S->C_cap, 1) * vsz, st));
  SEEDC(cudaMemcpyAsync(rec.Coff, S->Coff, (N + 1) * 8, cudaMemcpyDeviceToDevice, st));
  SEEDC(cudaMemcpyAsync(rec.Ccnt, S->Ccnt, N * 4, cudaMemcpyDeviceToDevice, st));
  if (S->C_cap) {
    SEEDC(cudaMemcpyAsync(rec.Crow, S->Crow, S->C_cap * 2, cudaMemcpyDeviceToDevice, st));
    SEEDC(cudaMemcpyAsync(rec.Cval, S->Cval, S->C_cap * vsz, cudaMemcpyDeviceToDevice, st));
  }
  D.steps.push_back(rec);
  D.t = 1;
  D.hist_k = S->dims[2];
  D.err_num = rec.err;
  D.err_den = rec.sq;
  D.sq_total = rec.sq;
  D.nnz_total = S->nnz_X;
  D.nnzC_total = S->nnz_C;
  D.all_positive = S->min_val > 0;
  D.max_T = rec.sq;
  F->nnz_X = S->nnz_X;
  F->T = S->T;
  F->nnz_C = S->nnz_C;
  F->have_err = true;
  F->err = S->err;
  SEED(sync(st));
#undef SEED
#undef SEEDC
  *state = F;
  return CTD_OK;
}

// Getters refuse a state that a failed step left part-way changed.
namespace ctd {
ctd_status dyn_check_complete(const ctd_factors* F) {
  if (F->kind == 1 && F->dyn && F->dyn->incomplete)
    return fail(CTD_EINVAL, "an earlier step on this state failed part-way; create a new state");
  return CTD_OK;
}
}  // namespace ctd

extern "C" ctd_status ctd_get_step(const ctd_factors* F, int64_t t, int64_t info[4],
                                   double sq[2]) {
  if (!F || !F->dyn) return fail(CTD_EINVAL, "not a CTD-D state");
  CTD_TRY(dyn_check_complete(F));
  if (t < 0 || t >= F->dyn->t) return fail(CTD_EINVAL, "step out of range");
  const StepRec& r = F->dyn->steps[t];
  if (info) {
    info[0] = r.d_unique;
    info[1] = r.d_kept;
    info[2] = r.d_before;
    info[3] = r.nnz;
  }
  if (sq) {
    sq[0] = r.sq;
    sq[1] = r.err;
  }
  return CTD_OK;
}

// M_{t+1} (as Y_K = L^(t)^{-T} W_K) of step t, formed on first request; the
// leading d_before block of the current L is L^(t), since L only grows.
static ctd_status ensure_M(const ctd_factors* Fc, int64_t t) {
  ctd_factors* F = const_cast<ctd_factors*>(Fc);
  StepRec& r = F->dyn->steps[t];
  if (r.M || r.d_before == 0 || r.d_kept == 0) return CTD_OK;
  if (!r.WK) return fail(CTD_EINVAL, "inconsistent step record");
  cudaStream_t st = F->stream;
  const size_t n = (size_t)r.d_before * r.d_kept;
  CTD_TRY(dalloc_n(&r.M, n, st));
  CTD_CUDA(cudaMemcpyAsync(r.M, r.WK, n * 8, cudaMemcpyDeviceToDevice, st));
  tri_solve_lower_T(F->L, F->dyn->cap_d, r.d_before, r.M, r.d_before, r.d_kept, st);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

extern "C" ctd_status ctd_get_M(const ctd_factors* F, int64_t t, double* M) {
  if (!F || !F->dyn) return fail(CTD_EINVAL, "not a CTD-D state");
  CTD_TRY(dyn_check_complete(F));
  if (t < 0 || t >= F->dyn->t) return fail(CTD_EINVAL, "step out of range");
  const StepRec& r = F->dyn->steps[t];
  const size_t n = (size_t)r.d_kept * r.d_before;
  if (n == 0) return CTD_OK;
  if (!M) return fail(CTD_EINVAL, "NULL argument");
  CTD_TRY(ensure_M(F, t));
  CTD_TRY(d2h(M, r.M, n, F->stream));
  return sync(F->stream);
}

// ---------------------------------------------------------------------------
// dynamic getters used by the common entry points
// ---------------------------------------------------------------------------
namespace ctd {

ctd_status dyn_sizes(const ctd_factors* F, ctd_sizes* o) {
  CTD_TRY(dyn_check_complete(F));
  const auto& D = *F->dyn;
  o->n_rows = F->n_rows;
  o->n_cols = F->n_cols;
  o->s_draws = D.last_d;
  o->s_unique = D.last_du;
  o->s_kept = F->s_kept;
  o->nnz_R = F->nnz_R;
  o->nnz_C = D.nnzC_total;
  o->t_steps = D.t;
  o->nnz_X = D.nnz_total;
  o->sqnorm_X = D.sq_total;
  return CTD_OK;
}

ctd_status dyn_samples(const ctd_factors* F, int64_t* I, int64_t* Iu) {
  CTD_TRY(dyn_check_complete(F));
  const auto& D = *F->dyn;
  if (I) CTD_TRY(d2h(I, D.lastI, (size_t)D.last_d, F->stream));
  if (Iu) CTD_TRY(d2h(Iu, D.lastIu, (size_t)D.last_du, F->stream));
  return sync(F->stream);
}

ctd_status dyn_fibers(const ctd_factors* F, int64_t* fiber, int64_t* step) {
  CTD_TRY(dyn_check_complete(F));
  const auto& D = *F->dyn;
  for (size_t c = 0; c < D.fiber_id.size(); ++c) {
    if (fiber) fiber[c] = D.fiber_id[c];
    if (step) step[c] = D.fiber_step[c];
  }
  return CTD_OK;
}

// U^(t) = (R^T R)^{-1} = L^{-T} L^{-1}, formed from the maintained factor on
// the first request after a step that kept fibers, then cached.
ctd_status dyn_U(const ctd_factors* Fc, double* U) {
  CTD_TRY(dyn_check_complete(Fc));
  ctd_factors* F = const_cast<ctd_factors*>(Fc);
  const int64_t n = F->s_kept;
  if (n == 0) return CTD_OK;
  cudaStream_t st = F->stream;
  if (!F->U_valid) {
    dfree(F->U, st);
    F->U = nullptr;
    CTD_TRY(dalloc_n(&F->U, (size_t)n * n, st));
    Arena a;
    a.st = st;
    double* Li;
    CTD_TRY(a.get(&Li, (size_t)n * n));
    CTD_TRY(tri_inverse(F->L, F->dyn->cap_d, n, Li, n, st));
    u_from_linv(Li, n, n, F->U, n, st);
    CTD_CUDA(cudaGetLastError());
    F->U_valid = true;
  }
  CTD_CUDA(cudaMemcpyAsync(U, F->U, (size_t)n * n * 8, cudaMemcpyDeviceToHost, st));
  return sync(st);
}

// Column (t, f) of C^(now): the step's exact block, then the rows each later
// step appends, M_{t'} times the column so far (Eq. C_t+1_final).
ctd_status dyn_C_columns(const ctd_factors* F, int64_t ncols, const int64_t* cols, double* out) {
  CTD_TRY(dyn_check_complete(F));
  const auto& D = *F->dyn;
  const int64_t h = F->s_kept;
  cudaStream_t st = F->stream;
  std::vector<std::vector<double>> Mh(D.steps.size());
  std::vector<int64_t> start(D.steps.size() + 1, 0);  // first column of each record
  for (size_t r = 0; r < D.steps.size(); ++r) start[r + 1] = start[r] + D.steps[r].ncols;
  for (int64_t c = 0; c < ncols; ++c) {
    if (cols[c] < 0 || cols[c] >= start.back()) return fail(CTD_EINVAL, "column out of range");
    const int64_t t =
        (int64_t)(std::upper_bound(start.begin(), start.end(), cols[c]) - start.begin()) - 1;
    const int64_t f = cols[c] - start[t];
    const StepRec& r = D.steps[t];
    std::vector<double> v(r.d_before + r.d_kept, 0.0);
    if (r.Coff) {
      uint64_t off = 0;
      uint32_t n = 0;
      CTD_TRY(d2h(&off, r.Coff + f, 1, st));
      CTD_TRY(d2h(&n, r.Ccnt + f, 1, st));
      CTD_TRY(sync(st));
      // a densely stored column holds every row's value (see C_DENSE)
      const bool dense = (n & C_DENSE) != 0;
      if (dense) n = (uint32_t)v.size();
      std::vector<uint16_t> rows(n);
      if (dense)
        for (uint32_t q = 0; q < n; ++q) rows[q] = (uint16_t)q;
      else
        CTD_TRY(d2h(rows.data(), r.Crow + off, n, st));
      if (F->precision == CTD_FP32_BULK) {
        std::vector<float> vals(n);
        CTD_TRY(d2h(vals.data(), static_cast<const float*>(r.Cval) + off, n, st));
        CTD_TRY(sync(st));
        for (uint32_t q = 0; q < n; ++q) v[rows[q]] = vals[q];
      } else {
        std::vector<double> vals(n);
        CTD_TRY(d2h(vals.data(), static_cast<const double*>(r.Cval) + off, n, st));
        CTD_TRY(sync(st));
        for (uint32_t q = 0; q < n; ++q) v[rows[q]] = vals[q];
      }
    } else if (r.d_before + r.d_kept > 0 && r.nnz > 0) {
      return fail(CTD_EINVAL, "this step's new columns were released (CTD_KEEP_LAST_C)");
    }
    for (int64_t t2 = t + 1; t2 < D.t; ++t2) {
      const StepRec& q = D.steps[t2];
      if (q.d_kept == 0) continue;
      if (q.d_before != (int64_t)v.size()) return fail(CTD_EINVAL, "inconsistent step record");
      std::vector<double>& Mq = Mh[t2];
      if (Mq.empty() && q.d_before > 0) {
        CTD_TRY(ensure_M(F, t2));
        Mq.resize((size_t)q.d_before * q.d_kept);
        CTD_TRY(d2h(Mq.data(), q.M, Mq.size(), st));
        CTD_TRY(sync(st));
      }
      const size_t base = v.size();
      v.resize(base + q.d_kept, 0.0);
      for (int64_t a = 0; a < q.d_kept; ++a) {
        double s = 0.0;
        for (int64_t b = 0; b < q.d_before; ++b) s += Mq[(size_t)a * q.d_before + b] * v[b];
        v[base + a] = s;
      }
    }
    if ((int64_t)v.size() != h) return fail(CTD_EINVAL, "inconsistent column height");
    std::copy(v.begin(), v.end(), out + c * h);
  }
  return CTD_OK;
}

ctd_status dyn_R(const ctd_factors* F, int64_t* colptr, int32_t* row, int32_t* val) {
  CTD_TRY(dyn_check_complete(F));
  const int64_t n = F->s_kept, nnz = F->nnz_R;
  std::vector<uint64_t> p(n + 1);
  std::vector<int32_t> r(nnz), v(nnz);
  CTD_TRY(d2h(p.data(), F->Rcolptr, n + 1, F->stream));
  CTD_TRY(d2h(r.data(), F->Rrow, nnz, F->stream));
  CTD_TRY(d2h(v.data(), F->Rval, nnz, F->stream));
  CTD_TRY(sync(F->stream));
  std::vector<int64_t> ord;
  for (int64_t c = 0; c < n; ++c) {
    const int64_t a = (int64_t)p[c], b = (int64_t)p[c + 1];
    ord.resize(b - a);
    std::iota(ord.begin(), ord.end(), a);
    std::sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return r[x] < r[y]; });
    for (int64_t q = a; q < b; ++q) {
      row[q] = r[ord[q - a]];
      val[q] = v[ord[q - a]];
    }
    colptr[c] = a;
  }
  colptr[n] = (int64_t)p[n];
  return CTD_OK;
}

}  // namespace ctd
