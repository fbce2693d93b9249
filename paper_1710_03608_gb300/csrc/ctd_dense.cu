// FP64 dense kernels for the independence filter and the middle factor U.
//
// Algorithm 1 lines 6-15 test each sampled fiber x_k, in order, against the
// span of the fibers kept so far: it is skipped iff ||res|| <= eps ||x_k||,
// res = x_k - R U R^T x_k.  With G = R'^T R' the Gram matrix of the
// candidates, ||res||^2 is the k-th diagonal entry of the Schur complement
// of G over the kept set, i.e. the pivot of a Cholesky factorization that
// only pivots on kept columns.  So the filter is an in-order Cholesky of G
// that skips a column whose pivot is <= eps^2 ||x_k||^2 (equality counts as
// dependent), and U = (R^T R)^{-1} = L^{-T} L^{-1} (Lemma 3.2, Colibri's
// Theorem 1).  In exact arithmetic this makes the same decisions and the
// same U as the sequential loop.
//
// The factorization is blocked by 32 columns: a one-warp kernel decides and
// factors the diagonal block in order, a row kernel forms the panel below
// it, and a tiled kernel applies the trailing update.  All arithmetic is
// FP64 on the CUDA cores.
#include "ctd_internal.cuh"

namespace ctd {

constexpr int NB = 32;

// ---------------------------------------------------------------------------
// generic FP64 GEMM: C = alpha op(A) op(B) + beta C (column-major)
// 64 x 64 tile, 16-deep k slices, 256 threads with 4 x 4 outputs each.
// `tri` = 1: only tiles on or below the diagonal of C, and k starts at the
// tile's first row/column block (for products of lower-triangular factors).
// ---------------------------------------------------------------------------
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256)
    k_dgemm(int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha,
            const double* __restrict__ A, int64_t lda, const double* __restrict__ B, int64_t ldb,
            double beta, double* __restrict__ C, int64_t ldc, int tri) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int64_t bm = (int64_t)blockIdx.x * GT, bn = (int64_t)blockIdx.y * GT;
  if (tri && bn > bm) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  const int64_t k0 = tri ? bm : 0;  // lower-triangular operand: terms need k >= max(row, col)
  for (int64_t kk = k0; kk < k; kk += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      const int r = e % GT, q = e / GT;
      const int64_t gr = bm + r, gq = kk + q;
      double av = 0.0;
      if (gr < m && gq < k) av = ta ? A[gq + gr * lda] : A[gr + gq * lda];
      As[q][r] = av;
      const int64_t gc = bn + r;
      double bv = 0.0;
      if (gc < n && gq < k) bv = tb ? B[gc + gq * ldb] : B[gq + gc * ldb];
      Bs[q][r] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = As[q][tx + 16 * u];
        b[u] = Bs[q][ty + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t r = bm + tx + 16 * u, c = bn + ty + 16 * v;
      if (r < m && c < n) {
        double* p = C + r + c * ldc;
        *p = alpha * acc[u][v] + (beta == 0.0 ? 0.0 : beta * *p);
      }
    }
}

void dgemm(bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
           int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
           cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  dim3 g((unsigned)((m + GT - 1) / GT), (unsigned)((n + GT - 1) / GT));
  CTD_LAUNCH(k_dgemm, (g), (256), 0, st, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0);
}

// Lower triangle (tile granularity) of C = Z^T Z for lower-triangular Z.
static void dgemm_tri_lower(const double* Z, int64_t n, int64_t ldz, double* C, int64_t ldc,
                            cudaStream_t st) {
  if (n <= 0) return;
  dim3 g((unsigned)((n + GT - 1) / GT), (unsigned)((n + GT - 1) / GT));
  CTD_LAUNCH(k_dgemm, (g), (256), 0, st, 1, 0, n, n, n, 1.0, Z, ldz, Z, ldz, 0.0, C, ldc, 1);
}

// ---------------------------------------------------------------------------
// Cholesky with skip
// ---------------------------------------------------------------------------
__global__ void k_chol_diag(double* __restrict__ A, int64_t n, int64_t lda, int64_t k0,
                            const double* __restrict__ thr, const int* __restrict__ force,
                            int* __restrict__ keep, double* __restrict__ piv,
                            unsigned* __restrict__ status) {
  __shared__ double D[NB][NB + 1];  // D[r][c], lower
  __shared__ int kp;
  __shared__ double inv;
  const int r = threadIdx.x;
  const int nb = (int)min((int64_t)NB, n - k0);
  if (r < nb)
    for (int c = 0; c <= r; ++c) D[r][c] = A[(k0 + r) + (k0 + c) * lda];
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    if (r == 0) {
      const double d = D[c][c];
      const int f = force ? force[k0 + c] : -1;
      int k = (d > thr[k0 + c] && d > 0.0) ? 1 : 0;
      if (f >= 0) k = f;
      if (k && !(d > 0.0)) {  // forced keep of a column with no positive pivot
        atomicOr(status, DEV_CAPACITY);
        k = 0;
      }
      kp = k;
      keep[k0 + c] = k;
      if (piv) piv[k0 + c] = d;
      const double l = k ? sqrt(d) : 0.0;
      D[c][c] = l;
      inv = k ? 1.0 / l : 0.0;
    }
    __syncthreads();
    if (r > c && r < nb) D[r][c] = kp ? D[r][c] * inv : 0.0;
    __syncthreads();
    if (kp && r > c && r < nb) {
      const double lrc = D[r][c];
      for (int j = c + 1; j <= r; ++j) D[r][j] = fma(-lrc, D[j][c], D[r][j]);
    }
    __syncthreads();
  }
  if (r < nb)
    for (int c = 0; c <= r; ++c) A[(k0 + r) + (k0 + c) * lda] = D[r][c];
}

// rows i >= k0 + nb: L21(i, :) = A21(i, :) L11^{-T} on kept columns
__global__ void k_chol_rows(double* __restrict__ A, int64_t n, int64_t lda, int64_t k0,
                            const int* __restrict__ keep) {
  __shared__ double L[NB][NB + 1];
  __shared__ int kp[NB];
  const int nb = (int)min((int64_t)NB, n - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    L[r][c] = (r < nb && c <= r) ? A[(k0 + r) + (k0 + c) * lda] : 0.0;
  }
  if (threadIdx.x < NB) kp[threadIdx.x] = threadIdx.x < nb ? keep[k0 + threadIdx.x] : 0;
  __syncthreads();
  const int64_t i = k0 + nb + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c) x[c] = c < nb ? A[i + (k0 + c) * lda] : 0.0;
#pragma unroll
  for (int c = 0; c < NB; ++c) {
    if (c < nb) {
      if (kp[c]) {
        double s = x[c];
#pragma unroll
        for (int j = 0; j < c; ++j) s -= x[j] * L[c][j];
        x[c] = s / L[c][c];
      } else {
        x[c] = 0.0;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NB; ++c)
    if (c < nb) A[i + (k0 + c) * lda] = x[c];
}

// trailing update of the lower triangle: A(r, c) -= sum_k L(r, k) L(c, k)
// over the panel columns, for r >= c >= k1.  One 32 x 32 tile per block.
__global__ void __launch_bounds__(256)
    k_chol_trailing(double* __restrict__ A, int64_t n, int64_t lda, int64_t k0, int nb) {
  __shared__ double Pr[NB][NB + 1];
  __shared__ double Pc[NB][NB + 1];
  const int64_t k1 = k0 + nb;
  const int64_t t = blockIdx.x;
  // tile (bi, bj) with bi >= bj from the linear index
  int64_t bi = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
  while (bi * (bi + 1) / 2 > t) --bi;
  const int64_t bj = t - bi * (bi + 1) / 2;
  const int64_t r0 = k1 + bi * NB, c0 = k1 + bj * NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int rr = e % NB, q = e / NB;
    Pr[rr][q] = (r0 + rr < n && q < nb) ? A[(r0 + rr) + (k0 + q) * lda] : 0.0;
    Pc[rr][q] = (c0 + rr < n && q < nb) ? A[(c0 + rr) + (k0 + q) * lda] : 0.0;
  }
  __syncthreads();
  const int rr = threadIdx.x & 31, cq = threadIdx.x >> 5;  // 8 column groups
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int cc = cq + 8 * v;
    const int64_t r = r0 + rr, c = c0 + cc;
    if (r < n && c < n && r >= c) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < NB; ++q) s = fma(Pr[rr][q], Pc[cc][q], s);
      A[r + c * lda] -= s;
    }
  }
}

void launch_chol_skip(double* A, int64_t n, int64_t lda, const double* thr, int* keep,
                      cudaStream_t st, const int* force, double* piv, unsigned* status) {
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int nb = (int)std::min<int64_t>(NB, n - k0);
    CTD_LAUNCH(k_chol_diag, (1), (NB), 0, st, A, n, lda, k0, thr, force, keep, piv, status);
    const int64_t rest = n - k0 - nb;
    if (rest > 0) {
      CTD_LAUNCH(k_chol_rows, ((unsigned)((rest + 127) / 128)), (128), 0, st, A, n, lda, k0, keep);
      const int64_t tb = (rest + NB - 1) / NB;
      CTD_LAUNCH(k_chol_trailing, ((unsigned)(tb * (tb + 1) / 2)), (256), 0, st, A, n, lda, k0,
                 nb);
    }
  }
}

// ---------------------------------------------------------------------------
// kept-set compaction and gathers
// ---------------------------------------------------------------------------
__global__ void k_compact_flags(const int* __restrict__ keep, int n, int* __restrict__ idx,
                                int* count) {
  __shared__ int wsum[32];
  __shared__ int base_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += blockDim.x) {
    const int e = c0 + threadIdx.x;
    const int flag = (e < n) ? (keep[e] != 0) : 0;
    const unsigned ball = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) wsum[warp] = __popc(ball);
    __syncthreads();
    int before = base_s, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) before += wsum[w];
      total += wsum[w];
    }
    if (flag) idx[before + __popc(ball & ((1u << lane) - 1))] = e;
    __syncthreads();
    if (threadIdx.x == 0) base_s += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = base_s;
}

void launch_compact_flags(const int* keep, int n, int* idx, int* count, cudaStream_t st) {
  CTD_LAUNCH(k_compact_flags, (1), (1024), 0, st, keep, n, idx, count);
}

__global__ void k_gather_lower(const double* __restrict__ A, int64_t lda, const int* __restrict__ idx,
                               const int* count_dev, int nk_max, double* __restrict__ B,
                               int64_t ldb) {
  const int nk = min(*count_dev, nk_max);
  const int64_t total = (int64_t)nk * nk;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % nk), c = (int)(e / nk);
    B[r + c * ldb] = (r >= c) ? A[idx[r] + (int64_t)idx[c] * lda] : 0.0;
  }
}

void launch_gather_lower(const double* A, int64_t lda, const int* idx, const int* count_dev,
                         int nk_max, double* B, int64_t ldb, cudaStream_t st) {
  if (nk_max <= 0) return;
  CTD_LAUNCH(k_gather_lower, (grid_for((int64_t)nk_max * nk_max, 256, (int64_t)num_sms() * 8)), (256), 0, st, 
      A, lda, idx, count_dev, nk_max, B, ldb);
}

// ---------------------------------------------------------------------------
// Z = L^{-1} (blocked by 32)
// ---------------------------------------------------------------------------
__global__ void k_trinv_diag(const double* __restrict__ L, int64_t ldl, int64_t n,
                             double* __restrict__ Z, int64_t ldz) {
  __shared__ double Lb[NB][NB + 1];
  __shared__ double Zb[NB][NB + 1];
  const int64_t b0 = (int64_t)blockIdx.x * NB;
  const int nb = (int)min((int64_t)NB, n - b0);
  const int j = threadIdx.x;
  for (int r = 0; r < NB; ++r) {
    Lb[r][j] = (r < nb && j < nb && j <= r) ? L[(b0 + r) + (b0 + j) * ldl] : 0.0;
    Zb[r][j] = 0.0;
  }
  __syncthreads();
  if (j < nb) {
    Zb[j][j] = 1.0 / Lb[j][j];
    for (int i = j + 1; i < nb; ++i) {
      double s = 0.0;
      for (int q = j; q < i; ++q) s = fma(Lb[i][q], Zb[q][j], s);
      Zb[i][j] = -s / Lb[i][i];
    }
  }
  __syncthreads();
  for (int r = 0; r < nb; ++r)
    if (j < nb) Z[(b0 + r) + (b0 + j) * ldz] = Zb[r][j];
}

// block row I: Z[I, J] = -Z[I, I] * sum_{K=J}^{I-1} L[I, K] Z[K, J], one block per J
__global__ void __launch_bounds__(256)
    k_trinv_row(const double* __restrict__ L, int64_t ldl, int64_t n, double* __restrict__ Z,
                int64_t ldz, int64_t bI) {
  __shared__ double Ls[NB][NB + 1];
  __shared__ double Zs[NB][NB + 1];
  __shared__ double Ts[NB][NB + 1];
  const int64_t bJ = blockIdx.x;
  const int64_t r0 = bI * NB;
  const int rr = threadIdx.x & 31, cq = threadIdx.x >> 5;
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t bK = bJ; bK < bI; ++bK) {
    for (int e = threadIdx.x; e < NB * NB; e += 256) {
      const int a = e % NB, b = e / NB;
      const int64_t lr = r0 + a, lc = bK * NB + b;
      Ls[a][b] = (lr < n && lc < n) ? L[lr + lc * ldl] : 0.0;
      const int64_t zr = bK * NB + a, zc = bJ * NB + b;
      Zs[a][b] = (zr < n && zc < n) ? Z[zr + zc * ldz] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int cc = cq + 8 * v;
      double s = t[v];
#pragma unroll
      for (int q = 0; q < NB; ++q) s = fma(Ls[rr][q], Zs[q][cc], s);
      t[v] = s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) Ts[rr][cq + 8 * v] = t[v];
  // diagonal block of Z
  for (int e = threadIdx.x; e < NB * NB; e += 256) {
    const int a = e % NB, b = e / NB;
    const int64_t zr = r0 + a, zc = r0 + b;
    Zs[a][b] = (zr < n && zc < n) ? Z[zr + zc * ldz] : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int cc = cq + 8 * v;
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < NB; ++q) s = fma(Zs[rr][q], Ts[q][cc], s);
    const int64_t zr = r0 + rr, zc = bJ * NB + cc;
    if (zr < n && zc < n) Z[zr + zc * ldz] = -s;
  }
}

void tri_inverse(const double* L, int64_t ldl, int64_t n, double* Z, int64_t ldz,
                 cudaStream_t st) {
  if (n <= 0) return;
  const int64_t nbk = (n + NB - 1) / NB;
  launch_zero_f64(Z, n, n, ldz, st);
  CTD_LAUNCH(k_trinv_diag, ((unsigned)nbk), (NB), 0, st, L, ldl, n, Z, ldz);
  for (int64_t bI = 1; bI < nbk; ++bI)
    CTD_LAUNCH(k_trinv_row, ((unsigned)bI), (256), 0, st, L, ldl, n, Z, ldz, bI);
}

// U = Z^T Z for Z = L^{-1}: lower tiles then mirror.
void u_from_linv(const double* Z, int64_t n, int64_t ldz, double* U, int64_t ldu,
                 cudaStream_t st) {
  dgemm_tri_lower(Z, n, ldz, U, ldu, st);
  launch_symmetrize(U, n, ldu, st);
}

// ---------------------------------------------------------------------------
// B <- L^{-1} B for lower-triangular L (n x n) and nrhs right-hand sides,
// by blocked forward substitution: each 32-row diagonal block is solved by
// substitution (one thread per right-hand side), then the rows below are
// updated with a GEMM.  Substitution keeps the solve backward stable, which
// the independence test needs: pivots ||x||^2 - ||L^{-1} R^T x||^2 then carry
// errors of order n u ||x||^2, not kappa(L) u ||x||^2.
// ---------------------------------------------------------------------------
__global__ void k_trsm_diag(const double* __restrict__ L, int64_t ldl, int64_t n, int64_t k0,
                            double* __restrict__ B, int64_t ldb, int64_t nrhs) {
  __shared__ double Ls[NB][NB + 1];
  const int nb = (int)min((int64_t)NB, n - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    Ls[r][c] = (r < nb && c <= r) ? L[(k0 + r) + (k0 + c) * ldl] : 0.0;
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs) return;
  double x[NB];
  double* col = B + j * ldb + k0;
#pragma unroll
  for (int r = 0; r < NB; ++r) x[r] = r < nb ? col[r] : 0.0;
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    if (r < nb) {
      double s = x[r];
#pragma unroll
      for (int c = 0; c < r; ++c) s = fma(-Ls[r][c], x[c], s);
      x[r] = s / Ls[r][r];
    }
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < nb) col[r] = x[r];
}

void tri_solve_lower(const double* L, int64_t ldl, int64_t n, double* B, int64_t ldb, int64_t nrhs,
                     cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int64_t nb = std::min<int64_t>(NB, n - k0);
    CTD_LAUNCH(k_trsm_diag, ((unsigned)((nrhs + 127) / 128)), (128), 0, st, L, ldl, n, k0, B, ldb,
               nrhs);
    const int64_t rest = n - k0 - nb;
    if (rest > 0)
      dgemm(false, false, rest, nrhs, nb, -1.0, L + (k0 + nb) + k0 * ldl, ldl, B + k0, ldb, 1.0,
            B + k0 + nb, ldb, st);
  }
}

// B <- L^{-T} B (backward substitution with the transpose of lower L).
__global__ void k_trsm_diag_T(const double* __restrict__ L, int64_t ldl, int64_t n, int64_t k0,
                              double* __restrict__ B, int64_t ldb, int64_t nrhs) {
  __shared__ double Ls[NB][NB + 1];
  const int nb = (int)min((int64_t)NB, n - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    Ls[r][c] = (r < nb && c <= r) ? L[(k0 + r) + (k0 + c) * ldl] : 0.0;
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nrhs) return;
  double x[NB];
  double* col = B + j * ldb + k0;
#pragma unroll
  for (int r = 0; r < NB; ++r) x[r] = r < nb ? col[r] : 0.0;
#pragma unroll
  for (int r = NB - 1; r >= 0; --r) {
    if (r < nb) {
      double s = x[r];
#pragma unroll
      for (int c = r + 1; c < NB; ++c)
        if (c < nb) s = fma(-Ls[c][r], x[c], s);
      x[r] = s / Ls[r][r];
    }
  }
#pragma unroll
  for (int r = 0; r < NB; ++r)
    if (r < nb) col[r] = x[r];
}

void tri_solve_lower_T(const double* L, int64_t ldl, int64_t n, double* B, int64_t ldb,
                       int64_t nrhs, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return;
  const int64_t last = ((n - 1) / NB) * NB;
  for (int64_t k0 = last; k0 >= 0; k0 -= NB) {
    const int64_t nb = std::min<int64_t>(NB, n - k0);
    CTD_LAUNCH(k_trsm_diag_T, ((unsigned)((nrhs + 127) / 128)), (128), 0, st, L, ldl, n, k0, B,
               ldb, nrhs);
    if (k0 > 0)  // B[0:k0] -= L[k0:k0+nb, 0:k0]^T B[k0:k0+nb]
      dgemm(true, false, k0, nrhs, nb, -1.0, L + k0, ldl, B + k0, ldb, 1.0, B, ldb, st);
  }
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__global__ void k_zero_f64(double* A, int64_t m, int64_t n, int64_t lda) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    A[(e % m) + (e / m) * lda] = 0.0;
}

void launch_zero_f64(double* A, int64_t m, int64_t n, int64_t lda, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  CTD_LAUNCH(k_zero_f64, (grid_for(m * n, 256, (int64_t)num_sms() * 8)), (256), 0, st, A, m, n, lda);
}

// mirror the lower triangle into the upper one; tiles strictly above the
// diagonal were never written by the tile-lower GEMM
__global__ void k_symmetrize(double* A, int64_t n, int64_t lda) {
  const int64_t total = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % n, c = e / n;
    if (r < c) A[r + c * lda] = A[c + r * lda];
  }
}

void launch_symmetrize(double* A, int64_t n, int64_t lda, cudaStream_t st) {
  if (n <= 1) return;
  CTD_LAUNCH(k_symmetrize, (grid_for(n * n, 256, (int64_t)num_sms() * 8)), (256), 0, st, A, n, lda);
}

__global__ void k_thresholds(const double* D, int64_t n, int64_t ldd, double eps2, double* thr) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    thr[e] = eps2 * D[e * (ldd + 1)];
}

void launch_thresholds(const double* D, int64_t n, int64_t ldd, double eps2, double* thr,
                       cudaStream_t st) {
  if (n <= 0) return;
  CTD_LAUNCH(k_thresholds, (grid_for(n, 256, 1024)), (256), 0, st, D, n, ldd, eps2, thr);
}

}  // namespace ctd
