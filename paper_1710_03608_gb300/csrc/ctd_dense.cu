// FP64 dense kernels for the independence filter and the middle factor U.
//
// Algorithm 1's independence test takes each sampled fiber x_k, in order, against the
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
// The factorization is one cooperative launch (a block per SM), blocked by
// 32 columns: four warps of block 0 (one per SM sub-partition) decide and
// factor each diagonal block in order, in registers, as soon as its update
// by the previous panel is done (lookahead): that update is split by rows
// over four blocks, which signal block 0 through a counter (a bounded
// wait), while the other blocks apply the rest of the trailing update in
// 32 x 32 tiles; the blocks then solve the next panel's rows.  Two bounded
// grid barriers per panel.  All arithmetic is FP64 on the CUDA cores.
#include "ctd_internal.cuh"

namespace ctd {

constexpr int NB = 32;
constexpr int TQ = 4;  // blocks that share the update of the next diagonal block

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

// 32 x 32 tile, 256 threads with 2 x 2 outputs each; blockIdx.z splits k
// into chunks of kchunk.  With splits > 1 each split writes its partial
// product to part + z * m * n (column-major, ld m) and k_splitk_reduce adds
// them in split order (deterministic).
constexpr int GS = 32;

__global__ void __launch_bounds__(256)
    k_dgemm32(int ta, int tb, int64_t m, int64_t n, int64_t k, double alpha,
              const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
              int64_t ldb, double beta, double* __restrict__ C, int64_t ldc, int tri,
              int64_t kchunk, double* __restrict__ part) {
  __shared__ double As[GK][GS + 1];
  __shared__ double Bs[GK][GS + 1];
  const int64_t bm = (int64_t)blockIdx.x * GS, bn = (int64_t)blockIdx.y * GS;
  if (tri && bn > bm) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {};
  int64_t kb = (int64_t)blockIdx.z * kchunk, ke = min(k, kb + kchunk);
  if (tri) kb = max(kb, bm);  // lower-triangular operand: terms need k >= max(row, col)
  for (int64_t kk = kb; kk < ke; kk += GK) {
    for (int e = threadIdx.x; e < GS * GK; e += 256) {
      const int r = e % GS, q = e / GS;
      const int64_t gr = bm + r, gq = kk + q;
      double av = 0.0;
      if (gr < m && gq < ke) av = ta ? A[gq + gr * lda] : A[gr + gq * lda];
      As[q][r] = av;
      const int64_t gc = bn + r;
      double bv = 0.0;
      if (gc < n && gq < ke) bv = tb ? B[gc + gq * ldb] : B[gq + gc * ldb];
      Bs[q][r] = bv;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GK; ++q) {
      const double a0 = As[q][tx], a1 = As[q][tx + 16];
      const double b0 = Bs[q][ty], b1 = Bs[q][ty + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int64_t r = bm + tx + 16 * u, c = bn + ty + 16 * v;
      if (r < m && c < n) {
        if (part) {
          part[(int64_t)blockIdx.z * m * n + r + c * m] = acc[u][v];
        } else {
          double* p = C + r + c * ldc;
          *p = alpha * acc[u][v] + (beta == 0.0 ? 0.0 : beta * *p);
        }
      }
    }
}

__global__ void k_splitk_reduce(const double* __restrict__ part, int splits, int64_t m, int64_t n,
                                double alpha, double beta, double* __restrict__ C, int64_t ldc,
                                int tri) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % m, c = e / m;
    if (tri && (c / GS) > (r / GS)) continue;
    double s = 0.0;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * total + e];
    double* p = C + r + c * ldc;
    *p = alpha * s + (beta == 0.0 ? 0.0 : beta * *p);
  }
}

static void dgemm_impl(bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha,
                       const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                       double* C, int64_t ldc, int tri, cudaStream_t st) {
  if (m <= 0 || n <= 0) return;
  const int64_t sms = num_sms();
  const int64_t t64 = ((m + GT - 1) / GT) * ((n + GT - 1) / GT);
  if (!tri && t64 >= 2 * sms) {
    dim3 g((unsigned)((m + GT - 1) / GT), (unsigned)((n + GT - 1) / GT));
    CTD_LAUNCH(k_dgemm, (g), (256), 0, st, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
               0);
    return;
  }
  const int64_t t32 = ((m + GS - 1) / GS) * ((n + GS - 1) / GS) / (tri ? 2 : 1) + 1;
  // split k so that about four blocks per SM have work, in chunks of >= 64
  int64_t splits = std::max<int64_t>(1, (4 * sms) / std::max<int64_t>(t32, 1));
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, k / 64));
  splits = std::min<int64_t>(splits, 16);
  int64_t kchunk = (k + splits - 1) / splits;
  kchunk = ((kchunk + GK - 1) / GK) * GK;
  splits = std::max<int64_t>(1, (k + kchunk - 1) / std::max<int64_t>(kchunk, 1));
  dim3 g((unsigned)((m + GS - 1) / GS), (unsigned)((n + GS - 1) / GS), (unsigned)splits);
  double* part = nullptr;
  if (splits > 1 && dalloc_n(&part, (size_t)splits * m * n, st) != CTD_OK) {
    part = nullptr;
    splits = 1;
    kchunk = std::max<int64_t>(k, 1);
    g.z = 1;
  }
  CTD_LAUNCH(k_dgemm32, (g), (256), 0, st, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
             tri, std::max<int64_t>(kchunk, 1), splits > 1 ? part : nullptr);
  if (splits > 1) {
    CTD_LAUNCH(k_splitk_reduce, (grid_for(m * n, 256, sms * 8)), (256), 0, st, part, (int)splits,
               m, n, alpha, beta, C, ldc, tri);
    dfree(part, st);
  }
}

void dgemm(bool ta, bool tb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
           int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
           cudaStream_t st) {
  dgemm_impl(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, 0, st);
}

// Lower tiles of C = Z^T Z for lower-triangular Z.
static void dgemm_tri_lower(const double* Z, int64_t n, int64_t ldz, double* C, int64_t ldc,
                            cudaStream_t st) {
  dgemm_impl(true, false, n, n, n, 1.0, Z, ldz, Z, ldz, 0.0, C, ldc, 1, st);
}

// ---------------------------------------------------------------------------
// Cholesky with skip
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// The whole skip-Cholesky in one cooperative launch (one block per SM): per
// 32-column panel, block 0 factors the diagonal block (in order, with the
// keep/skip decisions), every block then forms its share of the panel rows
// below and of the trailing update, separated by grid barriers.  The grid
// barrier spins a bounded number of times; if it gives up it records
// DEV_TIMEOUT and every block leaves, so the host reports CTD_ETIMEOUT.
// ---------------------------------------------------------------------------
constexpr long long BARRIER_SPIN_LIMIT = 1ll << 26;  // ~2 s of 32 ns naps

struct GridBar {
  unsigned* count;
  unsigned* gen;
  unsigned* status;
};

// returns false if the barrier timed out (or an earlier one did)
// Wait until *vgen differs from g, at most `limit` naps of ~32 ns; on giving
// up (or when another waiter already did) set DEV_TIMEOUT and return false.
__device__ bool bounded_wait_change(volatile unsigned* vgen, unsigned g, unsigned* status,
                                    long long limit) {
  volatile unsigned* vstat = status;
  long long spins = 0;
  while (*vgen == g) {
    if ((*vstat & DEV_TIMEOUT) || ++spins > limit) {
      atomicOr(status, DEV_TIMEOUT);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

__device__ bool grid_sync(const GridBar& gb) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = gb.gen;
    const unsigned g = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(gb.count, 1u);
    if (arrived == gridDim.x - 1) {
      *gb.count = 0;
      __threadfence();
      atomicAdd(gb.gen, 1u);
    } else if (!bounded_wait_change(vgen, g, gb.status, BARRIER_SPIN_LIMIT)) {
      ok = 0;
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// 1 / sqrt(d) for d > 0: an FP32 estimate y (relative error e0 below
// 2^-21) refined by one third-order step of the series
// (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + ..., with e = 1 - d y^2:
// y <- y (1 + e/2 + 3e^2/8), whose truncation error is about (5/16) e^3,
// far below FP64 rounding; four dependent FP64 operations against six for
// two Newton-Raphson steps.  Outside FP32's comfortable range the exact
// FP64 sqrt and division.  On GB300 a dependent FP64 operation costs over
// a hundred cycles on a narrow pipe, and the diagonal-block factorization
// takes one inverse square root per column in sequence.
__device__ __forceinline__ double rsqrt_fp64(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  // the FP32 estimate without FP64 <-> FP32 conversions (which would run on
  // the FP64 pipe): d's exponent rebiased and its mantissa truncated to 23
  // bits (relative error below 2^-23), and the estimate widened back
  // exactly, by integer operations on the bit patterns
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned fb = ((unsigned)(((b >> 52) & 0x7FF) - 1023 + 127) << 23) |
                      (unsigned)((b >> 29) & 0x7FFFFF);
  const unsigned yb = __float_as_uint(rsqrtf(__uint_as_float(fb)));
  const double y = __longlong_as_double(
      (long long)((((unsigned long long)((yb >> 23) & 0xFF) - 127 + 1023) << 52) |
                  ((unsigned long long)(yb & 0x7FFFFF) << 29)));
  const double t = d * y;
  const double e = fma(-t, y, 1.0);     // 1 - d y^2
  const double c = fma(e, 0.375, 0.5);  // 1/2 + 3e/8
  return fma(y * e, c, y);              // y (1 + e/2 + 3e^2/8)
}

// The diagonal block at k0, in order, by warp 0 of the calling block: lane r
// holds row r in registers; column c is finished left-looking (its entries
// reduced by the earlier columns, row c's values broadcast by shuffles),
// then decided and scaled.  No block barriers inside except the first.
struct CholShared {
  double D[NB][NB + 1];
  double Pc[NB][NB + 1];
  double invd[NB];
  int kp[NB];
  double thr_s[NB], piv_s[NB];
  int force_s[NB];
  double fpiv_s[NB];
  double colc[2][NB];  // the column just finished (double-buffered)
  int okq;             // block 0: the parts of the next diagonal block arrived
};

__device__ void chol_diag_block(double* __restrict__ A, int64_t n, int64_t lda, int64_t k0,
                                const double* __restrict__ thr, const int* __restrict__ force,
                                const double* __restrict__ fpiv, int* __restrict__ keep,
                                double* __restrict__ piv, unsigned* __restrict__ status,
                                CholShared& sh) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (int)min((int64_t)NB, n - k0);
  double* thr_s = sh.thr_s;
  int* force_s = sh.force_s;
  double* fpiv_s = sh.fpiv_s;
  int* kp = sh.kp;
  double* piv_s = sh.piv_s;
  if (tid < nb) {
    thr_s[tid] = thr[k0 + tid];
    force_s[tid] = force ? force[k0 + tid] : -1;
    fpiv_s[tid] = fpiv ? fpiv[k0 + tid] : 0.0;
  }
  __syncthreads();
  // Four warps, one per SM sub-partition (GB300's FP64 unit is narrow: a
  // warp-wide FP64 instruction occupies a sub-partition for ~64 cycles, so
  // one warp alone was the bottleneck).  Warp w holds columns j = 4 t + w,
  // lane r row r.  Column c's owner decides and scales it and publishes it
  // in shared memory; after a named barrier of the four warps every warp
  // updates its later columns (right-looking).
  constexpr int CW = 4, TPW = NB / CW;
  if (warp < CW) {
    double rowj[TPW];
#pragma unroll
    for (int t = 0; t < TPW; ++t) {
      const int j = CW * t + warp;
      rowj[t] = (lane < nb && j <= lane) ? A[(k0 + lane) + (k0 + j) * lda] : 0.0;
    }
#pragma unroll
    for (int c = 0; c < NB; ++c) {
      if (c < nb) {
        const int owner = c % CW, tc = c / CW;
        double* colc = sh.colc[c & 1];
        if (warp == owner) {
          double d = __shfl_sync(0xffffffffu, rowj[tc], c);
          int k = (d > thr_s[c] && d > 0.0) ? 1 : 0;
          if (force_s[c] >= 0) k = force_s[c];
          // a keep forced by the explicit residual takes that residual's
          // squared norm as its pivot (the Gram-based one lost it to rounding)
          if (force_s[c] == 1 && fpiv_s[c] > 0.0) d = fpiv_s[c];
          if (k && !(d > 0.0)) {
            if (lane == 0) atomicOr(status, DEV_CAPACITY);
            k = 0;
          }
          const double inv = k ? rsqrt_fp64(d) : 0.0;
          double v = 0.0;
          if (lane == c)
            v = k ? d * inv : 0.0;
          else if (lane > c)
            v = rowj[tc] * inv;
          rowj[tc] = v;
          colc[lane] = v;
          if (lane == 0) {
            kp[c] = k;
            piv_s[c] = d;
          }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(CW * 32));
        if (kp[c]) {
          const double lr = colc[lane];
#pragma unroll
          for (int t = 0; t < TPW; ++t) {
            const int j = CW * t + warp;
            if (j > c && lane >= j) rowj[t] = fma(-lr, colc[j], rowj[t]);
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < TPW; ++t) {
      const int j = CW * t + warp;
      if (lane < nb && j <= lane) A[(k0 + lane) + (k0 + j) * lda] = rowj[t];
    }
    asm volatile("bar.sync 1, %0;" ::"n"(CW * 32));
    if (warp == 0 && lane < nb) {
      keep[k0 + lane] = kp[lane];
      if (piv) piv[k0 + lane] = piv_s[lane];
    }
  }
  __threadfence();
}

__global__ void __launch_bounds__(256, 1)
    k_chol_coop(double* __restrict__ A, int64_t n, int64_t lda, const double* __restrict__ thr,
                const int* __restrict__ force, const double* __restrict__ fpiv,
                int* __restrict__ keep, double* __restrict__ piv,
                unsigned* __restrict__ status, GridBar gb) {
  __shared__ CholShared sh;
  double(*D)[NB + 1] = sh.D;
  double(*Pc)[NB + 1] = sh.Pc;
  double* invd = sh.invd;
  int* kp = sh.kp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned* handoff = status + 3;  // parts of the next diagonal block done
  int panels = 0;
  // the first diagonal block; every later one is factored by block 0 right
  // after its own trailing tile (tile 0 of the previous panel, which is that
  // diagonal block), overlapping the other blocks' trailing updates
  if (blockIdx.x == 0) chol_diag_block(A, n, lda, 0, thr, force, fpiv, keep, piv, status, sh);
  if (!grid_sync(gb)) return;
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int nb = (int)min((int64_t)NB, n - k0);
    const int64_t k1 = k0 + nb;
    const int64_t rest = n - k1;
    if (rest <= 0) break;
    // --- B: panel rows, L21(i, :) = A21(i, :) L11^{-T} on kept columns.
    // One warp per row: lane c holds column c's value; each step's dot
    // product over earlier columns is a warp reduction.
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      const int r = e % NB, c = e / NB;
      D[r][c] = (r < nb && c <= r) ? A[(k0 + r) + (k0 + c) * lda] : 0.0;
    }
    __syncthreads();  // D's diagonal is read below by other threads than wrote it
    if (tid < NB) {
      kp[tid] = tid < nb ? keep[k0 + tid] : 0;
      invd[tid] = (tid < nb && kp[tid]) ? 1.0 / D[tid][tid] : 0.0;
    }
    __syncthreads();
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = k1 + gw; i < n; i += nwarps) {
      // x L11^T = a, right-looking: x_c = a_c / L(c, c) is broadcast and
      // the lanes after c subtract their share at once
      double x = lane < nb ? A[i + (k0 + lane) * lda] : 0.0;
      for (int c = 0; c < nb; ++c) {
        const double xc = __shfl_sync(0xffffffffu, x * invd[c], c);
        if (lane == c)
          x = kp[c] ? xc : 0.0;
        else if (lane > c && kp[c])
          x = fma(-xc, D[lane][c], x);
      }
      if (lane < nb) A[i + (k0 + lane) * lda] = x;
    }
    __threadfence();
    if (!grid_sync(gb)) return;
    // --- C: trailing update of the lower triangle, 32 x 32 tiles.  Tile 0,
    // the next diagonal block (which the next panel's factorization waits
    // for), is split by rows over the first TQ blocks; block 0 then waits
    // (bounded) for the other parts and factors it while the other blocks
    // take the remaining tiles.  Every entry is the same fma sequence as in
    // a whole-tile update.
    const int64_t tb = (rest + NB - 1) / NB;
    const int64_t ntiles = tb * (tb + 1) / 2;
    const int tq = (int)min((int64_t)TQ, (int64_t)gridDim.x);
    if ((int)blockIdx.x < tq) {
      constexpr int QR = NB / TQ;  // rows of a part
      for (int qq = blockIdx.x; qq < TQ; qq += tq) {
        const int64_t ra = k1 + (int64_t)qq * QR;
        __syncthreads();
        for (int e = tid; e < NB * NB; e += blockDim.x) {
          const int rr = e % NB, q = e / NB;
          if (rr < QR) D[rr][q] = (ra + rr < n && q < nb) ? A[(ra + rr) + (k0 + q) * lda] : 0.0;
          Pc[rr][q] = (k1 + rr < n && q < nb) ? A[(k1 + rr) + (k0 + q) * lda] : 0.0;
        }
        __syncthreads();
        const int rr = tid % QR, cc = tid / QR;
        const int64_t r = ra + rr, c = k1 + cc;
        if (cc < NB && r < n && c < n && r >= c) {
          double s2 = 0.0;
#pragma unroll
          for (int q = 0; q < NB; ++q) s2 = fma(D[rr][q], Pc[cc][q], s2);
          A[r + c * lda] -= s2;
        }
      }
      if (blockIdx.x != 0) {
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          atomicAdd(handoff, (unsigned)((TQ - 1 - (int)blockIdx.x) / tq + 1));
        }
      }
    }
    const int first = gridDim.x > 1 ? 1 : 0;  // block 0 goes on to the diagonal block
    for (int64_t t = 1 + (int64_t)blockIdx.x - first; (int)blockIdx.x >= first && t < ntiles;
         t += (int64_t)gridDim.x - first) {
      int64_t bi = (int64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
      while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
      while (bi * (bi + 1) / 2 > t) --bi;
      const int64_t bj = t - bi * (bi + 1) / 2;
      const int64_t r0 = k1 + bi * NB, c0 = k1 + bj * NB;
      __syncthreads();
      for (int e = tid; e < NB * NB; e += blockDim.x) {
        const int rr = e % NB, q = e / NB;
        D[rr][q] = (r0 + rr < n && q < nb) ? A[(r0 + rr) + (k0 + q) * lda] : 0.0;
        Pc[rr][q] = (c0 + rr < n && q < nb) ? A[(c0 + rr) + (k0 + q) * lda] : 0.0;
      }
      __syncthreads();
      const int rr = tid & 31, cq = tid >> 5;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int cc = cq + 8 * v;
        const int64_t r = r0 + rr, c = c0 + cc;
        if (r < n && c < n && r >= c) {
          double s2 = 0.0;
#pragma unroll
          for (int q = 0; q < NB; ++q) s2 = fma(D[rr][q], Pc[cc][q], s2);
          A[r + c * lda] -= s2;
        }
      }
    }
    if (blockIdx.x == 0) {
      // the other parts of tile 0: a counter the part blocks raise, bounded wait
      ++panels;
      __syncthreads();
      if (tid == 0) {
        sh.okq = 1;
        const unsigned others = (unsigned)(TQ - (TQ + tq - 1) / tq);
        const unsigned target = others * (unsigned)panels;
        volatile unsigned* vh = handoff;
        volatile unsigned* vstat = status;
        long long spins = 0;
        while (*vh < target) {
          if ((*vstat & DEV_TIMEOUT) || ++spins > BARRIER_SPIN_LIMIT) {
            atomicOr(status, DEV_TIMEOUT);
            sh.okq = 0;
            break;
          }
          __nanosleep(32);
        }
        __threadfence();
      }
      __syncthreads();
      if (!sh.okq) return;
      chol_diag_block(A, n, lda, k1, thr, force, fpiv, keep, piv, status, sh);
    }
    __threadfence();
    if (!grid_sync(gb)) return;
  }
}

ctd_status launch_chol_skip(double* A, int64_t n, int64_t lda, const double* thr, int* keep,
                            cudaStream_t st, const int* force, double* piv, unsigned* status,
                            const double* fpiv) {
  if (n <= 0) return CTD_OK;
  // barrier words live in the status array's tail: status[1] count, status[2]
  // generation, status[3] the parts of each next diagonal block done
  GridBar gb{status + 1, status + 2, status};
  CTD_CUDA(cudaMemsetAsync(status + 1, 0, 3 * sizeof(unsigned), st));
  int per_sm = 0;
  CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chol_coop, 256, 0));
  if (per_sm <= 0) return fail(CTD_ECUDA, "the skip-Cholesky kernel cannot be resident");
  // one block per SM: measured on the 10^7-nonzero tensor (s' = 498), 152
  // blocks took 0.81 ms, 304 (two per SM) 0.97, 76 0.85, 38 0.97, 19 1.22
  const int nblocks = num_sms();
  void* args[] = {&A, &n, &lda, const_cast<double**>(&thr), const_cast<int**>(&force),
                  const_cast<double**>(&fpiv), &keep, &piv, &status, &gb};
  note_launch();
  // a failed cooperative launch leaves keep/piv unwritten: report it before
  // anything reads them
  CTD_CUDA(cudaLaunchCooperativeKernel((const void*)k_chol_coop, dim3(nblocks), dim3(256), args,
                                       0, st));
  return CTD_OK;
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

// U = Z^T Z for Z = L^{-1}: lower tiles then mirror.
void u_from_linv(const double* Z, int64_t n, int64_t ldz, double* U, int64_t ldu,
                 cudaStream_t st) {
  dgemm_tri_lower(Z, n, ldz, U, ldu, st);
  launch_symmetrize(U, n, ldu, st);
}

// ---------------------------------------------------------------------------
// Triangular solves.  Substitution keeps them backward stable, which the
// independence test needs: pivots ||x||^2 - ||L^{-1} R^T x||^2 then carry
// errors of order n u ||x||^2, not kappa(L) u ||x||^2.
// ---------------------------------------------------------------------------
// Z = L^{-1} in one launch: a block per column j of Z solves L z = e_j by
// blocked forward substitution from row j down (z is zero above row j), the
// column held in shared memory.  Warp 0 substitutes through each 32-row
// diagonal block (right-looking; lane r holds z_r, the reciprocal diagonal
// formed once per block), then every thread updates rows below with that
// block's 32 values in a fixed order.  Forward substitution keeps the
// inverse backward stable.  (Per-block substitution and GEMM launches took
// 29 latency-bound launches for n = 456.)
constexpr int TI_THREADS = 256;

__global__ void __launch_bounds__(TI_THREADS)
    k_tri_inv_cols(const double* __restrict__ L, int64_t ldl, int n, double* __restrict__ Z,
                   int64_t ldz) {
  extern __shared__ double zs[];  // [n]
  __shared__ double Ls[NB][NB + 1];  // the current diagonal block
  const int j = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int r = tid; r < n; r += TI_THREADS) zs[r] = r == j ? 1.0 : 0.0;
  for (int k0 = (j / NB) * NB; k0 < n; k0 += NB) {
    const int nb = min(NB, n - k0);
    for (int e = tid; e < NB * NB; e += TI_THREADS) {
      const int r = e % NB, c = e / NB;
      Ls[r][c] = (r < nb && c <= r) ? L[(k0 + r) + (int64_t)(k0 + c) * ldl] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
      double x = lane < nb ? zs[k0 + lane] : 0.0;
      const double rinv = lane < nb ? 1.0 / Ls[lane][lane] : 0.0;
      for (int c = 0; c < nb; ++c) {
        const double xc = __shfl_sync(0xffffffffu, x * rinv, c);
        if (lane == c)
          x = xc;
        else if (lane > c && lane < nb)
          x = fma(-Ls[lane][c], xc, x);
      }
      if (lane < nb) zs[k0 + lane] = x;
    }
    __syncthreads();
    for (int r = k0 + nb + tid; r < n; r += TI_THREADS) {
      double acc = zs[r];
      for (int c = 0; c < nb; ++c) acc = fma(-L[r + (int64_t)(k0 + c) * ldl], zs[k0 + c], acc);
      zs[r] = acc;
    }
    __syncthreads();
  }
  for (int r = tid; r < n; r += TI_THREADS) Z[r + (int64_t)j * ldz] = r < j ? 0.0 : zs[r];
}

ctd_status tri_inverse(const double* L, int64_t ldl, int64_t n, double* Z, int64_t ldz,
                       cudaStream_t st) {
  if (n <= 0) return CTD_OK;
  // the column lives in shared memory: n <= 28,000 or so
  const size_t smem = (size_t)n * sizeof(double);
  if (smem > 48 * 1024) {
    CTD_TRY(allow_max_smem((const void*)k_tri_inv_cols));
    int dev = 0, optin = 0;
    CTD_CUDA(cudaGetDevice(&dev));
    CTD_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (smem > (size_t)optin)
      return fail(CTD_ENOTSUP, "triangular inverse: more kept fibers than one column of shared memory holds");
  }
  CTD_LAUNCH(k_tri_inv_cols, ((unsigned)n), (TI_THREADS), smem, st, L, ldl, (int)n, Z, ldz);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

// B <- L^{-T} B (backward substitution with the transpose of lower L).
// Backward substitution on one 32-row block with L^T, a warp per right-hand
// side (lane r holds x_r; rows are finished from the bottom up).
__global__ void k_trsm_diag_T(const double* __restrict__ L, int64_t ldl, int64_t n, int64_t k0,
                              double* __restrict__ B, int64_t ldb, int64_t nrhs) {
  __shared__ double Ls[NB][NB + 1];
  __shared__ double inv[NB];
  const int nb = (int)min((int64_t)NB, n - k0);
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e % NB, c = e / NB;
    Ls[r][c] = (r < nb && c <= r) ? L[(k0 + r) + (k0 + c) * ldl] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < NB) inv[threadIdx.x] = threadIdx.x < nb ? 1.0 / Ls[threadIdx.x][threadIdx.x] : 0.0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= nrhs) return;
  double* col = B + j * ldb + k0;
  double x = lane < nb ? col[lane] : 0.0;
#pragma unroll
  for (int r = NB - 1; r >= 0; --r) {
    if (r < nb) {
      const double xr = __shfl_sync(0xffffffffu, x * inv[r], r);
      if (lane == r) x = xr;
      else if (lane < r) x = fma(-Ls[r][lane], xr, x);
    }
  }
  if (lane < nb) col[lane] = x;
}

void tri_solve_lower_T(const double* L, int64_t ldl, int64_t n, double* B, int64_t ldb,
                       int64_t nrhs, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return;
  const int64_t last = ((n - 1) / NB) * NB;
  for (int64_t k0 = last; k0 >= 0; k0 -= NB) {
    const int64_t nb = std::min<int64_t>(NB, n - k0);
    CTD_LAUNCH(k_trsm_diag_T, ((unsigned)((nrhs + 7) / 8)), (256), 0, st, L, ldl, n, k0, B,
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

// The failure path of the bounded waits, exercised on purpose: one thread
// waits, with the grid barrier's wait, on a word nothing changes.
__global__ void k_selftest_wait(unsigned* word, unsigned* status, long long limit) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    volatile unsigned* v = word;
    ctd::bounded_wait_change(v, *v, status, limit);
  }
}

namespace ctd {
__global__ void k_selftest_rsqrt(const double* __restrict__ d, int64_t n, double* __restrict__ out,
                                 double* __restrict__ ref) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[i] = rsqrt_fp64(d[i]);
    ref[i] = 1.0 / sqrt(d[i]);
  }
}
}  // namespace ctd

extern "C" ctd_status ctd_selftest_rsqrt(const double* d, int64_t n, double* out, double* ref) {
  using namespace ctd;
  if (n < 0 || n > (1 << 24) || (n > 0 && (!d || !out || !ref)))
    return fail(CTD_EINVAL, "rsqrt self-test: n out of range or NULL array");
  if (n == 0) return CTD_OK;
  double* dev = nullptr;
  CTD_TRY(dalloc(reinterpret_cast<void**>(&dev), (size_t)n * 3 * sizeof(double), nullptr));
  ctd_status rc = CTD_OK;
  cudaError_t e = cudaMemcpy(dev, d, (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    CTD_LAUNCH(ctd::k_selftest_rsqrt, (grid_for(n, 256, (int64_t)num_sms() * 8)), (256), 0,
               nullptr, dev, n, dev + n, dev + 2 * n);
    e = cudaMemcpy(out, dev + n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(ref, dev + 2 * n, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) rc = fail(CTD_ECUDA, std::string("rsqrt self-test: ") + cudaGetErrorString(e));
  cudaDeviceSynchronize();
  dfree(dev, nullptr);
  return rc;
}

extern "C" ctd_status ctd_selftest_bounded_wait(int64_t spin_limit, void* stream) {
  using namespace ctd;
  if (spin_limit < 1 || spin_limit > (1 << 24)) return fail(CTD_EINVAL, "spin_limit must be in [1, 2^24]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned* buf = nullptr;
  CTD_TRY(dalloc_n(&buf, 2, st));
  unsigned h = 0;
  ctd_status rc = CTD_OK;
  if (cudaMemsetAsync(buf, 0, 2 * sizeof(unsigned), st) != cudaSuccess) rc = fail(CTD_ECUDA, "memset failed");
  if (rc == CTD_OK) {
    CTD_LAUNCH(k_selftest_wait, (1), (32), 0, st, buf, buf + 1, (long long)spin_limit);
    rc = d2h(&h, buf + 1, 1, st);
    if (rc == CTD_OK) rc = sync(st);
  }
  dfree(buf, st);
  if (rc != CTD_OK) return rc;
  return status_from_device(h);
}
