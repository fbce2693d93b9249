// Sparse products with the factor R:
//   * dense columns  out(:, c) = R^T x_f      (the Gram matrices of the
//     independence filter of Algorithm 1 / Algorithm 2),
//   * the sparse core C_(alpha) = R^T X_(alpha) (Algorithm 1, Eq. 3),
//   * the error numerator ||P_R X||_F^2 = ||Q^T X_(alpha)||_F^2 with
//     Q = R L^{-T} (Eq. error, Lemma 3.2).
//
// Every product is an exact integer sum (int32 x int32 -> int64 terms).
// Column f of X is expanded into (row entry of R) work items which a warp
// spreads over its lanes; partial sums go to a dense int64 accumulator in
// shared memory and a bitmap marks the touched rows of R^T x_f, so results
// come out in ascending row order without a sort.
#include <algorithm>
#include <vector>

#include "ctd_internal.cuh"
#include "ctd_expand.cuh"

namespace ctd {

constexpr int WARP_MODE_MAX_WIDTH = 1024;  // accumulator per warp
constexpr int CTA_MODE_MAX_WIDTH = 24576;  // accumulator per block
constexpr int SPMM_THREADS = 256;

// Accumulate R^T x_f for column f into acc/bitmap; warps of the group
// [gwarp0, gwarp0 + gwarps) take interleaved 32-entry chunks.
__device__ __forceinline__ void accumulate_column(const CscDev& X, const CsrDev& R, int64_t f,
                                                  unsigned long long* acc, unsigned* bitmap,
                                                  int gwarp, int gwarps) {
  const unsigned long long a = X.colptr[f], b = X.colptr[f + 1];
  const int lane = threadIdx.x & 31;
  for (unsigned long long p0 = a + (unsigned long long)gwarp * 32; p0 < b;
       p0 += (unsigned long long)gwarps * 32) {
    const unsigned long long p = p0 + lane;
    unsigned long long rs = 0;
    int rl = 0, v = 0;
    if (p < b) {
      const int i = __ldg(X.row + p);
      v = __ldg(X.val + p);
      rs = __ldg(reinterpret_cast<const unsigned long long*>(R.rowptr) + i);
      rl = (int)(__ldg(reinterpret_cast<const unsigned long long*>(R.rowptr) + i + 1) - rs);
    }
    expand_chunk(rs, rl, v, R.col, R.val, [&](int m, long long prod) {
      atomicAdd(acc + m, (unsigned long long)prod);
      if (bitmap) atomicOr(bitmap + (m >> 5), 1u << (m & 31));
    });
  }
}

// ---------------------------------------------------------------------------
// dense output (one block per column)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SPMM_THREADS)
    k_spmm_dense(CscDev X, const int64_t* __restrict__ fibers, const int* nf_dev, int nf_max,
                 CsrDev R, double* __restrict__ out, int64_t ld) {
  extern __shared__ unsigned long long acc[];
  const int nf = min(*nf_dev, nf_max);
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int m = threadIdx.x; m < R.width; m += blockDim.x) acc[m] = 0;
  __syncthreads();
  for (int c = blockIdx.x; c < nf; c += gridDim.x) {
    accumulate_column(X, R, fibers[c], acc, nullptr, warp, nw);
    __syncthreads();
    for (int m = threadIdx.x; m < R.width; m += blockDim.x) {
      out[(int64_t)c * ld + m] = (double)(long long)acc[m];
      acc[m] = 0;
    }
    __syncthreads();
  }
}

// The same product with each column's entries spread over up to GS_SLICES
// blocks (block (c, s) takes the column's 32-entry chunks s, s + GS_SLICES,
// ... over its warps), so that the longest columns, those with the frequent
// mode-alpha indices, do not leave one block working alone; each block adds
// its integer partial sums into an int64 accumulator (exact in any order),
// which a second pass converts.
constexpr int GS_SLICES = 8;

__global__ void __launch_bounds__(SPMM_THREADS)
    k_spmm_dense_sliced(CscDev X, const int64_t* __restrict__ fibers, const int* nf_dev,
                        int nf_max, CsrDev R, unsigned long long* __restrict__ gacc) {
  extern __shared__ unsigned long long acc[];
  const int nf = min(*nf_dev, nf_max);
  const int c = blockIdx.x, sl = blockIdx.y;
  if (c >= nf) return;
  const int64_t f = fibers[c];
  const unsigned long long nchunk = (X.colptr[f + 1] - X.colptr[f] + 31) / 32;
  if ((unsigned long long)sl >= nchunk) return;  // uniform over the block
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int m = threadIdx.x; m < R.width; m += blockDim.x) acc[m] = 0;
  __syncthreads();
  accumulate_column(X, R, f, acc, nullptr, sl + GS_SLICES * warp, GS_SLICES * nw);
  __syncthreads();
  unsigned long long* g = gacc + (int64_t)c * R.width;
  for (int m = threadIdx.x; m < R.width; m += blockDim.x)
    if (acc[m]) atomicAdd(g + m, acc[m]);
}

__global__ void k_gram_convert(const unsigned long long* __restrict__ gacc, const int* nf_dev,
                               int nf_max, int width, double* __restrict__ out, int64_t ld) {
  const int nf = min(*nf_dev, nf_max);
  const int64_t total = (int64_t)nf * width;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / width, m = e % width;
    out[c * ld + m] = (double)(long long)gacc[e];
  }
}

ctd_status launch_spmm_dense(const CscDev& X, const int64_t* fibers, const int* nf_dev,
                             int nf_max, const CsrDev& R, double* out, int64_t ld,
                             cudaStream_t st, Arena* scratch) {
  if (nf_max <= 0 || R.width <= 0) return CTD_OK;
  if (scratch && (size_t)R.width * sizeof(unsigned long long) <= 48 * 1024) {
    unsigned long long* gacc;
    CTD_TRY(scratch->get(&gacc, (size_t)nf_max * R.width));
    CTD_CUDA(cudaMemsetAsync(gacc, 0, (size_t)nf_max * R.width * sizeof(unsigned long long), st));
    CTD_LAUNCH(k_spmm_dense_sliced, (dim3((unsigned)nf_max, GS_SLICES)), (SPMM_THREADS),
               (size_t)R.width * sizeof(unsigned long long), st, X, fibers, nf_dev, nf_max, R,
               gacc);
    CTD_LAUNCH(k_gram_convert, (grid_for((int64_t)nf_max * R.width, 256, (int64_t)num_sms() * 8)),
               (256), 0, st, gacc, nf_dev, nf_max, R.width, out, ld);
    CTD_CUDA(cudaGetLastError());
    return CTD_OK;
  }
  if (R.width > CTA_MODE_MAX_WIDTH)
    return fail(CTD_EINVAL, "factor wider than the supported maximum (24576 columns)");
  const size_t smem = (size_t)R.width * sizeof(unsigned long long);
  if (smem > 48 * 1024)
    CTD_TRY(allow_max_smem((const void*)k_spmm_dense));
  unsigned g = (unsigned)std::min<int64_t>(nf_max, (int64_t)num_sms() * 4);
  CTD_LAUNCH(k_spmm_dense, (g), (SPMM_THREADS), smem, st, X, fibers, nf_dev, nf_max, R, out, ld);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

// ---------------------------------------------------------------------------
// C bounds: ub[f] = min(width, sum over column f of R row lengths)
// ---------------------------------------------------------------------------
__global__ void k_c_bounds(CscDev X, int64_t n_cols, CsrDev R, unsigned* __restrict__ ub) {
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n_cols;
       f += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long a = X.colptr[f], b = X.colptr[f + 1];
    unsigned long long s = 0;
    for (unsigned long long p = a; p < b && s < (unsigned long long)R.width; ++p) {
      const int i = __ldg(X.row + p);
      s += __ldg(rp + i + 1) - __ldg(rp + i);
    }
    // capacity: the bound rounded up to a multiple of 4, so that every
    // column of C starts on a 16-byte boundary of its value array
    ub[f] = ((unsigned)min(s, (unsigned long long)R.width) + 3u) & ~3u;
  }
}

void launch_c_bounds(const CscDev& X, int64_t n_cols, const CsrDev& R, uint32_t* ub,
                     cudaStream_t st) {
  if (n_cols <= 0) return;
  CTD_LAUNCH(k_c_bounds, (grid_for(n_cols, 256, (int64_t)num_sms() * 16)), (256), 0, st, X, n_cols, R, ub);
}

// ---------------------------------------------------------------------------
// C fill
//
// Column f of C is written to [coff[f], coff[f] + ccnt[f]) with rows
// ascending (uint16 row index: s~ <= 24576).  Three paths:
//  * a column with one nonzero v in row i (all values positive) is
//    v * R(i, :), copied from R's row i (rows of R are sorted by column);
//  * other columns with fewer than HEAVY nonzeros: one warp each, with a
//    warp-private accumulator in shared memory;
//  * heavy columns: a whole block each.
// An output entry exists exactly where the accumulator is nonzero, so the
// emission is a sweep over the accumulator, 32 rows at a time, compacted
// with a ballot (ascending order, exact zeros dropped) -- no touched-set
// bookkeeping.  Accumulators are int32 when ||X||_F^2 < 2^31: by
// Cauchy-Schwarz every partial sum is at most ||x_f|| ||r_m|| <= ||X||_F^2.
// ---------------------------------------------------------------------------
constexpr int HEAVY = 128;

template <typename A>
__device__ __forceinline__ void acc_add(A* p, long long x);
template <>
__device__ __forceinline__ void acc_add<int>(int* p, long long x) {
  atomicAdd(p, (int)x);
}
template <>
__device__ __forceinline__ void acc_add<unsigned long long>(unsigned long long* p, long long x) {
  atomicAdd(p, (unsigned long long)x);
}
template <typename A>
__device__ __forceinline__ long long acc_val(A x) {
  return sizeof(A) == 4 ? (long long)(int)x : (long long)x;
}

// R rows with at least LONG_ROW entries are walked by the whole warp (one
// product per lane per step); shorter rows go through expand_chunk, which
// spreads the products of 32 short rows over the lanes.
constexpr int LONG_ROW = 16;

template <typename A>
__device__ __forceinline__ void accumulate_column_t(const CscDev& X, const CsrDev& R, int64_t f,
                                                    A* acc, int gwarp, int gwarps) {
  const unsigned long long a = X.colptr[f], b = X.colptr[f + 1];
  const int lane = threadIdx.x & 31;
  for (unsigned long long p0 = a + (unsigned long long)gwarp * 32; p0 < b;
       p0 += (unsigned long long)gwarps * 32) {
    const unsigned long long p = p0 + lane;
    unsigned long long rs = 0;
    int rl = 0, v = 0;
    if (p < b) {
      const int i = __ldg(X.row + p);
      v = __ldg(X.val + p);
      rs = __ldg(reinterpret_cast<const unsigned long long*>(R.rowptr) + i);
      rl = (int)(__ldg(reinterpret_cast<const unsigned long long*>(R.rowptr) + i + 1) - rs);
    }
    unsigned longs = __ballot_sync(0xffffffffu, rl >= LONG_ROW);
    while (longs) {
      const int src = __ffs(longs) - 1;
      longs &= longs - 1;
      const unsigned long long s0 = __shfl_sync(0xffffffffu, rs, src);
      const int n = __shfl_sync(0xffffffffu, rl, src);
      const long long vs = __shfl_sync(0xffffffffu, v, src);
      for (int q = lane; q < n; q += 32)
        acc_add<A>(acc + __ldg(R.col + s0 + q), vs * (long long)__ldg(R.val + s0 + q));
    }
    if (rl >= LONG_ROW) rl = 0;
    if (__any_sync(0xffffffffu, rl > 0))
      expand_chunk(rs, rl, v, R.col, R.val,
                   [&](int m, long long prod) { acc_add<A>(acc + m, prod); });
  }
}

// Warp-level emission of one column: sweep acc 32 rows at a time.
template <typename V, typename A>
__device__ __forceinline__ unsigned emit_warp(A* acc, int width, unsigned long long off,
                                              uint16_t* __restrict__ crow, V* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  unsigned pos = 0;
  for (int m0 = 0; m0 < width; m0 += 32) {
    const int m = m0 + lane;
    long long x = 0;
    if (m < width) {
      x = acc_val<A>(acc[m]);
      acc[m] = 0;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, x != 0);
    if (x != 0) {
      const unsigned q = pos + __popc(ball & ((1u << lane) - 1));
      crow[off + q] = (uint16_t)m;
      cval[off + q] = (V)x;
    }
    pos += __popc(ball);
  }
  return pos;
}

template <typename V, typename A>
__global__ void __launch_bounds__(SPMM_THREADS)
    k_c_fill_warp(CscDev X, int64_t n_cols, CsrDev R, const unsigned long long* __restrict__ coff,
                  unsigned* __restrict__ ccnt, uint16_t* __restrict__ crow, V* __restrict__ cval,
                  int positive, unsigned long long* work) {
  extern __shared__ unsigned long long smem_u64[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int width = R.width;
  const int accw = (width + 1) & ~1;  // keep 8-byte alignment between warps
  A* acc = reinterpret_cast<A*>(smem_u64) + (size_t)warp * accw;
  for (int m = lane; m < width; m += 32) acc[m] = 0;
  __syncwarp();
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  const unsigned long long* xp = reinterpret_cast<const unsigned long long*>(X.colptr);
  // 32 columns per grab; lane l prefetches column f0 + l's offsets and, for a
  // one-nonzero column, its entry and R-row range, so empty and one-nonzero
  // columns cost no dependent loads inside the walk below
  while (true) {
    unsigned long long f0 = 0;
    if (lane == 0) f0 = atomicAdd(work, 32ull);
    f0 = __shfl_sync(0xffffffffu, f0, 0);
    if (f0 >= (unsigned long long)n_cols) break;
    const int64_t f = (int64_t)f0 + lane;
    unsigned long long o = 0, xa = 0, rs = 0;
    int ub = 0, nx = 0, vv = 0, rl = 0;
    if (f < n_cols) {
      o = coff[f];
      ub = (int)(coff[f + 1] - o);
      xa = xp[f];
      nx = (int)min(xp[f + 1] - xa, (unsigned long long)0x7fffffff);
      if (ub > 0 && nx == 1 && positive) {
        const int i = __ldg(X.row + xa);
        vv = __ldg(X.val + xa);
        rs = __ldg(rp + i);
        rl = (int)(__ldg(rp + i + 1) - rs);
      }
      if (ub == 0) ccnt[f] = 0;
    }
    const int nf = (int)min((int64_t)32, n_cols - (int64_t)f0);
    for (int e = 0; e < nf; ++e) {
      const int ube = __shfl_sync(0xffffffffu, ub, e);
      const int nxe = __shfl_sync(0xffffffffu, nx, e);
      if (ube == 0 || nxe >= HEAVY) continue;  // empty here; heavy: block kernel
      const unsigned long long oe = __shfl_sync(0xffffffffu, o, e);
      if (nxe == 1 && positive) {
        const unsigned long long rse = __shfl_sync(0xffffffffu, rs, e);
        const int rle = __shfl_sync(0xffffffffu, rl, e);
        const long long ve = __shfl_sync(0xffffffffu, vv, e);
        for (int q = lane; q < rle; q += 32) {
          crow[oe + q] = (uint16_t)__ldg(R.col + rse + q);
          cval[oe + q] = (V)(ve * (long long)__ldg(R.val + rse + q));
        }
        if (lane == 0) ccnt[f0 + e] = (unsigned)rle;
        continue;
      }
      accumulate_column_t<A>(X, R, (int64_t)f0 + e, acc, 0, 1);
      __syncwarp();
      const unsigned n = emit_warp<V, A>(acc, width, oe, crow, cval);
      __syncwarp();
      if (lane == 0) ccnt[f0 + e] = n;
    }
  }
}

template <typename V, typename A>
__global__ void __launch_bounds__(SPMM_THREADS)
    k_c_fill_block(CscDev X, const int64_t* __restrict__ list, const unsigned* __restrict__ nlist,
                   CsrDev R, const unsigned long long* __restrict__ coff,
                   unsigned* __restrict__ ccnt, uint16_t* __restrict__ crow, V* __restrict__ cval,
                   unsigned long long* work) {
  extern __shared__ unsigned long long smem_u64[];
  const int width = R.width;
  A* acc = reinterpret_cast<A*>(smem_u64);
  __shared__ unsigned long long fcur;
  __shared__ unsigned wcount[SPMM_THREADS / 32];
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long n = *nlist;
  for (int m = threadIdx.x; m < width; m += blockDim.x) acc[m] = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) fcur = atomicAdd(work, 1ull);
    __syncthreads();
    const unsigned long long it = fcur;
    __syncthreads();
    if (it >= n) break;
    const int64_t f = list[it];
    accumulate_column_t<A>(X, R, f, acc, warp, nw);
    __syncthreads();
    // emission: warp w sweeps rows [w * span, (w + 1) * span) after counting
    const int span = (((width + nw - 1) / nw) + 31) & ~31;
    const int m_lo = min(width, warp * span), m_hi = min(width, m_lo + span);
    unsigned cnt = 0;
    for (int m0 = m_lo; m0 < m_hi; m0 += 32) {
      const int m = m0 + lane;
      const bool nz = m < m_hi && acc[m] != 0;
      cnt += __popc(__ballot_sync(0xffffffffu, nz));
    }
    if (lane == 0) wcount[warp] = cnt;
    __syncthreads();
    unsigned pos = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
      if (w < warp) pos += wcount[w];
      total += wcount[w];
    }
    const unsigned long long off = coff[f];
    for (int m0 = m_lo; m0 < m_hi; m0 += 32) {
      const int m = m0 + lane;
      long long x = 0;
      if (m < m_hi) {
        x = acc_val<A>(acc[m]);
        acc[m] = 0;
      }
      const unsigned ball = __ballot_sync(0xffffffffu, x != 0);
      if (x != 0) {
        const unsigned q = pos + __popc(ball & ((1u << lane) - 1));
        crow[off + q] = (uint16_t)m;
        cval[off + q] = (V)x;
      }
      pos += __popc(ball);
    }
    if (threadIdx.x == 0) ccnt[f] = total;
    __syncthreads();
  }
}

// Columns with at least `minc` nonzeros (and a nonzero bound): list + count.
__global__ void k_list_columns(const unsigned long long* __restrict__ colptr,
                               const unsigned long long* __restrict__ coff, int64_t n_cols,
                               unsigned long long minc, int64_t* __restrict__ list,
                               unsigned* __restrict__ count) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n_cols;
       f += (int64_t)gridDim.x * blockDim.x) {
    if (colptr[f + 1] - colptr[f] >= minc && coff[f + 1] > coff[f])
      list[atomicAdd(count, 1u)] = f;
  }
}

__global__ void k_list_columns_nnz(const unsigned long long* __restrict__ colptr, int64_t n_cols,
                                   unsigned long long minc, int64_t* __restrict__ list,
                                   unsigned* __restrict__ count) {
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n_cols;
       f += (int64_t)gridDim.x * blockDim.x)
    if (colptr[f + 1] - colptr[f] >= minc) list[atomicAdd(count, 1u)] = f;
}

void launch_list_columns_nnz(const uint64_t* colptr, int64_t n_cols, uint64_t minc, int64_t* list,
                             unsigned* count, cudaStream_t st) {
  if (n_cols <= 0) return;
  CTD_LAUNCH(k_list_columns_nnz, (grid_for(n_cols, 256, (int64_t)num_sms() * 8)), (256), 0, st,
             reinterpret_cast<const unsigned long long*>(colptr), n_cols,
             (unsigned long long)minc, list, count);
}

void launch_list_columns(const uint64_t* colptr, const uint64_t* coff, int64_t n_cols,
                         uint64_t minc, int64_t* list, unsigned* count, cudaStream_t st) {
  if (n_cols <= 0) return;
  CTD_LAUNCH(k_list_columns, (grid_for(n_cols, 256, (int64_t)num_sms() * 8)), (256), 0, st,
             reinterpret_cast<const unsigned long long*>(colptr),
             reinterpret_cast<const unsigned long long*>(coff), n_cols,
             (unsigned long long)minc, list, count);
}

template <typename V, typename A>
static ctd_status c_fill_impl(const CscDev& X, int64_t n_cols, const CsrDev& R,
                              const uint64_t* coff, uint32_t* ccnt, uint16_t* crow, V* cval,
                              int positive, unsigned long long* work, int64_t* heavy,
                              unsigned* nheavy, cudaStream_t st) {
  const int width = R.width;
  const int accw = (width + 1) & ~1;
  const unsigned long long* co = reinterpret_cast<const unsigned long long*>(coff);
  // heavy columns (and, if the warp accumulator would not fit, all columns)
  const bool warp_ok = width <= WARP_MODE_MAX_WIDTH;
  CTD_LAUNCH(k_list_columns, (grid_for(n_cols, 256, (int64_t)num_sms() * 8)), (256), 0, st,
             reinterpret_cast<const unsigned long long*>(X.colptr), co, n_cols,
             warp_ok ? (unsigned long long)HEAVY : 1ull, heavy, nheavy);
  if (warp_ok) {
    const int nw = SPMM_THREADS / 32;
    const size_t smem = (size_t)nw * accw * sizeof(A);
    if (smem > 48 * 1024)
      CTD_TRY(allow_max_smem((const void*)k_c_fill_warp<V, A>));
    int per_sm = 0;
    CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_c_fill_warp<V, A>,
                                                           SPMM_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    CTD_LAUNCH((k_c_fill_warp<V, A>), (num_sms() * per_sm), (SPMM_THREADS), smem, st, X, n_cols,
               R, co, ccnt, crow, cval, positive, work);
  } else {
    CTD_CUDA(cudaMemsetAsync(ccnt, 0, n_cols * sizeof(uint32_t), st));
  }
  if (width > CTA_MODE_MAX_WIDTH)
    return fail(CTD_EINVAL, "factor wider than the supported maximum (24576 columns)");
  const size_t smem = (size_t)accw * sizeof(A);
  if (smem > 48 * 1024)
    CTD_TRY(allow_max_smem((const void*)k_c_fill_block<V, A>));
  int per_sm = 0;
  CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_c_fill_block<V, A>,
                                                         SPMM_THREADS, smem));
  if (per_sm < 1) per_sm = 1;
  CTD_LAUNCH((k_c_fill_block<V, A>), (num_sms() * per_sm), (SPMM_THREADS), smem, st, X, heavy,
             nheavy, R, co, ccnt, crow, cval, work + 1);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

ctd_status launch_c_fill(const CscDev& X, int64_t n_cols, int64_t n_rows, int64_t nnz,
                         const CsrDev& R, const uint64_t* coff, uint32_t* ccnt, uint16_t* crow,
                         void* cval, int fp32, int positive, int x_int8, uint64_t sqnorm_X,
                         cudaStream_t st, const CfillLists* lists) {
  if (n_cols <= 0) return CTD_OK;
  if (R.width <= 0) {
    CTD_CUDA(cudaMemsetAsync(ccnt, 0, n_cols * sizeof(uint32_t), st));
    return CTD_OK;
  }
  if (R.width > 65535) return fail(CTD_EINVAL, "too many kept fibers for 16-bit row indices");
  // integer partial sums fit int32 (Cauchy-Schwarz) and the warp's register
  // accumulators cover the width: dense long rows + registers
  if (sqnorm_X < (1ull << 31) && R.width <= 1024)
    return c_fill_dense_rows(X, n_cols, n_rows, nnz, R, coff, ccnt, crow, cval, fp32, positive,
                             x_int8, st, lists);
  unsigned long long* work;
  int64_t* heavy;
  unsigned* nheavy;
  CTD_TRY(dalloc_n(&work, 2, st));
  CTD_TRY(dalloc_n(&heavy, n_cols, st));
  CTD_TRY(dalloc_n(&nheavy, 1, st));
  CTD_CUDA(cudaMemsetAsync(work, 0, 2 * sizeof(unsigned long long), st));
  CTD_CUDA(cudaMemsetAsync(nheavy, 0, sizeof(unsigned), st));
  const bool small = sqnorm_X < (1ull << 31);
  ctd_status rc;
  if (fp32)
    rc = small ? c_fill_impl<float, int>(X, n_cols, R, coff, ccnt, crow, static_cast<float*>(cval),
                                         positive, work, heavy, nheavy, st)
               : c_fill_impl<float, unsigned long long>(X, n_cols, R, coff, ccnt, crow,
                                                        static_cast<float*>(cval), positive, work,
                                                        heavy, nheavy, st);
  else
    rc = small ? c_fill_impl<double, int>(X, n_cols, R, coff, ccnt, crow,
                                          static_cast<double*>(cval), positive, work, heavy,
                                          nheavy, st)
               : c_fill_impl<double, unsigned long long>(X, n_cols, R, coff, ccnt, crow,
                                                         static_cast<double*>(cval), positive,
                                                         work, heavy, nheavy, st);
  dfree(work, st);
  dfree(heavy, st);
  dfree(nheavy, st);
  return rc;
}

// Sort each row of a row-major factor by column: one warp per row, each
// entry placed at its rank (the number of smaller columns; columns within a
// row are distinct).  When the columns lie in [col_base, col_base + ncols)
// with ncols <= SR_BITS, a row longer than SR_SHORT marks its columns in a
// bitmap in the warp's shared memory and takes each rank as the popcount of
// the bits below it (a prefix over the bitmap's words, then one word), so a
// row of n entries costs O(n + ncols/32) rather than O(n^2) (the long rows,
// those of the frequent mode-alpha indices, used to dominate).  Otherwise
// rows of up to SR_SMEM entries are ranked against a copy of their columns
// in shared memory and longer ones against global memory.  In/out arrays
// differ.
constexpr int SR_SMEM = 512;
constexpr int SR_SHORT = 64;
constexpr int SR_BITS = 8192;
constexpr int SR_WORDS = SR_BITS / 32;

__global__ void __launch_bounds__(256)
    k_sort_rows(const unsigned long long* __restrict__ rowptr, int64_t n_rows,
                const int32_t* __restrict__ col_in, const int32_t* __restrict__ val_in,
                int32_t* __restrict__ col_out, int32_t* __restrict__ val_out, int col_base,
                int ncols) {
  __shared__ int32_t keys[8][SR_SMEM];
  __shared__ unsigned bits[8][SR_WORDS];
  __shared__ unsigned pre[8][SR_WORDS];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t* kw = keys[wib];
  unsigned* bw = bits[wib];
  unsigned* pw = pre[wib];
  const bool use_bits = ncols > 0 && ncols <= SR_BITS;
  const int nwords = (ncols + 31) >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n_rows; i += nw) {
    const unsigned long long a = rowptr[i], b = rowptr[i + 1];
    const int len = (int)(b - a);
    if (use_bits && len > SR_SHORT) {
      for (int w = lane; w < nwords; w += 32) bw[w] = 0u;
      __syncwarp();
      for (int e = lane; e < len; e += 32) {
        const int m = col_in[a + e] - col_base;
        atomicOr(&bw[m >> 5], 1u << (m & 31));
      }
      __syncwarp();
      // exclusive prefix of the words' popcounts, 32 words per pass
      unsigned carry = 0;
      for (int w0 = 0; w0 < nwords; w0 += 32) {
        const int w = w0 + lane;
        const unsigned c = w < nwords ? (unsigned)__popc(bw[w]) : 0u;
        unsigned x = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const unsigned y = __shfl_up_sync(0xffffffffu, x, d);
          if (lane >= d) x += y;
        }
        if (w < nwords) pw[w] = carry + x - c;
        carry += __shfl_sync(0xffffffffu, x, 31);
      }
      __syncwarp();
      for (int e = lane; e < len; e += 32) {
        const int mc = col_in[a + e];
        const int m = mc - col_base;
        const int r = (int)pw[m >> 5] + __popc(bw[m >> 5] & ((1u << (m & 31)) - 1u));
        col_out[a + r] = mc;
        val_out[a + r] = val_in[a + e];
      }
      __syncwarp();
    } else if (len <= SR_SMEM) {
      for (int e = lane; e < len; e += 32) kw[e] = col_in[a + e];
      __syncwarp();
      for (int e = lane; e < len; e += 32) {
        const int m = kw[e];
        int r = 0;
        for (int q = 0; q < len; ++q) r += (kw[q] < m);
        col_out[a + r] = m;
        val_out[a + r] = val_in[a + e];
      }
      __syncwarp();
    } else {
      for (unsigned long long p = a + lane; p < b; p += 32) {
        const int m = col_in[p];
        unsigned long long r = 0;
        for (unsigned long long q = a; q < b; ++q) r += (col_in[q] < m);
        col_out[a + r] = m;
        val_out[a + r] = val_in[p];
      }
    }
  }
}

// Sort each segment of a compressed layout by index (values follow), in
// place: a block per segment.  When the indices lie in [0, nbits) with nbits
// <= SEG_BITS, a segment of more than 32 entries marks its indices in a
// bitmap in shared memory and places each entry at its rank, the popcount
// of the bits below it (a block-wide prefix over the bitmap's words, then
// one word): O(n + nbits/32) per segment.  Otherwise bitonic in shared
// memory up to 2048 entries, and longer segments rank each entry by
// counting (indices within a segment are distinct).  Used to give gathered
// columns a reproducible order.
constexpr int SEG_SORT_MAX = 2048;
constexpr int SEG_BITS = 65536;
constexpr int SEG_WORDS = SEG_BITS / 32;

__global__ void __launch_bounds__(256)
    k_sort_segments(const unsigned long long* __restrict__ ptr, int64_t nseg,
                    int32_t* __restrict__ idx, int32_t* __restrict__ val,
                    int32_t* __restrict__ tmp_idx, int32_t* __restrict__ tmp_val, int nbits) {
  __shared__ int32_t ks[SEG_SORT_MAX];
  __shared__ int32_t vs[SEG_SORT_MAX];
  __shared__ unsigned bits[SEG_WORDS];
  __shared__ unsigned pre[SEG_WORDS];
  __shared__ unsigned wtot[8];
  const int nwords = (nbits + 31) >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t g = blockIdx.x; g < nseg; g += gridDim.x) {
    const unsigned long long a = ptr[g], b = ptr[g + 1];
    const int n = (int)(b - a);
    if (n <= 1) continue;
    if (nbits > 0 && n > 32) {
      for (int w = threadIdx.x; w < nwords; w += blockDim.x) bits[w] = 0u;
      __syncthreads();
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int m = idx[a + e];
        atomicOr(&bits[m >> 5], 1u << (m & 31));
      }
      __syncthreads();
      // exclusive prefix of the words' popcounts: each thread a run of
      // consecutive words, then the threads' totals across the block
      const int per = (nwords + blockDim.x - 1) / blockDim.x;
      const int w0 = threadIdx.x * per;
      unsigned mine = 0;
      for (int w = w0; w < min(w0 + per, nwords); ++w) mine += __popc(bits[w]);
      unsigned inc = mine;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
      }
      if (lane == 31) wtot[warp] = inc;
      __syncthreads();
      unsigned off = inc - mine;
      for (int q = 0; q < warp; ++q) off += wtot[q];
      for (int w = w0; w < min(w0 + per, nwords); ++w) {
        pre[w] = off;
        off += __popc(bits[w]);
      }
      __syncthreads();
      const bool smem = n <= SEG_SORT_MAX;
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int m = idx[a + e];
        const int r = (int)pre[m >> 5] + __popc(bits[m >> 5] & ((1u << (m & 31)) - 1u));
        if (smem) {
          ks[r] = m;
          vs[r] = val[a + e];
        } else {
          tmp_idx[a + r] = m;
          tmp_val[a + r] = val[a + e];
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        idx[a + e] = smem ? ks[e] : tmp_idx[a + e];
        val[a + e] = smem ? vs[e] : tmp_val[a + e];
      }
      __syncthreads();
    } else if (n <= SEG_SORT_MAX) {
      int m = 1;
      while (m < n) m <<= 1;
      for (int e = threadIdx.x; e < m; e += blockDim.x) {
        ks[e] = e < n ? idx[a + e] : INT32_MAX;
        vs[e] = e < n ? val[a + e] : 0;
      }
      __syncthreads();
      for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const int o = e ^ j;
            if (o > e) {
              const bool up = (e & k) == 0;
              if ((ks[e] > ks[o]) == up) {
                const int32_t tk = ks[e], tv = vs[e];
                ks[e] = ks[o];
                vs[e] = vs[o];
                ks[o] = tk;
                vs[o] = tv;
              }
            }
          }
          __syncthreads();
        }
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        idx[a + e] = ks[e];
        val[a + e] = vs[e];
      }
      __syncthreads();
    } else {
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int32_t me = idx[a + e];
        int r = 0;
        for (int q = 0; q < n; ++q) r += idx[a + q] < me;
        tmp_idx[a + r] = me;
        tmp_val[a + r] = val[a + e];
      }
      __syncthreads();
      for (int e = threadIdx.x; e < n; e += blockDim.x) {
        idx[a + e] = tmp_idx[a + e];
        val[a + e] = tmp_val[a + e];
      }
      __syncthreads();
    }
  }
}

void launch_sort_segments(const uint64_t* ptr, int64_t nseg, int32_t* idx, int32_t* val,
                          int32_t* tmp_idx, int32_t* tmp_val, int64_t index_range,
                          cudaStream_t st) {
  if (nseg <= 0) return;
  const int nbits = index_range > 0 && index_range <= SEG_BITS ? (int)index_range : 0;
  CTD_LAUNCH(k_sort_segments, ((unsigned)std::min<int64_t>(nseg, (int64_t)num_sms() * 8)), (256), 0,
             st, reinterpret_cast<const unsigned long long*>(ptr), nseg, idx, val, tmp_idx,
             tmp_val, nbits);
}

void launch_sort_rows(const uint64_t* rowptr, int64_t n_rows, const int32_t* col_in,
                      const int32_t* val_in, int32_t* col_out, int32_t* val_out, int col_base,
                      int64_t ncols, cudaStream_t st) {
  if (n_rows <= 0) return;
  const int nc = ncols > 0 && ncols <= SR_BITS ? (int)ncols : 0;  // 0: no bitmap
  CTD_LAUNCH(k_sort_rows, (grid_for(n_rows * 32, 256, (int64_t)num_sms() * 16)), (256), 0, st,
             reinterpret_cast<const unsigned long long*>(rowptr), n_rows, col_in, val_in, col_out,
             val_out, col_base, nc);
}

// ---------------------------------------------------------------------------
// Error numerator in the Q form: ||P_R X||_F^2 = ||Q^T X_(alpha)||_F^2 with
// Q = R L^{-T} (orthonormal columns spanning range(R); L L^T = R^T R, Z =
// L^{-1}).  Q is dense I_alpha x s~, row-major with stride qs (a multiple of
// 32), computed in FP64 and stored as T.  The sum over columns f of
// ||Q^T x_f||^2 costs nnz * s~ multiply-adds; a column with one nonzero v in
// row i contributes v^2 ||Q(i, :)||^2, read from the precomputed row norms.
// ---------------------------------------------------------------------------
// One warp per (row i of R, group of 64 columns of Q): Q(i, c) = sum over
// the row's entries m <= c of R(i, m) Z(c, m) (Z lower triangular), in the
// row's entry order; lane l owns columns c0 + l and c0 + 32 + l.  The row's
// entries are loaded 32 at a time (coalesced) and broadcast by shuffles, so
// the Z loads of successive entries are independent and overlap; R's rows
// are sorted by column, so the walk stops at the first entry past the group.
template <typename T>
__global__ void k_build_q(CsrDev R, int64_t n_rows, const double* __restrict__ Z, int64_t ldz,
                          int qs, T* __restrict__ Q) {
  const int lane = threadIdx.x & 31;
  const int ng = qs / 64;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  for (int64_t w = gw; w < n_rows * ng; w += nw) {
    const int64_t i = w / ng;
    const int c0 = (int)(w % ng) * 64;
    const int cA = c0 + lane, cB = c0 + 32 + lane;
    const unsigned long long a = rp[i], b = rp[i + 1];
    double accA = 0.0, accB = 0.0;
    for (unsigned long long base = a; base < b; base += 32) {
      const int cnt = (int)min((unsigned long long)32, b - base);
      int mm = INT_MAX;
      double vv = 0.0;
      if (lane < cnt) {
        mm = R.col[base + lane];
        vv = (double)R.val[base + lane];
      }
      // the entries before the group's end form a prefix (sorted row)
      const int nlive = __popc(__ballot_sync(0xffffffffu, mm < c0 + 64));
#pragma unroll 4
      for (int e = 0; e < nlive; ++e) {
        const int m = __shfl_sync(0xffffffffu, mm, e);
        const double v = __shfl_sync(0xffffffffu, vv, e);
        const double* z = Z + (int64_t)m * ldz;
        if (cA >= m && cA < R.width) accA = fma(v, z[cA], accA);
        if (cB >= m && cB < R.width) accB = fma(v, z[cB], accB);
      }
      if (nlive < cnt) break;
    }
    Q[i * qs + cA] = (T)accA;
    Q[i * qs + cB] = (T)accB;
  }
}

// qn[i] = ||Q(i, :)||^2 of the stored (rounded) rows
template <typename T>
__global__ void k_q_rownorms(const T* __restrict__ Q, int64_t n_rows, int qs,
                             T* __restrict__ qn) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n_rows; i += nw) {
    double nrm = 0.0;
    for (int c = lane; c < qs; c += 32) {
      const double v = (double)Q[i * qs + c];
      nrm = fma(v, v, nrm);
    }
    for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (lane == 0) qn[i] = (T)nrm;
  }
}

// One warp per column, 32 columns per grab.  Hot rows of Q (slot >= 0 in
// `slot_of`, a global table read through the read-only cache) are staged
// in shared memory once per block.  Lane l owns the
// VEC consecutive Q columns at (l + 32 k) * VEC, read with 16-byte loads;
// a column's entries are loaded 32 at a time and broadcast by shuffles.
// Each 32-column chunk's sum goes to partial[chunk] (fixed order inside
// the warp), so the total does not depend on scheduling.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

// threads per block: one 32-warp block per SM for the register widths up
// to NK = 4 (one copy of the staged rows per SM), two 16-warp blocks at NK = 8
template <int NK>
constexpr int qf_threads() { return NK >= 8 ? 512 : 1024; }

// acc += sum over the chunks c = first, first + step, ... of the column
// entries [a, b) (32 per chunk) of v * Q(i, coff : coff + NK*32*VEC); lane l
// holds the VEC consecutive values at (l + 32 k) * VEC.  Rows with a slot
// (slot_of) are read from the staged copy Qs.
template <typename T, int NK>
__device__ __forceinline__ void qrows_accumulate(const CscDev& X, const T* __restrict__ Q, int qs,
                                                 int64_t coff, const T* __restrict__ Qs,
                                                 const short* __restrict__ slot_of,
                                                 unsigned long long a, unsigned long long b,
                                                 int first, int step,
                                                 T (&acc)[NK * Vec16<T>::n]) {
  using VT = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  const int lane = threadIdx.x & 31;
  for (unsigned long long base = a + (unsigned long long)first * 32; base < b;
       base += (unsigned long long)step * 32) {
    const int cnt = (int)min((unsigned long long)32, b - base);
    const T* myrow = nullptr;
    int myv = 0;
    if (lane < cnt) {
      const int i = __ldg(X.row + base + lane);
      myv = __ldg(X.val + base + lane);
      const int sl = slot_of ? (int)__ldg(slot_of + i) : -1;
      myrow = (sl >= 0 ? Qs + (int64_t)sl * qs : Q + (int64_t)i * qs) + coff;
    }
    int q = 0;
    for (; q + 1 < cnt; q += 2) {
      const VT* r0 = (const VT*)__shfl_sync(0xffffffffu, (unsigned long long)myrow, q);
      const VT* r1 = (const VT*)__shfl_sync(0xffffffffu, (unsigned long long)myrow, q + 1);
      const T v0 = (T)__shfl_sync(0xffffffffu, myv, q);
      const T v1 = (T)__shfl_sync(0xffffffffu, myv, q + 1);
      VT a0[NK], a1[NK];
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        a0[k] = r0[lane + 32 * k];
        a1[k] = r1[lane + 32 * k];
      }
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        const T* x0 = reinterpret_cast<const T*>(&a0[k]);
        const T* x1 = reinterpret_cast<const T*>(&a1[k]);
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          acc[k * VEC + u] = fma(v0, x0[u], acc[k * VEC + u]);
          acc[k * VEC + u] = fma(v1, x1[u], acc[k * VEC + u]);
        }
      }
    }
    if (q < cnt) {
      const VT* r0 = (const VT*)__shfl_sync(0xffffffffu, (unsigned long long)myrow, q);
      const T v0 = (T)__shfl_sync(0xffffffffu, myv, q);
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        const VT a0 = r0[lane + 32 * k];
        const T* x0 = reinterpret_cast<const T*>(&a0);
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[k * VEC + u] = fma(v0, x0[u], acc[k * VEC + u]);
      }
    }
  }
}



template <typename T, int NK>
__global__ void __launch_bounds__(qf_threads<NK>(), 1)
    k_qform(CscDev X, int64_t n_cols, const T* __restrict__ Q, int qs, int nblk,
            const T* __restrict__ qn, const short* __restrict__ slot_of,
            const int* __restrict__ hot_rows, int n_hot, int64_t n_rows, int grab,
            unsigned long long skip_above, const int64_t* __restrict__ hlist,
            const unsigned* __restrict__ nh, double* __restrict__ hval,
            unsigned long long* work, double* __restrict__ partial) {
  using VT = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* Qs = reinterpret_cast<T*>(smraw);  // [n_hot][qs]
  for (int64_t e = threadIdx.x; e < (int64_t)n_hot * qs; e += blockDim.x)
    Qs[e] = Q[(int64_t)hot_rows[e / qs] * qs + (e % qs)];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const unsigned long long* xp = reinterpret_cast<const unsigned long long*>(X.colptr);
  // first the heavy columns (more than skip_above nonzeros; `hlist`, in
  // column order), one per warp grab, so no long column is left for the end
  if (hlist) {
    const unsigned nhv = *nh;
    while (true) {
      unsigned h = 0;
      if (lane == 0) h = (unsigned)atomicAdd(work + 1, 1ull);
      h = __shfl_sync(0xffffffffu, h, 0);
      if (h >= nhv) break;
      const int64_t f = hlist[h];
      const unsigned long long a = xp[f], b = xp[f + 1];
      T ss = (T)0;
      for (int cb = 0; cb < nblk; ++cb) {
        T acc[NK * VEC];
#pragma unroll
        for (int k = 0; k < NK * VEC; ++k) acc[k] = (T)0;
        qrows_accumulate<T, NK>(X, Q, qs, (int64_t)cb * NK * 32 * VEC, Qs, slot_of, a, b, 0, 1,
                                acc);
#pragma unroll
        for (int k = 0; k < NK * VEC; ++k) ss = fma(acc[k], acc[k], ss);
      }
      for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) hval[h] = (double)ss;
    }
  }
  while (true) {
    unsigned long long f0 = 0;
    if (lane == 0) f0 = atomicAdd(work, (unsigned long long)grab);
    f0 = __shfl_sync(0xffffffffu, f0, 0);
    if (f0 >= (unsigned long long)n_cols) break;
    // lane l: column f0 + l's range; a one-nonzero column is settled here
    const int64_t fl = lane < grab ? (int64_t)f0 + lane : n_cols;  // lanes past the grab idle
    unsigned long long la = 0, lb = 0;
    T total = (T)0;  // this lane's column; FP32 sums on the FP32 path (GB300's FP64 pipe is narrow)
    if (fl < n_cols) {
      la = xp[fl];
      lb = xp[fl + 1];
      if (lb == la + 1) {
        const T v = (T)X.val[la];
        total = v * v * qn[X.row[la]];
        lb = la;  // done
      } else if (lb - la > skip_above) {
        lb = la;  // a heavy column: done first, or by the split kernels
      }
    }
    // columns with two or more nonzeros, one at a time
    unsigned todo = __ballot_sync(0xffffffffu, lb > la);
    while (todo) {
      const int e = __ffs(todo) - 1;
      todo &= todo - 1;
      const unsigned long long a = __shfl_sync(0xffffffffu, la, e);
      const unsigned long long b = __shfl_sync(0xffffffffu, lb, e);
      T ss = (T)0;
      for (int cb = 0; cb < nblk; ++cb) {  // column blocks of NK * 32 * VEC
      const int64_t coff = (int64_t)cb * NK * 32 * VEC;
      T acc[NK * VEC];
#pragma unroll
      for (int k = 0; k < NK * VEC; ++k) acc[k] = (T)0;
      qrows_accumulate<T, NK>(X, Q, qs, coff, Qs, slot_of, a, b, 0, 1, acc);
#pragma unroll
      for (int k = 0; k < NK * VEC; ++k) ss = fma(acc[k], acc[k], ss);
      }
      for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == e) total += ss;  // lane e owns column f0 + e
    }
    for (int o = 16; o; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
    if (lane == 0) partial[f0 / grab] = (double)total;
  }
}

// fixed-order two-level sum: block b adds its contiguous range of `in`
// (FP64 adds spread over many SMs: GB300's FP64 pipe is narrow)
__global__ void k_sum_f64_ranges(const double* __restrict__ in, int64_t n, int64_t per,
                                 double* __restrict__ out) {
  __shared__ double part[32];
  const int64_t a = (int64_t)blockIdx.x * per, b = min(n, a + per);
  double acc = 0.0;
  for (int64_t e = a + threadIdx.x; e < b; e += blockDim.x) acc += in[e];
  for (int w = 16; w; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    out[blockIdx.x] = t;
  }
}

// fixed-order sum of n doubles (one block)
__global__ void k_sum_f64_fixed(const double* __restrict__ in, int64_t n, double* out) {
  __shared__ double part[32];
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc += in[e];
  for (int w = 16; w; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    *out = t;
  }
}

__global__ void k_add2(const double* __restrict__ a, const double* __restrict__ b, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = *a + *b;
}

// *out = sum of n doubles, in an order fixed by n alone
ctd_status sum_f64(const double* in, int64_t n, double* out, Arena& scratch,
                          cudaStream_t st) {
  if (n <= 8192) {
    CTD_LAUNCH(k_sum_f64_fixed, (1), (1024), 0, st, in, n, out);
    return CTD_OK;
  }
  const int64_t nb = std::min<int64_t>(num_sms() * 2, (n + 1023) / 1024);
  const int64_t per = (n + nb - 1) / nb;
  double* mid;
  CTD_TRY(scratch.get(&mid, nb));
  CTD_LAUNCH(k_sum_f64_ranges, ((unsigned)nb), (256), 0, st, in, n, per, mid);
  CTD_LAUNCH(k_sum_f64_fixed, (1), (1024), 0, st, mid, nb, out);
  return CTD_OK;
}

// Columns per warp grab: 32 (one per lane's metadata prefetch) unless that
// would leave most warps idle (few columns, as in one CTD-D slice).
static int qform_grab(int64_t n_cols, int64_t warps) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(32, n_cols / std::max<int64_t>(warps * 4, 1)));
}

template <typename T, int NK>
static ctd_status qform_launch(const CscDev& X, int64_t n_cols, const T* Q, int qs, int nblk,
                               const T* qn, const short* slot_of, const int* hot, int n_hot,
                               int64_t n_rows, unsigned long long* work, double** partial,
                               int64_t* nparts, Arena& scratch, cudaStream_t st,
                               unsigned long long skip_above = ~0ull,
                               const int64_t* hlist = nullptr, const unsigned* nh = nullptr,
                               double* hval = nullptr) {
  const size_t smem = (size_t)n_hot * qs * sizeof(T);
  if (smem > 48 * 1024)
    CTD_TRY(allow_max_smem((const void*)k_qform<T, NK>));
  int per_sm = 0;
  constexpr int QF_THREADS = qf_threads<NK>();
  CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qform<T, NK>, QF_THREADS,
                                                         smem));
  if (per_sm < 1) return fail(CTD_ECUDA, "error kernel does not fit on an SM");
  const int64_t blocks = (int64_t)num_sms() * per_sm;
  const int grab = qform_grab(n_cols, blocks * (QF_THREADS / 32));
  *nparts = (n_cols + grab - 1) / grab;
  CTD_TRY(scratch.get(partial, *nparts));
  CTD_CUDA(cudaMemsetAsync(*partial, 0, *nparts * sizeof(double), st));
  CTD_LAUNCH((k_qform<T, NK>), (blocks), (QF_THREADS), smem, st, X, n_cols, Q, qs, nblk,
             qn, slot_of, hot, n_hot, n_rows, grab, skip_above, hlist, nh, hval, work, *partial);
  return CTD_OK;
}

// Columns with many nonzeros, split over blocks.  y_f = sum_p v_p Q(i_p, :)
// over the column's entries (Q by rows: row i at Qt + i * ld, d entries);
// block (h, s) forms the partial over the s-th of HS contiguous slices of
// heavy column list[h]'s entries, then one block per column adds the HS
// partials in order and either stores y_f (W(:, c), c = the column's index)
// or adds ||y_f||^2 to out[h].  Fixed order throughout.
constexpr int HS = 16;

__global__ void __launch_bounds__(256)
    k_heavy_partial(const int64_t* __restrict__ list, const unsigned* __restrict__ nlist,
                    const unsigned long long* __restrict__ cptr, const int32_t* __restrict__ crow,
                    const int32_t* __restrict__ cval, const double* __restrict__ Qt, int64_t ld,
                    int64_t d, double* __restrict__ P) {
  const unsigned h = blockIdx.x;
  if (h >= *nlist) return;
  const int s = blockIdx.y;
  const int64_t f = list[h];
  const unsigned long long a = cptr[f], b = cptr[f + 1];
  const unsigned long long len = b - a, chunk = (len + HS - 1) / HS;
  const unsigned long long p0 = a + min(len, chunk * s), p1 = a + min(len, chunk * (s + 1));
  double* out = P + ((int64_t)h * HS + s) * d;
  for (int64_t r0 = 0; r0 < d; r0 += 4 * (int64_t)blockDim.x) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (unsigned long long p = p0; p < p1; ++p) {
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
      if (r < d) out[r] = acc[u];
    }
  }
}

__global__ void __launch_bounds__(256)
    k_heavy_finish(const int64_t* __restrict__ list, const unsigned* __restrict__ nlist,
                   const double* __restrict__ P, int64_t d, double* __restrict__ W,
                   double* __restrict__ norms) {
  __shared__ double part[8];
  const unsigned h = blockIdx.x;
  if (h >= *nlist) return;
  const int64_t f = list[h];
  double ss = 0.0;
  for (int64_t r = threadIdx.x; r < d; r += blockDim.x) {
    double y = 0.0;
#pragma unroll
    for (int s = 0; s < HS; ++s) y += P[((int64_t)h * HS + s) * d + r];
    if (W) W[r + f * d] = y;
    ss = fma(y, y, ss);
  }
  if (!norms) return;
  for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    norms[h] = t;
  }
}

ctd_status launch_heavy_columns(const int64_t* list, const unsigned* nlist, int64_t max_heavy,
                                const uint64_t* cptr, const int32_t* crow, const int32_t* cval,
                                const double* Qt, int64_t ld, int64_t d, double* W,
                                double* norms, Arena& scratch, cudaStream_t st) {
  if (max_heavy <= 0 || d <= 0) return CTD_OK;
  double* P;
  CTD_TRY(scratch.get(&P, (size_t)max_heavy * HS * d));
  CTD_LAUNCH(k_heavy_partial, (dim3((unsigned)max_heavy, HS)), (256), 0, st, list, nlist,
             reinterpret_cast<const unsigned long long*>(cptr), crow, cval, Qt, ld, d, P);
  CTD_LAUNCH(k_heavy_finish, ((unsigned)max_heavy), (256), 0, st, list, nlist, P, d, W, norms);
  return CTD_OK;
}

// ||Q^T X_(alpha)||_F^2 for a dense FP64 Q given by rows (row i at
// Q + i * ld, ld a multiple of 512, entries past the used width zero) and
// its row norms qn; no shared-memory staging.
ctd_status launch_qform_rows(const CscDev& X, int64_t n_cols, int64_t nnz, const double* Q,
                             int64_t ld, int64_t width, const double* qn, int64_t n_rows,
                             double* out, Arena& scratch, cudaStream_t st) {
  CTD_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
  if (width <= 0 || n_cols <= 0) return CTD_OK;
  if (ld % 512 != 0 || ld < width) return fail(CTD_EINVAL, "Q row stride must be a multiple of 512");
  const int nblk = (int)((width + 255) / 256);  // 256 columns (4 loads per lane) per block
  // columns with more than HEAVY_SPLIT nonzeros go to the split kernels
  constexpr unsigned long long HEAVY_SPLIT = 256;
  const int64_t max_heavy = std::min<int64_t>(n_cols, nnz / (int64_t)(HEAVY_SPLIT + 1));
  unsigned long long* work;
  double* partial = nullptr;
  int64_t nchunks = 0;
  CTD_TRY(scratch.get(&work, 1));
  CTD_CUDA(cudaMemsetAsync(work, 0, 8, st));
  CTD_TRY((qform_launch<double, 4>(X, n_cols, Q, (int)ld, nblk, qn, nullptr, nullptr, 0, n_rows,
                                   work, &partial, &nchunks, scratch, st,
                                   max_heavy > 0 ? HEAVY_SPLIT : ~0ull)));
  if (max_heavy > 0) {
    int64_t* hl;
    unsigned* nh;
    double* all;  // the light partials, then one value per heavy column
    CTD_TRY(scratch.get(&hl, max_heavy));
    CTD_TRY(scratch.get(&nh, 1));
    CTD_TRY(scratch.get(&all, nchunks + max_heavy));
    CTD_CUDA(cudaMemsetAsync(nh, 0, sizeof(unsigned), st));
    CTD_CUDA(cudaMemsetAsync(all, 0, (nchunks + max_heavy) * sizeof(double), st));
    CTD_CUDA(cudaMemcpyAsync(all, partial, nchunks * sizeof(double), cudaMemcpyDeviceToDevice, st));
    launch_list_columns_nnz(X.colptr, n_cols, HEAVY_SPLIT + 1, hl, nh, st);
    CTD_TRY(launch_heavy_columns(hl, nh, max_heavy, X.colptr, X.row, X.val, Q, ld, width,
                                 nullptr, all + nchunks, scratch, st));
    partial = all;
    nchunks += max_heavy;
  }
  CTD_TRY(sum_f64(partial, nchunks, out, scratch, st));
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

// The columns with more than `minc` - 1 nonzeros, in ascending order: a
// count per 4096-column tile, an exclusive scan of the counts, then each
// tile writes its columns in order (deterministic, unlike atomic appends).
constexpr int HL_TILE = 4096;

__global__ void k_tile_counts(const unsigned long long* __restrict__ colptr, int64_t n_cols,
                              unsigned long long minc, unsigned* __restrict__ tcount) {
  __shared__ unsigned c;
  const int64_t t = blockIdx.x;
  if (threadIdx.x == 0) c = 0;
  __syncthreads();
  unsigned mine = 0;
  for (int64_t f = t * HL_TILE + threadIdx.x; f < min(n_cols, (t + 1) * HL_TILE); f += blockDim.x)
    mine += (colptr[f + 1] - colptr[f] >= minc);
  atomicAdd(&c, mine);
  __syncthreads();
  if (threadIdx.x == 0) tcount[t] = c;
}

__global__ void k_tile_write(const unsigned long long* __restrict__ colptr, int64_t n_cols,
                             unsigned long long minc, const unsigned long long* __restrict__ toff,
                             int64_t* __restrict__ list) {
  // one warp walks the tile in order; ballots keep the order inside it
  const int lane = threadIdx.x & 31;
  const int64_t t = blockIdx.x;
  unsigned long long pos = toff[t];
  for (int64_t f0 = t * HL_TILE; f0 < min(n_cols, (t + 1) * HL_TILE); f0 += 32) {
    const int64_t f = f0 + lane;
    const bool h = f < n_cols && colptr[f + 1] - colptr[f] >= minc;
    const unsigned m = __ballot_sync(0xffffffffu, h);
    if (h) list[pos + __popc(m & ((1u << lane) - 1))] = f;
    pos += __popc(m);
  }
}

__global__ void k_u64_to_u32(const unsigned long long* __restrict__ in, unsigned* out);

static ctd_status ordered_heavy_list(const uint64_t* colptr, int64_t n_cols, uint64_t minc,
                                     int64_t* list, unsigned* count, Arena& scratch,
                                     cudaStream_t st) {
  const int64_t tiles = (n_cols + HL_TILE - 1) / HL_TILE;
  unsigned* tc;
  uint64_t* toff;
  uint64_t* tmp;
  unsigned* status;
  CTD_TRY(scratch.get(&tc, tiles));
  CTD_TRY(scratch.get(&toff, tiles + 1));
  CTD_TRY(scratch.get(&tmp, scan_tmp_elems(tiles)));
  CTD_TRY(scratch.get(&status, 1));
  CTD_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
  CTD_LAUNCH(k_tile_counts, ((unsigned)tiles), (256), 0, st,
             reinterpret_cast<const unsigned long long*>(colptr), n_cols,
             (unsigned long long)minc, tc);
  launch_scan_u32(tc, toff, tiles, false, tmp, status, st);
  CTD_LAUNCH(k_tile_write, ((unsigned)tiles), (32), 0, st,
             reinterpret_cast<const unsigned long long*>(colptr), n_cols,
             (unsigned long long)minc, reinterpret_cast<const unsigned long long*>(toff), list);
  CTD_LAUNCH(k_u64_to_u32, (1), (32), 0, st, reinterpret_cast<const unsigned long long*>(toff) + tiles, count);
  return CTD_OK;
}

__global__ void k_u64_to_u32(const unsigned long long* __restrict__ in, unsigned* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = (unsigned)*in;
}

// Rows of X with the most nonzeros, chosen on the device: a histogram of
// min(count, HOT_BINS - 1), the smallest count L >= 1 with at most n_hot
// rows at or above it, and slots for those rows.
constexpr int HOT_BINS = 65536;

__global__ void k_hot_hist(const uint32_t* __restrict__ cnt, int64_t n, unsigned* __restrict__ hist) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (cnt[i]) atomicAdd(hist + min(cnt[i], (uint32_t)(HOT_BINS - 1)), 1u);
}

__global__ void __launch_bounds__(1024)
    k_hot_threshold(const unsigned* __restrict__ hist, int n_hot, int* __restrict__ thr) {
  constexpr int PER = HOT_BINS / 1024;
  __shared__ unsigned suf[1024];  // suf[g] = rows in groups >= g
  __shared__ int gstar;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  unsigned s = 0;
  for (int b = 0; b < PER; ++b) s += hist[t * PER + b];
  // inclusive suffix sum over the 1024 groups: within warps, then across
  unsigned x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_down_sync(0xffffffffu, x, o);
    if (lane + o < 32) x += y;
  }
  __shared__ unsigned wsum[32];
  if (lane == 0) wsum[warp] = x;  // the warp's total
  __syncthreads();
  unsigned later = 0;
  for (int w = warp + 1; w < 32; ++w) later += wsum[w];
  suf[t] = x + later;
  if (t == 0) gstar = 1024;
  __syncthreads();
  // the lowest group g whose suffix still fits in n_hot
  if (suf[t] <= (unsigned)n_hot && (t == 0 || suf[t - 1] > (unsigned)n_hot)) gstar = t;
  __syncthreads();
  if (t == 0) {
    const int g = gstar;  // groups >= g fit entirely
    unsigned above = g < 1024 ? suf[g] : 0;
    int L = g < 1024 ? g * PER : HOT_BINS;
    if (g > 0)
      for (int b = g * PER - 1; b >= (g - 1) * PER; --b) {
        if (above + hist[b] > (unsigned)n_hot) break;
        above += hist[b];
        L = b;
      }
    thr[0] = max(L, 1);
  }
}

__global__ void k_hot_assign(const uint32_t* __restrict__ cnt, int64_t n, const int* __restrict__ thr,
                             int n_hot, short* __restrict__ slot, int* __restrict__ hot,
                             int* __restrict__ used) {
  const uint32_t L = (uint32_t)thr[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (min(cnt[i], (uint32_t)(HOT_BINS - 1)) >= L) {
      const int s = atomicAdd(used, 1);
      if (s < n_hot) {
        slot[i] = (short)s;
        hot[s] = (int)i;
      }
    }
}

ctd_status launch_error_qform(const CscDev& X, int64_t n_cols, int64_t n_rows, int64_t X_nnz,
                              const CsrDev& R, const double* Z, int64_t ldz,
                              const uint32_t* rowcnt, int fp32, double* out, Arena& scratch,
                              cudaStream_t st) {
  CTD_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
  if (R.width <= 0 || n_cols <= 0) return CTD_OK;
  const size_t tsz = fp32 ? 4 : 8;
  const int span = 32 * (16 / (int)tsz);        // columns per 16-byte load across a warp
  int NK = (R.width + span - 1) / span;
  int nblk = 1;
  if (NK > 8) {  // wider than one register block: column blocks of 8 loads per lane
    nblk = (NK + 7) / 8;
    NK = 8;
  }
  NK = NK <= 1 ? 1 : NK <= 2 ? 2 : NK <= 4 ? 4 : 8;  // the kernel's compiled widths
  const int qs = nblk * NK * span;              // each Q row holds exactly NK loads per lane per block
  void *Q, *qn;
  double* partial = nullptr;
  int64_t nchunks = 0;
  short* slot_of;
  int* hot;
  unsigned long long* work;
  CTD_TRY(scratch.get(reinterpret_cast<unsigned char**>(&Q), (size_t)n_rows * qs * tsz));
  CTD_TRY(scratch.get(reinterpret_cast<unsigned char**>(&qn), (size_t)n_rows * tsz));
  CTD_TRY(scratch.get(&slot_of, n_rows));
  CTD_TRY(scratch.get(&work, 2));
  // hot rows (one register block wide only): as many as fit in ~200 KB of
  // shared memory (one block per SM; 100 KB each for two blocks at NK = 8),
  // or in the "qform_hot_kb" knob's budget when that is smaller
  const size_t budget = (size_t)std::min<int64_t>(tuning(TUNE_QFORM_HOT), NK >= 8 ? 100 : 200) * 1024;
  int n_hot = nblk == 1 ? (int)std::min<int64_t>((int64_t)(budget / ((size_t)qs * tsz)), n_rows)
                        : 0;
  CTD_TRY(scratch.get(&hot, std::max(n_hot, 1)));
  // the n_hot rows with the most nonzeros (ties by a threshold on the count:
  // rows at or above the smallest count that keeps the set within n_hot)
  CTD_CUDA(cudaMemsetAsync(slot_of, 0xff, n_rows * sizeof(short), st));  // -1
  CTD_CUDA(cudaMemsetAsync(hot, 0, std::max(n_hot, 1) * sizeof(int), st));  // unused slots: row 0
  if (n_hot > 0) {
    unsigned* hist;
    int *thr, *cnt;
    CTD_TRY(scratch.get(&hist, HOT_BINS));
    CTD_TRY(scratch.get(&thr, 1));
    CTD_TRY(scratch.get(&cnt, 1));
    CTD_CUDA(cudaMemsetAsync(hist, 0, HOT_BINS * sizeof(unsigned), st));
    CTD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), st));
    const unsigned g = grid_for(n_rows, 256, (int64_t)num_sms() * 4);
    CTD_LAUNCH(k_hot_hist, (g), (256), 0, st, rowcnt, n_rows, hist);
    CTD_LAUNCH(k_hot_threshold, (1), (1024), 0, st, hist, n_hot, thr);
    CTD_LAUNCH(k_hot_assign, (g), (256), 0, st, rowcnt, n_rows, thr, n_hot, slot_of, hot, cnt);
  }
  CTD_CUDA(cudaMemsetAsync(work, 0, 16, st));
  const unsigned gq = grid_for(n_rows * (qs / 64) * 32, 256, (int64_t)num_sms() * 16);
  const unsigned gn = grid_for(n_rows * 32, 256, (int64_t)num_sms() * 8);
  if (fp32) {
    CTD_LAUNCH(k_build_q<float>, (gq), (256), 0, st, R, n_rows, Z, ldz, qs,
               static_cast<float*>(Q));
    CTD_LAUNCH(k_q_rownorms<float>, (gn), (256), 0, st, static_cast<const float*>(Q), n_rows, qs,
               static_cast<float*>(qn));
  } else {
    CTD_LAUNCH(k_build_q<double>, (gq), (256), 0, st, R, n_rows, Z, ldz, qs,
               static_cast<double*>(Q));
    CTD_LAUNCH(k_q_rownorms<double>, (gn), (256), 0, st, static_cast<const double*>(Q), n_rows,
               qs, static_cast<double*>(qn));
  }
  // columns with more than QF_HEAVY nonzeros go first (a list in column
  // order, one value each), then the rest; both sums in a fixed order
  constexpr unsigned long long QF_HEAVY = 256;
  const int64_t max_heavy = std::max<int64_t>(1, std::min<int64_t>(n_cols, (int64_t)(X_nnz / (QF_HEAVY + 1))));
  int64_t* hlist;
  unsigned* nh;
  double* hval;
  CTD_TRY(scratch.get(&hlist, max_heavy));
  CTD_TRY(scratch.get(&nh, 1));
  CTD_TRY(scratch.get(&hval, max_heavy));
  CTD_CUDA(cudaMemsetAsync(hval, 0, max_heavy * sizeof(double), st));
  CTD_TRY(ordered_heavy_list(X.colptr, n_cols, QF_HEAVY + 1, hlist, nh, scratch, st));
  ctd_status rc;
#define QF(NKV)                                                                                 \
  rc = fp32 ? qform_launch<float, NKV>(X, n_cols, static_cast<const float*>(Q), qs, nblk,     \
                                       static_cast<const float*>(qn), slot_of, hot, n_hot,     \
                                       n_rows, work, &partial, &nchunks, scratch, st, QF_HEAVY, \
                                       hlist, nh, hval)                                         \
            : qform_launch<double, NKV>(X, n_cols, static_cast<const double*>(Q), qs, nblk,    \
                                        static_cast<const double*>(qn), slot_of, hot, n_hot,   \
                                        n_rows, work, &partial, &nchunks, scratch, st,         \
                                        QF_HEAVY, hlist, nh, hval)
  if (NK <= 1) {
    QF(1);
  } else if (NK <= 2) {
    QF(2);
  } else if (NK <= 4) {
    QF(4);
  } else {
    QF(8);
  }
#undef QF
  CTD_TRY(rc);
  double* two;
  CTD_TRY(scratch.get(&two, 2));
  CTD_TRY(sum_f64(partial, nchunks, two, scratch, st));
  CTD_TRY(sum_f64(hval, max_heavy, two + 1, scratch, st));
  CTD_LAUNCH(k_add2, (1), (32), 0, st, two, two + 1, out);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}


}  // namespace ctd
