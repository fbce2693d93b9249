// Sparse products with the factor R:
//   * dense columns  out(:, c) = R^T x_f      (the Gram matrices of the
//     independence filter, Algorithm 1 lines 6-15 / Algorithm 2 lines 6-16),
//   * the sparse core C_(alpha) = R^T X_(alpha) (Algorithm 1 line 16, Eq. 3),
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

namespace ctd {

constexpr int WARP_MODE_MAX_WIDTH = 1024;  // accumulator per warp
constexpr int CTA_MODE_MAX_WIDTH = 24576;  // accumulator per block
constexpr int SPMM_THREADS = 256;

// Expand 32 column entries (one per lane) into their R-row work items and
// apply fn(m, product) to every item.  Lanes without an entry pass rlen=0.
template <typename Fn>
__device__ __forceinline__ void expand_chunk(unsigned long long rstart, int rlen, int v,
                                             const int32_t* __restrict__ rcol,
                                             const int32_t* __restrict__ rval, Fn fn) {
  const int lane = threadIdx.x & 31;
  int incl = rlen;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const int excl = incl - rlen;
  for (int base = 0; base < total; base += 32) {
    const int t = base + lane;
    // owner = smallest lane with incl > t
    int lo = 0, hi = 31;
#pragma unroll
    for (int it = 0; it < 5; ++it) {
      const int mid = (lo + hi) >> 1;
      const int im = __shfl_sync(0xffffffffu, incl, mid);
      if (im > t)
        hi = mid;
      else
        lo = mid + 1;
    }
    const int owner = lo;
    const unsigned long long os = __shfl_sync(0xffffffffu, rstart, owner);
    const int oe = __shfl_sync(0xffffffffu, excl, owner);
    const int ov = __shfl_sync(0xffffffffu, v, owner);
    if (t < total) {
      const unsigned long long q = os + (unsigned long long)(t - oe);
      const int m = __ldg(rcol + q);
      const long long prod = (long long)ov * (long long)__ldg(rval + q);
      fn(m, prod);
    }
  }
}

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

ctd_status launch_spmm_dense(const CscDev& X, const int64_t* fibers, const int* nf_dev,
                             int nf_max, const CsrDev& R, double* out, int64_t ld,
                             cudaStream_t st) {
  if (nf_max <= 0 || R.width <= 0) return CTD_OK;
  if (R.width > CTA_MODE_MAX_WIDTH)
    return fail(CTD_EINVAL, "factor wider than the supported maximum (24576 columns)");
  const size_t smem = (size_t)R.width * sizeof(unsigned long long);
  if (smem > 48 * 1024)
    CTD_CUDA(cudaFuncSetAttribute(k_spmm_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
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
    ub[f] = (unsigned)min(s, (unsigned long long)R.width);
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
// ascending.  Three paths:
//  * a column with one nonzero v in row i (and all values positive) is
//    v * R(i, :), copied from R's row i (rows of R are sorted by column);
//  * other columns with fewer than HEAVY nonzeros: one warp each, with a
//    warp-private accumulator;
//  * heavy columns: a whole block each.
// Accumulators are int32 when ||X||_F^2 < 2^31: by Cauchy-Schwarz every
// partial sum is at most ||x_f|| ||r_m|| <= ||X||_F^2, so int32 is exact.
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
__device__ __forceinline__ long long acc_get(const A* p) {
  return sizeof(A) == 4 ? (long long)(*(const int*)p) : (long long)(*(const unsigned long long*)p);
}

template <typename A>
__device__ __forceinline__ void accumulate_column_t(const CscDev& X, const CsrDev& R, int64_t f,
                                                    A* acc, unsigned* bitmap, int gwarp,
                                                    int gwarps) {
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
      acc_add<A>(acc + m, prod);
      atomicOr(bitmap + (m >> 5), 1u << (m & 31));
    });
  }
}

// Emit the touched entries of one column in ascending row order and reset
// them.  Group = gthreads threads (a warp or the block).
template <typename V, typename A>
__device__ void emit_column_t(A* acc, unsigned* bitmap, int width, int* wpre, int gtid,
                              int gthreads, bool may_cancel, unsigned long long off,
                              int32_t* __restrict__ crow, V* __restrict__ cval, unsigned* count,
                              bool block_group) {
  const int nwords = (width + 31) >> 5;
  const int lane = gtid & 31;
  if (may_cancel) {  // drop exact zeros (only possible with signed inputs)
    for (int w = gtid; w < nwords; w += gthreads) {
      unsigned bits = bitmap[w], keep = bits;
      while (bits) {
        const int bpos = __ffs(bits) - 1;
        bits &= bits - 1;
        if (acc_get<A>(acc + w * 32 + bpos) == 0) keep &= ~(1u << bpos);
      }
      bitmap[w] = keep;
    }
    if (block_group) __syncthreads(); else __syncwarp();
  }
  int carry = 0;
  for (int w0 = 0; w0 < nwords; w0 += gthreads) {
    const int w = w0 + gtid;
    const int c = w < nwords ? __popc(bitmap[w]) : 0;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (block_group) {
      __shared__ int wtot[32];
      const int warp = gtid >> 5;
      if (lane == 31) wtot[warp] = incl;
      __syncthreads();
      int before = 0, all = 0;
      for (int q = 0; q < (gthreads >> 5); ++q) {
        if (q < warp) before += wtot[q];
        all += wtot[q];
      }
      if (w < nwords) wpre[w] = carry + before + incl - c;
      __syncthreads();
      carry += all;
    } else {
      if (w < nwords) wpre[w] = carry + incl - c;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  if (block_group) __syncthreads(); else __syncwarp();
  const int total = carry;
  for (int k = gtid; k < total; k += gthreads) {
    int lo = 0, hi = nwords - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (wpre[mid] <= k)
        lo = mid;
      else
        hi = mid - 1;
    }
    const int bpos = __fns(bitmap[lo], 0, k - wpre[lo] + 1);
    const int m = lo * 32 + bpos;
    crow[off + k] = m;
    cval[off + k] = (V)acc_get<A>(acc + m);
    acc[m] = 0;
  }
  if (block_group) __syncthreads(); else __syncwarp();
  if (may_cancel) {  // dropped zeros were reset already (their value is 0)
  }
  for (int w = gtid; w < nwords; w += gthreads) bitmap[w] = 0;
  if (block_group) __syncthreads(); else __syncwarp();
  if (gtid == 0) *count = (unsigned)total;
}

template <typename V, typename A>
__global__ void __launch_bounds__(SPMM_THREADS)
    k_c_fill_warp(CscDev X, int64_t n_cols, CsrDev R, const unsigned long long* __restrict__ coff,
                  unsigned* __restrict__ ccnt, int32_t* __restrict__ crow, V* __restrict__ cval,
                  int may_cancel, int positive, unsigned long long* work) {
  extern __shared__ unsigned long long smem_u64[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int width = R.width, nwords = (width + 31) >> 5;
  const int accw = (width + 1) & ~1;  // keep 8-byte alignment between warps
  A* acc = reinterpret_cast<A*>(smem_u64) + (size_t)warp * accw;
  unsigned* bitmaps = reinterpret_cast<unsigned*>(reinterpret_cast<A*>(smem_u64) + (size_t)nw * accw);
  unsigned* bitmap = bitmaps + warp * nwords;
  int* wpre = reinterpret_cast<int*>(bitmaps + nw * nwords) + warp * (nwords + 1);
  for (int m = lane; m < width; m += 32) acc[m] = 0;
  for (int w = lane; w < nwords; w += 32) bitmap[w] = 0;
  __syncwarp();
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  constexpr int CHUNK = 64;
  while (true) {
    unsigned long long f0 = 0;
    if (lane == 0) f0 = atomicAdd(work, (unsigned long long)CHUNK);
    f0 = __shfl_sync(0xffffffffu, f0, 0);
    if (f0 >= (unsigned long long)n_cols) break;
    const int64_t f1 = min((int64_t)f0 + CHUNK, n_cols);
    for (int64_t f = (int64_t)f0; f < f1; ++f) {
      const unsigned long long o = coff[f];
      if (coff[f + 1] == o) {
        if (lane == 0) ccnt[f] = 0;
        continue;
      }
      const unsigned long long a = X.colptr[f], b = X.colptr[f + 1];
      if (b - a >= (unsigned long long)HEAVY) continue;  // block kernel
      if (b - a == 1 && positive) {
        const int i = __ldg(X.row + a);
        const long long v = __ldg(X.val + a);
        const unsigned long long rs = __ldg(rp + i), n = __ldg(rp + i + 1) - rs;
        for (unsigned long long q = lane; q < n; q += 32) {
          crow[o + q] = __ldg(R.col + rs + q);
          cval[o + q] = (V)(v * (long long)__ldg(R.val + rs + q));
        }
        if (lane == 0) ccnt[f] = (unsigned)n;
        continue;
      }
      accumulate_column_t<A>(X, R, f, acc, bitmap, 0, 1);
      __syncwarp();
      emit_column_t<V, A>(acc, bitmap, width, wpre, lane, 32, may_cancel != 0, o, crow, cval,
                          ccnt + f, false);
    }
  }
}

template <typename V, typename A>
__global__ void __launch_bounds__(SPMM_THREADS)
    k_c_fill_block(CscDev X, const int64_t* __restrict__ list, const unsigned* __restrict__ nlist,
                   CsrDev R, const unsigned long long* __restrict__ coff,
                   unsigned* __restrict__ ccnt, int32_t* __restrict__ crow, V* __restrict__ cval,
                   int may_cancel, unsigned long long* work) {
  extern __shared__ unsigned long long smem_u64[];
  const int width = R.width, nwords = (width + 31) >> 5;
  A* acc = reinterpret_cast<A*>(smem_u64);
  unsigned* bitmap = reinterpret_cast<unsigned*>(acc + ((width + 1) & ~1));
  int* wpre = reinterpret_cast<int*>(bitmap + nwords);
  __shared__ unsigned long long fcur;
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long n = *nlist;
  for (int m = threadIdx.x; m < width; m += blockDim.x) acc[m] = 0;
  for (int w = threadIdx.x; w < nwords; w += blockDim.x) bitmap[w] = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) fcur = atomicAdd(work, 1ull);
    __syncthreads();
    const unsigned long long it = fcur;
    __syncthreads();
    if (it >= n) break;
    const int64_t f = list[it];
    accumulate_column_t<A>(X, R, f, acc, bitmap, warp, nw);
    __syncthreads();
    emit_column_t<V, A>(acc, bitmap, width, wpre, threadIdx.x, blockDim.x, may_cancel != 0,
                        coff[f], crow, cval, ccnt + f, true);
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

template <typename V, typename A>
static ctd_status c_fill_impl(const CscDev& X, int64_t n_cols, const CsrDev& R,
                              const uint64_t* coff, uint32_t* ccnt, int32_t* crow, V* cval,
                              int may_cancel, int positive, unsigned long long* work,
                              int64_t* heavy, unsigned* nheavy, cudaStream_t st) {
  const int width = R.width, nwords = (width + 31) >> 5;
  const int accw = (width + 1) & ~1;
  const unsigned long long* co = reinterpret_cast<const unsigned long long*>(coff);
  // heavy columns (and, if the warp accumulator would not fit, all columns)
  const bool warp_ok = width <= WARP_MODE_MAX_WIDTH;
  CTD_LAUNCH(k_list_columns, (grid_for(n_cols, 256, (int64_t)num_sms() * 8)), (256), 0, st,
             reinterpret_cast<const unsigned long long*>(X.colptr), co, n_cols,
             warp_ok ? (unsigned long long)HEAVY : 1ull, heavy, nheavy);
  if (warp_ok) {
    const int nw = SPMM_THREADS / 32;
    const size_t smem = (size_t)nw * accw * sizeof(A) + (size_t)nw * nwords * 4 +
                        (size_t)nw * (nwords + 1) * 4;
    if (smem > 48 * 1024)
      CTD_CUDA(cudaFuncSetAttribute(k_c_fill_warp<V, A>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_c_fill_warp<V, A>,
                                                           SPMM_THREADS, smem));
    if (per_sm < 1) per_sm = 1;
    CTD_LAUNCH((k_c_fill_warp<V, A>), (num_sms() * per_sm), (SPMM_THREADS), smem, st, X, n_cols,
               R, co, ccnt, crow, cval, may_cancel, positive, work);
  } else {
    CTD_CUDA(cudaMemsetAsync(ccnt, 0, n_cols * sizeof(uint32_t), st));
  }
  if (width > CTA_MODE_MAX_WIDTH)
    return fail(CTD_EINVAL, "factor wider than the supported maximum (24576 columns)");
  const size_t smem = (size_t)accw * sizeof(A) + (size_t)nwords * 4 + (size_t)(nwords + 1) * 4;
  if (smem > 48 * 1024)
    CTD_CUDA(cudaFuncSetAttribute(k_c_fill_block<V, A>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_c_fill_block<V, A>,
                                                         SPMM_THREADS, smem));
  if (per_sm < 1) per_sm = 1;
  CTD_LAUNCH((k_c_fill_block<V, A>), (num_sms() * per_sm), (SPMM_THREADS), smem, st, X, heavy,
             nheavy, R, co, ccnt, crow, cval, may_cancel, work + 1);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

ctd_status launch_c_fill(const CscDev& X, int64_t n_cols, const CsrDev& R, const uint64_t* coff,
                         uint32_t* ccnt, int32_t* crow, void* cval, int fp32, int may_cancel,
                         int positive, uint64_t sqnorm_X, cudaStream_t st) {
  if (n_cols <= 0) return CTD_OK;
  if (R.width <= 0) {
    CTD_CUDA(cudaMemsetAsync(ccnt, 0, n_cols * sizeof(uint32_t), st));
    return CTD_OK;
  }
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
                                         may_cancel, positive, work, heavy, nheavy, st)
               : c_fill_impl<float, unsigned long long>(X, n_cols, R, coff, ccnt, crow,
                                                        static_cast<float*>(cval), may_cancel,
                                                        positive, work, heavy, nheavy, st);
  else
    rc = small ? c_fill_impl<double, int>(X, n_cols, R, coff, ccnt, crow,
                                          static_cast<double*>(cval), may_cancel, positive, work,
                                          heavy, nheavy, st)
               : c_fill_impl<double, unsigned long long>(X, n_cols, R, coff, ccnt, crow,
                                                         static_cast<double*>(cval), may_cancel,
                                                         positive, work, heavy, nheavy, st);
  dfree(work, st);
  dfree(heavy, st);
  dfree(nheavy, st);
  return rc;
}

// Sort each row of a row-major factor by column (rank by counting; rows are
// short).  One warp per row; in/out arrays differ.
__global__ void k_sort_rows(const unsigned long long* __restrict__ rowptr, int64_t n_rows,
                            const int32_t* __restrict__ col_in, const int32_t* __restrict__ val_in,
                            int32_t* __restrict__ col_out, int32_t* __restrict__ val_out) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n_rows; i += nw) {
    const unsigned long long a = rowptr[i], b = rowptr[i + 1];
    for (unsigned long long p = a + lane; p < b; p += 32) {
      const int m = col_in[p];
      unsigned long long r = 0;
      for (unsigned long long q = a; q < b; ++q) r += (col_in[q] < m);
      col_out[a + r] = m;
      val_out[a + r] = val_in[p];
    }
  }
}

void launch_sort_rows(const uint64_t* rowptr, int64_t n_rows, const int32_t* col_in,
                      const int32_t* val_in, int32_t* col_out, int32_t* val_out, cudaStream_t st) {
  if (n_rows <= 0) return;
  CTD_LAUNCH(k_sort_rows, (grid_for(n_rows * 32, 256, (int64_t)num_sms() * 16)), (256), 0, st,
             reinterpret_cast<const unsigned long long*>(rowptr), n_rows, col_in, val_in, col_out,
             val_out);
}

// ---------------------------------------------------------------------------
// Error numerator in the Q form: ||P_R X||_F^2 = ||Q^T X_(alpha)||_F^2 with
// Q = R L^{-T} (orthonormal columns spanning range(R); L L^T = R^T R, Z =
// L^{-1}).  Q is dense I_alpha x s~, row-major with stride qs (a multiple of
// 32), computed in FP64 and stored as T.  The sum over columns f of
// ||Q^T x_f||^2 costs nnz * s~ multiply-adds; a column with one nonzero v in
// row i contributes v^2 ||Q(i, :)||^2, read from the precomputed row norms.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_build_q(CsrDev R, int64_t n_rows, const double* __restrict__ Z, int64_t ldz,
                          int qs, T* __restrict__ Q, double* __restrict__ qn) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  for (int64_t i = gw; i < n_rows; i += nw) {
    const unsigned long long a = rp[i], b = rp[i + 1];
    double nrm = 0.0;
    for (int c = lane; c < qs; c += 32) {
      double acc = 0.0;
      if (c < R.width)
        for (unsigned long long q = a; q < b; ++q) {
          const int m = R.col[q];
          if (c >= m) acc = fma((double)R.val[q], Z[c + (int64_t)m * ldz], acc);
        }
      const T tv = (T)acc;
      Q[i * qs + c] = tv;
      nrm = fma((double)tv, (double)tv, nrm);
    }
    for (int o = 16; o; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if (lane == 0) qn[i] = nrm;
  }
}

// One warp per column (dynamic chunks).  Hot rows of Q (slot >= 0 in
// `slot_of`) are staged in shared memory once per block.  A column's
// entries are loaded 32 at a time (one per lane) and broadcast by shuffles;
// two Q rows are in flight per step.
template <typename T, int NC>
__device__ __forceinline__ void qrow_fma(const T* __restrict__ qrow, float v, float* acc,
                                         double* accd, int lane, int qs) {
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const int c = lane + 32 * k;
    if (c < qs) {
      if (sizeof(T) == 4)
        acc[k] = fmaf(v, (float)qrow[c], acc[k]);
      else
        accd[k] = fma((double)v, (double)qrow[c], accd[k]);
    }
  }
}

template <typename T, int NC>
__global__ void __launch_bounds__(256)
    k_qform(CscDev X, int64_t n_cols, const T* __restrict__ Q, int qs,
            const double* __restrict__ qn, const short* __restrict__ slot_of,
            const int* __restrict__ hot_rows, int n_hot, int64_t n_rows,
            unsigned long long* work, double* __restrict__ block_sums) {
  extern __shared__ unsigned char smraw[];
  T* Qs = reinterpret_cast<T*>(smraw);                                   // [n_hot][qs]
  short* slot = reinterpret_cast<short*>(smraw + (size_t)n_hot * qs * sizeof(T));  // [n_rows]
  __shared__ double wsum[8];
  for (int64_t e = threadIdx.x; e < (int64_t)n_hot * qs; e += blockDim.x)
    Qs[e] = Q[(int64_t)hot_rows[e / qs] * qs + (e % qs)];
  for (int64_t e = threadIdx.x; e < n_rows; e += blockDim.x) slot[e] = slot_of[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double total = 0.0;
  constexpr int CHUNK = 64;
  while (true) {
    unsigned long long f0 = 0;
    if (lane == 0) f0 = atomicAdd(work, (unsigned long long)CHUNK);
    f0 = __shfl_sync(0xffffffffu, f0, 0);
    if (f0 >= (unsigned long long)n_cols) break;
    const int64_t f1 = min((int64_t)f0 + CHUNK, n_cols);
    for (int64_t f = (int64_t)f0; f < f1; ++f) {
      const unsigned long long a = X.colptr[f], b = X.colptr[f + 1];
      if (b == a) continue;
      if (b == a + 1) {
        const double v = (double)X.val[a];
        if (lane == 0) total = fma(v * v, qn[X.row[a]], total);
        continue;
      }
      float acc[NC];
      double accd[NC];
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        acc[k] = 0.f;
        accd[k] = 0.0;
      }
      for (unsigned long long base = a; base < b; base += 32) {
        const int cnt = (int)min((unsigned long long)32, b - base);
        const T* myrow = nullptr;
        int myv = 0;
        if (lane < cnt) {
          const int i = __ldg(X.row + base + lane);
          myv = __ldg(X.val + base + lane);
          const int sl = slot[i];
          myrow = sl >= 0 ? Qs + (int64_t)sl * qs : Q + (int64_t)i * qs;
        }
        int e = 0;
        for (; e + 1 < cnt; e += 2) {
          const T* r0 = (const T*)__shfl_sync(0xffffffffu, (unsigned long long)myrow, e);
          const T* r1 = (const T*)__shfl_sync(0xffffffffu, (unsigned long long)myrow, e + 1);
          const float v0 = (float)__shfl_sync(0xffffffffu, myv, e);
          const float v1 = (float)__shfl_sync(0xffffffffu, myv, e + 1);
          T q0[NC], q1[NC];
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            const int c = lane + 32 * k;
            q0[k] = c < qs ? r0[c] : (T)0;
            q1[k] = c < qs ? r1[c] : (T)0;
          }
#pragma unroll
          for (int k = 0; k < NC; ++k) {
            if (sizeof(T) == 4) {
              acc[k] = fmaf(v0, (float)q0[k], acc[k]);
              acc[k] = fmaf(v1, (float)q1[k], acc[k]);
            } else {
              accd[k] = fma((double)v0, (double)q0[k], accd[k]);
              accd[k] = fma((double)v1, (double)q1[k], accd[k]);
            }
          }
        }
        if (e < cnt) {
          const T* r0 = (const T*)__shfl_sync(0xffffffffu, (unsigned long long)myrow, e);
          const float v0 = (float)__shfl_sync(0xffffffffu, myv, e);
          qrow_fma<T, NC>(r0, v0, acc, accd, lane, qs);
        }
      }
      double ss = 0.0;
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        const double x = sizeof(T) == 4 ? (double)acc[k] : accd[k];
        ss = fma(x, x, ss);
      }
      for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if (lane == 0) total += ss;
    }
  }
  if (lane == 0) wsum[warp] = total;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    block_sums[blockIdx.x] = t;
  }
}

__global__ void k_sum_f64_small(const double* __restrict__ in, int n, double* out);

template <typename T, int NC>
static ctd_status qform_launch(const CscDev& X, int64_t n_cols, const T* Q, int qs,
                               const double* qn, const short* slot_of, const int* hot, int n_hot,
                               int64_t n_rows, unsigned long long* work, double* block_sums,
                               int* nblocks, cudaStream_t st) {
  const size_t smem = (size_t)n_hot * qs * sizeof(T) + (size_t)n_rows * sizeof(short);
  if (smem > 48 * 1024)
    CTD_CUDA(cudaFuncSetAttribute(k_qform<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  int per_sm = 0;
  CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qform<T, NC>, 256, smem));
  if (per_sm < 1) return fail(CTD_ECUDA, "error kernel does not fit on an SM");
  *nblocks = num_sms() * per_sm;
  CTD_LAUNCH((k_qform<T, NC>), (*nblocks), (256), smem, st, X, n_cols, Q, qs, qn, slot_of, hot,
             n_hot, n_rows, work, block_sums);
  return CTD_OK;
}

ctd_status launch_error_qform(const CscDev& X, int64_t n_cols, int64_t n_rows, const CsrDev& R,
                              const double* Z, int64_t ldz, const uint32_t* rowcnt_host_unused,
                              const int* hot_rows_host, int n_hot_req, int fp32, double* out,
                              Arena& scratch, cudaStream_t st) {
  (void)rowcnt_host_unused;
  CTD_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
  if (R.width <= 0 || n_cols <= 0) return CTD_OK;
  const int qs = (R.width + 31) & ~31;
  const int NCmax = qs / 32;
  if (NCmax > 32) return fail(CTD_ENOTSUP, "error kernel limited to s~ <= 1024");
  const size_t tsz = fp32 ? 4 : 8;
  void* Q;
  double* qn;
  short* slot_of;
  int* hot;
  unsigned long long* work;
  double* bsums;
  CTD_TRY(scratch.get(reinterpret_cast<unsigned char**>(&Q), (size_t)n_rows * qs * tsz));
  CTD_TRY(scratch.get(&qn, n_rows));
  CTD_TRY(scratch.get(&slot_of, n_rows));
  CTD_TRY(scratch.get(&work, 1));
  CTD_TRY(scratch.get(&bsums, 4096));
  // hot rows: as many as fit next to the slot table in ~100 KB of shared
  // memory, so two blocks (16 warps) stay resident per SM
  const size_t budget = 100 * 1024;
  const size_t table = (size_t)n_rows * sizeof(short);
  int n_hot = 0;
  if (table < budget) n_hot = (int)std::min<size_t>((budget - table) / ((size_t)qs * tsz), n_hot_req);
  n_hot = std::max(n_hot, 0);
  CTD_TRY(scratch.get(&hot, std::max(n_hot, 1)));
  std::vector<short> slots(n_rows, (short)-1);
  for (int q = 0; q < n_hot; ++q) slots[hot_rows_host[q]] = (short)q;
  CTD_CUDA(cudaMemcpyAsync(slot_of, slots.data(), n_rows * sizeof(short), cudaMemcpyHostToDevice, st));
  if (n_hot)
    CTD_CUDA(cudaMemcpyAsync(hot, hot_rows_host, n_hot * sizeof(int), cudaMemcpyHostToDevice, st));
  CTD_CUDA(cudaMemsetAsync(work, 0, 8, st));
  const unsigned gq = grid_for(n_rows * 32, 256, (int64_t)num_sms() * 8);
  if (fp32)
    CTD_LAUNCH(k_build_q<float>, (gq), (256), 0, st, R, n_rows, Z, ldz, qs,
               static_cast<float*>(Q), qn);
  else
    CTD_LAUNCH(k_build_q<double>, (gq), (256), 0, st, R, n_rows, Z, ldz, qs,
               static_cast<double*>(Q), qn);
  int nb = 0;
  ctd_status rc;
#define QF(NC)                                                                                  \
  rc = fp32 ? qform_launch<float, NC>(X, n_cols, static_cast<const float*>(Q), qs, qn, slot_of,  \
                                      hot, n_hot, n_rows, work, bsums, &nb, st)                  \
            : qform_launch<double, NC>(X, n_cols, static_cast<const double*>(Q), qs, qn,         \
                                       slot_of, hot, n_hot, n_rows, work, bsums, &nb, st)
  if (NCmax <= 4) {
    QF(4);
  } else if (NCmax <= 8) {
    QF(8);
  } else if (NCmax <= 16) {
    QF(16);
  } else {
    QF(32);
  }
#undef QF
  CTD_TRY(rc);
  if (nb > 4096) return fail(CTD_ECUDA, "too many blocks for the error reduction");
  CTD_LAUNCH(k_sum_f64_small, (1), (1024), 0, st, bsums, nb, out);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

__global__ void k_sum_f64_small(const double* __restrict__ in, int n, double* out) {
  __shared__ double part[32];
  double acc = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) acc += in[e];
  for (int w = 16; w; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    *out = t;
  }
}

// ---------------------------------------------------------------------------
// Quadratic form of a sparse C against U: sum_f c_f^T U c_f  (FP64).  One
// block per column; per-column results then a fixed-order reduction, so the
// sum does not depend on scheduling.
// ---------------------------------------------------------------------------
template <typename V>
__global__ void k_quad_cols(const unsigned long long* __restrict__ coff, const unsigned* __restrict__ ccnt,
                            const int32_t* __restrict__ crow, const V* __restrict__ cval,
                            int64_t n_cols, const double* __restrict__ U, int64_t ldu,
                            double* __restrict__ per_col) {
  __shared__ double part[32];
  for (int64_t f = blockIdx.x; f < n_cols; f += gridDim.x) {
    const unsigned long long o = coff[f];
    const unsigned n = ccnt[f];
    double acc = 0.0;
    for (unsigned p = threadIdx.x; p < n; p += blockDim.x) {
      const int mp = crow[o + p];
      const double vp = (double)cval[o + p];
      const double* Ucol = U + (int64_t)mp * ldu;
      double s = 0.0;
      for (unsigned q = 0; q < n; ++q) s = fma((double)cval[o + q], Ucol[crow[o + q]], s);
      acc = fma(vp, s, acc);
    }
    for (int w = 16; w; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
      per_col[f] = t;
    }
    __syncthreads();
  }
}

__global__ void k_sum_f64(const double* __restrict__ in, int64_t n, double* out) {
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

ctd_status launch_quad_form(const uint64_t* coff, const uint32_t* ccnt, const int32_t* crow,
                            const void* cval, int fp32, int64_t n_cols, const double* U,
                            int64_t ldu, double* out, cudaStream_t st) {
  CTD_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
  if (n_cols <= 0) return CTD_OK;
  double* per_col;
  CTD_TRY(dalloc_n(&per_col, n_cols, st));
  const unsigned g = grid_for(n_cols, 1, (int64_t)num_sms() * 16);
  if (fp32)
    CTD_LAUNCH(k_quad_cols<float>, (g), (256), 0, st,
               reinterpret_cast<const unsigned long long*>(coff), ccnt, crow,
               static_cast<const float*>(cval), n_cols, U, ldu, per_col);
  else
    CTD_LAUNCH(k_quad_cols<double>, (g), (256), 0, st,
               reinterpret_cast<const unsigned long long*>(coff), ccnt, crow,
               static_cast<const double*>(cval), n_cols, U, ldu, per_col);
  CTD_LAUNCH(k_sum_f64, (1), (1024), 0, st, per_col, n_cols, out);
  CTD_CUDA(cudaGetLastError());
  dfree(per_col, st);
  return CTD_OK;
}

}  // namespace ctd
