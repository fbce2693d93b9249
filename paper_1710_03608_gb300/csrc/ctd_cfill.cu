// C = R^T X_(alpha) (Algorithm 1 line 16, Eq. 3) with register accumulators.
//
// On count data the products are dominated by a few long rows of R (the
// frequent mode-alpha indices occur in many sampled fibers): on a Zipf(1.2)
// traffic tensor with 10^7 nonzeros and s~ = 456, the 100 longest of 8.5K
// nonempty rows carry 95% of the 1.5 * 10^9 products.  Walking such a row
// costs two global loads and one shared-memory atomic per product.  Here the
// H longest rows live densely in shared memory (int32, padded to NQ * 128
// columns), and lane l of a warp owns output rows m = 128 q + 4 l + {0..3}
// in registers: one dense row adds into them with NQ 128-bit shared loads
// and 4 NQ integer multiply-adds, no atomics.  The other rows go through the
// sparse walk into a per-warp shared accumulator as before, and the emission
// adds the two, compacts the nonzeros of each 128-row slab with a warp scan
// and writes them in ascending row order.
//
// Exactness: every partial sum is an integer of magnitude at most
// ||x_f|| ||r_m|| <= ||X||_F^2 < 2^31 (Cauchy-Schwarz); this path is taken
// only then.  Which rows are dense changes the order of integer additions
// only, so the result does not depend on the selection.
#include <algorithm>

#include "ctd_expand.cuh"
#include "ctd_internal.cuh"

namespace ctd {

namespace {

constexpr int CF_THREADS = 1024;  // one block per SM shares one copy of the dense rows
constexpr int CF_HEAVY_COL = 128;  // columns with at least this many nonzeros: one block each
constexpr int CF_LONG_ROW = 16;    // sparse rows at least this long: walked by the whole warp
constexpr int CF_MAX_DENSE = 64;   // dense rows at most

// --- selection of the dense rows -------------------------------------------
// hist[len] = number of rows of R with len entries (len >= minlen, capped at width)
__global__ void k_row_len_hist(const unsigned long long* __restrict__ rowptr, int64_t n_rows,
                               int minlen, int width, unsigned* __restrict__ hist) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int len = (int)min(rowptr[i + 1] - rowptr[i], (unsigned long long)width);
    if (len >= minlen) atomicAdd(hist + len, 1u);
  }
}

// thr[0] = the smallest length L >= minlen with #rows(len >= L) <= hmax
// (width + 1 if none qualifies)
__global__ void k_pick_len(const unsigned* __restrict__ hist, int width, int minlen, int hmax,
                           int* __restrict__ thr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned above = 0;
  int L = width + 1;
  for (int len = width; len >= minlen; --len) {
    if (above + hist[len] > (unsigned)hmax) break;
    above += hist[len];
    L = len;
  }
  thr[0] = L;
}

// slot[i] in [0, H) for the rows with len >= thr, -1 otherwise; rows[slot] = i
__global__ void k_assign_slots(const unsigned long long* __restrict__ rowptr, int64_t n_rows,
                               int width, const int* __restrict__ thr, int* __restrict__ slot,
                               int* __restrict__ rows, int* __restrict__ count) {
  const int L = thr[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int len = (int)min(rowptr[i + 1] - rowptr[i], (unsigned long long)width);
    int s = -1;
    if (len >= L) {
      s = (int)atomicAdd(reinterpret_cast<unsigned*>(count), 1u);
      rows[s] = (int)i;
    }
    slot[i] = s;
  }
}

struct Dense {
  const int* slot;   // per row of R
  const int* rows;   // per slot
  const int* count;  // number of dense rows (device)
  int hmax;          // shared memory is sized for this many
};

// Fill the dense rows (H x W ints at `dense`) and zero `acc_n` ints at `acc`.
__device__ __forceinline__ void load_dense(const CsrDev& R, const Dense& dn, int* dense, int W,
                                           int* acc, int acc_n) {
  const int H = min(*dn.count, dn.hmax);
  for (int e = threadIdx.x; e < H * W; e += blockDim.x) dense[e] = 0;
  for (int e = threadIdx.x; e < acc_n; e += blockDim.x) acc[e] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  for (int h = warp; h < H; h += nw) {
    const int i = dn.rows[h];
    for (unsigned long long p = rp[i] + lane; p < rp[i + 1]; p += 32)
      dense[h * W + __ldg(R.col + p)] = __ldg(R.val + p);
  }
  __syncthreads();
}


// Accumulate R^T x_f: dense rows into regs (lane's rows 128 q + 4 lane + k),
// other rows into the shared accumulator acc (atomics).  Warps of a group
// [gwarp, gwarp + gwarps) take interleaved 32-entry chunks of the column.
template <int NQ>
__device__ __forceinline__ void accumulate_reg(const CscDev& X, const CsrDev& R, const Dense& dn,
                                               const int4* __restrict__ dense4, int64_t f,
                                               int* acc, int (&regs)[4 * NQ], int gwarp,
                                               int gwarps) {
  constexpr int W4 = NQ * 32;  // int4 per dense row
  const unsigned long long a = X.colptr[f], b = X.colptr[f + 1];
  const int lane = threadIdx.x & 31;
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  for (unsigned long long p0 = a + (unsigned long long)gwarp * 32; p0 < b;
       p0 += (unsigned long long)gwarps * 32) {
    const unsigned long long p = p0 + lane;
    unsigned long long rs = 0;
    int rl = 0, v = 0, sl = -1;
    if (p < b) {
      const int i = __ldg(X.row + p);
      v = __ldg(X.val + p);
      sl = __ldg(dn.slot + i);
      if (sl < 0) {
        rs = __ldg(rp + i);
        rl = (int)(__ldg(rp + i + 1) - rs);
      }
    }
    unsigned dense_b = __ballot_sync(0xffffffffu, sl >= 0);
    while (dense_b) {
      const int src = __ffs(dense_b) - 1;
      dense_b &= dense_b - 1;
      const int h = __shfl_sync(0xffffffffu, sl, src);
      const int vs = __shfl_sync(0xffffffffu, v, src);
      const int4* d = dense4 + h * W4 + lane;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int4 x = d[q * 32];
        regs[4 * q + 0] += vs * x.x;
        regs[4 * q + 1] += vs * x.y;
        regs[4 * q + 2] += vs * x.z;
        regs[4 * q + 3] += vs * x.w;
      }
    }
    unsigned longs = __ballot_sync(0xffffffffu, rl >= CF_LONG_ROW);
    while (longs) {
      const int src = __ffs(longs) - 1;
      longs &= longs - 1;
      const unsigned long long s0 = __shfl_sync(0xffffffffu, rs, src);
      const int n = __shfl_sync(0xffffffffu, rl, src);
      const int vs = __shfl_sync(0xffffffffu, v, src);
      // four loads in flight per lane before the atomics
      int q = lane;
      for (; q + 96 < n; q += 128) {
        int c4[4], v4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          c4[u] = __ldg(R.col + s0 + q + 32 * u);
          v4[u] = __ldg(R.val + s0 + q + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) atomicAdd(acc + c4[u], vs * v4[u]);
      }
      for (; q < n; q += 32) atomicAdd(acc + __ldg(R.col + s0 + q), vs * __ldg(R.val + s0 + q));
    }
    if (rl >= CF_LONG_ROW) rl = 0;
    if (__any_sync(0xffffffffu, rl > 0))
      expand_chunk(rs, rl, v, R.col, R.val,
                   [&](int m, long long prod) { atomicAdd(acc + m, (int)prod); });
  }
}

// Emit one column from regs + acc (acc zeroed on the way, regs too): the
// nonzeros of rows [0, W) in ascending order at crow/cval + off.  Returns
// their count (same value in every lane).
template <typename V, int NQ>
__device__ __forceinline__ unsigned emit_reg(int* acc, int (&regs)[4 * NQ], unsigned long long off,
                                             uint16_t* __restrict__ crow, V* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  int4* acc4 = reinterpret_cast<int4*>(acc);
  unsigned pos = 0;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int4 s = acc4[q * 32 + lane];
    acc4[q * 32 + lane] = make_int4(0, 0, 0, 0);
    const int x0 = regs[4 * q] + s.x, x1 = regs[4 * q + 1] + s.y;
    const int x2 = regs[4 * q + 2] + s.z, x3 = regs[4 * q + 3] + s.w;
    regs[4 * q] = regs[4 * q + 1] = regs[4 * q + 2] = regs[4 * q + 3] = 0;
    const int c = (x0 != 0) + (x1 != 0) + (x2 != 0) + (x3 != 0);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long o = off + pos + (unsigned)(incl - c);
    const int m0 = q * 128 + 4 * lane;
    if (x0) { crow[o] = (uint16_t)m0;       cval[o] = (V)x0; ++o; }
    if (x1) { crow[o] = (uint16_t)(m0 + 1); cval[o] = (V)x1; ++o; }
    if (x2) { crow[o] = (uint16_t)(m0 + 2); cval[o] = (V)x2; ++o; }
    if (x3) { crow[o] = (uint16_t)(m0 + 3); cval[o] = (V)x3; }
    pos += (unsigned)total;
  }
  return pos;
}

// One persistent kernel, one 32-warp block per SM.  First the columns with
// at least CF_HEAVY_COL nonzeros (from `list`), a whole block each, the
// largest work items first; then every other column, a warp each, 32 at a
// time from a global counter (lane l prefetches column f0 + l's metadata).
// A column with a single nonzero v in row i and positive values is v R(i, :),
// copied.  The block accumulator of the first part is warp 0's accumulator
// of the second; emission leaves both zero.
template <typename V, int NQ>
__global__ void __launch_bounds__(CF_THREADS, 1)
    k_cf(CscDev X, int64_t n_cols, CsrDev R, Dense dn, const int64_t* __restrict__ list,
         const unsigned* __restrict__ nlist, const unsigned long long* __restrict__ coff,
         unsigned* __restrict__ ccnt, uint16_t* __restrict__ crow, V* __restrict__ cval,
         int positive, unsigned long long* work) {
  extern __shared__ int4 smem4[];
  constexpr int W = NQ * 128;
  int* dense = reinterpret_cast<int*>(smem4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int* accs = dense + (size_t)dn.hmax * W;
  load_dense(R, dn, dense, W, accs, nw * W);
  const int4* dense4 = reinterpret_cast<const int4*>(dense);
  int regs[4 * NQ];
#pragma unroll
  for (int k = 0; k < 4 * NQ; ++k) regs[k] = 0;
  __shared__ unsigned long long fcur;
  __shared__ unsigned wcount[CF_THREADS / 32];
  const int width = R.width;
  {
    int* acc = accs;
    const unsigned long long n = *nlist;
    while (true) {
      if (threadIdx.x == 0) fcur = atomicAdd(work + 1, 1ull);
      __syncthreads();
      const unsigned long long it = fcur;
      __syncthreads();
      if (it >= n) break;
      const int64_t f = list[it];
      accumulate_reg<NQ>(X, R, dn, dense4, f, acc, regs, warp, nw);
      // fold each warp's registers into the block accumulator
  #pragma unroll
      for (int q = 0; q < NQ; ++q)
  #pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (regs[4 * q + k] != 0) atomicAdd(acc + q * 128 + 4 * lane + k, regs[4 * q + k]);
          regs[4 * q + k] = 0;
        }
      __syncthreads();
      // emission: warp w sweeps rows [w * span, (w + 1) * span) after counting
      const int span = (((width + nw - 1) / nw) + 31) & ~31;
      const int m_lo = min(width, warp * span), m_hi = min(width, m_lo + span);
      unsigned cnt = 0;
      for (int m0 = m_lo; m0 < m_hi; m0 += 32) {
        const int m = m0 + lane;
        cnt += __popc(__ballot_sync(0xffffffffu, m < m_hi && acc[m] != 0));
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
        int x = 0;
        if (m < m_hi) {
          x = acc[m];
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
  __syncthreads();
  int* acc = accs + warp * W;
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  const unsigned long long* xp = reinterpret_cast<const unsigned long long*>(X.colptr);
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
    // columns with work here (empty ones are done, heavy ones were done first)
    unsigned todo = __ballot_sync(0xffffffffu, ub > 0 && nx < CF_HEAVY_COL);
    while (todo) {
      const int e = __ffs(todo) - 1;
      todo &= todo - 1;
      const unsigned long long oe = __shfl_sync(0xffffffffu, o, e);
      const int nxe = __shfl_sync(0xffffffffu, nx, e);
      if (nxe == 1 && positive) {
        const unsigned long long rse = __shfl_sync(0xffffffffu, rs, e);
        const int rle = __shfl_sync(0xffffffffu, rl, e);
        const int ve = __shfl_sync(0xffffffffu, vv, e);
        // a copy of R's row: four loads in flight per lane before the stores
        int q = lane;
        for (; q + 96 < rle; q += 128) {
          int c4[4], v4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            c4[u] = __ldg(R.col + rse + q + 32 * u);
            v4[u] = __ldg(R.val + rse + q + 32 * u);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            crow[oe + q + 32 * u] = (uint16_t)c4[u];
            cval[oe + q + 32 * u] = (V)(ve * v4[u]);
          }
        }
        for (; q < rle; q += 32) {
          crow[oe + q] = (uint16_t)__ldg(R.col + rse + q);
          cval[oe + q] = (V)(ve * __ldg(R.val + rse + q));
        }
        if (lane == 0) ccnt[f0 + e] = (unsigned)rle;
        continue;
      }
      accumulate_reg<NQ>(X, R, dn, dense4, (int64_t)f0 + e, acc, regs, 0, 1);
      __syncwarp();
      const unsigned n = emit_reg<V, NQ>(acc, regs, oe, crow, cval);
      __syncwarp();
      if (lane == 0) ccnt[f0 + e] = n;
    }
  }
}

template <typename V, int NQ>
ctd_status cf_launch(const CscDev& X, int64_t n_cols, const CsrDev& R, const Dense& dn,
                     const unsigned long long* coff, uint32_t* ccnt, uint16_t* crow, V* cval,
                     int positive, unsigned long long* work, const int64_t* heavy,
                     const unsigned* nheavy, cudaStream_t st) {
  constexpr int W = NQ * 128;
  const size_t smem = ((size_t)dn.hmax + CF_THREADS / 32) * (size_t)W * sizeof(int);
  CTD_TRY(allow_max_smem((const void*)k_cf<V, NQ>));
  int per_sm = 0;
  CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cf<V, NQ>, CF_THREADS, smem));
  if (per_sm < 1) return fail(CTD_ENOTSUP, "C fill: shared memory for the dense rows too large");
  CTD_LAUNCH((k_cf<V, NQ>), (num_sms() * per_sm), (CF_THREADS), smem, st, X, n_cols, R, dn, heavy,
             nheavy, coff, ccnt, crow, cval, positive, work);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

template <typename V>
ctd_status cf_dispatch(int nq, const CscDev& X, int64_t n_cols, const CsrDev& R, const Dense& dn,
                       const unsigned long long* coff, uint32_t* ccnt, uint16_t* crow, V* cval,
                       int positive, unsigned long long* work, const int64_t* heavy,
                       const unsigned* nheavy, cudaStream_t st) {
  switch (nq) {
    case 1: return cf_launch<V, 1>(X, n_cols, R, dn, coff, ccnt, crow, cval, positive, work, heavy, nheavy, st);
    case 2: return cf_launch<V, 2>(X, n_cols, R, dn, coff, ccnt, crow, cval, positive, work, heavy, nheavy, st);
    case 4: return cf_launch<V, 4>(X, n_cols, R, dn, coff, ccnt, crow, cval, positive, work, heavy, nheavy, st);
    default: return cf_launch<V, 8>(X, n_cols, R, dn, coff, ccnt, crow, cval, positive, work, heavy, nheavy, st);
  }
}

}  // namespace

// C fill with dense long rows and register accumulators; requires
// ||X||_F^2 < 2^31 and s~ <= 1024 (the caller checks).
ctd_status c_fill_dense_rows(const CscDev& X, int64_t n_cols, int64_t n_rows, const CsrDev& R,
                             const uint64_t* coff, uint32_t* ccnt, uint16_t* crow, void* cval,
                             int fp32, int positive, cudaStream_t st) {
  const int width = R.width;
  const int nq0 = (width + 127) / 128;
  const int nq = nq0 <= 1 ? 1 : nq0 <= 2 ? 2 : nq0 <= 4 ? 4 : 8;
  const int W = nq * 128;
  const size_t row_b = (size_t)W * sizeof(int);
  // one block of 32 warps per SM: dense rows + 32 warp accumulators in ~220 KB
  const int budget = 220 * 1024;
  int hmax = (int)(budget / (int64_t)row_b) - CF_THREADS / 32;
  hmax = std::max(0, std::min(hmax, CF_MAX_DENSE));
  const int minlen = std::max(16, 16 * nq);  // shorter rows are cheaper walked sparsely
  Arena a;
  a.st = st;
  unsigned *hist, *nheavy;
  int *thr, *slot, *rows, *count;
  unsigned long long* work;
  int64_t* heavy;
  CTD_TRY(a.get(&hist, width + 1));
  CTD_TRY(a.get(&thr, 1));
  CTD_TRY(a.get(&slot, std::max<int64_t>(n_rows, 1)));
  CTD_TRY(a.get(&rows, std::max(hmax, 1)));
  CTD_TRY(a.get(&count, 1));
  CTD_TRY(a.get(&work, 2));
  CTD_TRY(a.get(&heavy, std::max<int64_t>(n_cols, 1)));
  CTD_TRY(a.get(&nheavy, 1));
  CTD_CUDA(cudaMemsetAsync(hist, 0, (width + 1) * sizeof(unsigned), st));
  CTD_CUDA(cudaMemsetAsync(count, 0, sizeof(int), st));
  CTD_CUDA(cudaMemsetAsync(work, 0, 2 * sizeof(unsigned long long), st));
  CTD_CUDA(cudaMemsetAsync(nheavy, 0, sizeof(unsigned), st));
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  const unsigned g = grid_for(n_rows, 256, (int64_t)num_sms() * 4);
  CTD_LAUNCH(k_row_len_hist, (g), (256), 0, st, rp, n_rows, minlen, width, hist);
  CTD_LAUNCH(k_pick_len, (1), (32), 0, st, hist, width, minlen, hmax, thr);
  CTD_LAUNCH(k_assign_slots, (g), (256), 0, st, rp, n_rows, width, thr, slot, rows, count);
  launch_list_columns(X.colptr, coff, n_cols, CF_HEAVY_COL, heavy, nheavy, st);
  Dense dn{slot, rows, count, hmax};
  const unsigned long long* co = reinterpret_cast<const unsigned long long*>(coff);
  if (fp32)
    return cf_dispatch<float>(nq, X, n_cols, R, dn, co, ccnt, crow, static_cast<float*>(cval),
                              positive, work, heavy, nheavy, st);
  return cf_dispatch<double>(nq, X, n_cols, R, dn, co, ccnt, crow, static_cast<double*>(cval),
                             positive, work, heavy, nheavy, st);
}

}  // namespace ctd
