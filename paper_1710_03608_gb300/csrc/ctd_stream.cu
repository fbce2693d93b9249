// Streaming passes over the COO input: squared column norms (Algorithm 1
// Eq. 1), prefix sums (the column distribution's CDF and the
// counting-sort offsets), the counting-sort scatter into column- and
// row-major layouts (the matricization), and column gathers.
#include <algorithm>
#include <cstdlib>

#include "ctd_internal.cuh"

namespace ctd {

void mode_extents(const int64_t dims[3], int alpha, int64_t* n_rows, int64_t* n_cols) {
  if (alpha == 1) {
    *n_rows = dims[0];
    *n_cols = dims[1] * dims[2];
  } else if (alpha == 2) {
    *n_rows = dims[1];
    *n_cols = dims[0] * dims[2];
  } else {
    *n_rows = dims[2];
    *n_cols = dims[0] * dims[1];
  }
}

static ModeMap make_map(const CooDev& X) { return make_mode_map(X.dims, X.alpha); }

// The COO arrays are read with 16-byte loads (four entries per array per
// load) when all four start on a 16-byte boundary, with the streaming
// cache hint: each entry is read once, and the random-access arrays of the
// pass (counts, cursors, the column-major output) should keep L2.
static bool coo_vec4(const CooDev& X) {
  return ((reinterpret_cast<uintptr_t>(X.i) | reinterpret_cast<uintptr_t>(X.j) |
           reinterpret_cast<uintptr_t>(X.k) | reinterpret_cast<uintptr_t>(X.v)) & 15) == 0;
}

// ---------------------------------------------------------------------------
// K1a: entries per column and per row
// ---------------------------------------------------------------------------
// Row counts go to a per-block shared-memory histogram when the rows fit
// (Zipf sources put ~10% of all nonzeros on one row; global atomics on that
// one address would serialize), then one global add per touched row.
// Column counts are one non-returning 4-byte atomic per entry.
constexpr int NORMS_SMEM_ROWS = 16384;

template <bool VEC>
__global__ void __launch_bounds__(512)
    k_count(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj,
            const int32_t* __restrict__ kk, int64_t nnz, ModeMap mm, int64_t n_rows,
            unsigned* __restrict__ colcnt, unsigned* __restrict__ rowcnt, unsigned* status) {
  extern __shared__ unsigned rowhist[];
  const bool priv = n_rows <= NORMS_SMEM_ROWS;
  if (priv) {
    for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x) rowhist[r] = 0;
    __syncthreads();
  }
  bool bad = false;
  auto one = [&](int32_t a, int32_t b, int32_t c) {
    int32_t row;
    int64_t col;
    if (!mm.map(a, b, c, &row, &col)) {
      bad = true;
      return;
    }
    atomicAdd(colcnt + col, 1u);
    if (priv)
      atomicAdd(rowhist + row, 1u);
    else
      atomicAdd(rowcnt + row, 1u);
  };
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t tail0 = 0;
  if (VEC) {
    const int64_t nq = nnz >> 2;
    for (int64_t q = gt; q < nq; q += stride) {
      const int4 a = __ldcs(reinterpret_cast<const int4*>(ii) + q);
      const int4 b = __ldcs(reinterpret_cast<const int4*>(jj) + q);
      const int4 c = __ldcs(reinterpret_cast<const int4*>(kk) + q);
      one(a.x, b.x, c.x);
      one(a.y, b.y, c.y);
      one(a.z, b.z, c.z);
      one(a.w, b.w, c.w);
    }
    tail0 = nq << 2;
  }
  for (int64_t e = tail0 + gt; e < nnz; e += stride) one(__ldcs(ii + e), __ldcs(jj + e), __ldcs(kk + e));
  if (bad) atomicOr(status, DEV_BAD_INDEX);
  if (priv) {
    __syncthreads();
    for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x)
      if (rowhist[r]) atomicAdd(rowcnt + r, rowhist[r]);
  }
}

void launch_count(const CooDev& X, uint32_t* colcnt, uint32_t* rowcnt, unsigned* status,
                  cudaStream_t st) {
  if (X.nnz == 0) return;
  const int bs = 512;
  int64_t n_rows, n_cols;
  mode_extents(X.dims, X.alpha, &n_rows, &n_cols);
  const bool priv = n_rows <= NORMS_SMEM_ROWS;
  const size_t smem = priv ? (size_t)n_rows * 4 : 0;
  const bool vec = coo_vec4(X);
  const void* fn = vec ? (const void*)k_count<true> : (const void*)k_count<false>;
  if (smem > 48 * 1024) allow_max_smem(fn);
  // 4 entries per thread on the vector path; at most 2 blocks per SM (the
  // row histogram is zeroed and flushed once per block)
  const unsigned g = grid_for((X.nnz + 3) / (vec ? 4 : 1), bs, (int64_t)num_sms() * 2);
  if (vec)
    CTD_LAUNCH(k_count<true>, (g), (bs), smem, st, X.i, X.j, X.k, X.nnz, make_map(X), n_rows,
               colcnt, rowcnt, status);
  else
    CTD_LAUNCH(k_count<false>, (g), (bs), smem, st, X.i, X.j, X.k, X.nnz, make_map(X), n_rows,
               colcnt, rowcnt, status);
}

// ---------------------------------------------------------------------------
// K2: reduce-then-scan prefix sums (no inter-block waits).  Pass 1 writes
// every warp's sum (512 inputs) and every tile's sum (4096 inputs); one block
// scans the tile sums; pass 2 reads each input once more, starting from its
// tile's offset plus the sums of the warps before it in the tile.  Sums are
// saturating u64 additions: a total at or past 2^63 (the int64 range of the
// CDF) sets DEV_OVERFLOW, integer arithmetic only (GB300's FP64 pipe is
// narrow, and a double running sum per element made these passes FP64-bound).
// ---------------------------------------------------------------------------

// tmp layout: [ntiles + 1] tile sums (exclusive offsets after the tile scan,
// the total last), then [ntiles * SCAN_WARPS] warp sums
size_t scan_tmp_elems(int64_t n) {
  const size_t nt = (size_t)((n + SCAN_TILE - 1) / SCAN_TILE);
  return nt * (SCAN_WARPS + 1) + 4;
}

__device__ __forceinline__ unsigned long long sat_add(unsigned long long a, unsigned long long b) {
  const unsigned long long s = a + b;
  return s < a ? ~0ull : s;
}

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ unsigned long long warp_sat_sum(unsigned long long x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x = sat_add(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

template <typename Tin>
__global__ void k_scan_reduce(const Tin* __restrict__ in, int64_t n,
                              unsigned long long* __restrict__ tile_sum,
                              unsigned long long* __restrict__ warp_sums) {
  __shared__ unsigned long long ws[SCAN_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)warp * SCAN_PER_WARP;
  unsigned long long acc = 0;
#pragma unroll
  for (int it = 0; it < SCAN_PER_WARP / 32; ++it) {
    const int64_t e = base + it * 32 + lane;
    if (e < n) acc = sat_add(acc, (unsigned long long)in[e]);
  }
  acc = warp_sat_sum(acc);
  if (lane == 0) {
    ws[warp] = acc;
    warp_sums[(int64_t)blockIdx.x * SCAN_WARPS + warp] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < SCAN_WARPS; ++w) t = sat_add(t, ws[w]);
    tile_sum[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile sums in one block; flags a total past 2^63.
__global__ void k_scan_tiles(unsigned long long* tile_sum, int64_t ntiles, unsigned* status) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry_s;
  __shared__ int sat_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  if (threadIdx.x == 0) {
    carry_s = 0;
    sat_s = 0;
  }
  __syncthreads();
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    const int64_t e = base + threadIdx.x;
    const unsigned long long x = e < ntiles ? tile_sum[e] : 0ull;
    // a saturated tile, or a block sum that wraps, is an overflow
    if (x >= (1ull << 63)) sat_s = 1;
    unsigned long long inc = warp_incl_scan(x);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = lane < nw ? wsum[lane] : 0ull;
      unsigned long long wi = warp_incl_scan(w);
      if (lane < nw) wsum[lane] = wi - w;
    }
    __syncthreads();
    const unsigned long long excl = carry_s + wsum[warp] + inc - x;
    if (e < ntiles) tile_sum[e] = excl;
    // the first prefix to reach 2^63 is computed exactly (every earlier one
    // and every tile sum are below 2^63), so checking each prefix suffices
    if (excl + x >= (1ull << 63)) sat_s = 1;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry_s = excl + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tile_sum[ntiles] = carry_s;
    if (sat_s || carry_s >= (1ull << 63)) atomicOr(status, DEV_OVERFLOW);
  }
}

// `in` and `out` may be the same array (inclusive u64 scan), and cur32 may
// alias `in`: each element is read once, by the thread that then writes it,
// before that write, so neither pointer is declared __restrict__.
template <typename Tin>
__global__ void k_scan_apply(const Tin* in, unsigned long long* out, int64_t n,
                             const unsigned long long* __restrict__ tile_off,
                             const unsigned long long* __restrict__ warp_sums, bool inclusive,
                             uint32_t* cur32) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)warp * SCAN_PER_WARP;
  unsigned long long carry = tile_off[blockIdx.x];
  for (int w = 0; w < warp; ++w) carry += warp_sums[(int64_t)blockIdx.x * SCAN_WARPS + w];
  const int shift = inclusive ? 0 : 1;
#pragma unroll 4
  for (int it = 0; it < SCAN_PER_WARP / 32; ++it) {
    const int64_t e = base + it * 32 + lane;
    const unsigned long long x = e < n ? (unsigned long long)in[e] : 0ull;
    const unsigned long long inc = warp_incl_scan(x);
    if (e < n) {
      out[e + shift] = carry + inc;
      if (cur32) cur32[e] = (uint32_t)(carry + inc - x);
    }
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (!inclusive && blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

// Short inputs (at most SS_MAX elements) in one launch: one block of 32
// warps, warp w owns elements [512 w, 512 w + 512); the warps' sums, their
// exclusive offsets in shared memory, then each warp's running scan.  The
// same outputs, aliasing rules and overflow flag as the three-pass form.
constexpr int SS_WARPS = 32, SS_PER_WARP = 512, SS_MAX = SS_WARPS * SS_PER_WARP;

template <typename Tin>
__global__ void __launch_bounds__(SS_WARPS * 32)
    k_scan_small(const Tin* in, unsigned long long* out, int64_t n, bool inclusive,
                 uint32_t* cur32, unsigned* status) {
  __shared__ unsigned long long ws[SS_WARPS], wsat[SS_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)warp * SS_PER_WARP;
  unsigned long long acc = 0, accs = 0;
#pragma unroll 4
  for (int it = 0; it < SS_PER_WARP / 32; ++it) {
    const int64_t e = base + it * 32 + lane;
    if (e < n) {
      const unsigned long long x = (unsigned long long)in[e];
      acc += x;
      accs = sat_add(accs, x);
    }
  }
  acc = warp_sum(acc);
  accs = warp_sat_sum(accs);
  if (lane == 0) {
    ws[warp] = acc;
    wsat[warp] = accs;
  }
  __syncthreads();
  unsigned long long carry = 0;
  for (int w = 0; w < warp; ++w) carry += ws[w];
  if (threadIdx.x == 0) {
    // the exact total (saturating) at or past 2^63: every prefix is exact below it
    unsigned long long t = 0;
    for (int w = 0; w < SS_WARPS; ++w) t = sat_add(t, wsat[w]);
    if (t >= (1ull << 63)) atomicOr(status, DEV_OVERFLOW);
  }
  const int shift = inclusive ? 0 : 1;
#pragma unroll 4
  for (int it = 0; it < SS_PER_WARP / 32; ++it) {
    const int64_t e = base + it * 32 + lane;
    const unsigned long long x = e < n ? (unsigned long long)in[e] : 0ull;
    const unsigned long long inc = warp_incl_scan(x);
    if (e < n) {
      out[e + shift] = carry + inc;
      if (cur32) cur32[e] = (uint32_t)(carry + inc - x);
    }
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
  if (!inclusive && threadIdx.x == 0) out[0] = 0;
}

template <typename Tin>
static void scan_impl(const Tin* in, uint64_t* out, int64_t n, bool inclusive, uint64_t* tmp,
                      unsigned* status, cudaStream_t st, uint32_t* cur32 = nullptr) {
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (n == 0) {
    if (!inclusive) cudaMemsetAsync(out, 0, sizeof(uint64_t), st);
    return;
  }
  if (n <= SS_MAX) {
    CTD_LAUNCH(k_scan_small<Tin>, (1), (SS_WARPS * 32), 0, st, in,
               reinterpret_cast<unsigned long long*>(out), n, inclusive, cur32, status);
    return;
  }
  unsigned long long* ts = reinterpret_cast<unsigned long long*>(tmp);
  unsigned long long* wsums = ts + ntiles + 2;
  CTD_LAUNCH(k_scan_reduce<Tin>, ((unsigned)ntiles), (SCAN_WARPS * 32), 0, st, in, n, ts, wsums);
  CTD_LAUNCH(k_scan_tiles, (1), (1024), 0, st, ts, ntiles, status);
  CTD_LAUNCH(k_scan_apply<Tin>, ((unsigned)ntiles), (SCAN_WARPS * 32), 0, st, in,
             reinterpret_cast<unsigned long long*>(out), n, ts, wsums, inclusive, cur32);
}

// ---------------------------------------------------------------------------
// K1b: squared column norms (Eq. 1's numerators) from the column-major
// layout, as the first pass of the CDF's reduce-then-scan
// ---------------------------------------------------------------------------
// A warp takes 512 consecutive columns in 16 groups of 32 (a block of 8
// warps is one 4096-column scan tile), a lane per column.  Most columns of
// count data hold a few entries: each lane walks its own column if it has
// at most 32 (the group's entries are contiguous, so after the first touch
// these reads hit L1); longer columns are then summed by the whole warp,
// one at a time, with coalesced reads.  No atomics; every sum is a
// saturating u64 add, so a column whose exact sum reaches 2^64 stays
// saturated and the tile check flags the overflow.
__global__ void __launch_bounds__(SCAN_WARPS * 32)
    k_sqnorms_reduce(const unsigned long long* __restrict__ colptr,
                     const int32_t* __restrict__ val, int64_t n,
                     unsigned long long* __restrict__ norm2,
                     unsigned long long* __restrict__ tile_sum,
                     unsigned long long* __restrict__ warp_sums, unsigned* minkey,
                     int wshift) {
  const unsigned FULL = 0xffffffffu;
  __shared__ unsigned long long ws[SCAN_WARPS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)warp * SCAN_PER_WARP;
  const unsigned long long end_all = colptr[n];
  unsigned long long acc = 0;
  int vmin = INT32_MAX, vmax = INT32_MIN;
  unsigned long long a_next = base + lane < n ? colptr[base + lane] : end_all;
  for (int it = 0; it < SCAN_PER_WARP / 32; ++it) {
    const int64_t f = base + it * 32 + lane;
    const unsigned long long a = a_next;
    // start of the column after this lane's (lane 31: the next group's first)
    unsigned long long b = __shfl_down_sync(FULL, a, 1);
    if (lane == 31) b = f + 1 < n ? colptr[f + 1] : end_all;
    if (it + 1 < SCAN_PER_WARP / 32) a_next = f + 32 < n ? colptr[f + 32] : end_all;
    const int len = (int)min(b - a, 33ull);
    const int lshort = len <= 32 ? len : 0;
    const int maxs = (int)__reduce_max_sync(FULL, (unsigned)lshort);
    unsigned long long mine = 0;
    for (int t = 0; t < maxs; ++t)
      if (t < lshort) {
        const int v = __ldg(val + a + t);
        vmin = min(vmin, v);
        vmax = max(vmax, v);
        mine = sat_add(mine, sample_weight(v, wshift));
      }
    unsigned longs = __ballot_sync(FULL, len > 32);
    while (longs) {
      const int c = __ffs(longs) - 1;
      longs &= longs - 1;
      const unsigned long long la = __shfl_sync(FULL, a, c), lb = __shfl_sync(FULL, b, c);
      unsigned long long part = 0;
      for (unsigned long long p = la + lane; p < lb; p += 32) {
        const int v = __ldg(val + p);
        vmin = min(vmin, v);
        vmax = max(vmax, v);
        part = sat_add(part, sample_weight(v, wshift));
      }
      part = warp_sat_sum(part);
      if (lane == c) mine = part;
    }
    if (f < n) norm2[f] = mine;
    acc = sat_add(acc, mine);
  }
  acc = warp_sat_sum(acc);
  for (int o = 16; o; o >>= 1) {
    vmin = min(vmin, __shfl_xor_sync(FULL, vmin, o));
    vmax = max(vmax, __shfl_xor_sync(FULL, vmax, o));
  }
  if (lane == 0) {
    ws[warp] = acc;
    warp_sums[(int64_t)blockIdx.x * SCAN_WARPS + warp] = acc;
    if (vmin <= vmax) {
      atomicMin(minkey, (unsigned)vmin ^ 0x80000000u);
      atomicMin(minkey + 1, ~((unsigned)vmax ^ 0x80000000u));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < SCAN_WARPS; ++w) t = sat_add(t, ws[w]);
    tile_sum[blockIdx.x] = t;
  }
}

void launch_sqnorms_cdf(const uint64_t* colptr, const int32_t* val, int64_t n, uint64_t* norm2,
                        uint64_t* cdf, unsigned* minkey, uint64_t* tmp, unsigned* status,
                        cudaStream_t st, int wshift) {
  if (n == 0) return;
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  unsigned long long* ts = reinterpret_cast<unsigned long long*>(tmp);
  unsigned long long* wsums = ts + ntiles + 2;
  unsigned long long* nn = reinterpret_cast<unsigned long long*>(norm2);
  CTD_LAUNCH(k_sqnorms_reduce, ((unsigned)ntiles), (SCAN_WARPS * 32), 0, st,
             reinterpret_cast<const unsigned long long*>(colptr), val, n, nn, ts, wsums, minkey,
             wshift);
  CTD_LAUNCH(k_scan_tiles, (1), (1024), 0, st, ts, ntiles, status);
  CTD_LAUNCH(k_scan_apply<unsigned long long>, ((unsigned)ntiles), (SCAN_WARPS * 32), 0, st, nn,
             reinterpret_cast<unsigned long long*>(cdf), n, ts, wsums, true, (uint32_t*)nullptr);
}

// The last two passes of a scan whose first pass was fused into another
// kernel: that kernel wrote, per 4096-element tile, the tile's sum at
// tile_sum[t] and its eight 512-element warp sums at warp_sums[8 t + w]
// (tmp laid out as scan_impl's: tile sums first, warp sums after
// ntiles + 2 entries).
void launch_scan_finish(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* tmp,
                        unsigned* status, cudaStream_t st) {
  if (n == 0) return;
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  unsigned long long* ts = reinterpret_cast<unsigned long long*>(tmp);
  unsigned long long* wsums = ts + ntiles + 2;
  CTD_LAUNCH(k_scan_tiles, (1), (1024), 0, st, ts, ntiles, status);
  CTD_LAUNCH(k_scan_apply<unsigned long long>, ((unsigned)ntiles), (SCAN_WARPS * 32), 0, st,
             reinterpret_cast<const unsigned long long*>(in),
             reinterpret_cast<unsigned long long*>(out), n, ts, wsums, true, (uint32_t*)nullptr);
}

void launch_scan_u64(const uint64_t* in, uint64_t* out, int64_t n, bool inclusive, uint64_t* tmp,
                     unsigned* status, cudaStream_t st) {
  scan_impl<unsigned long long>(reinterpret_cast<const unsigned long long*>(in), out, n,
                                inclusive, tmp, status, st);
}
void launch_scan_u32(const uint32_t* in, uint64_t* out, int64_t n, bool inclusive, uint64_t* tmp,
                     unsigned* status, cudaStream_t st, uint32_t* cur32) {
  scan_impl<unsigned>(in, out, n, inclusive, tmp, status, st, cur32);
}

// ---------------------------------------------------------------------------
// K5a: counting-sort scatter into the column-major layout
// ---------------------------------------------------------------------------
// Each entry takes its place from its column's u32 cursor (one returning
// atomic) and writes its row and value there.  A thread takes four entries
// and issues their four atomics before any store, so their round trips
// overlap.  The random targets (cursors, rows, values) are kept L2-resident
// by splitting the columns into ranges, one pass over the COO per range:
// an entry is placed in the pass whose range holds its column.  Without
// the split the targets of a 10^7-entry tensor (120 MB) and the streamed
// COO do not fit in L2 together, and every partial-sector store becomes a
// DRAM read-modify-write.
template <bool VEC>
__global__ void __launch_bounds__(256)
    k_coo_scatter(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj,
                  const int32_t* __restrict__ kk, const int32_t* __restrict__ vv, int64_t nnz,
                  ModeMap mm, int64_t c_lo, int64_t c_hi, unsigned* __restrict__ cur,
                  int32_t* __restrict__ csc_row, int32_t* __restrict__ csc_val) {
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t tail0 = 0;
  if (VEC) {
    const int64_t nq = nnz >> 2;
    for (int64_t q = gt; q < nq; q += stride) {
      const int4 a = __ldcs(reinterpret_cast<const int4*>(ii) + q);
      const int4 b = __ldcs(reinterpret_cast<const int4*>(jj) + q);
      const int4 c = __ldcs(reinterpret_cast<const int4*>(kk) + q);
      const int32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w},
                    cv[4] = {c.x, c.y, c.z, c.w};
      int32_t row[4];
      int64_t col[4];
      bool ok[4];
      bool any = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        ok[u] = mm.map(av[u], bv[u], cv[u], &row[u], &col[u]) && col[u] >= c_lo && col[u] < c_hi;
        any |= ok[u];
      }
      if (!any) continue;
      const int4 v = __ldcs(reinterpret_cast<const int4*>(vv) + q);
      const int32_t vals[4] = {v.x, v.y, v.z, v.w};
      unsigned pos[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) pos[u] = ok[u] ? atomicAdd(cur + col[u], 1u) : 0u;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (ok[u]) {
          csc_row[pos[u]] = row[u];
          csc_val[pos[u]] = vals[u];
        }
    }
    tail0 = nq << 2;
  }
  for (int64_t e = tail0 + gt; e < nnz; e += stride) {
    int32_t row;
    int64_t col;
    if (!mm.map(__ldcs(ii + e), __ldcs(jj + e), __ldcs(kk + e), &row, &col)) continue;
    if (col < c_lo || col >= c_hi) continue;
    const unsigned p = atomicAdd(cur + col, 1u);
    csc_row[p] = row;
    csc_val[p] = __ldcs(vv + e);
  }
}

// Bytes of random targets one pass may hold in L2 (cursors and entries).
static int64_t scatter_l2_budget() {
  static int64_t b = [] {
    const char* e = getenv("CTD_SCATTER_L2_MB");  // tuning override
    const long mb = e ? atol(e) : 0;
    return (int64_t)(mb > 0 ? mb : 48) << 20;
  }();
  return b;
}

void launch_coo_scatter(const CooDev& X, uint32_t* cur, int32_t* csc_row, int32_t* csc_val,
                        cudaStream_t st) {
  if (X.nnz == 0) return;
  int64_t n_rows, n_cols;
  mode_extents(X.dims, X.alpha, &n_rows, &n_cols);
  const int bs = 256;
  const bool vec = coo_vec4(X);
  const unsigned g = grid_for((X.nnz + 3) / (vec ? 4 : 1), bs, (int64_t)num_sms() * 8);
  const int64_t targets = 4 * n_cols + 8 * X.nnz;
  const int64_t passes = std::max<int64_t>(1, std::min<int64_t>(8, (targets + scatter_l2_budget() - 1) / scatter_l2_budget()));
  const int64_t span = (n_cols + passes - 1) / passes;
  for (int64_t p = 0; p < passes; ++p) {
    const int64_t lo = p * span, hi = std::min(n_cols, lo + span);
    if (vec)
      CTD_LAUNCH(k_coo_scatter<true>, (g), (bs), 0, st, X.i, X.j, X.k, X.v, X.nnz, make_map(X),
                 lo, hi, cur, csc_row, csc_val);
    else
      CTD_LAUNCH(k_coo_scatter<false>, (g), (bs), 0, st, X.i, X.j, X.k, X.v, X.nnz, make_map(X),
                 lo, hi, cur, csc_row, csc_val);
  }
}

// ---------------------------------------------------------------------------
// K5b: one order inside every column
// ---------------------------------------------------------------------------
// The scatter leaves a column's entries in the order its cursor atomics were
// taken, which differs from run to run.  Integer work (the Gram matrix, C) is
// exact in any order, but floating-point sums over a column's entries (the
// error of Eq. 3 through Q, W = Q^T X_c of CTD-D) round differently.  These
// kernels sort each column's entries by (row, value), so those sums take one
// order whatever the scheduling.  Key: the row in the high 32 bits, the value
// mapped to an order-preserving unsigned in the low 32.
__device__ __forceinline__ unsigned long long col_key(int32_t r, int32_t v) {
  return ((unsigned long long)(uint32_t)r << 32) | (unsigned long long)((uint32_t)v ^ 0x80000000u);
}
__device__ __forceinline__ void col_key_split(unsigned long long k, int32_t* r, int32_t* v) {
  *r = (int32_t)(k >> 32);
  *v = (int32_t)((uint32_t)k ^ 0x80000000u);
}

constexpr int SC_WARP = 1024;   // longest column sorted by one warp
constexpr int SC_BLOCK = 4096;  // piece of a longer column sorted in one block's shared memory
constexpr int SC_WARPS = 4;     // warps per block of k_sort_cols_mid (8 KB of keys each)

// A warp per 32 consecutive columns.  Columns of 2..32 entries go in chunks
// of whole columns (at most 32 entries, one per lane), each entry ranked
// against its own column's entries by shuffles; longer columns are listed
// for k_sort_cols_mid (up to SC_WARP entries) or k_sort_cols_block.  A
// chunk is read whole before any of its entries is written.
__global__ void __launch_bounds__(256)
    k_sort_cols_short(const unsigned long long* __restrict__ colptr, int64_t n_cols,
                      int32_t* __restrict__ row, int32_t* __restrict__ val,
                      int64_t* __restrict__ mids, unsigned* __restrict__ n_mid,
                      int64_t* __restrict__ longs, unsigned* __restrict__ n_long) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f0 = gw * 32; f0 < n_cols; f0 += nw * 32) {
    const int64_t f = f0 + lane;
    unsigned long long a = 0, b = 0;
    if (f < n_cols) {
      a = colptr[f];
      b = colptr[f + 1];
    }
    const long long n = (long long)(b - a);
    if (n > SC_WARP) longs[atomicAdd(n_long, 1u)] = f;
    else if (n > 32) mids[atomicAdd(n_mid, 1u)] = f;
    // short columns: lane prefix sums of their lengths, then chunks
    const int ns = (n >= 2 && n <= 32) ? (int)n : 0;
    int incl = ns;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, d);
      if (lane >= d) incl += y;
    }
    const int excl = incl - ns;
    const int total = __shfl_sync(FULL, incl, 31);
    int base = 0;
    while (base < total) {
      // the chunk: the short columns that start at or after `base` and end
      // within base + 32 (at least one: each has at most 32 entries)
      const unsigned inm = __ballot_sync(FULL, ns > 0 && excl >= base && incl <= base + 32);
      const int end = __shfl_sync(FULL, incl, 31 - __clz(inm));
      const int g = base + lane;
      const bool valid = g < end;
      // the column (owner lane) of entry g: the lanes whose run ends at or before g
      int e = 0;
#pragma unroll
      for (int s = 16; s > 0; s >>= 1)
        if (__shfl_sync(FULL, incl, e + s - 1) <= g) e += s;
      e = min(e, 31);
      const unsigned long long ea = __shfl_sync(FULL, a, e);
      const int s0 = __shfl_sync(FULL, excl, e) - base;  // the column's first lane
      const int ne = __shfl_sync(FULL, ns, e);
      const int t = g - base - s0;                        // place in the column
      unsigned long long k = ~0ull;
      if (valid) k = col_key(row[ea + t], val[ea + t]);
      const int maxn = (int)__reduce_max_sync(FULL, valid ? (unsigned)ne : 0u);
      int r = 0;
      for (int j = 0; j < maxn; ++j) {
        const unsigned long long kj = __shfl_sync(FULL, k, min(s0 + j, 31));
        r += (j < ne) & ((kj < k) | ((kj == k) & (j < t)));
      }
      if (valid && r != t) {
        int32_t rr, vv;
        col_key_split(k, &rr, &vv);
        row[ea + r] = rr;
        val[ea + r] = vv;
      }
      base = end;
    }
  }
}

// A warp per listed column of 33..SC_WARP entries: bitonic sort of the
// keys in the warp's shared memory (padded to a power of two), the m/2
// compare-exchanges of each stage spread over the lanes.
__global__ void __launch_bounds__(SC_WARPS * 32)
    k_sort_cols_mid(const unsigned long long* __restrict__ colptr,
                    const int64_t* __restrict__ mids, const unsigned* __restrict__ n_mid,
                    int32_t* __restrict__ row, int32_t* __restrict__ val) {
  __shared__ unsigned long long ks_all[SC_WARPS][SC_WARP];
  unsigned long long* ks = ks_all[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nm = *n_mid;
  for (int64_t c = gw; c < nm; c += nw) {
    const int64_t f = mids[c];
    const unsigned long long a = colptr[f];
    const int n = (int)(colptr[f + 1] - a);
    int m = 64;
    while (m < n) m <<= 1;
    // loads eight at a time per lane, so their latencies overlap
    for (int p0 = 0; p0 < m; p0 += 256) {
      unsigned long long x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int p = p0 + 32 * u + lane;
        x[u] = p < n ? col_key(row[a + p], val[a + p]) : ~0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int p = p0 + 32 * u + lane;
        if (p < m) ks[p] = x[u];
      }
    }
    __syncwarp();
    for (int k = 2; k <= m; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int q = lane; q < (m >> 1); q += 32) {
          const int e = ((q & ~(j - 1)) << 1) | (q & (j - 1));  // bit j of e clear
          const int o = e | j;
          const bool up = (e & k) == 0;
          const unsigned long long x = ks[e], y = ks[o];
          if ((x > y) == up) {
            ks[e] = y;
            ks[o] = x;
          }
        }
        __syncwarp();
      }
    for (int p = lane; p < n; p += 32) {
      int32_t rr, vv;
      col_key_split(ks[p], &rr, &vv);
      row[a + p] = rr;
      val[a + p] = vv;
    }
    __syncwarp();
  }
}

// A block per listed column (more than SC_WARP entries): bitonic sort of
// SC_BLOCK-entry pieces in shared memory; a column of several pieces keeps
// the sorted pieces in `keys` (indexed like the entries) and puts each entry
// at its merged rank: its place in its piece plus, in every other piece, the
// entries below it (and the equal ones of earlier pieces).
__global__ void __launch_bounds__(1024)
    k_sort_cols_block(const unsigned long long* __restrict__ colptr,
                      const int64_t* __restrict__ longs, const unsigned* __restrict__ n_long,
                      int32_t* __restrict__ row, int32_t* __restrict__ val,
                      unsigned long long* __restrict__ keys) {
  __shared__ unsigned long long ks[SC_BLOCK];
  const unsigned nl = *n_long;
  for (unsigned g = blockIdx.x; g < nl; g += gridDim.x) {
    const int64_t f = longs[g];
    const unsigned long long a = colptr[f];
    const long long n = (long long)(colptr[f + 1] - a);
    const long long npc = (n + SC_BLOCK - 1) / SC_BLOCK;
    for (long long c = 0; c < npc; ++c) {
      const long long c0 = c * SC_BLOCK;
      const int len = (int)min((long long)SC_BLOCK, n - c0);
      int m = 1;
      while (m < len) m <<= 1;
      for (int e = threadIdx.x; e < m; e += blockDim.x)
        ks[e] = e < len ? col_key(row[a + c0 + e], val[a + c0 + e]) : ~0ull;
      __syncthreads();
      for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int q = threadIdx.x; q < (m >> 1); q += blockDim.x) {
            const int e = ((q & ~(j - 1)) << 1) | (q & (j - 1));
            const int o = e | j;
            const bool up = (e & k) == 0;
            const unsigned long long x = ks[e], y = ks[o];
            if ((x > y) == up) {
              ks[e] = y;
              ks[o] = x;
            }
          }
          __syncthreads();
        }
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        if (npc == 1) {
          int32_t rr, vv;
          col_key_split(ks[e], &rr, &vv);
          row[a + e] = rr;
          val[a + e] = vv;
        } else {
          keys[a + c0 + e] = ks[e];
        }
      }
      __syncthreads();
    }
    if (npc > 1) {
      for (long long p = threadIdx.x; p < n; p += blockDim.x) {
        const long long cp = p / SC_BLOCK;
        const unsigned long long k = keys[a + p];
        long long r = p - cp * SC_BLOCK;
        for (long long c = 0; c < npc; ++c) {
          if (c == cp) continue;
          const unsigned long long* ck = keys + a + c * SC_BLOCK;
          int lo = 0, hi = (int)min((long long)SC_BLOCK, n - c * SC_BLOCK);
          while (lo < hi) {
            const int md = (lo + hi) >> 1;
            const bool below = c < cp ? ck[md] <= k : ck[md] < k;
            if (below) lo = md + 1;
            else hi = md;
          }
          r += lo;
        }
        int32_t rr, vv;
        col_key_split(k, &rr, &vv);
        row[a + r] = rr;
        val[a + r] = vv;
      }
      __syncthreads();
    }
  }
}

ctd_status launch_sort_cols(const uint64_t* colptr, int64_t n_cols, int64_t nnz, int32_t* row,
                            int32_t* val, uint64_t* keys, Arena& A, cudaStream_t st) {
  if (nnz <= 1) return CTD_OK;
  int64_t *mids, *longs;
  unsigned* counts;
  CTD_TRY(A.get(&mids, nnz / 33 + 1));
  CTD_TRY(A.get(&longs, nnz / (SC_WARP + 1) + 1));
  CTD_TRY(A.get(&counts, 2));
  CTD_CUDA(cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned), st));
  const unsigned long long* cp = reinterpret_cast<const unsigned long long*>(colptr);
  CTD_LAUNCH(k_sort_cols_short, (grid_for(n_cols, 256, (int64_t)num_sms() * 8)), (256), 0, st,
             cp, n_cols, row, val, mids, counts, longs, counts + 1);
  CTD_LAUNCH(k_sort_cols_mid, ((unsigned)num_sms() * 6), (SC_WARPS * 32), 0, st, cp, mids, counts,
             row, val);
  CTD_LAUNCH(k_sort_cols_block, ((unsigned)num_sms()), (1024), 0, st, cp, longs, counts + 1, row,
             val, reinterpret_cast<unsigned long long*>(keys));
  return CTD_OK;
}

__global__ void k_copy_u64(const unsigned long long* __restrict__ in, unsigned long long* out,
                           int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride)
    out[e] = in[e];
}

void launch_copy_u64(const uint64_t* in, uint64_t* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  CTD_LAUNCH(k_copy_u64, (grid_for(n, 256, (int64_t)num_sms() * 8)), (256), 0, st, 
      reinterpret_cast<const unsigned long long*>(in), reinterpret_cast<unsigned long long*>(out),
      n);
}

// ---------------------------------------------------------------------------
// K5b: gather sampled columns
// ---------------------------------------------------------------------------
__global__ void k_column_sizes(const unsigned long long* __restrict__ colptr,
                               const int64_t* __restrict__ fibers, const int* nf_dev, int nf_max,
                               unsigned long long* sizes) {
  const int nf = min(*nf_dev, nf_max);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nf_max; c += gridDim.x * blockDim.x) {
    unsigned long long sz = 0;
    if (c < nf) {
      const int64_t f = fibers[c];
      sz = colptr[f + 1] - colptr[f];
    }
    sizes[c] = sz;
  }
}

void launch_column_sizes(const uint64_t* colptr, const int64_t* fibers, const int* nf_dev,
                         int nf_max, uint64_t* sizes, cudaStream_t st) {
  if (nf_max <= 0) return;
  CTD_LAUNCH(k_column_sizes, (grid_for(nf_max, 256, 1024)), (256), 0, st, 
      reinterpret_cast<const unsigned long long*>(colptr), fibers, nf_dev, nf_max,
      reinterpret_cast<unsigned long long*>(sizes));
}

// one warp per column
__global__ void k_gather_columns(const unsigned long long* __restrict__ colptr,
                                 const int32_t* __restrict__ row, const int32_t* __restrict__ val,
                                 const int64_t* __restrict__ fibers, const int* nf_dev, int nf_max,
                                 const unsigned long long* __restrict__ colptr_out,
                                 int32_t* __restrict__ row_out, int32_t* __restrict__ val_out) {
  const int nf = min(*nf_dev, nf_max);
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int c = gw; c < nf; c += nwarps) {
    const int64_t f = fibers[c];
    const unsigned long long a = colptr[f], b = colptr[f + 1];
    const unsigned long long o = colptr_out[c];
    for (unsigned long long p = a + lane; p < b; p += 32) {
      row_out[o + (p - a)] = row[p];
      val_out[o + (p - a)] = val[p];
    }
  }
}

void launch_gather_columns(const uint64_t* colptr, const int32_t* row, const int32_t* val,
                           const int64_t* fibers, const int* nf_dev, int nf_max,
                           const uint64_t* colptr_out, int32_t* row_out, int32_t* val_out,
                           cudaStream_t st) {
  if (nf_max <= 0) return;
  CTD_LAUNCH(k_gather_columns, (grid_for((int64_t)nf_max * 32, 256, 4096)), (256), 0, st, 
      reinterpret_cast<const unsigned long long*>(colptr), row, val, fibers, nf_dev, nf_max,
      reinterpret_cast<const unsigned long long*>(colptr_out), row_out, val_out);
}

// ---------------------------------------------------------------------------
// small CSC -> CSR transposition (for the factor R)
// ---------------------------------------------------------------------------
// row counts of a CSC layout, walking its columns (a warp per column), so
// the number of entries need not be known on the host
__global__ void k_row_counts(const unsigned long long* __restrict__ colptr,
                             const int32_t* __restrict__ row, int64_t ncols, unsigned* rowcnt) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = gw; c < ncols; c += nw)
    for (unsigned long long p = colptr[c] + lane; p < colptr[c + 1]; p += 32)
      atomicAdd(rowcnt + row[p], 1u);
}

// one warp per column: scatter its entries into their rows
__global__ void k_csc_to_csr(const unsigned long long* __restrict__ colptr,
                             const int32_t* __restrict__ row, const int32_t* __restrict__ val,
                             int64_t ncols, int col_base, unsigned long long* rowcur,
                             int32_t* __restrict__ col_out, int32_t* __restrict__ val_out) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = gw; c < ncols; c += nwarps) {
    for (unsigned long long p = colptr[c] + lane; p < colptr[c + 1]; p += 32) {
      unsigned long long pos = atomicAdd(rowcur + row[p], 1ull);
      col_out[pos] = (int32_t)(col_base + c);
      val_out[pos] = val[p];
    }
  }
}

ctd_status build_csr_from_csc(const uint64_t* colptr, const int32_t* row, const int32_t* val,
                              int64_t ncols, int64_t nnz, int64_t n_rows, int col_base,
                              uint64_t* rowptr_out, int32_t* col_out, int32_t* val_out,
                              Arena& scratch, cudaStream_t st) {
  unsigned* rowcnt;
  uint64_t* cur;
  uint64_t* tmp;
  unsigned* status;
  int32_t *col_tmp, *val_tmp;
  CTD_TRY(scratch.get(&rowcnt, n_rows));
  CTD_TRY(scratch.get(&cur, n_rows + 1));
  CTD_TRY(scratch.get(&tmp, scan_tmp_elems(n_rows)));
  CTD_TRY(scratch.get(&status, 1));
  CTD_TRY(scratch.get(&col_tmp, nnz));
  CTD_TRY(scratch.get(&val_tmp, nnz));
  CTD_CUDA(cudaMemsetAsync(rowcnt, 0, n_rows * sizeof(unsigned), st));
  CTD_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
  if (nnz > 0 && ncols > 0)
    CTD_LAUNCH(k_row_counts, (grid_for(ncols * 32, 256, 4096)), (256), 0, st,
               reinterpret_cast<const unsigned long long*>(colptr), row, ncols, rowcnt);
  launch_scan_u32(rowcnt, rowptr_out, n_rows, false, tmp, status, st);
  launch_copy_u64(rowptr_out, cur, n_rows, st);
  if (nnz > 0 && ncols > 0) {
    CTD_LAUNCH(k_csc_to_csr, (grid_for(ncols * 32, 256, 4096)), (256), 0, st,
               reinterpret_cast<const unsigned long long*>(colptr), row, val, ncols, col_base,
               reinterpret_cast<unsigned long long*>(cur), col_tmp, val_tmp);
    // rows sorted by column, so R(i, :) can be copied out in order
    launch_sort_rows(rowptr_out, n_rows, col_tmp, val_tmp, col_out, val_out, col_base, ncols,
                     st);
  }
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

// ---------------------------------------------------------------------------
// A factor by row restricted to a subset of its columns (R from R'): row i
// keeps the entries whose column c has kpos[c] >= 0, renumbered to kpos[c].
// kpos is increasing on the kept columns, so rows sorted by column stay
// sorted.  A warp per row; a kept entry's place is the count of kept
// entries before it (ballots), so the order is that of the input row.
// ---------------------------------------------------------------------------
__global__ void k_rsub_counts(const unsigned long long* __restrict__ rowptr,
                              const int32_t* __restrict__ col, const int* __restrict__ kpos,
                              int64_t n_rows, unsigned* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n_rows; i += nw) {
    const unsigned long long a = rowptr[i], b = rowptr[i + 1];
    unsigned c = 0;
    for (unsigned long long p = a + lane; p - lane < b; p += 32) {
      const bool k = p < b && kpos[col[p]] >= 0;
      c += __popc(__ballot_sync(0xffffffffu, k));
    }
    if (lane == 0) cnt[i] = c;
  }
}

__global__ void k_rsub_write(const unsigned long long* __restrict__ rowptr,
                             const int32_t* __restrict__ col, const int32_t* __restrict__ val,
                             const int* __restrict__ kpos, int64_t n_rows,
                             const unsigned long long* __restrict__ rowptr_out,
                             int32_t* __restrict__ col_out, int32_t* __restrict__ val_out) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n_rows; i += nw) {
    const unsigned long long a = rowptr[i], b = rowptr[i + 1];
    unsigned long long o = rowptr_out[i];
    for (unsigned long long p = a + lane; p - lane < b; p += 32) {
      const int kp = p < b ? kpos[col[p]] : -1;
      const unsigned m = __ballot_sync(0xffffffffu, kp >= 0);
      if (kp >= 0) {
        const unsigned long long q = o + __popc(m & lt);
        col_out[q] = kp;
        val_out[q] = val[p];
      }
      o += __popc(m);
    }
  }
}

ctd_status csr_keep_columns(const uint64_t* rowptr, const int32_t* col, const int32_t* val,
                            int64_t n_rows, const int* kpos, uint64_t* rowptr_out,
                            int32_t* col_out, int32_t* val_out, Arena& scratch,
                            cudaStream_t st) {
  unsigned* cnt;
  uint64_t* tmp;
  unsigned* status;
  CTD_TRY(scratch.get(&cnt, std::max<int64_t>(n_rows, 1)));
  CTD_TRY(scratch.get(&tmp, scan_tmp_elems(n_rows)));
  CTD_TRY(scratch.get(&status, 1));
  CTD_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
  const unsigned g = grid_for(n_rows * 32, 256, (int64_t)num_sms() * 8);
  const auto* rp = reinterpret_cast<const unsigned long long*>(rowptr);
  if (n_rows > 0) CTD_LAUNCH(k_rsub_counts, (g), (256), 0, st, rp, col, kpos, n_rows, cnt);
  launch_scan_u32(cnt, rowptr_out, n_rows, false, tmp, status, st);
  if (n_rows > 0)
    CTD_LAUNCH(k_rsub_write, (g), (256), 0, st, rp, col, val, kpos, n_rows,
               reinterpret_cast<const unsigned long long*>(rowptr_out), col_out, val_out);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

__global__ void k_sum_u32(const unsigned* __restrict__ in, int64_t n, unsigned long long* out,
                          unsigned mask) {
  __shared__ unsigned long long part[32];
  unsigned long long acc = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    acc += in[e] & mask;
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    atomicAdd(out, t);
  }
}

void launch_sum_u32(const uint32_t* in, int64_t n, uint64_t* out, cudaStream_t st,
                    uint32_t mask) {
  cudaMemsetAsync(out, 0, sizeof(uint64_t), st);
  if (n <= 0) return;
  CTD_LAUNCH(k_sum_u32, (grid_for(n, 1024, (int64_t)num_sms() * 2)), (1024), 0, st,
             in, n, reinterpret_cast<unsigned long long*>(out), mask);
}

__global__ void k_gather_i64(const int64_t* __restrict__ in, const int* __restrict__ idx,
                             const int* count, int nmax, int64_t* __restrict__ out) {
  const int n = min(*count, nmax);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
    out[c] = in[idx[c]];
}

void launch_gather_i64(const int64_t* in, const int* idx, const int* count, int nmax,
                       int64_t* out, cudaStream_t st) {
  if (nmax <= 0) return;
  CTD_LAUNCH(k_gather_i64, (grid_for(nmax, 256, 256)), (256), 0, st, in, idx, count, nmax, out);
}

}  // namespace ctd
