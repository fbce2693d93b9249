// Algorithm 1's matricization (X_(alpha) by column, Sec. 2.1) and its
// squared column norms (Eq. 1) for tensors with many columns, as a
// bucketed counting sort.
//
// A plain counting sort places every entry with one returning atomic on its
// column's cursor and two 4-byte stores at a random address: three small
// random L2 operations per entry, and GB300's L2 serves such operations at a
// fixed rate whatever the bytes.  Here the columns are cut into buckets of
// MB_W consecutive columns and the work is done in four passes:
//   count      entries per bucket (and per row) in shared-memory histograms;
//   scan       bucket offsets (the positions of each bucket's entries in
//              the column-major layout), with a u32 cursor per bucket;
//   partition  each block takes a chunk of entries, orders it by bucket in
//              shared memory and writes each bucket's run with consecutive
//              lanes on consecutive addresses, so stores coalesce;
//   place      one block per bucket counts its columns in shared memory,
//              writes their offsets, places the entries in shared memory in
//              column order and writes them out contiguously, then sums the
//              squares of each column's values (the norms) and writes the
//              tile and warp sums the CDF's prefix sum continues from.
// A bucket with more entries than the place kernel can stage writes its
// entries straight to global memory (its range is small and stays in L2).
#include <algorithm>

#include "ctd_internal.cuh"

namespace ctd {
namespace {

constexpr int MB_SHIFT = 13;
constexpr int MB_W = 1 << MB_SHIFT;     // columns per bucket: two scan tiles
static_assert(MB_W == 2 * SCAN_TILE, "a bucket is two scan tiles");
constexpr int MB_MAX_BUCKETS = 8192;    // bucket histogram in shared memory
constexpr int ROW_SMEM_MAX = 16384;     // row histogram in shared memory

constexpr int MC_THREADS = 512;         // count
constexpr int MP_THREADS = 1024;        // partition: 8 entries per thread
constexpr int MP_CHUNK = 8192;
constexpr int MQ_THREADS = 512;         // place
constexpr int MQ_SMEM = 112 * 1024;     // two blocks per SM
constexpr int MQ_CAP = (MQ_SMEM - MB_W * 4) / 8;  // entries staged per bucket

__device__ __forceinline__ unsigned long long sat_add64(unsigned long long a,
                                                        unsigned long long b) {
  const unsigned long long s = a + b;
  return s < a ? ~0ull : s;
}

// ---------------------------------------------------------------------------
// count: entries per bucket and per row
// ---------------------------------------------------------------------------
template <bool VEC>
__global__ void __launch_bounds__(MC_THREADS)
    k_mb_count(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj,
               const int32_t* __restrict__ kk, int64_t nnz, ModeMap mm, int64_t n_rows, int nb,
               unsigned* __restrict__ bcnt, unsigned* __restrict__ rowcnt, unsigned* status) {
  extern __shared__ unsigned sh[];
  unsigned* bh = sh;        // [nb]
  unsigned* rh = sh + nb;   // [n_rows] when they fit
  const bool priv = n_rows <= ROW_SMEM_MAX;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) bh[b] = 0;
  if (priv)
    for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x) rh[r] = 0;
  __syncthreads();
  bool bad = false;
  auto one = [&](int32_t a, int32_t b, int32_t c) {
    int32_t row;
    int64_t col;
    if (!mm.map(a, b, c, &row, &col)) {
      bad = true;
      return;
    }
    atomicAdd(bh + (col >> MB_SHIFT), 1u);
    if (priv)
      atomicAdd(rh + row, 1u);
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
  for (int64_t e = tail0 + gt; e < nnz; e += stride)
    one(__ldcs(ii + e), __ldcs(jj + e), __ldcs(kk + e));
  if (bad) atomicOr(status, DEV_BAD_INDEX);
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (bh[b]) atomicAdd(bcnt + b, bh[b]);
  if (priv)
    for (int64_t r = threadIdx.x; r < n_rows; r += blockDim.x)
      if (rh[r]) atomicAdd(rowcnt + r, rh[r]);
}

// Largest bucket (one block).
__global__ void k_mb_max(const unsigned* __restrict__ bcnt, int nb, unsigned* out) {
  unsigned m = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) m = max(m, bcnt[b]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Block-wide exclusive scan of `per` consecutive u32 values per thread,
// in place in shared memory (x[0 .. blockDim.x * per)); returns the total.
// wsum: 33 words of shared scratch.
template <int PER>
__device__ unsigned block_excl_scan(unsigned* x, unsigned* wsum) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  unsigned v[PER];
  unsigned run = 0;
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    v[u] = x[t * PER + u];
    const unsigned y = v[u];
    v[u] = run;
    run += y;
  }
  unsigned inc = run;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const unsigned w = lane < nw ? wsum[lane] : 0u;
    unsigned wi = w;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= d) wi += y;
    }
    wsum[lane] = wi - w;  // exclusive warp offsets; the total at [nw - 1] + last
    if (lane == 31) wsum[32] = wi;
  }
  __syncthreads();
  const unsigned off = wsum[warp] + inc - run;
#pragma unroll
  for (int u = 0; u < PER; ++u) x[t * PER + u] = off + v[u];
  const unsigned total = wsum[32];
  __syncthreads();
  return total;
}

// ---------------------------------------------------------------------------
// partition: each chunk of MP_CHUNK entries is ordered by bucket in shared
// memory, then each bucket's run is written to the staging arrays at the
// bucket's cursor, consecutive lanes on consecutive addresses.  Staged per
// entry: the column within its bucket (u16), the row and the value.
// Shared memory: hist and gbase (MB_MAX_BUCKETS each), the chunk's columns,
// rows and values (MP_CHUNK each): 160 KB.
// ---------------------------------------------------------------------------
constexpr int MP_SMEM = (2 * MB_MAX_BUCKETS + 3 * MP_CHUNK) * 4;

template <bool VEC>
__global__ void __launch_bounds__(MP_THREADS, 1)
    k_mb_part(const int32_t* __restrict__ ii, const int32_t* __restrict__ jj,
              const int32_t* __restrict__ kk, const int32_t* __restrict__ vv, int64_t nnz,
              ModeMap mm, int nb, unsigned* __restrict__ bcur, uint16_t* __restrict__ stg_lc,
              int32_t* __restrict__ stg_row, int32_t* __restrict__ stg_val) {
  extern __shared__ unsigned sp[];
  unsigned* hist = sp;                                    // counts, then local starts
  unsigned* gbase = hist + MB_MAX_BUCKETS;                // global start of each run
  int* s_f = reinterpret_cast<int*>(gbase + MB_MAX_BUCKETS);
  int* s_row = s_f + MP_CHUNK;
  int* s_val = s_row + MP_CHUNK;
  __shared__ unsigned wsum[33];
  const int t = threadIdx.x;
  constexpr int PER = MP_CHUNK / MP_THREADS;  // 8 entries per thread
  constexpr int HPER = MB_MAX_BUCKETS / MP_THREADS;
  for (int64_t c0 = (int64_t)blockIdx.x * MP_CHUNK; c0 < nnz;
       c0 += (int64_t)gridDim.x * MP_CHUNK) {
#pragma unroll
    for (int u = 0; u < HPER; ++u) hist[t * HPER + u] = 0;
    __syncthreads();
    int f[PER], row[PER], val[PER];
    unsigned r[PER];
#pragma unroll
    for (int g = 0; g < PER / 4; ++g) {
      const int64_t e = c0 + (int64_t)g * (MP_THREADS * 4) + 4 * t;  // entries e .. e+3
      int32_t a[4], b[4], c[4], v[4];
      if (VEC && e + 3 < nnz) {
        const int4 A = __ldcs(reinterpret_cast<const int4*>(ii + e));
        const int4 B = __ldcs(reinterpret_cast<const int4*>(jj + e));
        const int4 Cc = __ldcs(reinterpret_cast<const int4*>(kk + e));
        const int4 V = __ldcs(reinterpret_cast<const int4*>(vv + e));
        a[0] = A.x; a[1] = A.y; a[2] = A.z; a[3] = A.w;
        b[0] = B.x; b[1] = B.y; b[2] = B.z; b[3] = B.w;
        c[0] = Cc.x; c[1] = Cc.y; c[2] = Cc.z; c[3] = Cc.w;
        v[0] = V.x; v[1] = V.y; v[2] = V.z; v[3] = V.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool in = e + u < nnz;
          a[u] = in ? __ldcs(ii + e + u) : -1;  // -1 maps to "no entry"
          b[u] = in ? __ldcs(jj + e + u) : -1;
          c[u] = in ? __ldcs(kk + e + u) : -1;
          v[u] = in ? __ldcs(vv + e + u) : 0;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int32_t rw = 0;
        int64_t col = 0;
        const bool ok = mm.map(a[u], b[u], c[u], &rw, &col);
        f[4 * g + u] = ok ? (int)col : -1;
        row[4 * g + u] = rw;
        val[4 * g + u] = v[u];
        r[4 * g + u] = ok ? atomicAdd(hist + (col >> MB_SHIFT), 1u) : 0u;
      }
    }
    __syncthreads();
    // global start of each bucket's run (one atomic per bucket present)
    for (int b = t; b < nb; b += MP_THREADS) {
      const unsigned h = hist[b];
      gbase[b] = h ? atomicAdd(bcur + b, h) : 0u;
    }
    // local starts; the scan's own barriers order the reads above before its writes
    const unsigned n_valid = block_excl_scan<HPER>(hist, wsum);
    // the chunk in bucket order in shared memory
#pragma unroll
    for (int u = 0; u < PER; ++u)
      if (f[u] >= 0) {
        const unsigned p = hist[f[u] >> MB_SHIFT] + r[u];
        s_f[p] = f[u];
        s_row[p] = row[u];
        s_val[p] = val[u];
      }
    __syncthreads();
    // each bucket's run to its place: consecutive lanes, consecutive addresses
    for (unsigned p = t; p < n_valid; p += MP_THREADS) {
      const int fc = s_f[p];
      const int b = fc >> MB_SHIFT;
      const unsigned long long gpos = (unsigned long long)gbase[b] + (p - hist[b]);
      stg_lc[gpos] = (uint16_t)(fc & (MB_W - 1));
      stg_row[gpos] = s_row[p];
      stg_val[gpos] = s_val[p];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// place: one block per bucket.  Shared memory: a u32 per column of the
// bucket (counts, then starts, then cursors) and, when the bucket's entries
// fit, their rows and values in column order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(MQ_THREADS, 2)
    k_mb_place(const unsigned long long* __restrict__ bstart, int nb, int64_t n_cols,
               const uint16_t* __restrict__ stg_lc, const int32_t* __restrict__ stg_row,
               const int32_t* __restrict__ stg_val, unsigned long long* __restrict__ colptr,
               int32_t* __restrict__ csc_row, int32_t* __restrict__ csc_val,
               unsigned long long* __restrict__ norm2, unsigned long long* __restrict__ tile_sum,
               unsigned long long* __restrict__ warp_sums, unsigned* minkey, int wshift) {
  extern __shared__ unsigned sq[];
  unsigned* cnt = sq;                                          // [MB_W]
  int32_t* o_row = reinterpret_cast<int32_t*>(cnt + MB_W);     // [MQ_CAP]
  int32_t* o_val = o_row + MQ_CAP;                             // [MQ_CAP]
  __shared__ unsigned wsum[33];
  __shared__ unsigned long long segs[MQ_THREADS / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int b = blockIdx.x;
  const int64_t c0 = (int64_t)b << MB_SHIFT;
  const int ncols = (int)min((int64_t)MB_W, n_cols - c0);
  const unsigned long long s = bstart[b], e = bstart[b + 1];
  const unsigned E = (unsigned)(e - s);
  const bool staged = E <= (unsigned)MQ_CAP;
  constexpr int CPER = MB_W / MQ_THREADS;  // 16 columns per thread in the scan
#pragma unroll
  for (int u = 0; u < CPER; ++u) cnt[t * CPER + u] = 0;
  __syncthreads();
  // loads in batches ahead of the shared-memory atomics, so their round
  // trips overlap
  for (unsigned p0 = 0; p0 < E; p0 += MQ_THREADS * 16) {
    unsigned lc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const unsigned p = p0 + u * MQ_THREADS + t;
      lc[u] = p < E ? stg_lc[s + p] : 0xffffu;
    }
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (lc[u] != 0xffffu) atomicAdd(cnt + lc[u], 1u);
  }
  __syncthreads();
  block_excl_scan<CPER>(cnt, wsum);  // cnt[c] = start of column c within the bucket
  for (int c = t; c < ncols; c += MQ_THREADS) colptr[c0 + c] = s + cnt[c];
  if (b == nb - 1 && t == 0) colptr[n_cols] = e;
  __syncthreads();
  for (unsigned p0 = 0; p0 < E; p0 += MQ_THREADS * 8) {
    unsigned lc[8];
    int32_t rw[8], v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const unsigned p = p0 + u * MQ_THREADS + t;
      lc[u] = p < E ? stg_lc[s + p] : 0xffffu;
      rw[u] = p < E ? stg_row[s + p] : 0;
      v[u] = p < E ? stg_val[s + p] : 0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (lc[u] != 0xffffu) {
        const unsigned pos = atomicAdd(cnt + lc[u], 1u);
        if (staged) {
          o_row[pos] = rw[u];
          o_val[pos] = v[u];
        } else {
          csc_row[s + pos] = rw[u];
          csc_val[s + pos] = v[u];
        }
      }
  }
  __syncthreads();
  if (staged)
    for (unsigned p = t; p < E; p += MQ_THREADS) {
      csc_row[s + p] = o_row[p];
      csc_val[s + p] = o_val[p];
    }
  // cnt[c] is now the end of column c.  Squared norms (warp w takes the 512
  // columns of warp segment w of the bucket's two scan tiles): a lane walks
  // its own column when it has at most 32 entries; longer columns are then
  // summed by the whole warp.  The values come from shared memory, or from
  // the global copy this block wrote (visible to the block after the
  // barrier above).
  const int32_t* vals = staged ? o_val : csc_val + s;
  unsigned long long acc = 0;
  int vmin = INT32_MAX, vmax = INT32_MIN;
  for (int i = 0; i < SCAN_PER_WARP / 32; ++i) {
    const int c = warp * SCAN_PER_WARP + i * 32 + lane;
    const unsigned a = (c > 0 && c <= ncols) ? cnt[c - 1] : 0u;
    const unsigned z = c < ncols ? cnt[c] : a;
    const unsigned len = z - a;
    const unsigned lshort = len <= 32 ? len : 0u;
    const unsigned maxs = __reduce_max_sync(0xffffffffu, lshort);
    unsigned long long nrm = 0;
    for (unsigned q = 0; q < maxs; ++q)
      if (q < lshort) {
        const int v = vals[a + q];
        vmin = min(vmin, v);
        vmax = max(vmax, v);
        nrm = sat_add64(nrm, sample_weight(v, wshift));
      }
    unsigned longs = __ballot_sync(0xffffffffu, len > 32);
    while (longs) {
      const int l = __ffs(longs) - 1;
      longs &= longs - 1;
      const unsigned la = __shfl_sync(0xffffffffu, a, l), lz = __shfl_sync(0xffffffffu, z, l);
      unsigned long long part = 0;
      for (unsigned p = la + lane; p < lz; p += 32) {
        const int v = vals[p];
        vmin = min(vmin, v);
        vmax = max(vmax, v);
        part = sat_add64(part, sample_weight(v, wshift));
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) part = sat_add64(part, __shfl_xor_sync(0xffffffffu, part, o));
      if (lane == l) nrm = part;
    }
    if (c < ncols) {
      norm2[c0 + c] = nrm;
      acc = sat_add64(acc, nrm);
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    acc = sat_add64(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
    vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  }
  const int64_t ntiles = (n_cols + SCAN_TILE - 1) / SCAN_TILE;
  if (lane == 0) {
    segs[warp] = acc;
    const int64_t tile = (c0 / SCAN_TILE) + warp / SCAN_WARPS;
    if (tile < ntiles) warp_sums[tile * SCAN_WARPS + (warp % SCAN_WARPS)] = acc;
    if (vmin <= vmax) {
      atomicMin(minkey, (unsigned)vmin ^ 0x80000000u);
      atomicMin(minkey + 1, ~((unsigned)vmax ^ 0x80000000u));
    }
  }
  __syncthreads();
  if (t < MQ_THREADS / 32 / SCAN_WARPS) {
    const int64_t tile = (c0 / SCAN_TILE) + t;
    if (tile < ntiles) {
      unsigned long long x = 0;
      for (int w = 0; w < SCAN_WARPS; ++w) x = sat_add64(x, segs[t * SCAN_WARPS + w]);
      tile_sum[tile] = x;
    }
  }
}
static_assert(MQ_THREADS / 32 == 2 * SCAN_WARPS, "a place block covers two scan tiles");

}  // namespace

// The bucketed matricization, when the shape suits it: at least two buckets
// per SM, at most MB_MAX_BUCKETS, and no bucket above twice what a place
// block stages (checked on the device after the count; one read-back).
// Returns CTD_OK with *used = false, having written nothing the plain path
// needs, when it does not suit.  M's arrays are allocated by the caller;
// rowcnt, status and minval are zeroed / initialized by the caller.
ctd_status matricize_bucketed(const CooDev& X, Arena& A, cudaStream_t st, Matricized* M,
                              bool* used, int wshift) {
  *used = false;
  const int64_t nb64 = (M->n_cols + MB_W - 1) / MB_W;
  if (X.nnz == 0 || nb64 < 2 * (int64_t)num_sms() || nb64 > MB_MAX_BUCKETS) return CTD_OK;
  const int nb = (int)nb64;
  const bool vec = ((reinterpret_cast<uintptr_t>(X.i) | reinterpret_cast<uintptr_t>(X.j) |
                     reinterpret_cast<uintptr_t>(X.k) | reinterpret_cast<uintptr_t>(X.v)) & 15) == 0;
  const ModeMap mm = make_mode_map(X.dims, X.alpha);
  uint32_t* bcnt;
  uint64_t* bstart;
  unsigned* bmax;
  CTD_TRY(A.get(&bcnt, nb));
  CTD_TRY(A.get(&bstart, nb + 1));
  CTD_TRY(A.get(&bmax, 1));
  CTD_CUDA(cudaMemsetAsync(bcnt, 0, nb * sizeof(uint32_t), st));
  CTD_CUDA(cudaMemsetAsync(bmax, 0, sizeof(unsigned), st));
  {
    const bool priv = M->n_rows <= ROW_SMEM_MAX;
    const size_t smem = ((size_t)nb + (priv ? (size_t)M->n_rows : 0)) * 4;
    const void* fn = vec ? (const void*)k_mb_count<true> : (const void*)k_mb_count<false>;
    if (smem > 48 * 1024) CTD_TRY(allow_max_smem(fn));
    const unsigned g = grid_for((X.nnz + 3) / 4, MC_THREADS, (int64_t)num_sms() * 2);
    if (vec)
      CTD_LAUNCH(k_mb_count<true>, (g), (MC_THREADS), smem, st, X.i, X.j, X.k, X.nnz, mm,
                 M->n_rows, nb, bcnt, M->rowcnt, M->status);
    else
      CTD_LAUNCH(k_mb_count<false>, (g), (MC_THREADS), smem, st, X.i, X.j, X.k, X.nnz, mm,
                 M->n_rows, nb, bcnt, M->rowcnt, M->status);
  }
  CTD_LAUNCH(k_mb_max, (1), (1024), 0, st, bcnt, nb, bmax);
  unsigned h_max = 0;
  CTD_TRY(d2h(&h_max, bmax, 1, st));
  CTD_TRY(sync(st));
  if (h_max > 2u * (unsigned)MQ_CAP) {
    // skewed buckets: the plain passes recount the rows
    CTD_CUDA(cudaMemsetAsync(M->rowcnt, 0, M->n_rows * sizeof(uint32_t), st));
    return CTD_OK;
  }
  // bucket offsets; bcnt becomes each bucket's cursor
  launch_scan_u32(bcnt, bstart, nb, false, M->tmp, M->status, st, bcnt);
  uint16_t* stg_lc;
  int32_t *stg_row, *stg_val;
  CTD_TRY(A.get(&stg_lc, X.nnz));
  CTD_TRY(A.get(&stg_row, X.nnz));
  CTD_TRY(A.get(&stg_val, X.nnz));
  {
    const void* fn = vec ? (const void*)k_mb_part<true> : (const void*)k_mb_part<false>;
    CTD_TRY(allow_max_smem(fn));
    const int64_t chunks = (X.nnz + MP_CHUNK - 1) / MP_CHUNK;
    const unsigned g = (unsigned)std::min<int64_t>(chunks, (int64_t)num_sms());
    if (vec)
      CTD_LAUNCH(k_mb_part<true>, (g), (MP_THREADS), MP_SMEM, st, X.i, X.j, X.k, X.v, X.nnz, mm,
                 nb, bcnt, stg_lc, stg_row, stg_val);
    else
      CTD_LAUNCH(k_mb_part<false>, (g), (MP_THREADS), MP_SMEM, st, X.i, X.j, X.k, X.v, X.nnz, mm,
                 nb, bcnt, stg_lc, stg_row, stg_val);
  }
  {
    CTD_TRY(allow_max_smem((const void*)k_mb_place));
    const int64_t ntiles = (M->n_cols + SCAN_TILE - 1) / SCAN_TILE;
    unsigned long long* ts = reinterpret_cast<unsigned long long*>(M->tmp);
    CTD_LAUNCH(k_mb_place, (nb), (MQ_THREADS), MQ_SMEM, st,
               reinterpret_cast<const unsigned long long*>(bstart), nb, M->n_cols, stg_lc,
               stg_row, stg_val, reinterpret_cast<unsigned long long*>(M->colptr), M->csc_row,
               M->csc_val, reinterpret_cast<unsigned long long*>(M->norm2), ts, ts + ntiles + 2,
               M->minval, wshift);
  }
  *used = true;
  return CTD_OK;
}

}  // namespace ctd
