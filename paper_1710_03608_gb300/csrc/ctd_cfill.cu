// C = R^T X_(alpha) (Algorithm 1, Eq. 3) with register accumulators.
//
// On count data the products are dominated by a few long rows of R (the
// frequent mode-alpha indices occur in many sampled fibers): on a Zipf(1.2)
// traffic tensor with 10^7 nonzeros and s~ = 456, the 100 longest of 8.5K
// nonempty rows carry 95% of the 1.5 * 10^9 products.  Walking such a row
// costs two global loads and one shared-memory atomic per product.  Here the
// H longest rows live densely in shared memory (int8, int16 or int32, the
// narrowest R's values fit, padded to NQ * 128 columns), and lane l of a
// warp owns output rows m = 128 q + 4 l + {0..3} in registers: dense rows
// add into them from shared loads with integer multiply-adds (with int8
// rows and X's values in int8, four rows at a time by dp4a), no atomics.  The other rows go through a
// sparse walk into a per-warp shared accumulator, and the emission adds the
// two, compacts the nonzeros of each 128-row slab (ballots) through shared
// memory and writes them in ascending row order, consecutive lanes on
// consecutive entries.  A column with one nonzero v at row
// i is v R(i, :): those are copied from images of R's rows laid out so that
// every copy moves aligned 8- and 16-byte vectors (k_img_fill, k_copy_flat).
// The columns are sorted into those kinds by k_bounds_classify, in the pass
// that computes their capacities (or by k_classify where that pass is the
// plain one).
//
// Exactness: every partial sum is an integer of magnitude at most
// ||x_f|| ||r_m|| <= ||X||_F^2 < 2^31 (Cauchy-Schwarz); this path is taken
// only then.  Which rows are dense changes the order of integer additions
// only, so the result does not depend on the selection.
#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "ctd_expand.cuh"
#include "ctd_internal.cuh"

namespace ctd {

namespace {

// one 24-warp block per SM shares one copy of the dense rows (24 rather than
// 32 warps: 80 registers a thread instead of 64, and fewer accumulators
// leave room for more dense rows; measured faster on the traffic tensor)
constexpr int CF_THREADS = 768;
constexpr int CF_HEAVY_COL = 128;  // columns with at least this many nonzeros: taken first
constexpr int CF_LONG_ROW = 16;    // sparse rows at least this long: walked by the whole warp
constexpr int CF_LONG_GROUP = 2;   // long sparse rows walked together (loads in flight)
constexpr int CF_MAX_DENSE = 320;  // dense rows at most (shared memory bounds it first)

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
// (width + 1 if none qualifies).  One warp walks the lengths down from
// `width` 32 at a time: a prefix sum over the lanes gives #rows(len >= L)
// for each lane's L, and the first lane past hmax ends the walk (the count
// only grows as L falls).
__global__ void k_pick_len(const unsigned* __restrict__ hist, int width, int minlen, int hmax,
                           int* __restrict__ thr) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  unsigned long long carry = 0;
  int L = width + 1;
  for (int top = width; top >= minlen; top -= 32) {
    const int len = top - lane;
    unsigned long long x = len >= minlen ? hist[len] : 0ull;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    const bool over = len >= minlen && carry + x > (unsigned long long)hmax;
    const unsigned ob = __ballot_sync(0xffffffffu, over);
    const unsigned ok = __ballot_sync(0xffffffffu, len >= minlen && !over);
    if (ob) {
      // lanes before the first one over are fine: the last of them is L
      const int first = __ffs(ob) - 1;
      if (first > 0) L = top - (first - 1);
      break;
    }
    if (ok) L = top - (31 - __clz(ok));  // every length of this chunk is fine
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) thr[0] = L;
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

// Fill the dense rows (H x W entries of DB bytes at `dense`: int8, int16 or
// int32) and zero `acc_n` ints at `acc`.  R's values fit the entry type
// (checked on the host from max |R|).
template <int DB>
__device__ __forceinline__ void load_dense(const CsrDev& R, const Dense& dn, void* dense_v, int W,
                                           int* acc, int acc_n) {
  using DT = typename std::conditional<DB == 1, signed char,
                                       typename std::conditional<DB == 2, short, int>::type>::type;
  DT* dense = static_cast<DT*>(dense_v);
  const int H = min(*dn.count, dn.hmax);
  for (int e = threadIdx.x; e < H * W; e += blockDim.x) dense[e] = 0;
  for (int e = threadIdx.x; e < acc_n; e += blockDim.x) acc[e] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  for (int h = warp; h < H; h += nw) {
    const int i = dn.rows[h];
    for (unsigned long long p = rp[i] + lane; p < rp[i + 1]; p += 32)
      dense[h * W + __ldg(R.col + p)] = (DT)__ldg(R.val + p);
  }
  __syncthreads();
}


// Sort the columns by how C's column is formed (from the column bounds ub =
// coff[f+1] - coff[f] and the nonzero counts): ub = 0, the column is empty
// (count 0); one nonzero with positive values: a scaled copy of one row of
// R (`single`, count = ub); at least CF_HEAVY_COL nonzeros: `heavy`; else
// `multi`.  Appends are warp-aggregated; the order inside a list does not
// matter (every column writes its own output range).
constexpr int CL_ITEMS = 8;  // columns per thread in k_classify and k_bounds_classify

__global__ void __launch_bounds__(256)
    k_classify(const unsigned long long* __restrict__ xp,
               const unsigned long long* __restrict__ coff, int64_t n_cols, int positive,
               unsigned* __restrict__ ccnt, int64_t* __restrict__ single,
               unsigned* __restrict__ n_single, int64_t* __restrict__ heavy,
               unsigned* __restrict__ n_heavy, int64_t* __restrict__ multi,
               unsigned* __restrict__ n_multi) {
  __shared__ unsigned cnt[3], base[3];
  const int lane = threadIdx.x & 31;
  const int64_t span = (int64_t)blockDim.x * CL_ITEMS;
  for (int64_t b0 = (int64_t)blockIdx.x * span; b0 < n_cols; b0 += (int64_t)gridDim.x * span) {
    if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
    __syncthreads();
    int kind[CL_ITEMS];
    unsigned off[CL_ITEMS];
    // every item's offsets first, so their loads are in flight together
    unsigned long long ubs[CL_ITEMS], nxs[CL_ITEMS];
#pragma unroll
    for (int u = 0; u < CL_ITEMS; ++u) {
      const int64_t f = b0 + (int64_t)u * blockDim.x + threadIdx.x;
      ubs[u] = f < n_cols ? coff[f + 1] - coff[f] : 0ull;
      nxs[u] = f < n_cols ? xp[f + 1] - xp[f] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < CL_ITEMS; ++u) {
      const int64_t f = b0 + (int64_t)u * blockDim.x + threadIdx.x;
      int k = -1;  // -1 none, 0 single, 1 heavy, 2 multi
      if (f < n_cols) {
        const unsigned long long ub = ubs[u];
        const unsigned long long nx = nxs[u];
        if (ub == 0) {
          ccnt[f] = 0;
        } else if (nx == 1 && positive) {
          k = 0;  // the copy writes the count (R's row length)
        } else {
          k = nx >= (unsigned long long)CF_HEAVY_COL ? 1 : 2;
        }
      }
      kind[u] = k;
      off[u] = 0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const unsigned m = __ballot_sync(0xffffffffu, k == q);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        unsigned wb = 0;
        if (lane == leader) wb = atomicAdd(&cnt[q], (unsigned)__popc(m));
        wb = __shfl_sync(0xffffffffu, wb, leader);
        if (k == q) off[u] = wb + __popc(m & ((1u << lane) - 1));
      }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      unsigned* g = threadIdx.x == 0 ? n_single : threadIdx.x == 1 ? n_heavy : n_multi;
      base[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(g, cnt[threadIdx.x]) : 0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < CL_ITEMS; ++u) {
      const int k = kind[u];
      if (k < 0) continue;
      const int64_t f = b0 + (int64_t)u * blockDim.x + threadIdx.x;
      int64_t* out = k == 0 ? single : k == 1 ? heavy : multi;
      out[base[k] + off[u]] = f;
    }
    __syncthreads();
  }
}

// The C bounds and the column lists in one pass (what k_c_bounds and
// k_classify do separately): per column the bound ub = min(width, sum of
// the R row lengths of its entries) rounded up to a multiple of 4, written
// to ub; an empty bound gives ccnt = 0, else the column joins one of the
// three lists as k_classify would put it (appends warp-aggregated into
// shared counters, one global atomic per list per block and round).
__global__ void __launch_bounds__(256)
    k_bounds_classify(CscDev X, int64_t n_cols, CsrDev R, unsigned* __restrict__ ub, int positive,
                      unsigned* __restrict__ ccnt, int64_t* __restrict__ single,
                      int64_t* __restrict__ heavy, int64_t* __restrict__ multi,
                      unsigned* __restrict__ counts) {
  __shared__ unsigned cnt[3], base[3];
  const int lane = threadIdx.x & 31;
  const unsigned long long* xp = reinterpret_cast<const unsigned long long*>(X.colptr);
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  const unsigned long long width = (unsigned long long)R.width;
  const int64_t span = (int64_t)blockDim.x * CL_ITEMS;
  for (int64_t b0 = (int64_t)blockIdx.x * span; b0 < n_cols; b0 += (int64_t)gridDim.x * span) {
    if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
    __syncthreads();
    int kind[CL_ITEMS];
    unsigned off[CL_ITEMS];
    unsigned long long xa[CL_ITEMS], xb[CL_ITEMS];
#pragma unroll
    for (int u = 0; u < CL_ITEMS; ++u) {
      const int64_t f = b0 + (int64_t)u * blockDim.x + threadIdx.x;
      xa[u] = f < n_cols ? xp[f] : 0ull;
      xb[u] = f < n_cols ? xp[f + 1] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < CL_ITEMS; ++u) {
      const int64_t f = b0 + (int64_t)u * blockDim.x + threadIdx.x;
      int k = -1;  // -1 none, 0 single, 1 heavy, 2 multi
      if (f < n_cols) {
        unsigned long long sum = 0;
        for (unsigned long long p = xa[u]; p < xb[u] && sum < width; ++p) {
          const int i = __ldg(X.row + p);
          sum += __ldg(rp + i + 1) - __ldg(rp + i);
        }
        const unsigned bound = ((unsigned)min(sum, width) + 3u) & ~3u;
        ub[f] = bound;
        const unsigned long long nx = xb[u] - xa[u];
        if (bound == 0)
          ccnt[f] = 0;
        else if (nx == 1 && positive)
          k = 0;
        else
          k = nx >= (unsigned long long)CF_HEAVY_COL ? 1 : 2;
      }
      kind[u] = k;
      off[u] = 0;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const unsigned m = __ballot_sync(0xffffffffu, k == q);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        unsigned wb = 0;
        if (lane == leader) wb = atomicAdd(&cnt[q], (unsigned)__popc(m));
        wb = __shfl_sync(0xffffffffu, wb, leader);
        if (k == q) off[u] = wb + __popc(m & ((1u << lane) - 1));
      }
    }
    __syncthreads();
    if (threadIdx.x < 3)
      base[threadIdx.x] = cnt[threadIdx.x] ? atomicAdd(counts + threadIdx.x, cnt[threadIdx.x]) : 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < CL_ITEMS; ++u) {
      const int k = kind[u];
      if (k < 0) continue;
      const int64_t f = b0 + (int64_t)u * blockDim.x + threadIdx.x;
      int64_t* out = k == 0 ? single : k == 1 ? heavy : multi;
      out[base[k] + off[u]] = f;
    }
    __syncthreads();
  }
}

// four consecutive values, 16-byte aligned (float) or two 16-byte halves (double)
template <typename V>
__device__ __forceinline__ void store4(V* p, V a, V b, V c, V d);
template <>
__device__ __forceinline__ void store4<float>(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
template <>
__device__ __forceinline__ void store4<double>(double* p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

// R's rows at four alignments, for the copies: image k (k = 0..3) holds row
// i at ip[i] + k + e (e = 0..len-1) inside a slot of roundup(len + 3, 4)
// entries that starts at the 4-aligned ip[i], zeros elsewhere, columns as
// uint16.  An output run starting at o reads image (o mod 4), where every
// 4-aligned quad of the run lines up with a 4-aligned quad of the image:
// 8- and 16-byte loads and stores throughout.
__global__ void k_img_sizes(const unsigned long long* __restrict__ rp, int64_t n_rows,
                            unsigned long long* __restrict__ sz) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_rows;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long len = rp[i + 1] - rp[i];
    sz[i] = len ? ((len + 6ull) & ~3ull) : 0ull;
  }
}

__global__ void k_img_fill(CsrDev R, int64_t n_rows, const unsigned long long* __restrict__ ip,
                           int64_t P, uint16_t* __restrict__ icol, int* __restrict__ ival) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  for (int64_t i = gw; i < n_rows; i += nw) {
    const unsigned long long rs = rp[i];
    const long long len = (long long)(rp[i + 1] - rs);
    const unsigned long long b = ip[i], S = ip[i + 1] - b;
    for (unsigned long long j = lane; j < S; j += 32) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long long e = (long long)j - k;
        const bool in = e >= 0 && e < len;
        icol[(int64_t)k * P + b + j] = in ? (uint16_t)__ldg(R.col + rs + e) : (uint16_t)0;
        ival[(int64_t)k * P + b + j] = in ? __ldg(R.val + rs + e) : 0;
      }
    }
  }
}

template <typename V>
__device__ __forceinline__ void put_quad(uint16_t* crow, V* cval, unsigned long long o, ushort4 c,
                                         V a, V b, V d, V e);
template <>
__device__ __forceinline__ void put_quad<float>(uint16_t* crow, float* cval, unsigned long long o,
                                                ushort4 c, float a, float b, float d, float e) {
  *reinterpret_cast<ushort4*>(crow + o) = c;
  *reinterpret_cast<float4*>(cval + o) = make_float4(a, b, d, e);
}
template <>
__device__ __forceinline__ void put_quad<double>(uint16_t* crow, double* cval, unsigned long long o,
                                                 ushort4 c, double a, double b, double d, double e) {
  *reinterpret_cast<ushort4*>(crow + o) = c;
  reinterpret_cast<double2*>(cval + o)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(cval + o)[1] = make_double2(d, e);
}

// The copies of a warp's 32 list entries as one flat sequence of image
// quads: entry e's run is nq_e quads, and lane l owns quads l, l + 32, ...
// of the concatenated runs (found by a binary search over the lanes'
// inclusive prefix sums of nq), CP_UNROLL rounds of loads in flight before
// their stores.  The L2 latency of the image loads is then paid once per
// 32 * CP_UNROLL quads instead of once or twice per row.

__device__ __forceinline__ unsigned long long shfl64(unsigned long long x, int src) {
  return __shfl_sync(0xffffffffu, x, src);
}

template <typename V, int UNR, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_copy_flat(CscDev X, const unsigned long long* __restrict__ rp,
                const unsigned long long* __restrict__ ip, const uint16_t* __restrict__ icol,
                const int* __restrict__ ival, int64_t P, const int64_t* __restrict__ single,
                const unsigned* __restrict__ n_single,
                const unsigned long long* __restrict__ coff, unsigned* __restrict__ ccnt,
                uint16_t* __restrict__ crow, V* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned long long* xp = reinterpret_cast<const unsigned long long*>(X.colptr);
  const int64_t n = *n_single;
  for (int64_t w0 = gw * 32; w0 < n; w0 += nw * 32) {
    unsigned long long b = 0, o = 0;
    int rl = 0, v = 0;
    if (w0 + lane < n) {
      const int64_t f = single[w0 + lane];
      const unsigned long long xa = xp[f];
      o = coff[f];
      const int i = __ldg(X.row + xa);
      v = __ldg(X.val + xa);
      b = __ldg(ip + i);
      rl = (int)(__ldg(rp + i + 1) - __ldg(rp + i));
      ccnt[f] = (unsigned)rl;  // v > 0 and R > 0: every product is nonzero
    }
    const int nq = rl > 0 ? ((int)(o & 3ull) + rl + 3) >> 2 : 0;
    int incl = nq;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    const int excl = incl - nq;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    for (int g0 = 0; g0 < total; g0 += 32 * UNR) {
      ushort4 c[UNR];
      int4 w[UNR];
      unsigned long long oq[UNR];
      int lo[UNR], hi[UNR], vv[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int g = g0 + 32 * u + lane;
        const int gg = min(g, total - 1);
        // e = number of entries whose run ends at or before quad gg
        int e = 0;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1)
          if (__shfl_sync(0xffffffffu, incl, e + s - 1) <= gg) e += s;
        const int t = gg - __shfl_sync(0xffffffffu, excl, e);
        const unsigned long long be = shfl64(b, e), oe = shfl64(o, e);
        const int rle = __shfl_sync(0xffffffffu, rl, e);
        vv[u] = __shfl_sync(0xffffffffu, v, e);
        const int k = (int)(oe & 3ull);
        oq[u] = oe - (unsigned long long)k + 4ull * (unsigned long long)t;
        lo[u] = k - 4 * t;        // entries u' of the quad in [lo, hi) belong to the run
        hi[u] = k + rle - 4 * t;
        if (g >= total) hi[u] = -1;  // idle
        const int64_t off = (int64_t)k * P + (int64_t)be + 4 * (int64_t)t;
        if (g < total) {
          c[u] = *reinterpret_cast<const ushort4*>(icol + off);
          w[u] = *reinterpret_cast<const int4*>(ival + off);
        }
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        if (hi[u] <= 0) continue;
        const int ve = vv[u];
        const V a0 = (V)(ve * w[u].x), a1 = (V)(ve * w[u].y), a2 = (V)(ve * w[u].z),
                a3 = (V)(ve * w[u].w);
        const unsigned long long ot = oq[u];
        if (lo[u] <= 0 && hi[u] >= 4) {
          put_quad<V>(crow, cval, ot, c[u], a0, a1, a2, a3);
        } else {
          if (0 >= lo[u] && 0 < hi[u]) { crow[ot] = c[u].x; cval[ot] = a0; }
          if (1 >= lo[u] && 1 < hi[u]) { crow[ot + 1] = c[u].y; cval[ot + 1] = a1; }
          if (2 >= lo[u] && 2 < hi[u]) { crow[ot + 2] = c[u].z; cval[ot + 2] = a2; }
          if (3 >= lo[u] && 3 < hi[u]) { crow[ot + 3] = c[u].w; cval[ot + 3] = a3; }
        }
      }
    }
  }
}

// One chunk of up to 32 column entries, one per lane (sl = dense slot or -1;
// rs/rl = the R row's range for a sparse row; rl = 0 for idle lanes):
// dense rows into regs (lane's rows 128 q + 4 lane + k), other rows into the
// shared accumulator acc (atomics).  P4 (int8 dense rows, X's values in
// [-128, 127]): four entries at a time; each lane loads the four rows'
// words for its outputs 4 lane + {0..3}, transposes the 4 x 4 bytes with
// byte permutes so that each word holds one output's four row values, and
// adds the four products with one dp4a per output (exact int32 sums).
template <int NQ, int DB, bool P4>
__device__ __forceinline__ void chunk_reg(const CsrDev& R, const void* __restrict__ dense_v,
                                          int* acc, int (&regs)[4 * NQ], int v, int sl,
                                          unsigned long long rs, int rl) {
  constexpr int W4 = NQ * 32;  // 4-entry groups per dense row
  const int lane = threadIdx.x & 31;
  unsigned dense_b = __ballot_sync(0xffffffffu, sl >= 0);
  if (P4 && DB == 1) {
    while (dense_b) {
      int h[4], vp = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int src = dense_b ? __ffs(dense_b) - 1 : -1;
        if (dense_b) dense_b &= dense_b - 1;
        const int s = src < 0 ? 0 : src;
        const int hs = __shfl_sync(0xffffffffu, sl, s);
        const int vs = __shfl_sync(0xffffffffu, v, s);
        // a missing fourth entry repeats the first row with value 0
        h[u] = src < 0 ? h[0] : hs;
        vp |= ((src < 0 ? 0 : vs) & 0xff) << (8 * u);
      }
      const unsigned* d = static_cast<const unsigned*>(dense_v) + lane;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const unsigned w0 = d[h[0] * W4 + q * 32], w1 = d[h[1] * W4 + q * 32];
        const unsigned w2 = d[h[2] * W4 + q * 32], w3 = d[h[3] * W4 + q * 32];
        const unsigned lo01 = __byte_perm(w0, w1, 0x5140), hi01 = __byte_perm(w0, w1, 0x7362);
        const unsigned lo23 = __byte_perm(w2, w3, 0x5140), hi23 = __byte_perm(w2, w3, 0x7362);
        regs[4 * q + 0] = __dp4a((int)__byte_perm(lo01, lo23, 0x5410), vp, regs[4 * q + 0]);
        regs[4 * q + 1] = __dp4a((int)__byte_perm(lo01, lo23, 0x7632), vp, regs[4 * q + 1]);
        regs[4 * q + 2] = __dp4a((int)__byte_perm(hi01, hi23, 0x5410), vp, regs[4 * q + 2]);
        regs[4 * q + 3] = __dp4a((int)__byte_perm(hi01, hi23, 0x7632), vp, regs[4 * q + 3]);
      }
    }
  }
  while (dense_b) {
    const int src = __ffs(dense_b) - 1;
    dense_b &= dense_b - 1;
    const int h = __shfl_sync(0xffffffffu, sl, src);
    const int vs = __shfl_sync(0xffffffffu, v, src);
    if (DB == 1) {
      // four int8 per 4-byte load, sign-extended
      const unsigned* d = static_cast<const unsigned*>(dense_v) + h * W4 + lane;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int x = (int)d[q * 32];
        regs[4 * q + 0] += vs * ((x << 24) >> 24);
        regs[4 * q + 1] += vs * ((x << 16) >> 24);
        regs[4 * q + 2] += vs * ((x << 8) >> 24);
        regs[4 * q + 3] += vs * (x >> 24);
      }
    } else if (DB == 2) {
      // four int16 per 8-byte load, sign-extended
      const uint2* d = static_cast<const uint2*>(dense_v) + h * W4 + lane;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const uint2 x = d[q * 32];
        regs[4 * q + 0] += vs * (int)(short)(x.x & 0xffffu);
        regs[4 * q + 1] += vs * ((int)x.x >> 16);
        regs[4 * q + 2] += vs * (int)(short)(x.y & 0xffffu);
        regs[4 * q + 3] += vs * ((int)x.y >> 16);
      }
    } else {
      const int4* d = static_cast<const int4*>(dense_v) + h * W4 + lane;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int4 x = d[q * 32];
        regs[4 * q + 0] += vs * x.x;
        regs[4 * q + 1] += vs * x.y;
        regs[4 * q + 2] += vs * x.z;
        regs[4 * q + 3] += vs * x.w;
      }
    }
  }
  // the long sparse rows, CF_LONG_GROUP at a time: each lane loads its entries of
  // all of them before the atomics, so their L2 latencies overlap
  unsigned longs = __ballot_sync(0xffffffffu, rl >= CF_LONG_ROW);
  while (longs) {
    unsigned long long s0[CF_LONG_GROUP];
    int nn[CF_LONG_GROUP], vs[CF_LONG_GROUP];
    int maxn = 0;
#pragma unroll
    for (int u = 0; u < CF_LONG_GROUP; ++u) {
      const int src = longs ? __ffs(longs) - 1 : -1;
      if (longs) longs &= longs - 1;
      const int sl = src < 0 ? 0 : src;
      s0[u] = __shfl_sync(0xffffffffu, rs, sl);
      nn[u] = src < 0 ? 0 : __shfl_sync(0xffffffffu, rl, sl);
      vs[u] = __shfl_sync(0xffffffffu, v, sl);
      maxn = max(maxn, nn[u]);
    }
    for (int q = lane; q < maxn; q += 32) {
      int c4[CF_LONG_GROUP], v4[CF_LONG_GROUP];
#pragma unroll
      for (int u = 0; u < CF_LONG_GROUP; ++u)
        if (q < nn[u]) {
          c4[u] = __ldg(R.col + s0[u] + q);
          v4[u] = __ldg(R.val + s0[u] + q);
        }
#pragma unroll
      for (int u = 0; u < CF_LONG_GROUP; ++u)
        if (q < nn[u]) atomicAdd(acc + c4[u], vs[u] * v4[u]);
    }
  }
  if (rl >= CF_LONG_ROW) rl = 0;
  if (__any_sync(0xffffffffu, rl > 0))
    expand_chunk(rs, rl, v, R.col, R.val,
                 [&](int m, long long prod) { atomicAdd(acc + m, (int)prod); });
}

// Row metadata of one entry (row i): dense slot, else the R row's range.
__device__ __forceinline__ void entry_meta(const CsrDev& R, const Dense& dn, int i, int& sl,
                                           unsigned long long& rs, int& rl) {
  sl = -1;
  rs = 0;
  rl = 0;
  if (i < 0) return;
  sl = __ldg(dn.slot + i);
  if (sl < 0) {
    const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
    rs = __ldg(rp + i);
    rl = (int)(__ldg(rp + i + 1) - rs);
  }
}

// Accumulate R^T x_f over the column's entries [a, b): warps of a group
// [gwarp, gwarp + gwarps) take interleaved 32-entry chunks.
template <int NQ, int DB, bool P4>
__device__ __forceinline__ void accumulate_reg(const CscDev& X, const CsrDev& R, const Dense& dn,
                                               const void* __restrict__ dense4,
                                               unsigned long long a, unsigned long long b,
                                               int* acc, int (&regs)[4 * NQ], int gwarp,
                                               int gwarps) {
  const int lane = threadIdx.x & 31;
  for (unsigned long long p0 = a + (unsigned long long)gwarp * 32; p0 < b;
       p0 += (unsigned long long)gwarps * 32) {
    const unsigned long long p = p0 + lane;
    int i = -1, v = 0, sl, rl;
    unsigned long long rs;
    if (p < b) {
      i = __ldg(X.row + p);
      v = __ldg(X.val + p);
    }
    entry_meta(R, dn, i, sl, rs, rl);
    chunk_reg<NQ, DB, P4>(R, dense4, acc, regs, v, sl, rs, rl);
  }
}

template <typename V>
struct IsF32 { static constexpr bool v = false; };
template <>
struct IsF32<float> { static constexpr bool v = true; };

// Emit one column from regs + acc (both left zero).  First the final values
// (registers plus the warp's shared accumulator) and their nonzero count;
// then the column is stored densely (every row's value, zeros included,
// 16-byte stores straight from the registers; count | C_DENSE) when its
// capacity holds all rows and it is dense enough that this writes no more
// bytes than the sparse form (at least 2/3 nonzero with FP32 values, 4/5
// with FP64); otherwise as ascending (row, value) pairs, each lane's
// position from four ballots per 128-row slab, FP32 pairs staged in the
// slab's own accumulator words and the warp's row staging `srow` so that
// consecutive lanes store consecutive entries.
template <typename V, int NQ>
__device__ __forceinline__ unsigned emit_final(int* acc, int (&regs)[4 * NQ], uint16_t* srow,
                                               unsigned long long off, unsigned long long cap,
                                               int width, uint16_t* __restrict__ crow,
                                               V* __restrict__ cval) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int4* acc4 = reinterpret_cast<int4*>(acc);
  unsigned total = 0;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int4 s = acc4[q * 32 + lane];
    acc4[q * 32 + lane] = make_int4(0, 0, 0, 0);
    regs[4 * q] += s.x;
    regs[4 * q + 1] += s.y;
    regs[4 * q + 2] += s.z;
    regs[4 * q + 3] += s.w;
    total += __popc(__ballot_sync(FULL, regs[4 * q] != 0)) +
             __popc(__ballot_sync(FULL, regs[4 * q + 1] != 0)) +
             __popc(__ballot_sync(FULL, regs[4 * q + 2] != 0)) +
             __popc(__ballot_sync(FULL, regs[4 * q + 3] != 0));
  }
  const unsigned long long wpad = (unsigned long long)((width + 3) & ~3);
  const bool dense = cap >= wpad && (IsF32<V>::v ? 3ull * total >= 2ull * (unsigned)width
                                                 : 5ull * total >= 4ull * (unsigned)width);
  if (dense) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int m0 = q * 128 + 4 * lane;
      if (m0 < width)
        store4<V>(cval + off + m0, (V)regs[4 * q], (V)regs[4 * q + 1], (V)regs[4 * q + 2],
                  (V)regs[4 * q + 3]);
      regs[4 * q] = regs[4 * q + 1] = regs[4 * q + 2] = regs[4 * q + 3] = 0;
    }
    return total | C_DENSE;
  }
  __syncwarp();  // every lane's slab words are zero before any lane stages into them
  unsigned pos = 0;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int x0 = regs[4 * q], x1 = regs[4 * q + 1], x2 = regs[4 * q + 2], x3 = regs[4 * q + 3];
    regs[4 * q] = regs[4 * q + 1] = regs[4 * q + 2] = regs[4 * q + 3] = 0;
    const unsigned b0 = __ballot_sync(FULL, x0 != 0);
    const unsigned b1 = __ballot_sync(FULL, x1 != 0);
    const unsigned b2 = __ballot_sync(FULL, x2 != 0);
    const unsigned b3 = __ballot_sync(FULL, x3 != 0);
    const unsigned lt = (1u << lane) - 1;
    int p = __popc(b0 & lt) + __popc(b1 & lt) + __popc(b2 & lt) + __popc(b3 & lt);
    const int tot = __popc(b0) + __popc(b1) + __popc(b2) + __popc(b3);
    const int m0 = q * 128 + 4 * lane;
    if constexpr (IsF32<V>::v) {
      float* sv = reinterpret_cast<float*>(acc) + q * 128;  // the slab's words (zero)
      if (x0) { sv[p] = (float)x0; srow[p] = (uint16_t)m0;       ++p; }
      if (x1) { sv[p] = (float)x1; srow[p] = (uint16_t)(m0 + 1); ++p; }
      if (x2) { sv[p] = (float)x2; srow[p] = (uint16_t)(m0 + 2); ++p; }
      if (x3) { sv[p] = (float)x3; srow[p] = (uint16_t)(m0 + 3); }
      __syncwarp();
      const unsigned long long o = off + pos;
      for (int j = lane; j < tot; j += 32) {
        crow[o + j] = srow[j];
        cval[o + j] = sv[j];
      }
      __syncwarp();
      acc4[q * 32 + lane] = make_int4(0, 0, 0, 0);
    } else {
      unsigned long long o = off + pos + (unsigned)p;
      if (x0) { crow[o] = (uint16_t)m0;       cval[o] = (V)x0; ++o; }
      if (x1) { crow[o] = (uint16_t)(m0 + 1); cval[o] = (V)x1; ++o; }
      if (x2) { crow[o] = (uint16_t)(m0 + 2); cval[o] = (V)x2; ++o; }
      if (x3) { crow[o] = (uint16_t)(m0 + 3); cval[o] = (V)x3; }
    }
    pos += (unsigned)tot;
  }
  return pos;
}

// One persistent kernel, one block per SM sharing the dense rows; a
// warp per column, first the columns with at least CF_HEAVY_COL nonzeros
// (`list`, the longest work items), then the other multi-nonzero columns
// (`mlist`).  Each warp's accumulator is left zero by its emission.
template <typename V, int NQ, int DB, bool P4>
__global__ void __launch_bounds__(CF_THREADS, 1)
    k_cf(CscDev X, CsrDev R, Dense dn, const int64_t* __restrict__ list,
         const unsigned* __restrict__ nlist, const int64_t* __restrict__ mlist,
         const unsigned* __restrict__ mcount, const unsigned long long* __restrict__ coff,
         unsigned* __restrict__ ccnt, uint16_t* __restrict__ crow, V* __restrict__ cval,
         unsigned long long* work) {
  extern __shared__ int4 smem4[];
  constexpr int W = NQ * 128;
  unsigned char* dense = reinterpret_cast<unsigned char*>(smem4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  int* accs = reinterpret_cast<int*>(dense + (size_t)dn.hmax * W * DB);
  load_dense<DB>(R, dn, dense, W, accs, nw * W);
  const void* dense4 = dense;
  int regs[4 * NQ];
#pragma unroll
  for (int k = 0; k < 4 * NQ; ++k) regs[k] = 0;
  int* acc = accs + warp * W;
  // row staging of the emission: 128 entries per warp after the accumulators
  uint16_t* srow = reinterpret_cast<uint16_t*>(accs + nw * W) + warp * 128;
  // the columns of the heavy list, one per warp grab (the longest work items
  // first), then those of the multi list, `grab` per warp grab
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int64_t* lst = pass == 0 ? list : mlist;
    const unsigned long long nm = pass == 0 ? *nlist : *mcount;
    unsigned long long* counter = pass == 0 ? work + 1 : work;
    const unsigned long long warps_all = (unsigned long long)gridDim.x * nw;
    const int grab = pass == 0 ? 1 : (int)max(1ull, min(32ull, nm / (warps_all * 4ull)));
    while (true) {
      unsigned long long i0 = 0;
      if (lane == 0) i0 = atomicAdd(counter, (unsigned long long)grab);
      i0 = __shfl_sync(0xffffffffu, i0, 0);
      if (i0 >= nm) break;
      // lane l: list entry l's column, output offset and entry range
      unsigned long long o = 0, xa = 0, xb = 0;
      int64_t f = -1;
      if (lane < grab && i0 + lane < nm) {
        f = lst[i0 + lane];
        o = coff[f];
        xa = X.colptr[f];
        xb = X.colptr[f + 1];
      }
      unsigned todo = __ballot_sync(0xffffffffu, f >= 0);
      // software pipeline over the grabbed columns: the next column's first
      // chunk (entries, then their row metadata) is loaded while the current
      // one accumulates and emits
      int e = todo ? __ffs(todo) - 1 : 0;
      unsigned long long ea = __shfl_sync(0xffffffffu, xa, e);
      unsigned long long eb = __shfl_sync(0xffffffffu, xb, e);
      int ci = -1, cv = 0;
      if (todo && ea + lane < eb) {
        ci = __ldg(X.row + ea + lane);
        cv = __ldg(X.val + ea + lane);
      }
      int csl, crl;
      unsigned long long crs;
      entry_meta(R, dn, ci, csl, crs, crl);
      while (todo) {
        todo &= todo - 1;
        const unsigned long long oe = __shfl_sync(0xffffffffu, o, e);
        const int64_t fe = __shfl_sync(0xffffffffu, f, e);
        const unsigned long long ce = coff[fe + 1] - oe;  // capacity (read early)
        // issue the next column's first-chunk loads
        const int e2 = todo ? __ffs(todo) - 1 : 0;
        const unsigned long long na = __shfl_sync(0xffffffffu, xa, e2);
        const unsigned long long nb = __shfl_sync(0xffffffffu, xb, e2);
        int ni = -1, nv = 0;
        if (todo && na + lane < nb) {
          ni = __ldg(X.row + na + lane);
          nv = __ldg(X.val + na + lane);
        }
        chunk_reg<NQ, DB, P4>(R, dense4, acc, regs, cv, csl, crs, crl);
        if (eb - ea > 32)
          accumulate_reg<NQ, DB, P4>(X, R, dn, dense4, ea + 32, eb, acc, regs, 0, 1);
        // the next column's row metadata, then this column's emission
        entry_meta(R, dn, ni, csl, crs, crl);
        cv = nv;
        __syncwarp();
        const unsigned n = emit_final<V, NQ>(acc, regs, srow, oe, ce, R.width, crow, cval);
        __syncwarp();
        if (lane == 0) ccnt[fe] = n;
        e = e2;
        ea = na;
        eb = nb;
      }
    }
  }
}

template <typename V, int NQ, int DB, bool P4>
ctd_status cf_launch(const CscDev& X, const CsrDev& R, const Dense& dn,
                     const unsigned long long* coff, uint32_t* ccnt, uint16_t* crow, V* cval,
                     const int64_t* heavy, const unsigned* nheavy, const int64_t* multi,
                     const unsigned* nmulti, unsigned long long* work, cudaStream_t st) {
  constexpr int W = NQ * 128;
  const size_t smem = (size_t)dn.hmax * W * DB +
                      (size_t)(CF_THREADS / 32) * W * sizeof(int) +
                      (size_t)(CF_THREADS / 32) * 128 * sizeof(uint16_t);
  CTD_TRY(allow_max_smem((const void*)k_cf<V, NQ, DB, P4>));
  int per_sm = 0;
  CTD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cf<V, NQ, DB, P4>, CF_THREADS,
                                                         smem));
  if (per_sm < 1) return fail(CTD_ENOTSUP, "C fill: shared memory for the dense rows too large");
  CTD_LAUNCH((k_cf<V, NQ, DB, P4>), (num_sms() * per_sm), (CF_THREADS), smem, st, X, R, dn, heavy,
             nheavy, multi, nmulti, coff, ccnt, crow, cval, work);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

template <typename V>
ctd_status cf_all(int nq, int db, bool p4, const CscDev& X, int64_t n_cols, int64_t n_rows, const CsrDev& R,
                  const Dense& dn,
                  const unsigned long long* coff, uint32_t* ccnt, uint16_t* crow, V* cval,
                  int positive, int64_t list_cap, Arena& a, cudaStream_t st,
                  const CfillLists* lists) {
  int64_t *single, *heavy, *multi;
  unsigned* counts;
  unsigned long long* work;
  CTD_TRY(a.get(&work, 2));
  CTD_CUDA(cudaMemsetAsync(work, 0, 2 * sizeof(unsigned long long), st));
  if (lists) {  // built with the C bounds
    single = lists->single;
    heavy = lists->heavy;
    multi = lists->multi;
    counts = lists->counts;
  } else {
    CTD_TRY(a.get(&single, list_cap));
    CTD_TRY(a.get(&heavy, list_cap));
    CTD_TRY(a.get(&multi, list_cap));
    CTD_TRY(a.get(&counts, 3));
    CTD_CUDA(cudaMemsetAsync(counts, 0, 3 * sizeof(unsigned), st));
    CTD_LAUNCH(k_classify, (grid_for(n_cols, 256 * CL_ITEMS, (int64_t)num_sms() * 8)), (256), 0,
               st, reinterpret_cast<const unsigned long long*>(X.colptr), coff, n_cols, positive,
               ccnt, single, counts, heavy, counts + 1, multi, counts + 2);
  }
  // row images (see k_img_sizes): P entries per image, a multiple of 4
  unsigned long long *sz, *ip, *stmp;
  unsigned* sstat;
  CTD_TRY(a.get(&sz, n_rows));
  CTD_TRY(a.get(&ip, n_rows + 1));
  CTD_TRY(a.get(&stmp, scan_tmp_elems(n_rows)));
  CTD_TRY(a.get(&sstat, 1));
  const int64_t P = (R.nnz + 6 * n_rows + 3) & ~(int64_t)3;
  uint16_t* icol;
  int* ival;
  CTD_TRY(a.get(&icol, 4 * P));
  CTD_TRY(a.get(&ival, 4 * P));
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  const unsigned g = grid_for(n_rows, 256, (int64_t)num_sms() * 4);
  CTD_LAUNCH(k_img_sizes, (g), (256), 0, st, rp, n_rows, sz);
  // exclusive: n_rows + 1 outputs, ip[n_rows] = the images' total
  launch_scan_u64(reinterpret_cast<const uint64_t*>(sz), reinterpret_cast<uint64_t*>(ip),
                  n_rows, false, reinterpret_cast<uint64_t*>(stmp), sstat, st);
  CTD_LAUNCH(k_img_fill, (grid_for(n_rows * 32, 256, (int64_t)num_sms() * 8)), (256), 0, st, R,
             n_rows, ip, P, icol, ival);
  {
    PhaseScope ph("c_fill_copy", st);
    // four rounds of loads in flight; tighter register bounds (more warps
    // per SM) measured no faster: the copy is bound by its stores
    CTD_LAUNCH((k_copy_flat<V, 4, 1>), (num_sms() * (int)tuning(TUNE_COPY_BLOCKS)), (256), 0, st,
               X, rp, ip, icol, ival, P,
               single, counts, coff, ccnt, crow, cval);
  }
  PhaseScope ph("c_fill_multi", st);
#define CF_GO(NQV, DBV, P4V)                                                                  \
  return cf_launch<V, NQV, DBV, P4V>(X, R, dn, coff, ccnt, crow, cval, heavy, counts + 1, multi, \
                                     counts + 2, work, st)
#define CF_NQ(DBV, P4V)          \
  switch (nq) {                  \
    case 1: CF_GO(1, DBV, P4V);  \
    case 2: CF_GO(2, DBV, P4V);  \
    case 4: CF_GO(4, DBV, P4V);  \
    default: CF_GO(8, DBV, P4V); \
  }
  if (db == 1 && p4) CF_NQ(1, true)
  if (db == 1) CF_NQ(1, false)
  if (db == 2) CF_NQ(2, false)
  CF_NQ(4, false)
#undef CF_NQ
#undef CF_GO
}

}  // namespace

// C fill with dense long rows and register accumulators; requires
// ||X||_F^2 < 2^31 and s~ <= 1024 (the caller checks).
ctd_status c_fill_dense_rows(const CscDev& X, int64_t n_cols, int64_t n_rows, int64_t nnz,
                             const CsrDev& R, const uint64_t* coff, uint32_t* ccnt,
                             uint16_t* crow, void* cval, int fp32, int positive, int x_int8,
                             cudaStream_t st, const CfillLists* lists) {
  if (R.nnz < 0) return fail(CTD_EINVAL, "C fill: the entry count of R is not set");
  const int width = R.width;
  const int nq0 = (width + 127) / 128;
  const int nq = nq0 <= 1 ? 1 : nq0 <= 2 ? 2 : nq0 <= 4 ? 4 : 8;
  const int W = nq * 128;
  // dense rows in the narrowest integer type every value of R fits (int8 or
  // int16: four or two times as many rows in the same shared memory)
  const int db = (R.max_abs >= 0 && R.max_abs <= 127) ? 1
                 : (R.max_abs >= 0 && R.max_abs <= 32767) ? 2 : 4;
  const size_t row_b = (size_t)W * db;
  // one block per SM: dense rows, the warps' accumulators and row staging in
  // ~220 KB (a smaller budget keeps fewer rows dense: "cfill_dense_kb")
  const int budget = (int)tuning(TUNE_CFILL_DENSE) * 1024;
  int hmax = (int)((budget - (int64_t)(CF_THREADS / 32) * (256 + W * 4)) / (int64_t)row_b);
  hmax = std::max(0, std::min(hmax, CF_MAX_DENSE));
  const int minlen = std::max(16, 8 * nq);  // shorter rows are cheaper walked sparsely
  Arena a;
  a.st = st;
  unsigned* hist;
  int *thr, *slot, *rows, *count;
  CTD_TRY(a.get(&hist, width + 1));
  CTD_TRY(a.get(&thr, 1));
  CTD_TRY(a.get(&slot, std::max<int64_t>(n_rows, 1)));
  CTD_TRY(a.get(&rows, std::max(hmax, 1)));
  CTD_TRY(a.get(&count, 1));
  CTD_CUDA(cudaMemsetAsync(hist, 0, (width + 1) * sizeof(unsigned), st));
  CTD_CUDA(cudaMemsetAsync(count, 0, sizeof(int), st));
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(R.rowptr);
  const unsigned g = grid_for(n_rows, 256, (int64_t)num_sms() * 4);
  CTD_LAUNCH(k_row_len_hist, (g), (256), 0, st, rp, n_rows, minlen, width, hist);
  CTD_LAUNCH(k_pick_len, (1), (32), 0, st, hist, width, minlen, hmax, thr);
  CTD_LAUNCH(k_assign_slots, (g), (256), 0, st, rp, n_rows, width, thr, slot, rows, count);
  Dense dn{slot, rows, count, hmax};
  const unsigned long long* co = reinterpret_cast<const unsigned long long*>(coff);
  const int64_t list_cap = std::max<int64_t>(1, std::min(n_cols, nnz));
  if (fp32)
    return cf_all<float>(nq, db, x_int8 != 0, X, n_cols, n_rows, R, dn, co, ccnt, crow, static_cast<float*>(cval),
                         positive, list_cap, a, st, lists);
  return cf_all<double>(nq, db, x_int8 != 0, X, n_cols, n_rows, R, dn, co, ccnt, crow, static_cast<double*>(cval),
                        positive, list_cap, a, st, lists);
}

ctd_status launch_c_bounds_lists(const CscDev& X, int64_t n_cols, const CsrDev& R, uint32_t* ub,
                                 int positive, uint32_t* ccnt, const CfillLists& L,
                                 cudaStream_t st) {
  CTD_CUDA(cudaMemsetAsync(L.counts, 0, 3 * sizeof(unsigned), st));
  if (n_cols <= 0) return CTD_OK;
  CTD_LAUNCH(k_bounds_classify, (grid_for(n_cols, 256 * CL_ITEMS, (int64_t)num_sms() * 8)), (256),
             0, st, X, n_cols, R, ub, positive, ccnt, L.single, L.heavy, L.multi, L.counts);
  CTD_CUDA(cudaGetLastError());
  return CTD_OK;
}

}  // namespace ctd
