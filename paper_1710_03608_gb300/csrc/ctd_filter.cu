// The independence filter (Algorithm 1 and Algorithm 2)
// for a block of candidate fibers, with the sequential loop's decisions.
//
// Fast path: an in-order Cholesky with skip of the candidates' Schur
// complement S (see ctd_dense.cu); its pivot for candidate k is
// ||res_k||^2, the squared residual against R^(t) and the candidates kept
// before k.  A Gram-based pivot carries an absolute error of order
// u * |beta|^T |G| |beta| in the SQUARED residual, while the test compares
// ||res|| with eps ||x|| and the paper's eps = 1e-6 puts eps^2 = 1e-12 within
// reach of that error for fibers that depend on an ill-conditioned R.  So
// every candidate whose pivot is below 1e-4 ||x_k||^2 (residual ratio below
// 1e-2; independent fibers mostly sit far above) is re-tested the way the
// loop states it: the residual vector x_k - [R^(t), kept candidates before
// k] gamma is formed explicitly.  Against R^(t) (CTD-D) it is taken through
// the orthonormal basis Q of range(R^(t)) that the dynamic state keeps, so
// its accuracy does not depend on kappa(R^T R): near full row rank that
// condition number is huge, and coefficients on R itself (solved through
// the Cholesky factor of R^T R) lose every digit.  When some ratio is
// within a factor 4 of eps (or disagrees with the factorization), one step
// of iterative refinement (the least-squares correction for the residual,
// again through Q and the candidates' factor) removes most of the error
// left in gamma.  If that test disagrees with the pivot, the first
// disagreeing candidate's decision is fixed and the factorization is redone.
#include <algorithm>
#include <vector>

#include "ctd_internal.cuh"

namespace ctd {

namespace {

constexpr double SUSPECT = 1e-4;  // pivot / ||x||^2 below this is re-tested

// Stilde(:, c) = row k_c of the skip-Cholesky storage over kept columns
// before k_c (zero elsewhere), indexed by kept position.
__global__ void k_suspect_rows(const double* __restrict__ S, int64_t lds,
                               const int* __restrict__ kept_idx, int kept,
                               const int* __restrict__ sus, int nsus, double* __restrict__ out) {
  const int64_t total = (int64_t)kept * nsus;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % kept), c = (int)(e / kept);
    const int k = sus[c], j = kept_idx[p];
    out[e] = (j < k) ? S[k + (int64_t)j * lds] : 0.0;
  }
}

__global__ void k_gather_cols(const double* __restrict__ A, int64_t lda, int64_t m,
                              const int* __restrict__ idx, int n, double* __restrict__ out,
                              int64_t ldo) {
  const int64_t total = m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % m, c = e / m;
    out[r + c * ldo] = A[r + (int64_t)idx[c] * lda];
  }
}

// The candidate part of the explicit residuals, r_c = x_k - Xc[:, K] eta_c
// for every suspect c at once: a sparse-times-dense product by rows.  A
// warp takes row i of the candidates' by-row layout, broadcasts the row's
// entries (32 at a time, in column order) and each lane updates suspects
// c = lane, lane + 32, ... (32 NPL per pass) with the kept entries' eta
// rows (etaT, kept x ns row-major), the eta loads of eight entries in flight
// together, so a row is read once for all suspects; the order of operations
// per (i, c) is fixed (reproducible ratios and decisions).  sus_of[cc] = c if candidate cc is suspect c, else
// -1: that entry is x_k's own value.  With init = 0 the products are
// subtracted from the residual already in rbuf (the refinement step).  eta
// is zero for kept candidates after k_c.  The R^(t) part, Q gamma_c, is
// subtracted afterwards by a GEMM.  (A thread per (row, suspect) walked the
// long rows, those of the frequent mode-alpha indices, as chains of
// dependent loads, once per suspect.)
template <int NPL>  // suspects per lane per pass (32 * NPL per pass)
__global__ void __launch_bounds__(256)
    k_resid_rows(int64_t n_rows, const unsigned long long* __restrict__ crp,
                 const int32_t* __restrict__ ccol, const int32_t* __restrict__ cval,
                 const int* __restrict__ kpos, const int* __restrict__ sus_of,
                 const double* __restrict__ etaT, int ns, int init, int seg,
                 double* __restrict__ part, int real) {
  constexpr int CH = 32 * NPL;
  constexpr int EU = 8;  // entries whose eta loads are in flight together
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.y;  // the row's segment: entries [k seg, (k + 1) seg)
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = gw; i < n_rows; i += nw) {
    const unsigned long long a0 = crp[i], b0 = crp[i + 1];
    const unsigned long long a = a0 + (unsigned long long)k * seg;
    if (k > 0 && a >= b0) continue;  // no such segment (segment 0 always writes)
    const unsigned long long b = min(b0, a + (unsigned long long)seg);
    double* out = part + ((int64_t)k * n_rows + i) * ns;
    for (int c0 = 0; c0 < ns; c0 += CH) {
      double acc[NPL];
#pragma unroll
      for (int w = 0; w < NPL; ++w) acc[w] = 0.0;
      for (unsigned long long base = a; base < b; base += 32) {
        const int cnt = (int)min((unsigned long long)32, b - base);
        int q = -1, sc = -1;
        double v = 0.0;
        if (lane < cnt) {
          const int cc = ccol[base + lane];
          v = value_f64(cval[base + lane], real);
          q = kpos[cc];
          sc = sus_of[cc];
        }
        for (int e0 = 0; e0 < cnt; e0 += EU) {
          int qe[EU];
          double ve[EU], ld[EU][NPL];
#pragma unroll
          for (int u = 0; u < EU; ++u) {  // lanes past cnt carry q = -1
            qe[u] = __shfl_sync(0xffffffffu, q, e0 + u);
            ve[u] = __shfl_sync(0xffffffffu, v, e0 + u);
#pragma unroll
            for (int w = 0; w < NPL; ++w) {
              const int c = c0 + lane + 32 * w;
              ld[u][w] = (qe[u] >= 0 && c < ns) ? etaT[(int64_t)qe[u] * ns + c] : 0.0;
            }
          }
#pragma unroll
          for (int u = 0; u < EU; ++u)
#pragma unroll
            for (int w = 0; w < NPL; ++w) acc[w] = fma(-ve[u], ld[u][w], acc[w]);
          if (init) {
            // x_k(i), the suspect's own entry (static indices keep acc in registers)
#pragma unroll
            for (int u = 0; u < EU; ++u) {
              const int se = __shfl_sync(0xffffffffu, sc, e0 + u);
              if (se >= c0 && se < c0 + CH) {
                const int us = (se - c0) >> 5, ls = (se - c0) & 31;
#pragma unroll
                for (int w = 0; w < NPL; ++w) acc[w] += (w == us && lane == ls) ? ve[u] : 0.0;
              }
            }
          }
        }
      }
#pragma unroll
      for (int w = 0; w < NPL; ++w) {
        const int c = c0 + lane + 32 * w;
        if (c < ns) out[c] = acc[w];
      }
    }
  }
}

// rbuf(i, c) (=, or += with init = 0) the sum of row i's segment partials
// in segment order
__global__ void k_resid_combine(int64_t n_rows, const unsigned long long* __restrict__ crp,
                                int ns, int seg, const double* __restrict__ part, int init,
                                double* __restrict__ rbuf) {
  const int64_t total = n_rows * ns;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / ns;
    const int c = (int)(e % ns);
    const unsigned long long len = crp[i + 1] - crp[i];
    const int nseg = len == 0 ? 1 : (int)((len + seg - 1) / seg);
    double s = 0.0;
    for (int k = 0; k < nseg; ++k) s += part[((int64_t)k * n_rows + i) * ns + c];
    double* r = rbuf + (int64_t)c * n_rows + i;
    *r = init ? s : *r + s;
  }
}

// Rows are split into at most RS_SEGS segments of seg entries (a multiple of
// 32, at least 64), a warp per (row, segment): the long rows of the
// frequent mode-alpha indices no longer serialize on one warp (each entry
// costs NPL FP64 instructions of 64 cycles).
constexpr int RS_SEGS = 8;

static ctd_status launch_resid_rows(int64_t n_rows, int du, const uint64_t* crp,
                                    const int32_t* ccol, const int32_t* cval, const int* kpos,
                                    const int* sus_of, const double* etaT, int ns, int init,
                                    double* rbuf, int real, Arena& scratch, cudaStream_t st) {
  // at most RS_SEGS segments, and partials within 256 MB
  const int64_t per = std::max<int64_t>(1, n_rows * ns * (int64_t)sizeof(double));
  const int segs = (int)std::max<int64_t>(1, std::min<int64_t>(RS_SEGS, (256ll << 20) / per));
  int seg = (du + segs - 1) / segs;
  seg = std::max(64, (seg + 31) / 32 * 32);
  double* part;
  CTD_TRY(scratch.get(&part, (size_t)segs * n_rows * ns));
  const dim3 g(grid_for(n_rows * 32, 256, (int64_t)num_sms() * 16), segs);
  const unsigned long long* rp = reinterpret_cast<const unsigned long long*>(crp);
  if (ns <= 32)
    CTD_LAUNCH(k_resid_rows<1>, (g), (256), 0, st, n_rows, rp, ccol, cval, kpos, sus_of, etaT, ns,
               init, seg, part, real);
  else if (ns <= 64)
    CTD_LAUNCH(k_resid_rows<2>, (g), (256), 0, st, n_rows, rp, ccol, cval, kpos, sus_of, etaT, ns,
               init, seg, part, real);
  else
    CTD_LAUNCH(k_resid_rows<4>, (g), (256), 0, st, n_rows, rp, ccol, cval, kpos, sus_of, etaT, ns,
               init, seg, part, real);
  CTD_LAUNCH(k_resid_combine, (grid_for(n_rows * ns, 256, (int64_t)num_sms() * 16)), (256), 0, st,
             n_rows, rp, ns, seg, part, init, rbuf);
  return CTD_OK;
}

// etaT[q * ns + c] = eta[q + c * kept]
__global__ void k_transpose_eta(const double* __restrict__ eta, int kept, int ns,
                                double* __restrict__ etaT) {
  const int64_t total = (int64_t)kept * ns;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(e / ns), c = (int)(e % ns);
    etaT[e] = eta[q + (int64_t)c * kept];
  }
}

// sus_of[sus[c]] = c
__global__ void k_sus_of(const int* __restrict__ sus, int ns, int* __restrict__ sus_of) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ns; c += gridDim.x * blockDim.x)
    sus_of[sus[c]] = c;
}

__global__ void k_kpos(const int* __restrict__ idx, int kept, int* __restrict__ kpos) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < kept; p += gridDim.x * blockDim.x)
    kpos[idx[p]] = p;
}

__global__ void k_resid_norm(int64_t n_rows, const int* __restrict__ sus,
                             const double* __restrict__ xnorm2, const double* __restrict__ rbuf,
                             double* __restrict__ ratio) {
  __shared__ double part[32];
  const int c = blockIdx.x;
  const double* r = rbuf + (int64_t)c * n_rows;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n_rows; i += blockDim.x) acc = fma(r[i], r[i], acc);
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    const double xn = xnorm2[sus[c]];
    ratio[c] = xn > 0.0 ? sqrt(t) / sqrt(xn) : 0.0;
  }
}

// h_K(p, c) = x_{K[p]} . r_c for K[p] < k_c (else 0); a warp per kept
// column, grid (suspect, slice of columns)
__global__ void k_residual_dots(const unsigned long long* __restrict__ cptr,
                                const int32_t* __restrict__ crow, const int32_t* __restrict__ cval,
                                const int* __restrict__ kept_idx, int kept,
                                const int* __restrict__ sus, int64_t n_rows,
                                const double* __restrict__ rbuf, double* __restrict__ hK,
                                int real) {
  const int c = blockIdx.x;
  const int k = sus[c];
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.y * (blockDim.x >> 5);
  const double* r = rbuf + (int64_t)c * n_rows;
  for (int64_t j = gw; j < kept; j += nw) {
    unsigned long long a = 0, b = 0;
    const int col = kept_idx[j];
    if (col < k) {
      a = cptr[col];
      b = cptr[col + 1];
    }
    double s = 0.0;
    for (unsigned long long q = a + lane; q < b; q += 32) s = fma(value_f64(cval[q], real), r[crow[q]], s);
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) hK[j + (int64_t)c * kept] = s;
  }
}

// columns per suspect spread over this many blocks
unsigned slices_for(int64_t ncols, int ns) {
  const int64_t want = std::max<int64_t>(1, (int64_t)num_sms() * 4 / std::max(ns, 1));
  return (unsigned)std::min<int64_t>(want, std::max<int64_t>(1, (ncols + 7) / 8));
}

// zero entries (p, c) whose kept column is not before suspect c
__global__ void k_mask_before(double* __restrict__ A, int kept, const int* __restrict__ kept_idx,
                              const int* __restrict__ sus, int ns) {
  const int64_t total = (int64_t)kept * ns;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e % kept), c = (int)(e / kept);
    if (kept_idx[p] >= sus[c]) A[e] = 0.0;
  }
}

}  // namespace

ctd_status run_filter(const FilterIn& in, FilterOut& out, Arena& scratch, cudaStream_t st) {
  const int du = in.du;
  out.kept = 0;
  if (du <= 0) return CTD_OK;
  double *S0, *thr, *xn2, *piv, *fpiv;
  int* force;
  int*& count = out.count;
  unsigned* status;
  CTD_TRY(scratch.get(&S0, (size_t)du * du));
  CTD_TRY(scratch.get(&thr, du));
  CTD_TRY(scratch.get(&xn2, du));
  CTD_TRY(scratch.get(&piv, du));
  CTD_TRY(scratch.get(&force, du));
  CTD_TRY(scratch.get(&fpiv, du));
  CTD_TRY(scratch.get(&count, 1));
  CTD_TRY(scratch.get(&status, 4));
  CTD_TRY(scratch.get(&out.keep, du));
  CTD_TRY(scratch.get(&out.idx, du));
  CTD_CUDA(cudaMemcpyAsync(S0, in.S, (size_t)du * du * 8, cudaMemcpyDeviceToDevice, st));
  CTD_CUDA(cudaMemcpyAsync(xn2, in.xnorm2, (size_t)du * 8, cudaMemcpyDeviceToDevice, st));
  launch_thresholds(xn2, du, 0, in.eps * in.eps, thr, st);  // ld 0: a plain vector
  CTD_CUDA(cudaMemsetAsync(force, 0xff, (size_t)du * sizeof(int), st));  // -1
  CTD_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
  std::vector<int> h_force(du, -1), h_keep(du);
  std::vector<double> h_piv(du), h_xn(du), h_fpiv(du, 0.0);
  for (int iter = 0; iter <= du + 1; ++iter) {
    if (iter > 0) {
      CTD_CUDA(cudaMemcpyAsync(in.S, S0, (size_t)du * du * 8, cudaMemcpyDeviceToDevice, st));
      CTD_CUDA(cudaMemcpyAsync(force, h_force.data(), (size_t)du * sizeof(int),
                               cudaMemcpyHostToDevice, st));
      CTD_CUDA(cudaMemcpyAsync(fpiv, h_fpiv.data(), (size_t)du * sizeof(double),
                               cudaMemcpyHostToDevice, st));
    }
    {
      PhaseScope ph("filter_chol", st);
      CTD_TRY(launch_chol_skip(in.S, du, du, thr, out.keep, st, force, piv, status,
                               iter > 0 ? fpiv : nullptr));
      launch_compact_flags(out.keep, du, out.idx, count, st);
    }
    unsigned h_status = 0;
    int kept = 0;
    {
      Readback rb(st);
      if (iter == 0) CTD_TRY(rb.add(h_xn.data(), (const double*)xn2, du));
      CTD_TRY(rb.add(&kept, (const int*)count, 1));
      CTD_TRY(rb.add(&h_status, (const unsigned*)status, 1));
      CTD_TRY(rb.add(h_piv.data(), (const double*)piv, du));
      CTD_TRY(rb.add(h_keep.data(), (const int*)out.keep, du));
      CTD_CUDA(cudaGetLastError());
      CTD_TRY(rb.wait());
    }
    if (h_status & DEV_TIMEOUT) return fail(CTD_ETIMEOUT, "skip-Cholesky grid barrier gave up");
    if (h_status & DEV_CAPACITY)
      return fail(CTD_ENOTSUP,
                  "a fiber tested independent by its explicit residual has no positive pivot "
                  "(numerically ambiguous input)");
    out.kept = kept;
    CTD_TRY(scratch.get(&out.Lk, (size_t)std::max(kept, 1) * std::max(kept, 1)));
    CTD_TRY(scratch.get(&out.Li, (size_t)std::max(kept, 1) * std::max(kept, 1)));
    {
      PhaseScope ph("filter_inverse", st);
      launch_gather_lower(in.S, du, out.idx, count, kept, out.Lk, kept, st);
      CTD_TRY(tri_inverse(out.Lk, kept, kept, out.Li, kept, st));
    }
    std::vector<int> sus;
    for (int k = 0; k < du; ++k)
      if (h_xn[k] > 0.0 && h_piv[k] < SUSPECT * h_xn[k]) sus.push_back(k);
    if (sus.empty()) {
      out.keep_h = h_keep;
      out.piv_h = h_piv;
      out.xn_h = h_xn;
      return CTD_OK;
    }
    // explicit residuals of the suspects
    PhaseScope ph("filter_recheck", st);
    const int ns = (int)sus.size();
    const int kk = std::max(kept, 1);
    int* d_sus;
    double *Stil, *eta, *ratio, *rbuf, *gammaQ = nullptr, *WK = nullptr;
    CTD_TRY(scratch.get(&d_sus, ns));
    CTD_TRY(scratch.get(&Stil, (size_t)kk * ns));
    CTD_TRY(scratch.get(&eta, (size_t)kk * ns));
    CTD_TRY(scratch.get(&ratio, ns));
    CTD_TRY(scratch.get(&rbuf, (size_t)in.n_rows * ns));
    CTD_CUDA(cudaMemcpyAsync(d_sus, sus.data(), ns * sizeof(int), cudaMemcpyHostToDevice, st));
    CTD_CUDA(cudaMemsetAsync(eta, 0, (size_t)kk * ns * 8, st));
    if (kept > 0) {
      CTD_LAUNCH(k_suspect_rows, (grid_for((int64_t)kept * ns, 256, 4096)), (256), 0, st, in.S,
                 du, out.idx, kept, d_sus, ns, Stil);
      dgemm(true, false, kept, ns, kept, 1.0, out.Li, kept, Stil, kept, 0.0, eta, kept, st);
    }
    // coefficients on Q: gamma_c = Q^T (x_k - Xc[:, K] eta_c) = W_k - W_K eta_c
    if (in.dt > 0) {
      CTD_TRY(scratch.get(&gammaQ, (size_t)in.dt * ns));
      CTD_LAUNCH(k_gather_cols, (grid_for(in.dt * ns, 256, (int64_t)num_sms() * 8)), (256), 0, st,
                 in.W, in.dt, in.dt, d_sus, ns, gammaQ, in.dt);
      if (kept > 0) {
        CTD_TRY(scratch.get(&WK, (size_t)in.dt * kept));
        CTD_LAUNCH(k_gather_cols, (grid_for(in.dt * kept, 256, (int64_t)num_sms() * 8)), (256), 0,
                   st, in.W, in.dt, in.dt, out.idx, kept, WK, in.dt);
        dgemm(false, false, in.dt, ns, kept, -1.0, WK, in.dt, eta, kept, 1.0, gammaQ, in.dt, st);
      }
    }
    const unsigned ny = slices_for(kept, ns);
    int* kpos;
    CTD_TRY(scratch.get(&kpos, du));
    CTD_CUDA(cudaMemsetAsync(kpos, 0xff, (size_t)du * sizeof(int), st));  // -1
    if (kept > 0)
      CTD_LAUNCH(k_kpos, (grid_for(kept, 256, 64)), (256), 0, st, out.idx, kept, kpos);
    int* sus_of;
    double* etaT;
    CTD_TRY(scratch.get(&sus_of, du));
    CTD_TRY(scratch.get(&etaT, (size_t)kk * ns));
    CTD_CUDA(cudaMemsetAsync(sus_of, 0xff, (size_t)du * sizeof(int), st));  // -1
    CTD_LAUNCH(k_sus_of, (grid_for(ns, 256, 64)), (256), 0, st, d_sus, ns, sus_of);
    const unsigned gt = grid_for((int64_t)kk * ns, 256, (int64_t)num_sms() * 8);
    if (kept > 0) CTD_LAUNCH(k_transpose_eta, (gt), (256), 0, st, eta, kept, ns, etaT);
    CTD_TRY(launch_resid_rows(in.n_rows, du, in.c_rowptr, in.c_col, in.c_val, kpos, sus_of, etaT,
                              ns, 1, rbuf, in.real, scratch, st));
    // minus Q gamma (Q = Qt^T, n_rows x dt)
    if (in.dt > 0)
      dgemm(true, false, in.n_rows, ns, in.dt, -1.0, in.Qt, in.ldq, gammaQ, in.dt, 1.0, rbuf,
            in.n_rows, st);
    CTD_LAUNCH(k_resid_norm, (ns), (256), 0, st, in.n_rows, d_sus, xn2, rbuf, ratio);
    // one step of iterative refinement: the least-squares correction of the
    // residual against [Q, kept before k].  Its change to a ratio is of the
    // order of the rounding left in gamma; it is taken only when some ratio
    // lies within a factor 4 of eps or disagrees with the factorization's
    // decision (otherwise no decision can change).
    std::vector<double> h_ratio(ns);
    CTD_TRY(d2h(h_ratio.data(), ratio, ns, st));
    CTD_CUDA(cudaGetLastError());
    CTD_TRY(sync(st));
    bool refine = false;
    for (int c = 0; c < ns && !refine; ++c) {
      const double r = h_ratio[c];
      const int explicit_keep = r > in.eps ? 1 : 0;
      refine = (r >= 0.25 * in.eps && r <= 4.0 * in.eps) || explicit_keep != h_keep[sus[c]];
    }
    if (refine) {
      double *hQ = nullptr, *hK, *zK, *etad;
      CTD_TRY(scratch.get(&hK, (size_t)kk * ns));
      CTD_TRY(scratch.get(&zK, (size_t)kk * ns));
      CTD_TRY(scratch.get(&etad, (size_t)kk * ns));
      if (kept > 0)
        CTD_LAUNCH(k_residual_dots, (dim3(ns, ny)), (256), 0, st,
                   reinterpret_cast<const unsigned long long*>(in.cptr), in.crow, in.cval, out.idx,
                   kept, d_sus, in.n_rows, rbuf, hK, in.real);
      if (in.dt > 0) {
        // h_Q = Q^T r; the candidates' part of the correction sees the
        // residual projected off Q: h_K - W_K^T h_Q
        CTD_TRY(scratch.get(&hQ, (size_t)in.dt * ns));
        dgemm(false, false, in.dt, ns, in.n_rows, 1.0, in.Qt, in.ldq, rbuf, in.n_rows, 0.0, hQ,
              in.dt, st);
        if (kept > 0)
          dgemm(true, false, kept, ns, in.dt, -1.0, WK, in.dt, hQ, in.dt, 1.0, hK, kept, st);
      }
      CTD_CUDA(cudaMemsetAsync(etad, 0, (size_t)kk * ns * 8, st));
      if (kept > 0) {
        const unsigned gm = grid_for((int64_t)kept * ns, 256, 4096);
        CTD_LAUNCH(k_mask_before, (gm), (256), 0, st, hK, kept, out.idx, d_sus, ns);
        dgemm(false, false, kept, ns, kept, 1.0, out.Li, kept, hK, kept, 0.0, zK, kept, st);
        CTD_LAUNCH(k_mask_before, (gm), (256), 0, st, zK, kept, out.idx, d_sus, ns);
        dgemm(true, false, kept, ns, kept, 1.0, out.Li, kept, zK, kept, 0.0, etad, kept, st);
      }
      // r -= Xc[:, K] eta_d, then r -= Q (h_Q - W_K eta_d)
      if (kept > 0) CTD_LAUNCH(k_transpose_eta, (gt), (256), 0, st, etad, kept, ns, etaT);
      CTD_TRY(launch_resid_rows(in.n_rows, du, in.c_rowptr, in.c_col, in.c_val, kpos, sus_of,
                                etaT, ns, 0, rbuf, in.real, scratch, st));
      if (in.dt > 0) {
        if (kept > 0)
          dgemm(false, false, in.dt, ns, kept, -1.0, WK, in.dt, etad, kept, 1.0, hQ, in.dt, st);
        dgemm(true, false, in.n_rows, ns, in.dt, -1.0, in.Qt, in.ldq, hQ, in.dt, 1.0, rbuf,
              in.n_rows, st);
      }
      CTD_LAUNCH(k_resid_norm, (ns), (256), 0, st, in.n_rows, d_sus, xn2, rbuf, ratio);
      CTD_TRY(d2h(h_ratio.data(), ratio, ns, st));
      CTD_CUDA(cudaGetLastError());
      CTD_TRY(sync(st));
    }
    bool changed = false;
    for (int c = 0; c < ns && !changed; ++c) {
      const int k = sus[c];
      const int explicit_keep = h_ratio[c] > in.eps ? 1 : 0;  // ||res|| = eps ||x||: dependent
      if (explicit_keep != h_keep[k]) {
        h_force[k] = explicit_keep;
        h_fpiv[k] = h_ratio[c] * h_ratio[c] * h_xn[k];
        changed = true;
      }
    }
    if (out.ratios) out.ratios->assign(h_ratio.begin(), h_ratio.end());
    if (!changed) {
      out.keep_h = h_keep;
      out.piv_h = h_piv;
      out.xn_h = h_xn;
      return CTD_OK;
    }
  }
  return fail(CTD_ENOTSUP, "independence filter did not settle");
}

}  // namespace ctd
