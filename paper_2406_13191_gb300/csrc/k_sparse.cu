// FP64 sparse kernels on the LDL^T factor of the reduced Laplacian E^T Omega E.
//
// One CTA per instance; the solution vector lives in shared memory and the
// triangular solves walk the level schedules with one thread per row of a level.
//   k_base_flows : flows of the loads and of the mid-box dispatch,
//                  f0 = H_a (G mid - p_d) (Section 2, constraint (1c)), and for an
//                  outaged line k the rank-1 outage vector u (line outage
//                  distribution factors, f' = f + u f_k).
//   k_certify    : the FP64 dual bound through bus prices nu = lambda + H_a^T eta
//                  (eq. (4) with the closed-form inner minimum of eqs. (6)/(16);
//                  Remarks 1-2 make it a valid bound for mu >= 0).
#include "dev.cuh"
#include "kernels.h"

#include <algorithm>

namespace dcopf {

// The solve of a row at schedule position idx: its kEll packed entries (all loaded in
// one round trip, as they depend on idx only), then its overflow entries, in the same
// order as the row's CSR / CSC walk (unused slots subtract 0 x X[i]).
__device__ __forceinline__ void ell_row(int nr, int idx, int i, const int* __restrict__ ecol,
                                        const double* __restrict__ eval, const int* __restrict__ optr,
                                        const int* __restrict__ ocol, const double* __restrict__ oval,
                                        double* X) {
  constexpr int K = SparseFactor::kEll;
  int c[K];
  double w[K];
#pragma unroll
  for (int a = 0; a < K; ++a) {
    c[a] = ecol[(size_t)a * nr + idx];
    w[a] = eval[(size_t)a * nr + idx];
  }
  const int o0 = optr[idx], o1 = optr[idx + 1];
  double v = X[i];
#pragma unroll
  for (int a = 0; a < K; ++a) v -= w[a] * X[c[a]];
  for (int p = o0; p < o1; ++p) v -= oval[p] * X[ocol[p]];
  X[i] = v;
}

// One triangular sweep over a level schedule with the factor in global memory.  The
// rows near the root of the elimination tree are few per level but long (a separator
// row of the 10000-bus factor has up to ~100 entries), so each level splits its rows'
// entries over groups of G lanes, G the largest power of two up to 32 with one row per
// group covering the level in one pass: a long row's products are then summed by a
// group (each lane its strided share, then a shuffle tree) instead of one after another
// by one thread.  The next level's bounds are loaded a level ahead.
__device__ __forceinline__ void ell_sweep(int nr, int nlev, const int* __restrict__ lev,
                                          const int* __restrict__ rows, const int* __restrict__ ecol,
                                          const double* __restrict__ eval, const int* __restrict__ optr,
                                          const int* __restrict__ ocol, const double* __restrict__ oval,
                                          double* X) {
  if (nlev <= 0) return;
  constexpr int K = SparseFactor::kEll;
  const int tid = (int)threadIdx.x, bd = (int)blockDim.x;
  int s = lev[0], e = lev[1];
  for (int l = 0; l < nlev; ++l) {
    const int e_next = l + 2 <= nlev ? lev[l + 2] : e;
    const int w = e - s;
    int G = 1;
    while (G < 32 && 2 * G * w <= bd) G *= 2;
    const int gid = tid / G, gl = tid % G, ng = bd / G;
    for (int base = s; base < e; base += ng) {  // the same trip count for every lane
      const int idx = base + gid;
      const bool act = idx < e;
      double part = 0.0;
      int i = 0;
      if (act) {
        i = rows[idx];
        const int o0 = optr[idx], o1 = optr[idx + 1];
        for (int a = gl; a < K; a += G) part += eval[(size_t)a * nr + idx] * X[ecol[(size_t)a * nr + idx]];
        for (int p = o0 + gl; p < o1; p += G) part += oval[p] * X[ocol[p]];
      }
      for (int off = G >> 1; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
      if (act && gl == 0) X[i] -= part;
    }
    __syncthreads();
    s = e;
    e = e_next;
  }
}

// PF: the sweeps of ell_sweep; without, one thread per row in the stored order of its
// entries (fewer registers, for the kernels that inline several solves).
template <bool PF>
__device__ void ldl_solve_smem(const DevNet& N, double* X) {
  if (PF) {
    ell_sweep(N.nr, N.n_fwd_lev, N.fwd_lev, N.fwd_rows, N.fell_col, N.fell_val, N.fovf_ptr, N.fovf_col,
              N.fovf_val, X);
  } else {
    for (int lev = 0; lev < N.n_fwd_lev; ++lev) {
      int s = N.fwd_lev[lev], e = N.fwd_lev[lev + 1];
      for (int idx = s + threadIdx.x; idx < e; idx += blockDim.x)
        ell_row(N.nr, idx, N.fwd_rows[idx], N.fell_col, N.fell_val, N.fovf_ptr, N.fovf_col, N.fovf_val, X);
      __syncthreads();
    }
  }
  // with PF the diagonal scaling multiplies by the reciprocal (FP64 division is a long
  // instruction sequence here; the certificate bounds the prices' error from their
  // residual, whatever the solve's rounding)
  if (PF) {
    for (int i = threadIdx.x; i < N.nr; i += blockDim.x) X[i] *= N.inv_diag[i];
  } else {
    for (int i = threadIdx.x; i < N.nr; i += blockDim.x) X[i] /= N.diag[i];
  }
  __syncthreads();
  if (PF) {
    ell_sweep(N.nr, N.n_bwd_lev, N.bwd_lev, N.bwd_rows, N.bell_col, N.bell_val, N.bovf_ptr, N.bovf_col,
              N.bovf_val, X);
  } else {
    for (int lev = 0; lev < N.n_bwd_lev; ++lev) {
      int s = N.bwd_lev[lev], e = N.bwd_lev[lev + 1];
      for (int idx = s + threadIdx.x; idx < e; idx += blockDim.x)
        ell_row(N.nr, idx, N.bwd_rows[idx], N.bell_col, N.bell_val, N.bovf_ptr, N.bovf_col, N.bovf_val, X);
      __syncthreads();
    }
  }
}

// The factor staged in shared memory: FP64 values once in CSR order (the CSC walk
// reads them through cmap), 16-bit row/column indices, 32-bit pointers.
struct PackedFactor {
  const double* diag; const double* val;
  const uint32_t* rptr; const uint32_t* cptr; const uint32_t* cmap;
  const uint16_t* rcol; const uint16_t* crow; const uint16_t* frows; const uint16_t* brows;
  const uint16_t* flev; const uint16_t* blev;
};

// Copies the packed factor into shared memory (16-byte loads) and returns its view.
__device__ PackedFactor stage_factor(const DevNet& N, unsigned char* sm) {
  const int4* src = (const int4*)N.fac_blob;
  int4* dst = (int4*)sm;
  const int n16 = N.fac_bytes / 16;
  for (int base = 0; base < n16; base += 8 * blockDim.x) {  // 8 loads in flight per thread
    int4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = base + u * blockDim.x + threadIdx.x;
      if (q < n16) v[u] = __ldg(src + q);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = base + u * blockDim.x + threadIdx.x;
      if (q < n16) dst[q] = v[u];
    }
  }
  __syncthreads();
  PackedFactor F;
  F.diag = (const double*)(sm + N.off_diag); F.val = (const double*)(sm + N.off_val);
  F.rptr = (const uint32_t*)(sm + N.off_rptr); F.cptr = (const uint32_t*)(sm + N.off_cptr);
  F.cmap = (const uint32_t*)(sm + N.off_cmap);
  F.rcol = (const uint16_t*)(sm + N.off_rcol); F.crow = (const uint16_t*)(sm + N.off_crow);
  F.frows = (const uint16_t*)(sm + N.off_frows); F.brows = (const uint16_t*)(sm + N.off_brows);
  F.flev = (const uint16_t*)(sm + N.off_flev); F.blev = (const uint16_t*)(sm + N.off_blev);
  return F;
}

__device__ void ldl_solve_packed(const DevNet& N, const PackedFactor& F, double* X) {
  for (int lev = 0; lev < N.n_fwd_lev; ++lev) {
    const int s = F.flev[lev], e = F.flev[lev + 1];
    for (int idx = s + threadIdx.x; idx < e; idx += blockDim.x) {
      const int i = F.frows[idx];
      double v = X[i];
      for (uint32_t p = F.rptr[i]; p < F.rptr[i + 1]; ++p) v -= F.val[p] * X[F.rcol[p]];
      X[i] = v;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N.nr; i += blockDim.x) X[i] /= F.diag[i];
  __syncthreads();
  for (int lev = 0; lev < N.n_bwd_lev; ++lev) {
    const int s = F.blev[lev], e = F.blev[lev + 1];
    for (int idx = s + threadIdx.x; idx < e; idx += blockDim.x) {
      const int i = F.brows[idx];
      double v = X[i];
      for (uint32_t p = F.cptr[i]; p < F.cptr[i + 1]; ++p) v -= F.val[F.cmap[p]] * X[F.crow[p]];
      X[i] = v;
    }
    __syncthreads();
  }
}

// Solve with the staged factor when `staged`, else walk the factor in global memory
// (with ell_sweep when PF).
template <bool PF = true>
__device__ __forceinline__ void ldl_solve(const DevNet& N, const PackedFactor* F, double* X) {
  if (F) ldl_solve_packed(N, *F, X);
  else ldl_solve_smem<PF>(N, X);
}

__device__ __forceinline__ double theta_at(const DevNet& N, const double* X, int bus) {
  int p = N.pos_of_bus[bus];
  return p >= 0 ? X[p] : 0.0;
}

__global__ void __launch_bounds__(512, 2) k_base_flows(DevNet N, const double* __restrict__ loads,
                             const int* __restrict__ outage, double* __restrict__ f0,
                             float* __restrict__ f0_32, double* __restrict__ u64,
                             float* __restrict__ u32, double* __restrict__ demand, int* err,
                             int staged, double* __restrict__ wcache) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ double red[32];
  PackedFactor PF;
  const PackedFactor* pf = nullptr;
  if (staged) { PF = stage_factor(N, sm); pf = &PF; }
  double* X = (double*)(sm + (staged ? N.fac_bytes : 0));
  const int b = blockIdx.x;
  const int nl = N.n_line;
  const double* d = loads + (size_t)b * N.n_bus;
  double s = 0.0;
  for (int i = threadIdx.x; i < N.n_bus; i += blockDim.x) s += d[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) demand[b] = s;
  for (int k = threadIdx.x; k < N.nr; k += blockDim.x) X[k] = -d[N.bus_of_pos[k]];
  __syncthreads();
  ldl_solve(N, pf, X);
  double* frow = f0 + (size_t)b * nl;
  for (int l = threadIdx.x; l < nl; l += blockDim.x)
    frow[l] = N.phim[l] + N.line_b[l] * (theta_at(N, X, N.line_from[l]) - theta_at(N, X, N.line_to[l]));
  const int k = outage ? outage[b] : -1;
  __syncthreads();
  if (k >= 0) {
    for (int q = threadIdx.x; q < N.nr; q += blockDim.x) X[q] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
      int pa = N.pos_of_bus[N.line_from[k]], pb = N.pos_of_bus[N.line_to[k]];
      if (pa >= 0) X[pa] += 1.0;
      if (pb >= 0) X[pb] -= 1.0;
    }
    __syncthreads();
    ldl_solve(N, pf, X);
    if (wcache)  // kept for the certificates of this solve
      for (int q = threadIdx.x; q < N.nr; q += blockDim.x) wcache[(size_t)b * N.nr + q] = X[q];
    // PTDF of a transfer from the outaged line's from-bus to its to-bus
    const double ptdf_kk =
        N.line_b[k] * (theta_at(N, X, N.line_from[k]) - theta_at(N, X, N.line_to[k]));
    const double denom = 1.0 - ptdf_kk;
    const bool bridge = fabs(denom) < 1e-9;
    if (bridge && threadIdx.x == 0) atomicExch(err, (int)DCOPF_ERR_NETWORK);
    const double rden = bridge ? 0.0 : 1.0 / denom;
    const double f0k = frow[k];
    __syncthreads();
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      double u = 0.0;
      if (!bridge) {
        double ptdf = N.line_b[l] * (theta_at(N, X, N.line_from[l]) - theta_at(N, X, N.line_to[l]));
        u = (l == k) ? -1.0 : ptdf * rden;
      }
      if (u64) u64[(size_t)b * nl + l] = u;
      if (u32) u32[(size_t)b * nl + l] = (float)u;
      frow[l] += u * f0k;
    }
  } else {
    for (int l = threadIdx.x; l < nl; l += blockDim.x) {
      if (u64) u64[(size_t)b * nl + l] = 0.0;
      if (u32) u32[(size_t)b * nl + l] = 0.0f;
    }
  }
  __syncthreads();
  if (f0_32)
    for (int l = threadIdx.x; l < nl; l += blockDim.x) f0_32[(size_t)b * nl + l] = (float)frow[l];
}

// gamma_m = m u / (1 - m u), u = 2^-53: the classical bound on the relative error
// of m successive FP64 roundings.
__device__ __forceinline__ double gamma_fp64(double m) {
  const double u = 1.1102230246251565e-16;
  return (m * u) / (1.0 - m * u);
}

constexpr int kGamTab = 32;

// S is the storage type of the multipliers (double for the API, float for the FP32
// solver state); `mask` (nullable) selects the instances to certify (mask[b] != 0).
template <typename S>
__global__ void __launch_bounds__(512, 2)
    k_certify(DevNet N, const double* __restrict__ loads, const int* __restrict__ outage,
                          const double* __restrict__ lambda, const S* __restrict__ mu_hi,
                          const S* __restrict__ mu_lo, double* __restrict__ bound,
                          double* __restrict__ errb, const int* __restrict__ mask,
                          const int* __restrict__ done, int staged,
                          const double* __restrict__ wcache) {
  // shared memory: [staged factor] [nr] prices [nr] outage transfer
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ double red[32];
  // gamma of the residual's roundings per bus degree, evaluated once (the same values
  // the residual loop would compute per bus)
  __shared__ double gam_tab[kGamTab];
  const int b = blockIdx.x;
  if (mask && (mask[b] == 0 || (done && done[b]))) return;
  if (threadIdx.x < kGamTab) gam_tab[threadIdx.x] = gamma_fp64(2.0 * threadIdx.x + 6.0);
  PackedFactor PF;
  const PackedFactor* pf = nullptr;
  if (staged) { PF = stage_factor(N, sm); pf = &PF; }
  double* X = (double*)(sm + (staged ? N.fac_bytes : 0));
  const int nl = N.n_line;
  const int k = outage ? outage[b] : -1;
  const S* mh = mu_hi + (size_t)b * nl;
  const S* ml = mu_lo + (size_t)b * nl;
  const double* d = loads + (size_t)b * N.n_bus;
  const double lam = lambda[b];
  // rhs = E_r^T Omega eta with eta = max(mu_hi,0) - max(mu_lo,0), eta_k = 0; a
  // position's first kIncEll incidences load in one round trip, their multipliers in
  // the next (the sums keep the incidence order)
  auto eta_of = [&](int l) { return fmax((double)mh[l], 0.0) - fmax((double)ml[l], 0.0); };
  for (int q = threadIdx.x; q < N.nr; q += blockDim.x) {
    int ln[kIncEll];
    double cf[kIncEll];
#pragma unroll
    for (int a = 0; a < kIncEll; ++a) {
      ln[a] = N.qe_line[(size_t)a * N.nr + q];
      cf[a] = N.qe_coef[(size_t)a * N.nr + q];
    }
    const int o0 = N.qo_ptr[q], o1 = N.qo_ptr[q + 1];
    double et[kIncEll];
#pragma unroll
    for (int a = 0; a < kIncEll; ++a) et[a] = (ln[a] >= 0 && ln[a] != k) ? eta_of(ln[a]) : 0.0;
    double r = 0.0;
#pragma unroll
    for (int a = 0; a < kIncEll; ++a)
      if (ln[a] >= 0 && ln[a] != k) r += cf[a] * et[a];
    for (int p = o0; p < o1; ++p) {
      const int l = N.qo_line[p];
      if (l == k) continue;
      r += N.qo_coef[p] * eta_of(l);
    }
    X[q] = r;
  }
  __syncthreads();
  ldl_solve(N, pf, X);
  // B'^{-1} 1 bound for the post-outage network (Sherman-Morrison on B_r^{-1} 1, its
  // correction doubled as a margin over the rounding of W and denom): wq(q) =
  // winv1[q] + corr |W[q]|
  double corr = 0.0;
  const double* Wv = nullptr;
  if (k >= 0) {
    double* W = X + N.nr;
    Wv = W;
    const int a = N.line_from[k], c = N.line_to[k];
    if (wcache) {  // W = B_r^-1 (e_a - e_c) from the base flows of this solve
      for (int q = threadIdx.x; q < N.nr; q += blockDim.x) W[q] = wcache[(size_t)b * N.nr + q];
      __syncthreads();
    } else {
      for (int q = threadIdx.x; q < N.nr; q += blockDim.x) W[q] = 0.0;
      __syncthreads();
      if (threadIdx.x == 0) {
        int pa = N.pos_of_bus[a], pc = N.pos_of_bus[c];
        if (pa >= 0) W[pa] += 1.0;
        if (pc >= 0) W[pc] -= 1.0;
      }
      __syncthreads();
      ldl_solve(N, pf, W);
    }
    // eta'_k = u^T eta = (z_a - z_c) / (1 - PTDF_kk); z' = z + eta'_k b_k W
    const double denom = 1.0 - N.line_b[k] * (theta_at(N, W, a) - theta_at(N, W, c));
    const double s = (theta_at(N, X, a) - theta_at(N, X, c)) / denom;
    {
      // winv1 carries a 1e-6 relative margin: widen |w_a - w_c| by it
      const double wa = theta_at(N, N.winv1, a), wc = theta_at(N, N.winv1, c);
      corr = 2.0 * N.line_b[k] * (fabs(wa - wc) + 2e-6 * (wa + wc)) / fabs(denom);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < N.nr; q += blockDim.x) X[q] += s * N.line_b[k] * W[q];
    __syncthreads();
  }
  // Residual of the prices in the system they solve (the post-outage Laplacian B' and
  // right-hand side when k >= 0), plus the rounding of its own evaluation:
  // rmax >= |r - B' z^|_inf.  As B'^{-1} >= 0 elementwise, |z - z^| <= rmax B'^{-1} 1.
  double rmax = 0.0;
  for (int q = threadIdx.x; q < N.nr; q += blockDim.x) {
    int ln[kIncEll], op[kIncEll];
    double cf[kIncEll], bl[kIncEll];
#pragma unroll
    for (int a = 0; a < kIncEll; ++a) {
      ln[a] = N.qe_line[(size_t)a * N.nr + q];
      op[a] = N.qe_opos[(size_t)a * N.nr + q];
      cf[a] = N.qe_coef[(size_t)a * N.nr + q];
      bl[a] = N.qe_b[(size_t)a * N.nr + q];
    }
    const int o0 = N.qo_ptr[q], o1 = N.qo_ptr[q + 1];
    const double zi = X[q];
    double r = 0.0, bz = 0.0, acc = 0.0;
    int deg = 0;
    // one incidence: the line, the other end's position, +-b_l and b_l
    auto inc = [&](int l, int o, double c, double bv) {
      const double eta = eta_of(l);
      const double zo = o >= 0 ? X[o] : 0.0;
      r += c * eta;
      bz += bv * (zi - zo);
      acc += fabs(c * eta) + bv * (fabs(zi) + fabs(zo));
      ++deg;
    };
#pragma unroll
    for (int a = 0; a < kIncEll; ++a)
      if (ln[a] >= 0 && ln[a] != k) inc(ln[a], op[a], cf[a], bl[a]);
    for (int p = o0; p < o1; ++p)
      if (N.qo_line[p] != k) inc(N.qo_line[p], N.qo_opos[p], N.qo_coef[p], N.qo_b[p]);
    rmax = fmax(rmax, fabs(r - bz) + (deg < kGamTab ? gam_tab[deg] : gamma_fp64(2.0 * deg + 6.0)) * acc);
  }
  rmax = block_max(rmax, red);
  auto wq = [&](int bus) {
    const int q = N.pos_of_bus[bus];
    return q < 0 ? 0.0 : N.winv1[q] + (Wv ? corr * fabs(Wv[q]) : 0.0);
  };
  // K: how far the terms can move per unit of price error (a generator term is
  // max(|pmin|, |pmax|)-Lipschitz in its bus price, a bus term |d_i|-Lipschitz)
  double g = 0.0, A = 0.0, K = 0.0;
  for (int j = threadIdx.x; j < N.n_gen; j += blockDim.x) {
    double nu = lam + theta_at(N, X, N.gen_bus[j]);
    double p;
    double t = gen_min_value(nu, N.cost_quad[j], N.cost_lin[j], N.S, N.pmin[j], N.pmax[j], &p);
    g += t;
    A += fabs(t);
    K += fmax(fabs(N.pmin[j]), fabs(N.pmax[j])) * wq(N.gen_bus[j]);
  }
  for (int i = threadIdx.x; i < N.n_bus; i += blockDim.x) {
    double t = -(lam + theta_at(N, X, i)) * d[i];
    g += t;
    A += fabs(t);
    K += fabs(d[i]) * wq(i);
  }
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    if (l == k) continue;
    double t = -fmax((double)mh[l], 0.0) * N.fmax[l] + fmax((double)ml[l], 0.0) * N.fmin[l];
    g += t;
    A += fabs(t);
  }
  g = block_sum(g, red);
  A = block_sum(A, red);
  K = block_sum(K, red);
  if (threadIdx.x == 0) {
    int n_terms = N.n_gen + N.n_bus + nl;
    double m = (double)((n_terms + blockDim.x - 1) / blockDim.x) + 6.0 + 8.0;  // per-thread sums,
    // tree depth (<= 5 + 5), and the few roundings inside each term
    // summation bound, plus the prices' error through the terms (K is a rounded sum of
    // non-negative terms: one more gamma of its length)
    double e = gamma_fp64(m) * A + rmax * K * (1.0 + gamma_fp64(m + 4.0));
    bound[b] = g - e;
    if (errb) errb[b] = e;
  }
}

template __global__ void k_certify<double>(DevNet, const double*, const int*, const double*,
                                           const double*, const double*, double*, double*,
                                           const int*, const int*, int, const double*);
template __global__ void k_certify<float>(DevNet, const double*, const int*, const double*,
                                          const float*, const float*, double*, double*, const int*,
                                          const int*, int, const double*);

// Sparse operator form of the iteration: one CTA runs up to n_iters iterations of its
// instance with both operator products as level-scheduled triangular solves on the
// LDL^T factor of the reduced Laplacian, and no Phi~ (FP64 throughout):
//   adjoint  z = B_r^-1 E_r^T Omega eta' (eta'_k = u^T eta for an outaged line k),
//            pi~_j = sigma_j z_bus(j)                              (eq. (6): C^T mu)
//   minimiser x* from w = ctil + sigma lambda + pi~                (eq. (6) / eq. (16))
//   forward  theta = B_r^-1 (G sigma x*), f = Omega E theta + f0 (+ u f_k)  (constraint (1c))
//   value, supergradient, projected step and stop tests exactly as the per-phase path
//   (k_grad_value, k_step, k_close_iter), so the iterates are the same up to rounding.
// A CTA leaves its loop when its instance is done or a stop test fires (the host then
// certifies or stops it); the state stays in the solver's arrays between launches.
__global__ void k_sparse_iters(DevNet N, StepArgs P, SolveState<double> st,
                               const int* __restrict__ outage, const double* __restrict__ f0,
                               const double* __restrict__ u, const double* __restrict__ demand,
                               int n_iters, int max_iters, double tol, int staged) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ double red[32];
  __shared__ double s_pw[3];
  __shared__ int s_stop;
  const int b = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  PackedFactor PF;
  const PackedFactor* pf = nullptr;
  if (staged) { PF = stage_factor(N, sm); pf = &PF; }
  double* X = (double*)(sm + (staged ? N.fac_bytes : 0));  // [nr] solve vector
  double* xg = X + N.nr;                                    // [n_gen] minimiser
  const int nl = N.n_line, ng = N.n_gen;
  const int k = outage ? outage[b] : -1;
  const size_t o = (size_t)b * nl;
  double* mh = st.mu_hi + o;
  double* ml = st.mu_lo + o;
  const double* fr0 = f0 + o;
  const double* ur = u + o;
  const double D = demand[b];
  for (int it = 0; it < n_iters; ++it) {
    if (tid == 0) s_stop = st.done[b] || st.cand[b] != 0;
    __syncthreads();
    if (s_stop) break;
    // adjoint: the outaged line's multiplier is replaced by u^T eta (eta_k = 0)
    double ue = 0.0;
    if (k >= 0) {
      for (int l = tid; l < nl; l += nt)
        if (l != k) ue += ur[l] * (mh[l] - ml[l]);
      ue = block_sum(ue, red);
    }
    for (int q = tid; q < N.nr; q += nt) {
      const int bus = N.bus_of_pos[q];
      double r = 0.0;
      for (int p = N.bus_line_ptr[bus]; p < N.bus_line_ptr[bus + 1]; ++p) {
        const int l = N.bus_line_idx[p];
        r += N.bus_line_coef[p] * (l == k ? ue : mh[l] - ml[l]);
      }
      X[q] = r;
    }
    __syncthreads();
    ldl_solve<false>(N, pf, X);
    // minimiser, generation cost and dispatch
    const double lam = st.lam[b];
    const float kk = (float)(st.iter[b] + 1), wk = kk * kk;  // weight of the mean of minimisers
    double c = 0.0, ps = 0.0;
    for (int j = tid; j < ng; j += nt) {
      const double sg = N.sigma[j];
      const double w = N.ctil[j] + sg * lam + sg * theta_at(N, X, N.gen_bus[j]);
      const double x = inner_x<double>(w, N.mq[j]);
      xg[j] = x;
      c += (N.mq[j] * x + N.ctil[j]) * x + N.cconst[j];
      ps += N.mid[j] + sg * x;
      if (st.xsum) st.xsum[(size_t)b * ng + j] += wk * (float)x;
    }
    c = block_sum(c, red);   // (its barriers also publish xg and retire the reads of X)
    ps = block_sum(ps, red);
    if (tid == 0 && st.wsum) st.wsum[b] += (double)wk;
    // forward: injections sigma_j x_j at the generator buses (fixed order per bus)
    for (int q = tid; q < N.nr; q += nt) {
      const int bus = N.bus_of_pos[q];
      double y = 0.0;
      for (int p = N.bus_gen_ptr[bus]; p < N.bus_gen_ptr[bus + 1]; ++p) {
        const int j = N.bus_gen_idx[p];
        y += N.sigma[j] * xg[j];
      }
      X[q] = y;
    }
    __syncthreads();
    ldl_solve<false>(N, pf, X);
    auto flow = [&](int l) {  // Phi~ x on line l (pre-outage)
      return N.line_b[l] * (theta_at(N, X, N.line_from[l]) - theta_at(N, X, N.line_to[l]));
    };
    const double fk = k >= 0 ? flow(k) + fr0[k] : 0.0;
    // value (k_grad_value)
    double acc = 0.0;
    for (int l = tid; l < nl; l += nt) {
      if (l == k) continue;
      const double f = flow(l) + fr0[l] + (k >= 0 ? ur[l] * fk : 0.0);
      acc += mh[l] * (f - N.fmax[l]) + ml[l] * (N.fmin[l] - f);
    }
    acc = block_sum(acc, red);
    const double gl = ps - D;
    const double value = c + lam * gl + acc;
    // projected step (k_step): best point first, then mu and lambda
    const int t = st.iter[b] + 1;
    if (tid == 0) {
      s_pw[0] = pow(P.decay, (double)(t - 1));
      s_pw[1] = 1.0 - pow(P.beta1, (double)t);
      s_pw[2] = 1.0 - pow(P.beta2, (double)t);
      s_stop = value > st.best[b];  // reused: whether this point improves the best
    }
    __syncthreads();
    StepArgs Q = P;
    Q.bc1 = s_pw[1];
    Q.bc2 = s_pw[2];
    const double scale = s_pw[0];
    const bool better = s_stop != 0;
    const double am = P.alpha * scale;
    for (int l = tid; l < nl; l += nt) {
      const double h = mh[l], lo = ml[l];
      if (better) {
        st.best_hi[o + l] = h;
        st.best_lo[o + l] = lo;
      }
      double gh = 0.0, gll = 0.0;
      if (l != k) {
        const double f = flow(l) + fr0[l] + (k >= 0 ? ur[l] * fk : 0.0);
        gh = f - N.fmax[l];
        gll = N.fmin[l] - f;
      }
      const double h2 = rule_step<double>(Q, h, gh, st.s1_hi[o + l], st.s2_hi[o + l], am);
      const double l2 = rule_step<double>(Q, lo, gll, st.s1_lo[o + l], st.s2_lo[o + l], am);
      mh[l] = h2 > 0.0 ? h2 : 0.0;
      ml[l] = l2 > 0.0 ? l2 : 0.0;
    }
    if (tid == 0) {
      // lambda, best value and stop tests (k_step, k_close_iter)
      double lm = lam;
      if (better) {
        st.best[b] = value;
        st.best_lam[b] = lam;
        st.best_iter[b] = t;
      }
      double s1 = st.lam_s1[b], s2 = st.lam_s2[b];
      lm = rule_step<double>(Q, lm, gl, s1, s2, P.alpha_lambda * scale);
      st.lam[b] = lm;
      st.lam_s1[b] = s1;
      st.lam_s2[b] = s2;
      st.prev[b] = value;
      st.iter[b] = t;
      if (st.has_target && st.best[b] >= st.thresh[b] + st.margin[b]) st.cand[b] = 1;
      if (t >= max_iters) st.cand[b] = 2;
      if (tol > 0.0 && t > 1 && fabs(value - st.prev2[b]) < tol) st.cand[b] = 2;
      st.prev2[b] = value;
    }
    __syncthreads();  // the next loop reads mu, lambda and the flags
  }
}

// Shared memory of a sparse kernel with n_vec solution vectors; *staged tells whether
// the packed factor fits beside them.
static size_t sparse_smem(const dcopf_dual* h, int n_vec, int* staged) {
  size_t vec = (size_t)n_vec * (size_t)std::max(1, h->dev.nr) * sizeof(double);
  if (h->dev.fac_blob && (size_t)h->dev.fac_bytes + vec + 1024 <= h->smem_optin) {
    *staged = 1;
    return (size_t)h->dev.fac_bytes + vec;
  }
  *staged = 0;
  return vec;
}

size_t certify_smem(const dcopf_dual* h, bool outages) {
  int st = 0;
  return sparse_smem(h, outages ? 2 : 1, &st);
}

static int sparse_threads(const dcopf_dual* h) {
  // one thread per row of the widest level, rounded to warps, 128..512
  int w = 128;
  while (w < 512 && w < h->host.F.n / 8) w *= 2;
  return w;
}

dcopf_status run_iters_sparse(dcopf_dual* h, int B, const int* outage, const StepArgs& P,
                              SolveState<double>& st, int n_iters, int max_iters, double tol,
                              cudaStream_t s) {
  // [nr] solve vector plus [n_gen] minimiser, counted as whole vectors of nr doubles
  const int nvec = 1 + (h->dev.n_gen + h->dev.nr - 1) / std::max(1, h->dev.nr);
  int staged = 0;
  size_t smem = sparse_smem(h, nvec, &staged);
  if (smem > h->smem_optin) return DCOPF_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_sparse_iters, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DCOPF_ERR_CUDA;
  Workspace& w = h->ws;
  k_sparse_iters<<<B, sparse_threads(h), smem, s>>>(h->dev, P, st, outage, w.f0.as<double>(),
                                                     w.u64.as<double>(), w.demand.as<double>(),
                                                     n_iters, max_iters, tol, staged);
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

dcopf_status run_base_flows(dcopf_dual* h, int B, const double* loads, const int* outage,
                            cudaStream_t s) {
  if (dense_path_applies(h, B, outage)) return run_dense_base_flows(h, B, loads, s);
  int staged = 0;
  size_t smem = sparse_smem(h, 1, &staged);
  if (smem > h->smem_optin) return DCOPF_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_base_flows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DCOPF_ERR_CUDA;
  Workspace& w = h->ws;
  double* wc = nullptr;
  w.wcache_B = 0;
  w.wcache_outage = nullptr;
  if (outage) {
    if (w.wcache.alloc((size_t)B * h->dev.nr * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return DCOPF_ERR_OOM;
    }
    wc = w.wcache.as<double>();
  }
  k_base_flows<<<B, sparse_threads(h), smem, s>>>(h->dev, loads, outage, w.f0.as<double>(),
                                                  w.f0_32.as<float>(), w.u64.as<double>(),
                                                  w.u32.as<float>(), w.demand.as<double>(), h->d_err,
                                                  staged, wc);
  if (wc) {
    w.wcache_B = B;
    w.wcache_outage = outage;
  }
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

template <typename S>
dcopf_status run_certify_t(dcopf_dual* h, int B, const double* loads, const int* outage,
                           const double* lam, const S* mh, const S* ml, double* bound, double* errb,
                           const int* mask, const int* done, cudaStream_t s, bool use_wcache) {
  if (dense_path_applies(h, B, outage))
    return run_dense_certify<S>(h, B, loads, lam, mh, ml, bound, errb, mask, done, s);
  int staged = 0;
  size_t smem = sparse_smem(h, outage != nullptr ? 2 : 1, &staged);
  if (smem > h->smem_optin) return DCOPF_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_certify<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DCOPF_ERR_CUDA;
  const Workspace& w = h->ws;
  const double* wc = use_wcache && outage && w.wcache_B == B && w.wcache_outage == outage
                         ? w.wcache.as<double>()
                         : nullptr;
  k_certify<S><<<B, sparse_threads(h), smem, s>>>(h->dev, loads, outage, lam, mh, ml, bound, errb,
                                                  mask, done, staged, wc);
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}
template dcopf_status run_certify_t<double>(dcopf_dual*, int, const double*, const int*,
                                            const double*, const double*, const double*, double*,
                                            double*, const int*, const int*, cudaStream_t, bool);
template dcopf_status run_certify_t<float>(dcopf_dual*, int, const double*, const int*,
                                           const double*, const float*, const float*, double*,
                                           double*, const int*, const int*, cudaStream_t, bool);

// Base flows into caller-provided buffers (f0 and u64 [batch][n_line], demand [batch]);
// the same kernel as run_base_flows without touching the handle's workspace.
dcopf_status launch_base_flows_into(dcopf_dual* h, int B, const double* loads, const int* outage,
                                    double* f0, double* u64, double* demand, cudaStream_t s) {
  int staged = 0;
  size_t smem = sparse_smem(h, 1, &staged);
  if (smem > h->smem_optin) return DCOPF_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_base_flows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DCOPF_ERR_CUDA;
  k_base_flows<<<B, sparse_threads(h), smem, s>>>(h->dev, loads, outage, f0, nullptr, u64, nullptr,
                                                  demand, h->d_err, staged, nullptr);
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

}  // namespace dcopf
