// Constraint screening for the batched solves: Algorithm 1 writes the flow rows it
// iterates on as C_r, d_r, a subset of all 2 n_line rows.  A line whose flow stays
// strictly inside its limits for every dispatch of the generator box that meets the
// balance, at the loads of every instance of the batch, can never bind: dropping it
// leaves the primal optimum unchanged, and fixing its multipliers at zero keeps every
// dual point a valid bound (Remarks 1 and 2).  The certificate always evaluates the
// full problem, so a screen never affects the validity of a bound, only which rows the
// iterations carry.
//
// In the normalised variables (Appendix A1) the flow of line l is Phi~_l x + f0_l with
// x in [-1, 1]^n_gen and sigma^T x = R_b = D_b - sum_j mid_j.  For every t,
//   max { Phi~_l x : |x| <= 1, sigma^T x = R, R in [R_lo, R_hi] }
//     <= psi_l(t) = max(t R_lo, t R_hi) + sum_j |Phi~_lj - t sigma_j|
// (weak duality of the fractional knapsack for each R, then the max over R of a min
// over t is at most the min over t of the max).  psi_l is convex in t; a bisection on
// the sign of its subgradient in FP32 finds a good t, and psi_l(t) evaluated in FP64 is
// the bound, whatever the accuracy of the search.  The same with -Phi~_l bounds the
// flow from below.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "dev.cuh"
#include "kernels.h"

namespace dcopf {

namespace {

// Extremes over the batch of each line's base flow f0 and of the balance R.
__global__ void k_screen_envelope(int B, int nl, const double* __restrict__ f0,
                                  const double* __restrict__ demand, double sum_mid,
                                  double* __restrict__ lo, double* __restrict__ hi, double* __restrict__ r) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
    double a = INFINITY, z = -INFINITY;
    for (int b = 0; b < B; ++b) {
      const double v = f0[(size_t)b * nl + l];
      a = fmin(a, v);
      z = fmax(z, v);
    }
    lo[l] = a;
    hi[l] = z;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double a = INFINITY, z = -INFINITY;
    for (int b = 0; b < B; ++b) {
      a = fmin(a, demand[b] - sum_mid);
      z = fmax(z, demand[b] - sum_mid);
    }
    r[0] = a;
    r[1] = z;
  }
}

// Whether the knapsack bounds must be taken again: they hold for any balance range
// inside the one they were taken on (rng[0..1], valid when rng[2] != 0).  If the batch's
// range r[0..1] leaves it, the new range is the batch's widened a little (so that nearby
// batches reuse the bounds) and *redo = 1.  One thread.
__global__ void k_screen_range(const double* __restrict__ r, double* __restrict__ rng, int* __restrict__ redo) {
  if (rng[2] != 0.0 && r[0] >= rng[0] && r[1] <= rng[1]) {
    *redo = 0;
    return;
  }
  const double w = 0.02 * (fabs(r[0]) + fabs(r[1])) + 1e-9;
  rng[0] = r[0] - w;
  rng[1] = r[1] + w;
  rng[2] = 1.0;
  *redo = 1;
}

// One warp per line: the knapsack bounds up_l >= max Phi~_l x and dn_l >= max -Phi~_l x
// over the box and every balance R in [rng[0], rng[1]] (when *redo; else the bounds
// already in up / dn hold).
__global__ void __launch_bounds__(256) k_screen_knapsack(DevNet N, const double* __restrict__ rng,
                                                         const int* __restrict__ redo,
                                                         double* __restrict__ up, double* __restrict__ dn) {
  const int l = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (l >= N.n_line || !*redo) return;  // whole warps
  const double rlo = rng[0], rhi = rng[1];
  const int ng = N.n_gen;
  const float* p32 = N.phi32 + (size_t)l * ng;
  const double* p64 = N.phi64 + (size_t)l * ng;
  const float rlof = (float)rlo, rhif = (float)rhi;
  for (int dir = 0; dir < 2; ++dir) {
    const float sg = dir == 0 ? 1.f : -1.f;
    float rmin = INFINITY, rmax = -INFINITY;
    for (int j = lane; j < ng; j += 32) {
      const float s = N.sigma32[j];
      if (s > 0.f) {
        const float q = sg * p32[j] / s;
        rmin = fminf(rmin, q);
        rmax = fmaxf(rmax, q);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
      rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    float a = rmin < INFINITY ? rmin : 0.f, b = rmax > -INFINITY ? rmax : 0.f;
    // the subgradient (t > 0 ? R_hi : R_lo) - sum_j sigma_j sgn(Phi~_lj - t sigma_j) is
    // non-decreasing in t: bisection on its sign change
    for (int it = 0; it < 24; ++it) {
      const float t = 0.5f * (a + b);
      float g = 0.f;
      for (int j = lane; j < ng; j += 32) {
        const float s = N.sigma32[j], d = sg * p32[j] - t * s;
        g += d > 0.f ? s : (d < 0.f ? -s : 0.f);
      }
      g = warp_sum(g);
      const float sub = (t > 0.f ? rhif : rlof) - g;
      if (sub < 0.f) a = t;
      else b = t;
    }
    const double t = 0.5 * ((double)a + (double)b);
    double psi = 0.0;
    for (int j = lane; j < ng; j += 32) psi += fabs((double)sg * p64[j] - t * N.sigma[j]);
    psi = warp_sum(psi) + fmax(t * rlo, t * rhi);
    if (lane == 0) (dir == 0 ? up : dn)[l] = psi;
  }
}

// keep[l] = 0 when line l's flow provably stays inside its limits for the batch: its
// knapsack bounds plus the batch's extremes of its base flow, with a rounding margin.
__global__ void k_screen_decide(DevNet N, const double* __restrict__ up, const double* __restrict__ dn,
                                const double* __restrict__ lo, const double* __restrict__ hi,
                                unsigned char* __restrict__ keep) {
  const int nl = N.n_line, ng = N.n_gen;
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x) {
    const double fup = up[l] + hi[l], fdn = -dn[l] + lo[l];
    // psi is a sum of n_gen + 1 FP64 terms (each within a few units in the last place) and
    // the flow adds one more: 8 (n_gen + 2) units of 2^-53 of the magnitudes involved
    const double mag = fabs(up[l]) + fabs(dn[l]) + fabs(lo[l]) + fabs(hi[l]) + fabs(N.fmax[l]) + fabs(N.fmin[l]);
    const double margin = 8.0 * (ng + 2) * 1.1102230246251565e-16 * mag + 1e-12;
    keep[l] = (fup <= N.fmax[l] - margin && fdn >= N.fmin[l] + margin) ? 0 : 1;
  }
}

// *flag = 1 if a line that this batch must keep (keep[l]) is not in the kept set of the
// compact operands (pos[l] < 0): the solve that went ahead with them screens again.
__global__ void k_screen_cover(int nl, const unsigned char* __restrict__ keep, const int* __restrict__ pos,
                               int* __restrict__ flag) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += gridDim.x * blockDim.x)
    if (keep[l] && pos[l] < 0) *flag = 1;
}

// The products' B operands of the kept lines, from the network's (both in the blocked
// layout of blk_index, zero outside the matrix): rows of Phi~ (nk of n_line, K = ng)
// and columns of Phi~^T (ng rows, K = nk of n_line).
__device__ __forceinline__ void blk_coords(size_t q, int kb, int* r, int* c) {
  const size_t per = (size_t)kb * 512;
  const size_t rb = q / per;
  const int rem = (int)(q - rb * per);
  *r = (int)rb * 8 + ((rem >> 6) & 7);
  *c = (rem >> 9) * 64 + (rem & 63);
}
__global__ void k_screen_gather_rows_blk(int nk, int ng, int kb, const int* __restrict__ kept,
                                         const __nv_bfloat16* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  const size_t n = (size_t)((nk + 7) / 8) * kb * 512;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    int r, c;
    blk_coords(q, kb, &r, &c);
    dst[q] = (r < nk && c < ng) ? src[blk_index(kept[r], c, kb)] : z;
  }
}
__global__ void k_screen_gather_cols_blk(int rows, int nk, int kb_src, int kb, const int* __restrict__ kept,
                                         const __nv_bfloat16* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
  const size_t n = (size_t)((rows + 7) / 8) * kb * 512;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    int r, c;
    blk_coords(q, kb, &r, &c);
    dst[q] = (r < rows && c < nk) ? src[blk_index(r, kept[c], kb_src)] : z;
  }
}
__global__ void k_screen_gather_lines(int nk, const int* __restrict__ kept, const float* __restrict__ a,
                                      const float* __restrict__ b, float* __restrict__ ca, float* __restrict__ cb) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nk; r += gridDim.x * blockDim.x) {
    ca[r] = a[kept[r]];
    cb[r] = b[kept[r]];
  }
}

}  // namespace

// Per batch [B][n_line] FP32 rows -> [B][nk] compact rows (the base flows of the kept lines).
__global__ void k_screen_compact_rows(int B, int nl, int nk, const int* __restrict__ kept,
                                      const float* __restrict__ src, float* __restrict__ dst) {
  const size_t n = (size_t)B * nk;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const size_t b = q / nk, r = q - b * nk;
    dst[q] = src[b * nl + kept[r]];
  }
}

dcopf_status screen_batch(dcopf_dual* h, int B, cudaStream_t s) {
  LineScreen& S = h->scr;
  const int nl = h->host.n_line, ng = h->host.n_gen;
  const bool fresh = S.rng.p == nullptr;
  if (S.env.alloc((size_t)(2 * nl + 2) * sizeof(double)) != cudaSuccess ||
      S.knap.alloc((size_t)2 * nl * sizeof(double)) != cudaSuccess ||
      S.keep.alloc((size_t)nl) != cudaSuccess || S.rng.alloc(4 * sizeof(double)) != cudaSuccess ||
      S.flags.alloc(4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return DCOPF_ERR_OOM;
  }
  if (fresh && cudaMemsetAsync(S.rng.p, 0, 4 * sizeof(double), s) != cudaSuccess) return DCOPF_ERR_CUDA;
  double* lo = S.env.as<double>();
  double* hi = lo + nl;
  double* r = hi + nl;
  double sum_mid = 0.0;
  for (int j = 0; j < ng; ++j) sum_mid += h->host.mid[j];
  const unsigned grid = (unsigned)std::min(1024, (nl + 255) / 256);
  k_screen_envelope<<<grid, 256, 0, s>>>(B, nl, h->ws.f0.as<double>(), h->ws.demand.as<double>(), sum_mid,
                                         lo, hi, r);
  double* up = S.knap.as<double>();
  double* dn = up + nl;
  double* rng = S.rng.as<double>();
  int* redo = S.flags.as<int>();
  k_screen_range<<<1, 1, 0, s>>>(r, rng, redo);
  k_screen_knapsack<<<(unsigned)((nl + 7) / 8), 256, 0, s>>>(h->dev, rng, redo, up, dn);
  k_screen_decide<<<grid, 256, 0, s>>>(h->dev, up, dn, lo, hi, S.keep.as<unsigned char>());
  h->launches += 4;
  if (S.ready && !S.exact) {
    // go ahead with the kept set of the compact operands, and let the solve find out
    // (device error word [1]) whether this batch needs a line outside it
    k_screen_cover<<<grid, 256, 0, s>>>(nl, S.keep.as<unsigned char>(), S.pos.as<int>(), h->d_err + 1);
    h->launches += 1;
    return cudaGetLastError() == cudaSuccess ? DCOPF_OK : DCOPF_ERR_CUDA;
  }
  std::vector<unsigned char> keep(nl);
  if (cudaMemcpyAsync(keep.data(), S.keep.p, nl, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  std::vector<int> kept;
  for (int l = 0; l < nl; ++l)
    if (keep[l]) kept.push_back(l);
  // a multiple of 8 rows (16-byte row strides for TMA, four-line vector steps): the
  // first screened lines are kept as well, which only adds rows that cannot bind
  for (int l = 0; l < nl && (kept.size() % 8 != 0 || kept.empty()); ++l)
    if (!keep[l]) { keep[l] = 1; kept.push_back(l); }
  std::sort(kept.begin(), kept.end());
  if (S.ready && kept == S.kept_host) return DCOPF_OK;
  // the compact operands of this set of lines
  const int nk = (int)kept.size();
  TensorOps& T = h->tops;
  const int ld_lk = (nk + 7) & ~7;
  std::vector<int> pos(nl, -1);
  for (int q = 0; q < nk; ++q) pos[kept[q]] = q;
  S.ready = false;
  // the products' B operands in 8-row blocks of whole 64-column K blocks
  const int kb_g = (ng + 63) / 64, kb_l = (nk + 63) / 64;
  const size_t phi_bytes = (size_t)((nk + 7) / 8) * kb_g * 512 * 2;
  const size_t phit_bytes = (size_t)((ng + 7) / 8) * kb_l * 512 * 2;
  if (S.kept.alloc((size_t)nk * sizeof(int)) != cudaSuccess || S.pos.alloc((size_t)nl * sizeof(int)) != cudaSuccess ||
      S.phi_hi.alloc(phi_bytes) || S.phi_lo.alloc(phi_bytes) || S.phit_hi.alloc(phit_bytes) ||
      S.phit_lo.alloc(phit_bytes) ||
      S.lim.alloc((size_t)2 * nk * sizeof(float))) {
    cudaGetLastError();
    return DCOPF_ERR_OOM;
  }
  if (cudaMemcpyAsync(S.kept.p, kept.data(), (size_t)nk * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(S.pos.p, pos.data(), (size_t)nl * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  const int* kd = S.kept.as<int>();
  const int kb_n = (nl + 63) / 64;  // K blocks of the network's Phi~^T
  k_screen_gather_rows_blk<<<1024, 256, 0, s>>>(nk, ng, kb_g, kd, T.phi_hi.as<__nv_bfloat16>(),
                                                S.phi_hi.as<__nv_bfloat16>());
  k_screen_gather_rows_blk<<<1024, 256, 0, s>>>(nk, ng, kb_g, kd, T.phi_lo.as<__nv_bfloat16>(),
                                                S.phi_lo.as<__nv_bfloat16>());
  k_screen_gather_cols_blk<<<1024, 256, 0, s>>>(ng, nk, kb_n, kb_l, kd, T.phit_hi.as<__nv_bfloat16>(),
                                                S.phit_hi.as<__nv_bfloat16>());
  k_screen_gather_cols_blk<<<1024, 256, 0, s>>>(ng, nk, kb_n, kb_l, kd, T.phit_lo.as<__nv_bfloat16>(),
                                                S.phit_lo.as<__nv_bfloat16>());
  float* lim = S.lim.as<float>();
  k_screen_gather_lines<<<(nk + 255) / 256, 256, 0, s>>>(nk, kd, h->dev.fmax32, h->dev.fmin32, lim, lim + nk);
  h->launches += 5;
  if (cudaGetLastError() != cudaSuccess) return DCOPF_ERR_CUDA;
  bool mok = true;
  for (const uint32_t br : {128u, 96u, 80u, 72u}) {
    CUtensorMap* fh = br == 128 ? &S.m_phi_hi : br == 96 ? &S.m_phi_hi96 : br == 80 ? &S.m_phi_hi80 : &S.m_phi_hi72;
    CUtensorMap* fl = br == 128 ? &S.m_phi_lo : br == 96 ? &S.m_phi_lo96 : br == 80 ? &S.m_phi_lo80 : &S.m_phi_lo72;
    CUtensorMap* ah = br == 128 ? &S.m_phit_hi : br == 96 ? &S.m_phit_hi96 : br == 80 ? &S.m_phit_hi80 : &S.m_phit_hi72;
    CUtensorMap* al = br == 128 ? &S.m_phit_lo : br == 96 ? &S.m_phit_lo96 : br == 80 ? &S.m_phit_lo80 : &S.m_phit_lo72;
    mok = mok && tc_make_map_blocked(fh, S.phi_hi.p, nk, ng, br) && tc_make_map_blocked(fl, S.phi_lo.p, nk, ng, br) &&
          tc_make_map_blocked(ah, S.phit_hi.p, ng, nk, br) && tc_make_map_blocked(al, S.phit_lo.p, ng, nk, br);
  }
  if (!mok)
    return DCOPF_ERR_CUDA;
  S.nk = nk;
  S.ld_lk = ld_lk;
  S.kept_host = kept;
  S.ready = true;
  S.exact = false;
  S.map_B = 0;  // the per-batch A operand maps are made for the next batch size
  return DCOPF_OK;
}

}  // namespace dcopf
