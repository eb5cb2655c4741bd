// Base flows and the FP64 certificate through the dense PTDF H_a (all buses), for
// small batches without line outages.
//
// The sparse path (k_sparse.cu) walks the elimination levels of the LDL^T factor one
// after another; for one instance that chain of dependent FP64 steps costs a few
// hundred microseconds.  For a handful of instances it is cheaper to stream the FP64
// matrix H_a = Omega E (E^T Omega E)^{-1} (zero slack column; Section 2 below
// problem (1)) once per product:
//   f0 = Phi mid - H_a p_d                       (flows of the mid-box dispatch)
//   z  = H_a^T eta                               (bus prices of the line multipliers)
// and the certified bound (eq. (4) through the bus prices, as in k_certify).  H_a is
// built on first use from the same FP64 factor as Phi, so both paths evaluate the
// same problem data.
#include <algorithm>
#include <thread>
#include <vector>

#include "dev.cuh"
#include "kernels.h"

namespace dcopf {

constexpr int DN_TILE = 128;    // buses per column tile of the H_a^T eta product
constexpr int DN_SPLITS = 16;   // row splits of that product

// f0[b][i] = phim[i] - H_a[i,:] . d_b, demand[b] = sum d_b; a warp per (line, instance).
__global__ void k_dense_base_flows(int nb, int nl, const double* __restrict__ H,
                                   const double* __restrict__ phim, const double* __restrict__ loads,
                                   double* __restrict__ f0, float* __restrict__ f0_32,
                                   double* __restrict__ u64, float* __restrict__ u32,
                                   double* __restrict__ demand) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.y;
  const double* d = loads + (size_t)b * nb;
  if (warp == 0) {
    double s = 0.0;
    for (int j = lane; j < nb; j += 32) s += d[j];
    s = warp_sum(s);
    if (lane == 0) demand[b] = s;
  }
  if (warp >= nl) return;
  const double* row = H + (size_t)warp * nb;
  double s = 0.0;
  for (int j = lane; j < nb; j += 32) s = fma(row[j], d[j], s);
  s = warp_sum(s);
  if (lane == 0) {
    const size_t o = (size_t)b * nl + warp;
    const double v = phim[warp] - s;
    f0[o] = v;
    if (f0_32) f0_32[o] = (float)v;
    if (u64) u64[o] = 0.0;
    if (u32) u32[o] = 0.f;
  }
}

// Partial bus prices: part[b][split][j] = sum over the split's lines of H_a[i][j] eta_i,
// eta = max(mu_hi, 0) - max(mu_lo, 0), formed once per block in shared memory.
// Block = (column tile, row split, instance).
template <typename S>
__global__ void k_dense_prices(int nb, int nl, const double* __restrict__ H,
                               const S* __restrict__ mu_hi, const S* __restrict__ mu_lo,
                               double* __restrict__ part, const int* __restrict__ mask,
                               const int* __restrict__ done) {
  extern __shared__ double eta_s[];
  const int b = blockIdx.z;
  if (mask && (mask[b] == 0 || (done && done[b]))) return;
  const int j = blockIdx.x * DN_TILE + threadIdx.x;
  const int rows = (nl + DN_SPLITS - 1) / DN_SPLITS;
  const int i0 = blockIdx.y * rows, i1 = min(nl, i0 + rows);
  const S* mh = mu_hi + (size_t)b * nl;
  const S* ml = mu_lo + (size_t)b * nl;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x)
    eta_s[i - i0] = fmax((double)mh[i], 0.0) - fmax((double)ml[i], 0.0);
  __syncthreads();
  if (j >= nb) return;
  double s0 = 0.0, s1 = 0.0;
  int i = i0;
  for (; i + 8 <= i1; i += 8) {  // eight rows in flight, two chains
    double h[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) h[u] = H[(size_t)(i + u) * nb + j];
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      s0 = fma(h[u], eta_s[i + u - i0], s0);
      s1 = fma(h[u + 1], eta_s[i + u + 1 - i0], s1);
    }
  }
  for (; i < i1; ++i) s0 = fma(H[(size_t)i * nb + j], eta_s[i - i0], s0);
  part[((size_t)b * DN_SPLITS + blockIdx.y) * nb + j] = s0 + s1;
}

__device__ __forceinline__ double gamma_fp64_d(double m) {
  const double u = 1.1102230246251565e-16;
  return (m * u) / (1.0 - m * u);
}

// Certified bound from the bus prices: the same sum as k_certify (eq. (4) through nu).
template <typename S>
__global__ void k_dense_certify(DevNet N, const double* __restrict__ part,
                                const double* __restrict__ loads, const double* __restrict__ lambda,
                                const S* __restrict__ mu_hi, const S* __restrict__ mu_lo,
                                double* __restrict__ bound, double* __restrict__ errb,
                                const int* __restrict__ mask, const int* __restrict__ done) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  if (mask && (mask[b] == 0 || (done && done[b]))) return;
  const int nb = N.n_bus, nl = N.n_line;
  const double* pz = part + (size_t)b * DN_SPLITS * nb;
  const double* d = loads + (size_t)b * nb;
  const S* mh = mu_hi + (size_t)b * nl;
  const S* ml = mu_lo + (size_t)b * nl;
  const double lam = lambda[b];
  extern __shared__ double zs[];  // bus prices z = H_a^T eta, reduced once
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    double z = 0.0;
    for (int q0 = 0; q0 < DN_SPLITS; q0 += 8) {  // eight partials in flight
      double p[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) p[u] = pz[(size_t)(q0 + u) * nb + j];
#pragma unroll
      for (int u = 0; u < 8; ++u) z += p[u];
    }
    zs[j] = z;
  }
  __syncthreads();
  auto z_at = [&](int j) { return zs[j]; };
  double g = 0.0, A = 0.0;
  for (int j = threadIdx.x; j < N.n_gen; j += blockDim.x) {
    double p;
    const double t = gen_min_value(lam + z_at(N.gen_bus[j]), N.cost_quad[j], N.cost_lin[j], N.S,
                                   N.pmin[j], N.pmax[j], &p);
    g += t;
    A += fabs(t);
  }
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const double t = -(lam + z_at(i)) * d[i];
    g += t;
    A += fabs(t);
  }
  for (int l = threadIdx.x; l < nl; l += blockDim.x) {
    const double t = -fmax((double)mh[l], 0.0) * N.fmax[l] + fmax((double)ml[l], 0.0) * N.fmin[l];
    g += t;
    A += fabs(t);
  }
  g = block_sum(g, red);
  A = block_sum(A, red);
  if (threadIdx.x == 0) {
    const int n_terms = N.n_gen + nb + nl;
    const double m = (double)((n_terms + blockDim.x - 1) / blockDim.x) + 6.0 + 8.0 + DN_SPLITS;
    // (per-thread sums, the block tree, the roundings inside a term, and the row-split
    // partials of the prices)
    const double e = gamma_fp64_d(m) * A;
    bound[b] = g - e;
    if (errb) errb[b] = e;
  }
}

// ------------------------------------------------------------------ host side
dcopf_status ensure_dense_ha(dcopf_dual* h) {
  if (h->dense_ha.p) return DCOPF_OK;
  const HostNet& H = h->host;
  const SparseFactor& F = H.F;
  const int nb = H.n_bus, nl = H.n_line, n = F.n;
  std::vector<double> ha((size_t)nl * nb, 0.0);
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  auto worker = [&](int t) {
    std::vector<double> x(std::max(1, n));
    for (int j = t; j < nb; j += (int)nt) {
      const int p = F.pos_of_bus[j];
      if (p < 0) continue;  // slack column stays zero
      std::fill(x.begin(), x.end(), 0.0);
      x[p] = 1.0;
      host_ldl_solve(F, x.data());
      for (int l = 0; l < nl; ++l) {
        const int pf = F.pos_of_bus[H.line_from[l]], pt = F.pos_of_bus[H.line_to[l]];
        ha[(size_t)l * nb + j] = H.b[l] * ((pf >= 0 ? x[pf] : 0.0) - (pt >= 0 ? x[pt] : 0.0));
      }
    }
  };
  std::vector<std::thread> th;
  for (unsigned t = 1; t < nt; ++t) th.emplace_back(worker, (int)t);
  worker(0);
  for (auto& t : th) t.join();
  if (h->dense_ha.alloc(ha.size() * sizeof(double)) != cudaSuccess) return DCOPF_ERR_OOM;
  if (cudaMemcpy(h->dense_ha.p, ha.data(), ha.size() * sizeof(double), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return DCOPF_ERR_CUDA;
  return DCOPF_OK;
}

// Whether the dense path applies: few instances, no outages, H_a of modest size.
bool dense_path_applies(const dcopf_dual* h, int B, const int* outage) {
  const size_t bytes = (size_t)h->host.n_line * h->host.n_bus * sizeof(double);
  const size_t zs = (size_t)h->host.n_bus * sizeof(double);
  return outage == nullptr && B <= 8 && bytes <= ((size_t)2 << 30) && zs + 1024 <= h->smem_optin;
}

dcopf_status run_dense_base_flows(dcopf_dual* h, int B, const double* loads, cudaStream_t s) {
  dcopf_status r = ensure_dense_ha(h);
  if (r) return r;
  Workspace& w = h->ws;
  const int nl = h->host.n_line;
  dim3 grid((nl * 32 + 255) / 256, B);
  k_dense_base_flows<<<grid, 256, 0, s>>>(h->host.n_bus, nl, h->dense_ha.as<double>(), h->dev.phim,
                                          loads, w.f0.as<double>(), w.f0_32.as<float>(),
                                          w.u64.as<double>(), w.u32.as<float>(), w.demand.as<double>());
  h->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

template <typename S>
dcopf_status run_dense_certify(dcopf_dual* h, int B, const double* loads, const double* lam,
                               const S* mh, const S* ml, double* bound, double* errb,
                               const int* mask, const int* done, cudaStream_t s) {
  dcopf_status r = ensure_dense_ha(h);
  if (r) return r;
  const int nb = h->host.n_bus, nl = h->host.n_line;
  if (h->dense_part.alloc((size_t)std::max(B, 8) * DN_SPLITS * nb * sizeof(double)) != cudaSuccess)
    return DCOPF_ERR_OOM;
  dim3 grid((nb + DN_TILE - 1) / DN_TILE, DN_SPLITS, B);
  const size_t eta_smem = (size_t)((nl + DN_SPLITS - 1) / DN_SPLITS) * sizeof(double);
  const size_t z_smem = (size_t)nb * sizeof(double);
  if (eta_smem > h->smem_optin || z_smem > h->smem_optin) return DCOPF_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_dense_prices<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)eta_smem) != cudaSuccess ||
      cudaFuncSetAttribute(k_dense_certify<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)z_smem) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  k_dense_prices<S><<<grid, DN_TILE, eta_smem, s>>>(nb, nl, h->dense_ha.as<double>(), mh, ml,
                                                    h->dense_part.as<double>(), mask, done);
  k_dense_certify<S><<<B, 256, z_smem, s>>>(h->dev, h->dense_part.as<double>(), loads, lam, mh, ml,
                                            bound, errb, mask, done);
  h->launches += 2;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

template dcopf_status run_dense_certify<double>(dcopf_dual*, int, const double*, const double*,
                                                const double*, const double*, double*, double*,
                                                const int*, const int*, cudaStream_t);
template dcopf_status run_dense_certify<float>(dcopf_dual*, int, const double*, const double*,
                                               const float*, const float*, double*, double*,
                                               const int*, const int*, cudaStream_t);

}  // namespace dcopf
