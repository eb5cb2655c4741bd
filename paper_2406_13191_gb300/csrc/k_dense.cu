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
#include <cmath>
#include <thread>
#include <vector>

#include "dev.cuh"
#include "kernels.h"

namespace dcopf {

constexpr int DN_TILE = 128;    // buses per column tile of the H_a^T eta product
constexpr int DN_SPLITS = 64;   // row splits of that product
constexpr int DN_TERM_CTAS = 16;  // CTAs per instance summing the certificate's terms

// f0[b][i] = phim[i] - H_a[i,:] . d_b, demand[b] = sum d_b; a warp per (line, instance),
// four FMA chains with their loads in flight (FP64 latency is high on this part).
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
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int j = lane;
  for (; j + 224 < nb; j += 256) {  // eight row loads in flight per lane
    double a[8], e[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) { a[u] = row[j + 32 * u]; e[u] = d[j + 32 * u]; }
    s0 = fma(a[0], e[0], s0);
    s1 = fma(a[1], e[1], s1);
    s2 = fma(a[2], e[2], s2);
    s3 = fma(a[3], e[3], s3);
    s0 = fma(a[4], e[4], s0);
    s1 = fma(a[5], e[5], s1);
    s2 = fma(a[6], e[6], s2);
    s3 = fma(a[7], e[7], s3);
  }
  for (; j < nb; j += 32) s0 = fma(row[j], d[j], s0);
  double s = warp_sum((s0 + s1) + (s2 + s3));
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
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = i0;
  for (; i + 8 <= i1; i += 8) {  // eight rows in flight, four chains
    double h[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) h[u] = H[(size_t)(i + u) * nb + j];
#pragma unroll
    for (int u = 0; u < 8; u += 4) {
      s0 = fma(h[u], eta_s[i + u - i0], s0);
      s1 = fma(h[u + 1], eta_s[i + u + 1 - i0], s1);
      s2 = fma(h[u + 2], eta_s[i + u + 2 - i0], s2);
      s3 = fma(h[u + 3], eta_s[i + u + 3 - i0], s3);
    }
  }
  for (; i < i1; ++i) s0 = fma(H[(size_t)i * nb + j], eta_s[i - i0], s0);
  part[((size_t)b * DN_SPLITS + blockIdx.y) * nb + j] = (s0 + s1) + (s2 + s3);
}

// z[b][j] = sum of the row-split partials (fixed order, four chains).
__device__ __forceinline__ double dense_z(const double* __restrict__ part_b, int nb, int j) {
  const double* p = part_b + j;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll 4
  for (int q = 0; q < DN_SPLITS; q += 4) {
    a0 += p[(size_t)q * nb];
    a1 += p[(size_t)(q + 1) * nb];
    a2 += p[(size_t)(q + 2) * nb];
    a3 += p[(size_t)(q + 3) * nb];
  }
  return (a0 + a1) + (a2 + a3);
}

__device__ __forceinline__ double gamma_fp64_d(double m) {
  const double u = 1.1102230246251565e-16;
  return (m * u) / (1.0 - m * u);
}

// The certificate's terms (eq. (4) through the bus prices, as in k_certify) split over
// DN_TERM_CTAS blocks per instance: tpart[b][block] = (sum of terms, sum of |terms|,
// K, max |eta|).  Term t < n_gen: generator minimum; then n_bus bus terms; then n_line
// line terms.  A term's bus price is summed from the row-split partials on demand.  K
// bounds how the rounding of the prices moves the terms: a generator term is
// max(|pmin|, |pmax|)-Lipschitz in its bus price and a bus term |d_i|-Lipschitz, and
// |z^_j - z_j| <= gamma_k max|eta| colabs_j, so the terms move by at most
// gamma_k max|eta| K with K = sum_j max(|pmin_j|, |pmax_j|) colabs_bus(j) + sum_i |d_i| colabs_i.
// The last block of an instance to finish (arrival counter) adds the blocks' partials
// in block order and writes the bound: the result does not depend on which block is
// last.
template <typename S>
__global__ void k_dense_terms(DevNet N, const double* __restrict__ part,
                              const double* __restrict__ loads, const double* __restrict__ lambda,
                              const S* __restrict__ mu_hi, const S* __restrict__ mu_lo,
                              const double* __restrict__ colabs, double* __restrict__ tpart,
                              unsigned* __restrict__ arrive, int rows_per_split,
                              double* __restrict__ bound, double* __restrict__ errb,
                              const int* __restrict__ mask, const int* __restrict__ done) {
  __shared__ double red[32];
  __shared__ int s_last;
  const int b = blockIdx.y;
  if (mask && (mask[b] == 0 || (done && done[b]))) return;
  const int nb = N.n_bus, nl = N.n_line, ng = N.n_gen;
  const double* pb = part + (size_t)b * DN_SPLITS * nb;
  const double* d = loads + (size_t)b * nb;
  const S* mh = mu_hi + (size_t)b * nl;
  const S* ml = mu_lo + (size_t)b * nl;
  const double lam = lambda[b];
  const int nt = ng + nb + nl;
  const int stride = gridDim.x * blockDim.x;
  double g = 0.0, A = 0.0, K = 0.0, emax = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
    double v;
    if (t < ng) {
      double p;
      const int bus = N.gen_bus[t];
      const double z = N.pos_of_bus[bus] < 0 ? 0.0 : dense_z(pb, nb, bus);
      v = gen_min_value(lam + z, N.cost_quad[t], N.cost_lin[t], N.S, N.pmin[t], N.pmax[t], &p);
      K += fmax(fabs(N.pmin[t]), fabs(N.pmax[t])) * colabs[bus];
    } else if (t < ng + nb) {
      const int i = t - ng;
      const double z = N.pos_of_bus[i] < 0 ? 0.0 : dense_z(pb, nb, i);
      v = -(lam + z) * d[i];
      K += fabs(d[i]) * colabs[i];
    } else {
      const int l = t - ng - nb;
      const double eh = fmax((double)mh[l], 0.0), el = fmax((double)ml[l], 0.0);
      v = -eh * N.fmax[l] + el * N.fmin[l];
      emax = fmax(emax, fabs(eh - el));
    }
    g += v;
    A += fabs(v);
  }
  g = block_sum(g, red);
  A = block_sum(A, red);
  K = block_sum(K, red);
  emax = block_max(emax, red);
  if (threadIdx.x == 0) {
    double* o = tpart + ((size_t)b * DN_TERM_CTAS + blockIdx.x) * 4;
    o[0] = g;
    o[1] = A;
    o[2] = K;
    o[3] = emax;
    __threadfence();
    s_last = atomicAdd(arrive + b, 1u) == DN_TERM_CTAS - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double gs = 0.0, As = 0.0, Ks = 0.0, em = 0.0;
  for (int q = 0; q < DN_TERM_CTAS; ++q) {
    const double* o = tpart + ((size_t)b * DN_TERM_CTAS + q) * 4;
    gs += __ldcg(o);
    As += __ldcg(o + 1);
    Ks += __ldcg(o + 2);
    em = fmax(em, __ldcg(o + 3));
  }
  arrive[b] = 0u;  // ready for the next certification
  // summation: per-thread sums, the block tree, the blocks' sum, and the few
  // roundings inside a term
  const int total = DN_TERM_CTAS * blockDim.x;
  const double m = (double)((nt + total - 1) / total) + 8.0 + (double)DN_TERM_CTAS + 6.0;
  // prices: eta (1), the longest FMA chain of a row split (a quarter of its rows plus
  // up to 7 tail rows), the split's 4-chain merge (2), the split sum's chains and merge
  // (DN_SPLITS / 4 + 2); K is itself a rounded sum of non-negative terms (one more
  // gamma of its length)
  const double kz = 1.0 + (double)(rows_per_split / 4 + 8) + 2.0 + (double)(DN_SPLITS / 4 + 2);
  const double e = gamma_fp64_d(m) * As + gamma_fp64_d(kz) * em * Ks * (1.0 + gamma_fp64_d(m + kz));
  bound[b] = gs - e;
  if (errb) errb[b] = e;
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
  // column sums of |H_a| (rounded upward by a relative margin far above their rounding)
  std::vector<double> colabs(nb, 0.0);
  for (int l = 0; l < nl; ++l)
    for (int j = 0; j < nb; ++j) colabs[j] += std::fabs(ha[(size_t)l * nb + j]);
  for (double& c : colabs) c *= 1.0 + 1e-9;
  if (h->dense_colabs.alloc(colabs.size() * sizeof(double)) != cudaSuccess ||
      cudaMemcpy(h->dense_colabs.p, colabs.data(), colabs.size() * sizeof(double),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return DCOPF_ERR_OOM;
  if (h->dense_ha.alloc(ha.size() * sizeof(double)) != cudaSuccess) return DCOPF_ERR_OOM;
  if (cudaMemcpy(h->dense_ha.p, ha.data(), ha.size() * sizeof(double), cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return DCOPF_ERR_CUDA;
  return DCOPF_OK;
}

// Whether the dense path applies: few instances, no outages, H_a of modest size.
bool dense_path_applies(const dcopf_dual* h, int B, const int* outage) {
  const size_t bytes = (size_t)h->host.n_line * h->host.n_bus * sizeof(double);
  return outage == nullptr && B <= 8 && bytes <= ((size_t)2 << 30);
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
  const int Bc = std::max(B, 8);
  // [Bc][DN_SPLITS][nb] partials, [Bc][DN_TERM_CTAS][4] term sums, [Bc] arrival counters
  const size_t part_n = (size_t)Bc * DN_SPLITS * nb, tp_n = (size_t)Bc * DN_TERM_CTAS * 4;
  const size_t need = (part_n + tp_n + (size_t)Bc) * sizeof(double);
  if (h->dense_part.bytes < need) {
    if (h->dense_part.alloc(need) != cudaSuccess) return DCOPF_ERR_OOM;
    if (cudaMemset(h->dense_part.p, 0, need) != cudaSuccess) return DCOPF_ERR_CUDA;
  }
  double* part = h->dense_part.as<double>();
  double* tpart = part + part_n;
  unsigned* arrive = (unsigned*)(tpart + tp_n);
  const size_t eta_smem = (size_t)((nl + DN_SPLITS - 1) / DN_SPLITS) * sizeof(double);
  if (eta_smem > h->smem_optin) return DCOPF_ERR_UNSUPPORTED;
  if (eta_smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_dense_prices<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)eta_smem) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  dim3 grid((nb + DN_TILE - 1) / DN_TILE, DN_SPLITS, B);
  k_dense_prices<S><<<grid, DN_TILE, eta_smem, s>>>(nb, nl, h->dense_ha.as<double>(), mh, ml, part,
                                                    mask, done);
  k_dense_terms<S><<<dim3(DN_TERM_CTAS, B), 256, 0, s>>>(
      h->dev, part, loads, lam, mh, ml, h->dense_colabs.as<double>(), tpart, arrive,
      (nl + DN_SPLITS - 1) / DN_SPLITS, bound, errb, mask, done);
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
