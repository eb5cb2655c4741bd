// Fused persistent solve of one instance: every iteration of the projected dual
// ascent (Section 3.3, Algorithm 1 and the Adam / AdaGrad rules) runs inside one
// cooperative kernel with one CTA per SM.
//
// Data placement: CTA c owns a contiguous block of lines (rows of Phi~), keeps those
// rows of Phi~ (FP32) in shared memory for the whole solve, and owns the dual state
// of its lines (mu_hi, mu_lo, optimiser moments).  lambda and its moments are
// replicated in every CTA and updated identically.
//
// Iteration t (all CTAs):
//   A  eta = mu_hi - mu_lo on own rows; partial adjoint Phi~_c^T eta_c for all gens
//      -> Pp[j][c]                                   (eq. (6): C^T mu)
//   -- grid barrier 1 --
//   B  value of evaluation t-1 (sums of the per-CTA FP64 partials in a fixed order,
//      identical in every CTA) -> best-point tracking and the stop tests;
//      gens slice of CTA c: pi~_j = sum_c Pp[j][c], closed-form x*_j (eq. (6)/(16))
//      -> X[j], partial cost and dispatch sums -> Q[c]
//   -- grid barrier 2 --
//   C  forward f = Phi~_c X + f0 on own rows (constraint (1c)); supergradient and the
//      line part of the value -> R[c]; projected step of own mu and of lambda.
// The value of evaluation t is complete only after barrier 1 of iteration t+1, so
// the best point is taken from a copy of the previous iterate.
#include "dev.cuh"
#include "kernels.h"

namespace dcopf {

struct FusedArgs {
  DevNet N;
  StepArgs P;
  SolveState<float> st;
  const float* f0;        // [n_line]
  double demand;
  float* Pp;              // [n_gen][G]
  float* X;               // [n_gen]
  double* Q;              // [G][2]
  double* R;              // [G]
  unsigned* bar;
  int* err;
  int max_iters;
  double tol;
  int rows_per_cta;
  int gens_per_cta;
  int phi_in_smem;
  uint64_t timeout_ns;
};

template <typename S>
__device__ __forceinline__ S fused_rule(const StepArgs& P, S theta, S g, S& s1, S& s2, S a, S bc1,
                                        S bc2) {
  if (P.rule == DCOPF_GDM) {
    s1 = S(P.rho) * s1 + a * g;
    theta += s1;
    if (P.as_printed) theta += a * g;
  } else if (P.rule == DCOPF_ADAM) {
    s1 = S(P.beta1) * s1 + (S(1) - S(P.beta1)) * g;
    s2 = S(P.beta2) * s2 + (S(1) - S(P.beta2)) * g * g;
    theta += a * (s1 / bc1) / (sqrt(s2 / bc2) + S(P.eps));
  } else {
    s1 += g * g;
    theta += a * g / (sqrt(s1) + S(P.eps));
  }
  return theta;
}

__global__ void __launch_bounds__(256, 1) k_fused_solve(FusedArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const DevNet& N = A.N;
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
  const int nl = N.n_line, ng = N.n_gen;
  const int r0 = min(nl, c * A.rows_per_cta), r1 = min(nl, r0 + A.rows_per_cta);
  const int nr = r1 - r0;
  const int j0 = min(ng, c * A.gens_per_cta), j1 = min(ng, j0 + A.gens_per_cta);
  // shared memory carve-up
  float* xs = (float*)smem_raw;                                  // [ng]
  float* row = xs + ((ng + 3) & ~3);                             // per-row arrays, 12 x rpc
  const int rpc = A.rows_per_cta;
  float *eta = row, *mh = row + rpc, *ml = row + 2 * rpc, *h1 = row + 3 * rpc, *h2 = row + 4 * rpc,
        *l1 = row + 5 * rpc, *l2 = row + 6 * rpc, *ph = row + 7 * rpc, *pl = row + 8 * rpc,
        *fmx = row + 9 * rpc, *fmn = row + 10 * rpc, *f0 = row + 11 * rpc;
  float* phis = row + 12 * rpc;                                  // [rpc][ng] when resident
  __shared__ double red[32];
  __shared__ double s_lam[4];  // lam, s1, s2, lam_prev
  __shared__ int s_stop;

  const float* phi = A.phi_in_smem ? phis : (N.phi32 + (size_t)r0 * ng);
  if (A.phi_in_smem)
    for (int q = tid; q < nr * ng; q += blockDim.x) phis[q] = N.phi32[(size_t)r0 * ng + q];
  SolveState<float>& st = A.st;
  for (int r = tid; r < nr; r += blockDim.x) {
    int i = r0 + r;
    mh[r] = st.mu_hi[i]; ml[r] = st.mu_lo[i];
    h1[r] = st.s1_hi[i]; h2[r] = st.s2_hi[i]; l1[r] = st.s1_lo[i]; l2[r] = st.s2_lo[i];
    fmx[r] = N.fmax32[i]; fmn[r] = N.fmin32[i]; f0[r] = A.f0[i];
  }
  if (tid == 0) {
    s_lam[0] = st.lam[0]; s_lam[1] = st.lam_s1[0]; s_lam[2] = st.lam_s2[0]; s_lam[3] = st.lam[0];
    s_stop = 0;
  }
  double best = st.best[0];
  double prev_val = st.prev[0];
  int t = st.iter[0];
  int best_iter = st.best_iter[0];
  double best_lam = st.best_lam[0];
  int cand = 0;
  bool pending = false;         // an evaluation whose value is not yet assembled
  double cost_t = 0.0, psum_t = 0.0;
  unsigned epoch = 0;
  __syncthreads();

  for (;;) {
    // ---------------- phase A: partial adjoint over own rows
    for (int r = tid; r < nr; r += blockDim.x) eta[r] = mh[r] - ml[r];
    __syncthreads();
    for (int j = tid; j < ng; j += blockDim.x) {
      float s = 0.f;
      for (int r = 0; r < nr; ++r) s = fmaf(phi[(size_t)r * ng + j], eta[r], s);
      A.Pp[(size_t)j * G + c] = s;
    }
    if (!grid_barrier(A.bar, G, epoch, A.err, A.timeout_ns)) break;
    // ---------------- phase B: value of the pending evaluation, stop tests
    if (pending) {
      double lsum = 0.0;
      for (int q = tid; q < G; q += blockDim.x) lsum += A.R[q];
      // fixed-order reduction: identical in every CTA
      lsum = block_sum(lsum, red);
      double lamp = s_lam[3];
      double val = cost_t + lamp * (psum_t - A.demand) + lsum;
      bool better = val > best;
      if (better) {
        best = val; best_lam = lamp; best_iter = t;
        for (int r = tid; r < nr; r += blockDim.x) { st.best_hi[r0 + r] = ph[r]; st.best_lo[r0 + r] = pl[r]; }
      }
      if (st.has_target && best >= st.thresh[0] + st.margin[0]) cand = 1;
      if (t >= A.max_iters) cand = 2;
      if (A.tol > 0.0 && t > 1 && fabs(val - prev_val) < A.tol) cand = 2;
      if (best > 1e300) cand = 2;
      prev_val = val;
      pending = false;
      if (cand) break;
    }
    // gens slice: reduce partials, closed-form minimiser
    {
      const double lam = s_lam[0];
      double cs = 0.0, ps = 0.0;
      const int nj = j1 - j0;
      // (gen, part) pairs spread over the whole block; 8 lanes per gen
      const int lanes_per = 8;
      for (int base = 0; base < nj * lanes_per; base += blockDim.x) {
        int q = base + tid;
        int jj = q / lanes_per, part = q % lanes_per;
        float s = 0.f;
        if (jj < nj)
          for (int cc = part; cc < G; cc += lanes_per) s += A.Pp[(size_t)(j0 + jj) * G + cc];
        // reduce the 8 lanes of this gen (aligned groups of 8 inside a warp)
        s += __shfl_xor_sync(0xffffffffu, s, 1);
        s += __shfl_xor_sync(0xffffffffu, s, 2);
        s += __shfl_xor_sync(0xffffffffu, s, 4);
        if (jj < nj && part == 0) {
          int j = j0 + jj;
          double w = N.ctil[j] + N.sigma[j] * lam + (double)s;
          double x = inner_x<double>(w, N.mq[j]);
          A.X[j] = (float)x;
          cs += (N.mq[j] * x + N.ctil[j]) * x + N.cconst[j];
          ps += N.mid[j] + N.sigma[j] * x;
        }
      }
      cs = block_sum(cs, red);
      ps = block_sum(ps, red);
      if (tid == 0) { A.Q[2 * c] = cs; A.Q[2 * c + 1] = ps; }
    }
    if (!grid_barrier(A.bar, G, epoch, A.err, A.timeout_ns)) break;
    // ---------------- phase C: forward on own rows, supergradient, step
    for (int j = tid; j < ng; j += blockDim.x) xs[j] = A.X[j];
    {
      double cs = 0.0, ps = 0.0;
      for (int q = tid; q < G; q += blockDim.x) { cs += A.Q[2 * q]; ps += A.Q[2 * q + 1]; }
      cost_t = block_sum(cs, red);
      psum_t = block_sum(ps, red);
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    for (int r = warp; r < nr; r += nw) {
      float s = 0.f;
      const float* pr = phi + (size_t)r * ng;
      for (int j = lane; j < ng; j += 32) s = fmaf(pr[j], xs[j], s);
      s = warp_sum(s);
      if (lane == 0) eta[r] = s + f0[r];  // eta[] reused as the flow of own rows
    }
    __syncthreads();
    t += 1;
    const float scale = (float)pow(A.P.decay, (double)(t - 1));
    const float bc1 = (float)(1.0 - pow(A.P.beta1, (double)t));
    const float bc2 = (float)(1.0 - pow(A.P.beta2, (double)t));
    const float am = (float)(A.P.alpha * scale);
    double lacc = 0.0;
    for (int r = tid; r < nr; r += blockDim.x) {
      float f = eta[r];
      float gh = f - fmx[r], gl = fmn[r] - f;
      lacc += (double)mh[r] * (double)gh + (double)ml[r] * (double)gl;
      ph[r] = mh[r];
      pl[r] = ml[r];
      float nh = fused_rule<float>(A.P, mh[r], gh, h1[r], h2[r], am, bc1, bc2);
      float nlo = fused_rule<float>(A.P, ml[r], gl, l1[r], l2[r], am, bc1, bc2);
      mh[r] = nh > 0.f ? nh : 0.f;
      ml[r] = nlo > 0.f ? nlo : 0.f;
    }
    lacc = block_sum(lacc, red);
    if (tid == 0) {
      A.R[c] = lacc;
      double lam = s_lam[0], s1 = s_lam[1], s2 = s_lam[2];
      s_lam[3] = lam;
      double al = A.P.alpha_lambda * (double)pow(A.P.decay, (double)(t - 1));
      double gl = psum_t - A.demand;
      lam = fused_rule<double>(A.P, lam, gl, s1, s2, al, 1.0 - pow(A.P.beta1, (double)t),
                               1.0 - pow(A.P.beta2, (double)t));
      s_lam[0] = lam; s_lam[1] = s1; s_lam[2] = s2;
    }
    pending = true;
    __syncthreads();
  }
  // ---------------- write back (resumable state)
  __syncthreads();
  for (int r = tid; r < nr; r += blockDim.x) {
    int i = r0 + r;
    st.mu_hi[i] = mh[r]; st.mu_lo[i] = ml[r];
    st.s1_hi[i] = h1[r]; st.s2_hi[i] = h2[r]; st.s1_lo[i] = l1[r]; st.s2_lo[i] = l2[r];
  }
  if (c == 0 && tid == 0) {
    st.lam[0] = s_lam[0]; st.lam_s1[0] = s_lam[1]; st.lam_s2[0] = s_lam[2];
    st.best[0] = best; st.best_lam[0] = best_lam; st.best_iter[0] = best_iter;
    st.iter[0] = pending ? t - 1 : t;  // an unassembled evaluation is redone on resume
    st.prev[0] = prev_val;
    st.cand[0] = cand;
  }
}

dcopf_status run_iters_fused(dcopf_dual* h, const StepArgs& P, SolveState<float>& st, int max_iters,
                             double tol, cudaStream_t s) {
  const DevNet& N = h->dev;
  const int G = h->sm_count;
  const int nl = N.n_line, ng = N.n_gen;
  FusedArgs A{};
  A.N = N;
  A.P = P;
  A.st = st;
  A.f0 = h->ws.f0_32.as<float>();
  A.rows_per_cta = (nl + G - 1) / G;
  A.gens_per_cta = (ng + G - 1) / G;
  size_t base = (size_t)(((ng + 3) & ~3) + 12 * A.rows_per_cta) * sizeof(float);
  size_t phi_bytes = (size_t)A.rows_per_cta * ng * sizeof(float);
  A.phi_in_smem = (base + phi_bytes + 4096 <= h->smem_optin) ? 1 : 0;
  size_t smem = base + (A.phi_in_smem ? phi_bytes : 0);
  if (smem + 1024 > h->smem_optin) return DCOPF_ERR_UNSUPPORTED;
  // scratch: Pp [ng][G] f32, X [ng] f32, Q [G][2] f64, R [G] f64, demand read back below
  size_t need = (size_t)ng * G * 4 + (size_t)ng * 4 + 256 + (size_t)G * 24 + 256;
  if (h->ws.misc.alloc(need) != cudaSuccess) return DCOPF_ERR_OOM;
  char* m = h->ws.misc.as<char>();
  A.Pp = (float*)m;
  A.X = (float*)(m + (size_t)ng * G * 4);
  A.Q = (double*)(m + (((size_t)ng * G * 4 + (size_t)ng * 4 + 255) & ~(size_t)255));
  A.R = A.Q + 2 * G;
  A.bar = h->d_bar;
  A.err = h->d_err;
  A.max_iters = max_iters;
  A.tol = tol;
  A.timeout_ns = 2000000000ull;
  double demand = 0.0;
  if (cudaMemcpyAsync(&demand, h->ws.demand.as<double>(), sizeof(double), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  A.demand = demand;
  if (cudaFuncSetAttribute(k_fused_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return DCOPF_ERR_CUDA;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_solve, 256, smem);
  if (per_sm < 1) return DCOPF_ERR_UNSUPPORTED;
  if (cudaMemsetAsync(h->d_bar, 0, sizeof(unsigned), s) != cudaSuccess) return DCOPF_ERR_CUDA;
  void* args[] = {&A};
  cudaError_t e = cudaLaunchCooperativeKernel((void*)k_fused_solve, G, 256, args, smem, s);
  h->launches += 1;
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

}  // namespace dcopf
