// Per-phase kernels of one dual evaluation and one ascent step, batched over
// instances (row b of every [batch][n] array is instance b).
//
// One iteration of the method (Section 3.3, Algorithm 1) is
//   eta      = mu_hi - mu_lo  (+ rank-1 outage term)          k_eta
//   pi~      = Phi~^T eta          (adjoint, eq. (6) C^T mu)    k_adjoint
//   x*       = closed-form minimiser (eq. (6) / eq. (16))       k_minimize
//   f        = Phi~ x* + f0        (forward, constraint (1c))   k_forward
//   value, supergradient (FP64 accumulation)                    k_grad_value
//   projected GDM / Adam / AdaGrad step on (lambda, mu)         k_step
// These kernels are the unfused building blocks: dcopf_dual_eval and the plain
// path launch them one by one; the other paths replace the two operator products.
#include "dev.cuh"
#include "kernels.h"

namespace dcopf {

// eta[b][i] = mu_hi - mu_lo for i != k; for an outaged line k, eta'_k = u^T eta
// (the adjoint of the post-outage PTDF (I + u e_k^T) H_a is H_a^T (I + e_k u^T)).
template <typename T, typename S>
__global__ void k_eta(int nl, const S* __restrict__ mh, const S* __restrict__ ml,
                      const int* __restrict__ outage, const T* __restrict__ u,
                      T* __restrict__ eta) {
  __shared__ T red[32];
  const int b = blockIdx.x;
  const int k = outage ? outage[b] : -1;
  const S* h = mh + (size_t)b * nl;
  const S* lo = ml + (size_t)b * nl;
  T* e = eta + (size_t)b * nl;
  T s = T(0);
  for (int i = threadIdx.x; i < nl; i += blockDim.x) {
    T v = (i == k) ? T(0) : (T)((double)h[i] - (double)lo[i]);
    e[i] = v;
    if (k >= 0) s += u[(size_t)b * nl + i] * v;
  }
  if (k >= 0) {
    s = block_sum(s, red);
    if (threadIdx.x == 0) e[k] = s;
  }
}

// pit[b][j] = sum_i Phi~[i][j] eta[b][i]: one block per (j, b) over row j of Phi~^T,
// deterministic block reduction.
template <typename T>
__global__ void k_adjoint(int nl, int ng, const T* __restrict__ phit, const T* __restrict__ eta,
                          T* __restrict__ pit) {
  __shared__ T red[32];
  const int j = blockIdx.x, b = blockIdx.y;
  const T* row = phit + (size_t)j * nl;
  const T* e = eta + (size_t)b * nl;
  T s = T(0);
  for (int i = threadIdx.x; i < nl; i += blockDim.x) s += row[i] * e[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) pit[(size_t)b * ng + j] = s;
}

// x*[b][j] from w = ctil_j + sigma_j lambda_b + pi~_bj (FP64), plus per-instance
// sums of the generation cost and of the dispatch.
// sv (nullable, FP64 path): eq. (16)'s s.  With it the quadratic term M x^2 is replaced
// by its lower envelope -sqrt(M) s x - s^2 / 4 (equal at s = -2 sqrt(M) x), so the
// minimiser over the box is the vertex x = -sign(w - sqrt(M) s) (Remark 2).
template <typename T>
__global__ void k_minimize(DevNet N, const double* __restrict__ lambda, const T* __restrict__ pit,
                           T* __restrict__ x, double* __restrict__ sumcost,
                           double* __restrict__ sump, const int* __restrict__ done,
                           const double* __restrict__ sv) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  if (done && done[b]) return;
  const int ng = N.n_gen;
  const double lam = lambda[b];
  double c = 0.0, p = 0.0;
  for (int j = threadIdx.x; j < ng; j += blockDim.x) {
    double w = N.ctil[j] + N.sigma[j] * lam + (double)pit[(size_t)b * ng + j];
    double xx;
    if (sv) {
      const double sq = sqrt(N.mq[j]), sj = sv[(size_t)b * ng + j];
      xx = inner_x<double>(w - sq * sj, 0.0);
      c += (N.ctil[j] - sq * sj) * xx - 0.25 * sj * sj + N.cconst[j];
    } else {
      xx = inner_x<double>(w, N.mq[j]);
      c += (N.mq[j] * xx + N.ctil[j]) * xx + N.cconst[j];
    }
    x[(size_t)b * ng + j] = (T)xx;
    p += N.mid[j] + N.sigma[j] * xx;
  }
  c = block_sum(c, red);
  p = block_sum(p, red);
  if (threadIdx.x == 0) {
    sumcost[b] = c;
    sump[b] = p;
  }
}

// f[b][i] = sum_j Phi~[i][j] x[b][j] + f0[b][i]: one block per (i, b).
template <typename T>
__global__ void k_forward(int nl, int ng, const T* __restrict__ phi, const T* __restrict__ x,
                          const double* __restrict__ f0, double* __restrict__ f,
                          const int* __restrict__ done) {
  __shared__ T red[32];
  const int i = blockIdx.x, b = blockIdx.y;
  if (done && done[b]) return;
  const T* row = phi + (size_t)i * ng;
  const T* xx = x + (size_t)b * ng;
  T s = T(0);
  for (int j = threadIdx.x; j < ng; j += blockDim.x) s += row[j] * xx[j];
  s = block_sum(s, red);
  if (threadIdx.x == 0) f[(size_t)b * nl + i] = (double)s + f0[(size_t)b * nl + i];
}

// Outage correction f' = f + u f_k, supergradient (f - fmax, fmin - f; zero for the
// outaged line) and the FP64 dual value
//   g = sum_j cost_j(p*) + lambda (1^T p* - D) + mu_hi^T (f - fmax) + mu_lo^T (fmin - f).
template <typename S, typename G>
__global__ void k_grad_value(DevNet N, const int* __restrict__ outage, const double* __restrict__ u,
                             const double* __restrict__ lambda, const S* __restrict__ mh,
                             const S* __restrict__ ml, double* __restrict__ f,
                             const double* __restrict__ sumcost, const double* __restrict__ sump,
                             const double* __restrict__ demand, double* __restrict__ value,
                             double* __restrict__ glam, G* __restrict__ ghi, G* __restrict__ glo,
                             const int* __restrict__ done) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  if (done && done[b]) return;
  const int nl = N.n_line;
  const int k = outage ? outage[b] : -1;
  double* fr = f + (size_t)b * nl;
  double fk = 0.0;
  if (k >= 0) fk = fr[k];
  __syncthreads();
  double acc = 0.0;
  for (int i = threadIdx.x; i < nl; i += blockDim.x) {
    double fi = fr[i];
    if (k >= 0) fi += u[(size_t)b * nl + i] * fk;
    fr[i] = fi;
    double gh = fi - N.fmax[i], gl = N.fmin[i] - fi;
    if (i == k) { gh = 0.0; gl = 0.0; }
    if (ghi) ghi[(size_t)b * nl + i] = (G)gh;
    if (glo) glo[(size_t)b * nl + i] = (G)gl;
    acc += (double)mh[(size_t)b * nl + i] * gh + (double)ml[(size_t)b * nl + i] * gl;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) {
    double gl = sump[b] - demand[b];
    value[b] = sumcost[b] + lambda[b] * gl + acc;
    if (glam) glam[b] = gl;
  }
}

__global__ void k_to_float(long long n, const double* __restrict__ a, float* __restrict__ b) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) b[t] = (float)a[t];
}

__global__ void k_dispatch(DevNet N, int B, const double* __restrict__ x, double* __restrict__ p) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * N.n_gen) return;
  int j = t % N.n_gen;
  p[t] = N.mid[j] + N.sigma[j] * x[t];
}
__global__ void k_dispatch32(DevNet N, int B, const float* __restrict__ x, double* __restrict__ p) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * N.n_gen) return;
  int j = t % N.n_gen;
  p[t] = N.mid[j] + N.sigma[j] * (double)x[t];
}

// ---------------------------------------------------------------- ascent step
// (rule_step, the rule on one coordinate, is in kernels.h)

// Step kernel: records the best point (largest in-loop value) before stepping,
// then updates mu (projected to >= 0) and lambda.  Grid (ceil(nl/256), B).
template <typename S>
__global__ void k_step(int nl, StepArgs P, const double* __restrict__ value,
                       const double* __restrict__ glam, const double* __restrict__ ghi,
                       const double* __restrict__ glo, SolveState<S> st) {
  const int b = blockIdx.y;
  if (st.done[b] || st.cand[b] == 2) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = st.iter[b] + 1;  // evaluation count of this step (1-based)
  __shared__ double s_pw[3];       // step-size factors, once per block (FP64 pow is slow)
  if (threadIdx.x == 0) {
    s_pw[0] = pow(P.decay, (double)(t - 1));
    s_pw[1] = 1.0 - pow(P.beta1, (double)t);
    s_pw[2] = 1.0 - pow(P.beta2, (double)t);
  }
  __syncthreads();
  StepArgs Q = P;
  Q.bc1 = s_pw[1];
  Q.bc2 = s_pw[2];
  const double scale = s_pw[0];
  const bool better = value[b] > st.best[b];
  const size_t o = (size_t)b * nl + i;
  if (i < nl) {
    S h = st.mu_hi[o], l = st.mu_lo[o];
    if (better) {
      st.best_hi[o] = h;
      st.best_lo[o] = l;
    }
    S a = (S)(P.alpha * scale);
    S h2 = rule_step<S>(Q, h, (S)ghi[o], st.s1_hi[o], st.s2_hi[o], a);
    S l2 = rule_step<S>(Q, l, (S)glo[o], st.s1_lo[o], st.s2_lo[o], a);
    st.mu_hi[o] = h2 > S(0) ? h2 : S(0);
    st.mu_lo[o] = l2 > S(0) ? l2 : S(0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    // lambda and per-instance bookkeeping.  st.best is read by every block of this
    // instance row, so the new best value goes to st.best_next and is published by
    // k_close_iter after this kernel.
    double lam = st.lam[b];
    if (better) {
      st.best_next[b] = value[b];
      st.best_lam[b] = lam;
      st.best_iter[b] = t;
    }
    double a = P.alpha_lambda * scale;
    double s1 = st.lam_s1[b], s2 = st.lam_s2[b];
    lam = rule_step<double>(Q, lam, glam[b], s1, s2, a);
    st.lam[b] = lam;
    st.lam_s1[b] = s1;
    st.lam_s2[b] = s2;
    st.prev[b] = value[b];
    st.iter[b] = t;
  }
}

// Step of eq. (16)'s s (free, mu's step size): supergradient -sqrt(M) x* - s / 2 at the
// evaluated point.  Runs before k_step (which advances the iteration count).
__global__ void k_step_s(DevNet N, StepArgs P, const double* __restrict__ x, SolveStateBase st) {
  const int b = blockIdx.y;
  if (st.done[b] || st.cand[b] == 2) return;
  const int ng = N.n_gen;
  const int t = st.iter[b] + 1;
  __shared__ double s_pw[3];
  if (threadIdx.x == 0) {
    s_pw[0] = pow(P.decay, (double)(t - 1));
    s_pw[1] = 1.0 - pow(P.beta1, (double)t);
    s_pw[2] = 1.0 - pow(P.beta2, (double)t);
  }
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ng) return;
  StepArgs Q = P;
  Q.bc1 = s_pw[1];
  Q.bc2 = s_pw[2];
  const size_t o = (size_t)b * ng + j;
  const double sj = st.s[o];
  const double g = -sqrt(N.mq[j]) * x[o] - 0.5 * sj;
  st.s[o] = rule_step<double>(Q, sj, g, st.s1_s[o], st.s2_s[o], P.alpha * s_pw[0]);
}

// Closes an iteration: publishes best_next, applies the stop tests on the in-loop
// value (target crossing -> candidate for certification; |g_t - g_{t-1}| < tol;
// iteration cap).  One thread per instance.
__global__ void k_close_iter(int B, int max_iters, double tol, SolveStateBase st) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || st.done[b] || st.cand[b] == 2) return;
  double bn = st.best_next[b];
  if (bn > st.best[b]) st.best[b] = bn;
  if (st.has_target && st.best[b] >= st.thresh[b] + st.margin[b]) st.cand[b] = 1;
  if (st.iter[b] >= max_iters) st.cand[b] = 2;
  if (tol > 0.0 && st.iter[b] > 1 && fabs(st.prev[b] - st.prev2[b]) < tol) st.cand[b] = 2;
  st.prev2[b] = st.prev[b];
}

// ---------------------------------------------------------------- host drivers
namespace {
inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }
// threads per output of the reduction kernels: about 8 elements per thread, 32..256
inline int red_threads(int n) {
  int t = 32;
  while (t < 256 && t * 8 < n) t *= 2;
  return t;
}
}  // namespace

dcopf_status run_eval_unfused(dcopf_dual* h, int B, const int* outage, const double* lambda,
                              const double* mh, const double* ml, int precision, double* value,
                              double* glam, double* ghi, double* glo, double* dispatch,
                              cudaStream_t s) {
  const DevNet& N = h->dev;
  Workspace& w = h->ws;
  const int nl = N.n_line, ng = N.n_gen;
  dim3 gl(nl, B), gg(ng, B);
  const int ta = red_threads(nl), tf = red_threads(ng);
  if (precision == DCOPF_FP64) {
    k_eta<double, double><<<B, 256, 0, s>>>(nl, mh, ml, outage, w.u64.as<double>(), w.eta64.as<double>());
    k_adjoint<double><<<gg, ta, 0, s>>>(nl, ng, N.phit64, w.eta64.as<double>(), w.pit64.as<double>());
    k_minimize<double><<<B, 256, 0, s>>>(N, lambda, w.pit64.as<double>(), w.x64.as<double>(),
                                         w.sumcost.as<double>(), w.sump.as<double>(), nullptr, nullptr);
    k_forward<double><<<gl, tf, 0, s>>>(nl, ng, N.phi64, w.x64.as<double>(), w.f0.as<double>(),
                                         w.f.as<double>(), nullptr);
    if (dispatch) k_dispatch<<<cdiv((long long)B * ng, 256), 256, 0, s>>>(N, B, w.x64.as<double>(), dispatch);
  } else {
    k_eta<float, double><<<B, 256, 0, s>>>(nl, mh, ml, outage, w.u32.as<float>(), w.eta32.as<float>());
    k_adjoint<float><<<gg, ta, 0, s>>>(nl, ng, N.phit32, w.eta32.as<float>(), w.pit32.as<float>());
    k_minimize<float><<<B, 256, 0, s>>>(N, lambda, w.pit32.as<float>(), w.x32.as<float>(),
                                        w.sumcost.as<double>(), w.sump.as<double>(), nullptr, nullptr);
    k_forward<float><<<gl, tf, 0, s>>>(nl, ng, N.phi32, w.x32.as<float>(), w.f0.as<double>(),
                                        w.f.as<double>(), nullptr);
    if (dispatch) k_dispatch32<<<cdiv((long long)B * ng, 256), 256, 0, s>>>(N, B, w.x32.as<float>(), dispatch);
  }
  h->launches += 4 + (dispatch ? 1 : 0);
  return run_eval_finish(h, B, outage, lambda, mh, ml, value, glam, ghi, glo, nullptr, s);
}

// xsum[b][j] += k^2 x[b][j] and wsum[b] += k^2 for the k-th evaluation of every
// running instance (k = evaluations before this one + 1).
template <typename T>
__global__ void k_accum_mean(int ng, const T* __restrict__ x, SolveStateBase st) {
  const int b = blockIdx.x;
  if (st.done[b]) return;
  const float k = (float)(st.iter[b] + 1);
  const float wk = k * k;
  for (int j = threadIdx.x; j < ng; j += blockDim.x)
    st.xsum[(size_t)b * ng + j] += wk * (float)x[(size_t)b * ng + j];
  if (threadIdx.x == 0) st.wsum[b] += (double)wk;
}

__global__ void k_mean_out(DevNet N, const float* __restrict__ xsum, const double* __restrict__ wsum,
                           double* __restrict__ out) {
  const int b = blockIdx.x, ng = N.n_gen;
  const double w = wsum[b];
  for (int j = threadIdx.x; j < ng; j += blockDim.x) {
    const double x = w > 0.0 ? (double)xsum[(size_t)b * ng + j] / w : 0.0;
    out[(size_t)b * ng + j] = N.mid[j] + N.sigma[j] * x;
  }
}

template <typename T>
void launch_accum_mean(dcopf_dual* h, int B, const T* x, const SolveStateBase& st, cudaStream_t s) {
  k_accum_mean<T><<<B, 256, 0, s>>>(h->dev.n_gen, x, st);
  h->launches += 1;
}
template void launch_accum_mean<double>(dcopf_dual*, int, const double*, const SolveStateBase&, cudaStream_t);
template void launch_accum_mean<float>(dcopf_dual*, int, const float*, const SolveStateBase&, cudaStream_t);

void launch_mean_out(dcopf_dual* h, int B, const SolveStateBase& st, double* out, cudaStream_t s) {
  k_mean_out<<<B, 256, 0, s>>>(h->dev, st.xsum, st.wsum, out);
  h->launches += 1;
}

void launch_adjoint64(dcopf_dual* h, int B, const int* outage, const double* mh,
                      const double* ml, cudaStream_t s) {
  const DevNet& N = h->dev;
  Workspace& w = h->ws;
  const int nl = N.n_line, ng = N.n_gen;
  k_eta<double, double><<<B, 256, 0, s>>>(nl, mh, ml, outage, w.u64.as<double>(), w.eta64.as<double>());
  k_adjoint<double><<<dim3(ng, B), red_threads(nl), 0, s>>>(nl, ng, N.phit64, w.eta64.as<double>(),
                                                            w.pit64.as<double>());
  h->launches += 2;
}

void launch_forward64(dcopf_dual* h, int B, const double* x, const double* f0, double* f,
                      cudaStream_t s) {
  const DevNet& N = h->dev;
  const int nl = N.n_line, ng = N.n_gen;
  k_forward<double><<<dim3(nl, B), red_threads(ng), 0, s>>>(nl, ng, N.phi64, x, f0, f, nullptr);
  h->launches += 1;
}

// Tail of an evaluation once the flows f (FP64, before the outage correction) and the
// cost / dispatch sums are in the workspace; `dispatch` takes x from w.x64.
dcopf_status run_eval_finish(dcopf_dual* h, int B, const int* outage, const double* lambda,
                             const double* mh, const double* ml, double* value, double* glam,
                             double* ghi, double* glo, double* dispatch, cudaStream_t s) {
  const DevNet& N = h->dev;
  Workspace& w = h->ws;
  if (dispatch)
    k_dispatch<<<cdiv((long long)B * N.n_gen, 256), 256, 0, s>>>(N, B, w.x64.as<double>(), dispatch);
  k_grad_value<double, double><<<B, 256, 0, s>>>(N, outage, w.u64.as<double>(), lambda, mh, ml,
                                                 w.f.as<double>(), w.sumcost.as<double>(),
                                                 w.sump.as<double>(), w.demand.as<double>(), value,
                                                 glam, ghi, glo, nullptr);
  h->launches += 1 + (dispatch ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

template <typename S>
dcopf_status run_iters_unfused(dcopf_dual* h, int B, const int* outage, int precision,
                               const StepArgs& P, SolveState<S>& st, int n_iters, int max_iters,
                               double tol, cudaStream_t s) {
  const DevNet& N = h->dev;
  Workspace& w = h->ws;
  const int nl = N.n_line, ng = N.n_gen;
  dim3 gl(nl, B), gg(ng, B), gs(cdiv(nl, 256), B);
  const int ta = red_threads(nl), tf = red_threads(ng);
  for (int it = 0; it < n_iters; ++it) {
    if (precision == DCOPF_FP64) {
      k_eta<double, S><<<B, 256, 0, s>>>(nl, st.mu_hi, st.mu_lo, outage, w.u64.as<double>(), w.eta64.as<double>());
      k_adjoint<double><<<gg, ta, 0, s>>>(nl, ng, N.phit64, w.eta64.as<double>(), w.pit64.as<double>());
      k_minimize<double><<<B, 256, 0, s>>>(N, st.lam, w.pit64.as<double>(), w.x64.as<double>(),
                                           w.sumcost.as<double>(), w.sump.as<double>(), st.done, st.s);
      if (st.xsum) launch_accum_mean<double>(h, B, w.x64.as<double>(), st, s);
      k_forward<double><<<gl, tf, 0, s>>>(nl, ng, N.phi64, w.x64.as<double>(), w.f0.as<double>(),
                                           w.f.as<double>(), st.done);
    } else {
      k_eta<float, S><<<B, 256, 0, s>>>(nl, st.mu_hi, st.mu_lo, outage, w.u32.as<float>(), w.eta32.as<float>());
      k_adjoint<float><<<gg, ta, 0, s>>>(nl, ng, N.phit32, w.eta32.as<float>(), w.pit32.as<float>());
      k_minimize<float><<<B, 256, 0, s>>>(N, st.lam, w.pit32.as<float>(), w.x32.as<float>(),
                                          w.sumcost.as<double>(), w.sump.as<double>(), st.done, nullptr);
      if (st.xsum) launch_accum_mean<float>(h, B, w.x32.as<float>(), st, s);
      k_forward<float><<<gl, tf, 0, s>>>(nl, ng, N.phi32, w.x32.as<float>(), w.f0.as<double>(),
                                          w.f.as<double>(), st.done);
    }
    k_grad_value<S, double><<<B, 256, 0, s>>>(N, outage, w.u64.as<double>(), st.lam, st.mu_hi,
                                              st.mu_lo, w.f.as<double>(), w.sumcost.as<double>(),
                                              w.sump.as<double>(), w.demand.as<double>(),
                                              w.value.as<double>(), w.glam.as<double>(),
                                              w.ghi.as<double>(), w.glo.as<double>(), st.done);
    if (st.s && precision == DCOPF_FP64) {
      k_step_s<<<dim3(cdiv(ng, 256), B), 256, 0, s>>>(N, P, w.x64.as<double>(), st);
      h->launches += 1;
    }
    k_step<S><<<gs, 256, 0, s>>>(nl, P, w.value.as<double>(), w.glam.as<double>(),
                                 w.ghi.as<double>(), w.glo.as<double>(), st);
    k_close_iter<<<cdiv(B, 128), 128, 0, s>>>(B, max_iters, tol, st);
    h->launches += 7;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

// FP64 or FP32 evaluation with every intermediate in caller-provided buffers (same
// kernels as run_eval_unfused; nothing of the handle's workspace is used).
dcopf_status launch_eval_into(dcopf_dual* h, int B, const int* outage, const double* lambda,
                              const double* mh, const double* ml, int precision,
                              const EvalBuffers& E, double* value, double* glam, double* ghi,
                              double* glo, double* dispatch, cudaStream_t s) {
  const DevNet& N = h->dev;
  const int nl = N.n_line, ng = N.n_gen;
  dim3 gl(nl, B), gg(ng, B);
  const int ta = red_threads(nl), tf = red_threads(ng);
  if (precision == DCOPF_FP64) {
    k_eta<double, double><<<B, 256, 0, s>>>(nl, mh, ml, outage, E.u64, E.eta64);
    k_adjoint<double><<<gg, ta, 0, s>>>(nl, ng, N.phit64, E.eta64, E.pit64);
    k_minimize<double><<<B, 256, 0, s>>>(N, lambda, E.pit64, E.x64, E.sumcost, E.sump, nullptr, nullptr);
    k_forward<double><<<gl, tf, 0, s>>>(nl, ng, N.phi64, E.x64, E.f0, E.f, nullptr);
    if (dispatch) k_dispatch<<<cdiv((long long)B * ng, 256), 256, 0, s>>>(N, B, E.x64, dispatch);
  } else {
    k_to_float<<<cdiv((long long)B * nl, 256), 256, 0, s>>>((long long)B * nl, E.u64, E.u32);
    k_eta<float, double><<<B, 256, 0, s>>>(nl, mh, ml, outage, E.u32, E.eta32);
    k_adjoint<float><<<gg, ta, 0, s>>>(nl, ng, N.phit32, E.eta32, E.pit32);
    k_minimize<float><<<B, 256, 0, s>>>(N, lambda, E.pit32, E.x32, E.sumcost, E.sump, nullptr, nullptr);
    k_forward<float><<<gl, tf, 0, s>>>(nl, ng, N.phi32, E.x32, E.f0, E.f, nullptr);
    if (dispatch) k_dispatch32<<<cdiv((long long)B * ng, 256), 256, 0, s>>>(N, B, E.x32, dispatch);
    h->launches += 1;
  }
  k_grad_value<double, double><<<B, 256, 0, s>>>(N, outage, E.u64, lambda, mh, ml, E.f, E.sumcost,
                                                 E.sump, E.demand, value, glam, ghi, glo, nullptr);
  h->launches += 5 + (dispatch ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

template dcopf_status run_iters_unfused<double>(dcopf_dual*, int, const int*, int, const StepArgs&,
                                                SolveState<double>&, int, int, double, cudaStream_t);
template dcopf_status run_iters_unfused<float>(dcopf_dual*, int, const int*, int, const StepArgs&,
                                               SolveState<float>&, int, int, double, cudaStream_t);

// ---------------------------------------------------------------- instantiations
template __global__ void k_eta<double, double>(int, const double*, const double*, const int*,
                                               const double*, double*);
template __global__ void k_eta<float, double>(int, const double*, const double*, const int*,
                                              const float*, float*);
template __global__ void k_eta<float, float>(int, const float*, const float*, const int*,
                                             const float*, float*);
template __global__ void k_adjoint<double>(int, int, const double*, const double*, double*);
template __global__ void k_adjoint<float>(int, int, const float*, const float*, float*);
template __global__ void k_minimize<double>(DevNet, const double*, const double*, double*, double*,
                                            double*, const int*, const double*);
template __global__ void k_minimize<float>(DevNet, const double*, const float*, float*, double*,
                                           double*, const int*, const double*);
template __global__ void k_forward<double>(int, int, const double*, const double*, const double*,
                                           double*, const int*);
template __global__ void k_forward<float>(int, int, const float*, const float*, const double*,
                                          double*, const int*);
template __global__ void k_grad_value<double, double>(DevNet, const int*, const double*,
                                                      const double*, const double*, const double*,
                                                      double*, const double*, const double*,
                                                      const double*, double*, double*, double*,
                                                      double*, const int*);
template __global__ void k_grad_value<float, double>(DevNet, const int*, const double*,
                                                     const double*, const float*, const float*,
                                                     double*, const double*, const double*,
                                                     const double*, double*, double*, double*,
                                                     double*, const int*);
template __global__ void k_step<double>(int, StepArgs, const double*, const double*, const double*,
                                        const double*, SolveState<double>);
template __global__ void k_step<float>(int, StepArgs, const double*, const double*, const double*,
                                       const double*, SolveState<float>);

}  // namespace dcopf
