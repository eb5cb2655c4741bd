// C ABI of libdcopfdual.so: argument validation, handle and workspace management,
// and the solve driver that alternates device iterations with FP64 certification.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <vector>

#include "dcopf_dual.h"
#include "kernels.h"

using namespace dcopf;

dcopf_dual::~dcopf_dual() {
  for (auto* b : owned) delete b;
  if (d_err) cudaFree(d_err);
  if (d_bar) cudaFree(d_bar);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (tev) cudaEventDestroy(tev);
  for (cudaEvent_t e : kev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : kev2)
    if (e) cudaEventDestroy(e);
  if (tstream) cudaStreamDestroy(tstream);
  if (cstream) cudaStreamDestroy(cstream);
  if (cstream2) cudaStreamDestroy(cstream2);
  if (tstream2) cudaStreamDestroy(tstream2);
  if (fork_ev) cudaEventDestroy(fork_ev);
  if (join_ev) cudaEventDestroy(join_ev);
  if (h_pinned) cudaFreeHost(h_pinned);
}

namespace dcopf {

thread_local AllocAccount* tl_account = nullptr;

namespace {

#define CUDA_TRY(h, x)                                               \
  do {                                                               \
    cudaError_t e_ = (x);                                            \
    if (e_ != cudaSuccess) {                                         \
      (h)->last_error = cudaGetErrorString(e_);                      \
      return e_ == cudaErrorMemoryAllocation ? DCOPF_ERR_OOM : DCOPF_ERR_CUDA; \
    }                                                                \
  } while (0)

template <typename T>
dcopf_status upload(dcopf_dual* h, const std::vector<T>& v, const T** out) {
  auto* b = new DBuf();
  h->owned.push_back(b);
  CUDA_TRY(h, b->alloc(v.size() * sizeof(T)));
  if (!v.empty()) CUDA_TRY(h, cudaMemcpy(b->p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = (const T*)b->p;
  return DCOPF_OK;
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

static dcopf_status alloc_workspace(dcopf_dual* h, int B);

// A failed allocation may leave some buffers resized and one freed: the capacity is
// reset so that the next call allocates every buffer again.
dcopf_status ensure_workspace(dcopf_dual* h, int B) {
  if (B <= h->ws.cap) return DCOPF_OK;
  h->ws.cap = 0;
  const dcopf_status r = alloc_workspace(h, B);
  if (r == DCOPF_OK) h->ws.cap = B;
  else cudaGetLastError();
  return r;
}

static dcopf_status alloc_workspace(dcopf_dual* h, int B) {
  Workspace& w = h->ws;
  const size_t nl = h->dev.n_line, ng = h->dev.n_gen;
  const size_t bl = (size_t)B * nl, bg = (size_t)B * ng;
  CUDA_TRY(h, w.f0.alloc(bl * 8));
  CUDA_TRY(h, w.f0_32.alloc(bl * 4));
  CUDA_TRY(h, w.u64.alloc(bl * 8));
  CUDA_TRY(h, w.u32.alloc(bl * 4));
  CUDA_TRY(h, w.demand.alloc((size_t)B * 8));
  CUDA_TRY(h, w.eta64.alloc(bl * 8));
  CUDA_TRY(h, w.eta32.alloc(bl * 4));
  CUDA_TRY(h, w.pit64.alloc(bg * 8));
  CUDA_TRY(h, w.pit32.alloc(bg * 4));
  CUDA_TRY(h, w.x64.alloc(bg * 8));
  CUDA_TRY(h, w.x32.alloc(bg * 4));
  CUDA_TRY(h, w.f.alloc(bl * 8));
  CUDA_TRY(h, w.sumcost.alloc((size_t)B * 8));
  CUDA_TRY(h, w.sump.alloc((size_t)B * 8));
  CUDA_TRY(h, w.value.alloc((size_t)B * 8));
  CUDA_TRY(h, w.glam.alloc((size_t)B * 8));
  CUDA_TRY(h, w.ghi.alloc(bl * 8));
  CUDA_TRY(h, w.glo.alloc(bl * 8));
  return DCOPF_OK;
}

template <typename S>
dcopf_status ensure_state(dcopf_dual* h, int B, SolveState<S>* st) {
  StateBufs& sb = sizeof(S) == 8 ? h->st64 : h->st32;
  const size_t nl = h->dev.n_line;
  if (B > sb.cap) {
    sb.cap = 0;  // reset unless every buffer below is allocated
    if (sb.ints.alloc((size_t)B * 6 * sizeof(int)) != cudaSuccess ||
        sb.dbls.alloc((size_t)B * 12 * sizeof(double)) != cudaSuccess ||
        sb.mus.alloc((size_t)B * nl * 8 * sizeof(S)) != cudaSuccess) {
      cudaGetLastError();
      return DCOPF_ERR_OOM;
    }
    sb.cap = B;
  }
  int* I = sb.ints.as<int>();
  st->done = I; st->cand = I + B; st->iter = I + 2 * B; st->best_iter = I + 3 * B;
  st->status = I + 4 * B;
  double* D = sb.dbls.as<double>();
  st->best = D; st->best_next = D + B; st->best_lam = D + 2 * B; st->thresh = D + 3 * B;
  st->margin = D + 4 * B; st->prev = D + 5 * B; st->prev2 = D + 6 * B; st->lam = D + 7 * B;
  st->lam_s1 = D + 8 * B; st->lam_s2 = D + 9 * B; st->cert = D + 10 * B;
  S* M = sb.mus.as<S>();
  const size_t bl = (size_t)B * nl;
  st->mu_hi = M; st->mu_lo = M + bl; st->s1_hi = M + 2 * bl; st->s2_hi = M + 3 * bl;
  st->s1_lo = M + 4 * bl; st->s2_lo = M + 5 * bl; st->best_hi = M + 6 * bl; st->best_lo = M + 7 * bl;
  return DCOPF_OK;
}

dcopf_status ensure_mean(dcopf_dual* h, int B, SolveStateBase* st, bool f32, bool on,
                         cudaStream_t s) {
  st->xsum = nullptr;
  st->wsum = nullptr;
  if (!on) return DCOPF_OK;
  // the float state (fused, FP32 and BF16 paths) and the double state (FP64) keep
  // separate accumulators, like the rest of their state
  StateBufs& sb = f32 ? h->st32 : h->st64;
  const size_t ng = h->dev.n_gen;
  const size_t xs = ((size_t)B * ng * sizeof(float) + 255) & ~(size_t)255;
  CUDA_TRY(h, sb.avg.alloc(xs + (size_t)B * sizeof(double)));
  CUDA_TRY(h, cudaMemsetAsync(sb.avg.p, 0, xs + (size_t)B * sizeof(double), s));
  st->xsum = sb.avg.as<float>();
  st->wsum = (double*)(sb.avg.as<char>() + xs);
  return DCOPF_OK;
}

template dcopf_status ensure_state<float>(dcopf_dual*, int, SolveState<float>*);
template dcopf_status ensure_state<double>(dcopf_dual*, int, SolveState<double>*);

// ---------------------------------------------------------------- solver bookkeeping kernels
template <typename S>
__global__ void k_init_state(int B, int nl, int warm, const double* __restrict__ lam_in,
                             const double* __restrict__ mh_in, const double* __restrict__ ml_in,
                             const double* __restrict__ target, double gap, SolveState<S> st) {
  const size_t n = (size_t)B * nl;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    S h = warm ? (S)fmax(mh_in[q], 0.0) : S(0);
    S l = warm ? (S)fmax(ml_in[q], 0.0) : S(0);
    st.mu_hi[q] = h; st.mu_lo[q] = l;
    st.best_hi[q] = h; st.best_lo[q] = l;
    st.s1_hi[q] = S(0); st.s2_hi[q] = S(0); st.s1_lo[q] = S(0); st.s2_lo[q] = S(0);
  }
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    double lam = warm ? lam_in[b] : 0.0;
    st.lam[b] = lam; st.best_lam[b] = lam; st.lam_s1[b] = 0.0; st.lam_s2[b] = 0.0;
    st.best[b] = -INFINITY; st.best_next[b] = -INFINITY;
    st.iter[b] = 0; st.best_iter[b] = 0; st.done[b] = 0; st.cand[b] = 0; st.status[b] = 1;
    st.thresh[b] = target ? target[b] - gap * fabs(target[b]) : INFINITY;
    st.margin[b] = 0.0; st.prev[b] = 0.0; st.prev2[b] = 0.0; st.cert[b] = -INFINITY;
  }
}

// After certification of the candidates: accept (certified bound reaches the
// threshold), stop (cap / tol), or raise the in-loop margin and continue.
__global__ void k_accept(int B, double ub_any, SolveStateBase st, int* active, const int* err) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == 0) active[2] = *err;  // read back with the active count
  if (b >= B) return;
  if (!st.done[b] && st.cand[b]) {
    double c = st.cert[b];
    if (st.cand[b] == 1) {
      if (c >= st.thresh[b]) {
        st.done[b] = 1;
        st.status[b] = 0;
      } else {
        double short_by = st.thresh[b] - c;
        st.margin[b] += fmax(short_by, 1e-7 * fabs(st.thresh[b]));
        st.cand[b] = 0;
      }
    } else {
      st.done[b] = 1;
      st.status[b] = (c >= st.thresh[b]) ? 0 : 1;
    }
    if (c > ub_any) { st.done[b] = 1; st.status[b] = 2; }
  }
  if (!st.done[b]) atomicAdd(active, 1);
}

template <typename S>
__global__ void k_output(int B, int nl, SolveState<S> st, double* __restrict__ lam,
                         double* __restrict__ mh, double* __restrict__ ml, double* __restrict__ bound,
                         int* __restrict__ iters, int* __restrict__ status) {
  const size_t n = (size_t)B * nl;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    mh[q] = (double)st.best_hi[q];
    ml[q] = (double)st.best_lo[q];
  }
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    lam[b] = st.best_lam[b];
    if (bound) bound[b] = st.cert[b];
    if (iters) iters[b] = st.iter[b];
    if (status) status[b] = st.status[b];
  }
}

void k_init_state_f32(unsigned grid, cudaStream_t s, int B, int nl, int warm, const double* lam,
                      const double* mh, const double* ml, const double* target, double gap,
                      SolveState<float> st) {
  k_init_state<float><<<grid, 256, 0, s>>>(B, nl, warm, lam, mh, ml, target, gap, st);
}

void k_output_f32(unsigned grid, cudaStream_t s, int B, int nl, SolveState<float> st, double* lam,
                  double* mh, double* ml, double* bound, int* iters, int* status) {
  k_output<float><<<grid, 256, 0, s>>>(B, nl, st, lam, mh, ml, bound, iters, status);
}

// *out = sum of iters[0..B) (fixed order per thread, then a block tree)
__global__ void k_sum_iters(int B, const int* __restrict__ iters, int* __restrict__ out) {
  __shared__ long long sh[32];
  long long s = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) s += iters[b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = (int)s;
}

template <typename S>
dcopf_status solve_loop(dcopf_dual* h, int B, const double* loads, const int* outage,
                        const dcopf_solve_params& p, int path, double* lam, double* mh, double* ml,
                        double* bound, int* iters, int* status, cudaStream_t s) {
  SolveState<S> st{};
  dcopf_status r = ensure_state<S>(h, B, &st);
  if (r) return r;
  const int nl = h->dev.n_line;
  st.has_target = p.target_value != nullptr;
  unsigned g = std::min<unsigned>(cdiv((long long)B * nl, 256), 4096);
  k_init_state<S><<<g, 256, 0, s>>>(B, nl, p.warm_start, lam, mh, ml, p.target_value, p.gap, st);
  h->launches += 1;
  StepArgs P{};
  P.rule = p.rule;
  P.as_printed = p.as_printed;
  P.alpha = p.alpha;
  P.alpha_lambda = p.alpha_lambda > 0 ? p.alpha_lambda : p.alpha;
  P.rho = p.rho;
  P.beta1 = p.beta1;
  P.beta2 = p.beta2;
  P.eps = p.eps;
  P.decay = p.decay;
  if constexpr (sizeof(S) == 8) {
    if (p.qp_dual_s) {  // eq. (16)'s s and its moments, from s = 0
      const size_t n = (size_t)B * h->dev.n_gen;
      StateBufs& sb = h->st64;
      CUDA_TRY(h, sb.sbuf.alloc(3 * n * sizeof(double)));
      CUDA_TRY(h, cudaMemsetAsync(sb.sbuf.p, 0, 3 * n * sizeof(double), s));
      st.s = sb.sbuf.as<double>();
      st.s1_s = st.s + n;
      st.s2_s = st.s + 2 * n;
      P.qp_s = 1;
    }
  }
  CUDA_TRY(h, h->active.alloc(16));
  int* d_active = h->active.as<int>();
  // the sparse path iterates inside its kernel until a stop test fires: long rounds
  const int chunk = std::max(path == DCOPF_PATH_SPARSE ? 64 : 1, p.check_every);
  const double ub_any = h->ub_any;
  if (h->timing && !h->ev0) {
    CUDA_TRY(h, cudaEventCreate(&h->ev0));
    CUDA_TRY(h, cudaEventCreate(&h->ev1));
  }
  if constexpr (sizeof(S) == 4) {
    if (path == DCOPF_PATH_FUSED && h->fused_C == 0) {
      // Autotuner of the fused kernel's cluster shape (once per handle): every shape
      // the device keeps resident runs 40 iterations from the initial state, timed
      // with CUDA events; the fastest per iteration is kept and the state restarts.
      int Cs[9], Gs[9];
      const int n = fused_candidates(h, Cs, Gs, 9);
      if (n == 0) return DCOPF_ERR_UNSUPPORTED;
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      CUDA_TRY(h, cudaEventCreate(&e0));
      CUDA_TRY(h, cudaEventCreate(&e1));
      float best = 1e30f;
      int bi = 0;
      for (int i = 0; i < n; ++i) {
        h->fused_C = Cs[i];
        h->fused_G = Gs[i];
        float per = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          k_init_state<S><<<g, 256, 0, s>>>(B, nl, p.warm_start, lam, mh, ml, p.target_value, p.gap, st);
          h->launches += 1;
          cudaEventRecord(e0, s);
          dcopf_status rr = run_iters_fused(h, P, st, 40, 0.0, s);
          cudaEventRecord(e1, s);
          int done_iters = 0, derr = 0;
          if (rr || cudaEventSynchronize(e1) != cudaSuccess ||
              cudaMemcpy(&done_iters, st.iter, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
              cudaMemcpy(&derr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || derr) {
            if (h->verbose)
              fprintf(stderr, "[dcopf] fused tuning: cluster %d x %d CTAs failed (status %d, device %d)\n",
                      Gs[i] / Cs[i], Cs[i], (int)rr, derr);
            if (h->verbose) fused_report_refusal(h);
            cudaMemset(h->d_err, 0, sizeof(int));
            cudaGetLastError();
            if (derr == DCOPF_ERR_UNSUPPORTED && h->fused_coop != 0) {
              // the kernel refused the shape of a cooperative launch (profilers that
              // replay such launches drop the cluster shape): relaunch this candidate
              // as a plain cluster launch, whose shape they keep
              h->fused_coop = 0;
              --rep;
              continue;
            }
            per = 1e30f;
            break;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          per = std::min(per, ms / (float)std::max(1, done_iters));
        }
        if (h->verbose)
          fprintf(stderr, "[dcopf] fused tuning: cluster %d x %d CTAs: %.2f us per iteration\n",
                  Gs[i] / Cs[i], Cs[i], 1e3f * per);
        if (per < best) {
          best = per;
          bi = i;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (!(best < 1e30f)) {
        h->fused_C = 0;  // no shape ran: retune on the next fused solve
        return DCOPF_ERR_UNSUPPORTED;
      }
      h->fused_C = Cs[bi];
      h->fused_G = Gs[bi];
      k_init_state<S><<<g, 256, 0, s>>>(B, nl, p.warm_start, lam, mh, ml, p.target_value, p.gap, st);
      h->launches += 1;
    }
  }
  // the mean of the minimisers starts after any tuning runs
  if ((r = ensure_mean(h, B, &st, sizeof(S) == 4, p.mean_dispatch != nullptr, s))) return r;
  if (!h->h_pinned) CUDA_TRY(h, cudaMallocHost(&h->h_pinned, 4 * sizeof(int)));
  for (int round = 0;; ++round) {
    long long launches_before = h->launches;
    if (h->timing) CUDA_TRY(h, cudaEventRecord(h->ev0, s));
    if constexpr (sizeof(S) == 4) {
      if (path == DCOPF_PATH_FUSED) r = run_iters_fused(h, P, st, p.max_iters, p.tol, s);
    }
    if constexpr (sizeof(S) == 8) {
      if (path == DCOPF_PATH_SPARSE) r = run_iters_sparse(h, B, outage, P, st, chunk, p.max_iters, p.tol, s);
    }
    if (path != DCOPF_PATH_FUSED && path != DCOPF_PATH_SPARSE) {
      int prec = path == DCOPF_PATH_PLAIN ? DCOPF_FP64 : p.precision;
      r = run_iters_unfused<S>(h, B, outage, prec, P, st, chunk, p.max_iters, p.tol, s);
    }
    if (r) return r;
    if (h->timing) CUDA_TRY(h, cudaEventRecord(h->ev1, s));
    long long iter_launches = h->launches - launches_before;
    r = run_certify_t<S>(h, B, loads, outage, st.best_lam, st.best_hi, st.best_lo, st.cert, nullptr,
                         st.cand, st.done, s, true);
    if (r) return r;
    CUDA_TRY(h, cudaMemsetAsync(d_active, 0, sizeof(int), s));
    k_accept<<<cdiv(B, 128), 128, 0, s>>>(B, ub_any, st, d_active, h->d_err);
    // the outputs of the best points so far, written every round: when this round
    // finishes every instance (the usual case) nothing is left to do after the read
    // back (the caller's lambda / mu arrays were read only by the initialisation)
    k_output<S><<<std::min<unsigned>(cdiv((long long)B * nl, 256), 4096), 256, 0, s>>>(
        B, nl, st, lam, mh, ml, bound, iters, status);
    h->launches += 2;
    // the active count, the device error word (copied next to it by k_accept) and,
    // when timing, the evaluations so far: one copy, one synchronisation
    if (h->timing) {
      k_sum_iters<<<1, 256, 0, s>>>(B, st.iter, d_active + 1);
      h->launches += 1;
    }
    CUDA_TRY(h, cudaMemcpyAsync(h->h_pinned, d_active, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    const int active = h->h_pinned[0], derr = h->h_pinned[2];
    if (h->timing) {
      float ms = 0.f;
      CUDA_TRY(h, cudaEventElapsedTime(&ms, h->ev0, h->ev1));
      h->t_iter_ms += ms;
      h->t_iter_launches += iter_launches;
    }
    if (derr == DCOPF_ERR_UNSUPPORTED && path == DCOPF_PATH_FUSED && h->fused_coop != 0) {
      // the fused kernel refused this round's cooperative launch before touching any
      // state (its shape guard runs first): run the round again as a plain launch
      CUDA_TRY(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
      h->fused_coop = 0;
      continue;
    }
    if (derr) return (dcopf_status)derr;
    if (active == 0) break;
    if (round > 4 * (p.max_iters / chunk + 2) + 64) break;  // cannot happen unless stuck
  }
  if (p.mean_dispatch) launch_mean_out(h, B, st, p.mean_dispatch, s);
  CUDA_TRY(h, cudaGetLastError());
  if (h->timing) h->t_evals += h->h_pinned[1];
  return DCOPF_OK;
}

}  // namespace dcopf

// ==================================================================== C ABI
extern "C" {

const char* dcopf_version(void) { return "dcopfdual 0.1 (sm_103a)"; }

const char* dcopf_status_string(dcopf_status s) {
  switch (s) {
    case DCOPF_OK: return "ok";
    case DCOPF_ERR_INVALID_ARG: return "invalid argument";
    case DCOPF_ERR_NETWORK: return "invalid network (islanded, b <= 0, pmin > pmax or bridge outage)";
    case DCOPF_ERR_CUDA: return "CUDA error";
    case DCOPF_ERR_OOM: return "out of device memory";
    case DCOPF_ERR_TIMEOUT: return "bounded device wait timed out";
    case DCOPF_ERR_UNSUPPORTED: return "unsupported size or option";
  }
  return "unknown status";
}

void dcopf_solve_params_default(dcopf_solve_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->rule = DCOPF_ADAM;
  p->precision = DCOPF_FP32;
  p->path = DCOPF_PATH_AUTO;
  p->max_iters = 5000;
  p->check_every = 1;
  p->alpha = 1000.0;
  p->alpha_lambda = 0.0;
  p->rho = 0.9;
  p->beta1 = 0.9;
  p->beta2 = 0.999;
  p->eps = 1e-8;
  p->decay = 1.0;
  p->gap = 1e-3;
  p->tol = 0.0;
  p->target_value = nullptr;
}

dcopf_status dcopf_dual_create(const dcopf_network_desc* net, const dcopf_options* opt,
                               dcopf_dual_t* out) {
  if (!out) return DCOPF_ERR_INVALID_ARG;
  *out = nullptr;
  // host-side validation and setup first: invalid networks are rejected without
  // touching the GPU
  dcopf_dual* h = new dcopf_dual();
  h->verbose = opt && opt->verbose;
  {
    // DCOPF_FUSED_COOPERATIVE=0: launch the fused kernel as a plain cluster launch.
    // Co-residency then rests on the occupancy-sized grid alone (the bounded waits
    // still turn a missing cluster into DCOPF_ERR_TIMEOUT); profilers that rewrite
    // cooperative launches keep the cluster shape of a plain one.
    const char* e = getenv("DCOPF_FUSED_COOPERATIVE");
    if (e && e[0] == '0') h->fused_coop = 0;
    // DCOPF_FUSED_REFUSE=1 or 2: test hook that makes the fused kernel's shape guard
    // refuse cooperative launches (1, as profilers that rewrite such launches do) or
    // every launch (2), to exercise the fallbacks of dcopf_dual_solve_batch.
    const char* f = getenv("DCOPF_FUSED_REFUSE");
    if (f && (f[0] == '1' || f[0] == '2')) h->fused_refuse = f[0] - '0';
    // DCOPF_TENSOR_TILES=128, 256 or 192: the batched products on single CTAs only, or
    // on CTA pairs of 256 x 256 or 256 x 192 tiles only, instead of the shapes the first
    // solve of a batch size times fastest
    const char* t = getenv("DCOPF_TENSOR_TILES");
    if (t && strcmp(t, "128") == 0) h->tiles_mode = 1;
    if (t && strcmp(t, "256") == 0) h->tiles_mode = 2;
    if (t && strcmp(t, "192") == 0) h->tiles_mode = 3;
    if (t && strcmp(t, "160") == 0) h->tiles_mode = 4;
    if (t && strcmp(t, "144") == 0) h->tiles_mode = 5;
    const char* sh = getenv("DCOPF_TENSOR_SHAPE");
    int a = -1, sp = 0, fw = -1, br = 1;
    const int nf = sh ? sscanf(sh, "%d,%d,%d,%d", &a, &sp, &fw, &br) : 0;
    if (nf >= 3 && a >= 0 && a <= 8 && sp >= 1 && sp <= 64 && fw >= 0 && fw <= 8 && br >= 1 &&
        br <= 2) {
      h->shape_adj = a;
      h->shape_splits = sp;
      h->shape_fwd = fw;
      h->shape_branches = br;
    }
  }
  std::string err;
  h->sparse_only = opt && opt->operator_form == 1;
  if (opt && (opt->operator_form < 0 || opt->operator_form > 1)) { delete h; return DCOPF_ERR_INVALID_ARG; }
  dcopf_status st = build_host_net(net, &h->host, &err, h->verbose, !h->sparse_only);
  if (st != DCOPF_OK) {
    if (h->verbose) fprintf(stderr, "[dcopf] create: %s\n", err.c_str());
    delete h;
    return st;
  }
  int dev = opt && opt->device >= 0 ? opt->device : -1;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1 ||
      (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) || dev >= ndev) {
    delete h;
    return DCOPF_ERR_CUDA;
  }
  DeviceGuard guard(dev);
  h->device = dev;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) { delete h; return DCOPF_ERR_CUDA; }
  h->sm_count = prop.multiProcessorCount;
  h->smem_optin = prop.sharedMemPerBlockOptin;
  const HostNet& H = h->host;
  DevNet& D = h->dev;
  D.n_bus = H.n_bus; D.n_line = H.n_line; D.n_gen = H.n_gen; D.slack = H.slack; D.qp = H.qp;
  D.S = H.S;
  D.nr = H.F.n;
  D.n_fwd_lev = (int)H.F.fwd_level_ptr.size() - 1;
  D.n_bwd_lev = (int)H.F.bwd_level_ptr.size() - 1;
  const int nl = H.n_line, ng = H.n_gen;
  std::vector<float> fmax32(H.fmax.begin(), H.fmax.end()), fmin32(H.fmin.begin(), H.fmin.end());
  std::vector<float> sig32(H.sigma.begin(), H.sigma.end()), ctil32(H.ctil.begin(), H.ctil.end()),
      mq32(H.mq.begin(), H.mq.end()), cconst32(H.cconst.begin(), H.cconst.end()),
      mid32(H.mid.begin(), H.mid.end());
  std::vector<float> gen4(4 * (size_t)ng), gen2(2 * (size_t)ng);
  for (int j = 0; j < ng; ++j) {
    gen4[4 * j] = sig32[j]; gen4[4 * j + 1] = ctil32[j]; gen4[4 * j + 2] = mq32[j]; gen4[4 * j + 3] = cconst32[j];
    gen2[2 * j] = mid32[j];
    gen2[2 * j + 1] = mq32[j] > 0.f ? 1.0f / (2.0f * mq32[j]) : 0.f;
  }
  const size_t nphi = h->sparse_only ? 0 : (size_t)nl * ng;  // no PTDF on a sparse-only handle
  std::vector<double> phit(nphi);
  std::vector<float> phi32(nphi), phit32(nphi);
  for (int i = 0; i < nl && nphi; ++i)
    for (int j = 0; j < ng; ++j) {
      double v = H.phi[(size_t)i * ng + j];
      phit[(size_t)j * nl + i] = v;
      phi32[(size_t)i * ng + j] = (float)v;
      phit32[(size_t)j * nl + i] = (float)v;
    }
  // B_r^{-1} 1 (one FP64 solve), rounded up by a relative margin far above the solve's
  // error: bounds the price rounding of the certificate, |z - z^| <= |res|_inf B_r^{-1} 1
  std::vector<double> winv1(std::max(1, H.F.n), 1.0);
  if (H.F.n > 0) host_ldl_solve(H.F, winv1.data());
  for (double& v : winv1) v = std::fabs(v) * (1.0 + 1e-6);
  std::vector<double> inv_diag(H.F.diag.size());
  for (size_t i = 0; i < inv_diag.size(); ++i) inv_diag[i] = 1.0 / H.F.diag[i];
  // the bus incidences by elimination position (DevNet::qe_*, qo_*)
  const int nrp = std::max(1, H.F.n);
  std::vector<int> qe_line((size_t)kIncEll * nrp, -1), qe_opos((size_t)kIncEll * nrp, -1), qo_ptr(nrp + 1, 0);
  std::vector<double> qe_coef((size_t)kIncEll * nrp, 0.0), qe_b((size_t)kIncEll * nrp, 0.0);
  std::vector<int> qo_line, qo_opos;
  std::vector<double> qo_coef, qo_b;
  for (int q = 0; q < H.F.n; ++q) {
    const int bus = H.F.bus_of_pos[q];
    int a = 0;
    for (int p = H.bus_line_ptr[bus]; p < H.bus_line_ptr[bus + 1]; ++p, ++a) {
      const int l = H.bus_line_idx[p];
      const int o = H.line_from[l] == bus ? H.line_to[l] : H.line_from[l];
      const int op = H.F.pos_of_bus[o];
      if (a < kIncEll) {
        qe_line[(size_t)a * nrp + q] = l;
        qe_opos[(size_t)a * nrp + q] = op;
        qe_coef[(size_t)a * nrp + q] = H.bus_line_coef[p];
        qe_b[(size_t)a * nrp + q] = H.b[l];
      } else {
        qo_line.push_back(l);
        qo_opos.push_back(op);
        qo_coef.push_back(H.bus_line_coef[p]);
        qo_b.push_back(H.b[l]);
      }
    }
    qo_ptr[q + 1] = (int)qo_line.size();
  }
  if (qo_line.empty()) {  // keep every upload non-empty
    qo_line.push_back(0); qo_opos.push_back(-1); qo_coef.push_back(0.0); qo_b.push_back(0.0);
  }
#define UP(vec, field) \
  if ((st = upload(h, vec, &D.field)) != DCOPF_OK) { delete h; return st; }
  UP(winv1, winv1) UP(inv_diag, inv_diag)
  UP(qe_line, qe_line) UP(qe_opos, qe_opos) UP(qe_coef, qe_coef) UP(qe_b, qe_b)
  UP(qo_ptr, qo_ptr) UP(qo_line, qo_line) UP(qo_opos, qo_opos) UP(qo_coef, qo_coef) UP(qo_b, qo_b)
  UP(H.F.pos_of_bus, pos_of_bus) UP(H.F.bus_of_pos, bus_of_pos)
  UP(H.F.lrow_ptr, lrow_ptr) UP(H.F.lrow_col, lrow_col) UP(H.F.lrow_val, lrow_val)
  UP(H.F.lcol_ptr, lcol_ptr) UP(H.F.lcol_row, lcol_row) UP(H.F.lcol_val, lcol_val)
  UP(H.F.diag, diag) UP(H.F.fwd_rows, fwd_rows) UP(H.F.fwd_level_ptr, fwd_lev)
  UP(H.F.bwd_rows, bwd_rows) UP(H.F.bwd_level_ptr, bwd_lev)
  UP(H.F.fell_col, fell_col) UP(H.F.fell_val, fell_val) UP(H.F.fovf_ptr, fovf_ptr) UP(H.F.fovf_col, fovf_col)
  UP(H.F.fovf_val, fovf_val) UP(H.F.bell_col, bell_col) UP(H.F.bell_val, bell_val) UP(H.F.bovf_ptr, bovf_ptr)
  UP(H.F.bovf_col, bovf_col) UP(H.F.bovf_val, bovf_val)
  UP(H.line_from, line_from) UP(H.line_to, line_to) UP(H.b, line_b) UP(H.fmax, fmax)
  UP(H.fmin, fmin) UP(fmax32, fmax32) UP(fmin32, fmin32) UP(H.phim, phim)
  UP(H.bus_line_ptr, bus_line_ptr) UP(H.bus_line_idx, bus_line_idx)
  UP(H.bus_gen_ptr, bus_gen_ptr) UP(H.bus_gen_idx, bus_gen_idx)
  UP(H.bus_line_coef, bus_line_coef) UP(H.gen_bus, gen_bus) UP(H.pmin, pmin) UP(H.pmax, pmax)
  UP(H.cost_lin, cost_lin) UP(H.cost_quad, cost_quad) UP(H.sigma, sigma) UP(H.mid, mid)
  UP(H.ctil, ctil) UP(H.mq, mq) UP(H.cconst, cconst) UP(sig32, sigma32) UP(ctil32, ctil32)
  UP(mq32, mq32) UP(cconst32, cconst32) UP(mid32, mid32)
  {
    const float* g4 = nullptr;
    const float* g2 = nullptr;
    if ((st = upload(h, gen4, &g4)) != DCOPF_OK || (st = upload(h, gen2, &g2)) != DCOPF_OK) { delete h; return st; }
    D.gen4 = (const float4*)g4;
    D.gen2 = (const float2*)g2;
  } UP(H.phi, phi64) UP(phit, phit64) UP(phi32, phi32) UP(phit32, phit32)
#undef UP
  if (!H.F.blob.empty()) {
    if ((st = upload(h, H.F.blob, &D.fac_blob)) != DCOPF_OK) { delete h; return st; }
    D.fac_bytes = (int)H.F.blob.size();
    D.off_diag = H.F.off_diag; D.off_val = H.F.off_val; D.off_rptr = H.F.off_rptr;
    D.off_cptr = H.F.off_cptr; D.off_rcol = H.F.off_rcol; D.off_crow = H.F.off_crow;
    D.off_cmap = H.F.off_cmap; D.off_frows = H.F.off_frows; D.off_brows = H.F.off_brows;
    D.off_flev = H.F.off_flev; D.off_blev = H.F.off_blev;
  }
  if (cudaMalloc(&h->d_err, 16) != cudaSuccess || cudaMalloc(&h->d_bar, 64) != cudaSuccess ||
      cudaMemset(h->d_err, 0, 16) != cudaSuccess || cudaMemset(h->d_bar, 0, 64) != cudaSuccess) {
    delete h;
    return DCOPF_ERR_CUDA;
  }
  // an upper bound on the cost of any dispatch: a dual bound above it proves the
  // primal infeasible (Remarks 1-2 with weak duality)
  double ub = 0.0;
  for (int j = 0; j < ng; ++j) {
    auto cost = [&](double pp) {
      double sp = H.S * pp;
      return H.cost_quad[j] * sp * sp + H.cost_lin[j] * sp;
    };
    ub += std::max(cost(H.pmin[j]), cost(H.pmax[j]));
  }
  h->ub_any = ub + 1e-9 * std::fabs(ub) + 1e-9;
  if (cudaDeviceSynchronize() != cudaSuccess) { delete h; return DCOPF_ERR_CUDA; }
  *out = h;
  return DCOPF_OK;
}

dcopf_status dcopf_dual_destroy(dcopf_dual_t h) {
  if (!h) return DCOPF_OK;
  DeviceGuard guard(h->device);
  cudaDeviceSynchronize();
  delete h;
  return DCOPF_OK;
}

dcopf_status dcopf_dual_info(dcopf_dual_t h, int32_t* n_bus, int32_t* n_line, int32_t* n_gen,
                             int32_t* is_qp, uint8_t* bridge_mask) {
  if (!h) return DCOPF_ERR_INVALID_ARG;
  if (n_bus) *n_bus = h->host.n_bus;
  if (n_line) *n_line = h->host.n_line;
  if (n_gen) *n_gen = h->host.n_gen;
  if (is_qp) *is_qp = h->host.qp ? 1 : 0;
  if (bridge_mask) memcpy(bridge_mask, h->host.bridge.data(), h->host.bridge.size());
  return DCOPF_OK;
}

static dcopf_status check_batch(dcopf_dual_t h, int32_t batch, const double* loads) {
  if (!h || batch < 1 || !loads) return DCOPF_ERR_INVALID_ARG;
  if ((long long)batch * h->host.n_line > (1ll << 31)) return DCOPF_ERR_UNSUPPORTED;
  if (certify_smem(h, true) > h->smem_optin) return DCOPF_ERR_UNSUPPORTED;
  return DCOPF_OK;
}

// Outage indices arrive in device memory; they are copied back and checked on the
// host (range and bridges) before any kernel indexes arrays with them.
static dcopf_status check_outage(dcopf_dual_t h, int32_t batch, const int32_t* outage,
                                 cudaStream_t s) {
  if (!outage) return DCOPF_OK;
  std::vector<int32_t> o(batch);
  if (cudaMemcpyAsync(o.data(), outage, sizeof(int32_t) * batch, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();  // not a readable device pointer: leave no error behind
    return DCOPF_ERR_INVALID_ARG;
  }
  for (int32_t k : o) {
    if (k < -1 || k >= h->host.n_line) return DCOPF_ERR_INVALID_ARG;
    if (k >= 0 && h->host.bridge[k]) return DCOPF_ERR_NETWORK;
  }
  return DCOPF_OK;
}

static dcopf_status finish(dcopf_dual_t h, cudaStream_t s) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->last_error = cudaGetErrorString(e);
    return DCOPF_ERR_CUDA;
  }
  (void)s;
  return DCOPF_OK;
}

dcopf_status dcopf_dual_eval(dcopf_dual_t h, int32_t batch, const double* loads,
                             const int32_t* outage, const double* lambda, const double* mu_hi,
                             const double* mu_lo, int32_t precision, double* value,
                             double* g_lambda, double* g_mu_hi, double* g_mu_lo, double* dispatch,
                             void* stream) {
  dcopf_status r = check_batch(h, batch, loads);
  if (r) return r;
  if (!lambda || !mu_hi || !mu_lo || !value) return DCOPF_ERR_INVALID_ARG;
  if (precision != DCOPF_FP64 && precision != DCOPF_FP32 && precision != DCOPF_BF16X3)
    return DCOPF_ERR_INVALID_ARG;
  if (h->sparse_only) return DCOPF_ERR_UNSUPPORTED;  // the evaluation uses Phi~
  DeviceGuard guard(h->device);
  AccountScope account(&h->acct);
  cudaStream_t s = (cudaStream_t)stream;
  if ((r = check_outage(h, batch, outage, s))) return r;
  if ((r = ensure_workspace(h, batch))) return r;
  if ((r = run_base_flows(h, batch, loads, outage, s))) return r;
  if (precision == DCOPF_BF16X3)
    r = run_eval_tensor(h, batch, outage, lambda, mu_hi, mu_lo, value, g_lambda, g_mu_hi, g_mu_lo,
                        dispatch, s);
  else
    r = run_eval_unfused(h, batch, outage, lambda, mu_hi, mu_lo, precision, value, g_lambda,
                         g_mu_hi, g_mu_lo, dispatch, s);
  if (r) return r;
  return finish(h, s);
}

dcopf_status dcopf_dual_certify_bound(dcopf_dual_t h, int32_t batch, const double* loads,
                                      const int32_t* outage, const double* lambda,
                                      const double* mu_hi, const double* mu_lo, double* bound,
                                      double* err_bound, void* stream) {
  dcopf_status r = check_batch(h, batch, loads);
  if (r) return r;
  if (!lambda || !mu_hi || !mu_lo || !bound) return DCOPF_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  AccountScope account(&h->acct);
  cudaStream_t s = (cudaStream_t)stream;
  if ((r = check_outage(h, batch, outage, s))) return r;
  if ((r = run_certify_t<double>(h, batch, loads, outage, lambda, mu_hi, mu_lo, bound, err_bound,
                                 nullptr, nullptr, s)))
    return r;
  return finish(h, s);
}

dcopf_status dcopf_dual_primal_bound(dcopf_dual_t h, int32_t batch, const double* loads,
                                     const int32_t* outage, const double* lambda,
                                     const double* mu_hi, const double* mu_lo,
                                     const double* p_cand, const double* p_ref, double* upper,
                                     int32_t* pstatus, double* dispatch, double* max_violation,
                                     void* stream) {
  dcopf_status r = check_batch(h, batch, loads);
  if (r) return r;
  if (!upper || (!p_cand && (!lambda || !mu_hi || !mu_lo))) return DCOPF_ERR_INVALID_ARG;
  if (h->sparse_only) return DCOPF_ERR_UNSUPPORTED;  // the recovery's flows use Phi~
  DeviceGuard guard(h->device);
  AccountScope account(&h->acct);
  cudaStream_t s = (cudaStream_t)stream;
  if ((r = check_outage(h, batch, outage, s))) return r;
  if ((r = ensure_workspace(h, batch))) return r;
  if ((r = run_base_flows(h, batch, loads, outage, s))) return r;
  if ((r = run_primal(h, batch, outage, lambda, mu_hi, mu_lo, p_cand, p_ref, upper, pstatus,
                      dispatch, max_violation, s)))
    return r;
  return finish(h, s);
}

static dcopf_status check_params(const dcopf_solve_params& p) {
  if (p.rule < DCOPF_GDM || p.rule > DCOPF_ADAGRAD || p.max_iters < 1 || !(p.alpha > 0) ||
      !std::isfinite(p.alpha) || p.check_every < 0 || !(p.gap >= 0) || !(p.decay > 0) ||
      !(p.beta1 >= 0 && p.beta1 < 1) || !(p.beta2 >= 0 && p.beta2 < 1) || !(p.eps >= 0) ||
      p.path < DCOPF_PATH_AUTO || p.path > DCOPF_PATH_SPARSE || p.qp_dual_s < 0 || p.qp_dual_s > 1 ||
      p.screen_lines < 0 || p.screen_lines > 1)
    return DCOPF_ERR_INVALID_ARG;
  if (p.precision != DCOPF_FP64 && p.precision != DCOPF_FP32 && p.precision != DCOPF_BF16X3)
    return DCOPF_ERR_INVALID_ARG;
  return DCOPF_OK;
}

dcopf_status dcopf_dual_solve_batch(dcopf_dual_t h, int32_t batch, const double* loads,
                                    const int32_t* outage, const dcopf_solve_params* params,
                                    double* lambda, double* mu_hi, double* mu_lo,
                                    double* best_bound, int32_t* iters, int32_t* inst_status,
                                    void* stream) {
  dcopf_status r = check_batch(h, batch, loads);
  if (r) return r;
  if (!params || !lambda || !mu_hi || !mu_lo || !best_bound) return DCOPF_ERR_INVALID_ARG;
  const dcopf_solve_params& p = *params;
  if ((r = check_params(p))) return r;
  int path = p.path;
  if (path == DCOPF_PATH_AUTO)
    path = h->sparse_only ? DCOPF_PATH_SPARSE
                          : (batch == 1 && !outage) ? DCOPF_PATH_FUSED : DCOPF_PATH_BATCHED;
  if (h->sparse_only && path != DCOPF_PATH_SPARSE) return DCOPF_ERR_UNSUPPORTED;
  if (path == DCOPF_PATH_FUSED && (batch != 1 || outage)) return DCOPF_ERR_UNSUPPORTED;
  if (p.qp_dual_s && (path != DCOPF_PATH_PLAIN || !h->host.qp)) return DCOPF_ERR_UNSUPPORTED;
  int prec = p.precision;
  DeviceGuard guard(h->device);
  AccountScope account(&h->acct);
  cudaStream_t s = (cudaStream_t)stream;
  if ((r = check_outage(h, batch, outage, s))) return r;
  if ((r = ensure_workspace(h, batch))) return r;
  CUDA_TRY(h, cudaMemsetAsync(h->d_err, 0, 2 * sizeof(int), s));  // error word, re-screen flag
  if ((r = run_base_flows(h, batch, loads, outage, s))) return r;
  dcopf_solve_params q = p;
  q.precision = prec;
  if (path == DCOPF_PATH_PLAIN || path == DCOPF_PATH_SPARSE)
    return solve_loop<double>(h, batch, loads, outage, q, path, lambda, mu_hi, mu_lo, best_bound,
                              iters, inst_status, s);
  if (path == DCOPF_PATH_BATCHED && prec == DCOPF_BF16X3)
    return solve_tensor<float>(h, batch, loads, outage, q, lambda, mu_hi, mu_lo, best_bound, iters,
                               inst_status, s);
  if (path == DCOPF_PATH_FUSED && p.path == DCOPF_PATH_AUTO && h->fused_C == 0) {
    // AUTO: the fused kernel has no tuned shape yet.  If the tuner finds none that
    // runs (every shape refused), the same solve runs on the unfused FP32 kernels; the
    // tuner fails before any output is written, so a warm start is still intact.
    r = solve_loop<float>(h, batch, loads, outage, q, path, lambda, mu_hi, mu_lo, best_bound, iters,
                          inst_status, s);
    if (r != DCOPF_ERR_UNSUPPORTED || h->fused_C != 0) return r;
    if (h->verbose) fprintf(stderr, "[dcopf] no fused shape runs: unfused FP32 path\n");
    CUDA_TRY(h, cudaMemsetAsync(h->d_err, 0, sizeof(int), s));
    path = DCOPF_PATH_BATCHED;
  }
  return solve_loop<float>(h, batch, loads, outage, q, path, lambda, mu_hi, mu_lo, best_bound, iters,
                           inst_status, s);
}

dcopf_status dcopf_dual_solve_group(int32_t n_items, const dcopf_group_item* items,
                                    const dcopf_solve_params* params, void* stream) {
  if (n_items < 1 || !items || !params) return DCOPF_ERR_INVALID_ARG;
  dcopf_status r = check_params(*params);
  if (r) return r;
  if (params->precision != DCOPF_BF16X3 ||
      (params->path != DCOPF_PATH_AUTO && params->path != DCOPF_PATH_BATCHED))
    return DCOPF_ERR_UNSUPPORTED;
  std::vector<TensorItem> ti(n_items);
  for (int i = 0; i < n_items; ++i) {
    const dcopf_group_item& it = items[i];
    if ((r = check_batch(it.net, it.batch, it.loads))) return r;
    if (!it.lambda || !it.mu_hi || !it.mu_lo || !it.best_bound) return DCOPF_ERR_INVALID_ARG;
    if (it.net->sparse_only) return DCOPF_ERR_UNSUPPORTED;
    if (it.net->device != items[0].net->device) return DCOPF_ERR_INVALID_ARG;
    if (it.params) {
      if ((r = check_params(*it.params))) return r;
      if (it.params->precision != DCOPF_BF16X3 ||
          (it.params->path != DCOPF_PATH_AUTO && it.params->path != DCOPF_PATH_BATCHED))
        return DCOPF_ERR_UNSUPPORTED;
    }
    for (int j = 0; j < i; ++j)
      if (items[j].net == it.net) return DCOPF_ERR_INVALID_ARG;
    ti[i] = TensorItem{it.net,    it.params, it.batch,      it.loads, it.outage,
                       it.target_value, it.lambda, it.mu_hi, it.mu_lo, it.best_bound,
                       it.iters,  it.inst_status};
  }
  DeviceGuard guard(items[0].net->device);
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < n_items; ++i) {
    dcopf_dual* h = items[i].net;
    if ((r = check_outage(h, items[i].batch, items[i].outage, s))) return r;
    if ((r = ensure_workspace(h, items[i].batch))) return r;
    CUDA_TRY(h, cudaMemsetAsync(h->d_err, 0, 2 * sizeof(int), s));  // error word, re-screen flag
    if ((r = run_base_flows(h, items[i].batch, items[i].loads, items[i].outage, s))) return r;
  }
  return solve_tensor_group(ti.data(), n_items, *params, s);
}

int64_t dcopf_dual_kernel_launches(dcopf_dual_t h) { return h ? (int64_t)h->launches : 0; }

dcopf_status dcopf_dual_set_timing(dcopf_dual_t h, int32_t enable) {
  if (!h) return DCOPF_ERR_INVALID_ARG;
  h->timing = enable != 0;
  return DCOPF_OK;
}

dcopf_status dcopf_dual_read_timing(dcopf_dual_t h, double* iter_ms, int64_t* iter_launches,
                                    int64_t* evaluations) {
  if (!h) return DCOPF_ERR_INVALID_ARG;
  if (iter_ms) *iter_ms = h->t_iter_ms;
  if (iter_launches) *iter_launches = h->t_iter_launches;
  if (evaluations) *evaluations = h->t_evals;
  h->t_iter_ms = 0.0;
  h->t_iter_launches = 0;
  h->t_evals = 0;
  return DCOPF_OK;
}

dcopf_status dcopf_dual_screened_lines(dcopf_dual_t h, int32_t* n_kept, uint8_t* kept_mask) {
  if (!h) return DCOPF_ERR_INVALID_ARG;
  const LineScreen& S = h->scr;
  if (n_kept) *n_kept = S.ready ? S.nk : 0;
  if (kept_mask) {
    memset(kept_mask, 0, (size_t)h->host.n_line);
    if (S.ready)
      for (int l : S.kept_host) kept_mask[l] = 1;
  }
  return DCOPF_OK;
}

dcopf_status dcopf_dual_read_kernel_timing(dcopf_dual_t h, double* ms, int64_t* samples) {
  if (!h) return DCOPF_ERR_INVALID_ARG;
  if (ms)
    for (int q = 0; q < 5; ++q) ms[q] = h->t_kernel_ms[q];
  if (samples) *samples = h->t_kernel_samples;
  for (int q = 0; q < 5; ++q) h->t_kernel_ms[q] = 0.0;
  h->t_kernel_samples = 0;
  return DCOPF_OK;
}

dcopf_status dcopf_dual_tensor_shapes(dcopf_dual_t h, int32_t* shapes) {
  if (!h || !shapes) return DCOPF_ERR_INVALID_ARG;
  const int g0 = h->tune_branches > 1 ? tensor_first_group(h->tune_B) : h->tune_B;
  const int v[7] = {h->tune_B, h->tune_nl, h->tune_pair_adj, h->tune_splits, h->tune_pair_fwd,
                    h->tune_branches, g0};
  for (int q = 0; q < 7; ++q) shapes[q] = h->tune_B > 0 ? v[q] : 0;
  return DCOPF_OK;
}

dcopf_status dcopf_dual_workspace_limit(dcopf_dual_t h, int64_t limit_bytes, int64_t* used_bytes) {
  if (!h) return DCOPF_ERR_INVALID_ARG;
  if (limit_bytes >= 0) h->acct.limit = (size_t)limit_bytes;
  if (used_bytes) *used_bytes = (int64_t)h->acct.used;
  return DCOPF_OK;
}

dcopf_status dcopf_selftest_bounded_wait(dcopf_dual_t h, int64_t timeout_ns, void* stream) {
  if (!h || timeout_ns < 1000 || timeout_ns > 10000000000ll) return DCOPF_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  AccountScope account(&h->acct);
  return run_wait_selftest(h, (long long)timeout_ns, (cudaStream_t)stream);
}

dcopf_status dcopf_selftest_fused_timeout(dcopf_dual_t h, const double* loads, int64_t timeout_ns,
                                          void* stream) {
  if (!h || !loads || timeout_ns < 1000 || timeout_ns > 10000000000ll) return DCOPF_ERR_INVALID_ARG;
  if (h->sparse_only || h->fused_C == 0) return DCOPF_ERR_UNSUPPORTED;
  DeviceGuard guard(h->device);
  AccountScope account(&h->acct);
  const size_t nl = h->dev.n_line;
  CUDA_TRY(h, h->probe.alloc((2 * nl + 2) * sizeof(double) + 2 * sizeof(int)));
  double* lam = h->probe.as<double>();
  double* mh = lam + 1;
  double* ml = mh + nl;
  double* bound = ml + nl;
  int* it = (int*)(bound + 1);
  dcopf_solve_params p;
  dcopf_solve_params_default(&p);
  p.path = DCOPF_PATH_FUSED;
  p.max_iters = 10;
  h->fused_timeout_ns = (unsigned long long)timeout_ns;
  h->fused_arrive_extra = 1;
  const dcopf_status r = dcopf_dual_solve_batch(h, 1, loads, nullptr, &p, lam, mh, ml, bound, it,
                                                it + 1, stream);
  h->fused_timeout_ns = 2000000000ull;
  h->fused_arrive_extra = 0;
  return r;
}

dcopf_status dcopf_dual_device_error(dcopf_dual_t h) {
  if (!h) return DCOPF_ERR_INVALID_ARG;
  DeviceGuard guard(h->device);
  int e = 0;
  if (cudaMemcpy(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  return (dcopf_status)e;
}

}  // extern "C"
