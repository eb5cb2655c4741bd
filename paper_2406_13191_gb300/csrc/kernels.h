// Library handle, workspaces and the host-side drivers of each execution path.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "dev.cuh"
#include "internal.h"

namespace dcopf {

struct StepArgs {
  int rule, as_printed;
  int qp_s;         // 1 = eq. (16) with s as an ascent variable (plain path)
  double alpha, alpha_lambda, rho, beta1, beta2, eps, decay;
  double bc1, bc2;  // Adam bias corrections of the current step (set per step)
};

// One projected step of the chosen rule on one coordinate (Section 3.3):
//   GDM  (Algorithm 1, heavy ball): s1 <- rho s1 + a g;  theta <- theta + s1
//        (as printed: additionally theta <- theta + a g)
//   Adam: s1 <- b1 s1 + (1-b1) g; s2 <- b2 s2 + (1-b2) g^2;
//         theta <- theta + a (s1/c1) / (sqrt(s2/c2) + eps), c = 1 - beta^t
//   AdaGrad: s1 <- s1 + g^2; theta <- theta + a g / (sqrt(s1) + eps)
template <typename S>
__device__ __forceinline__ S rule_step(const StepArgs& P, S theta, S g, S& s1, S& s2, S a) {
  if (P.rule == DCOPF_GDM) {
    s1 = S(P.rho) * s1 + a * g;
    theta += s1;
    if (P.as_printed) theta += a * g;
  } else if (P.rule == DCOPF_ADAM) {
    s1 = S(P.beta1) * s1 + (S(1) - S(P.beta1)) * g;
    s2 = S(P.beta2) * s2 + (S(1) - S(P.beta2)) * g * g;
    theta += a * (s1 / S(P.bc1)) / (sqrt(s2 / S(P.bc2)) + S(P.eps));
  } else {
    s1 += g * g;
    theta += a * g / (sqrt(s1) + S(P.eps));
  }
  return theta;
}


// Per-instance solver bookkeeping (device pointers, [batch] each).
struct SolveStateBase {
  // eq. (16)'s s [batch][n_gen] and its two moments (plain FP64 path; null = closed form)
  double* s = nullptr;
  double* s1_s = nullptr;
  double* s2_s = nullptr;
  int* done;       // 1 once the instance has stopped
  int* cand;       // 1 = in-loop value reached the target (certify), 2 = stop (cap / tol)
  int* iter;       // evaluations so far
  int* best_iter;  // evaluation index of the best point
  int* status;     // per-instance result code
  double* best;    // best in-loop value
  double* best_next;
  double* best_lam;
  double* thresh;  // target - gap |target|
  double* margin;  // extra in-loop margin before certifying
  double* prev;
  double* prev2;
  double* lam;
  double* lam_s1;
  double* lam_s2;
  double* cert;    // certified bound of the best point
  int has_target;
  // mean of the minimisers (NULL = off): sum_k k^2 x_k [batch][n_gen] and sum_k k^2
  float* xsum = nullptr;
  double* wsum = nullptr;
};

template <typename S>
struct SolveState : SolveStateBase {
  S* mu_hi; S* mu_lo;      // [batch][n_line]
  S* s1_hi; S* s2_hi; S* s1_lo; S* s2_lo;
  S* best_hi; S* best_lo;
};

// Device-memory account of one handle's workspaces: the bytes its buffers hold and an
// optional limit (0 = none).  A handle's entry points make its account the calling
// thread's current one (AccountScope); buffers allocated under it are charged to it.
struct AllocAccount {
  size_t used = 0, limit = 0;
};
extern thread_local AllocAccount* tl_account;
struct AccountScope {
  AllocAccount* prev;
  explicit AccountScope(AllocAccount* a) : prev(tl_account) { tl_account = a; }
  ~AccountScope() { tl_account = prev; }
  AccountScope(const AccountScope&) = delete;
  AccountScope& operator=(const AccountScope&) = delete;
};

// Device buffer that frees itself.  Growing it under an account whose limit it would
// exceed fails with cudaErrorMemoryAllocation before anything is freed, so the
// buffer keeps its old size and contents.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  AllocAccount* acct = nullptr;  // the account its bytes are charged to, if any
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    if (acct) acct->used -= bytes;
    p = nullptr;
    bytes = 0;
    acct = nullptr;
  }
  cudaError_t alloc(size_t n) {
    if (n <= bytes && p) return cudaSuccess;
    AllocAccount* a = tl_account;
    if (a && a->limit && a->used - (acct == a ? bytes : 0) + n > a->limit)
      return cudaErrorMemoryAllocation;
    release();
    cudaError_t e = cudaMalloc(&p, n ? n : 16);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = n;
    if (a) {
      a->used += n;
      acct = a;
    }
    return e;
  }
  template <typename T> T* as() const { return (T*)p; }
};

struct Workspace {
  int cap = 0;  // batch capacity
  DBuf f0, f0_32, u64, u32, demand;
  DBuf eta64, eta32, pit64, pit32, x64, x32, f, sumcost, sump, value, glam, ghi, glo;
  DBuf misc;  // small per-batch scratch
  // B_r^-1 (e_from - e_to) of each instance's outaged line [batch][nr], left by the base
  // flows for the certificates of the same solve (valid for wcache_B, wcache_outage)
  DBuf wcache;
  int wcache_B = 0;
  const int* wcache_outage = nullptr;
};

// BF16 hi/lo operands and TMA descriptors of the tensor-core path.
struct TensorOps {
  bool ready = false;
  int ld_l = 0, ld_g = 0;  // padded row strides (elements) of [*][n_line] and [*][n_gen]
  int cap = 0;             // batch capacity of the per-batch operands
  DBuf phi_hi, phi_lo, phit_hi, phit_lo;
  CUtensorMap m_phi_hi, m_phi_lo, m_phit_hi, m_phit_lo;        // 128-row boxes
  CUtensorMap m_phi_hi96, m_phi_lo96, m_phit_hi96, m_phit_lo96;  // 96-row boxes (pair tiles of 192)
  CUtensorMap m_phi_hi80, m_phi_lo80, m_phit_hi80, m_phit_lo80;  // 80-row boxes (pair tiles of 160)
  CUtensorMap m_phi_hi72, m_phi_lo72, m_phit_hi72, m_phit_lo72;  // 72-row boxes (pair tiles of 144)
  DBuf H_hi, H_lo, X_hi, X_lo, P;
  CUtensorMap m_H_hi, m_H_lo, m_X_hi, m_X_lo;
};

// Constraint screening of the batched solve (k_screen.cu): the lines kept for the
// iterations and their compact operands, and the knapsack bounds of every line for a
// range of the balance right-hand side.
struct LineScreen {
  DBuf env, knap, keep;          // batch envelope [2][n_line] + range [2]; bounds [2][n_line]; flags
  DBuf rng;                      // balance range the knapsack bounds hold for [2], valid flag
  DBuf flags;                    // [0]: the knapsack bounds are taken again for this batch
  bool ready = false;            // the compact operands below match kept_host
  // the next screen builds the batch's own kept set (synchronously) rather than going
  // ahead with the current one: set after a solve found that its batch needs a line the
  // current set screens out
  bool exact = false;
  int nk = 0, ld_lk = 0;         // kept lines (a multiple of 8) and their row stride
  std::vector<int> kept_host;
  DBuf kept, pos;                // [nk] line of each compact row; [n_line] compact row or -1
  DBuf phi_hi, phi_lo, phit_hi, phit_lo, lim;  // compact BF16 operands; fmax, fmin [2][nk]
  CUtensorMap m_phi_hi, m_phi_lo, m_phit_hi, m_phit_lo;
  CUtensorMap m_phi_hi96, m_phi_lo96, m_phit_hi96, m_phit_lo96;
  CUtensorMap m_phi_hi80, m_phi_lo80, m_phit_hi80, m_phit_lo80;
  CUtensorMap m_phi_hi72, m_phi_lo72, m_phit_hi72, m_phit_lo72;
  int map_B = 0;                 // batch size of the maps below
  CUtensorMap m_H_hi, m_H_lo;    // the adjoint's A operand [B][ld_lk]
  DBuf f0c, full;                // compact base flows [B][nk]; full-length best point [2][B][n_line]
};

// Extra per-instance state of the batched tensor-core solve (device pointers).
struct BatchView {
  int n_tiles = 0;             // slices of lines of the step kernel
  int* frozen = nullptr;       // [B] done or waiting for certification
  int* pend = nullptr;         // [B] value partials of the evaluated point not yet finalised
  float* ueta = nullptr;       // [B] u^T eta of the point stepped to (outaged line's term)
  double* lam_eval = nullptr;  // [B] lambda of the evaluated point
  double* cost = nullptr;      // [B] generation cost at the minimiser
  double* psum = nullptr;      // [B] total dispatch
  double* pw = nullptr;        // [B][3] decay^t, beta1^t, beta2^t
  float* tout = nullptr;       // [B] pre-outage flow on the outaged line
  float* stepf = nullptr;      // [B][4] step factors of the current step
  float* mu2_hi = nullptr;     // [B][nl] second state buffer (iteration index % 3 == 1)
  float* mu2_lo = nullptr;
  float* mu3_hi = nullptr;     // [B][nl] third state buffer (index % 3 == 2)
  float* mu3_lo = nullptr;
  float* sv_hi = nullptr;      // [B][nl] the best point, saved when its buffer is reused
  float* sv_lo = nullptr;
  double* lam_best = nullptr;  // [B] lambda of the best point
  double* line_part = nullptr; // [B][n_tiles] per slice of lines of the step kernel
  double* out_part = nullptr;  // [B][n_tiles]
};

// Objects a batched solve reuses from call to call (kept by the first network's handle):
// the round loop's events and host-mapped read-back, and the iteration graph of the
// last solve with the bytes of the kernel arguments it was captured with.
struct RoundKit {
  int n = 0;  // networks the events and the read-back are made for
  std::vector<cudaEvent_t> ev, stage_ev, cert_ev;
  // per round parity [2][4n]: each network's running count, device error word,
  // re-screen flag and count of instances iterating (not frozen), written by its accept
  // kernel on the device and copied to pinned host memory on the read-back stream, off
  // the iterations' critical path
  int* rb_dev = nullptr;
  int* pin = nullptr;
  cudaStream_t rs = nullptr;
  cudaEvent_t acc[2] = {nullptr, nullptr};   // a round's accept kernels have run
  cudaEvent_t done[2] = {nullptr, nullptr};  // a round's read-back has landed
  cudaEvent_t t0[2] = {nullptr, nullptr}, t1[2] = {nullptr, nullptr};  // around a round's graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> sig;
  // the graph's per-kernel timing nodes: (node, network, event index)
  struct KNode {
    cudaGraphNode_t node;
    int net, q;
  };
  std::vector<KNode> knodes;
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    sig.clear();
    knodes.clear();
  }
  void release() {
    drop_graph();
    for (auto* v : {&ev, &stage_ev, &cert_ev})
      for (cudaEvent_t e : *v)
        if (e) cudaEventDestroy(e);
    ev.clear(); stage_ev.clear(); cert_ev.clear();
    for (cudaEvent_t* e : {&acc[0], &acc[1], &done[0], &done[1], &t0[0], &t0[1], &t1[0], &t1[1]}) {
      if (*e) cudaEventDestroy(*e);
      *e = nullptr;
    }
    if (rs) cudaStreamDestroy(rs);
    if (pin) cudaFreeHost(pin);
    if (rb_dev) cudaFree(rb_dev);
    rs = nullptr;
    pin = rb_dev = nullptr;
    n = 0;
  }
  ~RoundKit() { release(); }
};

struct BatchBufs {
  DBuf mu2, parts, small, F;
  DBuf snap;  // [B] instances staged for the certificate in flight
  BatchView v;
};

// Workspace of the primal recovery (dcopf_dual_primal_bound).
struct PrimalBufs {
  int cap = 0;
  DBuf xr, xu, fr, t, st;  // reference and repaired x [B][n_gen]; reference flows; t; status
};

struct StateBufs {
  int cap = 0;
  int elem = 0;  // sizeof(S) of the arrays below
  DBuf ints, dbls, mus;
  DBuf avg;      // xsum and wsum of the mean of the minimisers
  DBuf sbuf;     // eq. (16)'s s and its moments [3][batch][n_gen] (FP64 state only)
};

}  // namespace dcopf

struct dcopf_dual {
  // first member: outlives every buffer charged to it
  dcopf::AllocAccount acct;
  int device = 0;
  dcopf::HostNet host;
  dcopf::DevNet dev{};
  std::vector<dcopf::DBuf*> owned;  // network arrays
  dcopf::Workspace ws;
  dcopf::StateBufs st32, st64;
  dcopf::TensorOps tops;
  dcopf::DBuf dense_ha, dense_part;  // dense FP64 PTDF [n_line][n_bus] (built on first use)
  dcopf::DBuf dense_colabs;           // [n_bus] column sums of |H_a| (price rounding bound)
  dcopf::BatchBufs bb;
  dcopf::LineScreen scr;
  dcopf::PrimalBufs pb;
  int* d_err = nullptr;  // sticky device error word
  unsigned* d_bar = nullptr;  // grid-barrier counters
  dcopf::DBuf active;  // one int: instances still running
  int* h_pinned = nullptr;  // pinned host mirror of a round's read-back: [0] active count,
                            // [1] evaluations (timing), [2] device error word
  double ub_any = 0.0;  // cost of the dearest dispatch (upper bound on any primal cost)
  cudaStream_t tstream = nullptr;  // internal stream of the graph-captured batched solve
  // certificates of the batched solve, beside its iterations: one stream per round
  // parity, so that a round's certificates need not wait for the previous round's
  cudaStream_t cstream = nullptr, cstream2 = nullptr;
  // second branch of the batched solve's iteration graph (its second group of
  // instances), forked from tstream and joined back to it once per round
  cudaStream_t tstream2 = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  cudaEvent_t tev = nullptr;  // orders the internal stream after the caller's
  dcopf::RoundKit kit;         // round-loop objects and the cached iteration graph
  long long launches = 0;
  // optional event timing of the iteration kernels
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double t_iter_ms = 0.0;
  long long t_iter_launches = 0, t_evals = 0;
  // per-kernel timing of the batched solve (timing on): events around the adjoint,
  // minimiser, forward, step and value kernels of the last iteration of every round,
  // recorded inside the iteration graph
  cudaEvent_t kev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t kev2[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // odd rounds
  double t_kernel_ms[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  long long t_kernel_samples = 0;
  int sm_count = 0;
  int fused_C = 0, fused_G = 0;  // cluster shape of the fused kernel (chosen on first use)
  // layout of that shape, validated once (occupancy queries cost host time per solve)
  int fshape_C = 0, fshape_G = 0, fshape_phi = 0, fshape_rpc = 0, fshape_slice = 0;
  size_t fshape_smem = 0;
  bool sparse_only = false;      // created with operator_form 1: no Phi~ on the device
  int fused_coop = -1;           // -1 unknown, 1 cooperative+cluster launch accepted, 0 not
  // host-side refusal injection (DCOPF_FUSED_REFUSE, read at create): 1 sizes every
  // cooperative fused launch for another cluster shape, 2 every fused launch, so that
  // the kernel's shape guard refuses it (no device fault: the kernel returns a status)
  int fused_refuse = 0;
  // limit of the fused kernel's bounded waits, and extra arrivals its inter-cluster
  // wait expects (nonzero only inside dcopf_selftest_fused_timeout: a count that no
  // cluster reaches, so that the wait gives up)
  unsigned long long fused_timeout_ns = 2000000000ull;
  unsigned fused_arrive_extra = 0;
  dcopf::DBuf probe;  // outputs of the fused self-test
  // split-K of the batched adjoint GEMM chosen by timing (for batch size tune_B), and
  // whether the adjoint and the forward product run on CTA pairs (256 x 256 tiles)
  // rather than single CTAs (128 x 128)
  int tune_B = 0, tune_nl = 0, tune_splits = 0, tune_kbps = 0;
  int tune_pair_adj = 0, tune_pair_fwd = 0;  // 0 single CTAs; pairs of 1: 256 columns, 2: 192, 3: 160, 4: 144
  // instance groups iterated as parallel branches of the iteration graph (1 or 2); the
  // product shapes above are those of one group's batch
  int tune_branches = 1;
  // DCOPF_TENSOR_TILES (read at create): 0 = choose by timing, 1 = single CTAs only,
  // 2 / 3 / 4 / 5 = CTA pairs of 256 x 256 / 256 x 192 / 256 x 160 / 256 x 144 tiles
  // only (where the batch has more than 128 instances)
  int tiles_mode = 0;
  // DCOPF_TENSOR_SHAPE="a,s,f[,g]" (read at create): the adjoint's tiles (0 single, 1
  // pairs of 256, 2 pairs of 192, 3 pairs of 160, 4 pairs of 144), its split-K factor, the forward's tiles, the branches
  // (default 1); no timing (for profilers, whose per-launch overhead changes what the
  // timing would pick)
  int shape_adj = -1, shape_splits = 0, shape_fwd = -1, shape_branches = 1;
  size_t smem_optin = 0;
  bool verbose = false;
  std::string last_error;
  ~dcopf_dual();
};

namespace dcopf {

// Upload helpers and workspace management (api.cu).
dcopf_status ensure_workspace(dcopf_dual* h, int batch);
template <typename S>
dcopf_status ensure_state(dcopf_dual* h, int batch, SolveState<S>* st);

void k_init_state_f32(unsigned grid, cudaStream_t s, int B, int nl, int warm, const double* lam,
                      const double* mh, const double* ml, const double* target, double gap,
                      SolveState<float> st);
void k_output_f32(unsigned grid, cudaStream_t s, int B, int nl, SolveState<float> st, double* lam,
                  double* mh, double* ml, double* bound, int* iters, int* status);

// k_sparse.cu
dcopf_status run_base_flows(dcopf_dual* h, int batch, const double* loads, const int* outage,
                            cudaStream_t s);
// The mean of the minimisers over a solve (dcopf_solve_params.mean_dispatch): zeroed
// accumulators attached to st when `on`, detached otherwise; and the output
// p = mid + sigma (xsum / wsum) into out [B][n_gen].
dcopf_status ensure_mean(dcopf_dual* h, int B, SolveStateBase* st, bool f32, bool on,
                         cudaStream_t s);
void launch_mean_out(dcopf_dual* h, int B, const SolveStateBase& st, double* out, cudaStream_t s);
template <typename T>
void launch_accum_mean(dcopf_dual* h, int B, const T* x, const SolveStateBase& st, cudaStream_t s);
dcopf_status run_iters_sparse(dcopf_dual* h, int B, const int* outage, const StepArgs& P,
                              SolveState<double>& st, int n_iters, int max_iters, double tol,
                              cudaStream_t s);
dcopf_status run_primal(dcopf_dual* h, int B, const int* outage, const double* lambda,
                        const double* mh, const double* ml, const double* p_cand,
                        const double* p_ref, double* upper, int* pstatus, double* dispatch,
                        double* maxviol, cudaStream_t s);
// FP64 per-phase building blocks of k_phases.cu for other files: eta and the adjoint
// pi~ = Phi~^T eta into the workspace (eta64, pit64); and f = Phi~ x + f0.
void launch_adjoint64(dcopf_dual* h, int B, const int* outage, const double* mh,
                      const double* ml, cudaStream_t s);
void launch_forward64(dcopf_dual* h, int B, const double* x, const double* f0, double* f,
                      cudaStream_t s);
template <typename S>
dcopf_status run_certify_t(dcopf_dual* h, int batch, const double* loads, const int* outage,
                           const double* lam, const S* mh, const S* ml, double* bound, double* errb,
                           const int* mask, const int* done, cudaStream_t s,
                           bool use_wcache = false);
size_t certify_smem(const dcopf_dual* h, bool outages);

// Intermediate buffers of one evaluation, all caller-provided ([batch][n] arrays).
struct EvalBuffers {
  double *f0, *u64, *demand, *eta64, *pit64, *x64, *f, *sumcost, *sump;
  float *u32, *eta32, *pit32, *x32;
};
dcopf_status launch_base_flows_into(dcopf_dual* h, int B, const double* loads, const int* outage,
                                    double* f0, double* u64, double* demand, cudaStream_t s);
dcopf_status launch_eval_into(dcopf_dual* h, int B, const int* outage, const double* lambda,
                              const double* mh, const double* ml, int precision,
                              const EvalBuffers& E, double* value, double* glam, double* ghi,
                              double* glo, double* dispatch, cudaStream_t s);

// k_phases.cu
dcopf_status run_eval_unfused(dcopf_dual* h, int batch, const int* outage, const double* lambda,
                              const double* mh, const double* ml, int precision, double* value,
                              double* glam, double* ghi, double* glo, double* dispatch,
                              cudaStream_t s);
dcopf_status run_eval_finish(dcopf_dual* h, int batch, const int* outage, const double* lambda,
                             const double* mh, const double* ml, double* value, double* glam,
                             double* ghi, double* glo, double* dispatch, cudaStream_t s);
template <typename S>
dcopf_status run_iters_unfused(dcopf_dual* h, int batch, const int* outage, int precision,
                               const StepArgs& P, SolveState<S>& st, int n_iters, int max_iters,
                               double tol, cudaStream_t s);

// k_dense.cu
bool dense_path_applies(const dcopf_dual* h, int batch, const int* outage);
dcopf_status run_dense_base_flows(dcopf_dual* h, int batch, const double* loads, cudaStream_t s);
template <typename S>
dcopf_status run_dense_certify(dcopf_dual* h, int batch, const double* loads, const double* lam,
                               const S* mh, const S* ml, double* bound, double* errb,
                               const int* mask, const int* done, cudaStream_t s);

// k_tensor.cu
dcopf_status ensure_tensor_operands(dcopf_dual* h);
dcopf_status ensure_tensor_batch(dcopf_dual* h, int batch);
template <typename S>
dcopf_status solve_tensor(dcopf_dual* h, int batch, const double* loads, const int* outage,
                          const dcopf_solve_params& p, double* lam, double* mh, double* ml,
                          double* bound, int* iters, int* status, cudaStream_t s);
// tcgen05 GEMM with BF16 hi/lo split operands for other users (k_tensor.cu): tensor
// maps of row-major BF16 [rows][ld] with cols valid columns (K-major operands), and
// split-K partial products C = A B^T.
bool tc_make_map(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint64_t ld);
bool tc_make_map_rows(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint64_t ld,
                      uint32_t box_rows);
// A 4-D map over a rows x K BF16 matrix held in 8-row blocks of 64-column K blocks
// (element (r, c) at ((r / 8 * KB + c / 64) * 8 + r % 8) * 64 + c % 64, KB = ceil(K / 64)):
// dims {64, 8, KB, ceil(rows / 8)}, box {64, 8, 1, box_rows / 8}, 128-byte swizzle.
bool tc_make_map_blocked(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t K, uint32_t box_rows);
__host__ __device__ inline size_t blk_index(int r, int c, int kb) {
  return ((size_t)(r >> 3) * kb + (c >> 6)) * 512 + (size_t)(r & 7) * 64 + (c & 63);
}
// Constraint screening of a batch (k_screen.cu): base flows in ws.f0, demands in
// ws.demand; leaves h->scr ready with the kept lines and their compact operands.
dcopf_status screen_batch(dcopf_dual* h, int B, cudaStream_t s);
__global__ void k_screen_compact_rows(int B, int nl, int nk, const int* kept, const float* src, float* dst);
cudaError_t tc_gemm_partial(const CUtensorMap& Ah, const CUtensorMap& Al, const CUtensorMap& Bh,
                            const CUtensorMap& Bl, int M, int N, int K, float* P, int ldp,
                            int max_splits, int sm_count, int* err, int* splits_used,
                            cudaStream_t s);
cudaError_t tc_gemm_prepare();

// One network's instances in a group of batched solves (dcopf_dual_solve_group).
struct TensorItem {
  dcopf_dual* h;
  const dcopf_solve_params* p;  // this network's settings (nullptr: the group's)
  int B;
  const double* loads;
  const int* outage;
  const double* target;
  double *lam, *mh, *ml, *bound;
  int *iters, *status;
};
dcopf_status solve_tensor_group(const TensorItem* items, int n, const dcopf_solve_params& p,
                                cudaStream_t s);
// Instances in the first of the two groups a batch of B splits into.
int tensor_first_group(int B);
dcopf_status run_eval_tensor(dcopf_dual* h, int batch, const int* outage, const double* lambda,
                             const double* mh, const double* ml, double* value, double* glam,
                             double* ghi, double* glo, double* dispatch, cudaStream_t s);

// k_fused.cu
dcopf_status run_wait_selftest(dcopf_dual* h, long long timeout_ns, cudaStream_t s);
int fused_candidates(dcopf_dual* h, int* Cs, int* Gs, int cap);
void fused_report_refusal(dcopf_dual* h);
dcopf_status run_iters_fused(dcopf_dual* h, const StepArgs& P, SolveState<float>& st, int max_iters,
                             double tol, cudaStream_t s);

}  // namespace dcopf
