// Fused persistent solve of one instance: every iteration of the projected dual
// ascent (Section 3.3, Algorithm 1 and the Adam / AdaGrad rules) runs inside one
// kernel whose CTAs (one per SM) form thread-block clusters of C CTAs.
//
// Data placement: CTA c owns a contiguous block of lines (rows of Phi~), keeps those
// rows (FP32) in shared memory for the whole solve, and owns the dual state of its
// lines (mu_hi, mu_lo, optimiser moments).  lambda and its moments are replicated in
// every CTA and updated identically (same inputs, same order).
//
// Iteration k (all CTAs):
//   A   eta = mu_hi - mu_lo on own rows; partial adjoint Phi~_c^T eta_c for all gens,
//       each stored into the shared memory of the rank owning the gen's slice
//                                                             (eq. (6): C^T mu)
//   A2  [partials arrived] CTA r of a cluster sums its gens slice S_r over the
//       cluster's partials and publishes them -> Pc[j][cluster]
//   B   every cluster reads Pc for its slices and the line partials R of the previous
//       evaluation, sums the clusters in a fixed order, takes the closed-form
//       minimiser x*_j (eq. (6) / eq. (16)), stored into every rank of the
//       cluster, and partial cost / dispatch sums; the previous evaluation's dual
//       value -> best point, stop tests
//   C   [x* arrived] forward
//       f = Phi~_c x* + f0 on own rows (constraint (1c)); supergradient; FP64 line
//       partial -> R[c]; projected step of own mu and of lambda.
//
// Synchronisation between clusters: after publishing its slice, each CTA increments
// the arrival counter of its cluster rank with a release-add (which makes the CTA's
// writes visible); a CTA then waits, with acquire loads, until all C counters show
// every cluster's arrival for this loop, and
// reads the slice's partials (and the line partials R of the previous loop, written
// before the writer's arrival) from L2.  Pc and R are double-buffered by loop parity:
// a CTA can run at most one loop ahead of the slowest one, so a buffer is rewritten
// only after all its readers are done.
//
// Exchanges inside a cluster: asynchronous stores into the peers' shared memory
// (st.async), each counted on the receiving CTA's transaction barrier (an mbarrier
// whose phase completes when its own arrival and every expected byte are in); no
// cluster-wide barrier per loop.  Write-after-read safety of the receive buffers
// follows from the data dependencies: a peer stores loop k+1's partials only after it
// received this CTA's x* of loop k (sent after this CTA consumed loop k's partials),
// and loop k+1's x* only after it received this CTA's loop k+1 partials (sent after
// this CTA's forward of loop k read x*).
//
// Every wait is bounded.  Wait flags travel with x*, so a wait that gives up stops
// every CTA of the cluster at the same loop, or (when a CTA's own x* wait gives up)
// makes its peers' next waits give up; a final cluster barrier keeps every CTA's
// shared memory alive until no peer can store into it.
// Every cluster computes the same x* and the same dual value from the same data in
// the same order, so stop decisions are identical everywhere.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>

#include "dev.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace cg = cooperative_groups;

namespace dcopf {

struct FusedArgs {
  DevNet N;
  StepArgs P;
  SolveState<float> st;
  const float* f0;               // [n_line]
  const double* demand;          // [1] total demand of the instance (device)
  float* Pc;                     // [2][n_gen][NCLp] cluster partial adjoints
  double* R;                     // [2][G] line partials of the dual value
  unsigned* cnt;                 // [8] arrival counters, one per cluster rank; [16..19] the
                                 // shape a refused launch saw; [20..23] the first wait
                                 // that gave up
  int* err;
  double pscale, pinv;           // fixed-point scale of the dispatch sum and its inverse
  int max_iters;
  double tol;
  int rows_per_cta;
  int slice;                     // gens per cluster rank
  int phi_in_smem;
  int C, G;                      // launch shape the shared-memory layout was sized for
  unsigned smem_bytes;           // dynamic shared memory the layout needs
  uint64_t timeout_ns;
  unsigned arrive_extra;         // added to the inter-cluster arrival target (self-test)
};

// The ascent rule's constants in FP32, converted once per launch (FP64 conversions and
// arithmetic are slow on this part and every thread steps its lines each loop).
struct RuleF {
  int rule, as_printed;
  float rho, beta1, beta2, omb1, omb2, eps;
};
__device__ __forceinline__ RuleF rule_f(const StepArgs& P) {
  return RuleF{P.rule,           P.as_printed,           (float)P.rho,
               (float)P.beta1,   (float)P.beta2,         1.0f - (float)P.beta1,
               1.0f - (float)P.beta2, (float)P.eps};
}
__device__ __forceinline__ float fused_rule_f(const RuleF& R, float theta, float g, float& s1,
                                              float& s2, float a, float bc1, float bc2) {
  if (R.rule == DCOPF_GDM) {
    s1 = R.rho * s1 + a * g;
    theta += s1;
    if (R.as_printed) theta += a * g;
  } else if (R.rule == DCOPF_ADAM) {
    s1 = R.beta1 * s1 + R.omb1 * g;
    s2 = R.beta2 * s2 + R.omb2 * g * g;
    // bc1, bc2 are the reciprocals of the bias corrections 1 - beta^t (one division
    // fewer on the critical path of every line step)
    theta += (a * bc1) * s1 / (sqrtf(s2 * bc2) + R.eps);
  } else {
    s1 += g * g;
    theta += a * g / (sqrtf(s1) + R.eps);
  }
  return theta;
}


__global__ void __launch_bounds__(256, 1) k_fused_solve(FusedArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const DevNet& N = A.N;
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  // The layout below was sized on the host for (A.C, A.G); refuse any other shape.
  {
    unsigned dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    if (C != A.C || G != A.G || dyn < A.smem_bytes || C > 8 || G > (int)blockDim.x) {
      if (tid == 0) atomicExch(A.err, (int)DCOPF_ERR_UNSUPPORTED);
      if (tid == 0 && c == 0) {  // the shape this launch saw, for the host's diagnostics
        A.cnt[16] = (unsigned)C; A.cnt[17] = (unsigned)G; A.cnt[18] = dyn; A.cnt[19] = blockDim.x;
      }
      return;
    }
  }
  const int NCL = G / C, cid = c / C;
  const int NCLp = (NCL + 3) & ~3;
  const int nl = N.n_line, ng = N.n_gen;
  const int r0 = min(nl, c * A.rows_per_cta), r1 = min(nl, r0 + A.rows_per_cta);
  const int nr = r1 - r0;
  const int SL = A.slice;
  const int j0 = min(ng, rank * SL), j1 = min(ng, j0 + SL);
  const int nj = j1 - j0;
  const int ngp = (ng + 3) & ~3;
  const int rpc = A.rows_per_cta;
  // shared memory carve-up: per-slice generator constants (FP64), then floats
  double* gk = (double*)smem_raw;                // [7][SLp] ctil, sigma, mq, cconst, mid 2^e, sigma 2^e, 1/(2 mq)
  const int SLp = (SL + 1) & ~1;
  // [C][SL] partial adjoints of own slice, one row per cluster rank (written by peers)
  float* recv = (float*)(gk + 7 * SLp);
  float* xs = recv + ((C * SL + 3) & ~3);        // [ngp] x* of all gens (written by peers)
  float* tmp = xs + ngp;                         // [SL * NCLp] cluster partials of own slice
  float* xacc = tmp + SL * NCLp;                 // [SL] mean of the minimisers (cluster 0)
  float* row = xacc + ((SL + 3) & ~3);           // per-row arrays, 12 x rpc
  float *eta = row, *mh = row + rpc, *ml = row + 2 * rpc, *h1 = row + 3 * rpc, *h2 = row + 4 * rpc,
        *l1 = row + 5 * rpc, *l2 = row + 6 * rpc, *ph = row + 7 * rpc, *pl = row + 8 * rpc,
        *fmx = row + 9 * rpc, *fmn = row + 10 * rpc, *f0 = row + 11 * rpc;
  float* phis = row + 12 * rpc;                  // [rpc][ng] when resident
  __shared__ double rsh[256];   // line partials of the previous evaluation, one per CTA
  __shared__ double s_dec[2];   // [0] value of the evaluation, [1] 1 if it improved the best
  __shared__ double s_vbase;    // cost + lambda (sum p - D) of the pending evaluation
  __shared__ int s_cand;        // stop decision of this loop (made by the last warp)
  __shared__ double s_lam[4];   // lam, s1, s2, lam at the pending evaluation
  __shared__ float redf[32];
  __shared__ long long redq[32];
  __shared__ double s_csp[8];     // the cluster's slice cost sums (written by peers)
  __shared__ long long s_psp[8];  // the cluster's slice dispatch sums, fixed point (peers)
  __shared__ double s_cspc[8];    // copies of the two above for the lambda step, taken
  __shared__ long long s_pspc[8]; // before the peers can store the next loop's sums
  __shared__ int s_flags[8];      // the cluster's gave-up flags (written by peers)
  // transaction barriers: [0] the peers' asynchronous stores of adjoint partials of own
  // slice, [1] theirs of x* of the other slices with the slice sums and flags, [2] the
  // bulk copy of own slice's partials of every cluster
  __shared__ __align__(8) uint64_t s_mb[3];
  __shared__ double s_pw[6];    // decay^(t-1), 1 - beta1^t, 1 - beta2^t; running powers
  __shared__ float s_pwf[8];    // FP32 step factors by loop parity: alpha decay^(t-1), 1 / bias corrections, alpha_lambda decay^(t-1)

  const float* phig = N.phi32 + (size_t)r0 * ng;  // own rows in global memory
  if (A.phi_in_smem)
    for (int q = tid; q < nr * ng; q += blockDim.x) phis[q] = N.phi32[(size_t)r0 * ng + q];
  for (int jj = tid; jj < nj; jj += blockDim.x) {
    const int j = j0 + jj;
    gk[jj] = N.ctil[j]; gk[SLp + jj] = N.sigma[j]; gk[2 * SLp + jj] = N.mq[j];
    gk[3 * SLp + jj] = N.cconst[j];
    gk[6 * SLp + jj] = N.mq[j] > 0.0 ? 0.5 / N.mq[j] : 0.0;
    // the dispatch mid + sigma x in units of the fixed point (scaling by 2^e is exact,
    // so one FMA rounds exactly as the unscaled expression would)
    gk[4 * SLp + jj] = N.mid[j] * A.pscale; gk[5 * SLp + jj] = N.sigma[j] * A.pscale;
  }
  SolveState<float>& st = A.st;
  // the mean of the minimisers: cluster 0 keeps the running sum of each slice
  const bool mean_on = st.xsum != nullptr && cid == 0;
  if (mean_on)
    for (int jj = tid; jj < nj; jj += blockDim.x) xacc[jj] = st.xsum[j0 + jj];
  double wacc = 0.0;
  for (int r = tid; r < nr; r += blockDim.x) {
    int i = r0 + r;
    mh[r] = st.mu_hi[i]; ml[r] = st.mu_lo[i];
    h1[r] = st.s1_hi[i]; h2[r] = st.s2_hi[i]; l1[r] = st.s1_lo[i]; l2[r] = st.s2_lo[i];
    fmx[r] = N.fmax32[i]; fmn[r] = N.fmin32[i]; f0[r] = A.f0[i];
  }
  if (tid == 0) {
    s_lam[0] = st.lam[0]; s_lam[1] = st.lam_s1[0]; s_lam[2] = st.lam_s2[0]; s_lam[3] = st.lam[0];
    // running powers decay^t, beta1^t, beta2^t at the evaluation count of the state
    // (one pow each per launch; FP64 pow is slow on this part)
    const double t0 = (double)st.iter[0];
    s_pw[3] = pow(A.P.decay, t0);
    s_pw[4] = pow(A.P.beta1, t0);
    s_pw[5] = pow(A.P.beta2, t0);
  }
  // stop threshold of this launch (changed only between launches)
  const double stop_at = st.has_target ? st.thresh[0] + st.margin[0] : INFINITY;
  const double demand = A.demand[0];
  const RuleF RF = rule_f(A.P);
  double best = st.best[0];
  double prev_val = st.prev[0];
  int t = st.iter[0];
  int best_iter = st.best_iter[0];
  double best_lam = st.best_lam[0];
  int cand = 0;
  bool pending = false;
  const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
  // bytes the peers store into this CTA per loop: their partials of own slice, and
  // their x* slices with two 8-byte sums and a 4-byte flag each
  const uint32_t tx_part = (uint32_t)((C - 1) * nj * 4);
  const uint32_t tx_x = (uint32_t)((ng - nj) * 4 + (C - 1) * 20);
  if (tid == 0) {
    umma::mbar_init(&s_mb[0], 1);
    umma::mbar_init(&s_mb[1], 1);
    umma::mbar_init(&s_mb[2], 1);
    umma::fence_mbar_init();
  }
  cl.sync();  // every rank's barriers initialised before any store into it
  // the first wait that gives up records (which wait, loop, CTA, thread) for the host's
  // diagnostics: 1 partials of own slice, 2 arrival counters, 3 x* and sums, 4 the
  // bulk copy
  auto record_gave_up = [&](unsigned what, unsigned loop) {
    if (atomicCAS(A.cnt + 20, 0u, what) == 0u) {
      A.cnt[21] = loop; A.cnt[22] = (unsigned)c; A.cnt[23] = (unsigned)tid;
    }
  };

  for (unsigned k = 0;; ++k) {
    float* Pcb = A.Pc + (size_t)(k & 1u) * ng * NCLp;
    const double* Rprev = A.R + (size_t)((k + 1u) & 1u) * G;  // written in loop k-1
    double* Rcur = A.R + (size_t)(k & 1u) * G;
    // ---------------- A: partial adjoint of own rows (4 gens per thread in flight),
    // each sent straight into the shared memory of the rank that owns the gen's slice
    // by an asynchronous store counted on that rank's transaction barrier (no round
    // trip, no cluster-wide barrier)
    if (tid == 0) {
      // this loop's phase of both barriers: one arrival each, plus the bytes expected
      // (a peer's stores may land before this; the phase needs both)
      umma::mbar_arrive_expect_tx(&s_mb[0], tx_part);
      umma::mbar_arrive_expect_tx(&s_mb[1], tx_x);
    }
    for (int r = tid; r < nr; r += blockDim.x) eta[r] = mh[r] - ml[r];
    __syncthreads();
    auto push = [&](int j, float v) {
      const int q = j / SL;
      float* dst = recv + rank * SL + (j - q * SL);
      if (q == rank) *dst = v;
      else umma::st_async_b32(umma::cluster_addr(dst, q), __float_as_uint(v),
                              umma::cluster_addr(&s_mb[0], q));
    };
    // (instantiated once per home of Phi~ rows, so that shared-memory rows are read
    // with shared-memory loads rather than generic ones)
    auto adjoint = [&](const float* rows) {
      for (int jb = tid; jb < ng; jb += 4 * blockDim.x) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const int b = blockDim.x;
        const bool v1 = jb + b < ng, v2 = jb + 2 * b < ng, v3 = jb + 3 * b < ng;
#pragma unroll 4
        for (int r = 0; r < nr; ++r) {
          const float e = eta[r];
          const float* pr = rows + (size_t)r * ng + jb;
          a0 = fmaf(pr[0], e, a0);
          if (v1) a1 = fmaf(pr[b], e, a1);
          if (v2) a2 = fmaf(pr[2 * b], e, a2);
          if (v3) a3 = fmaf(pr[3 * b], e, a3);
        }
        push(jb, a0);
        if (v1) push(jb + b, a1);
        if (v2) push(jb + 2 * b, a2);
        if (v3) push(jb + 3 * b, a3);
      }
    };
    if (A.phi_in_smem) adjoint(phis);
    else adjoint(phig);
    __syncthreads();  // own rank's partials
    const bool part_ok = umma::mbar_wait_cluster(&s_mb[0], k & 1u, A.timeout_ns);
    if (!part_ok) record_gave_up(1, k);
    // ---------------- A2: cluster sum of own slice (fixed rank order), published
    for (int jj = tid; jj < nj; jj += blockDim.x) {
      const int j = j0 + jj;
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = q < C ? recv[q * SL + jj] : 0.f;
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) s += v[q];
      Pcb[(size_t)j * NCLp + cid] = s;
    }
    __syncthreads();
    if (tid == 0) red_release_add_u32(A.cnt + rank, 1u);  // releases the CTA's writes
    // ---------------- B: wait for every cluster's arrival, read partials (and R), x*
    {
      bool ok = part_ok;
      if (tid < C) {
        // counter `tid` counts the arrivals of rank-tid CTAs: NCL per loop
        // acquire loads; bar.sync below extends the ordering to the whole CTA
        const bool got = bounded_wait_geq(A.cnt + tid, (unsigned)NCL * (k + 1u) + A.arrive_extra,
                                          A.timeout_ns);
        if (!got) record_gave_up(2, k);
        ok = got && ok;
      }
      // Scalar work of the loop, by lane 0 of the last two warps while the counters
      // are polled (off the critical path):
      if (tid == (int)blockDim.x - 32 && pending) {
        // the previous loop's lambda step, from the cost and dispatch totals of its
        // evaluation (FP64 over the cluster's slice sums, the dispatch exactly in
        // fixed point): the value base cost + lambda (sum p - D), then the direction
        // in FP32 and the update of lambda in FP64
        double cost_t = 0.0;
        long long ps2 = 0;
        for (int q = 0; q < C; ++q) { cost_t += s_cspc[q]; ps2 += s_pspc[q]; }
        const double psum_t = (double)ps2 * A.pinv;
        double lam = s_lam[0];
        s_lam[3] = lam;
        s_vbase = cost_t + lam * (psum_t - demand);  // the value without its line sum
        float s1 = (float)s_lam[1], s2 = (float)s_lam[2];
        const float gl = (float)(psum_t - demand);
        const float* pf = s_pwf + ((k + 1u) & 1u) * 4;  // the previous loop's factors
        const float th = fused_rule_f(RF, 0.f, gl, s1, s2, pf[3], pf[1], pf[2]);
        lam += (double)th;
        s_lam[0] = lam; s_lam[1] = s1; s_lam[2] = s2;
      } else if (tid == (int)blockDim.x - 64) {
        // this loop's step-size factors from the running powers (FP64), with FP32
        // copies for every thread (double-buffered by loop parity: the lambda step
        // above reads the previous loop's at the same time)
        float* pf = s_pwf + (k & 1u) * 4;
        s_pw[0] = s_pw[3];
        s_pw[4] *= A.P.beta1;
        s_pw[5] *= A.P.beta2;
        s_pw[3] *= A.P.decay;
        s_pw[1] = 1.0 - s_pw[4];
        s_pw[2] = 1.0 - s_pw[5];
        pf[0] = (float)(A.P.alpha * s_pw[0]);
        pf[1] = (float)(1.0 / s_pw[1]);  // reciprocals of the bias corrections
        pf[2] = (float)(1.0 / s_pw[2]);
        pf[3] = (float)(A.P.alpha_lambda * s_pw[0]);
      }
      const int waited_out = __syncthreads_or(ok ? 0 : 1);
      ok = waited_out == 0;
      double rv = 0.0;
      if (tid == 0) {
        // the slice's partials of every cluster ([nj][NCLp] floats, contiguous) in one
        // bulk copy; after the acquire, a proxy fence orders it behind the data
        const uint32_t bytes = (uint32_t)(nj * NCLp * 4);
        if (ok && bytes > 0) {
          umma::fence_proxy_async_global();
          umma::mbar_arrive_expect_tx(&s_mb[2], bytes);
          umma::bulk_g2s(tmp, Pcb + (size_t)j0 * NCLp, bytes, &s_mb[2]);
        } else {
          umma::mbar_arrive(&s_mb[2]);  // keeps the phases in step
        }
      }
      if (ok && pending && tid < G) rv = __ldcg(Rprev + tid);
      if (!umma::mbar_wait_cluster(&s_mb[2], k & 1u, A.timeout_ns)) {
        record_gave_up(4, k);
        ok = false;
      }
      if (pending && tid < G) rsh[tid] = rv;
      __syncthreads();
      const double lam = s_lam[0];
      // one thread per generator of the slice: sum the clusters in a fixed order
      // (identical in every cluster), then the closed-form minimiser; the w that
      // cancels (ctil + sigma lambda + pi~) is formed in FP64.  The dispatch sum feeds
      // the lambda gradient sum(p) - D, a small difference of large sums: FP64 all the
      // way.  A generator's cost term only enters the in-loop value (which decides
      // when to certify; the certificate is FP64): FP32 within the CTA, FP64 across
      // the cluster.  Each thread's dispatch is formed in FP64 and rounded once to a
      // 64-bit fixed point whose range covers the sum of |p| over all generators; the
      // fixed-point sums are exact and independent of order, and integer shuffles
      // are several times faster than FP64 ones on this part.
      float csf = 0.f;
      long long psq = 0;
      for (int jj = tid; jj < nj; jj += blockDim.x) {
        const float4* tp = (const float4*)(tmp + jj * NCLp);
        float s = 0.f;
        for (int q = 0; q < NCLp / 4; ++q) {
          const float4 v = tp[q];
          const int b4 = 4 * q;
          s += v.x;
          if (b4 + 1 < NCL) s += v.y;
          if (b4 + 2 < NCL) s += v.z;
          if (b4 + 3 < NCL) s += v.w;
        }
        const double ct = gk[jj], sg = gk[SLp + jj], mq = gk[2 * SLp + jj];
        const double w = ct + sg * lam + (double)s;
        float x;
        if (mq > 0.0) {  // eq. (16): clip(-w / (2 mq), -1, 1), with 1 / (2 mq) precomputed
          x = -(float)w * (float)gk[6 * SLp + jj];
          x = x > 1.f ? 1.f : (x < -1.f ? -1.f : x);
        } else {
          x = inner_x<float>((float)w, 0.f);
        }
        xs[j0 + jj] = x;  // x* to every rank
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < C && q != rank)
            umma::st_async_b32(umma::cluster_addr(xs + j0 + jj, q), __float_as_uint(x),
                               umma::cluster_addr(&s_mb[1], q));
        csf += fmaf(fmaf((float)mq, x, (float)ct), x, (float)gk[3 * SLp + jj]);
        psq += __double2ll_rn(fma(gk[5 * SLp + jj], (double)x, gk[4 * SLp + jj]));
      }
      csf = warp_sum(csf);
      psq = warp_sum(psq);
      if (lane == 0) { redf[warp] = csf; redq[warp] = psq; }
      const int gave_up = __syncthreads_or(ok ? 0 : 1);
      if (warp == 0) {
        // the slice's cost and dispatch sums: a tree over the warp partials
        float cs = lane < nw ? redf[lane] : 0.f;
        long long ps = lane < nw ? redq[lane] : 0ll;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          cs += __shfl_xor_sync(0xffffffffu, cs, o);
          ps += __shfl_xor_sync(0xffffffffu, ps, o);
        }
        if (lane < C) {  // the slice's sums and flag to every rank
          const double csd = (double)cs;
          if (lane == rank) {
            s_csp[rank] = csd;
            s_psp[rank] = ps;
            s_flags[rank] = gave_up;
          } else {
            const uint32_t bar = umma::cluster_addr(&s_mb[1], lane);
            umma::st_async_b64(umma::cluster_addr(s_csp + rank, lane),
                               (uint64_t)__double_as_longlong(csd), bar);
            umma::st_async_b64(umma::cluster_addr(s_psp + rank, lane), (uint64_t)ps, bar);
            umma::st_async_b32(umma::cluster_addr(s_flags + rank, lane), (uint32_t)gave_up, bar);
          }
        }
      }
      // The value of the previous evaluation and the stop decision are made by the
      // last warp while the peers' x* and sums arrive.
      if (warp == nw - 1) {
        // line partials of the previous evaluation (FP64, fixed order), the value, the
        // best point and the stop decision, made once and broadcast
        double lsum = 0.0;
        if (pending) {
          double l2 = 0.0;  // two chains: FP64 add latency is high on this part
          int q = lane;
          for (; q + 32 < G; q += 64) { lsum += rsh[q]; l2 += rsh[q + 32]; }
          if (q < G) lsum += rsh[q];
          lsum = warp_sum(lsum + l2);
        }
        if (lane == 0) {
          int cd = cand;
          double val = 0.0;
          int imp = 0;
          if (pending) {
            val = s_vbase + lsum;
            imp = val > best;
            if ((imp ? val : best) >= stop_at) cd = 1;
            if (t >= A.max_iters) cd = 2;
            if (A.tol > 0.0 && t > 1 && fabs(val - prev_val) < A.tol) cd = 2;
          }
          s_dec[0] = val;
          s_dec[1] = (double)imp;
          s_cand = cd;
        }
      }
    }
    // ---------------- C: uniform exit decisions, forward, supergradient, step
    {
      // every rank's x* slice, sums and flag (peers' through the transaction barrier,
      // own through bar.sync), and the last warp's decision
      const bool x_ok = umma::mbar_wait_cluster(&s_mb[1], k & 1u, A.timeout_ns);
      if (!x_ok) record_gave_up(3, k);
      int any = __syncthreads_or(x_ok ? 0 : 1);
#pragma unroll
      for (int q = 0; q < 8; ++q) any |= (q < C) ? s_flags[q] : 0;
      if (any) {
        // uniform in the cluster when every rank's flag arrived; a rank whose own wait
        // gave up leaves alone and its peers' bounded waits for it give up next loop
        if (tid == 0) atomicExch(A.err, (int)DCOPF_ERR_TIMEOUT);
        break;
      }
    }
    if (pending) {
      const double val = s_dec[0];
      if (s_dec[1] != 0.0) {
        best = val; best_lam = s_lam[3]; best_iter = t;
        for (int r = tid; r < nr; r += blockDim.x) { st.best_hi[r0 + r] = ph[r]; st.best_lo[r0 + r] = pl[r]; }
      }
      cand = s_cand;
      prev_val = val;
      pending = false;
    }
    if (cand) break;  // uniform everywhere: every CTA assembled the same value
    if (mean_on) {  // this loop's minimiser, evaluation t + 1, weight (t + 1)^2
      const float kk = (float)(t + 1), wk = kk * kk;
      for (int jj = tid; jj < nj; jj += blockDim.x) xacc[jj] += wk * xs[j0 + jj];
      wacc += (double)wk;
    }
    if (tid == (int)blockDim.x - 32) {
      for (int q = 0; q < C; ++q) { s_cspc[q] = s_csp[q]; s_pspc[q] = s_psp[q]; }
    }
    // forward on own rows: a warp per row, 3 rows of a warp in flight
    auto forward = [&](const float* rows) {
      for (int rb = warp; rb < nr; rb += 3 * nw) {
        const bool v1 = rb + nw < nr, v2 = rb + 2 * nw < nr;
        const float* p0 = rows + (size_t)rb * ng;
        const float* p1 = p0 + (size_t)nw * ng;
        const float* p2 = p1 + (size_t)nw * ng;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 4
        for (int j = lane; j < ng; j += 32) {
          const float x = xs[j];
          a0 = fmaf(p0[j], x, a0);
          if (v1) a1 = fmaf(p1[j], x, a1);
          if (v2) a2 = fmaf(p2[j], x, a2);
        }
        a0 = warp_sum(a0);
        a1 = warp_sum(a1);
        a2 = warp_sum(a2);
        if (lane == 0) {
          eta[rb] = a0 + f0[rb];  // eta[] reused as the flow of own rows
          if (v1) eta[rb + nw] = a1 + f0[rb + nw];
          if (v2) eta[rb + 2 * nw] = a2 + f0[rb + 2 * nw];
        }
      }
    };
    if (A.phi_in_smem) forward(phis);
    else forward(phig);
    __syncthreads();
    t += 1;
    const float* pf = s_pwf + (k & 1u) * 4;
    const float bc1 = pf[1];
    const float bc2 = pf[2];
    const float am = pf[0];
    // projected steps of own lines: item i < nr steps mu_hi of row i, item nr + i
    // steps mu_lo of row i (two threads per line); the lambda step of this loop runs
    // in the next loop's A2
    float lacc = 0.f;
    for (int i = tid; i < 2 * nr; i += blockDim.x) {
      const bool hi = i < nr;
      const int r = hi ? i : i - nr;
      const float f = eta[r];
      const float g = hi ? f - fmx[r] : fmn[r] - f;
      float* mu = hi ? mh : ml;
      float* s1 = hi ? h1 : l1;
      float* s2 = hi ? h2 : l2;
      const float m0 = mu[r];
      lacc = fmaf(m0, g, lacc);
      (hi ? ph : pl)[r] = m0;
      const float nm = fused_rule_f(RF, m0, g, s1[r], s2[r], am, bc1, bc2);
      mu[r] = nm > 0.f ? nm : 0.f;
    }
    // the line partial: FP32 per thread and warp, FP64 across warps; published by
    // the release-add of the next arrival
    lacc = warp_sum(lacc);
    if (lane == 0) rsh[warp] = (double)lacc;  // rsh is free until the next phase B
    pending = true;
    __syncthreads();
    if (tid == 0) {
      // only the warps that own step items (item i belongs to thread i) contribute
      const int nwr = min(nw, (2 * nr + 31) >> 5);
      double l = 0.0;
      for (int q = 0; q < nwr; ++q) l += rsh[q];
      Rcur[c] = l;
    }
  }
  // ---------------- write back (resumable state); peers may still read our smem
  cl.sync();
  if (mean_on) {
    for (int jj = tid; jj < nj; jj += blockDim.x) st.xsum[j0 + jj] = xacc[jj];
    if (c == 0 && tid == 0) st.wsum[0] += wacc;
  }
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

// Largest cluster shape the device can keep resident with one CTA per SM.
struct FusedShape {
  int C = 0, G = 0;
  size_t smem = 0;
  int phi_in_smem = 0;
  int rows_per_cta = 0, slice = 0;
};

static size_t fused_smem(int ng, int rpc, int C, int NCL, bool phi) {
  int ngp = (ng + 3) & ~3;
  int SL = (ng + C - 1) / C;
  int SLp = (SL + 1) & ~1;
  int NCLp = (NCL + 3) & ~3;
  size_t f = (size_t)((C * SL + 3) & ~3) + ngp + (size_t)SL * NCLp + ((SL + 3) & ~3) +
             12 * (size_t)rpc;
  if (phi) f += (size_t)rpc * ng;
  return f * sizeof(float) + 7 * (size_t)SLp * sizeof(double);
}

// g_cap bounds the grid (fewer, larger CTAs: more rows each, fewer clusters to
// exchange with).
static cudaError_t fused_config(const dcopf_dual* h, int C, FusedShape* out, int g_cap = 1 << 30) {
  const int nl = h->dev.n_line, ng = h->dev.n_gen;
  const int sms = std::min(std::min(h->sm_count, 256), g_cap);  // R: one thread per CTA
  int G = (sms / C) * C;
  if (G < C) return cudaErrorInvalidValue;
  for (int pass = 0; pass < 2; ++pass) {
    const int rpc = (nl + G - 1) / G;
    const bool phi = fused_smem(ng, rpc, C, G / C, true) + 2048 <= h->smem_optin;
    const size_t smem = fused_smem(ng, rpc, C, G / C, phi);
    if (smem + 2048 > h->smem_optin) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_fused_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, k_fused_solve, &cfg);
    if (e != cudaSuccess) return e;
    if (ncl * C >= G) {
      out->C = C; out->G = G; out->smem = smem; out->phi_in_smem = phi ? 1 : 0;
      out->rows_per_cta = rpc; out->slice = (ng + C - 1) / C;
      return cudaSuccess;
    }
    if (ncl < 1 || pass == 1) return cudaErrorInvalidValue;
    G = ncl * C;  // fewer clusters fit: size the grid to what is resident
  }
  return cudaErrorInvalidValue;
}

// Cluster shapes (C, G) with C >= 2 the device keeps resident for this network,
// largest cluster first; returns how many were written.
int fused_candidates(dcopf_dual* h, int* Cs, int* Gs, int cap) {
  int n = 0;
  for (int C : {8, 4, 2}) {
    for (int div : {1, 2, 4}) {  // all SMs, or a half / quarter of them with more rows each
      FusedShape sh;
      if (n >= cap || fused_config(h, C, &sh, std::max(C, h->sm_count / div)) != cudaSuccess)
        continue;
      bool dup = false;
      for (int i = 0; i < n; ++i) dup |= Cs[i] == sh.C && Gs[i] == sh.G;
      if (dup || (div > 1 && !sh.phi_in_smem)) continue;  // smaller grids only with Phi resident
      Cs[n] = sh.C;
      Gs[n] = sh.G;
      ++n;
    }
  }
  cudaGetLastError();
  return n;
}

dcopf_status run_iters_fused(dcopf_dual* h, const StepArgs& P, SolveState<float>& st, int max_iters,
                             double tol, cudaStream_t s) {
  const DevNet& N = h->dev;
  const int ng = N.n_gen;
  if (h->fused_C == 0) {
    // Per iteration a CTA reduces (n_gen / C) generators over G / C cluster partials,
    // so larger clusters cut that work; accept a larger cluster unless it leaves
    // more than 1/8 of the SMs idle.
    FusedShape best;
    for (int C : {8, 4, 2, 1}) {
      FusedShape sh;
      if (fused_config(h, C, &sh) != cudaSuccess) continue;
      if (h->verbose)
        fprintf(stderr, "[dcopf] fused candidate: cluster %d, %d CTAs resident\n", C, sh.G);
      if (best.G == 0 || 8 * sh.G > 9 * best.G) best = sh;
    }
    cudaGetLastError();
    if (best.G == 0) return DCOPF_ERR_UNSUPPORTED;
    h->fused_C = best.C;
    h->fused_G = best.G;
    if (h->verbose)
      fprintf(stderr, "[dcopf] fused kernel: cluster %d x %d CTAs, %zu B shared, Phi rows %s, %d rows/CTA\n",
              best.G / best.C, best.C, best.smem, best.phi_in_smem ? "resident" : "streamed",
              best.rows_per_cta);
  }
  FusedShape sh;
  if (h->fshape_C == h->fused_C && h->fshape_G == h->fused_G) {
    sh.C = h->fshape_C; sh.G = h->fshape_G; sh.smem = h->fshape_smem; sh.phi_in_smem = h->fshape_phi;
    sh.rows_per_cta = h->fshape_rpc; sh.slice = h->fshape_slice;
    // the attribute is per function: another handle may have lowered it since
    if (cudaFuncSetAttribute(k_fused_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sh.smem) != cudaSuccess)
      return DCOPF_ERR_CUDA;
  } else {
    if (fused_config(h, h->fused_C, &sh, h->fused_G) != cudaSuccess || sh.G != h->fused_G) {
      cudaGetLastError();
      return DCOPF_ERR_UNSUPPORTED;
    }
    h->fshape_C = sh.C; h->fshape_G = sh.G; h->fshape_smem = sh.smem; h->fshape_phi = sh.phi_in_smem;
    h->fshape_rpc = sh.rows_per_cta; h->fshape_slice = sh.slice;
  }
  const int G = sh.G, C = sh.C, NCL = G / C;
  const int NCLp = (NCL + 3) & ~3;
  FusedArgs A{};
  A.N = N;
  A.P = P;
  A.st = st;
  A.f0 = h->ws.f0_32.as<float>();
  A.rows_per_cta = sh.rows_per_cta;
  A.slice = sh.slice;
  A.phi_in_smem = sh.phi_in_smem;
  A.C = C;
  A.G = G;
  A.smem_bytes = (unsigned)sh.smem;
  // exchange buffers; the arrival counters are zeroed before every launch
  const size_t pc_bytes = ((size_t)2 * ng * NCLp * 4 + 255) & ~(size_t)255;
  const size_t r_bytes = ((size_t)2 * G * 8 + 255) & ~(size_t)255;
  if (h->ws.misc.alloc(pc_bytes + r_bytes + 256) != cudaSuccess) return DCOPF_ERR_OOM;
  char* m = h->ws.misc.as<char>();
  A.Pc = (float*)m;
  A.R = (double*)(m + pc_bytes);
  A.cnt = (unsigned*)(m + pc_bytes + r_bytes);
  A.err = h->d_err;
  {
    // 2^e with sum_j (|mid_j| + |sigma_j|) * 2^e < 2^61, a bound on sum_j |p_j| 2^e:
    // no partial sum of the rounded dispatches can overflow 64 bits
    double pabs = 1.0;
    for (int j = 0; j < ng; ++j) pabs += fabs(h->host.mid[j]) + fabs(h->host.sigma[j]);
    const int e = 61 - (int)ceil(log2(pabs));
    A.pscale = ldexp(1.0, e);
    A.pinv = ldexp(1.0, -e);
  }
  A.max_iters = max_iters;
  A.tol = tol;
  A.timeout_ns = h->fused_timeout_ns;
  A.arrive_extra = h->fused_arrive_extra;
  A.demand = h->ws.demand.as<double>();  // read on the device: no host round trip
  if (cudaMemsetAsync(A.cnt, 0, 256, s) != cudaSuccess) return DCOPF_ERR_CUDA;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = sh.smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  // Co-residency of all clusters: requested from the driver (cooperative launch) when
  // it accepts that together with clusters; otherwise the grid is sized from
  // cudaOccupancyMaxActiveClusters and the bounded waits are the guard.
  cfg.numAttrs = h->fused_coop == 0 ? 1 : 2;
  // the refusal hook: a shape record that does not match the launch
  FusedArgs Ar = A;
  Ar.C = A.C + 1;
  const bool refuse_coop = h->fused_refuse >= 1, refuse_all = h->fused_refuse == 2;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_fused_solve,
                                     (refuse_all || (refuse_coop && cfg.numAttrs == 2)) ? Ar : A);
  if (e != cudaSuccess && cfg.numAttrs == 2) {
    cudaGetLastError();
    h->fused_coop = 0;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_fused_solve, refuse_all ? Ar : A);
  } else if (e == cudaSuccess && cfg.numAttrs == 2) {
    h->fused_coop = 1;
  }
  h->launches += 1;
  if (e != cudaSuccess) { h->last_error = cudaGetErrorString(e); return DCOPF_ERR_CUDA; }
  return DCOPF_OK;
}

// Self-test of the bounded wait: one thread waits for a counter that nothing
// increments; the wait must give up and report it.
__global__ void k_wait_selftest(const unsigned* ctr, uint64_t timeout_ns, int* gave_up) {
  if (threadIdx.x == 0) *gave_up = bounded_wait_geq(ctr, 1u, timeout_ns) ? 0 : 1;
}

// Prints the launch shape a refused fused launch saw and the first wait that gave up
// (both recorded in the counter block); for the verbose diagnostics of the shape tuner.
void fused_report_refusal(dcopf_dual* h) {
  unsigned v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const size_t ng = (size_t)h->dev.n_gen;
  const int G = h->fused_G, C = std::max(1, h->fused_C);
  const size_t NCLp = (size_t)((G / C + 3) & ~3);
  const size_t pc_bytes = (2 * ng * NCLp * 4 + 255) & ~(size_t)255;
  const size_t r_bytes = ((size_t)2 * G * 8 + 255) & ~(size_t)255;
  if (!h->ws.misc.p || h->ws.misc.bytes < pc_bytes + r_bytes + 256) return;
  if (cudaMemcpy(v, h->ws.misc.as<char>() + pc_bytes + r_bytes + 64, sizeof(v),
                 cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if (v[0])
    fprintf(stderr, "[dcopf] fused launch refused: saw cluster %u, grid %u, %u B dynamic shared, %u threads; "
                    "sized for cluster %d, grid %d\n", v[0], v[1], v[2], v[3], C, G);
  if (v[4])
    fprintf(stderr, "[dcopf] fused wait gave up: kind %u (1 partials, 2 arrivals, 3 x*), loop %u, CTA %u, "
                    "thread %u\n", v[4], v[5], v[6], v[7]);
}

dcopf_status run_wait_selftest(dcopf_dual* h, long long timeout_ns, cudaStream_t s) {
  if (h->ws.misc.alloc(std::max<size_t>(h->ws.misc.bytes, 256)) != cudaSuccess) return DCOPF_ERR_OOM;
  unsigned* ctr = (unsigned*)h->ws.misc.p;
  int* flag = (int*)((char*)h->ws.misc.p + 64);
  if (cudaMemsetAsync(h->ws.misc.p, 0, 128, s) != cudaSuccess) return DCOPF_ERR_CUDA;
  k_wait_selftest<<<1, 32, 0, s>>>(ctr, (uint64_t)timeout_ns, flag);
  h->launches += 1;
  int gave_up = 0;
  if (cudaMemcpyAsync(&gave_up, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  return gave_up ? DCOPF_ERR_TIMEOUT : DCOPF_OK;
}

}  // namespace dcopf
