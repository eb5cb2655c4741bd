// Batched operator products on tcgen05 tensor cores for many instances of one
// network: the adjoint Pi~ = H Phi~ (H = [batch][n_line] line multipliers) and the
// forward F = X Phi~^T (X = [batch][n_gen] normalised dispatch), the two dense
// contractions of every iteration (eq. (6): c + A^T lambda + C^T mu, and C x*).
//
// The products themselves (tcgen05, BF16 hi/lo split operands, single CTAs or CTA
// pairs) are in k_gemm.cuh; this file holds the iteration's other kernels (minimiser,
// step, value), the shape autotuner and the host driver of the batched solve.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <string>
#include <vector>

#include "dev.cuh"
#include "kernels.h"
#include "k_gemm.cuh"
#include "umma.cuh"

namespace dcopf {

// Internal status of a batched solve that must run again with a fresh constraint screen.
constexpr dcopf_status kRescreen = (dcopf_status)1000;

// Step-rule constants in FP32, converted once on the host (FP64 conversions per
// element are not free on this part).
struct StepArgsF {
  int rule, as_printed;
  float rho, beta1, omb1, beta2, omb2, eps;
};

static StepArgsF to_float_args(const StepArgs& P) {
  StepArgsF f;
  f.rule = P.rule;
  f.as_printed = P.as_printed;
  f.rho = (float)P.rho;
  f.beta1 = (float)P.beta1;
  f.omb1 = (float)(1.0 - P.beta1);
  f.beta2 = (float)P.beta2;
  f.omb2 = (float)(1.0 - P.beta2);
  f.eps = (float)P.eps;
  return f;
}

// One coordinate's step (Section 3.3) in FP32 with the instance's step factors of this
// step: a = alpha decay^(t-1) (GDM, AdaGrad), and for Adam a1 = a / (1 - beta1^t) and
// r2 = 1 / sqrt(1 - beta2^t), so that a (s1 / c1) / (sqrt(s2 / c2) + eps) is
// a1 s1 / (sqrt(s2) r2 + eps) with one division.  The division is the fast one
// (__fdividef, within two units in the last place for these operand ranges): the step
// only steers the iteration, the bound is certified in FP64.
__device__ __forceinline__ float step_rule(const StepArgsF& P, float theta, float g, float& s1,
                                           float& s2, float a, float a1, float r2) {
  if (P.rule == DCOPF_GDM) {
    s1 = P.rho * s1 + a * g;
    theta += s1;
    if (P.as_printed) theta += a * g;
  } else if (P.rule == DCOPF_ADAM) {
    s1 = P.beta1 * s1 + P.omb1 * g;
    s2 = P.beta2 * s2 + P.omb2 * g * g;
    theta += __fdividef(a1 * s1, fmaf(sqrtf(s2), r2, P.eps));
  } else {
    s1 += g * g;
    theta += __fdividef(a * g, sqrtf(s1) + P.eps);
  }
  return theta;
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16* hi, __nv_bfloat16* lo);
__device__ __forceinline__ int finalize_instance(int b, int lane, int max_iters, double tol,
                                                 const SolveStateBase& st, const BatchView& bb,
                                                 const double* __restrict__ demand);

// Step of the batched solve after the forward product: flows (with the rank-1 outage
// term), supergradient, line part of the dual value, projected step of mu into the
// parity-buffered state, BF16 split of the next eta, outage partial u^T eta.
struct StepEpi {
  StepArgsF P;
  const float* F;             // [B][ldF] forward product Phi~ x
  const float* f0;            // [B][nl] flows of the mid-box dispatch minus the loads
  int ldF;
  const float* u;             // [B][nl] outage vectors (rows of outage instances)
  const int* outage;          // [B] or null
  const float* tout;          // [B] pre-outage flow on the outaged line, (Phi~ x)_k
  const float* fmax; const float* fmin;
  const int* iter;            // [B] evaluations done: iter % 3 selects the state buffer
  const int* frozen;          // [B] done or waiting for certification
  const int* best_iter;       // [B] evaluation count of the best point so far
  const float* stepf;         // [B][4] step factors a, a1, r2 of step_rule
  // Three state buffers in turn: point t lives in buffer t % 3, so the two points
  // before the one being stepped are still there.  The step writing point t + 1
  // overwrites point t - 2; if that point is still the best (the value fell after
  // it), it is first copied to sv.  Points that are overtaken before their buffer
  // comes round are never copied.
  float* mu_hi[3]; float* mu_lo[3];
  float* sv_hi; float* sv_lo;
  float* s1_hi; float* s2_hi; float* s1_lo; float* s2_lo;
  __nv_bfloat16* Hh; __nv_bfloat16* Hl; int ldh;
  double* line_part; double* out_part; int n_tiles;   // [B][n_tiles] per slice of lines
  int B;                      // instances
  // [B]: the step has left the value partials of the instance's evaluated point (its
  // value and stop tests, finalize_instance, run in the next minimiser or at the end
  // of the round)
  int* pend;
};

// The step's work is a slice of STEP_SLICE lines of one instance per warp (four lines
// per lane, coalesced), elementwise; slices of an instance are numbered 0 .. n_tiles - 1
// and each leaves FP64 partials of the value and of u^T eta.
constexpr int STEP_THREADS = 256, STEP_SLICE = 128;

// The tail of both step kernels, per warp: the warp's partials go to slot `part` of the
// instance's [n_tiles], and the instance is marked as having partials to finalise (every
// warp stores the same flag; the kernels that read it run later in the stream).  No
// barrier and no fence: warps finish on their own.
__device__ __forceinline__ void step_tail(const StepEpi& E, int b, int part, float lacc, float oacc) {
  if ((threadIdx.x & 31) == 0) {
    E.line_part[(size_t)b * E.n_tiles + part] = (double)lacc;
    E.out_part[(size_t)b * E.n_tiles + part] = (double)oacc;
    E.pend[b] = 1;
  }
}

__device__ __forceinline__ void step_item(const StepEpi& E, int nl, int b, int part) {
  if (E.frozen[b]) return;
  const int k = E.outage ? E.outage[b] : -1;
  const float t_out = k >= 0 ? E.tout[b] : 0.f;
  const int it = E.iter[b], pb = it % 3, pn = (it + 1) % 3;
  const bool save = it >= 2 && E.best_iter[b] == it - 1;  // point it - 2 is the best
  const size_t o = (size_t)b * nl;
  const float* mhc = E.mu_hi[pb] + o;
  const float* mlc = E.mu_lo[pb] + o;
  float* mhn = E.mu_hi[pn] + o;
  float* mln = E.mu_lo[pn] + o;
  const float am = E.stepf[4 * b], a1s = E.stepf[4 * b + 1], r2 = E.stepf[4 * b + 2];
  const float* Fr = E.F + (size_t)b * E.ldF;
  // a lane's few terms are summed in FP32 and the warp's partial is FP64 (FP64
  // throughput is low on this part: per-element FP64 would dominate the kernel)
  float lacc = 0.f, oacc = 0.f;
  const int i0 = part * STEP_SLICE + (int)(threadIdx.x & 31);
  float fl[4], ui[4], mh[4], ml[4], a1[4], a2[4], b1[4], b2[4], fx[4], fn[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {  // all loads in flight before any arithmetic
    const int i = i0 + 32 * q;
    const bool in = i < nl;
    fl[q] = in ? Fr[i] + E.f0[o + i] : 0.f;
    ui[q] = (in && k >= 0) ? E.u[o + i] : 0.f;
    fx[q] = in ? E.fmax[i] : 0.f;
    fn[q] = in ? E.fmin[i] : 0.f;
    mh[q] = in ? mhc[i] : 0.f;
    ml[q] = in ? mlc[i] : 0.f;
    a1[q] = in ? E.s1_hi[o + i] : 0.f;
    a2[q] = in ? E.s2_hi[o + i] : 0.f;
    b1[q] = in ? E.s1_lo[o + i] : 0.f;
    b2[q] = in ? E.s2_lo[o + i] : 0.f;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + 32 * q;
    if (i >= nl) continue;
    const float f = fl[q] + ui[q] * t_out;
    const float gh = f - fx[q], gl = fn[q] - f;
    float nh = 0.f, nlo = 0.f;
    if (i != k) {
      lacc = fmaf(mh[q], gh, fmaf(ml[q], gl, lacc));
      nh = fmaxf(step_rule(E.P, mh[q], gh, a1[q], a2[q], am, a1s, r2), 0.f);
      nlo = fmaxf(step_rule(E.P, ml[q], gl, b1[q], b2[q], am, a1s, r2), 0.f);
      E.s1_hi[o + i] = a1[q]; E.s2_hi[o + i] = a2[q]; E.s1_lo[o + i] = b1[q]; E.s2_lo[o + i] = b2[q];
    }
    if (save) { E.sv_hi[o + i] = mhn[i]; E.sv_lo[o + i] = mln[i]; }
    mhn[i] = nh;
    mln[i] = nlo;
    const float eta = nh - nlo;
    split_bf16(eta, E.Hh + (size_t)b * E.ldh + i, E.Hl + (size_t)b * E.ldh + i);
    if (k >= 0) oacc = fmaf(ui[q], eta, oacc);
  }
  // a warp's terms in FP32, its partials in FP64 (summed in a fixed order by the value)
  lacc = warp_sum(lacc);
  oacc = warp_sum(oacc);
  step_tail(E, b, part, lacc, oacc);
}

// The per-instance scalars that a step item's loads depend on (whether it runs, the
// state buffer, the outage), loaded together in one round trip; the step factors, the
// outage flow and the best point's count then come with the data.
struct StepScalars {
  int frozen, k, it;
};
__device__ __forceinline__ StepScalars step_scalars(const StepEpi& E, int b) {
  StepScalars S;
  S.frozen = E.frozen[b];
  S.k = E.outage ? E.outage[b] : -1;
  S.it = E.iter[b];
  return S;
}

// The same step with four consecutive lines per lane: 16-byte loads and stores of every
// FP32 stream and 8-byte stores of the BF16 split (needs n_line, ldF and ldh multiples
// of 4).  The instance's scalars come in S; every load of the item is then issued at
// once.
__device__ __forceinline__ void step4_item(const StepEpi& E, int nl, int b, int part, const StepScalars& S) {
  if (S.frozen) return;
  const int k = S.k;
  const float t_out = k >= 0 ? E.tout[b] : 0.f;
  const int it = S.it, pb = it % 3, pn = (it + 1) % 3;
  const bool save = it >= 2 && E.best_iter[b] == it - 1;  // point it - 2 is the best
  const size_t o = (size_t)b * nl;
  const float am = E.stepf[4 * b], a1s = E.stepf[4 * b + 1], r2 = E.stepf[4 * b + 2];
  const int i = part * STEP_SLICE + 4 * (int)(threadIdx.x & 31);
  float lacc = 0.f, oacc = 0.f;
  if (i < nl) {
    auto ld4 = [](const float* p) { return *reinterpret_cast<const float4*>(p); };
    const float4 Fv = ld4(E.F + (size_t)b * E.ldF + i), f0 = ld4(E.f0 + o + i);
    const float4 uv = k >= 0 ? ld4(E.u + o + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 fx = ld4(E.fmax + i), fn = ld4(E.fmin + i);
    const float4 mh = ld4(E.mu_hi[pb] + o + i), ml = ld4(E.mu_lo[pb] + o + i);
    float4 a1 = ld4(E.s1_hi + o + i), a2 = ld4(E.s2_hi + o + i);
    float4 b1 = ld4(E.s1_lo + o + i), b2 = ld4(E.s2_lo + o + i);
    float F[4] = {Fv.x, Fv.y, Fv.z, Fv.w}, F0[4] = {f0.x, f0.y, f0.z, f0.w};
    float U[4] = {uv.x, uv.y, uv.z, uv.w}, FX[4] = {fx.x, fx.y, fx.z, fx.w};
    float FN[4] = {fn.x, fn.y, fn.z, fn.w}, MH[4] = {mh.x, mh.y, mh.z, mh.w};
    float ML[4] = {ml.x, ml.y, ml.z, ml.w}, A1[4] = {a1.x, a1.y, a1.z, a1.w};
    float A2[4] = {a2.x, a2.y, a2.z, a2.w}, B1[4] = {b1.x, b1.y, b1.z, b1.w};
    float B2[4] = {b2.x, b2.y, b2.z, b2.w};
    float NH[4], NL[4];
    __align__(8) __nv_bfloat16 hh[4], hl[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float f = F[q] + F0[q] + U[q] * t_out;
      const float gh = f - FX[q], gl = FN[q] - f;
      float nh = 0.f, nlo = 0.f;
      if (i + q != k) {
        lacc = fmaf(MH[q], gh, fmaf(ML[q], gl, lacc));
        nh = fmaxf(step_rule(E.P, MH[q], gh, A1[q], A2[q], am, a1s, r2), 0.f);
        nlo = fmaxf(step_rule(E.P, ML[q], gl, B1[q], B2[q], am, a1s, r2), 0.f);
      }
      NH[q] = nh;
      NL[q] = nlo;
      const float eta = nh - nlo;
      hh[q] = __float2bfloat16_rn(eta);
      hl[q] = __float2bfloat16_rn(eta - __bfloat162float(hh[q]));
      if (k >= 0) oacc = fmaf(U[q], eta, oacc);
    }
    // moments of the outaged line stay as they were: their new values equal the loaded
    // ones there, since step_rule only ran for the other lines
    auto st4 = [](float* p, const float* v) {
      *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    };
    if (save) {  // the best point's buffer is about to be reused: keep a copy
      *reinterpret_cast<float4*>(E.sv_hi + o + i) = ld4(E.mu_hi[pn] + o + i);
      *reinterpret_cast<float4*>(E.sv_lo + o + i) = ld4(E.mu_lo[pn] + o + i);
    }
    st4(E.mu_hi[pn] + o + i, NH);
    st4(E.mu_lo[pn] + o + i, NL);
    st4(E.s1_hi + o + i, A1);
    st4(E.s2_hi + o + i, A2);
    st4(E.s1_lo + o + i, B1);
    st4(E.s2_lo + o + i, B2);
    *reinterpret_cast<uint2*>(E.Hh + (size_t)b * E.ldh + i) = *reinterpret_cast<const uint2*>(hh);
    *reinterpret_cast<uint2*>(E.Hl + (size_t)b * E.ldh + i) = *reinterpret_cast<const uint2*>(hl);
  }
  // a warp's terms in FP32, its partials in FP64 (summed in a fixed order by the value)
  lacc = warp_sum(lacc);
  oacc = warp_sum(oacc);
  step_tail(E, b, part, lacc, oacc);
}

// The step kernels: slice w = (instance w / n_tiles, slice w % n_tiles of its lines),
// one per warp of the grid, or taken in turn by the warps of a smaller grid (that leaves
// room on the SMs for another instance group's products; a block holds 64 registers x
// 256 threads).  An instance's slices run in any order (its last one runs the value).
__global__ void __launch_bounds__(STEP_THREADS) k_bt_step(StepEpi E, int nl) {
  const int nw = blockDim.x >> 5, total = E.n_tiles * E.B;
  for (int w = blockIdx.x * nw + (int)(threadIdx.x >> 5); w < total; w += gridDim.x * nw)
    step_item(E, nl, w / E.n_tiles, w % E.n_tiles);
}

__global__ void __launch_bounds__(STEP_THREADS, 4) k_bt_step4(StepEpi E, int nl) {
  const int nw = blockDim.x >> 5, total = E.n_tiles * E.B;
  for (int w = blockIdx.x * nw + (int)(threadIdx.x >> 5); w < total; w += gridDim.x * nw) {
    const int b = w / E.n_tiles;
    step4_item(E, nl, b, w % E.n_tiles, step_scalars(E, b));
  }
}

// ------------------------------------------------------------------ operand preparation
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  *hi = h;
  *lo = __float2bfloat16_rn(v - __bfloat162float(h));
}

// H[b][i] = mu_hi - mu_lo (outaged line: u^T eta, the adjoint of the post-outage PTDF),
// split into BF16 hi/lo rows of stride ld.
template <typename S>
__global__ void k_split_eta(int nl, int ld, const S* __restrict__ mh, const S* __restrict__ ml,
                            const int* __restrict__ outage, const float* __restrict__ u,
                            __nv_bfloat16* __restrict__ Hh, __nv_bfloat16* __restrict__ Hl) {
  __shared__ float red[32];
  const int b = blockIdx.x;
  const int k = outage ? outage[b] : -1;
  float s = 0.f;
  for (int i = threadIdx.x; i < nl; i += blockDim.x) {
    const float v = (i == k) ? 0.f : (float)((double)mh[(size_t)b * nl + i] - (double)ml[(size_t)b * nl + i]);
    split_bf16(v, Hh + (size_t)b * ld + i, Hl + (size_t)b * ld + i);
    if (k >= 0) s += u[(size_t)b * nl + i] * v;
  }
  if (k >= 0) {
    s = block_sum(s, red);
    if (threadIdx.x == 0) split_bf16(s, Hh + (size_t)b * ld + k, Hl + (size_t)b * ld + k);
  }
}

// pi~ = sum of the split-K partials, closed-form minimiser, BF16 split of x, FP64
// x for the dispatch output, per-instance cost and dispatch sums.
__global__ void k_reduce_min(DevNet N, int splits, int M, int ldp, const float* __restrict__ P,
                             const double* __restrict__ lambda, int ldx,
                             __nv_bfloat16* __restrict__ Xh, __nv_bfloat16* __restrict__ Xl,
                             double* __restrict__ x64, double* __restrict__ sumcost,
                             double* __restrict__ sump) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  const int ng = N.n_gen;
  const double lam = lambda[b];
  double c = 0.0, p = 0.0;
  for (int j = threadIdx.x; j < ng; j += blockDim.x) {
    float s = 0.f;
    for (int q = 0; q < splits; ++q) s += P[((size_t)q * M + b) * ldp + j];
    const double w = N.ctil[j] + N.sigma[j] * lam + (double)s;
    const double x = inner_x<double>(w, N.mq[j]);
    split_bf16((float)x, Xh + (size_t)b * ldx + j, Xl + (size_t)b * ldx + j);
    if (x64) x64[(size_t)b * ng + j] = x;
    c += (N.mq[j] * x + N.ctil[j]) * x + N.cconst[j];
    p += N.mid[j] + N.sigma[j] * x;
  }
  c = block_sum(c, red);
  p = block_sum(p, red);
  if (threadIdx.x == 0) {
    sumcost[b] = c;
    sump[b] = p;
  }
}

// ------------------------------------------------------------------ host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 2-D BF16 tensor map over [rows][cols] with row stride ld elements (ld * 2 bytes a
// multiple of 16), box of 64 columns x box_rows rows, 128-byte swizzle, zero fill
// outside the tensor.
static bool make_map(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint64_t ld,
                     uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || ((uintptr_t)ptr & 15) || ((ld * 2) & 15)) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {64, box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static int round8(int n) { return (n + 7) & ~7; }
static cudaError_t prepare_gemm();

// BF16 hi/lo copies of Phi~ (forward B operand, n_line x n_gen) and Phi~^T (adjoint B
// operand, n_gen x n_line), built once per handle, in 8-row blocks of 64-column K blocks
// (blk_index): a TMA box of 64 columns and 8 j rows is then j contiguous 1 KB runs.
dcopf_status ensure_tensor_operands(dcopf_dual* h) {
  TensorOps& T = h->tops;
  if (T.ready) return DCOPF_OK;
  const HostNet& H = h->host;
  const int nl = H.n_line, ng = H.n_gen;
  T.ld_l = round8(nl);
  T.ld_g = round8(ng);
  const int kb_g = (ng + 63) / 64, kb_l = (nl + 63) / 64;
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  std::vector<__nv_bfloat16> ph((size_t)round8(nl) * kb_g * 64, z), pl(ph.size(), z);
  std::vector<__nv_bfloat16> th((size_t)round8(ng) * kb_l * 64, z), tl(th.size(), z);
  for (int i = 0; i < nl; ++i)
    for (int j = 0; j < ng; ++j) {
      const float v = (float)H.phi[(size_t)i * ng + j];
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      const size_t f = blk_index(i, j, kb_g), a = blk_index(j, i, kb_l);
      ph[f] = hi; pl[f] = lo;
      th[a] = hi; tl[a] = lo;
    }
  auto up = [&](DBuf& d, const std::vector<__nv_bfloat16>& v) {
    if (d.alloc(v.size() * 2) != cudaSuccess) return false;
    return cudaMemcpy(d.p, v.data(), v.size() * 2, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!up(T.phi_hi, ph) || !up(T.phi_lo, pl) || !up(T.phit_hi, th) || !up(T.phit_lo, tl))
    return DCOPF_ERR_OOM;
  bool mok = true;
  for (const uint32_t br : {128u, 96u, 80u, 72u}) {
    CUtensorMap* fh = br == 128 ? &T.m_phi_hi : br == 96 ? &T.m_phi_hi96 : br == 80 ? &T.m_phi_hi80 : &T.m_phi_hi72;
    CUtensorMap* fl = br == 128 ? &T.m_phi_lo : br == 96 ? &T.m_phi_lo96 : br == 80 ? &T.m_phi_lo80 : &T.m_phi_lo72;
    CUtensorMap* ah = br == 128 ? &T.m_phit_hi : br == 96 ? &T.m_phit_hi96 : br == 80 ? &T.m_phit_hi80 : &T.m_phit_hi72;
    CUtensorMap* al = br == 128 ? &T.m_phit_lo : br == 96 ? &T.m_phit_lo96 : br == 80 ? &T.m_phit_lo80 : &T.m_phit_lo72;
    mok = mok && tc_make_map_blocked(fh, T.phi_hi.p, nl, ng, br) && tc_make_map_blocked(fl, T.phi_lo.p, nl, ng, br) &&
          tc_make_map_blocked(ah, T.phit_hi.p, ng, nl, br) && tc_make_map_blocked(al, T.phit_lo.p, ng, nl, br);
  }
  if (!mok) return DCOPF_ERR_CUDA;
  if (prepare_gemm() != cudaSuccess) return DCOPF_ERR_CUDA;
  T.ready = true;
  return DCOPF_OK;
}

// Per-batch BF16 operands and split-K partials.
dcopf_status ensure_tensor_batch(dcopf_dual* h, int B) {
  TensorOps& T = h->tops;
  if (B <= T.cap) return DCOPF_OK;
  const int nl = h->host.n_line, ng = h->host.n_gen;
  const int ldp = (ng + 3) & ~3;
  T.cap = 0;  // reset unless every buffer and tensor map below is made
  if (T.H_hi.alloc((size_t)B * T.ld_l * 2) || T.H_lo.alloc((size_t)B * T.ld_l * 2) ||
      T.X_hi.alloc((size_t)B * T.ld_g * 2) || T.X_lo.alloc((size_t)B * T.ld_g * 2) ||
      T.P.alloc((size_t)64 * B * ldp * 4)) {
    cudaGetLastError();
    return DCOPF_ERR_OOM;
  }
  cudaMemset(T.H_hi.p, 0, (size_t)B * T.ld_l * 2);
  cudaMemset(T.H_lo.p, 0, (size_t)B * T.ld_l * 2);
  cudaMemset(T.X_hi.p, 0, (size_t)B * T.ld_g * 2);
  cudaMemset(T.X_lo.p, 0, (size_t)B * T.ld_g * 2);
  if (!make_map(&T.m_H_hi, T.H_hi.p, B, nl, T.ld_l, GBM) ||
      !make_map(&T.m_H_lo, T.H_lo.p, B, nl, T.ld_l, GBM) ||
      !make_map(&T.m_X_hi, T.X_hi.p, B, ng, T.ld_g, GBM) ||
      !make_map(&T.m_X_lo, T.X_lo.p, B, ng, T.ld_g, GBM))
    return DCOPF_ERR_CUDA;
  T.cap = B;
  return DCOPF_OK;
}

// Sets the GEMM kernels' shared-memory limits (outside any stream capture).
static cudaError_t prepare_gemm() {
  cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16x<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)GemmCfg<2, 2>::SMEM);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_gemm_bf16x<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)GemmCfg<3>::SMEM);
  if (e != cudaSuccess) return e;
#define DCOPF_PAIR_SMEM(NP, BN)                                                                     \
  if ((e = cudaFuncSetAttribute(k_gemm_pair<NP, BN, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                (int)PairCfg<NP, BN>::SMEM)) != cudaSuccess ||                         \
      (e = cudaFuncSetAttribute(k_gemm_pair<NP, BN, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                (int)PairCfg<NP, BN>::SMEM)) != cudaSuccess)                           \
    return e;
  DCOPF_PAIR_SMEM(2, 256)
  DCOPF_PAIR_SMEM(3, 256)
  DCOPF_PAIR_SMEM(2, 192)
  DCOPF_PAIR_SMEM(3, 192)
  DCOPF_PAIR_SMEM(2, 160)
  DCOPF_PAIR_SMEM(3, 160)
  DCOPF_PAIR_SMEM(2, 144)
  DCOPF_PAIR_SMEM(3, 144)
#undef DCOPF_PAIR_SMEM
  return cudaSuccess;
}

// The CTA-pair products: clusters of two CTAs, grid (2 x pair columns, pair rows, splits).
template <int NPROD, int PBN>
static cudaError_t launch_gemm_pair(dcopf_dual* h, const CUtensorMap& Ah, const CUtensorMap& Al,
                                    const CUtensorMap& Bh, const CUtensorMap& Bl, GemmArgs g, int splits,
                                    cudaStream_t s, int mc) {
  // mc = 2: two pairs per cluster share their A boxes (the column tiles rounded up to an
  // even count; a tile past N loads zeros and stores nothing)
  const int pairs = (g.N + PBN - 1) / PBN;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(2 * ((pairs + mc - 1) / mc * mc), (g.M + PBM - 1) / PBM, splits);
  cfg.blockDim = dim3(192);
  cfg.dynamicSmemBytes = PairCfg<NPROD, PBN>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2 * mc;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  h->launches += 1;
  if (mc == 2) return cudaLaunchKernelEx(&cfg, k_gemm_pair<NPROD, PBN, 2>, Ah, Al, Bh, Bl, g);
  return cudaLaunchKernelEx(&cfg, k_gemm_pair<NPROD, PBN, 1>, Ah, Al, Bh, Bl, g);
}

template <int NPROD, int OCC = 1>
static cudaError_t launch_gemm(dcopf_dual* h, const CUtensorMap& Ah, const CUtensorMap& Al,
                               const CUtensorMap& Bh, const CUtensorMap& Bl, GemmArgs g, int splits,
                               cudaStream_t s) {
  using Cfg = GemmCfg<NPROD, OCC>;
  dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM, splits);
  k_gemm_bf16x<NPROD, OCC><<<grid, 192, Cfg::SMEM, s>>>(Ah, Al, Bh, Bl, g);
  h->launches += 1;
  return cudaGetLastError();
}

// The adjoint Pi~ = H Phi~ (split-K partials) and the forward F = X Phi~^T, each on
// single CTAs or on CTA pairs.
// The lines a batched solve iterates on: every line of the network, or the lines a
// constraint screen kept (k_screen.cu), with the operands, limits and base flows of
// those lines in compact [*][nl] layouts.
struct LineSet {
  int nl = 0, ld_l = 0;            // lines iterated on, row stride of [*][nl] BF16 operands
  const CUtensorMap *H_hi = nullptr, *H_lo = nullptr;   // adjoint A operand [B][ld_l]
  const CUtensorMap *phit_hi = nullptr, *phit_lo = nullptr, *phit_hi96 = nullptr, *phit_lo96 = nullptr;
  const CUtensorMap *phi_hi = nullptr, *phi_lo = nullptr, *phi_hi96 = nullptr, *phi_lo96 = nullptr;
  const CUtensorMap *phit_hi80 = nullptr, *phit_lo80 = nullptr, *phi_hi80 = nullptr, *phi_lo80 = nullptr;
  const CUtensorMap *phit_hi72 = nullptr, *phit_lo72 = nullptr, *phi_hi72 = nullptr, *phi_lo72 = nullptr;
  const float* fmax = nullptr;     // [nl]
  const float* fmin = nullptr;
  const float* f0 = nullptr;       // [B][nl] base flows
  const int* kept = nullptr;       // [nl] network line of each row (null: all lines)
  const int* pos = nullptr;        // [n_line] row of each line or -1 (null: all lines)
  int blocked = 0;                 // the B operands' maps are 4-D over 8-row blocks
};

static LineSet full_lines(dcopf_dual* h) {
  TensorOps& T = h->tops;
  LineSet L;
  L.nl = h->host.n_line;
  L.ld_l = T.ld_l;
  L.H_hi = &T.m_H_hi; L.H_lo = &T.m_H_lo;
  L.phit_hi = &T.m_phit_hi; L.phit_lo = &T.m_phit_lo; L.phit_hi96 = &T.m_phit_hi96; L.phit_lo96 = &T.m_phit_lo96;
  L.phi_hi = &T.m_phi_hi; L.phi_lo = &T.m_phi_lo; L.phi_hi96 = &T.m_phi_hi96; L.phi_lo96 = &T.m_phi_lo96;
  L.phit_hi80 = &T.m_phit_hi80; L.phit_lo80 = &T.m_phit_lo80; L.phi_hi80 = &T.m_phi_hi80; L.phi_lo80 = &T.m_phi_lo80;
  L.phit_hi72 = &T.m_phit_hi72; L.phit_lo72 = &T.m_phit_lo72; L.phi_hi72 = &T.m_phi_hi72; L.phi_lo72 = &T.m_phi_lo72;
  L.fmax = h->dev.fmax32;
  L.fmin = h->dev.fmin32;
  L.f0 = h->ws.f0_32.as<float>();
  L.blocked = 1;
  return L;
}

// `tiles`: 0 single CTAs (128 x 128), 1 / 2 / 3 / 4 CTA pairs of 256 x 256 / 192 / 160 / 144.
// Ah / Al: the A operand's rows (the batch's, or one group's of it).
// `tiles` 5 .. 8: the widths of 1 .. 4 with two pairs per cluster sharing A.
static cudaError_t launch_adjoint(dcopf_dual* h, const LineSet& L, const CUtensorMap& Ah, const CUtensorMap& Al,
                                  const GemmArgs& g, int splits, int tiles, cudaStream_t s) {
  const int mc = tiles > 4 ? 2 : 1, w = tiles > 4 ? tiles - 4 : tiles;
  if (w == 1) return launch_gemm_pair<3, 256>(h, Ah, Al, *L.phit_hi, *L.phit_lo, g, splits, s, mc);
  if (w == 2) return launch_gemm_pair<3, 192>(h, Ah, Al, *L.phit_hi96, *L.phit_lo96, g, splits, s, mc);
  if (w == 3) return launch_gemm_pair<3, 160>(h, Ah, Al, *L.phit_hi80, *L.phit_lo80, g, splits, s, mc);
  if (w == 4) return launch_gemm_pair<3, 144>(h, Ah, Al, *L.phit_hi72, *L.phit_lo72, g, splits, s, mc);
  return launch_gemm<3>(h, Ah, Al, *L.phit_hi, *L.phit_lo, g, splits, s);
}
static cudaError_t launch_forward(dcopf_dual* h, const LineSet& L, const CUtensorMap& Ah, const CUtensorMap& Al,
                                  const GemmArgs& g, int tiles, cudaStream_t s) {
  const int mc = tiles > 4 ? 2 : 1, w = tiles > 4 ? tiles - 4 : tiles;
  if (h->host.qp) {
    if (w == 1) return launch_gemm_pair<3, 256>(h, Ah, Al, *L.phi_hi, *L.phi_lo, g, 1, s, mc);
    if (w == 2) return launch_gemm_pair<3, 192>(h, Ah, Al, *L.phi_hi96, *L.phi_lo96, g, 1, s, mc);
    if (w == 3) return launch_gemm_pair<3, 160>(h, Ah, Al, *L.phi_hi80, *L.phi_lo80, g, 1, s, mc);
    if (w == 4) return launch_gemm_pair<3, 144>(h, Ah, Al, *L.phi_hi72, *L.phi_lo72, g, 1, s, mc);
    return launch_gemm<3>(h, Ah, Al, *L.phi_hi, *L.phi_lo, g, 1, s);
  }
  if (w == 1) return launch_gemm_pair<2, 256>(h, Ah, Al, *L.phi_hi, *L.phi_lo, g, 1, s, mc);
  if (w == 2) return launch_gemm_pair<2, 192>(h, Ah, Al, *L.phi_hi96, *L.phi_lo96, g, 1, s, mc);
  if (w == 3) return launch_gemm_pair<2, 160>(h, Ah, Al, *L.phi_hi80, *L.phi_lo80, g, 1, s, mc);
  if (w == 4) return launch_gemm_pair<2, 144>(h, Ah, Al, *L.phi_hi72, *L.phi_lo72, g, 1, s, mc);
  // the LP forward on single CTAs (two products: x is exact in BF16): its K = n_gen is
  // short, so a CTA spends much of its time in the epilogue; two CTAs per SM (a 2-stage
  // ring each) let one CTA's epilogue run beside the other's main loop
  return launch_gemm<2, 2>(h, Ah, Al, *L.phi_hi, *L.phi_lo, g, 1, s);
}

// Split-K factor of the adjoint over nl lines: enough CTAs to cover the SMs twice.
static void adjoint_split(const dcopf_dual* h, int B, int nl, int* splits, int* kbps) {
  const int tiles = ((B + GBM - 1) / GBM) * ((h->host.n_gen + GBN - 1) / GBN);
  const int kb = (nl + GBK - 1) / GBK;
  int s = std::max(1, std::min(kb, std::min(64, (2 * h->sm_count + tiles - 1) / tiles)));
  int per = (kb + s - 1) / s;
  *kbps = per;
  *splits = (kb + per - 1) / per;
}

// dcopf_dual_eval with BF16 split tensor-core products.
dcopf_status run_eval_tensor(dcopf_dual* h, int B, const int* outage, const double* lambda,
                             const double* mh, const double* ml, double* value, double* glam,
                             double* ghi, double* glo, double* dispatch, cudaStream_t s) {
  dcopf_status r;
  if ((r = ensure_tensor_operands(h)) || (r = ensure_tensor_batch(h, B))) return r;
  TensorOps& T = h->tops;
  Workspace& w = h->ws;
  const int nl = h->host.n_line, ng = h->host.n_gen;
  k_split_eta<double><<<B, 256, 0, s>>>(nl, T.ld_l, mh, ml, outage, w.u32.as<float>(),
                                        T.H_hi.as<__nv_bfloat16>(), T.H_lo.as<__nv_bfloat16>());
  h->launches += 1;
  int splits, kbps;
  adjoint_split(h, B, nl, &splits, &kbps);
  const LineSet L = full_lines(h);
  int pair_adj = (h->tiles_mode >= 2 && B > GBM) ? h->tiles_mode - 1 : 0, pair_fwd = pair_adj;
  if (h->tune_B == B && h->tune_nl == nl && h->tune_splits > 0 && h->tune_branches == 1) {
    // the shapes a solve of this batch chose
    splits = h->tune_splits;
    kbps = h->tune_kbps;
    pair_adj = h->tune_pair_adj;
    pair_fwd = h->tune_pair_fwd;
  }
  GemmArgs g{};
  g.M = B; g.N = ng; g.K = nl; g.kb_per_split = kbps; g.epi = EPI_PARTIAL;
  g.P = T.P.as<float>(); g.ldp = (ng + 3) & ~3; g.err = h->d_err; g.timeout_ns = 2000000000ull;
  g.bblk = L.blocked;
  if (launch_adjoint(h, L, *L.H_hi, *L.H_lo, g, splits, pair_adj, s) != cudaSuccess) return DCOPF_ERR_CUDA;
  k_reduce_min<<<B, 256, 0, s>>>(h->dev, splits, B, g.ldp, T.P.as<float>(), lambda, T.ld_g,
                                 T.X_hi.as<__nv_bfloat16>(), T.X_lo.as<__nv_bfloat16>(),
                                 w.x64.as<double>(), w.sumcost.as<double>(), w.sump.as<double>());
  h->launches += 1;
  GemmArgs f{};
  f.M = B; f.N = nl; f.K = ng; f.kb_per_split = (ng + GBK - 1) / GBK; f.epi = EPI_FLOW;
  f.f0 = w.f0.as<double>(); f.f = w.f.as<double>(); f.ldf = nl; f.err = h->d_err;
  f.timeout_ns = 2000000000ull;
  f.bblk = L.blocked;
  if (launch_forward(h, L, T.m_X_hi, T.m_X_lo, f, pair_fwd, s) != cudaSuccess) return DCOPF_ERR_CUDA;
  return run_eval_finish(h, B, outage, lambda, mh, ml, value, glam, ghi, glo, dispatch, s);
}

// ------------------------------------------------------------------ for other users
bool tc_make_map(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint64_t ld) {
  return make_map(m, ptr, rows, cols, ld, GBM);
}
bool tc_make_map_rows(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t cols, uint64_t ld,
                      uint32_t box_rows) {
  return make_map(m, ptr, rows, cols, ld, box_rows);
}
bool tc_make_map_blocked(CUtensorMap* m, const void* ptr, uint64_t rows, uint64_t K, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || ((uintptr_t)ptr & 15) || box_rows % 8 || box_rows > 256) return false;
  const uint64_t kb = (K + 63) / 64, rb = (rows + 7) / 8;
  cuuint64_t dims[4] = {64, 8, kb, rb};
  cuuint64_t strides[3] = {128, 1024, kb * 1024};
  cuuint32_t box[4] = {64, 8, 1, box_rows / 8};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// P[s][m][ldp] = the K-slice s of A[m][:] . B[n][:] (BF16 hi/lo split operands, three
// products, FP32 accumulation in TMEM) for 0 <= m < M, 0 <= n < N; the number of K
// slices is chosen to fill the SMs twice (at most max_splits) and returned.
cudaError_t tc_gemm_partial(const CUtensorMap& Ah, const CUtensorMap& Al, const CUtensorMap& Bh,
                            const CUtensorMap& Bl, int M, int N, int K, float* P, int ldp,
                            int max_splits, int sm_count, int* err, int* splits_used,
                            cudaStream_t s) {
  const int tiles = ((M + GBM - 1) / GBM) * ((N + GBN - 1) / GBN);
  const int kb = (K + GBK - 1) / GBK;
  int sp = std::max(1, std::min(std::min(kb, max_splits), (2 * sm_count + tiles - 1) / tiles));
  const int per = (kb + sp - 1) / sp;
  sp = (kb + per - 1) / per;  // every slice has at least one K block
  GemmArgs g{};
  g.M = M; g.N = N; g.K = K; g.kb_per_split = per; g.epi = EPI_PARTIAL;
  g.P = P; g.ldp = ldp; g.err = err; g.timeout_ns = 2000000000ull;
  using Cfg = GemmCfg<3>;
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, sp);
  k_gemm_bf16x<3><<<grid, 192, Cfg::SMEM, s>>>(Ah, Al, Bh, Bl, g);
  *splits_used = sp;
  return cudaGetLastError();
}

// Allows the three-product GEMM its shared memory (once per process).
cudaError_t tc_gemm_prepare() {
  return cudaFuncSetAttribute(k_gemm_bf16x<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)GemmCfg<3>::SMEM);
}

template __global__ void k_split_eta<float>(int, int, const float*, const float*, const int*,
                                            const float*, __nv_bfloat16*, __nv_bfloat16*);


// Block size of the minimiser (one block per instance, at most 512 threads).  256
// threads unless the batch exceeds the blocks of that size the SMs hold at once (four
// per SM at 64 registers); then 128, which halves the waves for twice the generators
// per thread.  Measured on the same machine: 1024 4600-bus instances 175.7 -> 170.8 us
// per batched iteration, 4096 2000-bus ones 438.8 -> 421.1 us, while 256 4600-bus or
// 10000-bus instances run slower with 128 (4992 -> 4780 instances/s to the gap;
// 194.7 -> 208.9 us).  A batch that leaves SMs idle with thousands of generators per
// instance (the 10000-bus batch of 256) takes 512 threads instead: fewer generators
// per thread on the same single wave.
constexpr int MIN_MAX_THREADS = 512;
static int minimize_threads(const dcopf_dual* h, int B) {
  if (B > 4 * h->sm_count) return 128;
  return (h->host.n_gen >= 1024 && B <= 2 * h->sm_count) ? MIN_MAX_THREADS : 256;
}

// ------------------------------------------------------------------ batched solve
// pi~ from the split-K partials, minimiser, BF16 split of x, per-instance cost and
// dispatch, the pre-outage flow (Phi~ x)_k of an outaged line, the step factors of
// this step (running powers), and the lambda step (Section 3.3).
template <int SG, int MG>
__device__ __forceinline__ void minimize_item(const DevNet& N, int splits, int M, int ldp,
                                              const float* __restrict__ P, const SolveStateBase& st,
                                              const BatchView& bb, const StepArgs& SP, int ldx,
                                              __nv_bfloat16* __restrict__ Xh, __nv_bfloat16* __restrict__ Xl,
                                              const int* __restrict__ outage,
                                              const double* __restrict__ demand, int max_iters, double tol,
                                              int b, double* red) {
  // Warp 0 first runs the value and stop tests of the point the last step evaluated,
  // while the other warps start on the generators (whose terms do not depend on them);
  // the block's step at the end is skipped if those tests stopped the instance.  With
  // the mean of the minimisers on, whose weight is the iteration count the tests
  // advance, every warp waits for them instead.  (pend and frozen are read by every
  // thread before warp 0 changes them; an instance frozen on entry has nothing pending.)
  // Every per-instance scalar that the generator warps need is loaded here, with pend
  // and frozen, in one round trip (none of them is written by the tests: ueta is, but it
  // is only used when nothing is pending).
  const int pend = bb.pend[b];
  const int frozen0 = bb.frozen[b];
  const int k = outage ? outage[b] : -1;
  const float ueta_st = outage ? bb.ueta[b] : 0.f;
  const double lam = st.lam[b];
  __syncthreads();
  if (frozen0) return;
  // warp 0, lane 0: whether its tests froze the instance
  int froze = 0;
  if (pend && threadIdx.x < 32) {
    froze = finalize_instance(b, (int)threadIdx.x, max_iters, tol, st, bb, demand);
    if (threadIdx.x == 0) bb.pend[b] = 0;
  }
  if (st.xsum) {
    __syncthreads();
    if (bb.frozen[b]) return;
  }
  const int ng = N.n_gen;
  // the outaged line's term of the adjoint: the step left its multiplier difference out
  // of H (0 there) and its u^T eta in the slices' partials (summed here in the value
  // tests' order, so that it is their ueta), else ueta holds it (0 before the first step,
  // when H holds it)
  float ueta = 0.f;
  if (k >= 0) {
    if (pend) {
      const int nt = bb.n_tiles, ln = threadIdx.x & 31;
      double os = 0.0;
      for (int q = ln; q < nt; q += 32) os += bb.out_part[(size_t)b * nt + q];
      ueta = (float)warp_sum(os);
    } else {
      ueta = ueta_st;
    }
  }
  // The in-loop value and the lambda gradient only steer the iteration (the bound is
  // certified in FP64 later): per-generator terms and warp sums in FP32, FP64 across
  // warps.  The reduced cost w = ctil + sigma lambda + pi~ is formed in FP32: its
  // rounding there (a few 2^-24 of |ctil| + |sigma lambda|) is far below the error of
  // the split BF16 products that give pi~.
  const float lamf = (float)lam;
  float c = 0.f, p = 0.f, to = 0.f;
  float wk = 0.f;  // weight of the mean of the minimisers, (iteration + 1)^2
  if (st.xsum || st.wsum) {
    const float kk = (float)(st.iter[b] + 1);
    wk = kk * kk;
  }
  // MG generators per thread and pass, every split-K partial of a group of SG splits in
  // flight before the arithmetic, summed in split order (a missing term adds +0).  While
  // warp 0 runs the value and stop tests, the other warps take all the generators.
  const bool w0_busy = pend && !st.xsum;
  const int nt = w0_busy ? (int)blockDim.x - 32 : (int)blockDim.x;
  const int tg = w0_busy ? (int)threadIdx.x - 32 : (int)threadIdx.x;
  auto gen = [&](int j, float sj) {
    const float4 g = N.gen4[j];   // sigma, ctil, mq, cconst
    const float2 g2 = N.gen2[j];  // mid, 1 / (2 mq) (0 for a linear cost)
    if (k >= 0) sj = fmaf(N.phi32[(size_t)k * ng + j], ueta, sj);
    const float w = fmaf(g.x, lamf, g.y) + sj;
    // the closed-form minimiser of eq. (6) / (16) on the normalised box [-1, 1]
    const float x = g.z > 0.f ? fminf(1.f, fmaxf(-1.f, -w * g2.y)) : (w > 0.f ? -1.f : (w < 0.f ? 1.f : 0.f));
    if (st.xsum) st.xsum[(size_t)b * ng + j] += wk * x;
    split_bf16(x, Xh + (size_t)b * ldx + j, Xl + (size_t)b * ldx + j);
    c += fmaf(fmaf(g.z, x, g.y), x, g.w);
    p += fmaf(g.x, x, g2.x);
    if (k >= 0) to = fmaf(N.phi32[(size_t)k * ng + j], x, to);
  };
  for (int j0 = tg; tg >= 0 && j0 < ng; j0 += MG * nt) {
    float sg[MG];
#pragma unroll
    for (int u = 0; u < MG; ++u) sg[u] = 0.f;
    for (int q0 = 0; q0 < splits; q0 += SG) {
      float t[SG][MG];
#pragma unroll
      for (int v = 0; v < SG; ++v)
#pragma unroll
        for (int u = 0; u < MG; ++u) {
          const int j = j0 + u * nt;
          t[v][u] = (q0 + v < splits && j < ng) ? P[((size_t)(q0 + v) * M + b) * ldp + j] : 0.f;
        }
#pragma unroll
      for (int v = 0; v < SG; ++v)
#pragma unroll
        for (int u = 0; u < MG; ++u) sg[u] += t[v][u];
    }
#pragma unroll
    for (int u = 0; u < MG; ++u)
      if (j0 + u * nt < ng) gen(j0 + u * nt, sg[u]);
  }
  c = warp_sum(c); p = warp_sum(p); to = warp_sum(to);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int RW = MIN_MAX_THREADS / 32;
  // the lambda step's state, loaded by the thread that takes the step before it waits
  // for the other warps
  double pw0 = 0.0, pw1 = 0.0, pw2 = 0.0, ls1 = 0.0, ls2 = 0.0, dem = 0.0;
  if (threadIdx.x == 0) {
    pw0 = bb.pw[3 * b];
    pw1 = bb.pw[3 * b + 1];
    pw2 = bb.pw[3 * b + 2];
    ls1 = st.lam_s1[b];
    ls2 = st.lam_s2[b];
    dem = demand[b];
  }
  if (lane == 0) { red[wid] = c; red[RW + wid] = p; red[2 * RW + wid] = to; }
  __syncthreads();
  if (wid == 0) {
    // the warps' partials in FP64, a shuffle tree over lanes (fixed order)
    const int nw = (int)(blockDim.x >> 5);
    double cs = lane < nw ? red[lane] : 0.0, ps = lane < nw ? red[RW + lane] : 0.0,
           ts = lane < nw ? red[2 * RW + lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cs += __shfl_xor_sync(0xffffffffu, cs, o);
      ps += __shfl_xor_sync(0xffffffffu, ps, o);
      ts += __shfl_xor_sync(0xffffffffu, ts, o);
    }
    if (lane != 0) return;
    if (froze) return;  // stopped by this kernel's value tests
    bb.cost[b] = cs;
    bb.psum[b] = ps;
    if (st.wsum) st.wsum[b] += (double)wk;
    bb.tout[b] = (float)ts;
    bb.lam_eval[b] = lam;
    // step t = iter + 1: scale decay^(t-1), bias corrections 1 - beta^t
    const double d = pw0, b1 = pw1 * SP.beta1, b2 = pw2 * SP.beta2;
    const float bc1 = (float)(1.0 - b1), bc2 = (float)(1.0 - b2);
    const float am = (float)(SP.alpha * d);
    bb.stepf[4 * b] = am;
    bb.stepf[4 * b + 1] = am / bc1;             // Adam: alpha decay^(t-1) / (1 - beta1^t)
    bb.stepf[4 * b + 2] = 1.0f / sqrtf(bc2);    // and 1 / sqrt(1 - beta2^t)
    bb.pw[3 * b] = d * SP.decay;
    bb.pw[3 * b + 1] = b1;
    bb.pw[3 * b + 2] = b2;
    // lambda's step: the moments and lambda in FP64, the Adam / AdaGrad direction in
    // FP32 (FP64 division and square root are slow on this part)
    const double g = ps - dem, a = SP.alpha_lambda * d;
    double s1 = ls1, s2 = ls2, l = lam;
    if (SP.rule == DCOPF_GDM) {
      s1 = SP.rho * s1 + a * g;
      l += s1;
      if (SP.as_printed) l += a * g;
    } else if (SP.rule == DCOPF_ADAM) {
      s1 = SP.beta1 * s1 + (1.0 - SP.beta1) * g;
      s2 = SP.beta2 * s2 + (1.0 - SP.beta2) * g * g;
      l += a * (double)(((float)s1 / bc1) / (sqrtf((float)s2 / bc2) + (float)SP.eps));
    } else {
      s1 += g * g;
      l += a * (double)((float)g / (sqrtf((float)s1) + (float)SP.eps));
    }
    st.lam[b] = l;
    st.lam_s1[b] = s1;
    st.lam_s2[b] = s2;
  }
}

// The minimiser kernel: instance b taken in turn by the launched blocks (one per
// instance, or fewer to leave room for another instance group's products).
__global__ void __launch_bounds__(MIN_MAX_THREADS, 2)
    k_bt_minimize(DevNet N, int splits, int M, int ldp, const float* __restrict__ P,
                  SolveStateBase st, BatchView bb, StepArgs SP, int ldx,
                  __nv_bfloat16* __restrict__ Xh, __nv_bfloat16* __restrict__ Xl,
                  const int* __restrict__ outage, const double* __restrict__ demand, int max_iters,
                  double tol) {
  __shared__ double red[3 * (MIN_MAX_THREADS / 32)];
  for (int b = blockIdx.x; b < M; b += gridDim.x) {
    if (splits <= 4)
      minimize_item<4, 6>(N, splits, M, ldp, P, st, bb, SP, ldx, Xh, Xl, outage, demand, max_iters, tol, b, red);
    else
      minimize_item<3, 6>(N, splits, M, ldp, P, st, bb, SP, ldx, Xh, Xl, outage, demand, max_iters, tol, b, red);
    __syncthreads();  // red is read by warp 0 before the next instance's partials land
  }
}

// Dual value of the evaluated point (FP64), best value and its lambda, u^T eta of the
// point stepped to, stop tests, for instance b, by one warp: of the next iteration's
// minimiser block for the instance, or of the end-of-round kernel.  A stopping instance
// is frozen: one that reached its target with the point just evaluated (state buffer
// iter % 3), one stopped by the iteration cap or the tol test with its best point.
// Lane 0 loads the instance's scalars before the partial sums (one round trip for
// both) and returns 1 if the tests froze the instance (0 on the other lanes).
__device__ __forceinline__ int finalize_instance(int b, int lane, int max_iters, double tol,
                                                 const SolveStateBase& st, const BatchView& bb,
                                                 const double* __restrict__ demand) {
  const int nt = bb.n_tiles;
  double cost = 0.0, lam_e = 0.0, psum = 0.0, dem = 0.0, best = 0.0, prev = 0.0, thr = 0.0;
  int iter = 0;
  if (lane == 0) {
    cost = bb.cost[b];
    lam_e = bb.lam_eval[b];
    psum = bb.psum[b];
    dem = demand[b];
    best = st.best[b];
    prev = st.prev[b];
    iter = st.iter[b];
    if (st.has_target) thr = st.thresh[b] + st.margin[b];
  }
  double ls = 0.0, os = 0.0;
  for (int q = lane; q < nt; q += 32) {
    ls += bb.line_part[(size_t)b * nt + q];
    os += bb.out_part[(size_t)b * nt + q];
  }
  ls = warp_sum(ls);
  os = warp_sum(os);
  if (lane != 0) return 0;
  const double val = cost + lam_e * (psum - dem) + ls;
  const int t = iter + 1;
  if (val > best) { st.best[b] = val; st.best_iter[b] = t; bb.lam_best[b] = lam_e; }
  // u^T eta of the point stepped to, the outaged line's multiplier difference in the
  // post-outage adjoint: the next minimiser adds its column of the product
  bb.ueta[b] = (float)os;
  int c = 0;
  if (st.has_target && val >= thr) c = 1;
  else if (t >= max_iters) c = 2;
  else if (tol > 0.0 && t > 1 && fabs(val - prev) < tol) c = 2;
  st.prev[b] = val;
  if (c) {
    st.cand[b] = c;
    bb.frozen[b] = 1;
    st.best_lam[b] = c == 1 ? lam_e : bb.lam_best[b];
    return 1;
  }
  st.iter[b] = t;
  return 0;
}

// The value and stop tests of the points the last step of a round evaluated (those
// the next round's first minimiser would otherwise take), so that the round's staging
// sees them.  One warp per instance.
__global__ void k_bt_finalize(int B, int max_iters, double tol, SolveStateBase st, BatchView bb,
                              const double* __restrict__ demand) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (b >= B) return;
  if (!__shfl_sync(0xffffffffu, lane == 0 ? bb.pend[b] : 0, 0)) return;
  finalize_instance(b, lane, max_iters, tol, st, bb, demand);
  if (lane == 0) bb.pend[b] = 0;
}

// Stages the frozen candidates whose certificate is not already pending (snap_prev,
// the set of the round before): snap[b] = 1 for each (the certificate and, two rounds
// later, the accept step act on exactly those, while the next rounds' iterations may
// freeze others), and copies each one's point into rows of dh / dl ([B][len]): its compact row
// (pos null, len = nl) or, behind a constraint screen, its full-length row (len = n_line,
// pos the compact row of each line or -1, zero on the screened lines).  A candidate that
// reached its target is the point just evaluated (state buffer iter % 3); one stopped by
// the iteration cap or the tol test is its best point: point iter or iter - 1 (still in
// their buffers) or an older one (its saved copy).
__global__ void k_bt_stage(int B, int nl, int len, const int* __restrict__ pos, SolveState<float> st,
                           BatchView bb, int* snap, const int* __restrict__ snap_prev, float* __restrict__ dh,
                           float* __restrict__ dl) {
  const int b = blockIdx.y;
  const bool staged = st.cand[b] && !st.done[b] && !snap_prev[b];
  if (blockIdx.x == 0 && threadIdx.x == 0) snap[b] = staged ? 1 : 0;
  if (!staged) return;
  const int it = st.iter[b];
  // how many points before the last one the staged point is (0 with no best yet)
  const int back = (st.cand[b] == 1 || st.best_iter[b] < 1) ? 0 : it + 1 - st.best_iter[b];
  const float* bh[3] = {st.mu_hi, bb.mu2_hi, bb.mu3_hi};
  const float* bl[3] = {st.mu_lo, bb.mu2_lo, bb.mu3_lo};
  const float* sh = (back <= 1 ? bh[(it - back) % 3] : bb.sv_hi) + (size_t)b * nl;
  const float* sl = (back <= 1 ? bl[(it - back) % 3] : bb.sv_lo) + (size_t)b * nl;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
    const int r = pos ? pos[i] : i;
    dh[(size_t)b * len + i] = r >= 0 ? sh[r] : 0.f;
    dl[(size_t)b * len + i] = r >= 0 ? sl[r] : 0.f;
  }
}

// After certification: accept, stop, or unfreeze with a larger in-loop margin each
// staged instance (when `accept`; the evaluation of a frozen point counts, and an
// unfrozen instance moves on to the point already stepped to); then the number of
// instances still running into *out_active, the device error word into *out_err and
// the re-screen flag (error word [1]) into *out_flag.  One block.
constexpr int ACCEPT_THREADS = 512;
__global__ void __launch_bounds__(ACCEPT_THREADS)
    k_bt_accept(int B, int accept, double ub_any, SolveStateBase st, BatchView bb,
                const int* __restrict__ snap, const int* __restrict__ err, int* out_active,
                int* out_err, int* out_flag, int* out_iter) {
  __shared__ int red[ACCEPT_THREADS / 32], red2[ACCEPT_THREADS / 32];
  int running = 0, iterating = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    if (accept && snap[b] && !st.done[b] && st.cand[b]) {
      const double c = st.cert[b];
      if (st.cand[b] == 1) {
        if (c >= st.thresh[b]) {
          st.done[b] = 1;
          st.status[b] = 0;
        } else {
          st.margin[b] += fmax(st.thresh[b] - c, 1e-7 * fabs(st.thresh[b]));
          st.cand[b] = 0;
          bb.frozen[b] = 0;
        }
      } else {
        st.done[b] = 1;
        st.status[b] = (c >= st.thresh[b]) ? 0 : 1;
      }
      if (c > ub_any) { st.done[b] = 1; st.status[b] = 2; bb.frozen[b] = 1; }
      st.iter[b] += 1;
    }
    running += st.done[b] ? 0 : 1;
    iterating += bb.frozen[b] ? 0 : 1;
  }
  running = __reduce_add_sync(0xffffffffu, running);
  iterating = __reduce_add_sync(0xffffffffu, iterating);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = running;
    red2[threadIdx.x >> 5] = iterating;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0, m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      n += red[w];
      m += red2[w];
    }
    *out_active = n;
    *out_err = err[0];
    *out_flag = err[1];
    *out_iter = m;
  }
}

__global__ void k_bt_init(int B, BatchView bb) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    bb.frozen[b] = 0;
    bb.pend[b] = 0;
    bb.ueta[b] = 0.f;
    bb.pw[3 * b] = 1.0;
    bb.pw[3 * b + 1] = 1.0;
    bb.pw[3 * b + 2] = 1.0;
  }
}

static dcopf_status ensure_batch_bufs(dcopf_dual* h, int B, int n_tiles) {
  BatchBufs& bb = h->bb;
  BatchView& v = bb.v;
  const size_t nl = h->host.n_line;
  if (bb.mu2.alloc((size_t)B * nl * 6 * sizeof(float)) ||
      bb.parts.alloc((size_t)B * n_tiles * 2 * sizeof(double)) ||
      bb.small.alloc((size_t)B * 7 * sizeof(double) + (size_t)B * 8 * sizeof(float) + 1024)) {
    cudaGetLastError();
    return DCOPF_ERR_OOM;
  }
  v.mu2_hi = bb.mu2.as<float>();
  v.mu2_lo = v.mu2_hi + (size_t)B * nl;
  v.mu3_hi = v.mu2_hi + 2 * (size_t)B * nl;
  v.mu3_lo = v.mu2_hi + 3 * (size_t)B * nl;
  v.sv_hi = v.mu2_hi + 4 * (size_t)B * nl;
  v.sv_lo = v.mu2_hi + 5 * (size_t)B * nl;
  v.line_part = bb.parts.as<double>();
  v.out_part = v.line_part + (size_t)B * n_tiles;
  double* d = bb.small.as<double>();
  v.lam_eval = d; v.cost = d + B; v.psum = d + 2 * (size_t)B; v.pw = d + 3 * (size_t)B;  // pw: [B][3]
  v.lam_best = d + 6 * (size_t)B;
  float* f = (float*)(d + 7 * (size_t)B);
  v.tout = f; v.stepf = f + B;  // stepf: [B][4]
  v.frozen = (int*)(f + 5 * (size_t)B);
  v.pend = (int*)(f + 6 * (size_t)B);
  v.ueta = f + 7 * (size_t)B;
  v.n_tiles = n_tiles;
  return DCOPF_OK;
}

// One group of a batch's instances, [b0, b0 + B): the kernel arguments of its
// iteration chain, every per-instance pointer advanced to the group's first instance.
struct IterView {
  int b0 = 0, B = 0;
  SolveState<float> st{};
  BatchView bb{};
  GemmArgs ga{}, gf{};
  StepEpi E{};
  CUtensorMap Hh{}, Hl{}, Xh{}, Xl{};  // the group's rows of the two products' A operands
  const int* outage = nullptr;         // [B] or null
  const double* demand = nullptr;      // [B]
  __nv_bfloat16 *Xhp = nullptr, *Xlp = nullptr, *Hhp = nullptr, *Hlp = nullptr;
};
// A batch runs as one group, or as two whose iteration chains are parallel branches of
// the iteration graph: one group's HBM-bound step and latency-bound minimiser then run
// beside the other's tensor-core products.
constexpr int MAX_BRANCHES = 2;

// Product shapes of the batched iteration, as launch_adjoint's `tiles`.
struct TensorShapes {
  int adj = 0, splits = 1, kbps = 1, fwd = 0;
};
// The tuner's two fastest adjoint shapes and forward tiles, each timed on its own.
struct ShapeChoices {
  TensorShapes best;
  int adj2 = -1, splits2 = 1, kbps2 = 1;  // the second adjoint (adj2 < 0: none)
  int fwd2 = -1;                          // the second forward (< 0: none)
};

// One network's share of a batched tensor-core solve: the instances, the kernel
// arguments of one iteration, and the solve state.
struct TensorRun {
  TensorItem it{};
  dcopf_solve_params p{};
  SolveState<float> st{};
  StepArgs P{};
  GemmArgs ga{}, gf{};
  StepEpi E{};
  int splits = 1, n_tiles = 0;
  int pair_adj = 0, pair_fwd = 0;  // product shapes, as launch_adjoint's `tiles`
  LineSet ls;                      // the lines iterated on
  unsigned gi = 1;
  bool running = true;
  int nv = 1;                      // instance groups, iterated as parallel graph branches
  IterView v[MAX_BRANCHES];
  // blocks of the step and the minimiser kernels (0: one per work item); with two
  // groups, two step blocks and one minimiser block per SM, which leaves each SM the
  // registers of a product CTA of the other group
  int step_blocks = 0, min_blocks = 0;
};

template <typename T>
static void adv(T*& p, size_t n) {
  if (p) p += n;
}

// The view of instances [b0, b0 + Bg) of R's batch.
static bool make_view(TensorRun& R, int b0, int Bg, IterView* V) {
  dcopf_dual* h = R.it.h;
  TensorOps& T = h->tops;
  const size_t nl = R.ls.nl, ng = h->host.n_gen, nt = R.n_tiles, o = b0;
  IterView& W = *V;
  W = IterView{};
  W.b0 = b0;
  W.B = Bg;
  SolveState<float>& st = W.st;
  st = R.st;
  adv(st.s, o * ng); adv(st.s1_s, o * ng); adv(st.s2_s, o * ng);
  for (int** q : {&st.done, &st.cand, &st.iter, &st.best_iter, &st.status}) adv(*q, o);
  for (double** q : {&st.best, &st.best_next, &st.best_lam, &st.thresh, &st.margin, &st.prev,
                     &st.prev2, &st.lam, &st.lam_s1, &st.lam_s2, &st.cert, &st.wsum})
    adv(*q, o);
  adv(st.xsum, o * ng);
  for (float** q : {&st.mu_hi, &st.mu_lo, &st.s1_hi, &st.s2_hi, &st.s1_lo, &st.s2_lo, &st.best_hi,
                    &st.best_lo})
    adv(*q, o * nl);
  BatchView& bb = W.bb;
  bb = h->bb.v;
  adv(bb.frozen, o); adv(bb.lam_eval, o); adv(bb.cost, o); adv(bb.psum, o); adv(bb.pw, 3 * o);
  adv(bb.tout, o); adv(bb.stepf, 4 * o); adv(bb.lam_best, o); adv(bb.pend, o); adv(bb.ueta, o);
  for (float** q : {&bb.mu2_hi, &bb.mu2_lo, &bb.mu3_hi, &bb.mu3_lo, &bb.sv_hi, &bb.sv_lo}) adv(*q, o * nl);
  adv(bb.line_part, o * nt); adv(bb.out_part, o * nt);
  W.ga = R.ga;
  W.ga.M = Bg;
  W.ga.P = R.ga.P + (size_t)64 * o * R.ga.ldp;  // the partials' [64][B][ldp] share of the group
  W.ga.skip = bb.frozen;
  W.gf = R.gf;
  W.gf.M = Bg;
  W.gf.F32 = R.gf.F32 + o * R.gf.ldf32;
  W.gf.skip = bb.frozen;
  StepEpi& E = W.E;
  E = R.E;
  E.F = R.E.F + o * R.E.ldF;
  E.f0 = R.E.f0 + o * nl;
  adv(E.u, o * nl);
  adv(E.outage, o);
  E.tout = bb.tout; E.iter = st.iter; E.frozen = bb.frozen; E.best_iter = st.best_iter; E.stepf = bb.stepf;
  E.mu_hi[0] = st.mu_hi; E.mu_hi[1] = bb.mu2_hi; E.mu_hi[2] = bb.mu3_hi;
  E.mu_lo[0] = st.mu_lo; E.mu_lo[1] = bb.mu2_lo; E.mu_lo[2] = bb.mu3_lo;
  E.sv_hi = bb.sv_hi; E.sv_lo = bb.sv_lo;
  E.s1_hi = st.s1_hi; E.s2_hi = st.s2_hi; E.s1_lo = st.s1_lo; E.s2_lo = st.s2_lo;
  E.Hh = R.E.Hh + o * E.ldh;
  E.Hl = R.E.Hl + o * E.ldh;
  E.line_part = bb.line_part; E.out_part = bb.out_part;
  E.B = Bg;
  E.pend = bb.pend;
  W.outage = R.it.outage ? R.it.outage + o : nullptr;
  W.demand = h->ws.demand.as<double>() + o;

  W.Xhp = T.X_hi.as<__nv_bfloat16>() + o * T.ld_g;
  W.Xlp = T.X_lo.as<__nv_bfloat16>() + o * T.ld_g;
  W.Hhp = E.Hh;
  W.Hlp = E.Hl;
  return make_map(&W.Hh, W.Hhp, Bg, nl, R.ls.ld_l, GBM) && make_map(&W.Hl, W.Hlp, Bg, nl, R.ls.ld_l, GBM) &&
         make_map(&W.Xh, W.Xhp, Bg, ng, T.ld_g, GBM) && make_map(&W.Xl, W.Xlp, Bg, ng, T.ld_g, GBM);
}

// The first group's size when the batch runs as two: half the batch, rounded up to
// whole 256-row pair tiles where the batch has at least 1024 instances, else to
// 128-row tiles.
int tensor_first_group(int B) {
  const int q = B >= 1024 ? 256 : 128;
  return std::min(B - 1, ((B + 1) / 2 + q - 1) / q * q);
}

// R's groups: the whole batch (nv = 1) or its two groups (nv = 2).
static dcopf_status make_views(TensorRun& R, int nv) {
  const int B = R.it.B;
  R.nv = nv;
  R.step_blocks = nv > 1 ? 2 * R.it.h->sm_count : 0;
  R.min_blocks = nv > 1 ? R.it.h->sm_count : 0;
  if (nv == 1) return make_view(R, 0, B, &R.v[0]) ? DCOPF_OK : DCOPF_ERR_CUDA;
  const int b1 = tensor_first_group(B);
  return make_view(R, 0, b1, &R.v[0]) && make_view(R, b1, B - b1, &R.v[1]) ? DCOPF_OK : DCOPF_ERR_CUDA;
}

static void apply_shapes(TensorRun& R, const TensorShapes& S) {
  R.splits = S.splits;
  R.pair_adj = S.adj;
  R.pair_fwd = S.fwd;
  for (IterView& V : R.v) V.ga.kb_per_split = S.kbps;
}

// Enqueues n iterations of group V's chain (adjoint GEMM, minimiser, forward GEMM,
// step, value) on cs; with `mark`, the timing events around the kernels of the last.
static bool enqueue_iters(TensorRun& R, IterView& V, int n, cudaStream_t cs, bool mark_last) {
  dcopf_dual* h = R.it.h;
  const int nl = R.ls.nl;
  TensorOps& T = h->tops;
  bool ok = true;
  for (int it = 0; it < n && ok; ++it) {
    // timing on: event nodes around the kernels of the round's last iteration
    const bool mark = mark_last && h->timing && h->kev[0] && it == n - 1;
    // (external event-record nodes: a plain record during capture only orders streams)
    auto ev = [&](int q) {
      if (mark) ok &= cudaEventRecordWithFlags(h->kev[q], cs, cudaEventRecordExternal) == cudaSuccess;
    };
    ev(0);
    ok &= launch_adjoint(h, R.ls, V.Hh, V.Hl, V.ga, R.splits, R.pair_adj, cs) == cudaSuccess;
    ev(1);
    const int mb = R.min_blocks ? std::min(V.B, R.min_blocks) : V.B;
    k_bt_minimize<<<mb, minimize_threads(h, V.B), 0, cs>>>(h->dev, R.splits, V.B, V.ga.ldp, V.ga.P, V.st,
                                                           V.bb, R.P, T.ld_g, V.Xhp, V.Xlp, V.outage,
                                                           V.demand, R.p.max_iters, R.p.tol);
    ev(2);
    ok &= launch_forward(h, R.ls, V.Xh, V.Xl, V.gf, R.pair_fwd, cs) == cudaSuccess;
    ev(3);
    const int blocks = (R.n_tiles * V.B + STEP_THREADS / 32 - 1) / (STEP_THREADS / 32);
    const int sb = R.step_blocks ? std::min(blocks, R.step_blocks) : blocks;
    if (nl % 4 == 0 && V.E.ldF % 4 == 0 && V.E.ldh % 4 == 0)
      k_bt_step4<<<sb, STEP_THREADS, 0, cs>>>(V.E, nl);
    else
      k_bt_step<<<sb, STEP_THREADS, 0, cs>>>(V.E, nl);
    ev(4);  // the value and stop tests run in the next minimiser (or below, for the last)
    ev(5);
  }
  // the value and stop tests of the round's last step
  k_bt_finalize<<<(V.B + 3) / 4, 128, 0, cs>>>(V.B, R.p.max_iters, R.p.tol, V.st, V.bb, V.demand);
  return ok && cudaGetLastError() == cudaSuccess;
}

// Enqueues `chunk` iterations of every group on cs (the groups after the first on the
// handle's second stream, forked from cs and joined back to it).
static bool tensor_enqueue_chunk(TensorRun& R, int chunk, cudaStream_t cs) {
  dcopf_dual* h = R.it.h;
  if (R.nv == 1) return enqueue_iters(R, R.v[0], chunk, cs, true);
  bool ok = cudaEventRecord(h->fork_ev, cs) == cudaSuccess &&
            cudaStreamWaitEvent(h->tstream2, h->fork_ev, 0) == cudaSuccess;
  ok = ok && enqueue_iters(R, R.v[0], chunk, cs, true);
  ok = ok && enqueue_iters(R, R.v[1], chunk, h->tstream2, false);
  ok = ok && cudaEventRecord(h->join_ev, h->tstream2) == cudaSuccess &&
       cudaStreamWaitEvent(cs, h->join_ev, 0) == cudaSuccess;
  return ok;
}

// Initial state (cold or warm start), per-instance flags, and the BF16 split of the
// first eta, on stream cs.
static void tensor_init_state(TensorRun& R, cudaStream_t cs) {
  dcopf_dual* h = R.it.h;
  const int B = R.it.B, nl = h->host.n_line, nk = R.ls.nl;
  TensorOps& T = h->tops;
  if (R.ls.kept) {
    // the warm start of every line into the (still unused) saved-point buffers, then
    // the rows of the kept lines into the compact state; the moments start at zero
    SolveState<float> tmp = R.st;
    tmp.mu_hi = h->bb.v.sv_hi;
    tmp.mu_lo = h->bb.v.sv_lo;
    tmp.best_hi = h->scr.full.as<float>();
    tmp.best_lo = tmp.best_hi + (size_t)B * nl;
    k_init_state_f32(R.gi, cs, B, nl, R.p.warm_start, R.it.lam, R.it.mh, R.it.ml, R.it.target, R.p.gap,
                     tmp);
    const unsigned g = (unsigned)std::min<long long>(((long long)B * nk + 255) / 256, 4096);
    k_screen_compact_rows<<<g, 256, 0, cs>>>(B, nl, nk, R.ls.kept, tmp.mu_hi, R.st.mu_hi);
    k_screen_compact_rows<<<g, 256, 0, cs>>>(B, nl, nk, R.ls.kept, tmp.mu_lo, R.st.mu_lo);
    k_screen_compact_rows<<<g, 256, 0, cs>>>(B, nl, nk, R.ls.kept, tmp.best_hi, R.st.best_hi);
    k_screen_compact_rows<<<g, 256, 0, cs>>>(B, nl, nk, R.ls.kept, tmp.best_lo, R.st.best_lo);
    h->launches += 4;
  } else {
    k_init_state_f32(R.gi, cs, B, nl, R.p.warm_start, R.it.lam, R.it.mh, R.it.ml, R.it.target, R.p.gap,
                     R.st);
  }
  k_bt_init<<<(B + 255) / 256, 256, 0, cs>>>(B, h->bb.v);
  k_split_eta<float><<<B, 256, 0, cs>>>(nk, R.ls.ld_l, R.st.mu_hi, R.st.mu_lo, R.it.outage,
                                        h->ws.u32.as<float>(), T.H_hi.as<__nv_bfloat16>(),
                                        T.H_lo.as<__nv_bfloat16>());
  h->launches += 3;
}

// Autotuner of the batched products' shapes for the instances of group V, on the
// first solve of a batch size:
//  - the adjoint: single CTAs (128 x 128 tiles) or CTA pairs (256 x 256 or 256 x 192),
//    each with split-K factors around a heuristic and the factors that fill whole
//    waves; more splits fill the SMs with CTAs but add FP32 partial traffic to the
//    minimiser's reduction, so each candidate is timed as adjoint + minimiser;
//  - the forward product: single CTAs or CTA pairs.
// Timed with CUDA events on the solve's stream; the fastest of each goes to *out.
static dcopf_status tune_view_shapes(TensorRun& R, IterView& V, cudaStream_t cs, ShapeChoices* out) {
  dcopf_dual* h = R.it.h;
  const int B = V.B, ng = h->host.n_gen;
  TensorOps& T = h->tops;
  const int kb = (R.ls.nl + GBK - 1) / GBK;
  const bool pair_ok = B > GBM && h->tiles_mode != 1;
  const bool single_ok = h->tiles_mode <= 1 || B <= GBM;
  // pair widths tried: tiles codes tv_lo .. tv_hi (all three unless DCOPF_TENSOR_TILES fixes one)
  const int tv_lo = h->tiles_mode >= 2 ? h->tiles_mode - 1 : 1, tv_hi = h->tiles_mode >= 2 ? h->tiles_mode - 1 : 4;
  struct Cand { int tiles; int splits; };  // tiles as launch_adjoint's
  std::vector<Cand> cand;
  auto add = [&](int tiles, int sp) {
    sp = std::max(1, std::min(std::min(kb, 64), sp));
    const int per = (kb + sp - 1) / sp;
    const int se = (kb + per - 1) / per;
    for (const Cand& c : cand)
      if (c.tiles == tiles && c.splits == se) return;
    cand.push_back({tiles, se});
  };
  if (single_ok) {
    int s0 = 1, kb0 = 1;
    adjoint_split(h, B, R.ls.nl, &s0, &kb0);
    for (int num : {1, 2, 3, 4, 6, 8}) add(0, (s0 * num + 2) / 4);
    // and the splits that fill whole waves (one CTA per SM): the last wave of a grid of
    // tiles x splits CTAs is then full rather than a few CTAs on an idle GPU
    const int tiles = ((B + GBM - 1) / GBM) * ((ng + GBN - 1) / GBN);
    for (int wv = 1; wv <= 4; ++wv) add(0, wv * h->sm_count / tiles);
  }
  if (pair_ok) {
    for (int tv = tv_lo; tv <= tv_hi; ++tv) {
      const int bn = tv == 1 ? 256 : tv == 2 ? 192 : tv == 3 ? 160 : 144;
      const int ptiles = ((B + PBM - 1) / PBM) * ((ng + bn - 1) / bn);
      const int slots = h->sm_count / 2;  // one pair per two SMs
      const int s0 = std::max(1, (slots + ptiles - 1) / ptiles);
      for (int mc : {0, 4})  // one pair per cluster, or two sharing A
        if (mc == 0 || ptiles >= 2) {
          for (int num : {2, 3, 4, 6}) add(tv + mc, (s0 * num + 2) / 4);
          for (int wv = 1; wv <= 3; ++wv) add(tv + mc, wv * slots / ptiles);
        }
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return DCOPF_ERR_CUDA;
  }
  auto timed = [&](auto&& body, float* ms) -> dcopf_status {
    *ms = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {  // the first pass warms up; the fastest of the others
      float t = 0.f;
      if (cudaEventRecord(e0, cs) != cudaSuccess) return DCOPF_ERR_CUDA;
      for (int k = 0; k < 3; ++k)
        if (body() != cudaSuccess) return DCOPF_ERR_CUDA;
      if (cudaEventRecord(e1, cs) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        return DCOPF_ERR_CUDA;
      if (rep > 0) *ms = std::min(*ms, t);
    }
    return DCOPF_OK;
  };
  static const char* kTiles[9] = {"single 128x128", "pairs 256x256", "pairs 256x192", "pairs 256x160",
                                  "pairs 256x144", "2 pairs 256x256", "2 pairs 256x192", "2 pairs 256x160",
                                  "2 pairs 256x144"};
  float best = 1e30f, second = 1e30f;
  Cand bc = cand.empty() ? Cand{0, 1} : cand[0], bc2{-1, 1};
  int best_per = (kb + bc.splits - 1) / bc.splits, per2 = 1;
  dcopf_status res = DCOPF_OK;
  for (const Cand& c : cand) {
    GemmArgs g = V.ga;
    g.kb_per_split = (kb + c.splits - 1) / c.splits;
    float ms = 0.f;
    res = timed(
        [&] {
          cudaError_t e = launch_adjoint(h, R.ls, V.Hh, V.Hl, g, c.splits, c.tiles, cs);
          k_bt_minimize<<<B, minimize_threads(h, B), 0, cs>>>(h->dev, c.splits, B, g.ldp, g.P, V.st, V.bb, R.P,
                                                              T.ld_g, V.Xhp, V.Xlp, V.outage, V.demand,
                                                              R.p.max_iters, R.p.tol);
          h->launches += 1;
          return e != cudaSuccess ? e : cudaGetLastError();
        },
        &ms);
    if (res != DCOPF_OK) break;
    if (h->verbose)
      fprintf(stderr, "dcopf: batch %d adjoint %s split-K %d: %.1f us per GEMM+min\n", B,
              kTiles[c.tiles], c.splits, 1e3f * ms / 3.f);
    if (ms < best) {
      second = best;
      bc2 = bc;
      per2 = best_per;
      best = ms;
      bc = c;
      best_per = g.kb_per_split;
    } else if (ms < second) {
      second = ms;
      bc2 = c;
      per2 = g.kb_per_split;
    }
  }
  if (second >= 1e30f) bc2.tiles = -1;
  // the forward product, on the operands the runs above left
  int fwd = (pair_ok && !single_ok) ? tv_lo : 0, fwd2 = -1;
  if (res == DCOPF_OK && pair_ok) {
    float bf = 1e30f, bf2 = 1e30f;
    std::vector<int> tvs;
    if (single_ok) tvs.push_back(0);
    for (int tv = tv_lo; tv <= tv_hi; ++tv) tvs.push_back(tv);
    for (int tv = tv_lo; tv <= tv_hi; ++tv) tvs.push_back(tv + 4);
    for (int tv : tvs) {
      if (res != DCOPF_OK) break;
      float ms = 0.f;
      res = timed([&] { return launch_forward(h, R.ls, V.Xh, V.Xl, V.gf, tv, cs); }, &ms);
      if (h->verbose) fprintf(stderr, "dcopf: batch %d forward %s: %.1f us\n", B, kTiles[tv], 1e3f * ms / 3.f);
      if (res == DCOPF_OK && ms < bf) {
        bf2 = bf;
        fwd2 = bf < 1e30f ? fwd : -1;
        bf = ms;
        fwd = tv;
      } else if (res == DCOPF_OK && ms < bf2) {
        bf2 = ms;
        fwd2 = tv;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (res != DCOPF_OK) return res;
  int derr = 0;
  if (cudaMemcpy(&derr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  if (derr) return (dcopf_status)derr;
  out->best = TensorShapes{bc.tiles, bc.splits, best_per, fwd};
  out->adj2 = bc2.tiles;
  out->splits2 = bc2.splits;
  out->kbps2 = per2;
  out->fwd2 = fwd2;
  if (h->verbose)
    fprintf(stderr, "dcopf: batch %d adjoint %s split-K %d (%.1f us per GEMM+min), forward %s\n", B,
            kTiles[bc.tiles], bc.splits, 1e3f * best / 3.f, kTiles[fwd]);
  return DCOPF_OK;
}

// Milliseconds of 6 whole iterations of every group of R: the fastest of three runs
// after one that warms up, each from the initial state (so that no instance has stopped
// and had its work skipped).
static dcopf_status time_iterations(TensorRun& R, cudaStream_t cs, float* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return DCOPF_ERR_CUDA;
  }
  dcopf_status res = DCOPF_OK;
  *ms = 1e30f;
  for (int rep = 0; rep < 4 && res == DCOPF_OK; ++rep) {
    float t = 0.f;
    tensor_init_state(R, cs);
    if (cudaEventRecord(e0, cs) != cudaSuccess || !tensor_enqueue_chunk(R, 6, cs) ||
        cudaEventRecord(e1, cs) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
      res = DCOPF_ERR_CUDA;
    if (rep > 0) *ms = std::min(*ms, t);
  }
  R.it.h->launches += 4LL * (6 * 2 + 1) * R.nv;  // the products count themselves
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return res;
}

// The shapes and the grouping of the batch: each grouping's product shapes by
// tune_view_shapes, then the whole iteration under each grouping, timed; the faster
// is kept per handle.
static dcopf_status tune_tensor(TensorRun& R, cudaStream_t cs) {
  dcopf_dual* h = R.it.h;
  const int B = R.it.B;
  dcopf_status r;
  ShapeChoices c1, c2;
  if ((r = make_views(R, 1)) || (r = tune_view_shapes(R, R.v[0], cs, &c1))) return r;
  int nv = 1;
  // the two fastest of each product, each timed on its own, combined and timed as whole
  // iterations: a product's time beside the others' differs from its own
  std::vector<TensorShapes> combos{c1.best};
  if (c1.adj2 >= 0) combos.push_back(TensorShapes{c1.adj2, c1.splits2, c1.kbps2, c1.best.fwd});
  if (c1.fwd2 >= 0) combos.push_back(TensorShapes{c1.best.adj, c1.best.splits, c1.best.kbps, c1.fwd2});
  if (c1.adj2 >= 0 && c1.fwd2 >= 0) combos.push_back(TensorShapes{c1.adj2, c1.splits2, c1.kbps2, c1.fwd2});
  TensorShapes best = c1.best;
  float t1 = 1e30f;
  for (const TensorShapes& c : combos) {
    float t = 0.f;
    apply_shapes(R, c);
    if ((r = time_iterations(R, cs, &t))) return r;
    if (h->verbose)
      fprintf(stderr, "dcopf: batch %d shapes %d,%d,%d: %.1f us per iteration\n", B, c.adj, c.splits, c.fwd,
              1e3f * t / 6.f);
    if (t < t1) {
      t1 = t;
      best = c;
    }
  }
  if (B >= 2 * GBM) {
    float t2 = 0.f;
    if ((r = make_views(R, 2)) || (r = tune_view_shapes(R, R.v[0], cs, &c2))) return r;
    const TensorShapes s2 = c2.best;
    apply_shapes(R, s2);
    if ((r = time_iterations(R, cs, &t2))) return r;
    if (h->verbose)
      fprintf(stderr, "dcopf: batch %d one group %.1f us, two groups %.1f us per iteration\n", B,
              1e3f * t1 / 6.f, 1e3f * t2 / 6.f);
    if (t2 < t1) {
      nv = 2;
      best = s2;
    }
  }
  h->tune_B = B;
  h->tune_nl = R.ls.nl;
  h->tune_splits = best.splits;
  h->tune_kbps = best.kbps;
  h->tune_pair_adj = best.adj;
  h->tune_pair_fwd = best.fwd;
  h->tune_branches = nv;
  return DCOPF_OK;
}

// Buffers, state initialisation and the iteration's kernel arguments; the work is
// enqueued on the handle's internal stream, ordered after the caller's stream s.
static dcopf_status tensor_setup(TensorRun& R, cudaStream_t s) {
  dcopf_dual* h = R.it.h;
  const int B = R.it.B;
  dcopf_status r;
  if ((r = ensure_tensor_operands(h)) || (r = ensure_tensor_batch(h, B))) return r;
  if ((r = ensure_state<float>(h, B, &R.st))) return r;
  const int n_line = h->host.n_line, ng = h->host.n_gen;
  TensorOps& T = h->tops;
  Workspace& w = h->ws;
  const dcopf_solve_params& p = R.p;
  R.ls = full_lines(h);
  if (p.screen_lines && !R.it.outage) {
    // constraint screening: the iterations carry only the lines that can bind
    if ((r = screen_batch(h, B, s))) return r;
    LineScreen& S = h->scr;
    const int nk = S.nk;
    if (S.f0c.alloc((size_t)B * nk * sizeof(float)) != cudaSuccess ||
        S.full.alloc((size_t)2 * B * n_line * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return DCOPF_ERR_OOM;
    }
    if (S.map_B != B) {
      if (!tc_make_map(&S.m_H_hi, T.H_hi.p, B, nk, S.ld_lk) || !tc_make_map(&S.m_H_lo, T.H_lo.p, B, nk, S.ld_lk))
        return DCOPF_ERR_CUDA;
      S.map_B = B;
    }
    const unsigned g = (unsigned)std::min<long long>(((long long)B * nk + 255) / 256, 4096);
    k_screen_compact_rows<<<g, 256, 0, s>>>(B, n_line, nk, S.kept.as<int>(), w.f0_32.as<float>(),
                                            S.f0c.as<float>());
    h->launches += 1;
    LineSet& L = R.ls;
    L.nl = nk;
    L.ld_l = S.ld_lk;
    L.H_hi = &S.m_H_hi; L.H_lo = &S.m_H_lo;
    L.phit_hi = &S.m_phit_hi; L.phit_lo = &S.m_phit_lo; L.phit_hi96 = &S.m_phit_hi96; L.phit_lo96 = &S.m_phit_lo96;
    L.phi_hi = &S.m_phi_hi; L.phi_lo = &S.m_phi_lo; L.phi_hi96 = &S.m_phi_hi96; L.phi_lo96 = &S.m_phi_lo96;
    L.phit_hi80 = &S.m_phit_hi80; L.phit_lo80 = &S.m_phit_lo80; L.phi_hi80 = &S.m_phi_hi80; L.phi_lo80 = &S.m_phi_lo80;
    L.phit_hi72 = &S.m_phit_hi72; L.phit_lo72 = &S.m_phit_lo72; L.phi_hi72 = &S.m_phi_hi72; L.phi_lo72 = &S.m_phi_lo72;
    L.fmax = S.lim.as<float>();
    L.fmin = S.lim.as<float>() + nk;
    L.f0 = S.f0c.as<float>();
    L.kept = S.kept.as<int>();
    L.pos = S.pos.as<int>();
  }
  const int nl = R.ls.nl;
  R.n_tiles = (nl + STEP_SLICE - 1) / STEP_SLICE;
  if ((r = ensure_batch_bufs(h, B, R.n_tiles))) return r;
  const int ldF = (nl + 3) & ~3;
  if (h->bb.F.alloc((size_t)B * ldF * sizeof(float)) != cudaSuccess) return DCOPF_ERR_OOM;
  BatchView& bb = h->bb.v;
  R.st.has_target = R.it.target != nullptr;
  StepArgs& P = R.P;
  P.rule = p.rule; P.as_printed = p.as_printed; P.alpha = p.alpha;
  P.alpha_lambda = p.alpha_lambda > 0 ? p.alpha_lambda : p.alpha;
  P.rho = p.rho; P.beta1 = p.beta1; P.beta2 = p.beta2; P.eps = p.eps; P.decay = p.decay;
  // work on an internal stream (graph capture needs a capturable stream)
  if (!h->tstream && cudaStreamCreateWithFlags(&h->tstream, cudaStreamNonBlocking) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  cudaStream_t cs = h->tstream;
  if (!h->tev && cudaEventCreateWithFlags(&h->tev, cudaEventDisableTiming) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  if (cudaEventRecord(h->tev, s) != cudaSuccess || cudaStreamWaitEvent(cs, h->tev, 0) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  R.gi = std::min<unsigned>((unsigned)(((long long)B * n_line + 255) / 256), 4096);
  tensor_init_state(R, cs);
  int kbps;
  adjoint_split(h, B, nl, &R.splits, &kbps);
  GemmArgs& ga = R.ga;
  ga.M = B; ga.N = ng; ga.K = nl; ga.kb_per_split = kbps; ga.epi = EPI_PARTIAL;
  ga.P = T.P.as<float>(); ga.ldp = (ng + 3) & ~3; ga.err = h->d_err; ga.timeout_ns = 2000000000ull;
  GemmArgs& gf = R.gf;
  gf.M = B; gf.N = nl; gf.K = ng; gf.kb_per_split = (ng + GBK - 1) / GBK; gf.epi = EPI_TILE;
  gf.F32 = h->bb.F.as<float>(); gf.ldf32 = ldF;
  gf.err = h->d_err; gf.timeout_ns = 2000000000ull;
  ga.bblk = gf.bblk = R.ls.blocked;
  // the CTA-pair products keep Phi~'s high part in L2 in preference to its low part
  // (the two layouts' high parts, 99 MB on the 10000-bus batch, fit where all four do
  // not)
  ga.bpol = gf.bpol = 3;
  StepEpi& E = R.E;
  E.P = to_float_args(P); E.F = gf.F32; E.ldF = ldF; E.f0 = R.ls.f0; E.u = w.u32.as<float>();
  E.outage = R.it.outage; E.tout = bb.tout;
  E.fmax = R.ls.fmax; E.fmin = R.ls.fmin; E.iter = R.st.iter; E.frozen = bb.frozen;
  E.stepf = bb.stepf;
  E.best_iter = R.st.best_iter;
  E.mu_hi[0] = R.st.mu_hi; E.mu_hi[1] = bb.mu2_hi; E.mu_hi[2] = bb.mu3_hi;
  E.mu_lo[0] = R.st.mu_lo; E.mu_lo[1] = bb.mu2_lo; E.mu_lo[2] = bb.mu3_lo;
  E.sv_hi = bb.sv_hi; E.sv_lo = bb.sv_lo;
  E.s1_hi = R.st.s1_hi; E.s2_hi = R.st.s2_hi; E.s1_lo = R.st.s1_lo; E.s2_lo = R.st.s2_lo;
  E.Hh = T.H_hi.as<__nv_bfloat16>(); E.Hl = T.H_lo.as<__nv_bfloat16>(); E.ldh = R.ls.ld_l;
  E.line_part = bb.line_part; E.out_part = bb.out_part; E.n_tiles = R.n_tiles;
  E.pend = bb.pend; E.B = B;
  if (h->timing && !h->kev[0])
    for (int q = 0; q < 6; ++q)
      if (cudaEventCreate(&h->kev[q]) != cudaSuccess) return DCOPF_ERR_CUDA;
  if (h->shape_adj >= 0 && (h->tune_B != B || h->tune_nl != nl)) {  // shapes fixed at create: no timing
    const int kb = (nl + GBK - 1) / GBK;
    const int nv = B >= 2 * GBM ? h->shape_branches : 1;
    const bool pairs_fit = (nv == 1 ? B : tensor_first_group(B)) > GBM;
    h->tune_B = B;
    h->tune_nl = nl;
    h->tune_kbps = (kb + h->shape_splits - 1) / h->shape_splits;
    h->tune_splits = (kb + h->tune_kbps - 1) / h->tune_kbps;
    h->tune_pair_adj = pairs_fit ? h->shape_adj : 0;
    h->tune_pair_fwd = pairs_fit ? h->shape_fwd : 0;
    h->tune_branches = nv;
  }
  if (!h->tstream2 && cudaStreamCreateWithFlags(&h->tstream2, cudaStreamNonBlocking) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  if ((!h->fork_ev && cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming) != cudaSuccess) ||
      (!h->join_ev && cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming) != cudaSuccess))
    return DCOPF_ERR_CUDA;
  if (h->tune_B != B || h->tune_nl != nl) {
    if ((r = tune_tensor(R, cs))) return r;
    tensor_init_state(R, cs);  // the timed runs stepped lambda: start again
  }
  R.ga.skip = bb.frozen;
  R.gf.skip = bb.frozen;
  // the mean of the minimisers starts after the tuning runs
  if ((r = ensure_mean(h, B, &R.st, true, p.mean_dispatch != nullptr, cs))) return r;
  if ((r = make_views(R, h->tune_branches))) return r;
  apply_shapes(R, TensorShapes{h->tune_pair_adj, h->tune_splits, h->tune_kbps, h->tune_pair_fwd});
  return DCOPF_OK;
}

// After round `round`'s chunk: stage and snapshot the frozen candidates (on the solve's
// stream cs) into the snapshot of the round's parity, then certify them in FP64 on the
// certificate stream cc, which runs beside the next two chunks of iterations (the staged
// instances stay frozen meanwhile; round + 2 accepts them).  `done_ev` is recorded on cc
// when the certificate has finished.
static dcopf_status tensor_stage_certify(TensorRun& R, int round, cudaStream_t cs, cudaStream_t cc,
                                         cudaEvent_t staged_ev, cudaEvent_t done_ev) {
  dcopf_dual* h = R.it.h;
  const int B = R.it.B, nl = R.ls.nl, n_line = h->host.n_line;
  BatchView& bb = h->bb.v;
  int* snap = h->bb.snap.as<int>() + (size_t)(round & 1) * B;
  const int* snap_prev = h->bb.snap.as<int>() + (size_t)((round + 1) & 1) * B;
  // the certificate evaluates the full problem: behind a screen, the staged points on
  // every line, zero on the screened ones
  float* bh = R.st.best_hi;
  float* bl = R.st.best_lo;
  int len = nl;
  if (R.ls.kept) {
    bh = h->scr.full.as<float>();
    bl = bh + (size_t)B * n_line;
    len = n_line;
  }
  k_bt_stage<<<dim3((len + 1023) / 1024, B), 256, 0, cs>>>(B, nl, len, R.ls.kept ? R.ls.pos : nullptr, R.st, bb,
                                                          snap, snap_prev, bh, bl);
  h->launches += 1;
  if (cudaEventRecord(staged_ev, cs) != cudaSuccess || cudaStreamWaitEvent(cc, staged_ev, 0) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  dcopf_status r = run_certify_t<float>(h, B, R.it.loads, R.it.outage, R.st.best_lam, bh, bl, R.st.cert,
                                        nullptr, snap, R.st.done, cc, true);
  if (r) return r;
  h->launches += 1;
  if (cudaEventRecord(done_ev, cc) != cudaSuccess) return DCOPF_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? DCOPF_OK : DCOPF_ERR_CUDA;
}

// The stream of round `round`'s certificates: one per round parity, so that two rounds'
// certificates can run at once; the dense certificate (small batches without outages)
// keeps one stream, as its launches share the handle's partial-sum buffer.
static cudaStream_t cert_stream(const TensorRun& R, int round) {
  dcopf_dual* h = R.it.h;
  const bool two = h->cstream2 && !dense_path_applies(h, R.it.B, R.it.outage);
  return (round & 1) && two ? h->cstream2 : h->cstream;
}

// Once the certificate of the instances staged in round `staged` is in (done_ev): accept,
// stop or resume each of them (when `accept`), on cs; the count of instances still
// running, the device error word and the re-screen flag go to *out_active, *out_err,
// *out_flag (device memory).
static dcopf_status tensor_accept(TensorRun& R, bool accept, int staged, int* out_active, int* out_err,
                                  int* out_flag, int* out_iter, cudaStream_t cs, cudaEvent_t done_ev) {
  dcopf_dual* h = R.it.h;
  if (accept && cudaStreamWaitEvent(cs, done_ev, 0) != cudaSuccess) return DCOPF_ERR_CUDA;
  const int* snap = h->bb.snap.as<int>() + (size_t)(staged & 1) * R.it.B;
  k_bt_accept<<<1, ACCEPT_THREADS, 0, cs>>>(R.it.B, accept ? 1 : 0, h->ub_any, R.st, h->bb.v, snap, h->d_err,
                                           out_active, out_err, out_flag, out_iter);
  h->launches += 1;
  return cudaGetLastError() == cudaSuccess ? DCOPF_OK : DCOPF_ERR_CUDA;
}

static dcopf_status tensor_finish(TensorRun& R, cudaStream_t s) {
  dcopf_dual* h = R.it.h;
  cudaStream_t cs = h->tstream;
  SolveState<float> out = R.st;
  if (R.ls.kept) {  // the full-length copies of the last staged points
    out.best_hi = h->scr.full.as<float>();
    out.best_lo = out.best_hi + (size_t)R.it.B * h->host.n_line;
  }
  k_output_f32(R.gi, cs, R.it.B, h->host.n_line, out, R.it.lam, R.it.mh, R.it.ml, R.it.bound,
               R.it.iters, R.it.status);
  h->launches += 1;
  if (R.p.mean_dispatch) launch_mean_out(h, R.it.B, R.st, R.p.mean_dispatch, cs);
  if (cudaEventRecord(h->tev, cs) != cudaSuccess || cudaStreamWaitEvent(s, h->tev, 0) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  if (h->timing) {
    std::vector<int> its(R.it.B);
    cudaMemcpy(its.data(), R.st.iter, sizeof(int) * R.it.B, cudaMemcpyDeviceToHost);
    for (int v : its) h->t_evals += v;
  }
  return DCOPF_OK;
}

// Verbose diagnostics of one group solve: events around every round's graph.
struct GroupObjects {
  std::vector<cudaEvent_t> vev;
  ~GroupObjects() {
    for (cudaEvent_t e : vev) if (e) cudaEventDestroy(e);
  }
};

// The bytes of every kernel argument of the iteration graph of runs[0..n) (the views,
// the step rule, the stop parameters, the shapes, the operand maps, the network's device
// data): a later solve with the same bytes replays the graph captured for them.
static std::vector<unsigned char> graph_signature(const std::vector<TensorRun>& runs, int chunk) {
  std::vector<unsigned char> sig;
  auto put = [&](const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    sig.insert(sig.end(), c, c + n);
  };
  put(&chunk, sizeof chunk);
  for (const TensorRun& R : runs) {
    const dcopf_dual* h = R.it.h;
    put(&h, sizeof h);
    const int timed = h->timing && h->kev[0];
    put(&timed, sizeof timed);
    if (timed) put(h->kev, sizeof h->kev);
    put(&R.nv, sizeof R.nv);
    put(R.v, sizeof(IterView) * R.nv);
    put(&R.P, sizeof R.P);
    put(&R.p.max_iters, sizeof R.p.max_iters);  // arguments of the minimiser and the value kernel
    put(&R.p.tol, sizeof R.p.tol);
    put(&h->dev, sizeof h->dev);
    const int ints[7] = {R.splits, R.pair_adj, R.pair_fwd, R.n_tiles, R.step_blocks, R.min_blocks, R.ls.nl};
    put(ints, sizeof ints);
    for (const CUtensorMap* m : {R.ls.phit_hi, R.ls.phit_lo, R.ls.phit_hi96, R.ls.phit_lo96, R.ls.phit_hi80,
                                 R.ls.phit_lo80, R.ls.phi_hi, R.ls.phi_lo, R.ls.phi_hi96, R.ls.phi_lo96,
                                 R.ls.phi_hi80, R.ls.phi_lo80, R.ls.phit_hi72, R.ls.phit_lo72, R.ls.phi_hi72,
                                 R.ls.phi_lo72})
      if (m) put(m, sizeof(CUtensorMap));
  }
  return sig;
}

// Batched solves of several networks (distinct handles on one device) that advance
// together: each round is ONE launch of a CUDA graph holding every network's chunk
// of iterations as parallel branches, followed by each network's FP64 certification.
static dcopf_status solve_tensor_group_once(const TensorItem* items, int n, const dcopf_solve_params& p,
                                           cudaStream_t s) {
  const auto t_start = std::chrono::steady_clock::now();
  auto host_ms = [t_start] {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  };
  std::vector<TensorRun> runs(n);
  for (int i = 0; i < n; ++i) {
    runs[i].it = items[i];
    runs[i].p = items[i].p ? *items[i].p : p;
    dcopf_status r = tensor_setup(runs[i], s);
    if (r) return r;
  }
  dcopf_dual* h0 = items[0].h;
  cudaStream_t cs0 = h0->tstream;
  const int chunk = std::max(16, p.check_every);
  GroupObjects G;
  RoundKit& K = h0->kit;
  const double t_setup = host_ms();
  if (K.n != n) {  // events and read-back for n networks
    K.release();
    K.ev.assign(2 * n + 1, nullptr);
    K.stage_ev.assign(n, nullptr);
    K.cert_ev.assign(2 * n, nullptr);  // per network and round parity
    for (auto* v : {&K.ev, &K.stage_ev, &K.cert_ev})
      for (cudaEvent_t& e : *v)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return DCOPF_ERR_CUDA;
    for (int q = 0; q < 2; ++q)
      if (cudaEventCreateWithFlags(&K.done[q], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&K.acc[q], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreate(&K.t0[q]) != cudaSuccess || cudaEventCreate(&K.t1[q]) != cudaSuccess)
        return DCOPF_ERR_CUDA;
    if (cudaStreamCreateWithFlags(&K.rs, cudaStreamNonBlocking) != cudaSuccess) return DCOPF_ERR_CUDA;
    if (cudaMallocHost(&K.pin, 8 * sizeof(int) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&K.rb_dev, 8 * sizeof(int) * (size_t)n) != cudaSuccess) {
      cudaGetLastError();
      K.release();
      return DCOPF_ERR_OOM;
    }
    K.n = n;
  }
  // every stream starts after every setup
  for (int i = 1; i < n; ++i) {
    if (cudaEventRecord(K.ev[i], items[i].h->tstream) != cudaSuccess ||
        cudaStreamWaitEvent(cs0, K.ev[i], 0) != cudaSuccess)
      return DCOPF_ERR_CUDA;
  }
  std::vector<unsigned char> sig = graph_signature(runs, chunk);
  const bool reuse = K.exec && sig == K.sig;
  if (!reuse) {
    K.drop_graph();
    std::vector<long long> before(n);
    for (int i = 0; i < n; ++i) before[i] = items[i].h->launches;
    if (cudaStreamBeginCapture(cs0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return DCOPF_ERR_CUDA;
    bool cap_ok = cudaEventRecord(K.ev[0], cs0) == cudaSuccess;
    for (int i = 1; i < n && cap_ok; ++i)
      cap_ok = cudaStreamWaitEvent(items[i].h->tstream, K.ev[0], 0) == cudaSuccess;
    for (int i = 0; i < n && cap_ok; ++i) cap_ok = tensor_enqueue_chunk(runs[i], chunk, items[i].h->tstream);
    for (int i = 1; i < n && cap_ok; ++i)
      cap_ok = cudaEventRecord(K.ev[n + i], items[i].h->tstream) == cudaSuccess &&
               cudaStreamWaitEvent(cs0, K.ev[n + i], 0) == cudaSuccess;
    cudaError_t ce = cudaStreamEndCapture(cs0, &K.graph);
    for (int i = 0; i < n; ++i) items[i].h->launches = before[i];  // counted per replay below
    if (!cap_ok || ce != cudaSuccess || cudaGraphInstantiate(&K.exec, K.graph, 0) != cudaSuccess) {
      cudaGetLastError();
      K.drop_graph();
      return DCOPF_ERR_CUDA;
    }
    // the per-kernel timing nodes of the graph
    bool ktimed = false;
    for (int i = 0; i < n; ++i) ktimed |= items[i].h->timing && items[i].h->kev[0];
    if (ktimed) {
      size_t nn = 0;
      if (cudaGraphGetNodes(K.graph, nullptr, &nn) != cudaSuccess) return DCOPF_ERR_CUDA;
      std::vector<cudaGraphNode_t> nodes(nn);
      if (nn && cudaGraphGetNodes(K.graph, nodes.data(), &nn) != cudaSuccess) return DCOPF_ERR_CUDA;
      for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        cudaEvent_t e = nullptr;
        if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeEventRecord ||
            cudaGraphEventRecordNodeGetEvent(nd, &e) != cudaSuccess)
          continue;
        for (int i = 0; i < n; ++i)
          for (int q = 0; q < 6; ++q)
            if (items[i].h->kev[q] && e == items[i].h->kev[q]) K.knodes.push_back({nd, i, q});
      }
    }
    K.sig = std::move(sig);
  }
  // each timed network's second event set (odd rounds)
  for (int i = 0; i < n; ++i) {
    dcopf_dual* hi = items[i].h;
    if (!hi->timing || !hi->kev[0]) continue;
    for (int q = 0; q < 6; ++q)
      if (!hi->kev2[q] && cudaEventCreate(&hi->kev2[q]) != cudaSuccess) return DCOPF_ERR_CUDA;
  }
  const bool verbose = h0->verbose;
  const double t_captured = host_ms();
  double t_wait = 0.0;
  long long max_iters = 0;
  for (const TensorRun& R : runs) max_iters = std::max<long long>(max_iters, R.p.max_iters);
  // The certificate of round r's candidates runs on a side stream (one per round parity)
  // beside the next rounds' iterations (the candidates stay frozen meanwhile); round
  // r + 2 then accepts them.
  for (int i = 0; i < n; ++i) {
    dcopf_dual* hi = items[i].h;
    // the certificates at the highest stream priority: their CTAs take SMs as the
    // iterations' blocks retire, so that they are in when the next round accepts them
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    for (cudaStream_t* cst : {&hi->cstream, &hi->cstream2})
      if (!*cst && cudaStreamCreateWithPriority(cst, cudaStreamNonBlocking, hi_prio) != cudaSuccess)
        return DCOPF_ERR_CUDA;
    if (hi->bb.snap.alloc(2 * sizeof(int) * (size_t)items[i].B) != cudaSuccess ||
        cudaMemsetAsync(hi->bb.snap.p, 0, 2 * sizeof(int) * (size_t)items[i].B, hi->tstream) != cudaSuccess)
      return DCOPF_ERR_OOM;
  }
  // Rounds are pipelined: the host enqueues round r (its graph, the accept of the
  // certificates of round r - 2's candidates, the staging and certificate of round r's,
  // the read-back of the running counts and device error words) and only then waits for
  // round r - 1's read-back, so that the GPU does not idle while the host turns a round
  // around.  A certificate has two rounds of iterations to run beside (it competes with
  // them for SMs), so that its accept does not wait for it.  A batch whose last instance
  // was accepted in round r - 1 thus also runs round r, whose iterations skip every
  // (frozen) instance.  A round whose graph would find every instance frozen (by the
  // latest read-back, round r - 2's: none was iterating after its accept) launches no
  // graph, only its accept, staging and read-back; an instance that a later accept
  // resumes (its certificate fell short) iterates again from the round after the
  // read-back that shows it.
  std::vector<int> act(n, 1), iterating(n, 1);
  bool ran[2] = {true, true};
  int rounds = 0;
  for (int round = 0;; ++round) {
    const int sl = round & 1;
    rounds = round + 1;
    bool run_graph = round < 2;
    for (int i = 0; i < n; ++i) run_graph |= act[i] && iterating[i] > 0;
    ran[sl] = run_graph;
    for (const RoundKit::KNode& k : K.knodes) {
      dcopf_dual* hk = items[k.net].h;
      if (cudaGraphExecEventRecordNodeSetEvent(K.exec, k.node, sl ? hk->kev2[k.q] : hk->kev[k.q]) != cudaSuccess)
        return DCOPF_ERR_CUDA;
    }
    if (verbose) {
      cudaEvent_t a = nullptr, b = nullptr, c = nullptr;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventCreate(&c);
      G.vev.push_back(a);
      G.vev.push_back(b);
      G.vev.push_back(c);
      cudaEventRecord(a, cs0);
    }
    if (h0->timing) cudaEventRecord(K.t0[sl], cs0);
    if (run_graph && cudaGraphLaunch(K.exec, cs0) != cudaSuccess) return DCOPF_ERR_CUDA;
    long long round_launches = 0;
    for (int i = 0; i < n && run_graph; ++i) {
      items[i].h->launches += (4LL * chunk + 1) * runs[i].nv;
      round_launches += (4LL * chunk + 1) * runs[i].nv;
    }
    if (h0->timing) cudaEventRecord(K.t1[sl], cs0);
    if (verbose) cudaEventRecord(G.vev[G.vev.size() - 2], cs0);
    int* slot = K.rb_dev + (size_t)sl * 4 * n;
    if (cudaEventRecord(K.ev[2 * n], cs0) != cudaSuccess) return DCOPF_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
      cudaStream_t si = items[i].h->tstream;
      if (i > 0 && cudaStreamWaitEvent(si, K.ev[2 * n], 0) != cudaSuccess) return DCOPF_ERR_CUDA;
      // every network reports its count and error word; a network still running accepts
      // the certificates of the last round and stages this round's candidates
      dcopf_status r;
      if ((r = tensor_accept(runs[i], round > 1 && act[i], round - 2, slot + i, slot + n + i, slot + 2 * n + i,
                             slot + 3 * n + i, si, K.cert_ev[2 * i + (round & 1)])))
        return r;
      if (verbose && i == 0) cudaEventRecord(G.vev.back(), cs0);
      if (act[i] &&
          (r = tensor_stage_certify(runs[i], round, si, cert_stream(runs[i], round), K.stage_ev[i],
                                    K.cert_ev[2 * i + (round & 1)])))
        return r;
    }
    for (int i = 1; i < n; ++i)
      if (cudaEventRecord(K.ev[n + i], items[i].h->tstream) != cudaSuccess ||
          cudaStreamWaitEvent(cs0, K.ev[n + i], 0) != cudaSuccess)
        return DCOPF_ERR_CUDA;
    // the read-back of this round's counts, on its own stream
    if (cudaEventRecord(K.acc[sl], cs0) != cudaSuccess || cudaStreamWaitEvent(K.rs, K.acc[sl], 0) != cudaSuccess ||
        cudaMemcpyAsync(K.pin + (size_t)sl * 4 * n, slot, 4 * sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost,
                        K.rs) != cudaSuccess ||
        cudaEventRecord(K.done[sl], K.rs) != cudaSuccess)
      return DCOPF_ERR_CUDA;
    if ((long long)round * chunk > 4LL * max_iters + 64) {  // a cap no solve should reach
      if (cudaEventSynchronize(K.done[sl]) != cudaSuccess) return DCOPF_ERR_CUDA;
      break;
    }
    if (round == 0) continue;
    // round r - 1's read-back (round r is already queued behind it)
    const int pv_sl = sl ^ 1;
    const double tw = verbose ? host_ms() : 0.0;
    if (cudaEventSynchronize(K.done[pv_sl]) != cudaSuccess) return DCOPF_ERR_CUDA;
    if (verbose) t_wait += host_ms() - tw;
    const int* pv = K.pin + (size_t)pv_sl * 4 * n;
    for (int i = 0; i < n; ++i)
      if (pv[n + i]) return (dcopf_status)pv[n + i];
    for (int i = 0; i < n; ++i) iterating[i] = pv[3 * n + i];
    bool rescreen = false;
    for (int i = 0; i < n; ++i)
      if (pv[2 * n + i]) {  // this batch needs a line the network's kept set screens out
        items[i].h->scr.exact = true;
        rescreen = true;
      }
    if (rescreen) {
      for (int i = 0; i < n; ++i)
        if (cudaStreamSynchronize(items[i].h->tstream) != cudaSuccess ||
            (items[i].h->tstream2 && cudaStreamSynchronize(items[i].h->tstream2) != cudaSuccess) ||
            (items[i].h->cstream && cudaStreamSynchronize(items[i].h->cstream) != cudaSuccess) ||
            (items[i].h->cstream2 && cudaStreamSynchronize(items[i].h->cstream2) != cudaSuccess) ||
            cudaMemset(items[i].h->d_err + 1, 0, sizeof(int)) != cudaSuccess)
          return DCOPF_ERR_CUDA;
      if (cudaStreamSynchronize(K.rs) != cudaSuccess) return DCOPF_ERR_CUDA;
      return kRescreen;
    }
    if (h0->timing) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, K.t0[pv_sl], K.t1[pv_sl]);
      h0->t_iter_ms += ms;
      h0->t_iter_launches += round_launches;
    }
    for (int i = 0; i < n && ran[pv_sl]; ++i) {
      dcopf_dual* hi = items[i].h;
      if (!hi->timing || !hi->kev[0] || !act[i] || K.knodes.empty()) continue;
      cudaEvent_t* ks = pv_sl ? hi->kev2 : hi->kev;
      float km[5];
      bool kok = true;
      for (int q = 0; q < 5; ++q) kok &= cudaEventElapsedTime(&km[q], ks[q], ks[q + 1]) == cudaSuccess;
      if (!kok) { cudaGetLastError(); continue; }
      for (int q = 0; q < 5; ++q) hi->t_kernel_ms[q] += km[q];
      hi->t_kernel_samples += 1;
    }
    if (round < 2) continue;  // round 0's read-back counts no accept
    int any = 0;
    for (int i = 0; i < n; ++i) {
      act[i] = pv[i];
      any |= act[i];
    }
    if (!any) break;
  }
  // the last round's graph time (timing), once everything queued has run
  if (cudaStreamSynchronize(cs0) != cudaSuccess || cudaStreamSynchronize(K.rs) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  if (h0->timing) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, K.t0[(rounds - 1) & 1], K.t1[(rounds - 1) & 1]);
    h0->t_iter_ms += ms;
  }
  if (verbose) {
    double graphs = 0.0, gaps = 0.0, accepts = 0.0;
    std::string per_round;
    for (size_t q = 0; q + 2 < G.vev.size(); q += 3) {
      float a = 0.f, b = 0.f, c = 0.f;
      cudaEventElapsedTime(&a, G.vev[q], G.vev[q + 1]);
      graphs += a;
      char buf[16];
      snprintf(buf, sizeof buf, " %.2f", a);
      per_round += buf;
      if (cudaEventElapsedTime(&c, G.vev[q + 1], G.vev[q + 2]) == cudaSuccess) accepts += c;
      if (q + 3 < G.vev.size() && cudaEventElapsedTime(&b, G.vev[q + 1], G.vev[q + 3]) == cudaSuccess) gaps += b;
    }
    fprintf(stderr,
            "dcopf: group solve: setup %.2f ms, graph %s %.2f ms (host), %d rounds: graphs %.2f ms, "
            "between graphs %.2f ms (of which accepts, with their wait for the certificates, %.2f ms; "
            "GPU), host waits %.2f ms, loop %.2f ms (host)\n",
            t_setup, reuse ? "reused" : "captured", t_captured - t_setup, rounds, graphs, gaps, accepts, t_wait,
            host_ms() - t_captured);
    fprintf(stderr, "dcopf: graph ms per round:%s\n", per_round.c_str());
  }
  // the last two rounds' certificates: accept what they staged (nothing, when every
  // instance had stopped before those rounds)
  for (int i = 0; i < n; ++i)
    for (int q = std::max(0, rounds - 2); q < rounds; ++q) {
      int* slot = K.rb_dev;  // free: everything queued has run
      dcopf_status r = tensor_accept(runs[i], true, q, slot + i, slot + n + i, slot + 2 * n + i, slot + 3 * n + i,
                                     items[i].h->tstream, K.cert_ev[2 * i + (q & 1)]);
      if (r) return r;
    }
  for (int i = 0; i < n; ++i) {
    dcopf_status r = tensor_finish(runs[i], s);
    if (r) return r;
  }
  return DCOPF_OK;
}

dcopf_status solve_tensor_group(const TensorItem* items, int n, const dcopf_solve_params& p,
                                cudaStream_t s) {
  dcopf_status r = solve_tensor_group_once(items, n, p, s);
  // a screen that went ahead with a kept set this batch outgrew: again, with the batch's own
  if (r == kRescreen) r = solve_tensor_group_once(items, n, p, s);
  return r == kRescreen ? DCOPF_ERR_CUDA : r;
}

template <typename S>
dcopf_status solve_tensor(dcopf_dual* h, int B, const double* loads, const int* outage,
                          const dcopf_solve_params& p, double* lam, double* mh, double* ml,
                          double* bound, int* iters, int* status, cudaStream_t s) {
  static_assert(sizeof(S) == 4, "the tensor-core solve keeps FP32 state");
  TensorItem it{h, nullptr, B, loads, outage, p.target_value, lam, mh, ml, bound, iters, status};
  return solve_tensor_group(&it, 1, p, s);
}

template dcopf_status solve_tensor<float>(dcopf_dual*, int, const double*, const int*,
                                          const dcopf_solve_params&, double*, double*, double*,
                                          double*, int*, int*, cudaStream_t);

}  // namespace dcopf
