// Batched operator products on tcgen05 tensor cores for many instances of one
// network: the adjoint Pi~ = H Phi~ (H = [batch][n_line] line multipliers) and the
// forward F = X Phi~^T (X = [batch][n_gen] normalised dispatch), the two dense
// contractions of every iteration (eq. (6): c + A^T lambda + C^T mu, and C x*).
//
// Precision: each FP32 operand v is split into BF16 v_hi = bf16(v) and
// v_lo = bf16(v - v_hi) and the product is hi*hi + hi*lo + lo*hi with FP32 accumulation
// in TMEM (3 MMAs per K step).  When one operand is exact in BF16 (the LP dispatch
// x in {-1, 0, 1}) its lo part is zero and 2 MMAs suffice.
//
// Kernel shape: one 128 x 128 output tile per CTA (split along K for the adjoint,
// whose K = n_line is long and whose N = n_gen is short), 6 warps: warp 0 issues TMA
// loads of the BF16 tiles of a 64-wide K block into a ring with 128-byte swizzle,
// warp 1 allocates TMEM and one of its threads issues the MMAs, warps 2-5 read the
// accumulator from TMEM (tcgen05.ld) and run the epilogue.  The three-product GEMMs
// run one CTA per SM with a 3-stage ring; the two-product LP forward runs two CTAs per
// SM with a 2-stage ring each, so that one CTA's epilogue overlaps the other's loads.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "dev.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace dcopf {

enum { EPI_PARTIAL = 0, EPI_FLOW = 1, EPI_TILE = 2 };

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

__device__ __forceinline__ float step_rule(const StepArgsF& P, float theta, float g, float& s1,
                                           float& s2, float a, float bc1, float bc2) {
  if (P.rule == DCOPF_GDM) {
    s1 = P.rho * s1 + a * g;
    theta += s1;
    if (P.as_printed) theta += a * g;
  } else if (P.rule == DCOPF_ADAM) {
    s1 = P.beta1 * s1 + P.omb1 * g;
    s2 = P.beta2 * s2 + P.omb2 * g * g;
    theta += a * (s1 / bc1) / (sqrtf(s2 / bc2) + P.eps);
  } else {
    s1 += g * g;
    theta += a * g / (sqrtf(s1) + P.eps);
  }
  return theta;
}

// Step of the batched solve after the forward product: flows (with the rank-1 outage
// term), supergradient, line part of the dual value, projected step of mu into the
// parity-buffered state, BF16 split of the next eta, outage partial u^T eta.
struct StepEpi {
  StepArgsF P;
  const float* F;             // [B][ldF] forward product Phi~ x
  int ldF;
  const float* f0;            // [B][nl] flows of the mid-box dispatch minus the loads
  const float* u;             // [B][nl] outage vectors (rows of outage instances)
  const int* outage;          // [B] or null
  const float* tout;          // [B] pre-outage flow on the outaged line, (Phi~ x)_k
  const float* fmax; const float* fmin;
  const int* iter;            // [B] evaluations done: iter % 3 selects the state buffer
  const int* frozen;          // [B] done or waiting for certification
  const int* best_iter;       // [B] evaluation count of the best point so far
  const float* stepf;         // [B][4] alpha scale, 1 - beta1^t, 1 - beta2^t
  // Three state buffers in turn: point t lives in buffer t % 3, so the two points
  // before the one being stepped are still there.  The step writing point t + 1
  // overwrites point t - 2; if that point is still the best (the value fell after
  // it), it is first copied to sv.  Points that are overtaken before their buffer
  // comes round are never copied.
  float* mu_hi[3]; float* mu_lo[3];
  float* sv_hi; float* sv_lo;
  float* s1_hi; float* s2_hi; float* s1_lo; float* s2_lo;
  __nv_bfloat16* Hh; __nv_bfloat16* Hl; int ldh;
  double* line_part; double* out_part; int n_tiles;   // [B][n_tiles] per chunk of lines
};

struct GemmArgs {
  int M, N, K;           // rows of A (instances), rows of B (outputs), contraction length
  int kb_per_split;      // 64-wide K blocks per split
  int epi;
  float* P; int ldp;     // EPI_PARTIAL: P[split][M][ldp]
  const double* f0; double* f; int ldf;  // EPI_FLOW: f = acc + f0, [M][ldf]
  float* F32; int ldf32;  // EPI_TILE: raw accumulator, [M][ldf32]
  int* err;
  uint64_t timeout_ns;
  const int* skip;       // nullable [M]: rows whose instance is frozen (a tile of them is skipped)
};

constexpr int GBM = 128, GBN = 128, GBK = 64;
constexpr uint32_t TILE_BYTES = GBM * GBK * 2;  // 16 KB, also GBN * GBK * 2

template <int NPROD, int OCC = 1>
struct GemmCfg {
  static constexpr int STAGES = NPROD == 3 ? 3 : (OCC == 2 ? 2 : 4);
  static constexpr uint32_t STAGE_BYTES = (NPROD == 3 ? 4 : 3) * TILE_BYTES;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
  static_assert(STAGES * STAGE_BYTES >= GBM * (GBN + 1) * 4, "the ring stages the output tile");
};

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16* hi, __nv_bfloat16* lo);



template <int NPROD, int OCC = 1>
__global__ void __launch_bounds__(192, OCC)
    k_gemm_bf16x(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                 const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                 GemmArgs g) {
  using Cfg = GemmCfg<NPROD, OCC>;
  constexpr int ST = Cfg::STAGES;
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[ST], empty[ST], accf;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int kb_total = (g.K + GBK - 1) / GBK;
  const int kb0 = blockIdx.z * g.kb_per_split;
  const int nkb = min(kb_total, kb0 + g.kb_per_split) - kb0;
  auto a_hi = [&](int s) { return base + (size_t)s * Cfg::STAGE_BYTES; };
  auto a_lo = [&](int s) { return a_hi(s) + TILE_BYTES; };
  auto b_hi = [&](int s) { return a_hi(s) + (NPROD == 3 ? 2 : 1) * TILE_BYTES; };
  auto b_lo = [&](int s) { return b_hi(s) + TILE_BYTES; };

  if (g.skip) {
    // a tile whose instances are all frozen has nothing to compute: the kernels that
    // read its output skip frozen instances too.  Decided before any barrier, TMA or
    // TMEM work, by every thread alike.
    int live = 0;
    for (int r = threadIdx.x; r < GBM; r += blockDim.x)
      live |= (m0 + r < g.M && !g.skip[m0 + r]) ? 1 : 0;
    if (!__syncthreads_or(live)) return;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(&accf, 1);
    s_abort = 0;
    umma::fence_mbar_init();
  }
  if (warp == 1) umma::tmem_alloc(&tmem_base, GBN);
  __syncthreads();
  umma::tc_fence_after();
  const uint32_t tmem = tmem_base;
  int issued = 0;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int i = 0; i < nkb && nkb > 0; ++i) {
      const int s = i % ST;
      if (i >= ST && !umma::mbar_wait(&empty[s], ((i / ST) & 1) ^ 1, g.timeout_ns)) {
        s_abort = 1;
        break;
      }
      umma::mbar_arrive_expect_tx(&full[s], Cfg::STAGE_BYTES);
      const int x = (kb0 + i) * GBK;
      umma::tma_load_2d(&tAh, &full[s], a_hi(s), x, m0);
      if (NPROD == 3) umma::tma_load_2d(&tAl, &full[s], a_lo(s), x, m0);
      umma::tma_load_2d(&tBh, &full[s], b_hi(s), x, n0);
      umma::tma_load_2d(&tBl, &full[s], b_lo(s), x, n0);
      ++issued;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = umma::idesc_bf16_f32(GBN);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % ST;
      if (!umma::mbar_wait(&full[s], (i / ST) & 1, g.timeout_ns)) {
        s_abort = 1;
        break;
      }
      umma::tc_fence_after();
      const uint64_t dah = umma::desc_sw128(umma::smem_u32(a_hi(s)));
      const uint64_t dal = umma::desc_sw128(umma::smem_u32(a_lo(s)));
      const uint64_t dbh = umma::desc_sw128(umma::smem_u32(b_hi(s)));
      const uint64_t dbl = umma::desc_sw128(umma::smem_u32(b_lo(s)));
#pragma unroll
      for (int kk = 0; kk < GBK / 16; ++kk) {
        const uint64_t o = (uint64_t)(kk * 32) >> 4;  // 16 BF16 = 32 bytes along the row
        umma::mma_bf16(tmem, dah + o, dbh + o, idesc, (i > 0 || kk > 0) ? 1u : 0u);
        umma::mma_bf16(tmem, dah + o, dbl + o, idesc, 1u);
        if (NPROD == 3) umma::mma_bf16(tmem, dal + o, dbh + o, idesc, 1u);
      }
      umma::mma_commit(&empty[s]);
    }
    umma::mma_commit(&accf);
  } else if (warp >= 2) {
    // ---------------- epilogue: warp w reads TMEM lanes 32*(w%4) .. +31
    const bool ready = __all_sync(0xffffffffu, umma::mbar_wait(&accf, 0, g.timeout_ns));
    umma::tc_fence_after();
    const int q = warp & 3;
    const int row = m0 + 32 * q + lane;
    if (!ready) s_abort = 1;
    if (ready && nkb > 0) {
#pragma unroll 1
      for (int cc = 0; cc < GBN / 32; ++cc) {
        float v[32];
        umma::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * cc), v);
        const int col0 = n0 + 32 * cc;
        if (g.epi == EPI_TILE) {
          // stage the accumulator in the (now idle) pipeline ring, stride GBN + 1
          float* tile = (float*)base;
#pragma unroll
          for (int u = 0; u < 32; ++u) tile[(32 * q + lane) * (GBN + 1) + 32 * cc + u] = v[u];
        } else if (row < g.M) {
          if (g.epi == EPI_PARTIAL) {
            float* dst = g.P + ((size_t)blockIdx.z * g.M + row) * g.ldp + col0;
            if (col0 + 32 <= g.N) {
#pragma unroll
              for (int u = 0; u < 8; ++u)
                reinterpret_cast<float4*>(dst)[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            } else {  // ragged tail: predicated, unrolled (v stays in registers)
#pragma unroll
              for (int u = 0; u < 32; ++u)
                if (col0 + u < g.N) dst[u] = v[u];
            }
          } else {
            const double* f0 = g.f0 + (size_t)row * g.ldf + col0;
            double* f = g.f + (size_t)row * g.ldf + col0;
#pragma unroll
            for (int u = 0; u < 32; ++u)
              if (col0 + u < g.N) f[u] = (double)v[u] + f0[u];
          }
        }
      }
    }
  }
  umma::tc_fence_before();  // order this thread's tcgen05 work before the teardown barrier
  __syncthreads();
  if (g.epi == EPI_TILE && !s_abort && nkb > 0) {
    // coalesced store of the staged tile: a warp per row, lanes along columns
    const float* tile = (const float*)base;
    for (int m = warp; m < GBM; m += 6) {
      const int r = m0 + m;
      if (r >= g.M) break;
      float* dst = g.F32 + (size_t)r * g.ldf32;
#pragma unroll
      for (int q = 0; q < GBN / 32; ++q) {
        const int c = lane + 32 * q;
        if (n0 + c < g.N) dst[n0 + c] = tile[m * (GBN + 1) + c];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_abort) {
    atomicExch(g.err, (int)DCOPF_ERR_TIMEOUT);
    // let the copies still in flight land before the CTA's shared memory is released
    for (int i = max(0, issued - ST); i < issued; ++i)
      umma::mbar_wait(&full[i % ST], (i / ST) & 1, g.timeout_ns);
  }
  __syncthreads();
  if (warp == 1) {
    umma::tc_fence_after();
    umma::tmem_dealloc(tmem, GBN);
  }
}

// ------------------------------------------------------------------ CTA-pair products
// The same products on pairs of CTAs (clusters of 2, tcgen05 cta_group::2): a pair
// computes a 256 x 256 output tile.  Each CTA loads its own 128 rows of A and its own
// 128 of the tile's 256 rows of B, so that per byte fed from L2 each CTA does twice the
// MMA work of a 128 x 128 tile.  The even-ranked CTA issues every MMA; both CTAs'
// loads count on its "full" barriers; its commits arrive on the "empty" and
// accumulator barriers of both CTAs.  Each CTA's TMEM holds its 128 rows x 256 columns
// of the accumulator and each CTA runs the epilogue of its rows.
constexpr int PBM = 256;

// PBN: the pair tile's width (256 or 192 output columns; each CTA loads PBN / 2 rows of B).
template <int NPROD, int PBN>
struct PairCfg {
  static constexpr uint32_t B_TILE = (uint32_t)(PBN / 2) * GBK * 2;
  static constexpr uint32_t STAGE_BYTES = (NPROD == 3 ? 2 : 1) * TILE_BYTES + 2 * B_TILE;
  // as many stages as fit in 224 KB of the 227 KB a CTA may hold (at most five)
  static constexpr int STAGES = (224u * 1024u / STAGE_BYTES) < 5 ? (224u * 1024u / STAGE_BYTES) : 5;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
  static constexpr uint32_t TMEM_COLS = PBN <= 128 ? 128 : 256;  // a power of two
  static_assert(STAGES >= 2, "a ring of at least two stages");
  static_assert(B_TILE % 1024 == 0, "tiles start on 1024-byte (swizzle atom) boundaries");
  static_assert(STAGES * STAGE_BYTES >= 128 * (PBN + 1) * 4, "the ring stages the output tile");
};

template <int NPROD, int PBN>
__global__ void __launch_bounds__(192, 1)
    k_gemm_pair(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                GemmArgs g) {
  using Cfg = PairCfg<NPROD, PBN>;
  constexpr int ST = Cfg::STAGES;
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[ST], empty[ST], accf;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = umma::cluster_ctarank();  // 0: issues the MMAs
  const int m0 = blockIdx.y * PBM, n0 = (blockIdx.x >> 1) * PBN;
  const int my_m = m0 + 128 * (int)rank;  // this CTA's rows of A and of the output
  const int my_n = n0 + (PBN / 2) * (int)rank;  // this CTA's rows of B
  const int kb_total = (g.K + GBK - 1) / GBK;
  const int kb0 = blockIdx.z * g.kb_per_split;
  const int nkb = min(kb_total, kb0 + g.kb_per_split) - kb0;
  auto a_hi = [&](int s) { return base + (size_t)s * Cfg::STAGE_BYTES; };
  auto a_lo = [&](int s) { return a_hi(s) + TILE_BYTES; };
  auto b_hi = [&](int s) { return a_hi(s) + (NPROD == 3 ? 2 : 1) * TILE_BYTES; };
  auto b_lo = [&](int s) { return b_hi(s) + Cfg::B_TILE; };

  if (g.skip) {
    // both CTAs decide on all 256 rows of the pair, so that they leave together
    int live = 0;
    for (int r = threadIdx.x; r < PBM; r += blockDim.x)
      live |= (m0 + r < g.M && !g.skip[m0 + r]) ? 1 : 0;
    if (!__syncthreads_or(live)) return;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(&accf, 1);
    s_abort = 0;
    umma::fence_mbar_init();
  }
  if (warp == 1) umma::tmem_alloc_pair(&tmem_base, Cfg::TMEM_COLS);
  __syncthreads();
  umma::tc_fence_before();
  umma::cluster_sync_all();  // both CTAs' barriers and TMEM exist before any remote signal
  umma::tc_fence_after();
  const uint32_t tmem = tmem_base;
  int issued = 0;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer (both CTAs; completion counted on rank 0's barrier)
    for (int i = 0; i < nkb; ++i) {
      const int s = i % ST;
      if (i >= ST && !umma::mbar_wait(&empty[s], ((i / ST) & 1) ^ 1, g.timeout_ns)) {
        s_abort = 1;
        break;
      }
      if (rank == 0) umma::mbar_arrive_expect_tx(&full[s], 2 * Cfg::STAGE_BYTES);
      const uint32_t bar = umma::cluster_addr(&full[s], 0);
      const int x = (kb0 + i) * GBK;
      umma::tma_load_2d_pair(&tAh, bar, a_hi(s), x, my_m);
      if (NPROD == 3) umma::tma_load_2d_pair(&tAl, bar, a_lo(s), x, my_m);
      umma::tma_load_2d_pair(&tBh, bar, b_hi(s), x, my_n);
      umma::tma_load_2d_pair(&tBl, bar, b_lo(s), x, my_n);
      ++issued;
    }
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---------------- MMA issuer (rank 0 only): M = 256 over the pair, N = PBN
    constexpr uint32_t idesc = umma::idesc_bf16_f32(PBN, PBM);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % ST;
      if (!umma::mbar_wait(&full[s], (i / ST) & 1, g.timeout_ns)) {
        s_abort = 1;
        break;
      }
      umma::tc_fence_after();
      const uint64_t dah = umma::desc_sw128(umma::smem_u32(a_hi(s)));
      const uint64_t dal = umma::desc_sw128(umma::smem_u32(a_lo(s)));
      const uint64_t dbh = umma::desc_sw128(umma::smem_u32(b_hi(s)));
      const uint64_t dbl = umma::desc_sw128(umma::smem_u32(b_lo(s)));
#pragma unroll
      for (int kk = 0; kk < GBK / 16; ++kk) {
        const uint64_t o = (uint64_t)(kk * 32) >> 4;
        umma::mma_bf16_pair(tmem, dah + o, dbh + o, idesc, (i > 0 || kk > 0) ? 1u : 0u);
        umma::mma_bf16_pair(tmem, dah + o, dbl + o, idesc, 1u);
        if (NPROD == 3) umma::mma_bf16_pair(tmem, dal + o, dbh + o, idesc, 1u);
      }
      umma::mma_commit_pair(&empty[s], (uint16_t)0x3);
    }
    umma::mma_commit_pair(&accf, (uint16_t)0x3);
  } else if (warp >= 2) {
    // ---------------- epilogue (both CTAs): warp w reads TMEM lanes 32*(w%4) .. +31
    const bool ready = __all_sync(0xffffffffu, umma::mbar_wait(&accf, 0, g.timeout_ns));
    umma::tc_fence_after();
    const int q = warp & 3;
    const int row = my_m + 32 * q + lane;
    if (!ready) s_abort = 1;
    if (ready && nkb > 0) {
#pragma unroll 1
      for (int cc = 0; cc < PBN / 32; ++cc) {
        float v[32];
        umma::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * cc), v);
        const int col0 = n0 + 32 * cc;
        if (g.epi == EPI_TILE) {
          float* tile = (float*)base;
#pragma unroll
          for (int u = 0; u < 32; ++u) tile[(32 * q + lane) * (PBN + 1) + 32 * cc + u] = v[u];
        } else if (row < g.M) {
          if (g.epi == EPI_PARTIAL) {
            float* dst = g.P + ((size_t)blockIdx.z * g.M + row) * g.ldp + col0;
            if (col0 + 32 <= g.N) {
#pragma unroll
              for (int u = 0; u < 8; ++u)
                reinterpret_cast<float4*>(dst)[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            } else {
#pragma unroll
              for (int u = 0; u < 32; ++u)
                if (col0 + u < g.N) dst[u] = v[u];
            }
          } else {
            const double* f0 = g.f0 + (size_t)row * g.ldf + col0;
            double* f = g.f + (size_t)row * g.ldf + col0;
#pragma unroll
            for (int u = 0; u < 32; ++u)
              if (col0 + u < g.N) f[u] = (double)v[u] + f0[u];
          }
        }
      }
    }
  }
  umma::tc_fence_before();
  __syncthreads();
  if (g.epi == EPI_TILE && !s_abort && nkb > 0) {
    const float* tile = (const float*)base;
    for (int m = warp; m < 128; m += 6) {
      const int r = my_m + m;
      if (r >= g.M) break;
      float* dst = g.F32 + (size_t)r * g.ldf32;
#pragma unroll
      for (int q = 0; q < PBN / 32; ++q) {
        const int c = lane + 32 * q;
        if (n0 + c < g.N) dst[n0 + c] = tile[m * (PBN + 1) + c];
      }
    }
  }
  if (threadIdx.x == 0 && s_abort) {
    atomicExch(g.err, (int)DCOPF_ERR_TIMEOUT);
    // rank 0's full barriers count both CTAs' copies: let those in flight land
    if (rank == 0)
      for (int i = max(0, issued - ST); i < issued; ++i)
        umma::mbar_wait(&full[i % ST], (i / ST) & 1, g.timeout_ns);
  }
  __syncthreads();
  // neither CTA releases its shared memory or TMEM while the pair's copies or MMAs may
  // still reach it
  umma::tc_fence_before();
  umma::cluster_sync_all();
  if (warp == 1) {
    umma::tc_fence_after();
    umma::tmem_dealloc_pair(tmem, Cfg::TMEM_COLS);
  }
}

// One block per (chunk of STEP_CHUNK lines, instance): elementwise, full occupancy,
// coalesced; per-chunk FP64 partials of the value and of u^T eta.
constexpr int STEP_THREADS = 256, STEP_PER_THREAD = 4;
constexpr int STEP_CHUNK = STEP_THREADS * STEP_PER_THREAD;

__global__ void __launch_bounds__(STEP_THREADS) k_bt_step(StepEpi E, int nl) {
  __shared__ double red[32];
  const int b = blockIdx.y, chunk = blockIdx.x;
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
  const float am = E.stepf[4 * b], bc1 = E.stepf[4 * b + 1], bc2 = E.stepf[4 * b + 2];
  const float* Fr = E.F + (size_t)b * E.ldF;
  // a thread's few terms are summed in FP32 and the block sum is FP64 (FP64 throughput
  // is low on this part: per-element FP64 would dominate the kernel)
  float lacc = 0.f, oacc = 0.f;
  const int i0 = chunk * STEP_CHUNK + threadIdx.x;
  float fl[STEP_PER_THREAD], ui[STEP_PER_THREAD], mh[STEP_PER_THREAD], ml[STEP_PER_THREAD],
      a1[STEP_PER_THREAD], a2[STEP_PER_THREAD], b1[STEP_PER_THREAD], b2[STEP_PER_THREAD],
      fx[STEP_PER_THREAD], fn[STEP_PER_THREAD];
#pragma unroll
  for (int q = 0; q < STEP_PER_THREAD; ++q) {  // all loads in flight before any arithmetic
    const int i = i0 + q * STEP_THREADS;
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
  for (int q = 0; q < STEP_PER_THREAD; ++q) {
    const int i = i0 + q * STEP_THREADS;
    if (i >= nl) continue;
    const float f = fl[q] + ui[q] * t_out;
    const float gh = f - fx[q], gl = fn[q] - f;
    float nh = 0.f, nlo = 0.f;
    if (i != k) {
      lacc = fmaf(mh[q], gh, fmaf(ml[q], gl, lacc));
      nh = fmaxf(step_rule(E.P, mh[q], gh, a1[q], a2[q], am, bc1, bc2), 0.f);
      nlo = fmaxf(step_rule(E.P, ml[q], gl, b1[q], b2[q], am, bc1, bc2), 0.f);
      E.s1_hi[o + i] = a1[q]; E.s2_hi[o + i] = a2[q]; E.s1_lo[o + i] = b1[q]; E.s2_lo[o + i] = b2[q];
    }
    if (save) { E.sv_hi[o + i] = mhn[i]; E.sv_lo[o + i] = mln[i]; }
    mhn[i] = nh;
    mln[i] = nlo;
    const float eta = nh - nlo;
    split_bf16(eta, E.Hh + (size_t)b * E.ldh + i, E.Hl + (size_t)b * E.ldh + i);
    if (k >= 0) oacc = fmaf(ui[q], eta, oacc);
  }
  // warp sums in FP32, the 8 warp partials in FP64 (fixed order)
  lacc = warp_sum(lacc);
  oacc = warp_sum(oacc);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[w] = (double)lacc;
    red[16 + w] = (double)oacc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // the warps' partials in FP64, a shuffle tree (fixed order)
    const int l = threadIdx.x;
    double ls = l < STEP_THREADS / 32 ? red[l] : 0.0, os = l < STEP_THREADS / 32 ? red[16 + l] : 0.0;
#pragma unroll
    for (int o = STEP_THREADS / 64; o > 0; o >>= 1) {
      ls += __shfl_xor_sync(0xffffffffu, ls, o);
      os += __shfl_xor_sync(0xffffffffu, os, o);
    }
    if (l == 0) {
      E.line_part[(size_t)b * E.n_tiles + chunk] = ls;
      E.out_part[(size_t)b * E.n_tiles + chunk] = os;
    }
  }
}

// The same step with four consecutive lines per thread: 16-byte loads and stores of every
// FP32 stream and 8-byte stores of the BF16 split (needs n_line, ldF and ldh multiples
// of 4; the chunk of a block is the same 1024 lines as k_bt_step's).
__global__ void __launch_bounds__(STEP_THREADS, 4) k_bt_step4(StepEpi E, int nl) {
  __shared__ double red[32];
  const int b = blockIdx.y, chunk = blockIdx.x;
  if (E.frozen[b]) return;
  const int k = E.outage ? E.outage[b] : -1;
  const float t_out = k >= 0 ? E.tout[b] : 0.f;
  const int it = E.iter[b], pb = it % 3, pn = (it + 1) % 3;
  const bool save = it >= 2 && E.best_iter[b] == it - 1;  // point it - 2 is the best
  const size_t o = (size_t)b * nl;
  const float am = E.stepf[4 * b], bc1 = E.stepf[4 * b + 1], bc2 = E.stepf[4 * b + 2];
  const int i = 4 * (chunk * STEP_THREADS + threadIdx.x);
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
        nh = fmaxf(step_rule(E.P, MH[q], gh, A1[q], A2[q], am, bc1, bc2), 0.f);
        nlo = fmaxf(step_rule(E.P, ML[q], gl, B1[q], B2[q], am, bc1, bc2), 0.f);
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
  lacc = warp_sum(lacc);
  oacc = warp_sum(oacc);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[w] = (double)lacc;
    red[16 + w] = (double)oacc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // the warps' partials in FP64, a shuffle tree (fixed order)
    const int l = threadIdx.x;
    double ls = l < STEP_THREADS / 32 ? red[l] : 0.0, os = l < STEP_THREADS / 32 ? red[16 + l] : 0.0;
#pragma unroll
    for (int o = STEP_THREADS / 64; o > 0; o >>= 1) {
      ls += __shfl_xor_sync(0xffffffffu, ls, o);
      os += __shfl_xor_sync(0xffffffffu, os, o);
    }
    if (l == 0) {
      E.line_part[(size_t)b * E.n_tiles + chunk] = ls;
      E.out_part[(size_t)b * E.n_tiles + chunk] = os;
    }
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

// BF16 hi/lo copies of Phi~ (forward B operand, [n_line][ld_g]) and Phi~^T (adjoint B
// operand, [n_gen][ld_l]), built once per handle.
dcopf_status ensure_tensor_operands(dcopf_dual* h) {
  TensorOps& T = h->tops;
  if (T.ready) return DCOPF_OK;
  const HostNet& H = h->host;
  const int nl = H.n_line, ng = H.n_gen;
  T.ld_l = round8(nl);
  T.ld_g = round8(ng);
  std::vector<__nv_bfloat16> ph((size_t)nl * T.ld_g), pl((size_t)nl * T.ld_g);
  std::vector<__nv_bfloat16> th((size_t)ng * T.ld_l), tl((size_t)ng * T.ld_l);
  const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
  std::fill(ph.begin(), ph.end(), z); std::fill(pl.begin(), pl.end(), z);
  std::fill(th.begin(), th.end(), z); std::fill(tl.begin(), tl.end(), z);
  for (int i = 0; i < nl; ++i)
    for (int j = 0; j < ng; ++j) {
      const float v = (float)H.phi[(size_t)i * ng + j];
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
      ph[(size_t)i * T.ld_g + j] = hi; pl[(size_t)i * T.ld_g + j] = lo;
      th[(size_t)j * T.ld_l + i] = hi; tl[(size_t)j * T.ld_l + i] = lo;
    }
  auto up = [&](DBuf& d, const std::vector<__nv_bfloat16>& v) {
    if (d.alloc(v.size() * 2) != cudaSuccess) return false;
    return cudaMemcpy(d.p, v.data(), v.size() * 2, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  if (!up(T.phi_hi, ph) || !up(T.phi_lo, pl) || !up(T.phit_hi, th) || !up(T.phit_lo, tl))
    return DCOPF_ERR_OOM;
  if (!make_map(&T.m_phi_hi, T.phi_hi.p, nl, ng, T.ld_g, GBN) ||
      !make_map(&T.m_phi_lo, T.phi_lo.p, nl, ng, T.ld_g, GBN) ||
      !make_map(&T.m_phit_hi, T.phit_hi.p, ng, nl, T.ld_l, GBN) ||
      !make_map(&T.m_phit_lo, T.phit_lo.p, ng, nl, T.ld_l, GBN) ||
      !make_map(&T.m_phi_hi96, T.phi_hi.p, nl, ng, T.ld_g, 96) ||
      !make_map(&T.m_phi_lo96, T.phi_lo.p, nl, ng, T.ld_g, 96) ||
      !make_map(&T.m_phit_hi96, T.phit_hi.p, ng, nl, T.ld_l, 96) ||
      !make_map(&T.m_phit_lo96, T.phit_lo.p, ng, nl, T.ld_l, 96))
    return DCOPF_ERR_CUDA;
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
#define DCOPF_PAIR_SMEM(NP, BN)                                                                  \
  if ((e = cudaFuncSetAttribute(k_gemm_pair<NP, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                (int)PairCfg<NP, BN>::SMEM)) != cudaSuccess)                        \
    return e;
  DCOPF_PAIR_SMEM(2, 256)
  DCOPF_PAIR_SMEM(3, 256)
  DCOPF_PAIR_SMEM(2, 192)
  DCOPF_PAIR_SMEM(3, 192)
#undef DCOPF_PAIR_SMEM
  return cudaSuccess;
}

// The CTA-pair products: clusters of two CTAs, grid (2 x pair columns, pair rows, splits).
template <int NPROD, int PBN>
static cudaError_t launch_gemm_pair(dcopf_dual* h, const CUtensorMap& Ah, const CUtensorMap& Al,
                                    const CUtensorMap& Bh, const CUtensorMap& Bl, GemmArgs g, int splits,
                                    cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(2 * ((g.N + PBN - 1) / PBN), (g.M + PBM - 1) / PBM, splits);
  cfg.blockDim = dim3(192);
  cfg.dynamicSmemBytes = PairCfg<NPROD, PBN>::SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  h->launches += 1;
  return cudaLaunchKernelEx(&cfg, k_gemm_pair<NPROD, PBN>, Ah, Al, Bh, Bl, g);
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
  const float* fmax = nullptr;     // [nl]
  const float* fmin = nullptr;
  const float* f0 = nullptr;       // [B][nl] base flows
  const int* kept = nullptr;       // [nl] network line of each row (null: all lines)
  const int* pos = nullptr;        // [n_line] row of each line or -1 (null: all lines)
};

static LineSet full_lines(dcopf_dual* h) {
  TensorOps& T = h->tops;
  LineSet L;
  L.nl = h->host.n_line;
  L.ld_l = T.ld_l;
  L.H_hi = &T.m_H_hi; L.H_lo = &T.m_H_lo;
  L.phit_hi = &T.m_phit_hi; L.phit_lo = &T.m_phit_lo; L.phit_hi96 = &T.m_phit_hi96; L.phit_lo96 = &T.m_phit_lo96;
  L.phi_hi = &T.m_phi_hi; L.phi_lo = &T.m_phi_lo; L.phi_hi96 = &T.m_phi_hi96; L.phi_lo96 = &T.m_phi_lo96;
  L.fmax = h->dev.fmax32;
  L.fmin = h->dev.fmin32;
  L.f0 = h->ws.f0_32.as<float>();
  return L;
}

// `tiles`: 0 single CTAs (128 x 128), 1 CTA pairs of 256 x 256, 2 CTA pairs of 256 x 192.
static cudaError_t launch_adjoint(dcopf_dual* h, const LineSet& L, const GemmArgs& g, int splits, int tiles,
                                  cudaStream_t s) {
  if (tiles == 1) return launch_gemm_pair<3, 256>(h, *L.H_hi, *L.H_lo, *L.phit_hi, *L.phit_lo, g, splits, s);
  if (tiles == 2) return launch_gemm_pair<3, 192>(h, *L.H_hi, *L.H_lo, *L.phit_hi96, *L.phit_lo96, g, splits, s);
  return launch_gemm<3>(h, *L.H_hi, *L.H_lo, *L.phit_hi, *L.phit_lo, g, splits, s);
}
static cudaError_t launch_forward(dcopf_dual* h, const LineSet& L, const GemmArgs& g, int tiles, cudaStream_t s) {
  TensorOps& T = h->tops;
  if (h->host.qp) {
    if (tiles == 1) return launch_gemm_pair<3, 256>(h, T.m_X_hi, T.m_X_lo, *L.phi_hi, *L.phi_lo, g, 1, s);
    if (tiles == 2) return launch_gemm_pair<3, 192>(h, T.m_X_hi, T.m_X_lo, *L.phi_hi96, *L.phi_lo96, g, 1, s);
    return launch_gemm<3>(h, T.m_X_hi, T.m_X_lo, *L.phi_hi, *L.phi_lo, g, 1, s);
  }
  if (tiles == 1) return launch_gemm_pair<2, 256>(h, T.m_X_hi, T.m_X_lo, *L.phi_hi, *L.phi_lo, g, 1, s);
  if (tiles == 2) return launch_gemm_pair<2, 192>(h, T.m_X_hi, T.m_X_lo, *L.phi_hi96, *L.phi_lo96, g, 1, s);
  // the LP forward on single CTAs (two products: x is exact in BF16): its K = n_gen is
  // short, so a CTA spends much of its time in the epilogue; two CTAs per SM (a 2-stage
  // ring each) let one CTA's epilogue run beside the other's main loop
  return launch_gemm<2, 2>(h, T.m_X_hi, T.m_X_lo, *L.phi_hi, *L.phi_lo, g, 1, s);
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
  if (h->tune_B == B && h->tune_nl == nl && h->tune_splits > 0) {  // the shapes a solve of this batch chose
    splits = h->tune_splits;
    kbps = h->tune_kbps;
    pair_adj = h->tune_pair_adj;
    pair_fwd = h->tune_pair_fwd;
  }
  GemmArgs g{};
  g.M = B; g.N = ng; g.K = nl; g.kb_per_split = kbps; g.epi = EPI_PARTIAL;
  g.P = T.P.as<float>(); g.ldp = (ng + 3) & ~3; g.err = h->d_err; g.timeout_ns = 2000000000ull;
  if (launch_adjoint(h, L, g, splits, pair_adj, s) != cudaSuccess) return DCOPF_ERR_CUDA;
  k_reduce_min<<<B, 256, 0, s>>>(h->dev, splits, B, g.ldp, T.P.as<float>(), lambda, T.ld_g,
                                 T.X_hi.as<__nv_bfloat16>(), T.X_lo.as<__nv_bfloat16>(),
                                 w.x64.as<double>(), w.sumcost.as<double>(), w.sump.as<double>());
  h->launches += 1;
  GemmArgs f{};
  f.M = B; f.N = nl; f.K = ng; f.kb_per_split = (ng + GBK - 1) / GBK; f.epi = EPI_FLOW;
  f.f0 = w.f0.as<double>(); f.f = w.f.as<double>(); f.ldf = nl; f.err = h->d_err;
  f.timeout_ns = 2000000000ull;
  if (launch_forward(h, L, f, pair_fwd, s) != cudaSuccess) return DCOPF_ERR_CUDA;
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
__global__ void __launch_bounds__(MIN_MAX_THREADS, 2)
    k_bt_minimize(DevNet N, int splits, int M, int ldp, const float* __restrict__ P,
                              SolveStateBase st, BatchView bb, StepArgs SP, int ldx,
                              __nv_bfloat16* __restrict__ Xh, __nv_bfloat16* __restrict__ Xl,
                              const int* __restrict__ outage, const double* __restrict__ demand) {
  __shared__ double red[3 * (MIN_MAX_THREADS / 32)];
  const int b = blockIdx.x;
  if (bb.frozen[b]) return;
  const int ng = N.n_gen;
  const int k = outage ? outage[b] : -1;
  const double lam = st.lam[b];
  // The in-loop value and the lambda gradient only steer the iteration (the bound is
  // certified in FP64 later): per-generator terms and warp sums in FP32, FP64 across
  // warps.  The reduced cost w = ctil + sigma lambda + pi~ is formed in FP32: its
  // rounding there (a few 2^-24 of |ctil| + |sigma lambda|) is far below the error of
  // the split BF16 products that give pi~.
  const float lamf = (float)lam;
  float c = 0.f, p = 0.f, to = 0.f;
  const float kk = (float)(st.iter[b] + 1), wk = kk * kk;  // weight of the mean of the minimisers
  const int nt = blockDim.x;
  // two generators per thread and loop, every load in flight before the arithmetic;
  // split-K partials summed in split order (a missing term adds +0)
  for (int ja = threadIdx.x; ja < ng; ja += 2 * nt) {
    const int jb = ja + nt;
    const bool vb = jb < ng;
    float sa = 0.f, sb = 0.f;
    for (int q0 = 0; q0 < splits; q0 += 8) {
      float ta[8], tb[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const size_t row = ((size_t)(q0 + u) * M + b) * ldp;
        ta[u] = q0 + u < splits ? P[row + ja] : 0.f;
        tb[u] = (q0 + u < splits && vb) ? P[row + jb] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) { sa += ta[u]; sb += tb[u]; }
    }
    auto gen = [&](int j, float sj) {
      const float mq = N.mq32[j];
      const float w = fmaf(N.sigma32[j], lamf, N.ctil32[j]) + sj;
      const float x = inner_x<float>(w, mq);
      if (st.xsum) st.xsum[(size_t)b * ng + j] += wk * x;
      split_bf16(x, Xh + (size_t)b * ldx + j, Xl + (size_t)b * ldx + j);
      c += fmaf(fmaf(mq, x, N.ctil32[j]), x, N.cconst32[j]);
      p += fmaf(N.sigma32[j], x, N.mid32[j]);
      if (k >= 0) to = fmaf(N.phi32[(size_t)k * ng + j], x, to);
    };
    gen(ja, sa);
    if (vb) gen(jb, sb);
  }
  c = warp_sum(c); p = warp_sum(p); to = warp_sum(to);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int RW = MIN_MAX_THREADS / 32;
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
    bb.cost[b] = cs;
    bb.psum[b] = ps;
    if (st.wsum) st.wsum[b] += (double)wk;
    bb.tout[b] = (float)ts;
    bb.lam_eval[b] = lam;
    // step t = iter + 1: scale decay^(t-1), bias corrections 1 - beta^t
    const double d = bb.pw[3 * b], b1 = bb.pw[3 * b + 1] * SP.beta1, b2 = bb.pw[3 * b + 2] * SP.beta2;
    const float bc1 = (float)(1.0 - b1), bc2 = (float)(1.0 - b2);
    bb.stepf[4 * b] = (float)(SP.alpha * d);
    bb.stepf[4 * b + 1] = bc1;
    bb.stepf[4 * b + 2] = bc2;
    bb.pw[3 * b] = d * SP.decay;
    bb.pw[3 * b + 1] = b1;
    bb.pw[3 * b + 2] = b2;
    // lambda's step: the moments and lambda in FP64, the Adam / AdaGrad direction in
    // FP32 (FP64 division and square root are slow on this part)
    const double g = ps - demand[b], a = SP.alpha_lambda * d;
    double s1 = st.lam_s1[b], s2 = st.lam_s2[b], l = lam;
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

// Dual value of the evaluated point (FP64), best value and its lambda, outage patch of
// the next eta, stop tests.  A stopping instance is frozen: one that reached its
// target with the point just evaluated (state buffer iter % 3), one stopped by the
// iteration cap or the tol test with its best point.  One warp per instance.
__global__ void k_bt_finalize(int B, int ld_l, int max_iters, double tol, SolveStateBase st,
                              BatchView bb, const int* __restrict__ outage,
                              const double* __restrict__ demand,
                              __nv_bfloat16* __restrict__ Hh, __nv_bfloat16* __restrict__ Hl) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (b >= B || bb.frozen[b]) return;
  const int nt = bb.n_tiles;
  double ls = 0.0, os = 0.0;
  for (int q = lane; q < nt; q += 32) {
    ls += bb.line_part[(size_t)b * nt + q];
    os += bb.out_part[(size_t)b * nt + q];
  }
  ls = warp_sum(ls);
  os = warp_sum(os);
  if (lane != 0) return;
  const double val = bb.cost[b] + bb.lam_eval[b] * (bb.psum[b] - demand[b]) + ls;
  const int t = st.iter[b] + 1;
  if (val > st.best[b]) { st.best[b] = val; st.best_iter[b] = t; bb.lam_best[b] = bb.lam_eval[b]; }
  const int k = outage ? outage[b] : -1;
  if (k >= 0) split_bf16((float)os, Hh + (size_t)b * ld_l + k, Hl + (size_t)b * ld_l + k);
  int c = 0;
  if (st.has_target && val >= st.thresh[b] + st.margin[b]) c = 1;
  else if (t >= max_iters) c = 2;
  else if (tol > 0.0 && t > 1 && fabs(val - st.prev[b]) < tol) c = 2;
  st.prev[b] = val;
  if (c) {
    st.cand[b] = c;
    bb.frozen[b] = 1;
    st.best_lam[b] = c == 1 ? bb.lam_eval[b] : bb.lam_best[b];
  } else {
    st.iter[b] = t;
  }
}

// Copies the frozen candidates' points to best_* and snapshots which instances are
// staged (snap[b] = 1): the certificate and the accept step of this round act on
// exactly those, while the next round's iterations may freeze others.  A candidate
// that reached its target is the point just evaluated (state buffer iter % 3); one
// stopped by the iteration cap or the tol test is its best point: point iter or
// iter - 1 (still in their buffers) or an older one (its saved copy).
__global__ void k_bt_select(int B, int nl, SolveState<float> st, BatchView bb, int* snap) {
  const int b = blockIdx.y;
  const bool staged = st.cand[b] && !st.done[b];
  if (blockIdx.x == 0 && threadIdx.x == 0) snap[b] = staged ? 1 : 0;
  if (!staged) return;
  const int it = st.iter[b];
  // how many points before the last one the staged point is (0 with no best yet)
  const int back = (st.cand[b] == 1 || st.best_iter[b] < 1) ? 0 : it + 1 - st.best_iter[b];
  const float* bh[3] = {st.mu_hi, bb.mu2_hi, bb.mu3_hi};
  const float* bl[3] = {st.mu_lo, bb.mu2_lo, bb.mu3_lo};
  const float* sh = back <= 1 ? bh[(it - back) % 3] : bb.sv_hi;
  const float* sl = back <= 1 ? bl[(it - back) % 3] : bb.sv_lo;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
    st.best_hi[(size_t)b * nl + i] = sh[(size_t)b * nl + i];
    st.best_lo[(size_t)b * nl + i] = sl[(size_t)b * nl + i];
  }
}

// After certification: accept, stop, or unfreeze with a larger in-loop margin.  The
// evaluation of a frozen point counts; an unfrozen instance moves on to the point
// already stepped to.
__global__ void k_bt_accept(int B, double ub_any, SolveStateBase st, BatchView bb,
                            const int* __restrict__ snap, int* active) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (snap[b] && !st.done[b] && st.cand[b]) {
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
  if (!st.done[b]) atomicAdd(active, 1);
}

__global__ void k_bt_init(int B, BatchView bb) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    bb.frozen[b] = 0;
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
      bb.small.alloc((size_t)B * 7 * sizeof(double) + (size_t)B * 6 * sizeof(float) + 1024)) {
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
  v.n_tiles = n_tiles;
  return DCOPF_OK;
}

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
};

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

// Autotuner of the batched products' shapes, on the first solve of a batch size:
//  - the adjoint: single CTAs (128 x 128 tiles) or CTA pairs (256 x 256), each with
//    split-K factors around a heuristic and the factors that fill whole waves; more
//    splits fill the SMs with CTAs but add FP32 partial traffic to the minimiser's
//    reduction, so each candidate is timed as adjoint + minimiser;
//  - the forward product: single CTAs or CTA pairs.
// Timed with CUDA events on the solve's stream; the fastest of each is kept per handle.
static dcopf_status tune_tensor_shapes(TensorRun& R, cudaStream_t cs) {
  dcopf_dual* h = R.it.h;
  const int B = R.it.B, ng = h->host.n_gen;
  TensorOps& T = h->tops;
  Workspace& w = h->ws;
  const int kb = (R.ls.nl + GBK - 1) / GBK;
  const bool pair_ok = B > GBM && h->tiles_mode != 1;
  const bool single_ok = h->tiles_mode <= 1 || B <= GBM;
  const int tv_lo = h->tiles_mode == 3 ? 2 : 1, tv_hi = h->tiles_mode == 2 ? 1 : 2;
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
    const int s0 = R.splits;
    for (int num : {1, 2, 3, 4, 6, 8}) add(0, (s0 * num + 2) / 4);
    // and the splits that fill whole waves (one CTA per SM): the last wave of a grid of
    // tiles x splits CTAs is then full rather than a few CTAs on an idle GPU
    const int tiles = ((B + GBM - 1) / GBM) * ((ng + GBN - 1) / GBN);
    for (int wv = 1; wv <= 4; ++wv) add(0, wv * h->sm_count / tiles);
  }
  if (pair_ok) {
    for (int tv = tv_lo; tv <= tv_hi; ++tv) {
      const int bn = tv == 1 ? 256 : 192;
      const int ptiles = ((B + PBM - 1) / PBM) * ((ng + bn - 1) / bn);
      const int slots = h->sm_count / 2;  // one pair per two SMs
      const int s0 = std::max(1, (slots + ptiles - 1) / ptiles);
      for (int num : {2, 3, 4, 6}) add(tv, (s0 * num + 2) / 4);
      for (int wv = 1; wv <= 3; ++wv) add(tv, wv * slots / ptiles);
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return DCOPF_ERR_CUDA;
  }
  auto timed = [&](auto&& body, float* ms) -> dcopf_status {
    for (int rep = 0; rep < 2; ++rep) {  // the first pass warms up
      if (cudaEventRecord(e0, cs) != cudaSuccess) return DCOPF_ERR_CUDA;
      for (int k = 0; k < 3; ++k)
        if (body() != cudaSuccess) return DCOPF_ERR_CUDA;
      if (cudaEventRecord(e1, cs) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
        return DCOPF_ERR_CUDA;
    }
    return DCOPF_OK;
  };
  static const char* kTiles[3] = {"single 128x128", "pairs 256x256", "pairs 256x192"};
  float best = 1e30f;
  Cand bc = cand.empty() ? Cand{0, 1} : cand[0];
  int best_per = (kb + bc.splits - 1) / bc.splits;
  dcopf_status out = DCOPF_OK;
  for (const Cand& c : cand) {
    GemmArgs g = R.ga;
    g.kb_per_split = (kb + c.splits - 1) / c.splits;
    float ms = 0.f;
    out = timed(
        [&] {
          cudaError_t e = launch_adjoint(h, R.ls, g, c.splits, c.tiles, cs);
          k_bt_minimize<<<B, minimize_threads(h, B), 0, cs>>>(h->dev, c.splits, B, g.ldp, T.P.as<float>(),
                                                              R.st, h->bb.v, R.P, T.ld_g,
                                                              T.X_hi.as<__nv_bfloat16>(),
                                                              T.X_lo.as<__nv_bfloat16>(), R.it.outage,
                                                              w.demand.as<double>());
          h->launches += 1;
          return e != cudaSuccess ? e : cudaGetLastError();
        },
        &ms);
    if (out != DCOPF_OK) break;
    if (h->verbose)
      fprintf(stderr, "dcopf: batch %d adjoint %s split-K %d: %.1f us per GEMM+min\n", B,
              kTiles[c.tiles], c.splits, 1e3f * ms / 3.f);
    if (ms < best) {
      best = ms;
      bc = c;
      best_per = g.kb_per_split;
    }
  }
  // the forward product, on the operands the runs above left
  int fwd = (pair_ok && !single_ok) ? tv_lo : 0;
  if (out == DCOPF_OK && pair_ok) {
    float bf = 1e30f;
    for (int tv = single_ok ? 0 : tv_lo; tv <= tv_hi && out == DCOPF_OK; ++tv) {
      if (tv > 0 && tv < tv_lo) continue;
      float ms = 0.f;
      out = timed([&] { return launch_forward(h, R.ls, R.gf, tv, cs); }, &ms);
      if (h->verbose) fprintf(stderr, "dcopf: batch %d forward %s: %.1f us\n", B, kTiles[tv], 1e3f * ms / 3.f);
      if (out == DCOPF_OK && ms < bf) {
        bf = ms;
        fwd = tv;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (out != DCOPF_OK) return out;
  int derr = 0;
  if (cudaMemcpy(&derr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  if (derr) return (dcopf_status)derr;
  h->tune_B = B;
  h->tune_nl = R.ls.nl;
  h->tune_splits = bc.splits;
  h->tune_kbps = best_per;
  h->tune_pair_adj = bc.tiles;
  h->tune_pair_fwd = fwd;
  if (h->verbose)
    fprintf(stderr, "dcopf: batch %d adjoint %s split-K %d (%.1f us per GEMM+min), forward %s\n", B,
            kTiles[bc.tiles], bc.splits, 1e3f * best / 3.f, kTiles[fwd]);
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
    L.fmax = S.lim.as<float>();
    L.fmin = S.lim.as<float>() + nk;
    L.f0 = S.f0c.as<float>();
    L.kept = S.kept.as<int>();
    L.pos = S.pos.as<int>();
  }
  const int nl = R.ls.nl;
  R.n_tiles = (nl + STEP_CHUNK - 1) / STEP_CHUNK;
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
  if (h->timing && !h->kev[0])
    for (int q = 0; q < 6; ++q)
      if (cudaEventCreate(&h->kev[q]) != cudaSuccess) return DCOPF_ERR_CUDA;
  if (h->shape_adj >= 0 && (h->tune_B != B || h->tune_nl != nl)) {  // shapes fixed at create: no timing
    const int kb = (nl + GBK - 1) / GBK;
    const bool pairs_fit = B > GBM;
    h->tune_B = B;
    h->tune_nl = nl;
    h->tune_kbps = (kb + h->shape_splits - 1) / h->shape_splits;
    h->tune_splits = (kb + h->tune_kbps - 1) / h->tune_kbps;
    h->tune_pair_adj = pairs_fit ? h->shape_adj : 0;
    h->tune_pair_fwd = pairs_fit ? h->shape_fwd : 0;
  }
  if (h->tune_B != B || h->tune_nl != nl) {
    if ((r = tune_tensor_shapes(R, cs))) return r;
    tensor_init_state(R, cs);  // the timed runs stepped lambda: start again
  }
  R.splits = h->tune_splits;
  R.ga.kb_per_split = h->tune_kbps;
  R.pair_adj = h->tune_pair_adj;
  R.pair_fwd = h->tune_pair_fwd;
  R.ga.skip = bb.frozen;
  R.gf.skip = bb.frozen;
  // the mean of the minimisers starts after the tuning runs
  return ensure_mean(h, B, &R.st, true, p.mean_dispatch != nullptr, cs);
}

// Enqueues `chunk` iterations (adjoint GEMM, minimiser, forward GEMM, step, value) on
// cs, which is capturing.
static bool tensor_enqueue_chunk(TensorRun& R, int chunk, cudaStream_t cs) {
  dcopf_dual* h = R.it.h;
  const int B = R.it.B, nl = R.ls.nl;
  TensorOps& T = h->tops;
  Workspace& w = h->ws;
  BatchView& bb = h->bb.v;
  bool ok = true;
  for (int it = 0; it < chunk && ok; ++it) {
    // timing on: event nodes around the kernels of the round's last iteration
    const bool mark = h->timing && h->kev[0] && it == chunk - 1;
    // (external event-record nodes: a plain record during capture only orders streams)
    auto ev = [&](int q) {
      if (mark) ok &= cudaEventRecordWithFlags(h->kev[q], cs, cudaEventRecordExternal) == cudaSuccess;
    };
    ev(0);
    ok &= launch_adjoint(h, R.ls, R.ga, R.splits, R.pair_adj, cs) == cudaSuccess;
    ev(1);
    k_bt_minimize<<<B, minimize_threads(h, B), 0, cs>>>(h->dev, R.splits, B, R.ga.ldp, T.P.as<float>(), R.st, bb, R.P,
                                     T.ld_g, T.X_hi.as<__nv_bfloat16>(), T.X_lo.as<__nv_bfloat16>(),
                                     R.it.outage, w.demand.as<double>());
    ev(2);
    ok &= launch_forward(h, R.ls, R.gf, R.pair_fwd, cs) == cudaSuccess;
    ev(3);
    if (nl % 4 == 0 && R.E.ldF % 4 == 0 && R.E.ldh % 4 == 0)
      k_bt_step4<<<dim3(R.n_tiles, B), STEP_THREADS, 0, cs>>>(R.E, nl);
    else
      k_bt_step<<<dim3(R.n_tiles, B), STEP_THREADS, 0, cs>>>(R.E, nl);
    ev(4);
    k_bt_finalize<<<(B + 3) / 4, 128, 0, cs>>>(B, R.ls.ld_l, R.p.max_iters, R.p.tol, R.st, bb,
                                               R.it.outage, w.demand.as<double>(),
                                               T.H_hi.as<__nv_bfloat16>(),
                                               T.H_lo.as<__nv_bfloat16>());
    ev(5);
  }
  return ok;
}

// After a chunk: stage and snapshot the frozen candidates (on the solve's stream cs),
// then certify them in FP64 on the certificate stream cc, which runs beside the next
// chunk of iterations (the staged instances stay frozen meanwhile).  `done_ev` is
// recorded on cc when the certificate has finished.
static dcopf_status tensor_stage_certify(TensorRun& R, cudaStream_t cs, cudaStream_t cc,
                                         cudaEvent_t staged_ev, cudaEvent_t done_ev) {
  dcopf_dual* h = R.it.h;
  const int B = R.it.B, nl = R.ls.nl, n_line = h->host.n_line;
  BatchView& bb = h->bb.v;
  int* snap = h->bb.snap.as<int>();
  k_bt_select<<<dim3((nl + 255) / 256, B), 256, 0, cs>>>(B, nl, R.st, bb, snap);
  const float* bh = R.st.best_hi;
  const float* bl = R.st.best_lo;
  if (R.ls.kept) {
    // the certificate evaluates the full problem: the staged points on every line,
    // zero on the screened ones
    float* fh = h->scr.full.as<float>();
    float* fl = fh + (size_t)B * n_line;
    const unsigned g = (unsigned)std::min<long long>(((long long)B * n_line + 255) / 256, 4096);
    k_screen_scatter_rows<<<g, 256, 0, cs>>>(B, n_line, nl, R.ls.pos, R.st.best_hi, fh);
    k_screen_scatter_rows<<<g, 256, 0, cs>>>(B, n_line, nl, R.ls.pos, R.st.best_lo, fl);
    h->launches += 2;
    bh = fh;
    bl = fl;
  }
  if (cudaEventRecord(staged_ev, cs) != cudaSuccess || cudaStreamWaitEvent(cc, staged_ev, 0) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  dcopf_status r = run_certify_t<float>(h, B, R.it.loads, R.it.outage, R.st.best_lam, bh, bl, R.st.cert,
                                        nullptr, snap, R.st.done, cc, true);
  if (r) return r;
  h->launches += 1;
  if (cudaEventRecord(done_ev, cc) != cudaSuccess) return DCOPF_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? DCOPF_OK : DCOPF_ERR_CUDA;
}

// Once the certificate of the staged instances is in (done_ev): accept, stop or resume
// each of them, on cs; adds the count of instances still running to *d_active.
static dcopf_status tensor_accept(TensorRun& R, int* d_active, cudaStream_t cs, cudaEvent_t done_ev) {
  dcopf_dual* h = R.it.h;
  const int B = R.it.B;
  if (cudaStreamWaitEvent(cs, done_ev, 0) != cudaSuccess) return DCOPF_ERR_CUDA;
  k_bt_accept<<<(B + 127) / 128, 128, 0, cs>>>(B, h->ub_any, R.st, h->bb.v, h->bb.snap.as<int>(),
                                               d_active);
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

// Owns the CUDA objects of one group solve.
struct GroupObjects {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev, stage_ev, cert_ev;
  DBuf active;
  ~GroupObjects() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    for (cudaEvent_t e : stage_ev) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : cert_ev) if (e) cudaEventDestroy(e);
  }
};

// Batched solves of several networks (distinct handles on one device) that advance
// together: each round is ONE launch of a CUDA graph holding every network's chunk
// of iterations as parallel branches, followed by each network's FP64 certification.
dcopf_status solve_tensor_group(const TensorItem* items, int n, const dcopf_solve_params& p,
                                cudaStream_t s) {
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
  G.ev.resize(2 * n + 1, nullptr);
  for (auto& e : G.ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return DCOPF_ERR_CUDA;
  if (G.active.alloc(sizeof(int) * (size_t)n) != cudaSuccess) return DCOPF_ERR_OOM;
  int* d_active = G.active.as<int>();
  // every stream starts after every setup
  for (int i = 1; i < n; ++i) {
    if (cudaEventRecord(G.ev[i], items[i].h->tstream) != cudaSuccess ||
        cudaStreamWaitEvent(cs0, G.ev[i], 0) != cudaSuccess)
      return DCOPF_ERR_CUDA;
  }
  std::vector<long long> before(n);
  for (int i = 0; i < n; ++i) before[i] = items[i].h->launches;
  if (cudaStreamBeginCapture(cs0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  bool cap_ok = cudaEventRecord(G.ev[0], cs0) == cudaSuccess;
  for (int i = 1; i < n && cap_ok; ++i)
    cap_ok = cudaStreamWaitEvent(items[i].h->tstream, G.ev[0], 0) == cudaSuccess;
  for (int i = 0; i < n && cap_ok; ++i) cap_ok = tensor_enqueue_chunk(runs[i], chunk, items[i].h->tstream);
  for (int i = 1; i < n && cap_ok; ++i)
    cap_ok = cudaEventRecord(G.ev[n + i], items[i].h->tstream) == cudaSuccess &&
             cudaStreamWaitEvent(cs0, G.ev[n + i], 0) == cudaSuccess;
  cudaError_t ce = cudaStreamEndCapture(cs0, &G.graph);
  for (int i = 0; i < n; ++i) items[i].h->launches = before[i];  // counted per replay below
  if (!cap_ok || ce != cudaSuccess || cudaGraphInstantiate(&G.exec, G.graph, 0) != cudaSuccess) {
    cudaGetLastError();
    return DCOPF_ERR_CUDA;
  }
  if (h0->timing && !h0->ev0) {
    cudaEventCreate(&h0->ev0);
    cudaEventCreate(&h0->ev1);
  }
  const long long per_chunk = 5LL * chunk;
  long long max_iters = 0;
  for (const TensorRun& R : runs) max_iters = std::max<long long>(max_iters, R.p.max_iters);
  // The certificate of round r's candidates runs on a side stream beside round r + 1's
  // iterations (the candidates stay frozen meanwhile); round r + 1 then accepts them.
  for (int i = 0; i < n; ++i) {
    dcopf_dual* hi = items[i].h;
    if (!hi->cstream && cudaStreamCreateWithFlags(&hi->cstream, cudaStreamNonBlocking) != cudaSuccess)
      return DCOPF_ERR_CUDA;
    if (hi->bb.snap.alloc(sizeof(int) * (size_t)items[i].B) != cudaSuccess) return DCOPF_ERR_OOM;
  }
  G.stage_ev.resize(n, nullptr);
  G.cert_ev.resize(n, nullptr);
  for (int i = 0; i < n; ++i)
    if (cudaEventCreateWithFlags(&G.stage_ev[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&G.cert_ev[i], cudaEventDisableTiming) != cudaSuccess)
      return DCOPF_ERR_CUDA;
  std::vector<int> act(n, 1);
  for (int round = 0;; ++round) {
    if (h0->timing) cudaEventRecord(h0->ev0, cs0);
    if (cudaGraphLaunch(G.exec, cs0) != cudaSuccess) return DCOPF_ERR_CUDA;
    for (int i = 0; i < n; ++i) items[i].h->launches += per_chunk;
    if (h0->timing) cudaEventRecord(h0->ev1, cs0);
    if (cudaMemsetAsync(d_active, 0, sizeof(int) * (size_t)n, cs0) != cudaSuccess ||
        cudaEventRecord(G.ev[2 * n], cs0) != cudaSuccess)
      return DCOPF_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
      cudaStream_t si = items[i].h->tstream;
      if (i > 0 && cudaStreamWaitEvent(si, G.ev[2 * n], 0) != cudaSuccess) return DCOPF_ERR_CUDA;
      if (!act[i]) continue;
      dcopf_status r;
      if (round > 0 && (r = tensor_accept(runs[i], d_active + i, si, G.cert_ev[i]))) return r;
      if ((r = tensor_stage_certify(runs[i], si, items[i].h->cstream, G.stage_ev[i], G.cert_ev[i])))
        return r;
    }
    for (int i = 1; i < n; ++i)
      if (cudaEventRecord(G.ev[n + i], items[i].h->tstream) != cudaSuccess ||
          cudaStreamWaitEvent(cs0, G.ev[n + i], 0) != cudaSuccess)
        return DCOPF_ERR_CUDA;
    if (round > 0 &&
        cudaMemcpyAsync(act.data(), d_active, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, cs0) !=
            cudaSuccess)
      return DCOPF_ERR_CUDA;
    if (cudaStreamSynchronize(cs0) != cudaSuccess) return DCOPF_ERR_CUDA;
    if (h0->timing) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, h0->ev0, h0->ev1);
      h0->t_iter_ms += ms;
      h0->t_iter_launches += per_chunk * n;
    }
    for (int i = 0; i < n; ++i) {
      dcopf_dual* hi = items[i].h;
      if (!hi->timing || !hi->kev[0] || !act[i]) continue;
      float km[5];
      bool kok = true;
      for (int q = 0; q < 5; ++q) kok &= cudaEventElapsedTime(&km[q], hi->kev[q], hi->kev[q + 1]) == cudaSuccess;
      if (!kok) { cudaGetLastError(); continue; }
      for (int q = 0; q < 5; ++q) hi->t_kernel_ms[q] += km[q];
      hi->t_kernel_samples += 1;
    }
    int any = 0;
    for (int i = 0; i < n; ++i) {
      int derr = 0;
      cudaMemcpy(&derr, items[i].h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
      if (derr) return (dcopf_status)derr;
      any |= act[i];
    }
    if (round > 0 && !any) break;
    if ((long long)round * chunk > 4LL * max_iters + 64) break;
  }
  // the last round's certificates: accept what they staged (nothing, when every
  // instance had stopped before that round)
  for (int i = 0; i < n; ++i) {
    dcopf_status r = tensor_accept(runs[i], d_active + i, items[i].h->tstream, G.cert_ev[i]);
    if (r) return r;
  }
  for (int i = 0; i < n; ++i) {
    dcopf_status r = tensor_finish(runs[i], s);
    if (r) return r;
  }
  return DCOPF_OK;
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
