// tcgen05 GEMMs of the batched solve with BF16 hi/lo split operands: C = A B^T over
// row-major [rows][K] operands (K-major), FP32 accumulation in TMEM.
//
// Precision: each FP32 operand v is split into BF16 v_hi = bf16(v) and
// v_lo = bf16(v - v_hi) and the product is hi*hi + hi*lo + lo*hi (NPROD = 3 MMAs per
// K step).  When one operand is exact in BF16 (the LP dispatch x in {-1, 0, 1}) its
// lo part is zero and NPROD = 2 suffices.
//
// k_gemm_bf16x: one 128 x 128 output tile per CTA (split along K where K is long and
// N short), 6 warps: warp 0 issues TMA loads of the BF16 tiles of a 64-wide K block
// into a ring with 128-byte swizzle, warp 1 allocates TMEM and one of its threads
// issues the MMAs, warps 2-5 read the accumulator from TMEM (tcgen05.ld) and run the
// epilogue.  The three-product GEMMs run one CTA per SM with a 3-stage ring; the
// two-product LP forward runs two CTAs per SM with a 2-stage ring each, so that one
// CTA's epilogue overlaps the other's loads.
// k_gemm_pair: the same on CTA pairs (cta_group::2), 256-row tiles.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>

#include "dev.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace dcopf {

enum { EPI_PARTIAL = 0, EPI_FLOW = 1, EPI_TILE = 2 };

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
  int bblk;              // B in 8-row blocks (4-D maps: element (r, c) at ((r/8 KB + c/64) 8 + r%8) 64 + c%64)
  int bpol;              // L2 policy of the CTA-pair B loads: 0 none, 1 evict_last, 2 evict_first,
                         // 3 evict_last for B's high part and evict_first for its low part
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
      if (g.bblk) {
        umma::tma_load_4d(&tBh, &full[s], b_hi(s), kb0 + i, n0 >> 3);
        umma::tma_load_4d(&tBl, &full[s], b_lo(s), kb0 + i, n0 >> 3);
      } else {
        umma::tma_load_2d(&tBh, &full[s], b_hi(s), x, n0);
        umma::tma_load_2d(&tBl, &full[s], b_lo(s), x, n0);
      }
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

// PBN: the pair tile's width (256, 192, 160 or 144 output columns, a multiple of 16;
// each CTA loads PBN / 2 rows of B).  The epilogue reads TMEM 32 columns at a time: for a
// width that is not a multiple of 32 the last read runs past the tile's columns into
// the rest of the (256-column) allocation, and those columns are not stored.
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
  static_assert(PBN % 16 == 0 && PBN <= 256 && (PBN + 31) / 32 * 32 <= (int)TMEM_COLS,
                "the epilogue's 32-column TMEM reads stay inside the allocation");
  static_assert(STAGES * STAGE_BYTES >= 128 * (PBN + 1) * 4, "the ring stages the output tile");
};

// MC pairs per cluster (1 or 2).  With two, the pairs of a cluster compute neighbouring
// column tiles from the same A rows, and each A box is loaded once for both: the CTA of
// the first pair multicasts A's high part, the CTA of the second its low part, to the
// CTAs of the same rank in both pairs.  A stage is then free only when both pairs' MMAs
// have read it: every MMA commit arrives on the empty barriers of all four CTAs.
template <int NPROD, int PBN, int MC = 1>
__global__ void __launch_bounds__(192, 1)
    k_gemm_pair(const __grid_constant__ CUtensorMap tAh, const __grid_constant__ CUtensorMap tAl,
                const __grid_constant__ CUtensorMap tBh, const __grid_constant__ CUtensorMap tBl,
                GemmArgs g) {
  static_assert(MC == 1 || MC == 2, "one or two pairs per cluster");
  using Cfg = PairCfg<NPROD, PBN>;
  constexpr int ST = Cfg::STAGES;
  extern __shared__ __align__(16) unsigned char gsm_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)gsm_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[ST], empty[ST], accf;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t crank = umma::cluster_ctarank();
  const uint32_t rank = crank & 1u;  // in the pair; 0 issues the pair's MMAs
  const uint32_t pc = crank >> 1;    // the pair in the cluster
  const uint16_t pair_mask = (uint16_t)(0x3u << (2 * pc)), all_mask = MC == 2 ? 0xF : 0x3;
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
      umma::mbar_init(&empty[s], MC);
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
    const uint64_t pol_last = umma::l2_policy_evict_last(), pol_first = umma::l2_policy_evict_first();
    for (int i = 0; i < nkb; ++i) {
      const int s = i % ST;
      if (i >= ST && !umma::mbar_wait(&empty[s], ((i / ST) & 1) ^ 1, g.timeout_ns)) {
        s_abort = 1;
        break;
      }
      if (rank == 0) umma::mbar_arrive_expect_tx(&full[s], 2 * Cfg::STAGE_BYTES);
      const uint32_t bar = umma::cluster_addr(&full[s], (int)(crank & ~1u));
      const int x = (kb0 + i) * GBK;
      if (MC == 1) {
        umma::tma_load_2d_pair(&tAh, bar, a_hi(s), x, my_m);
        if (NPROD == 3) umma::tma_load_2d_pair(&tAl, bar, a_lo(s), x, my_m);
      } else {
        const uint16_t amask = (uint16_t)((1u << crank) | (1u << (crank ^ 2u)));
        if (pc == 0) umma::tma_load_2d_pair_mc(&tAh, bar, a_hi(s), x, my_m, amask);
        if (NPROD == 3 && pc == 1) umma::tma_load_2d_pair_mc(&tAl, bar, a_lo(s), x, my_m, amask);
      }
      if (g.bpol) {
        const uint64_t ph = g.bpol == 2 ? pol_first : pol_last, pl = g.bpol == 1 ? pol_last : pol_first;
        if (g.bblk) {
          umma::tma_load_4d_pair_hint(&tBh, bar, b_hi(s), kb0 + i, my_n >> 3, ph);
          umma::tma_load_4d_pair_hint(&tBl, bar, b_lo(s), kb0 + i, my_n >> 3, pl);
        } else {
          umma::tma_load_2d_pair_hint(&tBh, bar, b_hi(s), x, my_n, ph);
          umma::tma_load_2d_pair_hint(&tBl, bar, b_lo(s), x, my_n, pl);
        }
      } else if (g.bblk) {
        umma::tma_load_4d_pair(&tBh, bar, b_hi(s), kb0 + i, my_n >> 3);
        umma::tma_load_4d_pair(&tBl, bar, b_lo(s), kb0 + i, my_n >> 3);
      } else {
        umma::tma_load_2d_pair(&tBh, bar, b_hi(s), x, my_n);
        umma::tma_load_2d_pair(&tBl, bar, b_lo(s), x, my_n);
      }
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
      umma::mma_commit_pair(&empty[s], all_mask);
    }
    umma::mma_commit_pair(&accf, pair_mask);
  } else if (warp >= 2) {
    // ---------------- epilogue (both CTAs): warp w reads TMEM lanes 32*(w%4) .. +31
    const bool ready = __all_sync(0xffffffffu, umma::mbar_wait(&accf, 0, g.timeout_ns));
    umma::tc_fence_after();
    const int q = warp & 3;
    const int row = my_m + 32 * q + lane;
    if (!ready) s_abort = 1;
    if (ready && nkb > 0) {
#pragma unroll 1
      for (int cc = 0; cc < (PBN + 31) / 32; ++cc) {
        float v[32];
        umma::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * cc), v);
        const int col0 = n0 + 32 * cc;
        const int lim = min(PBN - 32 * cc, g.N - col0);  // columns of this read that are output
        if (g.epi == EPI_TILE) {
          float* tile = (float*)base;
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (u < PBN - 32 * cc) tile[(32 * q + lane) * (PBN + 1) + 32 * cc + u] = v[u];
        } else if (row < g.M) {
          if (g.epi == EPI_PARTIAL) {
            float* dst = g.P + ((size_t)blockIdx.z * g.M + row) * g.ldp + col0;
            if (lim >= 32) {
#pragma unroll
              for (int u = 0; u < 8; ++u)
                reinterpret_cast<float4*>(dst)[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
            } else {
#pragma unroll
              for (int u = 0; u < 32; ++u)
                if (u < lim) dst[u] = v[u];
            }
          } else {
            const double* f0 = g.f0 + (size_t)row * g.ldf + col0;
            double* f = g.f + (size_t)row * g.ldf + col0;
#pragma unroll
            for (int u = 0; u < 32; ++u)
              if (u < lim) f[u] = (double)v[u] + f0[u];
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
      for (int q = 0; q < (PBN + 31) / 32; ++q) {
        const int c = lane + 32 * q;
        if (c < PBN && n0 + c < g.N) dst[n0 + c] = tile[m * (PBN + 1) + c];
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

}  // namespace dcopf
