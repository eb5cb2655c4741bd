// Micro-benchmarks of the GPU limits that bound this library's kernels (no
// counterpart in the paper): streaming reads from L2 or HBM, shared-memory reads,
// FP64 and FP32 FMA throughput and dependent-chain latency, the TMA tile feed from L2
// into shared memory that the tensor-core products run on, and one loop of the fused
// solve's exchange (in-cluster transaction-barrier pushes, arrival counters between
// clusters, a bulk copy) with no arithmetic around it.  Every wait is bounded.
#include <cooperative_groups.h>
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdio>

#include "dcopf_probe.h"
#include "dev.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace cg = cooperative_groups;

namespace dcopf {
namespace {

// Timed with CUDA events on the legacy default stream, after one warm-up launch.
template <typename F>
dcopf_status time_ms(F&& launch, int reps, double* ms_out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return DCOPF_ERR_CUDA;
  }
  launch();
  cudaEventRecord(e0, 0);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(e1, 0);
  float ms = 0.f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                  cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok) return DCOPF_ERR_CUDA;
  *ms_out = (double)ms / reps;
  return DCOPF_OK;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

struct DevMem {
  void* p = nullptr;
  ~DevMem() { if (p) cudaFree(p); }
};

// ---------------------------------------------------------------- streaming read
__global__ void k_probe_read(const float4* __restrict__ buf, size_t n4, int passes, float* sink) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
  if (acc.x + acc.y + acc.z + acc.w == 1234.5f) *sink = acc.x;  // keeps the loads
}

// ---------------------------------------------------------------- shared memory
__global__ void __launch_bounds__(256) k_probe_smem(int iters, float* sink) {
  __shared__ float4 s[2048];  // 32 KB
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) s[i] = make_float4(i, i, i, i);
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int idx = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {  // consecutive threads, consecutive 16-byte words
      const float4 v = s[(idx + u * 256) & 2047];
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    idx = (idx + 97) & 2047;
  }
  if (acc.x + acc.y + acc.z + acc.w == 1234.5f) *sink = acc.x;
}

// ---------------------------------------------------------------- FMA
template <typename T>
__global__ void __launch_bounds__(256) k_probe_fma(int iters, T b, T c, T* sink) {
  T a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = (T)(threadIdx.x + q);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = fma(a[q], b, c);
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  if (s == (T)1234.5) *sink = s;
}

template <typename T>
__global__ void k_probe_fma_chain(int iters, T b, T c, T* sink) {
  T a = (T)threadIdx.x;
  for (int it = 0; it < iters; ++it) a = fma(a, b, c);
  if (a == (T)1234.5) *sink = a;
}

// ---------------------------------------------------------------- TMA feed
// One CTA per SM keeps a ring of `ST` stages of four 16 KB BF16 tiles (128 x 64, 128-byte
// swizzle, the tensor-core GEMM's operand tiles) filled from an L2-resident matrix;
// a consumer thread releases each stage as soon as it lands.
constexpr int FEED_ST = 3;
constexpr uint32_t FEED_TILE = 128 * 64 * 2;

__global__ void __launch_bounds__(64, 1) k_probe_feed(const __grid_constant__ CUtensorMap map, int rows,
                                                     int cols, int n_stages, uint64_t timeout_ns,
                                                     int* err) {
  extern __shared__ __align__(16) unsigned char raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[FEED_ST], empty[FEED_ST];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < FEED_ST; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::fence_mbar_init();
  }
  __syncthreads();
  const int kx = cols / 64, ry = rows / 128;
  __shared__ int s_issued, s_landed;
  if (threadIdx.x == 0) { s_issued = 0; s_landed = 0; }
  __syncthreads();
  bool ok = true;
  if (warp == 0 && lane == 0) {
    for (int i = 0; i < n_stages && ok; ++i) {
      const int s = i % FEED_ST;
      if (i >= FEED_ST && !umma::mbar_wait(&empty[s], ((i / FEED_ST) & 1) ^ 1, timeout_ns)) {
        ok = false;
        break;
      }
      umma::mbar_arrive_expect_tx(&full[s], 4 * FEED_TILE);
      unsigned char* st = base + (size_t)s * 4 * FEED_TILE;
      for (int t = 0; t < 4; ++t) {
        const int x = ((blockIdx.x * 7 + i * 3 + t) % kx) * 64;
        const int y = ((blockIdx.x + i + 5 * t) % ry) * 128;
        umma::tma_load_2d(&map, &full[s], st + t * FEED_TILE, x, y);
      }
      s_issued = i + 1;
    }
  } else if (warp == 1 && lane == 0) {
    for (int i = 0; i < n_stages && ok; ++i) {
      const int s = i % FEED_ST;
      if (!umma::mbar_wait(&full[s], (i / FEED_ST) & 1, timeout_ns)) {
        ok = false;
        break;
      }
      s_landed = i + 1;
      umma::mbar_arrive(&empty[s]);
    }
  }
  const int failed = __syncthreads_or(ok ? 0 : 1);
  if (failed && threadIdx.x == 0) {
    atomicExch(err, (int)DCOPF_ERR_TIMEOUT);
    // no CTA leaves with its own copies in flight: wait (bounded) for every stage
    // issued but not yet seen to land
    for (int i = s_landed; i < s_issued; ++i)
      umma::mbar_wait(&full[i % FEED_ST], (i / FEED_ST) & 1, timeout_ns);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- exchange
struct ExArgs {
  float* Pc;          // [2][n_gen][NCLp]
  unsigned* cnt;      // [8] arrival counters, one per cluster rank
  int* err;
  int ng, SL, NCLp, loops;
  uint64_t timeout_ns;
};

// The fused solve's exchange with the arithmetic left out: per loop, every CTA pushes
// one float per generator into the shared memory of the rank owning the generator's
// slice (st.async on that rank's transaction barrier), waits for its slice, publishes
// the slice's cluster sum, release-adds its arrival, waits for every cluster's arrival
// (acquire polling), bulk-copies its slice's partials of every cluster, and pushes its
// slice's values and two sums and a flag to every peer (second transaction barrier).
__global__ void __launch_bounds__(256, 1) k_probe_exchange(ExArgs A) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int G = gridDim.x, c = blockIdx.x, cid = c / C, NCL = G / C, tid = threadIdx.x;
  const int ng = A.ng, SL = A.SL, NCLp = A.NCLp;
  const int j0 = min(ng, rank * SL), j1 = min(ng, j0 + SL), nj = j1 - j0;
  float* recv = (float*)sm_raw;                  // [C][SL]
  float* xs = recv + ((C * SL + 3) & ~3);        // [ng]
  float* tmp = xs + ((ng + 3) & ~3);             // [SL][NCLp]
  __shared__ __align__(8) uint64_t mb[3];
  __shared__ double s_sum[2 * 8];
  __shared__ int s_flag[8];
  const uint32_t tx_part = (uint32_t)((C - 1) * nj * 4);
  const uint32_t tx_x = (uint32_t)((ng - nj) * 4 + (C - 1) * 20);
  if (tid == 0) {
    for (int q = 0; q < 3; ++q) umma::mbar_init(&mb[q], 1);
    umma::fence_mbar_init();
  }
  cl.sync();
  for (int k = 0; k < A.loops; ++k) {
    float* Pcb = A.Pc + (size_t)(k & 1) * ng * NCLp;
    if (tid == 0) {
      umma::mbar_arrive_expect_tx(&mb[0], tx_part);
      umma::mbar_arrive_expect_tx(&mb[1], tx_x);
    }
    __syncthreads();
    for (int j = tid; j < ng; j += blockDim.x) {
      const int q = j / SL;
      float* dst = recv + rank * SL + (j - q * SL);
      const float v = (float)(j + k);
      if (q == rank) *dst = v;
      else umma::st_async_b32(umma::cluster_addr(dst, q), __float_as_uint(v), umma::cluster_addr(&mb[0], q));
    }
    __syncthreads();
    bool ok = umma::mbar_wait_cluster(&mb[0], k & 1, A.timeout_ns);
    for (int jj = tid; jj < nj; jj += blockDim.x) {
      float s = 0.f;
      for (int q = 0; q < C; ++q) s += recv[q * SL + jj];
      Pcb[(size_t)(j0 + jj) * NCLp + cid] = s;
    }
    __syncthreads();
    if (tid == 0) red_release_add_u32(A.cnt + rank, 1u);
    if (tid < C && !bounded_wait_geq(A.cnt + tid, (unsigned)NCL * (unsigned)(k + 1), A.timeout_ns)) ok = false;
    ok = __syncthreads_or(ok ? 0 : 1) == 0;
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)(nj * NCLp * 4);
      if (ok && bytes > 0) {
        umma::fence_proxy_async_global();
        umma::mbar_arrive_expect_tx(&mb[2], bytes);
        umma::bulk_g2s(tmp, Pcb + (size_t)j0 * NCLp, bytes, &mb[2]);
      } else {
        umma::mbar_arrive(&mb[2]);
      }
    }
    if (!umma::mbar_wait_cluster(&mb[2], k & 1, A.timeout_ns)) ok = false;
    __syncthreads();
    float part = 0.f;
    for (int jj = tid; jj < nj; jj += blockDim.x) {
      float s = 0.f;
      for (int q = 0; q < NCL; ++q) s += tmp[jj * NCLp + q];
      xs[j0 + jj] = s;
      part += s;
      for (int q = 0; q < C; ++q)
        if (q != rank)
          umma::st_async_b32(umma::cluster_addr(xs + j0 + jj, q), __float_as_uint(s),
                             umma::cluster_addr(&mb[1], q));
    }
    part = warp_sum(part);
    const int bad = __syncthreads_or(ok ? 0 : 1);
    if (tid < C) {  // two 8-byte sums and a flag to every rank
      const double v = (double)part;
      if (tid == rank) {
        s_sum[2 * rank] = v; s_sum[2 * rank + 1] = v; s_flag[rank] = bad;
      } else {
        const uint32_t bar = umma::cluster_addr(&mb[1], tid);
        umma::st_async_b64(umma::cluster_addr(s_sum + 2 * rank, tid), (uint64_t)__double_as_longlong(v), bar);
        umma::st_async_b64(umma::cluster_addr(s_sum + 2 * rank + 1, tid), (uint64_t)__double_as_longlong(v), bar);
        umma::st_async_b32(umma::cluster_addr(s_flag + rank, tid), (uint32_t)bad, bar);
      }
    }
    const bool x_ok = umma::mbar_wait_cluster(&mb[1], k & 1, A.timeout_ns);
    int any = __syncthreads_or(x_ok ? 0 : 1);
    for (int q = 0; q < C; ++q) any |= s_flag[q];
    if (any) {
      if (tid == 0) atomicExch(A.err, (int)DCOPF_ERR_TIMEOUT);
      break;
    }
  }
  cl.sync();  // no CTA leaves while a peer may still store into it
}

}  // namespace
}  // namespace dcopf

using namespace dcopf;

extern "C" {

dcopf_status dcopf_probe_read(int64_t footprint_bytes, int32_t passes, double* gbs) {
  if (footprint_bytes < (1 << 20) || footprint_bytes > (1ll << 36) || passes < 1 || passes > 1000 || !gbs)
    return DCOPF_ERR_INVALID_ARG;
  const size_t n4 = (size_t)footprint_bytes / 16;
  DevMem buf, sink;
  if (cudaMalloc(&buf.p, n4 * 16) != cudaSuccess || cudaMalloc(&sink.p, 16) != cudaSuccess)
    return DCOPF_ERR_OOM;
  if (cudaMemset(buf.p, 0, n4 * 16) != cudaSuccess) return DCOPF_ERR_CUDA;
  const int grid = 4 * sm_count();
  double ms = 0.0;
  dcopf_status r = time_ms([&] { k_probe_read<<<grid, 512>>>((const float4*)buf.p, n4, passes, (float*)sink.p); },
                           5, &ms);
  if (r) return r;
  *gbs = (double)n4 * 16.0 * passes / (ms * 1e-3) / 1e9;
  return DCOPF_OK;
}

dcopf_status dcopf_probe_smem(double* gbs) {
  if (!gbs) return DCOPF_ERR_INVALID_ARG;
  DevMem sink;
  if (cudaMalloc(&sink.p, 16) != cudaSuccess) return DCOPF_ERR_OOM;
  const int grid = 4 * sm_count(), iters = 4096;
  double ms = 0.0;
  dcopf_status r = time_ms([&] { k_probe_smem<<<grid, 256>>>(iters, (float*)sink.p); }, 5, &ms);
  if (r) return r;
  *gbs = (double)grid * 256 * iters * 8 * 16 / (ms * 1e-3) / 1e9;
  return DCOPF_OK;
}

dcopf_status dcopf_probe_fma(int32_t fp64, double* tflops, double* chain_ns) {
  if (!tflops || !chain_ns) return DCOPF_ERR_INVALID_ARG;
  DevMem sink;
  if (cudaMalloc(&sink.p, 16) != cudaSuccess) return DCOPF_ERR_OOM;
  const int grid = 8 * sm_count(), iters = fp64 ? 4096 : 65536, chain = 1 << 16;
  double ms = 0.0, ms_chain = 0.0;
  dcopf_status r;
  if (fp64) {
    r = time_ms([&] { k_probe_fma<double><<<grid, 256>>>(iters, 0.999999, 1e-7, (double*)sink.p); }, 3, &ms);
    if (!r) r = time_ms([&] { k_probe_fma_chain<double><<<1, 1>>>(chain, 0.999999, 1e-7, (double*)sink.p); }, 3, &ms_chain);
  } else {
    r = time_ms([&] { k_probe_fma<float><<<grid, 256>>>(iters, 0.999999f, 1e-7f, (float*)sink.p); }, 3, &ms);
    if (!r) r = time_ms([&] { k_probe_fma_chain<float><<<1, 1>>>(chain, 0.999999f, 1e-7f, (float*)sink.p); }, 3, &ms_chain);
  }
  if (r) return r;
  *tflops = 2.0 * 8.0 * grid * 256.0 * iters / (ms * 1e-3) / 1e12;
  *chain_ns = ms_chain * 1e6 / chain;
  return DCOPF_OK;
}

dcopf_status dcopf_probe_tma_feed(int64_t footprint_bytes, double* gbs) {
  if (footprint_bytes < (4 << 20) || footprint_bytes > (1ll << 32) || !gbs) return DCOPF_ERR_INVALID_ARG;
  const int cols = 12800;  // BF16 elements per row (200 tiles of 64)
  const int rows = std::max(128, (int)(footprint_bytes / (2 * cols)) / 128 * 128);
  DevMem buf, err;
  if (cudaMalloc(&buf.p, (size_t)rows * cols * 2) != cudaSuccess || cudaMalloc(&err.p, 16) != cudaSuccess)
    return DCOPF_ERR_OOM;
  if (cudaMemset(buf.p, 0, (size_t)rows * cols * 2) != cudaSuccess || cudaMemset(err.p, 0, 16) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  CUtensorMap map;
  if (!tc_make_map(&map, buf.p, rows, cols, cols)) return DCOPF_ERR_CUDA;
  const size_t smem = (size_t)FEED_ST * 4 * FEED_TILE + 1024;
  if (cudaFuncSetAttribute(k_probe_feed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  const int grid = sm_count(), stages = 2000;
  double ms = 0.0;
  dcopf_status r = time_ms(
      [&] { k_probe_feed<<<grid, 64, smem>>>(map, rows, cols, stages, 2000000000ull, (int*)err.p); }, 5, &ms);
  if (r) return r;
  int e = 0;
  if (cudaMemcpy(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DCOPF_ERR_CUDA;
  if (e) return (dcopf_status)e;
  *gbs = (double)grid * stages * 4.0 * FEED_TILE / (ms * 1e-3) / 1e9;
  return DCOPF_OK;
}

dcopf_status dcopf_probe_exchange(int32_t cluster, int32_t grid, int32_t n_gen, int32_t loops,
                                  double* us_per_loop) {
  if (!us_per_loop || (cluster != 2 && cluster != 4 && cluster != 8) || n_gen < cluster ||
      n_gen > 100000 || loops < 1 || loops > 100000)
    return DCOPF_ERR_INVALID_ARG;
  const int sms = sm_count();
  const int G = grid > 0 ? grid : sms / cluster * cluster;
  if (G % cluster || G > 256 || G > sms) return DCOPF_ERR_INVALID_ARG;
  const int NCL = G / cluster, NCLp = (NCL + 3) & ~3, SL = (n_gen + cluster - 1) / cluster;
  const size_t smem = ((size_t)((cluster * SL + 3) & ~3) + ((n_gen + 3) & ~3) + (size_t)SL * NCLp) * 4;
  if (smem > 200 * 1024) return DCOPF_ERR_UNSUPPORTED;
  DevMem pc, cnt;
  if (cudaMalloc(&pc.p, (size_t)2 * n_gen * NCLp * 4) != cudaSuccess || cudaMalloc(&cnt.p, 256) != cudaSuccess)
    return DCOPF_ERR_OOM;
  if (cudaFuncSetAttribute(k_probe_exchange, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  ExArgs A{};
  A.Pc = (float*)pc.p;
  A.cnt = (unsigned*)cnt.p;
  A.err = (int*)((char*)cnt.p + 128);
  A.ng = n_gen; A.SL = SL; A.NCLp = NCLp; A.loops = loops;
  A.timeout_ns = 200000000ull;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  bool coop_ok = true;
  auto launch = [&] {
    cudaMemsetAsync(cnt.p, 0, 256, 0);
    cfg.numAttrs = coop_ok ? 2 : 1;
    if (cudaLaunchKernelEx(&cfg, k_probe_exchange, A) != cudaSuccess && coop_ok) {
      cudaGetLastError();
      coop_ok = false;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_probe_exchange, A);
    }
  };
  double ms = 0.0;
  dcopf_status r = time_ms(launch, 5, &ms);
  if (r) return r;
  int e = 0;
  if (cudaMemcpy(&e, A.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DCOPF_ERR_CUDA;
  if (e) return (dcopf_status)e;
  *us_per_loop = ms * 1e3 / loops;
  return DCOPF_OK;
}

}  // extern "C"
