// dcopf_dual_eval_noalloc: the dual evaluation of dcopf_dual_eval for callers that
// cannot allocate device memory themselves (for instance code running inside a host
// framework that owns every allocation, or a real-time loop where cudaMalloc's
// implicit synchronisation and latency are not allowed).  Its intermediate arrays
// live in one file-scope device array of fixed size instead of the handle's
// workspace, so the call performs no allocation at all.
#include <cstring>
#include <mutex>

#include "dcopf_dual.h"
#include "kernels.h"

namespace dcopf {

// Fixed scratch shared by every call of dcopf_dual_eval_noalloc on a device.  Every
// GPU that loads the library holds these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_addr_mutex;
void* g_addr[64] = {nullptr};  // device address of g_noalloc_scratch, per device ordinal

// The scratch array's device address for the current device, looked up once per
// device.  In host code the array's name is only a host-side stand-in, so kernels
// must get this address, never &g_noalloc_scratch.
dcopf_status scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= 64) return DCOPF_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return DCOPF_ERR_CUDA;
    }
    g_addr[device] = p;
  }
  *out = (unsigned char*)g_addr[device];
  return DCOPF_OK;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }
}  // namespace

}  // namespace dcopf

using namespace dcopf;

extern "C" dcopf_status dcopf_dual_eval_noalloc(dcopf_dual_t h, int32_t batch, const double* loads,
                                                const int32_t* outage, const double* lambda,
                                                const double* mu_hi, const double* mu_lo,
                                                int32_t precision, double* value, double* g_lambda,
                                                double* g_mu_hi, double* g_mu_lo, double* dispatch,
                                                void* stream) {
  // the same host checks, in the same order, as dcopf_dual_eval
  if (!h || batch < 1 || !loads) return DCOPF_ERR_INVALID_ARG;
  if ((long long)batch * h->host.n_line > (1ll << 31)) return DCOPF_ERR_UNSUPPORTED;
  if (certify_smem(h, true) > h->smem_optin) return DCOPF_ERR_UNSUPPORTED;
  if (!lambda || !mu_hi || !mu_lo || !value) return DCOPF_ERR_INVALID_ARG;
  if (precision != DCOPF_FP64 && precision != DCOPF_FP32 && precision != DCOPF_BF16X3)
    return DCOPF_ERR_INVALID_ARG;
  if (h->sparse_only) return DCOPF_ERR_UNSUPPORTED;  // the evaluation uses Phi~
  if (precision == DCOPF_BF16X3) return DCOPF_ERR_UNSUPPORTED;  // its operands need a workspace
  const size_t B = (size_t)batch, nl = (size_t)h->host.n_line, ng = (size_t)h->host.n_gen;
  // scratch carve-up: every section 256-byte aligned
  size_t need = 0;
  auto take = [&](size_t bytes) { size_t o = need; need += align256(bytes); return o; };
  const size_t o_f0 = take(B * nl * 8), o_u64 = take(B * nl * 8), o_dem = take(B * 8),
               o_f = take(B * nl * 8), o_sc = take(B * 8), o_sp = take(B * 8);
  size_t o_eta = 0, o_pit = 0, o_x = 0, o_u32 = 0;
  if (precision == DCOPF_FP64) {
    o_eta = take(B * nl * 8); o_pit = take(B * ng * 8); o_x = take(B * ng * 8);
  } else {
    o_eta = take(B * nl * 4); o_pit = take(B * ng * 4); o_x = take(B * ng * 4); o_u32 = take(B * nl * 4);
  }
  if (need > kNoAllocScratchBytes) return DCOPF_ERR_INVALID_ARG;  // batch too large for the scratch
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != h->device && cudaSetDevice(h->device) != cudaSuccess) return DCOPF_ERR_CUDA;
  dcopf_status r = DCOPF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  if ((r = scratch_address(h->device, &base)) == DCOPF_OK) {
    // outage indices: checked on the host in chunks through a fixed stack buffer
    if (outage) {
      int32_t chunk[1024];
      for (size_t b0 = 0; b0 < B && r == DCOPF_OK; b0 += 1024) {
        const size_t n = B - b0 < 1024 ? B - b0 : 1024;
        if (cudaMemcpyAsync(chunk, outage + b0, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
          cudaGetLastError();  // not a readable device pointer: leave no error behind
          r = DCOPF_ERR_INVALID_ARG;
          break;
        }
        for (size_t q = 0; q < n; ++q) {
          const int32_t k = chunk[q];
          if (k < -1 || k >= h->host.n_line) { r = DCOPF_ERR_INVALID_ARG; break; }
          if (k >= 0 && h->host.bridge[k]) { r = DCOPF_ERR_NETWORK; break; }
        }
      }
    }
  }
  if (r == DCOPF_OK) {
    EvalBuffers E{};
    E.f0 = (double*)(base + o_f0);
    E.u64 = (double*)(base + o_u64);
    E.demand = (double*)(base + o_dem);
    E.f = (double*)(base + o_f);
    E.sumcost = (double*)(base + o_sc);
    E.sump = (double*)(base + o_sp);
    if (precision == DCOPF_FP64) {
      E.eta64 = (double*)(base + o_eta); E.pit64 = (double*)(base + o_pit); E.x64 = (double*)(base + o_x);
    } else {
      E.eta32 = (float*)(base + o_eta); E.pit32 = (float*)(base + o_pit); E.x32 = (float*)(base + o_x);
      E.u32 = (float*)(base + o_u32);
    }
    // Every array is fully written by the kernels before it is read (the base-flow
    // kernel writes f0, u64 and demand for every instance), so nothing needs clearing.
    r = launch_base_flows_into(h, batch, loads, outage, E.f0, E.u64, E.demand, s);
    if (r == DCOPF_OK)
      r = launch_eval_into(h, batch, outage, lambda, mu_hi, mu_lo, precision, E, value, g_lambda,
                           g_mu_hi, g_mu_lo, dispatch, s);
  }
  if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
  return r;
}
