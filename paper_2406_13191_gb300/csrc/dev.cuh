// Device-side data structures and helpers shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "dcopf_dual.h"

namespace dcopf {

// Everything the kernels need to know about one network, as device pointers.
// Layouts: Phi~ row-major [n_line][n_gen] ("phi*"), its transpose [n_gen][n_line]
// ("phit*"); per-line and per-generator vectors are plain arrays.
constexpr int kIncEll = 4;

struct DevNet {
  int n_bus, n_line, n_gen, slack, qp;
  double S;
  // sparse LDL^T of the reduced Laplacian (elimination positions 0..nr-1)
  int nr;
  const int* pos_of_bus;   // [n_bus], -1 for slack
  const int* bus_of_pos;   // [nr]
  const int* lrow_ptr; const int* lrow_col; const double* lrow_val;
  const int* lcol_ptr; const int* lcol_row; const double* lcol_val;
  const double* diag;
  const int* fwd_rows; const int* fwd_lev; int n_fwd_lev;
  const int* bwd_rows; const int* bwd_lev; int n_bwd_lev;
  // the same schedules ELL-packed (SparseFactor::kEll slots per row, then an overflow)
  const int* fell_col; const double* fell_val; const int* fovf_ptr; const int* fovf_col; const double* fovf_val;
  const int* bell_col; const double* bell_val; const int* bovf_ptr; const int* bovf_col; const double* bovf_val;
  const double* winv1;     // [nr] upper bound of B_r^{-1} 1 (entries >= 0: B_r is an M-matrix)
  const double* inv_diag;  // [nr] 1 / diag (the solves that scale by a product)
  // packed copy of the factor for shared-memory staging (nullptr when unavailable)
  const unsigned char* fac_blob; int fac_bytes;
  int off_diag, off_val, off_rptr, off_cptr, off_rcol, off_crow, off_cmap, off_frows, off_brows,
      off_flev, off_blev;
  // lines
  const int* line_from; const int* line_to;
  const double* line_b;
  const double* fmax; const double* fmin;
  const float* fmax32; const float* fmin32;
  const double* phim;       // Phi mid [n_line]
  const int* bus_line_ptr; const int* bus_line_idx; const double* bus_line_coef;
  // the same incidences by elimination position q (the bus at q), in the same order: the
  // first kIncEll in slots [a * nr + q] (line -1 and coefficient 0 where unused), the rest
  // in an overflow CSR; each with the line, the other end's position (-1 for the slack
  // bus), the coefficient +-b_l and b_l
  const int* qe_line; const int* qe_opos; const double* qe_coef; const double* qe_b;
  const int* qo_ptr; const int* qo_line; const int* qo_opos; const double* qo_coef; const double* qo_b;
  const int* bus_gen_ptr; const int* bus_gen_idx;
  // generators
  const int* gen_bus;
  const double* pmin; const double* pmax; const double* cost_lin; const double* cost_quad;
  const double* sigma; const double* mid; const double* ctil; const double* mq; const double* cconst;
  const float* sigma32; const float* ctil32; const float* mq32; const float* cconst32;
  const float* mid32;
  // the minimiser's constants packed per generator: (sigma, ctil, mq, cconst) and
  // (mid, 1 / (2 mq), 0 for a linear cost)
  const float4* gen4; const float2* gen2;
  // dense operators
  const double* phi64; const double* phit64;
  const float* phi32; const float* phit32;
};

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block maximum; `sh` needs blockDim.x/32 slots.  All threads receive the result.
template <typename T>
__device__ __forceinline__ T block_max(T v, T* sh) {
  v = warp_max(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (w == 0) r = warp_max(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// Deterministic block sum (fixed tree); `sh` needs blockDim.x/32 slots.  All threads
// receive the result.  Must be called by every thread of the block.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (w == 0) r = warp_sum(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------- inner minimiser
// Normalised generator j (Appendix A1): p = mid + sigma x, |x| <= 1, cost
// mq x^2 + ctil x + cconst.  With w = ctil + sigma (lambda + pi_j) the Lagrangian
// term is mq x^2 + w x + const: eq. (6) gives x = -sign(w) for mq = 0 (tie -> 0,
// the box midpoint); eq. (16) maximised over s gives x = clip(-w / (2 mq), -1, 1).
template <typename T>
__device__ __forceinline__ T inner_x(T w, T mq) {
  if (mq > T(0)) {
    T x = -w / (T(2) * mq);
    return x > T(1) ? T(1) : (x < T(-1) ? T(-1) : x);
  }
  return w > T(0) ? T(-1) : (w < T(0) ? T(1) : T(0));
}

// FP64 minimum of cost_j(p) + nu p over [pmin, pmax] in physical units, used by
// the certificate (cost_j(p) = a (S p)^2 + c S p).
__device__ __forceinline__ double gen_min_value(double nu, double a, double c, double S,
                                                double pmin, double pmax, double* pstar) {
  double k = c * S + nu;
  double p;
  if (a > 0.0) {
    p = -k / (2.0 * a * S * S);
    p = p > pmax ? pmax : (p < pmin ? pmin : p);
    *pstar = p;
    return a * S * S * p * p + k * p;
  }
  p = k > 0.0 ? pmin : (k < 0.0 ? pmax : 0.5 * (pmin + pmax));
  *pstar = p;
  return k * p;
}

// ---------------------------------------------------------------- grid barrier
// Barrier over all CTAs of a cooperative launch.  `counter` is zero at launch and
// only grows; `epoch` is the caller's private count of barriers passed.  The wait is
// bounded by `timeout_ns` of wall-clock time: on expiry it records DCOPF_ERR_TIMEOUT
// in *err and returns false, so callers can leave their loops.
// Release-add at GPU scope: the writes that happen before it (the thread's own and,
// through bar.sync, the CTA's) are visible to any thread whose acquire load reads the
// result (PTX memory model, release pattern with cumulativity).
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits until *ctr >= target (wrap-safe), reading it with acquire semantics; gives up
// after timeout_ns of wall-clock time and returns false.  Used by every cross-CTA wait
// of the persistent kernels.
__device__ __forceinline__ bool bounded_wait_geq(const unsigned* ctr, unsigned target,
                                                 uint64_t timeout_ns) {
  uint64_t t0 = 0;
  int spins = 0;
  while ((int)(ld_acquire_u32(ctr) - target) < 0) {
    if ((++spins & 31) == 0) {
      const uint64_t now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > timeout_ns) return false;
    }
  }
  return true;
}

__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned nblocks, unsigned& epoch,
                                             int* err, uint64_t timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  epoch += 1;
  if (threadIdx.x == 0) {
    unsigned target = epoch * nblocks;
    __threadfence();
    atomicAdd(counter, 1u);
    int ok = 1;
    uint64_t t0 = 0;
    int spins = 0;
    while ((int)(ld_acquire_u32(counter) - target) < 0) {
      if (++spins == 64) { t0 = global_ns(); }
      if (spins > 64 && (spins & 255) == 0) {
        if (global_ns() - t0 > timeout_ns) { atomicExch(err, (int)DCOPF_ERR_TIMEOUT); ok = 0; break; }
        if (ld_relaxed_s32(err) != 0) { ok = 0; break; }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace dcopf
