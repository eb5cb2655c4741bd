// Learned warm start: a two-hidden-layer GELU perceptron from bus loads to a dual
// point, with its training (forward, mean-squared-error gradient, Adam) on the GPU.
// Two modes: every product on the tcgen05 tensor cores with BF16 hi/lo split operands
// and FP32 accumulation (the tcgen05 GEMM of the batched solve), or FP32 SIMT.
// Any proposal with mu >= 0 is a valid dual point (Section 3, Remarks 1-2), so the
// network only changes where the ascent of Algorithm 1 starts.
//
// Every product is one FP32 SIMT GEMM kernel with a fused epilogue (bias, GELU and
// the stored pre-activation on the way forward; the GELU derivative on the way
// back); the small kernels around it gather and normalise a minibatch, form the
// output gradient and loss, sum bias gradients and apply Adam.  All reductions have
// a fixed order, so a call is deterministic for a given launch shape.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <new>

#include "dcopf_mlp.h"
#include "kernels.h"

using namespace dcopf;

namespace {

constexpr int TBM = 64, TBN = 64, TBK = 16, GEMM_THREADS = 256;
enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_BACK = 3 };

// GELU(z) = z Phi(z), Phi the standard normal CDF, and its derivative
// Phi(z) + z phi(z).
__device__ __forceinline__ float gelu_f(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
  return cdf + z * pdf;
}

__device__ __forceinline__ float epilogue(int epi, float v, int m, int n, const float* bias, float* Z,
                                          int ldz) {
  if (epi == EPI_BIAS || epi == EPI_BIAS_GELU) v += bias[n];
  if (epi == EPI_BIAS_GELU) {
    Z[(size_t)m * ldz + n] = v;
    v = gelu_f(v);
  }
  if (epi == EPI_GELU_BACK) v *= gelu_grad_f(Z[(size_t)m * ldz + n]);
  return v;
}

// C[M][N] = op(A)[M][K] op(B)[K][N] with the epilogue EPI.  op(A)(m, k) is
// A[m*lda + k], or A[k*lda + m] when TA; op(B)(k, n) is B[k*ldb + n], or B[n*ldb + k]
// when TB.  64 x 64 output tile per block, 16-deep K slices staged in shared memory,
// a 4 x 4 register tile per thread (rows ty + 16i, columns tx + 16j).  Split K: block
// z covers k in [z kper, (z+1) kper) and writes C + z czs (then EPI is EPI_STORE and
// k_splitk_reduce finishes the sum in a fixed order).
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GEMM_THREADS)
    k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda, const float* __restrict__ B,
            int ldb, float* __restrict__ C, int ldc, const float* __restrict__ bias,
            float* __restrict__ Z, int ldz, int kper, size_t czs) {
  __shared__ float As[TBK][TBM + 1];
  __shared__ float Bs[TBK][TBN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const int kbeg = blockIdx.z * kper;
  const int kend = min(K, kbeg + kper);
  C += blockIdx.z * czs;
  float acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += TBK) {
#pragma unroll
    for (int e = 0; e < (TBM * TBK) / GEMM_THREADS; ++e) {
      const int q = tid + e * GEMM_THREADS;
      int m, k;
      if (TA) { m = q % TBM; k = q / TBM; } else { k = q % TBK; m = q / TBK; }
      const int gm = m0 + m, gk = k0 + k;
      float v = 0.f;
      if (gm < M && gk < kend) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[k][m] = v;
    }
#pragma unroll
    for (int e = 0; e < (TBN * TBK) / GEMM_THREADS; ++e) {
      const int q = tid + e * GEMM_THREADS;
      int n, k;
      if (TB) { k = q % TBK; n = q / TBK; } else { n = q % TBN; k = q / TBN; }
      const int gn = n0 + n, gk = k0 + k;
      float v = 0.f;
      if (gn < N && gk < kend) v = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      C[(size_t)m * ldc + n] = epilogue(EPI, acc[i][j], m, n, bias, Z, ldz);
    }
  }
}

// C[m][n] = epilogue(sum over z = 0..S-1 of Pz[m][n]), slices S apart by M*N.
template <int EPI>
__global__ void k_splitk_reduce(int M, int N, int S, const float* __restrict__ Pz,
                                float* __restrict__ C, int ldc, const float* __restrict__ bias,
                                float* __restrict__ Z, int ldz) {
  const size_t MN = (size_t)M * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < MN;
       e += (size_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int z = 0; z < S; ++z) v += Pz[z * MN + e];
    const int m = (int)(e / N), n = (int)(e - (size_t)m * N);
    C[(size_t)m * ldc + n] = epilogue(EPI, v, m, n, bias, Z, ldz);
  }
}

// ---- tensor-core mode: BF16 hi/lo split operands for the tcgen05 GEMM
//
// BF16 hi/lo split of an FP32 matrix S [M][N] (leading dimension lds): row-major copies
// (hi, lo, ld ldr) and/or transposed copies (hiT, loT: [N][ldt]).  The transposed copies
// get zeros in columns [M, Mpad): the padding of a contraction over M.  32 x 32 tiles
// through shared memory; block (32, 8).
__global__ void k_split2d(int M, int N, int Mpad, const float* __restrict__ S, int lds,
                          __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int ldr,
                          __nv_bfloat16* __restrict__ hiT, __nv_bfloat16* __restrict__ loT,
                          int ldt) {
  __shared__ float t[32][33];
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < 32; r += 8) {
    const int m = m0 + r, n = n0 + tx;
    const bool in = m < M && n < N;
    const float v = in ? S[(size_t)m * lds + n] : 0.f;
    t[r][tx] = v;
    if (hi && in) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hi[(size_t)m * ldr + n] = h;
      lo[(size_t)m * ldr + n] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
  if (!hiT) return;  // uniform across the block
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int n = n0 + r, m = m0 + tx;
    if (n < N && m < Mpad) {
      const float v = t[tx][r];
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hiT[(size_t)n * ldt + m] = h;
      loT[(size_t)n * ldt + m] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

// out[m][n] = epilogue(sum over the K slices s = 0..S-1 of P[s][m][n]) (fixed order).
template <int EPI>
__global__ void k_reduce_epi(int M, int N, int S, const float* __restrict__ P, int ldp,
                             const float* __restrict__ bias, float* __restrict__ Z, int ldz,
                             float* __restrict__ out, int ldo) {
  const size_t MN = (size_t)M * N;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < MN;
       e += (size_t)gridDim.x * blockDim.x) {
    const int m = (int)(e / N), n = (int)(e - (size_t)m * N);
    float v = 0.f;
    for (int sl = 0; sl < S; ++sl) v += P[((size_t)sl * M + m) * ldp + n];
    out[(size_t)m * ldo + n] = epilogue(EPI, v, m, n, bias, Z, ldz);
  }
}

// Xn[b][i] = (X[r][i] - shift[i]) * scale[i], r = idx[b] (or b without idx).  A row
// index outside [0, n_rows) records DCOPF_ERR_INVALID_ARG and yields a zero row.
template <typename T>
__global__ void k_mlp_in(int Bn, int n_in, const int* __restrict__ idx, int64_t n_rows,
                         const T* __restrict__ X, const float* __restrict__ shift,
                         const float* __restrict__ scale, float* __restrict__ Xn, int* err) {
  const int b = blockIdx.y;
  const int64_t r = idx ? (int64_t)idx[b] : (int64_t)b;
  const bool ok = r >= 0 && r < n_rows;
  if (!ok && blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(err, 0, (int)DCOPF_ERR_INVALID_ARG);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_in; i += gridDim.x * blockDim.x)
    Xn[(size_t)b * n_in + i] = ok ? ((float)X[r * n_in + i] - shift[i]) * scale[i] : 0.f;
}

constexpr int OUT_BLOCKS = 296, OUT_THREADS = 256;

// dU = 2 / (B n_out) (U - T) with T the normalised targets of rows idx; the squared
// error summed per block (FP32 per thread, FP64 across the block) into part[block].
__global__ void __launch_bounds__(OUT_THREADS)
    k_mlp_out_grad(int Bn, int n_out, const float* __restrict__ U, const int* __restrict__ idx,
                   int64_t n_rows, const float* __restrict__ Y, const float* __restrict__ shift,
                   const float* __restrict__ inv_scale, float* __restrict__ dU, double* part) {
  __shared__ double sh[OUT_THREADS / 32];
  const int64_t total = (int64_t)Bn * n_out;
  const float g = 2.0f / (float)total;
  float s = 0.f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / n_out), o = (int)(e - (int64_t)b * n_out);
    const int64_t r = idx ? (int64_t)idx[b] : (int64_t)b;
    float d = 0.f;
    if (r >= 0 && r < n_rows) d = U[e] - (Y[r * n_out + o] - shift[o]) * inv_scale[o];
    dU[e] = g * d;
    s = fmaf(d, d, s);
  }
  const double t = block_sum((double)s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_mlp_loss(int nparts, const double* __restrict__ part, double denom, float* loss) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int q = threadIdx.x; q < nparts; q += blockDim.x) s += part[q];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *loss = (float)(s / denom);
}

// db[n] = sum over rows of D[m][n] (fixed row order).
__global__ void k_colsum(int M, int N, const float* __restrict__ D, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += D[(size_t)m * N + n];
  db[n] = s;
}

__global__ void k_adam(int64_t P, float* __restrict__ p, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float b1, float b2, float c1,
                       float c2, float eps) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= c1 * mi / (sqrtf(vi * c2) + eps);
  }
}

__global__ void k_out_map(int64_t total, int n_out, const float* __restrict__ U,
                          const float* __restrict__ shift, const float* __restrict__ scale,
                          float* __restrict__ Yo) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int o = (int)(e % n_out);
    Yo[e] = fmaf(scale[o], U[e], shift[o]);
  }
}

// (lambda, eta) = output map of U; mu_hi = max(eta, 0), mu_lo = max(-eta, 0).
__global__ void k_to_duals(int Bn, int n_out, const float* __restrict__ U,
                           const float* __restrict__ shift, const float* __restrict__ scale,
                           double* __restrict__ lam, double* __restrict__ mh,
                           double* __restrict__ ml) {
  const int b = blockIdx.y, nl = n_out - 1;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x) {
    const double y = (double)shift[o] + (double)scale[o] * (double)U[(size_t)b * n_out + o];
    if (o == 0) {
      lam[b] = y;
    } else {
      mh[(size_t)b * nl + o - 1] = y > 0.0 ? y : 0.0;
      ml[(size_t)b * nl + o - 1] = y < 0.0 ? -y : 0.0;
    }
  }
}

__global__ void k_recip(int n, const float* __restrict__ a, float* __restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = 1.0f / a[i];
}

__global__ void k_fill(int64_t n, float* __restrict__ a, float v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = v;
}

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace

// A BF16 hi/lo split operand of the tcgen05 GEMM and its tensor maps.
struct TcOp {
  DBuf hi, lo;
  CUtensorMap mh, ml;
  int ld = 0;
};

struct dcopf_mlp {
  int n_in = 0, nh = 0, n_out = 0, max_batch = 0;
  // tensor-core mode: every product on tcgen05 with BF16 hi/lo split operands
  int tensor = 0;
  int ldi = 0, ldh = 0, ldo = 0, ldb = 0;  // padded leading dimensions (BF16 elements)
  TcOp XnS, H1S, H2S, dUS, dZ2S;           // activations as A operands, [max_batch][features]
  TcOp XnT, H1T, H2T, dZ2T, dZ1T, dUT;     // transposed, [features][ldb] (contractions over the batch)
  TcOp W1T, W2T, W3T, W2R, W3R;            // weights: transposed for the forward, as stored for the backward
  DBuf tcP;                                // split-K partial products
  int64_t P = 0, o_b1 = 0, o_W2 = 0, o_b2 = 0, o_W3 = 0, o_b3 = 0;
  int64_t adam_t = 0;
  int64_t launches = 0;
  int sm_count = 1;
  size_t splitk_cap = 0;  // floats in `splitk`
  DBuf params, grad, mom1, mom2, norm, part, err, splitk;
  DBuf Xn, Z1, H1, Z2, H2, U, dU, D1, D2;
  float* in_shift() const { return norm.as<float>(); }
  float* in_scale() const { return norm.as<float>() + n_in; }
  float* out_shift() const { return norm.as<float>() + 2 * n_in; }
  float* out_scale() const { return norm.as<float>() + 2 * n_in + n_out; }
  float* out_inv() const { return norm.as<float>() + 2 * n_in + 2 * n_out; }
};

namespace {

constexpr int TC_MAX_SPLITS = 16;

inline int pad_to(int v, int q) { return (v + q - 1) / q * q; }

// K slices tc_gemm_partial uses for an M x N x K product (the same rule).
int tc_splits(int M, int N, int K, int sms) {
  const int tiles = cdiv(M, 128) * cdiv(N, 128);
  const int kb = cdiv(K, 64);
  int sp = std::max(1, std::min(std::min(kb, TC_MAX_SPLITS), (int)cdiv(2 * sms, tiles)));
  const int per = cdiv(kb, sp);
  return (int)cdiv(kb, per);
}

bool tc_op_alloc(TcOp& o, int rows, int cols, int ld) {
  o.ld = ld;
  const size_t bytes = (size_t)rows * ld * 2;
  if (o.hi.alloc(bytes) != cudaSuccess || o.lo.alloc(bytes) != cudaSuccess) return false;
  if (cudaMemset(o.hi.p, 0, bytes) != cudaSuccess || cudaMemset(o.lo.p, 0, bytes) != cudaSuccess)
    return false;
  return tc_make_map(&o.mh, o.hi.p, rows, cols, ld) && tc_make_map(&o.ml, o.lo.p, rows, cols, ld);
}

// BF16 hi/lo copies of an FP32 matrix (row-major R and/or transposed T, see k_split2d).
void tc_split(dcopf_mlp* h, cudaStream_t s, int M, int N, int Mpad, const float* S, int lds,
              TcOp* R, TcOp* T) {
  dim3 grid(cdiv(N, 32), cdiv(std::max(M, Mpad), 32));
  k_split2d<<<grid, dim3(32, 8), 0, s>>>(
      M, N, Mpad, S, lds, R ? R->hi.as<__nv_bfloat16>() : nullptr,
      R ? R->lo.as<__nv_bfloat16>() : nullptr, R ? R->ld : 0, T ? T->hi.as<__nv_bfloat16>() : nullptr,
      T ? T->lo.as<__nv_bfloat16>() : nullptr, T ? T->ld : 0);
  h->launches += 1;
}

// out = epilogue(A B^T) for A [M][K], B [N][K] split operands; fixed-order K slices.
template <int EPI>
void tc_product(dcopf_mlp* h, cudaStream_t s, const TcOp& A, const TcOp& B, int M, int N, int K,
                const float* bias, float* Z, int ldz, float* out, int ldo) {
  const int ldp = pad_to(N, 4);
  int sp = 1;
  tc_gemm_partial(A.mh, A.ml, B.mh, B.ml, M, N, K, h->tcP.as<float>(), ldp, TC_MAX_SPLITS,
                  h->sm_count, h->err.as<int>(), &sp, s);
  const int64_t total = (int64_t)M * N;
  k_reduce_epi<EPI><<<(int)std::min<int64_t>(cdiv(total, 256), 8 * h->sm_count), 256, 0, s>>>(
      M, N, sp, h->tcP.as<float>(), ldp, bias, Z, ldz, out, ldo);
  h->launches += 2;
}

// Weight operands from the FP32 parameters (after every change of the parameters).
void tc_refresh_weights(dcopf_mlp* h, cudaStream_t s) {
  const float* P = h->params.as<float>();
  const int ni = h->n_in, nh = h->nh, no = h->n_out;
  tc_split(h, s, ni, nh, ni, P, nh, nullptr, &h->W1T);
  tc_split(h, s, nh, nh, nh, P + h->o_W2, nh, &h->W2R, &h->W2T);
  tc_split(h, s, nh, no, nh, P + h->o_W3, no, &h->W3R, &h->W3T);
}

// Forward pass of the rows in Xn on the tensor cores; with `train`, also the
// transposed operands the backward pass contracts over the batch.
void forward_rows_tc(dcopf_mlp* h, cudaStream_t s, int Bn, bool train) {
  const float* P = h->params.as<float>();
  const int ni = h->n_in, nh = h->nh, no = h->n_out;
  const int Bp = train ? pad_to(Bn, 64) : Bn;
  tc_split(h, s, Bn, ni, Bp, h->Xn.as<float>(), ni, &h->XnS, train ? &h->XnT : nullptr);
  tc_product<EPI_BIAS_GELU>(h, s, h->XnS, h->W1T, Bn, nh, ni, P + h->o_b1, h->Z1.as<float>(), nh,
                            h->H1.as<float>(), nh);
  tc_split(h, s, Bn, nh, Bp, h->H1.as<float>(), nh, &h->H1S, train ? &h->H1T : nullptr);
  tc_product<EPI_BIAS_GELU>(h, s, h->H1S, h->W2T, Bn, nh, nh, P + h->o_b2, h->Z2.as<float>(), nh,
                            h->H2.as<float>(), nh);
  tc_split(h, s, Bn, nh, Bp, h->H2.as<float>(), nh, &h->H2S, train ? &h->H2T : nullptr);
  tc_product<EPI_BIAS>(h, s, h->H2S, h->W3T, Bn, no, nh, P + h->o_b3, nullptr, 0, h->U.as<float>(), no);
}

// Splits of the products (and thus the partial buffer) for every product of a call
// with batch Bn: the largest over the batches a handle accepts sizes the buffer.
size_t tc_partial_floats(const dcopf_mlp* h) {
  const int ni = h->n_in, nh = h->nh, no = h->n_out, sms = h->sm_count;
  size_t most = 0;
  for (int Bn = 1; Bn <= h->max_batch; ++Bn) {  // every batch: the maxima sit at tile edges
    const int prod[8][3] = {{Bn, nh, ni}, {Bn, nh, nh}, {Bn, no, nh}, {nh, no, Bn},
                            {Bn, nh, no}, {nh, nh, Bn}, {Bn, nh, nh}, {ni, nh, Bn}};
    for (auto& q : prod)
      most = std::max(most, (size_t)tc_splits(q[0], q[1], q[2], sms) * q[0] * pad_to(q[1], 4));
  }
  return most;
}

// One product with its epilogue.  When the output tiles cannot fill the SMs twice,
// K is split into S slices (multiples of the K tile, at least 256 deep) written to the
// split-K buffer and summed by k_splitk_reduce, which applies the epilogue.
template <bool TA, bool TB, int EPI>
void gemm(dcopf_mlp* h, cudaStream_t s, int M, int N, int K, const float* A, int lda,
          const float* B, int ldb, float* C, int ldc, const float* bias = nullptr,
          float* Z = nullptr, int ldz = 0) {
  const int tiles = cdiv(N, TBN) * cdiv(M, TBM);
  int S = 1;
  if (tiles < 2 * h->sm_count) {
    S = std::min(cdiv(2 * h->sm_count, tiles), std::max(1, K / 256));
    while (S > 1 && (size_t)S * M * N > h->splitk_cap) --S;
  }
  if (S <= 1) {
    dim3 grid(cdiv(N, TBN), cdiv(M, TBM), 1);
    k_sgemm<TA, TB, EPI><<<grid, GEMM_THREADS, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Z, ldz,
                                                       K, 0);
    h->launches += 1;
    return;
  }
  const int kper = cdiv(cdiv(K, S), TBK) * TBK;
  S = cdiv(K, kper);
  float* P = h->splitk.as<float>();
  dim3 grid(cdiv(N, TBN), cdiv(M, TBM), S);
  k_sgemm<TA, TB, EPI_STORE><<<grid, GEMM_THREADS, 0, s>>>(M, N, K, A, lda, B, ldb, P, N, nullptr,
                                                           nullptr, 0, kper, (size_t)M * N);
  const int rb = (int)std::min<int64_t>(cdiv((int64_t)M * N, 256), 8 * h->sm_count);
  k_splitk_reduce<EPI><<<rb, 256, 0, s>>>(M, N, S, P, C, ldc, bias, Z, ldz);
  h->launches += 2;
}

// Forward pass of the rows already normalised in Xn: Z1, H1, Z2, H2 and U (the
// normalised output).
void forward_rows(dcopf_mlp* h, cudaStream_t s, int Bn, bool train = false) {
  if (h->tensor) {
    forward_rows_tc(h, s, Bn, train);
    return;
  }
  const float* P = h->params.as<float>();
  const int ni = h->n_in, nh = h->nh, no = h->n_out;
  gemm<false, false, EPI_BIAS_GELU>(h, s, Bn, nh, ni, h->Xn.as<float>(), ni, P, nh,
                                    h->H1.as<float>(), nh, P + h->o_b1, h->Z1.as<float>(), nh);
  gemm<false, false, EPI_BIAS_GELU>(h, s, Bn, nh, nh, h->H1.as<float>(), nh, P + h->o_W2, nh,
                                    h->H2.as<float>(), nh, P + h->o_b2, h->Z2.as<float>(), nh);
  gemm<false, false, EPI_BIAS>(h, s, Bn, no, nh, h->H2.as<float>(), nh, P + h->o_W3, no,
                               h->U.as<float>(), no, P + h->o_b3);
}

template <typename T>
void gather_rows(dcopf_mlp* h, cudaStream_t s, int Bn, const int* idx, int64_t n_rows, const T* X) {
  dim3 grid(cdiv(h->n_in, 256), Bn);
  k_mlp_in<T><<<grid, 256, 0, s>>>(Bn, h->n_in, idx, n_rows, X, h->in_shift(), h->in_scale(),
                                   h->Xn.as<float>(), h->err.as<int>());
  h->launches += 1;
}

// Loss and gradient into h->grad (and *loss when given).
void loss_grad_rows(dcopf_mlp* h, cudaStream_t s, int Bn, const int* idx, int64_t n_rows,
                    const float* X, const float* Y, float* loss) {
  const float* P = h->params.as<float>();
  float* G = h->grad.as<float>();
  const int ni = h->n_in, nh = h->nh, no = h->n_out;
  gather_rows<float>(h, s, Bn, idx, n_rows, X);
  forward_rows(h, s, Bn, true);
  k_mlp_out_grad<<<OUT_BLOCKS, OUT_THREADS, 0, s>>>(Bn, no, h->U.as<float>(), idx, n_rows, Y,
                                                    h->out_shift(), h->out_inv(),
                                                    h->dU.as<float>(), h->part.as<double>());
  h->launches += 1;
  if (loss) {
    k_mlp_loss<<<1, 256, 0, s>>>(OUT_BLOCKS, h->part.as<double>(), (double)Bn * no, loss);
    h->launches += 1;
  }
  if (h->tensor) {
    // the same chain rule on the tensor cores: weight gradients contract over the batch
    // (transposed operands, zero-padded to the K tile), input gradients over the outputs
    const int Bp = pad_to(Bn, 64);
    tc_split(h, s, Bn, no, Bp, h->dU.as<float>(), no, &h->dUS, &h->dUT);
    tc_product<EPI_STORE>(h, s, h->H2T, h->dUT, nh, no, Bn, nullptr, nullptr, 0, G + h->o_W3, no);
    k_colsum<<<cdiv(no, 256), 256, 0, s>>>(Bn, no, h->dU.as<float>(), G + h->o_b3);
    tc_product<EPI_GELU_BACK>(h, s, h->dUS, h->W3R, Bn, nh, no, nullptr, h->Z2.as<float>(), nh,
                              h->D2.as<float>(), nh);
    tc_split(h, s, Bn, nh, Bp, h->D2.as<float>(), nh, &h->dZ2S, &h->dZ2T);
    tc_product<EPI_STORE>(h, s, h->H1T, h->dZ2T, nh, nh, Bn, nullptr, nullptr, 0, G + h->o_W2, nh);
    k_colsum<<<cdiv(nh, 256), 256, 0, s>>>(Bn, nh, h->D2.as<float>(), G + h->o_b2);
    tc_product<EPI_GELU_BACK>(h, s, h->dZ2S, h->W2R, Bn, nh, nh, nullptr, h->Z1.as<float>(), nh,
                              h->D1.as<float>(), nh);
    tc_split(h, s, Bn, nh, Bp, h->D1.as<float>(), nh, nullptr, &h->dZ1T);
    tc_product<EPI_STORE>(h, s, h->XnT, h->dZ1T, ni, nh, Bn, nullptr, nullptr, 0, G, nh);
    k_colsum<<<cdiv(nh, 256), 256, 0, s>>>(Bn, nh, h->D1.as<float>(), G + h->o_b1);
    h->launches += 3;
    return;
  }
  // layer 3: dW3 = H2^T dU, db3 = column sums of dU, dZ2 = (dU W3^T) * GELU'(Z2)
  gemm<true, false, EPI_STORE>(h, s, nh, no, Bn, h->H2.as<float>(), nh, h->dU.as<float>(), no,
                               G + h->o_W3, no);
  k_colsum<<<cdiv(no, 256), 256, 0, s>>>(Bn, no, h->dU.as<float>(), G + h->o_b3);
  h->launches += 1;
  gemm<false, true, EPI_GELU_BACK>(h, s, Bn, nh, no, h->dU.as<float>(), no, P + h->o_W3, no,
                                   h->D2.as<float>(), nh, nullptr, h->Z2.as<float>(), nh);
  // layer 2
  gemm<true, false, EPI_STORE>(h, s, nh, nh, Bn, h->H1.as<float>(), nh, h->D2.as<float>(), nh,
                               G + h->o_W2, nh);
  k_colsum<<<cdiv(nh, 256), 256, 0, s>>>(Bn, nh, h->D2.as<float>(), G + h->o_b2);
  h->launches += 1;
  gemm<false, true, EPI_GELU_BACK>(h, s, Bn, nh, nh, h->D2.as<float>(), nh, P + h->o_W2, nh,
                                   h->D1.as<float>(), nh, nullptr, h->Z1.as<float>(), nh);
  // layer 1
  gemm<true, false, EPI_STORE>(h, s, ni, nh, Bn, h->Xn.as<float>(), ni, h->D1.as<float>(), nh, G,
                               nh);
  k_colsum<<<cdiv(nh, 256), 256, 0, s>>>(Bn, nh, h->D1.as<float>(), G + h->o_b1);
  h->launches += 1;
}

dcopf_status launch_status() {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return DCOPF_OK;
  return e == cudaErrorMemoryAllocation ? DCOPF_ERR_OOM : DCOPF_ERR_CUDA;
}

bool valid(const dcopf_mlp* h, int Bn) { return h && Bn >= 1 && Bn <= h->max_batch; }

}  // namespace

extern "C" {

dcopf_status dcopf_mlp_create(const dcopf_mlp_desc* d, dcopf_mlp_t* out) {
  if (!d || !out) return DCOPF_ERR_INVALID_ARG;
  *out = nullptr;
  if (d->n_in < 1 || d->n_hidden < 1 || d->n_out < 1 || d->max_batch < 1) return DCOPF_ERR_INVALID_ARG;
  if (d->precision != DCOPF_FP32 && d->precision != DCOPF_BF16X3) return DCOPF_ERR_INVALID_ARG;
  const int64_t ni = d->n_in, nh = d->n_hidden, no = d->n_out, mb = d->max_batch;
  if (ni * nh > (1LL << 31) || nh * no > (1LL << 31) || mb * (ni > no ? ni : no) > (1LL << 31))
    return DCOPF_ERR_INVALID_ARG;
  dcopf_mlp* h = new (std::nothrow) dcopf_mlp();
  if (!h) return DCOPF_ERR_OOM;
  h->tensor = d->precision == DCOPF_BF16X3 ? 1 : 0;
  h->n_in = d->n_in;
  h->nh = d->n_hidden;
  h->n_out = d->n_out;
  h->max_batch = d->max_batch;
  h->o_b1 = ni * nh;
  h->o_W2 = h->o_b1 + nh;
  h->o_b2 = h->o_W2 + nh * nh;
  h->o_W3 = h->o_b2 + nh;
  h->o_b3 = h->o_W3 + nh * no;
  h->P = h->o_b3 + no;
  const size_t P4 = (size_t)h->P * 4;
  bool ok = h->params.alloc(P4) == cudaSuccess && h->grad.alloc(P4) == cudaSuccess &&
            h->mom1.alloc(P4) == cudaSuccess && h->mom2.alloc(P4) == cudaSuccess &&
            h->norm.alloc((size_t)(2 * ni + 3 * no) * 4) == cudaSuccess &&
            h->part.alloc(OUT_BLOCKS * 8) == cudaSuccess && h->err.alloc(16) == cudaSuccess &&
            h->Xn.alloc((size_t)mb * ni * 4) == cudaSuccess &&
            h->U.alloc((size_t)mb * no * 4) == cudaSuccess &&
            h->dU.alloc((size_t)mb * no * 4) == cudaSuccess;
  for (DBuf* b : {&h->Z1, &h->H1, &h->Z2, &h->H2, &h->D1, &h->D2})
    ok = ok && b->alloc((size_t)mb * nh * 4) == cudaSuccess;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    ok = false;
  // split K only where tiles < 2 SMs: S * M * N < (2 SMs + tiles) * 64 * 64 <= 4 SMs * 4096
  h->splitk_cap = (size_t)4 * h->sm_count * TBM * TBN;
  ok = ok && h->splitk.alloc(h->splitk_cap * 4) == cudaSuccess;
  if (ok && h->tensor) {
    const int ni_ = h->n_in, nh_ = h->nh, no_ = h->n_out, mb_ = h->max_batch;
    h->ldi = pad_to(ni_, 8);
    h->ldh = pad_to(nh_, 8);
    h->ldo = pad_to(no_, 8);
    h->ldb = pad_to(mb_, 64);
    ok = tc_gemm_prepare() == cudaSuccess &&
         tc_op_alloc(h->XnS, mb_, ni_, h->ldi) && tc_op_alloc(h->H1S, mb_, nh_, h->ldh) &&
         tc_op_alloc(h->H2S, mb_, nh_, h->ldh) && tc_op_alloc(h->dUS, mb_, no_, h->ldo) &&
         tc_op_alloc(h->dZ2S, mb_, nh_, h->ldh) && tc_op_alloc(h->XnT, ni_, h->ldb, h->ldb) &&
         tc_op_alloc(h->H1T, nh_, h->ldb, h->ldb) && tc_op_alloc(h->H2T, nh_, h->ldb, h->ldb) &&
         tc_op_alloc(h->dZ2T, nh_, h->ldb, h->ldb) && tc_op_alloc(h->dZ1T, nh_, h->ldb, h->ldb) &&
         tc_op_alloc(h->dUT, no_, h->ldb, h->ldb) && tc_op_alloc(h->W1T, nh_, ni_, h->ldi) &&
         tc_op_alloc(h->W2T, nh_, nh_, h->ldh) && tc_op_alloc(h->W2R, nh_, nh_, h->ldh) &&
         tc_op_alloc(h->W3T, no_, nh_, h->ldh) && tc_op_alloc(h->W3R, nh_, no_, h->ldo) &&
         h->tcP.alloc(tc_partial_floats(h) * 4) == cudaSuccess;
  }
  if (!ok) {
    delete h;
    cudaGetLastError();
    return DCOPF_ERR_OOM;
  }
  cudaMemset(h->params.p, 0, P4);
  cudaMemset(h->grad.p, 0, P4);
  cudaMemset(h->mom1.p, 0, P4);
  cudaMemset(h->mom2.p, 0, P4);
  cudaMemset(h->err.p, 0, 16);
  cudaMemset(h->norm.p, 0, (size_t)(2 * ni + 3 * no) * 4);
  k_fill<<<cdiv(ni, 256), 256>>>(ni, h->in_scale(), 1.f);
  k_fill<<<cdiv(no, 256), 256>>>(no, h->out_scale(), 1.f);
  k_fill<<<cdiv(no, 256), 256>>>(no, h->out_inv(), 1.f);
  h->launches += 3;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    delete h;
    return DCOPF_ERR_CUDA;
  }
  *out = h;
  return DCOPF_OK;
}

dcopf_status dcopf_mlp_destroy(dcopf_mlp_t h) {
  if (!h) return DCOPF_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  delete h;
  return DCOPF_OK;
}

int64_t dcopf_mlp_num_params(dcopf_mlp_t h) { return h ? h->P : -1; }

dcopf_status dcopf_mlp_set_params(dcopf_mlp_t h, const float* params, void* stream) {
  if (!h || !params) return DCOPF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P4 = (size_t)h->P * 4;
  if (cudaMemcpyAsync(h->params.p, params, P4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(h->mom1.p, 0, P4, s) != cudaSuccess ||
      cudaMemsetAsync(h->mom2.p, 0, P4, s) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  h->adam_t = 0;
  if (h->tensor) tc_refresh_weights(h, s);
  return launch_status();
}

dcopf_status dcopf_mlp_get_params(dcopf_mlp_t h, float* params, void* stream) {
  if (!h || !params) return DCOPF_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(params, h->params.p, (size_t)h->P * 4, cudaMemcpyDeviceToDevice,
                      (cudaStream_t)stream) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  return DCOPF_OK;
}

dcopf_status dcopf_mlp_set_normalization(dcopf_mlp_t h, const float* in_shift, const float* in_scale,
                                         const float* out_shift, const float* out_scale,
                                         void* stream) {
  if (!h || !in_shift || !in_scale || !out_shift || !out_scale) return DCOPF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ni4 = (size_t)h->n_in * 4, no4 = (size_t)h->n_out * 4;
  if (cudaMemcpyAsync(h->in_shift(), in_shift, ni4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(h->in_scale(), in_scale, ni4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(h->out_shift(), out_shift, no4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(h->out_scale(), out_scale, no4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  k_recip<<<cdiv(h->n_out, 256), 256, 0, s>>>(h->n_out, h->out_scale(), h->out_inv());
  h->launches += 1;
  return launch_status();
}

dcopf_status dcopf_mlp_forward(dcopf_mlp_t h, int32_t batch, const float* x, float* y, void* stream) {
  if (!valid(h, batch) || !x || !y) return DCOPF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  gather_rows<float>(h, s, batch, nullptr, batch, x);
  forward_rows(h, s, batch);
  const int64_t total = (int64_t)batch * h->n_out;
  k_out_map<<<cdiv(total, 256) < 2048 ? cdiv(total, 256) : 2048, 256, 0, s>>>(
      total, h->n_out, h->U.as<float>(), h->out_shift(), h->out_scale(), y);
  h->launches += 1;
  return launch_status();
}

dcopf_status dcopf_mlp_loss_grad(dcopf_mlp_t h, int32_t batch, const int32_t* idx, int64_t n_rows,
                                 const float* X, const float* Y, float* loss, float* grad,
                                 void* stream) {
  if (!valid(h, batch) || !idx || n_rows < 1 || !X || !Y) return DCOPF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  loss_grad_rows(h, s, batch, idx, n_rows, X, Y, loss);
  if (grad && cudaMemcpyAsync(grad, h->grad.p, (size_t)h->P * 4, cudaMemcpyDeviceToDevice, s) !=
                  cudaSuccess)
    return DCOPF_ERR_CUDA;
  return launch_status();
}

dcopf_status dcopf_mlp_train_step(dcopf_mlp_t h, int32_t batch, const int32_t* idx, int64_t n_rows,
                                  const float* X, const float* Y, const dcopf_adam_params* a,
                                  float* loss, void* stream) {
  if (!valid(h, batch) || !idx || n_rows < 1 || !X || !Y || !a) return DCOPF_ERR_INVALID_ARG;
  if (!(a->lr > 0.0) || !(a->beta1 >= 0.0 && a->beta1 < 1.0) || !(a->beta2 >= 0.0 && a->beta2 < 1.0) ||
      !(a->eps > 0.0))
    return DCOPF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  loss_grad_rows(h, s, batch, idx, n_rows, X, Y, loss);
  h->adam_t += 1;
  const double c1 = a->lr / (1.0 - pow(a->beta1, (double)h->adam_t));
  const double c2 = 1.0 / (1.0 - pow(a->beta2, (double)h->adam_t));
  k_adam<<<cdiv(h->P, 256) < 4096 ? cdiv(h->P, 256) : 4096, 256, 0, s>>>(
      h->P, h->params.as<float>(), h->grad.as<float>(), h->mom1.as<float>(), h->mom2.as<float>(),
      (float)a->beta1, (float)a->beta2, (float)c1, (float)c2, (float)a->eps);
  h->launches += 1;
  if (h->tensor) tc_refresh_weights(h, s);
  return launch_status();
}

dcopf_status dcopf_mlp_warm_start(dcopf_mlp_t h, int32_t batch, const double* loads, double* lambda,
                                  double* mu_hi, double* mu_lo, void* stream) {
  if (!valid(h, batch) || !loads || !lambda || !mu_hi || !mu_lo || h->n_out < 2)
    return DCOPF_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  gather_rows<double>(h, s, batch, nullptr, batch, loads);
  forward_rows(h, s, batch);
  dim3 grid(cdiv(h->n_out, 256), batch);
  k_to_duals<<<grid, 256, 0, s>>>(batch, h->n_out, h->U.as<float>(), h->out_shift(),
                                  h->out_scale(), lambda, mu_hi, mu_lo);
  h->launches += 1;
  return launch_status();
}

dcopf_status dcopf_mlp_device_error(dcopf_mlp_t h) {
  if (!h) return DCOPF_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return DCOPF_ERR_CUDA;
  int e = 0;
  if (cudaMemcpy(&e, h->err.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(h->err.p, 0, sizeof(int)) != cudaSuccess)
    return DCOPF_ERR_CUDA;
  return (dcopf_status)e;
}

int64_t dcopf_mlp_kernel_launches(dcopf_mlp_t h) { return h ? h->launches : -1; }

}  // extern "C"
