/* Learned warm start for the dual ascent: a small multilayer perceptron that maps
 * bus loads to a dual point (lambda, mu_hi, mu_lo).
 *
 * The paper has no counterpart.  Its Remarks 1-2 (Section 3) state the fact this
 * relies on: every dual point with mu >= 0 gives a valid lower bound.  A proposal
 * from the network therefore never changes what a solve certifies; it changes only
 * where the ascent of Algorithm 1 starts and so how many iterations it needs.  Cold
 * start (lambda = mu = 0) remains the fallback.
 *
 * Architecture: x (n_in loads) -> Linear(n_in, n_hidden) -> GELU -> Linear(n_hidden,
 * n_hidden) -> GELU -> Linear(n_hidden, n_out).  GELU(z) = z * Phi(z) with Phi the
 * standard normal CDF (the exact form, through erf).  The output is (lambda, eta)
 * with n_out = 1 + n_line, and the dual point is mu_hi = max(eta, 0),
 * mu_lo = max(-eta, 0).
 *
 * Normalisation: inputs are mapped to (x - in_shift) * in_scale before the first
 * layer; the last layer's output u is mapped to out_shift + out_scale * u.  Training
 * minimises the mean squared error in the normalised output space,
 *   L = 1 / (B * n_out) * sum_b sum_o (u_bo - (y_bo - out_shift_o) / out_scale_o)^2.
 *
 * Precision: FP32 storage of parameters, moments and activations; products either on
 * the tensor cores with BF16 hi/lo split operands (about 16 significant bits) or in
 * FP32 SIMT; FP64 loss accumulation.
 *
 * Parameters: one flat FP32 vector, in this order, each matrix row-major:
 *   W1 [n_in][n_hidden], b1 [n_hidden], W2 [n_hidden][n_hidden], b2 [n_hidden],
 *   W3 [n_hidden][n_out], b3 [n_out].
 * The same layout is used for gradients.
 *
 * Conventions (as in dcopf_dual.h): array arguments are caller-owned DEVICE
 * pointers unless stated, row-major; every call is asynchronous on the given stream
 * (a cudaStream_t passed as void*, NULL for the legacy default stream); host-side
 * argument errors return immediately with DCOPF_ERR_INVALID_ARG and launch nothing.
 * A handle's workspace is sized for max_batch rows and shared by all its calls:
 * calls on one handle must not overlap on the device (issue them on one stream).
 */
#ifndef DCOPF_MLP_H
#define DCOPF_MLP_H

#include <stdint.h>

#include "dcopf_dual.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dcopf_mlp* dcopf_mlp_t; /* opaque; owned by the library */

typedef struct {
  int32_t n_in;      /* input width (number of buses), >= 1 */
  int32_t n_hidden;  /* width of both hidden layers, >= 1 */
  int32_t n_out;     /* output width (1 + number of lines), >= 1 */
  int32_t max_batch; /* largest batch of any call on this handle, >= 1 */
  int32_t precision; /* DCOPF_BF16X3: every product on the tcgen05 tensor cores with BF16
                        hi/lo split operands (three products, FP32 accumulation);
                        DCOPF_FP32: FP32 SIMT products */
} dcopf_mlp_desc;

typedef struct {
  double lr;    /* Adam step size */
  double beta1; /* first-moment decay */
  double beta2; /* second-moment decay */
  double eps;   /* added to the root of the second moment */
} dcopf_adam_params;

/* Allocates parameters (zero), Adam moments (zero), normalisation (identity) and the
 * workspace on the current device.  Errors: INVALID_ARG (sizes), OOM, CUDA. */
dcopf_status dcopf_mlp_create(const dcopf_mlp_desc* desc, dcopf_mlp_t* out);
dcopf_status dcopf_mlp_destroy(dcopf_mlp_t h);

/* Number of FP32 parameters:
 * n_in*n_hidden + n_hidden + n_hidden*n_hidden + n_hidden + n_hidden*n_out + n_out. */
int64_t dcopf_mlp_num_params(dcopf_mlp_t h);

/* Copies params [num_params] in; resets the Adam moments and step count. */
dcopf_status dcopf_mlp_set_params(dcopf_mlp_t h, const float* params, void* stream);
/* Copies the parameters out to params [num_params]. */
dcopf_status dcopf_mlp_get_params(dcopf_mlp_t h, float* params, void* stream);

/* Input map (x - in_shift) * in_scale ([n_in] each) and output map
 * out_shift + out_scale * u ([n_out] each). */
dcopf_status dcopf_mlp_set_normalization(dcopf_mlp_t h, const float* in_shift,
                                         const float* in_scale, const float* out_shift,
                                         const float* out_scale, void* stream);

/* y [batch][n_out] = output map of the network at the input map of x [batch][n_in].
 * 1 <= batch <= max_batch. */
dcopf_status dcopf_mlp_forward(dcopf_mlp_t h, int32_t batch, const float* x, float* y,
                               void* stream);

/* Loss and gradient on the rows idx [batch] of a data set X [n_rows][n_in], Y
 * [n_rows][n_out] (raw, un-normalised values).  loss [1] (FP32, nullable) receives L;
 * grad [num_params] (nullable) receives dL/dparams.  Parameters are not changed.
 * Every idx entry must lie in [0, n_rows): the call checks this on the device and
 * reports DCOPF_ERR_INVALID_ARG through dcopf_mlp_device_error. */
dcopf_status dcopf_mlp_loss_grad(dcopf_mlp_t h, int32_t batch, const int32_t* idx,
                                 int64_t n_rows, const float* X, const float* Y, float* loss,
                                 float* grad, void* stream);

/* One Adam step (bias-corrected, Kingma and Ba) on the loss of dcopf_mlp_loss_grad:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, t += 1,
 * p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * loss [1] (nullable) receives the loss before the step. */
dcopf_status dcopf_mlp_train_step(dcopf_mlp_t h, int32_t batch, const int32_t* idx,
                                  int64_t n_rows, const float* X, const float* Y,
                                  const dcopf_adam_params* adam, float* loss, void* stream);

/* Warm-start proposal for dcopf_dual_solve_batch: runs the network on loads
 * [batch][n_in] (FP64, p.u.) and writes lambda [batch], mu_hi and mu_lo
 * [batch][n_out - 1] (FP64) with mu_hi = max(eta, 0), mu_lo = max(-eta, 0). */
dcopf_status dcopf_mlp_warm_start(dcopf_mlp_t h, int32_t batch, const double* loads,
                                  double* lambda, double* mu_hi, double* mu_lo, void* stream);

/* First device-side error recorded by this handle's kernels since the last call
 * (DCOPF_OK if none); synchronises the device and clears the record. */
dcopf_status dcopf_mlp_device_error(dcopf_mlp_t h);

/* Number of kernels this handle has launched. */
int64_t dcopf_mlp_kernel_launches(dcopf_mlp_t h);

#ifdef __cplusplus
}
#endif

#endif /* DCOPF_MLP_H */
