/*
 * dcopf_probe.h -- micro-benchmarks of the GPU limits that bound libdcopfdual's
 * kernels.  The paper has no counterpart: these calls measure the denominators of
 * the library's roofline figures (the fused single-instance solve is bound by the
 * latency of its exchange between CTAs, the batched products by the tensor cores and
 * the feed of their operands from L2, the step by HBM).
 *
 * Every call runs on the calling thread's current CUDA device, allocates and frees
 * its own device memory, enqueues on the legacy default stream, times with CUDA
 * events after one warm-up launch, synchronises the device and returns a
 * dcopf_status (dcopf_dual.h).  Outputs are host pointers.  Every device wait is
 * bounded; a wait that gives up returns DCOPF_ERR_TIMEOUT.
 */
#ifndef DCOPF_PROBE_H
#define DCOPF_PROBE_H

#include <stdint.h>

#include "dcopf_dual.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Streaming read bandwidth: every SM reads a buffer of footprint_bytes (1 MiB .. 64 GiB)
 * `passes` times (1 .. 1000) with 16-byte loads that bypass L1.  A footprint well
 * below the L2 size measures L2, one well above it HBM.  *gbs = bytes read / s / 1e9. */
dcopf_status dcopf_probe_read(int64_t footprint_bytes, int32_t passes, double* gbs);

/* Shared-memory read bandwidth over all SMs (conflict-free 16-byte loads). */
dcopf_status dcopf_probe_smem(double* gbs);

/* FMA throughput (*tflops, 2 flops per FMA, eight independent chains per thread on
 * every SM) and the latency of one dependent FMA (*chain_ns, one thread), in FP64
 * (fp64 != 0) or FP32. */
dcopf_status dcopf_probe_fma(int32_t fp64, double* tflops, double* chain_ns);

/* The tensor-core products' operand feed: one CTA per SM keeps a ring of three stages
 * of four 128 x 64 BF16 tiles (128-byte swizzle, as the products load them) filled by
 * TMA from a matrix of footprint_bytes (4 MiB .. 4 GiB) and releases each stage as it
 * lands.  *gbs = bytes landed in shared memory / s / 1e9. */
dcopf_status dcopf_probe_tma_feed(int64_t footprint_bytes, double* gbs);

/* One loop of the fused solve's exchange without its arithmetic: clusters of
 * `cluster` CTAs (2, 4 or 8) on a grid of `grid` CTAs (0 = the SM count rounded down
 * to a multiple of the cluster), n_gen generators split into cluster slices;
 * asynchronous stores into the peers' shared memory on transaction barriers, a
 * release-add arrival per CTA and acquire polling of every cluster's arrival, one
 * bulk copy of the slice's partials, and a second round of stores.  *us_per_loop =
 * the launch time of `loops` loops / loops.  Errors: INVALID_ARG (sizes),
 * UNSUPPORTED (shared memory), TIMEOUT, CUDA. */
dcopf_status dcopf_probe_exchange(int32_t cluster, int32_t grid, int32_t n_gen, int32_t loops,
                                  double* us_per_loop);

#ifdef __cplusplus
}
#endif

#endif /* DCOPF_PROBE_H */
