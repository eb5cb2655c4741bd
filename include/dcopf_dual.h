/*
 * dcopf_dual.h -- C ABI of the GB300 Lagrange-dual DCOPF library (libdcopfdual.so).
 *
 * The library computes lower bounds on the cost of DC optimal power flow by
 * projected gradient ascent on the Lagrange dual of
 *
 *     min  sum_j cost_j(p_j)
 *     s.t. 1^T p - 1^T p_d = 0                        : lambda   (power balance)
 *          f_min <= H_a (G p - p_d) <= f_max           : mu_lo, mu_hi >= 0
 *          p_min <= p <= p_max
 *
 * ("GPU-Accelerated DCOPF using Gradient-Based Optimization", arXiv 2406.13191,
 * Section 2 problem (1); PTDF H = Omega E (E^T Omega E)^{-1} with a zero slack
 * column; cost_j(p) = a_j (S p)^2 + b_j S p, a_j = 0 for linear costs, S = base MVA).
 * The dual function g(lambda, mu) = inf_p L(p, lambda, mu) (Section 3, eqs. (3)-(5))
 * is evaluated in closed form: the inner minimiser is the box-clipped dispatch
 * (eq. (6) via the dual norm for linear costs, eq. (16) for quadratic costs).
 * Any lambda and any mu >= 0 give a valid lower bound (Remarks 1 and 2).
 *
 * Conventions shared by every entry point:
 *  - Powers are in p.u. on base_mva; costs in $/h; multipliers in $/h per p.u.
 *  - Batched arrays are row-major [batch][n]: instance b's row starts at b*n.
 *  - Unless stated otherwise, array arguments of eval / solve_batch /
 *    certify_bound are caller-owned DEVICE pointers on the handle's device; the
 *    library never frees them.  They must not alias one another.
 *  - All device work is enqueued on the caller's stream `stream` (a cudaStream_t
 *    passed as void*; NULL = legacy default stream) and is asynchronous unless the
 *    entry point says it synchronises.  Host-side validation errors return before
 *    anything is enqueued.
 *  - No C++ exception crosses this ABI.  Every entry point returns a dcopf_status.
 *  - A handle may be used from one host thread at a time.
 */
#ifndef DCOPF_DUAL_H
#define DCOPF_DUAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dcopf_dual* dcopf_dual_t; /* opaque; owned by the library */

typedef enum {
  DCOPF_OK = 0,
  DCOPF_ERR_INVALID_ARG = 1, /* null pointer, size out of range, bad enum value, NaN */
  DCOPF_ERR_NETWORK = 2,     /* islanded network, b <= 0, pmin > pmax, bridge outage */
  DCOPF_ERR_CUDA = 3,        /* a CUDA runtime/driver call failed */
  DCOPF_ERR_OOM = 4,         /* device allocation failed */
  DCOPF_ERR_TIMEOUT = 5,     /* a bounded device wait (grid barrier, mbarrier) gave up */
  DCOPF_ERR_UNSUPPORTED = 6  /* size or option combination this build does not handle */
} dcopf_status;

/* Arithmetic of the operator products (adjoint Phi^T eta, forward Phi x).
 * The dual value is always accumulated in FP64. */
typedef enum {
  DCOPF_FP64 = 0,  /* FP64 products on CUDA cores */
  DCOPF_FP32 = 1,  /* FP32 products with FP32 accumulation on CUDA cores */
  DCOPF_BF16X3 = 2 /* BF16 hi/lo split products on tcgen05 tensor cores, FP32 accumulation */
} dcopf_precision;

/* Ascent rule (Section 3.3). */
typedef enum {
  DCOPF_GDM = 0,    /* Algorithm 1 read as heavy-ball momentum */
  DCOPF_ADAM = 1,   /* Adam, bias-corrected moments */
  DCOPF_ADAGRAD = 2 /* AdaGrad */
} dcopf_rule;

/* Execution path of dcopf_dual_solve_batch. */
typedef enum {
  DCOPF_PATH_AUTO = 0,   /* fused persistent kernel for batch 1, batched kernels otherwise;
                            a single instance whose fused kernel cannot run (no cluster
                            shape fits, or every shape is refused) runs on the unfused
                            FP32 kernels instead */
  DCOPF_PATH_PLAIN = 1,  /* one launch per phase per iteration (the unfused baseline) */
  DCOPF_PATH_FUSED = 2,  /* one persistent thread-block-cluster kernel per instance; it
                            is launched cooperatively when the driver accepts that,
                            unless the environment sets DCOPF_FUSED_COOPERATIVE=0
                            (read by dcopf_dual_create).  The kernel refuses a launch
                            whose cluster shape is not the one its shared-memory layout
                            was sized for (profilers that replay cooperative launches
                            drop the shape); such a launch is repeated as a plain
                            cluster launch.  Test hook: DCOPF_FUSED_REFUSE=1 (or 2),
                            read by dcopf_dual_create, makes the host size every
                            cooperative (or every) fused launch for another shape, so
                            that the kernel refuses it */
  DCOPF_PATH_BATCHED = 3, /* batched contraction kernels replayed from a CUDA graph */
  DCOPF_PATH_SPARSE = 4   /* one CTA per instance runs the iterations with both operator
                             products as level-scheduled triangular solves on the sparse
                             LDL^T factor of the reduced Laplacian (no PTDF); FP64; the
                             iterates equal the plain path's up to rounding */
} dcopf_path;

/* Network description (Section 2, problem (1)).  Host pointers, copied by
 * dcopf_dual_create; the caller may free them afterwards. */
typedef struct {
  int32_t n_bus, n_line, n_gen;
  int32_t slack_bus;          /* 0-based; the zero column of H_a */
  const int32_t* line_from;   /* [n_line] 0-based bus index */
  const int32_t* line_to;     /* [n_line] */
  const double* line_b;       /* [n_line] susceptance, p.u., > 0 */
  const double* flow_max;     /* [n_line] upper flow limit, p.u. */
  const double* flow_min;     /* [n_line] lower flow limit; NULL => -flow_max */
  const int32_t* gen_bus;     /* [n_gen] 0-based bus of each generator */
  const double* pmin;         /* [n_gen] p.u. */
  const double* pmax;         /* [n_gen] p.u., >= pmin */
  const double* cost_lin;     /* [n_gen] b_j, $/MWh */
  const double* cost_quad;    /* [n_gen] a_j >= 0, $/MW^2h; NULL => linear costs */
  double base_mva;            /* S, MVA (> 0) */
} dcopf_network_desc;

typedef struct {
  int32_t device;    /* CUDA device ordinal; -1 = current device */
  int32_t max_batch; /* largest batch the handle will see (workspaces sized lazily anyway) */
  int32_t verbose;   /* 1 = print setup statistics to stderr */
  int32_t operator_form; /* 0 = the PTDF Phi~ and the sparse factor (every call);
                            1 = the sparse factor only: no Phi~ is built or stored (for
                            networks whose n_line x n_gen PTDF does not fit); then only
                            DCOPF_PATH_SPARSE (and PATH_AUTO, which picks it) and
                            dcopf_dual_certify_bound run, the rest return UNSUPPORTED */
} dcopf_options;

/* Parameters of dcopf_dual_solve_batch.  Zero-initialise and set what you need;
 * dcopf_solve_params_default fills the documented defaults. */
typedef struct {
  int32_t rule;        /* dcopf_rule */
  int32_t precision;   /* dcopf_precision of the in-loop operator products */
  int32_t path;        /* dcopf_path */
  int32_t max_iters;   /* iteration cap per instance (> 0) */
  int32_t warm_start;  /* 1 = start from lambda/mu given in the in/out arrays */
  int32_t as_printed;  /* 1 = GDM applies Algorithm 1's printed extra gradient update */
  int32_t check_every; /* certify a candidate at most every k iterations (>= 1) */
  int32_t screen_lines; /* 1 = constraint screening on the batched tensor-core path
                           (DCOPF_BF16X3, batches without outages): lines whose flow
                           provably stays inside its limits for every dispatch of the
                           generator box that meets the balance, at every instance's
                           loads, are left out of the iterations (their multipliers stay
                           0, so every point is still a valid bound, Remarks 1 and 2;
                           the certificate evaluates the full problem); 0 = every line
                           (Algorithm 1's C_r, d_r read as all flow rows) */
  double alpha;        /* step size for mu (and lambda unless alpha_lambda > 0) */
  double alpha_lambda; /* step size for lambda; <= 0 => alpha */
  double rho;          /* GDM momentum */
  double beta1, beta2; /* Adam moments */
  double eps;          /* Adam / AdaGrad denominator guard */
  double decay;        /* step size multiplied by decay every iteration (1 = none) */
  double gap;          /* stop when certified bound >= target - gap*|target| */
  double tol;          /* > 0: also stop when |g_k - g_{k-1}| < tol (Algorithm 1 stop test) */
  const double* target_value; /* DEVICE [batch] optimal costs to stop at; NULL => run max_iters
                                 or until the tol test */
  double* mean_dispatch;      /* DEVICE [batch][n_gen] or NULL: receives the mean of the
                                 minimisers p*(lambda_k, mu_k) of the solve's evaluations,
                                 the k-th weighted by k^2 (p.u.); a candidate for
                                 dcopf_dual_primal_bound (averages of a dual method's
                                 minimisers approach the primal optimum) */
  int32_t qp_dual_s;  /* 1 = quadratic costs: ascend on eq. (16)'s dual g_q(lambda, mu, s)
                         with s (one per generator, free, starting at 0, mu's step size)
                         as a third ascent variable (Section 3.2, Remark 2) instead of
                         the closed form max_s g_q; the in-loop value is g_q, the
                         certificate still evaluates (lambda, mu) in closed form, which
                         bounds at least as tightly.  DCOPF_PATH_PLAIN only, else
                         DCOPF_ERR_UNSUPPORTED; 0 = the closed form */
  int32_t reserved;
} dcopf_solve_params;

/* Library version string. */
const char* dcopf_version(void);

/* Human-readable text of a status code (static storage). */
const char* dcopf_status_string(dcopf_status s);

/* Fills p with the defaults: ADAM, FP32, PATH_AUTO, max_iters 5000, alpha 1000,
 * rho 0.9, beta1 0.9, beta2 0.999, eps 1e-8, decay 1, gap 1e-3, check_every 1. */
void dcopf_solve_params_default(dcopf_solve_params* p);

/* Validates the network, factorises the reduced Laplacian E^T Omega E (FP64 sparse
 * LDL^T, minimum-degree order, slack removed), builds Phi = H_a G (the PTDF at the
 * generator buses, Section 2 below problem (1)) in FP64, normalises generator
 * outputs to the unit box (Appendix A1), uploads everything to the device and
 * returns a handle in *out.  Synchronises the device.  Errors: INVALID_ARG (null
 * pointers, sizes < 1, NaN/Inf, bad slack index), NETWORK (islanded network, b <= 0,
 * pmin > pmax, flow_min > flow_max), UNSUPPORTED (no lines: a single bus, whose dual
 * has lambda alone and is solved by merit order; or sizes beyond the limits), OOM,
 * CUDA. */
dcopf_status dcopf_dual_create(const dcopf_network_desc* net, const dcopf_options* opt,
                               dcopf_dual_t* out);

/* Frees the handle and all device memory it owns.  NULL is accepted. */
dcopf_status dcopf_dual_destroy(dcopf_dual_t h);

/* Network sizes and flags of a handle (host pointers; NULL outputs are skipped).
 * bridge_mask: host array [n_line] receiving 1 for lines whose outage islands the
 * network (such outages are rejected by every entry point). */
dcopf_status dcopf_dual_info(dcopf_dual_t h, int32_t* n_bus, int32_t* n_line, int32_t* n_gen,
                             int32_t* is_qp, uint8_t* bridge_mask);

/* One evaluation of the dual function and its supergradient at given multipliers
 * (Section 3.1 eq. (6) / Section 3.2 eq. (16) in closed form; gradient as in
 * Algorithm 1's gradient lines, read as the primal residuals).
 *   loads    [batch][n_bus]  p_d of each instance
 *   outage   [batch] or NULL line index removed from instance b (-1 = none); the
 *            outaged line's multipliers are ignored and its gradient is 0
 *   lambda   [batch]; mu_hi, mu_lo [batch][n_line], used as given (negative mu are
 *            allowed: the dual function is defined for them, they just do not bound)
 *   precision dcopf_precision of the operator products
 * Outputs (NULL = skip, except value):
 *   value    [batch]  g(lambda, mu) = sum_j cost_j(p*) + lambda (1^T p* - 1^T p_d)
 *                     + mu_hi^T (f - f_max) + mu_lo^T (f_min - f), FP64 accumulation
 *   g_lambda [batch]  1^T p* - 1^T p_d
 *   g_mu_hi, g_mu_lo [batch][n_line]  f - f_max, f_min - f
 *   dispatch [batch][n_gen]  the minimiser p* (ties take the box midpoint)
 * Errors: INVALID_ARG, NETWORK (bridge outage), UNSUPPORTED, OOM, CUDA. */
dcopf_status dcopf_dual_eval(dcopf_dual_t h, int32_t batch, const double* loads,
                             const int32_t* outage, const double* lambda, const double* mu_hi,
                             const double* mu_lo, int32_t precision, double* value,
                             double* g_lambda, double* g_mu_hi, double* g_mu_lo,
                             double* dispatch, void* stream);

/* Certified FP64 lower bound at given multipliers (Remarks 1 and 2): mu is first
 * projected to mu >= 0, the bus prices nu = lambda + H_a^T (mu_hi - mu_lo) are
 * computed in FP64 by sparse triangular solves, and
 *   bound = sum_j min_p [cost_j(p) + nu_bus(j) p] - nu^T p_d - mu_hi^T f_max + mu_lo^T f_min
 * is accumulated in FP64 (eq. (4) evaluated through the bus prices).  err_bound
 * receives an upper bound on the total rounding error of that evaluation: of the
 * final accumulation and each term, and of the computed bus prices nu (the residual
 * of the sparse triangular solves, or the accumulation in the dense H_a^T products,
 * times how much each term can move with its price).  The reported bound already
 * has it subtracted.
 *   loads [batch][n_bus]; outage [batch] or NULL; lambda [batch]; mu_hi, mu_lo
 *   [batch][n_line]; bound [batch] (required); err_bound [batch] (NULL = skip). */
dcopf_status dcopf_dual_certify_bound(dcopf_dual_t h, int32_t batch, const double* loads,
                                      const int32_t* outage, const double* lambda,
                                      const double* mu_hi, const double* mu_lo, double* bound,
                                      double* err_bound, void* stream);

/* Upper bound from a dual point (primal recovery).  The paper builds no primal point;
 * by its Remarks 1 and 2 no feasible dispatch costs less than any dual value, so the
 * cost of the dispatch returned here, with dcopf_dual_certify_bound's lower bound,
 * brackets gamma* without a stored optimum.  Steps, in FP64, per instance:
 *   1. the closed-form minimiser (eq. (6) / eq. (16)) at the bus prices of
 *      (lambda, mu) plus a uniform price shift, the shift found by bisection until
 *      two adjacent shifts bracket the demand; the convex combination of those two
 *      dispatches that meets the demand exactly (box and balance hold);
 *   2. the smallest move t in [0, 1] towards the reference dispatch that brings
 *      every flow within its limits (the feasible set is convex);
 *   3. the flows of the result recomputed, and its cost.
 *   loads [batch][n_bus]; outage [batch] or NULL (as in dcopf_dual_eval); lambda
 *   [batch]; mu_hi, mu_lo [batch][n_line], used as given (NULL allowed with p_cand).
 *   p_cand [batch][n_gen] or NULL: a candidate dispatch (p.u.; e.g. the solve's
 *            mean_dispatch) that replaces step 1: clipped to the box, then moved
 *            towards pmax (total below the demand) or pmin (above) until it meets
 *            the demand
 *   p_ref [batch][n_gen] or NULL: a dispatch in p.u. that meets the box, the balance
 *            (to 1e-9 max(1, demand)) and every flow limit (to 1e-9 p.u.), e.g. the
 *            current operating point; NULL = the proportional dispatch
 *            pmin + theta (pmax - pmin) with sum = demand
 * Outputs:
 *   upper    [batch] (required)  the cost ($/h) of the recovered dispatch; +inf
 *            where there is no bound
 *   pstatus  [batch] or NULL     0 bound; 1 the demand lies outside
 *            [sum pmin, sum pmax]; 2 the reference breaks the box, the balance or a
 *            flow limit
 *   dispatch [batch][n_gen] or NULL  the recovered dispatch (p.u.; NaN where there
 *            is no bound)
 *   max_violation [batch] or NULL  the largest flow-limit violation of that dispatch
 *            with its flows recomputed (rounding only; NaN where there is no bound)
 * Errors: INVALID_ARG, NETWORK (bridge outage), UNSUPPORTED, OOM, CUDA. */
dcopf_status dcopf_dual_primal_bound(dcopf_dual_t h, int32_t batch, const double* loads,
                                     const int32_t* outage, const double* lambda,
                                     const double* mu_hi, const double* mu_lo,
                                     const double* p_cand, const double* p_ref, double* upper,
                                     int32_t* pstatus, double* dispatch, double* max_violation,
                                     void* stream);

/* Projected gradient ascent on the dual for a batch of instances of one network
 * (Section 3.3, Algorithm 1 and the Adam / AdaGrad rules), from the cold start
 * lambda = mu = 0 (Algorithm 1, Require) or from the given warm start.
 *   loads [batch][n_bus]; outage [batch] or NULL
 *   lambda [batch], mu_hi, mu_lo [batch][n_line]: in = warm start (if
 *     params->warm_start), out = the best iterate found (largest certified bound)
 *   best_bound [batch]: certified FP64 bound at that iterate (dcopf_dual_certify_bound)
 *   iters [batch]: iterations taken; inst_status [batch]: 0 = reached target,
 *     1 = stopped at max_iters or by the tol test, 2 = dual unbounded (infeasible
 *     primal suspected: the bound exceeded the cost of any dispatch)
 * Stopping: when target_value is given, an instance stops once its certified bound
 * is >= target - gap*|target|; candidates are certified when the in-loop value
 * (reduced precision) first reaches the target.  All output arrays are device
 * pointers.  The call enqueues its work on `stream` and synchronises that stream
 * before returning (the iteration count is data dependent).
 * Errors: INVALID_ARG, NETWORK, UNSUPPORTED, OOM, CUDA, TIMEOUT. */
dcopf_status dcopf_dual_solve_batch(dcopf_dual_t h, int32_t batch, const double* loads,
                                    const int32_t* outage, const dcopf_solve_params* params,
                                    double* lambda, double* mu_hi, double* mu_lo,
                                    double* best_bound, int32_t* iters, int32_t* inst_status,
                                    void* stream);

/* One network's instances in a group solve (dcopf_dual_solve_group).  Arrays as in
 * dcopf_dual_solve_batch, for this item's handle; target_value [batch] (DEVICE,
 * nullable) plays the role of params->target_value for these instances; params
 * (HOST, nullable) overrides the group's ascent settings for this network (its
 * check_every and target_value are ignored). */
typedef struct {
  dcopf_dual_t net;
  int32_t batch;
  int32_t reserved;
  const dcopf_solve_params* params;
  const double* loads;
  const int32_t* outage;
  const double* target_value;
  double* lambda;
  double* mu_hi;
  double* mu_lo;
  double* best_bound;
  int32_t* iters;
  int32_t* inst_status;
} dcopf_group_item;

/* Batched solves of several networks of different sizes in one go: the same method
 * and results as dcopf_dual_solve_batch on each item (Section 3.3, Algorithm 1 and
 * Adam / AdaGrad), with the iterations of every network issued together.  Each round
 * of check_every (at least 16) iterations is ONE launch of a CUDA graph that holds
 * every network's iteration kernels as parallel branches; the FP64 certification of
 * the round's candidates follows per network.  The paper solves one instance at a
 * time; this is the batching it leaves to future work.
 *   n_items >= 1 items with pairwise distinct handles, all created on one device
 *   params: shared ascent settings (items may override them); precision must be
 *     DCOPF_BF16X3 and path DCOPF_PATH_AUTO or DCOPF_PATH_BATCHED in every set used
 *     (else DCOPF_ERR_UNSUPPORTED); params->target_value is ignored (each item has
 *     its own); the round length is the shared check_every
 * Synchronises `stream` before returning.
 * Errors: INVALID_ARG (a NULL or repeated handle, handles on different devices, bad
 * sizes or parameters), NETWORK, UNSUPPORTED, OOM, CUDA, TIMEOUT. */
dcopf_status dcopf_dual_solve_group(int32_t n_items, const dcopf_group_item* items,
                                    const dcopf_solve_params* params, void* stream);

/* dcopf_dual_eval without any device allocation, for callers that cannot allocate
 * device memory (a host framework that owns every allocation, or a real-time loop
 * where cudaMalloc's implicit synchronisation and latency are not acceptable).  The
 * paper has no counterpart: this is an interface convenience.
 *
 * Same arguments, host checks, results and errors as dcopf_dual_eval, for precision
 * DCOPF_FP64 or DCOPF_FP32 (DCOPF_BF16X3 returns DCOPF_ERR_UNSUPPORTED: its BF16
 * operands live in the handle's workspace).  Instead of the handle's
 * workspace, every intermediate array lives in one fixed device array of 16 MiB
 * compiled into the library (each GPU that loads the library holds it until the
 * process exits).  A call needs 256-byte-aligned sections of about
 * batch * (8 * (4 * n_line + 2 * n_gen) + 24) bytes for FP64 (less for FP32); a batch
 * that does not fit returns DCOPF_ERR_INVALID_ARG before anything is enqueued.
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, which may also load the library's device code); make that
 * first call before any stream capture.  All calls on a device share the one array
 * and it keeps the last call's contents, which every call fully overwrites before
 * reading: calls whose device work overlaps (different streams, or different host
 * threads) race on it and must be serialised by the caller.  Outage indices are
 * copied back and checked on the host, which synchronises `stream`. */
dcopf_status dcopf_dual_eval_noalloc(dcopf_dual_t h, int32_t batch, const double* loads,
                                     const int32_t* outage, const double* lambda,
                                     const double* mu_hi, const double* mu_lo, int32_t precision,
                                     double* value, double* g_lambda, double* g_mu_hi,
                                     double* g_mu_lo, double* dispatch, void* stream);

/* Number of kernels this handle has launched since creation (for launch accounting). */
int64_t dcopf_dual_kernel_launches(dcopf_dual_t h);

/* Timing of the iteration kernels of dcopf_dual_solve_batch (the fused persistent
 * kernel, or the per-iteration kernels of the plain and batched paths), measured
 * with CUDA events recorded on the caller's stream around each launch group.
 * enable != 0 switches it on (off by default; it adds no synchronisation). */
dcopf_status dcopf_dual_set_timing(dcopf_dual_t h, int32_t enable);

/* Reads and resets the accumulated timing: total milliseconds of the iteration
 * kernels, the number of iteration-kernel launches, and the dual evaluations they
 * performed summed over instances.  Host pointers; NULL outputs are skipped. */
dcopf_status dcopf_dual_read_timing(dcopf_dual_t h, double* iter_ms, int64_t* iter_launches,
                                    int64_t* evaluations);

/* The lines the last screened solve (screen_lines = 1) iterated on: *n_kept (host,
 * nullable) their number, kept_mask (host [n_line], nullable) 1 for each of them.  The
 * kept set is a multiple of 8 lines: besides every line that may bind it holds the
 * first lines that cannot, up to that multiple.  0 kept lines: no screen yet. */
dcopf_status dcopf_dual_screened_lines(dcopf_dual_t h, int32_t* n_kept, uint8_t* kept_mask);

/* Per-kernel timing of the batched tensor-core solve, while dcopf_dual_set_timing is
 * on: CUDA events recorded inside the iteration graph around the kernels of the last
 * iteration of every round of the first instance group (the adjoint product, the
 * minimiser, the forward product, the step, and a fifth slot for the dual value and
 * stop tests, which run beside the next iteration's minimiser, so that it reads only
 * the events' own cost, about 2 us).  A round in which every instance was frozen
 * launches no graph and adds no sample.  ms (host
 * [5], nullable) receives the summed milliseconds of each over the sampled iterations,
 * samples (host, nullable) their count; both are then reset.  Host only. */
dcopf_status dcopf_dual_read_kernel_timing(dcopf_dual_t h, double* ms, int64_t* samples);

/* The shapes the batched tensor-core solve chose for its last batch (by timing on the
 * first solve of a batch size, or as DCOPF_TENSOR_SHAPE fixed them), into shapes (host
 * [7]): the batch, the lines iterated on, the adjoint product's tiles (0 single CTAs of
 * 128 x 128; CTA pairs of 1: 256 x 256, 2: 256 x 192, 3: 256 x 160, 4: 256 x 144;
 * 5 .. 8: the widths of 1 .. 4 in clusters of two pairs that load each box of the batch
 * operand once for both), its split-K factor, the forward product's tiles (same codes),
 * the number of instance groups iterated as
 * parallel branches of the iteration graph (1 or 2; the tiles are those of one group's
 * share of the batch), and the first group's instances (its kernels are the ones that
 * dcopf_dual_read_kernel_timing times).  All zero before the first batched solve.
 * Host only. */
dcopf_status dcopf_dual_tensor_shapes(dcopf_dual_t h, int32_t* shapes);

/* Device-memory budget of a handle's workspaces: the buffers that eval,
 * certify_bound, primal_bound, solve_batch and the self-tests allocate on first use
 * or when a larger batch arrives (the network data uploaded by dcopf_dual_create and
 * the buffers of dcopf_dual_solve_group are not counted).  limit_bytes > 0 sets the
 * largest number of bytes they may hold together, 0 removes the limit, < 0 leaves it
 * unchanged.  A call that would need a workspace beyond the limit returns
 * DCOPF_ERR_OOM before it enqueues any work and leaves the handle usable: later calls
 * whose workspaces fit run normally.  used_bytes (host, nullable) receives the bytes
 * the workspaces hold now.  Host only; does not synchronise. */
dcopf_status dcopf_dual_workspace_limit(dcopf_dual_t h, int64_t limit_bytes, int64_t* used_bytes);

/* Self-test of the bounded device wait used by every cross-CTA synchronisation of
 * the persistent kernels: one thread waits, with an acquire load in a loop, for a
 * device counter that nothing increments, and must give up after timeout_ns
 * (1 us .. 10 s) of wall-clock time.  Returns DCOPF_ERR_TIMEOUT when the wait gave up
 * (the expected outcome), DCOPF_OK if it did not.  The device stays usable
 * either way.  Synchronises `stream`. */
dcopf_status dcopf_selftest_bounded_wait(dcopf_dual_t h, int64_t timeout_ns, void* stream);

/* Self-test of the fused persistent kernel's failure path: one fused solve of the
 * instance `loads` (DEVICE [n_bus]) in which the wait for every cluster's arrival
 * expects one arrival more than the clusters make, with the kernel's waits limited to
 * timeout_ns (1 us .. 10 s).  Every cluster gives up at the first loop, the CTAs of
 * each cluster leave together through the kernel's final cluster barrier, and the
 * solve returns DCOPF_ERR_TIMEOUT (the expected outcome; DCOPF_OK would mean the
 * wait did not give up).  The handle stays usable.  Needs a handle whose fused shape
 * is already chosen (after one fused solve), else DCOPF_ERR_UNSUPPORTED.
 * Synchronises `stream`. */
dcopf_status dcopf_selftest_fused_timeout(dcopf_dual_t h, const double* loads, int64_t timeout_ns,
                                          void* stream);

/* Sticky device-side error word of the handle's last solve (0 = none, else a
 * dcopf_status value such as DCOPF_ERR_TIMEOUT).  Synchronises the device. */
dcopf_status dcopf_dual_device_error(dcopf_dual_t h);

#ifdef __cplusplus
}
#endif

#endif /* DCOPF_DUAL_H */
