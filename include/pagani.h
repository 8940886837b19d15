/*
 * pagani.h - C ABI of the GB300 (sm_103a) PAGANI adaptive integrator.
 *
 * PAGANI (Sakiotis et al., "PAGANI: A Parallel Adaptive GPU Algorithm for
 * Numerical Integration", SC'21) integrates f over the unit hypercube [0,1]^n
 * by evaluating a degree-9 fully symmetric cubature rule and its null-rule
 * error estimate on every active sub-region at once, classifying regions as
 * active or finished, filtering the finished ones out with a prefix scan and
 * bisecting the survivors along an axis chosen by fourth divided
 * differences (Sec. 3, Algorithm 2; threshold search Sec. 3.5.3, Algorithm 3).
 *
 * Every step of that loop runs in this library's CUDA kernels on one GPU; the
 * loop itself stays on the device (a CUDA graph with conditional nodes).
 * All arithmetic is IEEE double precision.
 *
 * Conventions for every entry point:
 *  - Return value: a status code (>= 0 success or a non-converged but valid
 *    result, < 0 error; see PAGANI_STATUS_*).  No C++ exception crosses the
 *    ABI.  On error pagani_last_error() describes the failure.
 *  - Host pointers are read (or written) during the call only; the caller
 *    keeps ownership.  Device pointers must be CUDA device memory of the
 *    current device, sized as stated, and stay valid until the call returns.
 *  - cuda_stream: a cudaStream_t (NULL = a non-blocking stream the library
 *    owns).  The calls below synchronise that stream before they return.
 *  - Calls are serialised on an internal lock; the workspace is owned by the
 *    library and reused across calls.
 */
#ifndef PAGANI_GB300_H
#define PAGANI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Integrand families (the Genz families and the box-integral family of the
 * test integrands f1..f8, Sec. 4.1).  params layout (float64, n = dim):
 *   PRODUCT_PEAK  f = prod_j 1/(c_j^-2 + (x_j - w_j)^2)   params = c[n], w[n]
 *   GAUSSIAN      f = exp(-sum_j a_j^2 (x_j - w_j)^2)     params = a[n], w[n]
 *   OSCILLATORY   f = cos(2 pi u + sum_j a_j x_j)         params = u, a[n]
 *   CORNER_PEAK   f = (1 + sum_j a_j x_j)^-(n+1)          params = a[n]
 *   C0            f = exp(-sum_j a_j |x_j - w_j|)         params = a[n], w[n]
 *   DISCONTINUOUS f = exp(sum_j a_j x_j) if every x_j < w_j, else 0
 *                                                         params = a[n], w[n]
 *   BOX_POWER     f = (sum_j x_j^2)^q                     params = q (q >= 0)
 * Parameters must be finite; PRODUCT_PEAK needs c_j != 0.                     */
#define PAGANI_PRODUCT_PEAK 0
#define PAGANI_GAUSSIAN 1
#define PAGANI_OSCILLATORY 2
#define PAGANI_CORNER_PEAK 3
#define PAGANI_C0 4
#define PAGANI_DISCONTINUOUS 5
#define PAGANI_BOX_POWER 6

#define PAGANI_MIN_DIM 2
#define PAGANI_MAX_DIM 8

/* Status codes.  0..2 come with valid estimates (Algorithm 2 returns the
 * latest v + v_f, e + e_f in each case). */
#define PAGANI_STATUS_CONVERGED 0    /* (e+e_f)/|v+v_f| <= epsrel or e+e_f <= epsabs */
#define PAGANI_STATUS_IT_MAX 1       /* it_max iterations without convergence, or no
                                        region left to refine (rel-err filtering on a
                                        sign-changing integrand, Sec. 3.5.1): later
                                        iterations could not change the estimates */
#define PAGANI_STATUS_MEMORY 2       /* splitting the actives would exceed max_regions (Sec. 3.5.2) */
#define PAGANI_ERR_DIM (-1)          /* dim outside [PAGANI_MIN_DIM, PAGANI_MAX_DIM] */
#define PAGANI_ERR_INTEGRAND (-2)    /* unknown integrand_id or invalid params */
#define PAGANI_ERR_TOLERANCE (-3)    /* epsrel <= 0 / NaN, or epsabs < 0 / NaN */
#define PAGANI_ERR_CUDA (-4)         /* CUDA error or device allocation failure */
#define PAGANI_ERR_WATCHDOG (-5)     /* a device-side consistency check failed */
#define PAGANI_ERR_NONFINITE (-6)    /* the integrand produced NaN or Inf */
#define PAGANI_ERR_CAPACITY (-7)     /* max_regions below the initial uniform split */
#define PAGANI_ERR_ARGUMENT (-8)     /* other invalid argument (null pointer, size) */

typedef struct {
  double estimate;        /* v + v_f                                          */
  double errorest;        /* e + e_f                                          */
  int32_t status;         /* PAGANI_STATUS_* / PAGANI_ERR_*                   */
  int32_t iterations;     /* Evaluate passes performed                       */
  int64_t n_regions;      /* regions evaluated, summed over iterations       */
  int64_t n_active_last;  /* regions evaluated in the last iteration         */
  double finished_volume; /* volume of the regions classified finished       */
  double eval_ms;         /* host-driven loop only: summed device time of the Evaluate
                             launches, CUDA events on the launching stream; -1 otherwise */
  int32_t eval_launches;  /* Evaluate launches of this call                   */
  int32_t kernel_launches;/* kernels of this library launched by this call   */
  int64_t h2d_bytes;      /* host-to-device bytes copied by this call        */
  int64_t d2h_bytes;      /* device-to-host bytes copied by this call        */
  double active_volume;   /* volume of the regions of the last iteration; with
                             finished_volume it sums to the volume of the
                             integration region (dyadic boxes)              */
  int64_t n_leaves;       /* with keep_leaves: boxes of the converged leaf set
                             (see pagani_leaves); -1 otherwise             */
  double phase_ms[4];     /* host-driven loop only (use_graph = 0): summed device
                             time, CUDA events on the launching stream, of the
                             other phases of Algorithm 2 (the performance
                             breakdown of Sec. 4.2): [0] factor-cache fill,
                             [1] Threshold-Classify probes, [2] finished sums
                             and survivor count, [3] filter and split; -1
                             otherwise                                       */
} pagani_result;

typedef struct {
  int32_t relerr_filter;    /* 1 (default): Rel-Err-Classify on; 0 for sign-changing f (Sec. 3.5.1) */
  int32_t heuristic_filter; /* Threshold-Classify (Sec. 3.5.2-3.5.3) and its triggers: 1 (default)
                               both triggers, the estimate's digits unchanged and memory about to
                               be exhausted; 2 the memory trigger only; 3 the digits trigger only;
                               0 off (the filtering ablation of Sec. 4.2).  Other values:
                               PAGANI_ERR_ARGUMENT                                                */
  int32_t init_div;         /* divisions per axis of the Uniform-Split; 0 = largest power of two
                               d >= 2 with d^dim <= 4096 (Sec. 3.1)                                 */
  int32_t it_max;           /* iteration limit (default 100)                                       */
  int32_t use_graph;        /* 1 (default): device-resident loop in one CUDA graph; 0: host-driven */
  int32_t keep_leaves;      /* 1: keep the converged leaf set for pagani_leaves / differentiation;
                               0 (default); needs rule_degree 9                                   */
  int32_t rule_degree;      /* cubature rule: 9 (default; 0 means the same) the degree-9 rule with
                               four null rules (Sec. 2.1, 3.2); 7 the Genz-Malik degree-7 rule of
                               Cuhre, 2^dim + 2 dim^2 + 2 dim + 1 points, error |R7 - R5| with its
                               embedded degree-5 rule.  Other values: PAGANI_ERR_ARGUMENT          */
} pagani_options;

/* One record per iteration (Algorithm 2 scalars after that iteration). */
typedef struct {
  int32_t it, trigger, probes, search_ok;
  int64_t s, n_relerr_active, n_survivors;
  double v, e, vf, ef, threshold, direction_changes;
  int32_t probe_passes;   /* probe kernel launches of this iteration's threshold search */
  int32_t reserved;
} pagani_trace_record;

/* Fills *opt with the defaults listed above. */
void pagani_default_options(pagani_options* opt);

/* Integrate family `integrand_id` with parameters `params` (host array,
 * layout above) over [0,1]^dim to relative tolerance epsrel or absolute
 * tolerance epsabs (Algorithm 2, Sec. 3.1).  max_regions caps the regions
 * held in one iteration (memory requirement of Sec. 3.5.2).  Writes *out and
 * returns out->status.  Uses default options and the library's stream. */
int pagani_integrate(int dim, int integrand_id, const double* params, double epsrel, double epsabs,
                     int64_t max_regions, pagani_result* out);

/* As pagani_integrate with explicit options (NULL = defaults), a CUDA stream,
 * and an optional per-iteration trace: trace (host array of trace_cap
 * records, may be NULL) receives min(iterations, trace_cap) records. */
int pagani_integrate_ex(int dim, int integrand_id, const double* params, double epsrel, double epsabs,
                        int64_t max_regions, const pagani_options* opt, void* cuda_stream, pagani_result* out,
                        pagani_trace_record* trace, int trace_cap);

/* As pagani_integrate_ex over the box [lower, upper] (host arrays of dim
 * doubles; both NULL = the unit cube): Algorithm 2 takes the bounds a, b of
 * the integration region (Sec. 3.1) and starts with the Uniform-Split of
 * that box.  Regions are kept as dyadic sub-boxes of the unit cube and every
 * rule point x is evaluated at lower + (upper - lower) x, so a region's
 * volume is its unit-cube volume times prod (upper - lower); estimates,
 * errors, trace sums and the finished/active volumes are in that measure
 * (epsabs too).  Needs lower[j] < upper[j], both finite, and a finite
 * non-zero product of the lengths, else PAGANI_ERR_ARGUMENT.  The leaf set
 * kept with keep_leaves is in unit-cube coordinates of that map. */
int pagani_integrate_box(int dim, int integrand_id, const double* params, const double* lower,
                         const double* upper, double epsrel, double epsabs, int64_t max_regions,
                         const pagani_options* opt, void* cuda_stream, pagani_result* out,
                         pagani_trace_record* trace, int trace_cap);

/* Allocation-free integration, for callers that cannot allocate device
 * memory: applications whose own allocator owns all of the device memory (a
 * framework's caching allocator, a memory pool sized at start-up), and
 * service loops that must never pay for an allocation or risk an
 * out-of-memory failure mid-request.  The paper has no counterpart; it is a
 * deployment variant of pagani_integrate.
 *
 * Same arguments and result as pagani_integrate (default options; rel-err
 * filtering is off for the oscillatory family, on otherwise), plus a stream
 * (NULL = the legacy default stream).  Instead of the library workspace it
 * uses a 32 MiB array in the library's device memory, which every GPU that
 * loads the library holds until the process exits.  It runs the loop kernels
 * host-driven (no CUDA graph): after each step it copies the loop state to
 * the host and synchronises the stream.  It calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * max_regions is limited by the array: on a 152-SM GPU about 540,000
 * regions at dim 2, 420,000 at dim 3, 290,000 at dim 5 and 190,000 at dim 8;
 * larger values return PAGANI_ERR_CAPACITY with the limit in
 * pagani_last_error().  The first call on a device looks the array's
 * address up with that device current; make that first call before any
 * stream capture.  All calls share the array: calls whose GPU work overlaps
 * (other streams, other host threads with their own device contexts) race
 * on it.  Each call rewrites everything it reads, so the previous call's
 * contents do not leak into a result; a call that fails after its first
 * launch waits for its queued kernels before it returns.  The looked-up
 * address belongs to the device's context: after the application resets a
 * device (cudaDeviceReset), do not call this entry point on it again in the
 * same process.  Returns out->status. */
int pagani_integrate_noalloc(int dim, int integrand_id, const double* params, double epsrel, double epsabs,
                             int64_t max_regions, void* cuda_stream, pagani_result* out);

/* Batched integration: many independent integrals in one CUDA-graph
 * launch.  Not in the paper: a throughput form of Algorithm 2 for workloads
 * made of many small integrals.  Every item runs its own Algorithm 2/3 state
 * (same decisions as pagani_integrate) in a fixed region pool of
 * max_regions_per_item regions (its memory requirement, Sec. 3.5.2).  Items
 * are grouped by (integrand_id, dim); per iteration one Evaluate kernel runs
 * per group over all its items' regions, then one block per item reduces,
 * classifies, searches a threshold, compacts and splits.  Each group's
 * Evaluate grid is chosen by an autotuner on the first batch that contains
 * the group (timed on that batch's first iteration) and cached.
 * items: host array of count items; results: host array of count results (in
 * item order).  opt: NULL = defaults (heuristic_filter, it_max and
 * use_graph are used; rule_degree must be 9 or 0, the degree-9 rule).
 * device_ms (may be NULL) receives the device time of
 * the loop (CUDA events on the stream).  Returns 0 when the batch ran (each
 * item's status in its result), < 0 on an argument or CUDA error. */
typedef struct {
  int32_t dim;
  int32_t integrand_id;
  int32_t relerr_filter;  /* 1: Rel-Err-Classify on; 0 for sign-changing integrands */
  int32_t reserved;
  double epsrel, epsabs;
  double params[17];      /* family layout (see above) */
} pagani_batch_item;

typedef struct {
  double estimate, errorest;
  int32_t status, iterations;
  int64_t n_regions;
} pagani_batch_result;

int pagani_integrate_batch(int64_t count, const pagani_batch_item* items, int64_t max_regions_per_item,
                           const pagani_options* opt, void* cuda_stream, pagani_batch_result* results,
                           double* device_ms);

/* Allocates (or grows) the library workspace for up to max_regions regions
 * of dimension dim so that later calls do not allocate (the paper times
 * integration without workspace set-up, Sec. 4).  Returns 0 or < 0. */
int pagani_workspace_reserve(int64_t max_regions, int dim);

/* Frees the workspace and every cached CUDA graph.  Returns 0. */
int pagani_workspace_release(void);

/* Evaluate (Sec. 3.2) on a caller-given list of m boxes: lower and width are
 * DEVICE arrays in SoA layout [dim][m] (box i spans lower[j*m+i] ..
 * lower[j*m+i] + width[j*m+i] on axis j).  Writes, per box, the rule
 * estimate V[i], the null-rule error E[i] (before the two-level refinement)
 * and the split axis K[i] (fourth differences).  diag (device, may be NULL)
 * receives, SoA [(8 + dim)][m], the null-rule values N_1..N_4, their noise
 * floors (values at or below count as zero in the error formula) and the
 * fourth differences D_0..D_{dim-1}.  params is a host array.  Returns 0 or
 * < 0. */
int pagani_evaluate(int dim, int integrand_id, const double* params, int64_t m, const double* lower,
                    const double* width, double* V, double* E, int32_t* K, double* diag, void* cuda_stream);

/* As pagani_evaluate with the rule chosen by rule_degree (9 or 7, as in
 * pagani_options).  With 7, E is |R7 - R5| and diag row 0 holds that
 * difference (rows 1..3 and their floors are zero). */
int pagani_evaluate_ex(int dim, int integrand_id, const double* params, int rule_degree, int64_t m,
                       const double* lower, const double* width, double* V, double* E, int32_t* K, double* diag,
                       void* cuda_stream);

/* The converged leaf set of the last integration run with keep_leaves: the
 * boxes whose rule values make up the estimate v + v_f of Algorithm 2 (every
 * box classified finished, in the iteration it finished, and every box of
 * the last iteration).  Writes the count to *n_out; with lower and level
 * non-NULL also copies the boxes into those DEVICE arrays, SoA [dim][cap]
 * (box i: lower[j*cap+i] and width 2^-level[j*cap+i] on axis j; cap >=
 * count).  Returns 0, or < 0 if no leaf set was kept or dim differs. */
int pagani_leaves(int dim, int64_t cap, double* lower, uint8_t* level, int64_t* n_out, void* cuda_stream);

/* Differentiation of the rule estimate over a fixed box list (typically the
 * leaf set above): out[0] = sum over boxes of the basic-rule value V, and
 * out[1 + k] = its derivative with respect to params[k] (the family's own
 * parameter layout: out[1..dim] for the first vector, out[dim+1..2 dim] for
 * the second), i.e. sum vol sum_points w d f/d theta.  Defined for the
 * positive product families (PRODUCT_PEAK, GAUSSIAN, C0): f is a product of
 * per-axis factors, so d f/d theta_j = f d log phi_j / d theta_j.  lower
 * (f64) and level (u8) are DEVICE arrays SoA [dim][m]; params and out (2 dim
 * + 1 doubles) are host arrays.  The paper defines no derivative; this is
 * the backward pass of the converged integral with the region set frozen.
 * Returns 0 or < 0. */
int pagani_gradient(int dim, int integrand_id, const double* params, int64_t m, const double* lower,
                    const uint8_t* level, double* out, void* cuda_stream);

/* The rule tables this library generated for dimension dim (host outputs):
 * radius[5] = generator radii sqrt(l1), sqrt(l2), sqrt(l3), sqrt(lp), sqrt(l0);
 * weights[9*5] = per generator orbit (centre, l1, l2, l3, lp, l1l1, l1l2,
 * l1l1l1, l0^n) the basic rule and null rules 1..4 on the unit-volume cube;
 * counts[9] = orbit sizes.  Host computation only (no GPU needed).  Returns
 * the number of rule points N(dim), or < 0 on error. */
int pagani_rule_tables(int dim, double* radius, double* weights, int64_t* counts);

/* As pagani_rule_tables for rule_degree 9 or 7.  For 7 the Genz-Malik orbits
 * sit on the slots of the same structure (centre; one axis at sqrt(9/70) in
 * slot lp and at sqrt(9/10) in slot l2; pairs at sqrt(9/10) in slot l1l1;
 * every axis at sqrt(9/19) in slot l0^n), column 1 holds w7 - w5 and
 * columns 2..4 are zero. */
int pagani_rule_tables_ex(int dim, int rule_degree, double* radius, double* weights, int64_t* counts);

/* Measures this GPU's FP64 throughput with independent-chain
 * microbenchmarks (the roofline denominators of Evaluate).  Writes up to
 * n_out values to out: [0] FMA TFLOP/s (2 flops per FMA), [1] exp calls/s,
 * [2] sincos calls/s, [3] divisions/s (each in units of 1e9).  Returns 0 or
 * < 0. */
int pagani_fp64_peak(double* out, int n_out, void* cuda_stream);

/* Human-readable description of the last error on this thread. */
const char* pagani_last_error(void);

/* Library build identification. */
const char* pagani_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PAGANI_GB300_H */
