/*
 * gbselect — exact order statistics of large real vectors on one GB300 (sm_103a).
 *
 * Method: G. Beliakov, "Parallel calculation of the median and order statistics on
 * GPUs with application to robust regression", arXiv:1104.2732.  The k-th order
 * statistic x_(k) is the minimiser of the convex piecewise-linear cost of
 * Eq. (med_objOS); Kelley's cutting plane (Algorithm 1, Sec. 3) minimises it, one
 * fused pass over x per iterate computing #(x<t), #(x<=t) and the cost; the final
 * bracket is compacted and the answer selected inside it (Sec. 3, hybrid finish).
 *
 * Conventions for every entry point:
 *  - Array pointers are DEVICE pointers owned by the caller; inputs are never
 *    written.  Outputs are device pointers, written asynchronously on `stream`.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *  - k is 1-based (Sec. 1).  The median is x_(k) with k = floor((n+1)/2) (Sec. 1).
 *  - Results are elements of x, bit for bit: ties, -0/+0 and +-inf are ordered by
 *    IEEE-754 totalOrder (-inf < ... < -0 < +0 < ... < +inf).
 *  - Argument errors are detected on the host before any launch and return
 *    GBS_EINVAL (nothing is launched).  Data-dependent errors (NaN in the input,
 *    an internal wait that gave up) are recorded on the device; gbs_last_stats()
 *    synchronises the stream of the last call and returns them.  On GBS_ENAN the
 *    output holds a quiet NaN.
 *  - A context owns a device workspace.  Calls on one context must not overlap in
 *    time (issue them on one stream, or use one context per stream).  A call that
 *    needs more workspace than reserved allocates it (synchronously); call
 *    gbs_reserve() first to keep later calls allocation-free.
 *  - No exception crosses this interface.
 */
#ifndef GBSELECT_H
#define GBSELECT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBS_OK = 0,
    GBS_EINVAL = 1,   /* bad argument (n < 1, k outside [1,n], NULL pointer, ...) */
    GBS_ENAN = 2,     /* the input holds a NaN: it has no rank */
    GBS_ENOMEM = 3,   /* workspace allocation failed */
    GBS_ECUDA = 4,    /* a CUDA runtime call failed */
    GBS_ETIMEOUT = 5, /* a bounded device-side wait gave up; the result is not valid */
    GBS_EINTERNAL = 6 /* an internal consistency check failed; the result is not valid */
} gbs_status;

typedef struct gbs_ctx gbs_ctx;

/* How a selection ended (gbs_run_stats.how). */
enum {
    GBS_HOW_NONE = 0,
    GBS_HOW_NEGINF = 1, /* k <= #(x = -inf) */
    GBS_HOW_POSINF = 2, /* k > n - #(x = +inf) */
    GBS_HOW_MIN = 3,    /* x_(k) is the finite minimum (Sec. 3, step 0 extremes) */
    GBS_HOW_MAX = 4,    /* x_(k) is the finite maximum */
    GBS_HOW_HIT = 5,    /* an iterate t had 0 in dF(t) (Algorithm 1, step 1.3) */
    GBS_HOW_FINISH = 6  /* compaction of the bracket and radix select (Sec. 3, hybrid) */
};

/* Tuning knobs.  Zero fields take the defaults given beside them. */
typedef struct {
    int64_t cap;         /* the pass that sees a bracket of <= cap elements compacts it and
                            the cutting plane stops (Sec. 3 ends the iterations once one more
                            would cost more than it saves the finish); 0 = max(n/4, 4096) for
                            float32, max(n/8, 4096) for float64 */
    int32_t maxit;       /* cutting-plane iterations before compaction is forced; 0 = 64 */
    int32_t blocks_per_sm; /* CTAs per SM of the persistent kernel; 0 = 1 below 32 MiB of
                              input, else 2 (at most what fits) */
    int32_t use_learned; /* 1 = start from the bracket proposed by the loaded model (if any);
                            a proposed bracket that passes its count check and holds at most
                            max(cap, n/8) elements goes straight to the finish */
    int32_t lms_start;   /* fused LMS/LTS objectives (n >= 65536): 0 = each candidate starts from
                            a bracket proposed by order statistics of its squared residuals on
                            8192 sampled rows and checked by counts in the first pass (a
                            candidate whose check fails goes to the materialising form);
                            1 = start from the extremes (Algorithm 1, step 0) */
    int32_t knn_start;   /* kNN (n >= 65536): 0 = each query starts from a bracket of sampled
                            distance order statistics, checked by counts in one fused pass (a
                            query whose check fails takes the plain form); 1 = the plain form
                            for every query: its distance row written out, d_(k) by the
                            segmented select, then the indicator reduction */
    int32_t reserved[5];
} gbs_config;

/* Per-call record of the last selection on a context (host copy). */
typedef struct {
    int32_t status;        /* gbs_status of the device work */
    int32_t how;           /* GBS_HOW_* */
    int32_t passes;        /* full passes over x, the min/max/count pass included */
    int32_t kelley_steps;  /* iterates from the tangent intersection (Algorithm 1, step 1.1) */
    int32_t bisect_steps;  /* safeguard iterates (bracket midpoint in totalOrder keys) */
    int32_t finish_rounds; /* 12-bit radix rounds of the finish */
    int32_t grid;          /* CTAs of the persistent launch */
    int32_t learned;       /* 1 if a proposed bracket was used, 2 if it failed its count check */
    int64_t n, k;
    int64_t finish_pop;    /* elements compacted for the finish */
    int64_t pops[64];      /* bracket population after each iterate */
    double iterates[64];   /* the evaluated points t */
    uint64_t t_ns[72];     /* device timestamps (globaltimer, ns) at each grid-wide step */
    uint64_t t_stream_ns[64]; /* CTA 0: end of the streaming part of each cutting-plane pass */
    int32_t n_t;           /* valid entries of t_ns */
    int32_t pad;
} gbs_run_stats;

/* Pass 0 of Algorithm 1 (Sec. 3, step 0): extremes and sums over x. */
typedef struct {
    int64_t n;
    int64_t n_nan, n_neginf, n_posinf, n_negzero, n_finite;
    double min, max;        /* finite minimum / maximum (0 if no finite element); a zero
                               extreme is reported as +0, see n_negzero */
    int64_t c_le_min;       /* #(x <= min) under IEEE comparison (infinities included) */
    int64_t c_lt_max;       /* #(x <  max) */
    double sum;             /* sum of the finite elements (float32 partials, float64 total) */
} gbs_array_stats;

/* One fused cost + count pass (Algorithm 1, step 1.2; the figure's Objective()). */
typedef struct {
    int64_t c_lt_t;   /* #(x <  t) */
    int64_t c_le_t;   /* #(x <= t) */
    int64_t c_le_a;   /* #(x <= a) */
    int64_t pad;
    double S;         /* sum over a < x_i < t of (t - x_i) */
    double dphi;      /* Phi(t) - Phi(a) = (c_le_a - k + 1/2)(t - a) + S, Phi = F/n of Eq. (med_objOS) */
} gbs_cost_eval;

/* State of a sharded selection (see gbs_shard_begin).  Plain data: it may be copied,
 * broadcast between processes or inspected; only the functions below change it. */
enum {
    GBS_SHARD_ITERATE = 0, /* evaluate t on every shard (gbs_cost_pass_*), then gbs_shard_update */
    GBS_SHARD_DONE = 1,    /* result holds x_(k) */
    GBS_SHARD_COMPACT = 2, /* compact (a, b] on every shard; x_(k) is the (k - cle_a)-th of them */
    GBS_SHARD_NAN = 3      /* x holds a NaN: no rank */
};
typedef struct {
    int64_t n, k;          /* global length and rank */
    int64_t cap;           /* compaction threshold on the bracket population */
    int32_t maxit;         /* iterates before compaction is forced */
    int32_t elem_bytes;    /* 4 (float32) or 8 (float64): the grid of the iterates */
    int32_t phase;         /* GBS_SHARD_* */
    int32_t how;           /* GBS_HOW_* once DONE */
    int32_t it;            /* iterates evaluated */
    int32_t use_bisect, stalled, dfv; /* safeguards, as in the single-array kernel */
    int64_t n_neginf, n_negzero;      /* #(x = -inf), #(x = -0) */
    int64_t cle_a, clt_b, cle_b;      /* #(x <= a) (-1 until counted), #(x < b), #(x <= b) */
    double a, b;           /* bracket: x_(k) lies in (a, b] */
    double t;              /* next point to evaluate (after gbs_shard_next) */
    double dF;             /* Phi(b) - Phi(a), Phi = F/n of Eq. (med_objOS) (in u = log1p(x - xmin) for
                              the log driver) */
    double result;         /* x_(k) once DONE */
    int32_t driver;        /* GBS_DRIVER_*: how the next point is chosen (gbs_shard_set_driver) */
    int32_t pad2;
    double xmin;           /* finite minimum of x (the log driver's origin) */
    double px, pg;         /* root-finding driver: the last point evaluated and its g */
    double step1, step2;   /* root-finding driver: the last two steps */
} gbs_shard_state;

/* How the sharded state machine picks the next point (gbs_shard_set_driver).  The
 * paper compares Kelley's cutting plane with minimisers and root-finders of the same
 * objective (Sec. 2, Sec. 4 Tables 1-2 and Discussion); all share the exact finish, so
 * they differ only in the passes taken. */
enum {
    GBS_DRIVER_KELLEY = 0,   /* tangent intersection (Algorithm 1, step 1.1), the default */
    GBS_DRIVER_BISECT = 1,   /* bisection of 0 in g(y): the midpoint of (a, b) in value */
    GBS_DRIVER_BRENT = 2,    /* Brent's root-finder on g(y): inverse quadratic or secant
                                interpolation of the subgradient counts, bisection when the
                                interpolant leaves the bracket or does not halve the step */
    GBS_DRIVER_LOG = 3       /* Kelley's method on the monotone image u = log(1 + x - xmin)
                                (Sec. 4 Discussion): the cost is evaluated by
                                gbs_cost_pass_log_*, the iterate mapped back by
                                x = xmin + expm1(u) */
};

/* Context lifetime.  gbs_create makes a context for CUDA ordinal `device`.  Creation
 * touches only the host: the device workspace is allocated on first use or by
 * gbs_reserve.  Errors:
 *  - EINVAL for a NULL ctx or an ordinal outside [0, device count);
 *  - ECUDA when the device cannot be queried or lacks cooperative launch;
 *  - ENOMEM when the host record cannot be allocated.
 * gbs_destroy synchronises the device and frees everything the context holds; NULL is a
 * no-op. */
gbs_status gbs_create(gbs_ctx** ctx, int device);
void gbs_destroy(gbs_ctx* ctx);

/* Grows the workspace so that selections of up to n elements of elem_bytes (4 or 8)
 * run without allocating.  Synchronous. */
gbs_status gbs_reserve(gbs_ctx* ctx, int64_t n, int32_t elem_bytes);

/* Replaces or reads the context's gbs_config; cfg is a host struct, copied.  The values
 * apply from the next call.  EINVAL for NULL pointers, a negative cap, maxit or
 * blocks_per_sm, or lms_start or knn_start outside {0, 1}. */
gbs_status gbs_set_config(gbs_ctx* ctx, const gbs_config* cfg);
gbs_status gbs_get_config(gbs_ctx* ctx, gbs_config* cfg);

/* x_(k) of x[0..n) (Sec. 1; Algorithm 1 and the hybrid finish of Sec. 3).
 * x: n elements, device, contiguous, aligned to its element size (any 16-byte phase).
 * out: 1 element, device.  EINVAL for NULL pointers, n < 1, k outside [1, n] or a
 * misaligned x; ENAN (device record) when x holds a NaN. */
gbs_status gbs_select_kth_f32(gbs_ctx* ctx, const float* x, int64_t n, int64_t k, float* out,
                              void* stream);
gbs_status gbs_select_kth_f64(gbs_ctx* ctx, const double* x, int64_t n, int64_t k, double* out,
                              void* stream);

/* Med(x) = x_(floor((n+1)/2)) (Sec. 1, Eq. (med_obj)). */
gbs_status gbs_median_f32(gbs_ctx* ctx, const float* x, int64_t n, float* out, void* stream);
gbs_status gbs_median_f64(gbs_ctx* ctx, const double* x, int64_t n, double* out, void* stream);

/* Pass 0 alone (Sec. 3, step 0).  out: device pointer to one gbs_array_stats. */
gbs_status gbs_array_stats_f32(gbs_ctx* ctx, const float* x, int64_t n, gbs_array_stats* out,
                               void* stream);
gbs_status gbs_array_stats_f64(gbs_ctx* ctx, const double* x, int64_t n, gbs_array_stats* out,
                               void* stream);

/* One fused pass at the points a < t for rank k (Algorithm 1, step 1.2; Sec. 4 figure,
 * Objective()).  a and t are converted to the element type.  out: device pointer to one
 * gbs_cost_eval.  EINVAL unless a < t and 1 <= k <= n. */
gbs_status gbs_cost_pass_f32(gbs_ctx* ctx, const float* x, int64_t n, int64_t k, double a,
                             double t, gbs_cost_eval* out, void* stream);
gbs_status gbs_cost_pass_f64(gbs_ctx* ctx, const double* x, int64_t n, int64_t k, double a,
                             double t, gbs_cost_eval* out, void* stream);

/* x_(k) of float32 x[0..n) without allocating anything: no context, no cudaMalloc,
 * cudaFree or allocating library call.  The paper has no counterpart; this is for
 * callers that cannot let a library allocate device memory (hosts whose device memory
 * belongs to their own arena or caching allocator, runtimes with a fixed device budget,
 * loops where an allocation's implicit device synchronisation is not acceptable).
 * Same kernel and same result as gbs_select_kth_f32.  Its scratch is one static device
 * array of about 4.1 MiB that every GPU loading the library holds until process exit.
 * Limits: 1 <= k <= n <= 1048576 (2^20), else GBS_EINVAL before any launch.
 * Runs on the current device.  The first call on a device resolves the array's address
 * there (cudaGetSymbolAddress).
 * All calls share the array: calls whose GPU work overlaps in time (different streams,
 * several threads) race and give wrong results; serialise them.  There is no per-call
 * record to read back: a NaN result means that x holds a NaN or that the device work
 * failed (a bounded wait gave up, an internal check failed). */
gbs_status gbs_select_kth_f32_noalloc(const float* x, int64_t n, int64_t k, float* out, void* stream);

/* Segmented batched select: out[s] = x_(k[s]) of the segment x[offsets[s], offsets[s+1])
 * for s = 0..S-1, all in one persistent launch (Sec. 2 notes that many medians of
 * different vectors are a workload of their own).  offsets: S+1 int64, device,
 * non-decreasing; k: S int64, device, 1-based, or NULL for the medians
 * floor((n_s+1)/2); out: S floats, device.  Each CTA takes whole segments, largest
 * first; a segment that fits in shared memory is radix-selected there, a larger one runs
 * the cutting plane (Algorithm 1) with CTA-wide reductions and compacts its final
 * bracket into shared memory, or, once it holds at most n_s/2 elements, into the CTA's
 * share of a 1 GiB device-memory area of the workspace.  A segment with n_s = 0 or k
 * outside [1, n_s] gets a NaN and GBS_EINVAL in the device status (gbs_last_stats).  The
 * call launches two kernels and no host synchronisation, so it can be captured in a CUDA
 * graph once the workspace holds 8*S bytes plus that area (gbs_reserve or a first call). */
gbs_status gbs_select_segmented_f32(gbs_ctx* ctx, const float* x, const int64_t* offsets, int32_t S,
                                    const int64_t* k, float* out, void* stream);

/* Autotuner of the segmented select: times every launch variant (CTA size and the
 * shared-memory capacity of the in-CTA select) on this batch, keeps the fastest for later
 * calls on ctx and leaves its results in out.  Synchronous.  chosen (may be NULL)
 * receives the variant; ms_per_variant (n_variants floats, may be NULL) the times. */
gbs_status gbs_segmented_autotune_f32(gbs_ctx* ctx, const float* x, const int64_t* offsets, int32_t S,
                                      const int64_t* k, float* out, void* stream, int32_t* chosen,
                                      float* ms_per_variant, int32_t n_variants);
/* The launch variant of later segmented calls on ctx (0 .. n_variants-1; a new context
 * uses variant 0: 512 threads, 12288-element shared-memory capacity).  EINVAL otherwise. */
gbs_status gbs_segmented_set_variant(gbs_ctx* ctx, int32_t variant);
gbs_status gbs_segmented_get_variant(gbs_ctx* ctx, int32_t* variant, int32_t* threads, int32_t* smem_cap,
                                     int32_t* n_variants);
/* Passes over each segment of the last segmented call (1 = loaded once into shared
 * memory).  Synchronises that call's stream.  passes: S int32, host. */
gbs_status gbs_segmented_passes(gbs_ctx* ctx, int32_t* passes, int32_t S);

/* Squared residuals of the linear model (Sec. 5, Eq. (model)) for C candidates:
 * S[c*n + i] = (y_i - sum_j X[i*p + j] * theta[c*p + j])^2, candidate-major.
 * X: n x p row-major float32; y: n; theta: p x C column-major (candidate c's p
 * coefficients contiguous); S: C*n floats; all device.  1 <= p <= 16.
 * precision 0: float32 FMAs on the CUDA cores; 1: the product X*theta on the tensor
 * cores as three TF32 products (hi*hi + hi*lo + lo*hi of a two-term split of each
 * operand, float32 accumulation), which keeps float32 accuracy. */
gbs_status gbs_residual_sq_f32(gbs_ctx* ctx, const float* X, const float* y, int64_t n, int32_t p,
                               const float* theta, int32_t C, float* S, int32_t precision, void* stream);

/* LMS and LTS objectives (Sec. 5) of C candidates: lms_out[c] = s_(k_lms) and
 * lts_out[c] = sum of the h_lts smallest s_i, where s_i are the squared residuals of
 * candidate c computed as in gbs_residual_sq_f32 (float32) and the LTS sum is accumulated
 * in float64 (Eq. (med_reg): all s below q = s_(h) plus (h - #(s < q)) q).
 * lms_out: C floats, lts_out: C doubles, device.  precision as in gbs_residual_sq_f32.
 * batched 1: one segmented select over all candidates in its trimmed-sum mode (the LMS
 * rank from the same compacted bracket when it lies inside, else a second batched
 * select for the few candidates where it does not); batched 0: one single-array select
 * per candidate and rank plus a summing kernel.  Allocates a C*n-float buffer on first
 * use (synchronously); 1 <= k_lms, h_lts <= n. */
gbs_status gbs_lms_lts_f32(gbs_ctx* ctx, const float* X, const float* y, int64_t n, int32_t p, const float* theta,
                           int32_t C, int64_t k_lms, int64_t h_lts, float* lms_out, double* lts_out,
                           int32_t precision, int32_t batched, void* stream);

/* The same objectives without writing the residual matrix: every pass of the cutting
 * plane (Algorithm 1, Sec. 3) recomputes s_ic = (y_i - x_i . theta_c)^2 on the tensor
 * cores (TF32 x 3 split, as precision 1 above) and reduces it per candidate in the
 * product's epilogue; the passes bracket the ranks k_lms and h_lts together, compact each
 * candidate's bracket and finish in the segmented select's trimmed-sum mode.  With
 * gbs_config.lms_start 0 (the default), n >= 65536 and ranks close enough that the
 * expected bracket fits the compaction buffer, the starting brackets are instead order
 * statistics of each candidate's squares on 8192 sampled rows, and a single pass over
 * the rows checks them by exact counts and compacts them.  Candidates whose residuals are
 * not all finite, whose sampled bracket misses a rank, or whose bracket does not fit the
 * compaction buffer (49152 elements), are recomputed by the batched form of
 * gbs_lms_lts_f32.  X: n x p row-major, y: n, theta: C x p row-major, all float32 device
 * arrays (any alignment; p <= 16, n <= 2^31).  Outputs as gbs_lms_lts_f32.  passes (host
 * pointer, may be NULL) receives the number of passes over the rows.  Synchronises
 * `stream` once per cutting-plane pass (the host stops when every candidate is ready to
 * compact) and once at the end. */
gbs_status gbs_lms_lts_fused_f32(gbs_ctx* ctx, const float* X, const float* y, int64_t n, int32_t p,
                                 const float* theta, int32_t C, int64_t k_lms, int64_t h_lts,
                                 float* lms_out, double* lts_out, int32_t* passes, void* stream);

/* Host record of the last gbs_lms_lts_fused_f32 call on ctx (synchronises its stream):
 * passes over the rows, launches of the fused pass kernels, their device time (CUDA
 * events recorded on the call's stream around each launch), and of that the time of the
 * compaction pass (the one pass of the sampled start). */
typedef struct {
    int32_t passes;
    int32_t pass_launches;
    double pass_ms;
    double write_ms;
} gbs_lms_stats;
gbs_status gbs_lms_last_stats(gbs_ctx* ctx, gbs_lms_stats* out);

/* ---- The LMS / LTS estimator search (Sec. 5: computing the estimator takes many
 * evaluations of F(theta)).  Candidates theta_c (C x p row-major float32, device; elemental
 * fits, for instance) are given.
 * C-steps (concentration steps) refine an LTS fit: refit the model by least squares on
 * the h observations the objective retains -- the rows weighted by the rho of
 * Eq. (med_reg), 1 below q = s_(h), a/b at q, 0 above -- and repeat while the objective
 * decreases; it cannot increase.  Which rows are retained is decided on float32 squared
 * residuals formed in a stated order (for j = 0..p-1, acc = acc + x_j * theta_j, each
 * product and sum rounded, no fused multiply-add; r = y - acc; s = r * r); the refit is
 * solved in float64 (normal equations, Cholesky) and rounded to float32; objectives are
 * float64 sums of those squares. */

/* For each candidate c: theta_out[c] (C x p float32, device) = the best fit reached from
 * theta[c] by at most max_steps refits, obj_out[c] (C float64, device) its LTS objective,
 * refits_out[c] (C int32, device, may be NULL) the refits kept.  1 <= p <= 16,
 * 1 <= h <= n <= 2^31, 0 <= max_steps <= 1000.  A refit whose retained rows do not
 * determine the coefficients (a non-positive Cholesky pivot) ends that candidate.  Squares
 * of up to 1 GiB of candidates at a time are written to the workspace.  Synchronises
 * `stream` once per refit round. */
gbs_status gbs_lts_csteps_f32(gbs_ctx* ctx, const float* X, const float* y, int64_t n, int32_t p, const float* theta,
                              int32_t C, int64_t h, int32_t max_steps, float* theta_out, double* obj_out,
                              int32_t* refits_out, void* stream);
/* The estimators: both objectives of every candidate by gbs_lms_lts_fused_f32; LMS: the
 * candidate of least LMS objective (the smallest index among equal values) -> lms_theta
 * (p floats), lms_value, lms_index; LTS: the n_refine candidates of least LTS objective
 * (smaller index first on ties) refined by C-steps, the refined fit of least objective
 * (the better-ranked start on ties) -> lts_theta (p floats), lts_value (float64),
 * lts_index (its start).  All outputs are device pointers; lms_index and lts_index may be
 * NULL.  1 <= C <= 65536 (candidates are ranked by counting); other limits as above. */
gbs_status gbs_lms_lts_search_f32(gbs_ctx* ctx, const float* X, const float* y, int64_t n, int32_t p,
                                  const float* theta, int32_t C, int64_t k_lms, int64_t h_lts, int32_t n_refine,
                                  int32_t max_steps, float* lms_theta, float* lms_value, int32_t* lms_index,
                                  float* lts_theta, double* lts_value, int32_t* lts_index, void* stream);

/* ---- k-nearest-neighbour regression and classification through the k-th order
 * statistic of the distances (Sec. 5, last application).  For each query q_j the k
 * nearest of the n points x_i (Euclidean) are marked by an indicator against d_(k), the
 * k-th smallest distance: 1 below it, 0 above it, and (k - #(d < d_(k))) / #(d = d_(k))
 * for every point exactly at it (the a/b weight at the order statistic of
 * Eq. (med_reg)), so that exactly k points count whatever the ties.
 * Distances: the squared distance is formed in float32 in a fixed order -- for
 * t = 0..p-1, e = q_t - x_t, acc = acc + e*e, every operation rounded on its own, no
 * fused multiply-add -- and the order statistic is taken on it; which points count is
 * therefore decided exactly on those float32 values.
 * Layout: X n x p and Q m x p row-major float32, device; 1 <= p <= 32, 1 <= k <= n < 2^31,
 * m >= 1.  kth_d2 (m floats, device, may be NULL) receives d_(k)^2 per query.
 * Route: with gbs_config.knn_start 0 (default) and n >= 65536, each query's distances to
 * 8192 evenly spread rows propose a bracket around rank k; one fused pass counts the
 * points below it and at its upper end and compacts those inside, and a finish per query
 * selects d_(k) among them.  A query whose bracket fails its count check (or outgrows its
 * buffer) takes the plain form: its distance row is written to the workspace, the
 * segmented select finds d_(k), and the pass reduces the points below and at d_(k).
 * Device-side errors (gbs_last_stats): GBS_ENAN for a non-finite coordinate in X or Q
 * (the outputs then hold NaN, class -1); GBS_EINVAL for a label outside [0, n_classes).
 * The workspace grows on demand (synchronously); the call synchronises `stream` once per
 * 16384 queries to read how many queries need the plain form. */

/* Regression: pred[j] = sum_i rho_ij w_ij f_i / sum_i rho_ij w_ij, rho the indicator above,
 * w = 1 (weight 0) or w = 1 / (d + eps) with d = sqrt(d^2) in float64 (weight 1, eps > 0).
 * f: n float32, device; pred: m float64, device (sums in float64).  EINVAL for NULL X, Q,
 * f or pred, a bad size or rank, weight outside {0, 1}, or a non-positive eps with
 * weight 1. */
gbs_status gbs_knn_regress_f32(gbs_ctx* ctx, const float* X, int64_t n, int32_t p, const float* f, const float* Q,
                               int32_t m, int64_t k, int32_t weight, double eps, double* pred, float* kth_d2,
                               void* stream);
/* Classification: votes[j][c] = sum_i rho_ij [label_i = c] (m x n_classes float64, device,
 * may be NULL; each the correctly rounded value of an exact rational), cls[j] = the class
 * with the largest vote, the smallest label among equal votes (decided on the exact
 * rationals; m int32, device).  labels: n int32 in [0, n_classes), device;
 * 1 <= n_classes <= 1024. */
gbs_status gbs_knn_classify_f32(gbs_ctx* ctx, const float* X, int64_t n, int32_t p, const int32_t* labels,
                                int32_t n_classes, const float* Q, int32_t m, int64_t k, int32_t* cls,
                                double* votes, float* kth_d2, void* stream);

/* Host record of the last kNN call on ctx (synchronises its stream): queries, queries that
 * took the plain form, full passes over the points for the first 16384 queries (the
 * fused pass counts 1; the plain form adds its distance rows and its second pass), and
 * the device time of the sampled start's fused pass launches (CUDA events recorded on the
 * call's stream around each launch), with their count. */
typedef struct {
    int64_t queries;
    int64_t plain_queries;
    int32_t passes;
    int32_t pass_launches;
    double pass_ms;
} gbs_knn_stats;
gbs_status gbs_knn_last_stats(gbs_ctx* ctx, gbs_knn_stats* out);

/* ---- Learned starting bracket (no counterpart in the paper; it replaces the starting
 * bracket of Algorithm 1, step 0).  A sketch of x -- 1024 samples x[j*floor(n/1024)],
 * sorted; features: the 32 sample quantiles at sorted positions 16+32i standardised by
 * the sample mean mu and population spread sd, asinh of the standardised sample min and
 * max, asinh(mu/sd) and log(sd)/16 -- feeds a 36-64-64-2 MLP with GELU hidden layers
 * whose outputs (c, omega) propose (mu + sd(c - e^omega), mu + sd(c + e^omega)] for the
 * median.  With gbs_config.use_learned set and a model loaded, a median select of
 * n >= 65536 checks the proposal by counts in its first pass (and compacts it when it
 * holds the answer); a side that fails falls back to the data's extreme.  Results are
 * identical with or without a model; only the pass count changes.
 * Parameters: 6658 float32, order W1[64][36], b1[64], W2[64][64], b2[64], W3[2][64], b3[2]. */
gbs_status gbs_bracket_model_set(gbs_ctx* ctx, const float* weights, int32_t count);   /* host array */
gbs_status gbs_bracket_model_get(gbs_ctx* ctx, float* weights, int32_t count);         /* host array */
/* Checkpoint: "GBSBRKT1", u32 version 1, n_in, n_hid, n_out, n_params, u64 Adam step, then
 * weights, Adam first and second moments (float32, little-endian). */
gbs_status gbs_bracket_model_save(gbs_ctx* ctx, const char* path);
gbs_status gbs_bracket_model_load(gbs_ctx* ctx, const char* path);
/* Sketch features of x (n >= 1024): feat 36 floats, musd {mu, sd} 2 doubles; device. */
gbs_status gbs_bracket_features_f32(gbs_ctx* ctx, const float* x, int64_t n, float* feat, double* musd,
                                    void* stream);
/* Proposed bracket for the median of x: out = {a, b, valid} (3 doubles, device). */
gbs_status gbs_bracket_propose_f32(gbs_ctx* ctx, const float* x, int64_t n, double* out, void* stream);
/* Network outputs (c, omega) for B feature rows: F B x 36, out B x 2 (device). */
gbs_status gbs_bracket_forward(gbs_ctx* ctx, const float* F, int32_t B, float* out, void* stream);
/* Gradient of the mean batch loss (z - c)^2 + rho_0.99(|z - c| - e^omega),
 * rho_tau(u) = u (tau - [u < 0]), for B rows F (B x 36) and labels Z (B): grad 6658 floats,
 * loss 1 double (device). */
gbs_status gbs_bracket_grad(gbs_ctx* ctx, const float* F, const float* Z, int32_t B, float* grad, double* loss,
                            void* stream);
/* Trains the loaded model with Adam (beta 0.9 / 0.999, eps 1e-8) for `steps` batches of
 * `batch` rows of (F, Z) (device, N rows), reshuffled every epoch from `seed`.
 * loss_hist: `steps` floats (host) or NULL.  Synchronous. */
gbs_status gbs_bracket_train(gbs_ctx* ctx, const float* F, const float* Z, int32_t N, int32_t batch,
                             int32_t steps, float lr, uint64_t seed, float* loss_hist, void* stream);
/* Training array on the device from Philox4x32-10 (counters (i, j, hi(i), 0), key seed):
 * family 0 N(0,1); 1 Student-t with integer nu = p0 in [1, 64]; 2 lognormal(0, p0);
 * 3 N(0,1) replaced with probability p0 by N(p1, p2); then loc + scale * value. */
gbs_status gbs_generate_training_array_f32(gbs_ctx* ctx, float* x, int64_t n, int32_t family, float p0, float p1,
                                           float p2, float loc, float scale, uint64_t seed, void* stream);
/* Raw Philox4x32-10 (Salmon et al., SC'11) for m (counter, key) pairs: counters 4m,
 * keys 2m, out 4m uint32 (device). */
gbs_status gbs_philox4x32_10(gbs_ctx* ctx, const uint32_t* counters, const uint32_t* keys, uint32_t* out, int32_t m,
                             void* stream);

/* Synchronises the stream of the last call on ctx and copies its record to *out. */
gbs_status gbs_last_stats(gbs_ctx* ctx, gbs_run_stats* out);

/* Static, human-readable name of a status code. */
const char* gbs_status_string(gbs_status s);

/* Failure-path check (no paper counterpart): one device-side wait that cannot complete (a
 * grid barrier of one CTA counting two arrivals) gives up after limit_ns nanoseconds
 * (1e3 .. 1e9), as every wait of the persistent kernels does after 2 s, and records
 * GBS_ETIMEOUT in the device status, copied to *device_status (host pointer).
 * Synchronises stream; the context stays usable.  EINVAL for a bad argument. */
gbs_status gbs_check_wait_timeout(gbs_ctx* ctx, int64_t limit_ns, int32_t* device_status, void* stream);

/* ---------------------------------------------------------------------------------
 * Sharded selection.  Algorithm 1 (Sec. 3) over a vector split into shards that are
 * reduced separately -- on several devices, in several processes, or as sub-ranges of
 * one array -- with the per-pass results summed by the caller (an all-reduce), as the
 * paper's multi-GPU remark (Sec. 4) sums the per-device reductions on the host.  The
 * state functions are host code and need no device; every per-element pass is one of
 * the library's own kernels on a shard:
 *   1. every shard: gbs_array_stats_*.  Totals: sums of n, n_nan, n_neginf, n_posinf,
 *      n_negzero, n_finite and sum; the least `min` and the greatest `max` over the
 *      shards that hold a finite element (c_le_min and c_lt_max are not used).  Then
 *      gbs_shard_begin().
 *   2. while phase == GBS_SHARD_ITERATE: gbs_shard_next() sets t (or moves the state to
 *      GBS_SHARD_COMPACT); every shard runs gbs_cost_pass_*(k = any valid rank, a, t);
 *      totals: sums of c_lt_t, c_le_t, c_le_a and S; then gbs_shard_update().
 *   3. GBS_SHARD_COMPACT: every shard copies its elements of (a, b] with gbs_compact_*;
 *      x_(k) is element k - cle_a of their union (gbs_select_kth_* on it).
 * The result is the single-array result bit for bit; the iterates may differ from the
 * single-array kernel's, whose cost partials are summed in another order.
 * --------------------------------------------------------------------------------- */

/* Trivial resolution and the starting bracket from the pass-0 totals (Sec. 3, step 0).
 * cap <= 0 selects max(n/16, 4096); maxit <= 0 selects 64.  EINVAL for bad arguments
 * or totals whose counts do not add up to n. */
gbs_status gbs_shard_begin(gbs_shard_state* s, int32_t elem_bytes, int64_t n, int64_t k,
                           const gbs_array_stats* total, int64_t cap, int32_t maxit);
/* The next point t strictly inside (a, b) on the element grid: the tangent intersection
 * of Algorithm 1, step 1.1, or the bracket midpoint in totalOrder keys after a slow
 * step.  Moves the state to GBS_SHARD_COMPACT instead once (a, b] holds at most cap
 * elements, after maxit iterates, or after two stalled steps.  EINVAL unless ITERATE. */
gbs_status gbs_shard_next(gbs_shard_state* s);
/* Steps 1.3-1.4 from the totals of the pass at (a, t).  EINTERNAL when the totals are
 * inconsistent (c_le_a differs from the state's, or counts out of order). */
gbs_status gbs_shard_update(gbs_shard_state* s, const gbs_cost_eval* total);
/* Selects the driver (GBS_DRIVER_*) of a state made by gbs_shard_begin, before its first
 * gbs_shard_next.  The log driver starts from a bisection (its cost difference over the
 * starting bracket is not known from pass 0) and needs the passes of
 * gbs_cost_pass_log_*.  EINVAL for an unknown driver or a state that has iterated. */
gbs_status gbs_shard_set_driver(gbs_shard_state* s, int32_t driver);

/* Device-resident loop (step 2 above without a host round trip per pass).  The state
 * (made on the host by gbs_shard_begin, gbs_shard_set_driver and one gbs_shard_next) is
 * copied to device memory, d_state, 8-byte aligned; d_acc is a device array of 8 int64,
 * zeroed before the first pass, both owned by the caller.  Per pass, stream-ordered:
 *   a. every shard: gbs_shard_pass_dev_*: if the state is ITERATE and d_acc[4] == 0, adds
 *      the shard's #(x < t), #(x <= t), #(x <= a) to d_acc[0..2] and its S (the cost of
 *      gbs_cost_pass_*, or of gbs_cost_pass_log_* for the log driver, on the float32
 *      images of the elements) to d_acc[3] in fixed point: each block's part times
 *      2^fx rounded to an integer, fx = 61 - e where n (t - a) < 2^e, the same in
 *      every process, so the totals do not depend on the order of the additions;
 *   b. the caller sums d_acc[0..3] over its processes in place (an all-reduce);
 *   c. gbs_shard_step_dev: steps 1.3-1.4 from those totals, then step 1.1 (the code of
 *      gbs_shard_update and gbs_shard_next), and clears d_acc[0..3].  An update or next
 *      that fails leaves the state as it was and stores its status in d_acc[4], which
 *      stops the loop.
 * Once the state leaves ITERATE both calls do nothing, so the host may enqueue several
 * passes and read the phase (and d_acc[4]) back now and then.  Step 3 is as above.
 * EINVAL for a null or misaligned pointer or n < 0 (n = 0: nothing to do). */
gbs_status gbs_shard_pass_dev_f32(gbs_ctx* ctx, const float* x, int64_t n, const gbs_shard_state* d_state,
                                  int64_t* d_acc, void* stream);
gbs_status gbs_shard_pass_dev_f64(gbs_ctx* ctx, const double* x, int64_t n, const gbs_shard_state* d_state,
                                  int64_t* d_acc, void* stream);
gbs_status gbs_shard_step_dev(gbs_ctx* ctx, gbs_shard_state* d_state, int64_t* d_acc, void* stream);
/* A pass over several shards in one call: gbs_shard_pass_dev_* on shards[i] (device
 * pointers) of lens[i] elements for i < count (host arrays), then, when step != 0,
 * gbs_shard_step_dev (for a process that sums nothing with others).  Stops at the first
 * failing launch and returns its status. */
gbs_status gbs_shard_passes_dev_f32(gbs_ctx* ctx, const float* const* shards, const int64_t* lens, int32_t count,
                                   gbs_shard_state* d_state, int64_t* d_acc, int32_t step, void* stream);
gbs_status gbs_shard_passes_dev_f64(gbs_ctx* ctx, const double* const* shards, const int64_t* lens, int32_t count,
                                   gbs_shard_state* d_state, int64_t* d_acc, int32_t step, void* stream);

/* One pass at the points a < t for rank k in the coordinates u = log1p(x - xmin)
 * (Sec. 4 Discussion: order statistics commute with increasing maps, and the log map
 * keeps huge elements from swamping the cost sums): the counts #(x < t), #(x <= t),
 * #(x <= a) as gbs_cost_pass_*, S = sum over a < x_i < t of (u(t) - u(x_i)) and
 * dphi = (c_le_a - k + 1/2)(u(t) - u(a)) + S; u is taken of the elements inside (a, t)
 * only (float32 arithmetic: the cost steers iterates, never results).  out: device
 * pointer to one gbs_cost_eval.  EINVAL unless xmin - 1 < a < t, both finite. */
gbs_status gbs_cost_pass_log_f32(gbs_ctx* ctx, const float* x, int64_t n, int64_t k, double a, double t,
                                 double xmin, gbs_cost_eval* out, void* stream);
gbs_status gbs_cost_pass_log_f64(gbs_ctx* ctx, const double* x, int64_t n, int64_t k, double a, double t,
                                 double xmin, gbs_cost_eval* out, void* stream);

/* Copies the elements x_i with a < x_i <= b (IEEE comparison; NaN never qualifies) into
 * z[0..z_cap) in no particular order, and stores how many qualify in *count (host
 * pointer; the call synchronises `stream`).  x: n elements, device.  z: device, z_cap
 * elements, owned by the caller.  GBS_ENOMEM when more than z_cap qualify (z then holds
 * z_cap of them); EINVAL unless a < b. */
gbs_status gbs_compact_f32(gbs_ctx* ctx, const float* x, int64_t n, double a, double b, float* z,
                           int64_t z_cap, int64_t* count, void* stream);
gbs_status gbs_compact_f64(gbs_ctx* ctx, const double* x, int64_t n, double a, double b, double* z,
                           int64_t z_cap, int64_t* count, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GBSELECT_H */
