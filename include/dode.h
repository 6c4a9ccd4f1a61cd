/*
 * dode.h -- C ABI of libdode: per-day dynamic OD demand estimation (DODE) by
 * stochastic projected gradient descent (SPGD) on GB300 (sm_103a).
 *
 * Method: Ma & Qian, "Estimating multi-year 24/7 origin-destination demand using
 * high-granular multi-source traffic data" (arXiv 1901.09266).  For each day
 * independently (Sec. 2.7) the library solves the NNLS problem of Eq. (opt) /
 * Eq. (nnls):
 *
 *     min_{q >= 0}  sum_{a in A^o} sum_{h2} m[h2][a] (x[h2][a] - (B q)[h2][a])^2
 *
 * where B = delta * rho * p (Eq. (assign)) is rebuilt from the day's link speeds:
 * link travel times (Sec. 2.4), leading-vehicle trajectories (Eq. (cost)), the
 * dynamic assignment ratio rho (Eq. (dar)) and logit route choice (Eq. (logit)).
 * Algorithm 1 (Sec. 3.3) with Adagrad and projection max(q, 0) is the solver.
 *
 * Conventions for every entry point:
 *  - Return value: DODE_OK (0) or a negative DODE_ERR_* code.  No entry point
 *    throws; dode_last_error() returns a message for the last failed call on a
 *    context.
 *  - Layouts are time-major as in the paper's Table "DODE framework variable
 *    vectorization": q[d][h][od] (entry (h-1)|K| + od of day d), link arrays
 *    x[d][h][o] with o the position of the link in dode_network.obs_links, speed
 *    arrays [d][h][a] over all links.  All arrays are dense, C-contiguous.
 *  - Pointer arguments tagged "ptr_kind" are host pointers (DODE_PTR_HOST) or
 *    device pointers on the context's GPU (DODE_PTR_DEVICE); all others are host
 *    pointers.  Inputs are borrowed only for the duration of the call (copied or
 *    uploaded); outputs are caller-allocated.
 *  - All device work is issued on the context's stream (dode_options.stream,
 *    NULL = legacy default stream).  Every call returns after its work on that
 *    stream has completed (device errors are reported by the call that caused
 *    them).
 *  - A context owns all its device memory.  Calls on one context are not
 *    thread-safe; distinct contexts are independent.
 *  - Time: ticks of 1/ticks_per_s s; an interval is interval_s * ticks_per_s
 *    ticks (4800 for 5-minute intervals at 16 ticks/s).
 */
#ifndef DODE_H
#define DODE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes -------------------------------------------------------- */
#define DODE_OK 0
#define DODE_ERR_ARG -1                  /* bad argument / size / pointer */
#define DODE_ERR_ROUTE_NOT_CONTIGUOUS -2 /* head of link j != tail of link j+1 */
#define DODE_ERR_ROUTE_REPEATS_LINK -3   /* a route uses a link twice (not a simple path) */
#define DODE_ERR_BAD_SPEED -4            /* speed <= 0, NaN or Inf */
#define DODE_ERR_TICK_OVERFLOW -5        /* a link travel time above 2^24 ticks */
#define DODE_ERR_OOM -6                  /* device allocation failed */
#define DODE_ERR_CUDA -7                 /* CUDA runtime error (message in dode_last_error) */
#define DODE_ERR_DEVICE_TIMEOUT -8       /* a bounded device wait gave up */
#define DODE_ERR_STATE -9                /* call order: e.g. solve before set_days */
#define DODE_ERR_UNSUPPORTED -10         /* valid input this form does not handle */
#define DODE_ERR_BOUNDS -11              /* debug build only (-DDODE_CHECK_BOUNDS): a device index check
                                            failed; dode_last_error names the site and the index, and
                                            the access was skipped */

/* ---- enums ------------------------------------------------------------------ */
#define DODE_PTR_HOST 0
#define DODE_PTR_DEVICE 1

#define DODE_FORM_FUSED 0  /* one persistent kernel, DAR recomputed on chip every pass */
#define DODE_FORM_PLAIN 1  /* separate kernels over a DAR materialised in HBM */

#define DODE_PREC_FP32 0   /* FP32 operands and accumulation */
#define DODE_PREC_BF16 1   /* BF16 DAR fractions, demands and residuals; FP32 accumulation */

#define DODE_MAX_ROUTE_LINKS 64

/* ---- inputs ----------------------------------------------------------------- */

/* Directed graph (Sec. 4, Step 0) and the observed link set A^o.            */
typedef struct {
    int32_t n_nodes;
    int32_t n_links;
    const int32_t *link_tail;   /* [n_links] node ids in [0, n_nodes) */
    const int32_t *link_head;   /* [n_links] */
    const float *link_len_mi;   /* [n_links] length in miles, finite, > 0 */
    int32_t n_obs;              /* |A^o| >= 1 */
    const int32_t *obs_links;   /* [n_obs] distinct link ids; column order of counts / mask */
} dode_network;

/* Path sets K_rs (Sec. 4, Step 0) in CSR form.                              */
typedef struct {
    int32_t n_od;               /* |K_q| */
    int32_t n_routes;           /* Pi */
    const int32_t *route_od;    /* [n_routes] OD pair of each route, in [0, n_od); every OD has >= 1 route */
    const int32_t *route_ptr;   /* [n_routes + 1] offsets into route_links, route_ptr[0] = 0 */
    const int32_t *route_links; /* links of route k in travel order, route_ptr[k] .. route_ptr[k+1]-1;
                                   1 .. DODE_MAX_ROUTE_LINKS contiguous, distinct links */
} dode_routes;

typedef struct {
    int32_t n_intervals;     /* N intervals per day (288) */
    int32_t interval_s;      /* Delta H in seconds (300) */
    int32_t ticks_per_s;     /* time resolution (16) */
    float theta_per_min;     /* logit dispersion of Eq. (logit) on minutes (0.1); 0 = uniform split */
    float eps;               /* Adagrad epsilon (1e-10) */
    int32_t row_chunk;       /* Algorithm 1 batch size b in rows; 0 = all rows each update */
    uint64_t seed;           /* row permutation seed (row_chunk > 0) */
    int32_t form;            /* DODE_FORM_* */
    int32_t precision;       /* DODE_PREC_* (fused form only) */
    int32_t block_threads;   /* fused kernel CTA size (0 = tuned default) */
    int32_t ctas_per_sm;     /* fused kernel CTAs per SM (0 = tuned default) */
    int32_t device;          /* CUDA device ordinal (-1 = current) */
    void *stream;            /* cudaStream_t for all work (NULL = default stream) */
    int32_t use_graph;       /* 1: dode_solve with DEVICE outputs replays a CUDA graph of its device
                                work (captured on first use, re-captured when iters, step, theta or
                                the launch shape change) */
    int32_t max_ctas;        /* cap on resident CTAs of the fused kernel (0 = as many as fit) */
    int32_t day_base;        /* index of the first loaded day in the caller's day numbering (>= 0);
                                seeds the row permutation of row_chunk > 0 */
    int32_t couple_days;     /* 1: the loaded days are consecutive and are solved jointly -- the
                                whole-period NNLS of Sec. 2.7 without its cut at midnight.  A trip
                                that departs on day d and is still travelling after midnight takes
                                day d + 1's link times and counts on day d + 1's links (its first
                                maxoff + 2 intervals); the gradient of day d's demand then includes
                                day d + 1's residuals.  The last loaded day drops mass after its
                                midnight as the per-day problem does.  Needs the fused form and
                                row_chunk = 0 (else dode_create returns DODE_ERR_ARG), and a
                                network whose accumulator ring and tick window fit in shared
                                memory (else DODE_ERR_UNSUPPORTED at the first evaluation).
                                Each epoch then takes two launches; use_graph is ignored.
                                dode_dar_distance, dode_get_dar and dode_loss_static_scratch
                                refuse coupled days.  0 = independent days (default). */
    int32_t epoch_slices;    /* fused solve of independent days: cut each day's epochs into this many
                                slices, handed out slice-major so that no CTA idles while the last
                                days run (slice s of a day starts when its slice s - 1 is done; a
                                wait past 20 s gives DODE_ERR_DEVICE_TIMEOUT).  Results are
                                bitwise the same for any value.  0 = automatic (min(16, iters / 4)
                                slices when there are more days than CTAs and iters >= 8, else 1);
                                1 = whole days. */
} dode_options;

typedef struct dode_ctx dode_ctx;

/* Fill *opt with the defaults listed above.                                   */
void dode_default_options(dode_options *opt);

/*
 * dode_create -- validate the network and route sets and build a context.
 * Network and routes are copied; the device copies of the route tables are
 * built once here (OD-major route order, link -> observed column map).
 * Errors: DODE_ERR_ARG (sizes, ids out of range, duplicated observed link, bad
 * option), DODE_ERR_ROUTE_NOT_CONTIGUOUS, DODE_ERR_ROUTE_REPEATS_LINK,
 * DODE_ERR_CUDA / DODE_ERR_OOM.  On error *out is NULL.
 * Limits checked here, before any device call (DODE_ERR_ARG):
 *   - every link length finite and > 0; every OD pair has at least one route;
 *   - a route has 1 .. 64 links; fewer than 2^22 OD pairs;
 *   - an interval of 2 .. 2^24 ticks (interval_s * ticks_per_s), a day of at
 *     most 2^29 ticks;
 *   - row_chunk > 0 needs n_intervals * n_obs < 2^31 (row ids are int32);
 *   - couple_days = 1 needs the fused form and row_chunk = 0.
 */
int dode_create(const dode_network *net, const dode_routes *routes, const dode_options *opt,
                dode_ctx **out);

/*
 * dode_set_days -- load D days of observations and speeds (Sec. 4, Steps 1 and 4).
 *   counts [D][N][n_obs] link counts x (vehicles per interval), FP32
 *   speeds [D][N][n_links] link speeds in mph (Sec. 2.4), FP32, finite, > 0
 *   mask   [D][N][n_obs] 1 = observed, 0 = missing (excluded from the loss); NULL = all observed
 * Computes the travel-time tick table and each day's route times once
 * (Sec. 3.2 DAR construction inputs), and resets the solver state (q = 0,
 * Adagrad accumulator = 0).  Errors: DODE_ERR_ARG, DODE_ERR_BAD_SPEED (first bad
 * value reported in the message), DODE_ERR_TICK_OVERFLOW, DODE_ERR_OOM, DODE_ERR_CUDA.
 */
int dode_set_days(dode_ctx *ctx, int32_t n_days, const float *counts, const float *speeds,
                  const uint8_t *mask, int32_t ptr_kind);

/*
 * dode_prefetch_days -- start copying the next batch of days to the device
 * while the current one solves.  Host pointers, same layouts as dode_set_days;
 * pinned host memory makes the copies asynchronous.  The copies run on a
 * stream of the context's own and the call returns at once.  The next
 * dode_set_days with DODE_PTR_HOST and the same n_days, counts, speeds and
 * mask pointers waits for them and uses the device copies instead of copying
 * again; a dode_set_days with other inputs lets them finish and ignores them.
 * The host buffers must stay valid and unchanged until that dode_set_days
 * call.  Keeps one device copy of the inputs (D N (n_links + n_obs) 4 bytes +
 * D N n_obs for the mask).  Errors: DODE_ERR_ARG, DODE_ERR_OOM, DODE_ERR_CUDA.
 */
int dode_prefetch_days(dode_ctx *ctx, int32_t n_days, const float *counts, const float *speeds,
                       const uint8_t *mask);

/* Replace the counts (and mask, if not NULL) of the loaded days; speeds and
 * solver state are kept.  Same layouts as dode_set_days. */
int dode_set_counts(dode_ctx *ctx, const float *counts, const uint8_t *mask, int32_t ptr_kind);

/*
 * dode_solve -- run `iters` epochs of Algorithm 1 (Sec. 3.3) on every loaded day,
 * continuing from the current state (q, G), with step size `step` (eta, > 0).
 *   batch     days per minibatch of the outer loop over days (>= 1, or 0 = all).
 *             Days are independent problems (Sec. 2.7), so the minibatch order
 *             changes no iterate; the device drains all days through one work
 *             queue and runs each day's epochs back to back.
 *   q_out     [D][N][n_od] final OD flows (ptr_kind), may be NULL
 *   loss_out  [D] masked squared loss of the final q, FP64 (ptr_kind), may be NULL
 * One epoch with row_chunk = 0 is one full-row update per day.  With
 * row_chunk = b > 0 (fused form) each epoch permutes the day's observed rows
 * (Algorithm 1's permutate: row r = h * n_obs + o gets the key SplitMix64
 * output number r of the stream seeded with seed ^ (day << 32 | epoch), day =
 * day_base + index in the loaded set; rows go in ascending (key, r)) and
 * makes one update per run of b consecutive rows (the last run partial);
 * the loss trace still reports the full masked loss at each epoch start.
 * iters = 0 takes no step: q_out is the current state and loss_out its loss.
 * Errors: DODE_ERR_STATE (no days loaded), DODE_ERR_ARG, DODE_ERR_UNSUPPORTED
 * (row_chunk > 0 with the plain form), DODE_ERR_CUDA.
 */
int dode_solve(dode_ctx *ctx, int32_t iters, float step, int32_t batch, float *q_out,
               double *loss_out, int32_t ptr_kind);

/* Per-epoch loss trace of the last dode_solve: trace[e][d] = masked loss of day d
 * at the start of epoch e (FP32), host pointer [iters][D].  DODE_ERR_STATE if no
 * solve has run since the days were loaded. */
int dode_get_loss_trace(dode_ctx *ctx, float *trace, int32_t iters);

/* Solver state: q and the Adagrad accumulator G, both [D][N][n_od] FP32.      */
int dode_get_state(dode_ctx *ctx, float *q, float *G, int32_t ptr_kind);
int dode_set_state(dode_ctx *ctx, const float *q, const float *G, int32_t ptr_kind);

/* xhat[d][h][o] = (B_d q_d)[h][o], the link counts implied by q (Eq. (reverse)
 * with Eq. (flow)); q [D][N][n_od], xhat [D][N][n_obs], same ptr_kind. */
int dode_forward(dode_ctx *ctx, const float *q, float *xhat, int32_t ptr_kind);

/*
 * Differentiable form.  L(q, theta) = sum_d sum m (B_d(theta) q_d - x_d)^2 with
 * the logit dispersion `theta` (per minute) in place of the context's.
 *   loss   [D] per-day loss, FP64 (host)
 *   dq     [D][N][n_od] dL/dq = 2 B^T r (ptr_kind), may be NULL
 *   dtheta [D] dL/dtheta per day, FP64 (host), may be NULL
 * The DAR is recomputed on the fly in both passes (nothing is checkpointed).
 */
int dode_loss(dode_ctx *ctx, const float *q, float theta, double *loss, int32_t ptr_kind);
int dode_loss_grad(dode_ctx *ctx, const float *q, float theta, double *loss, float *dq,
                   double *dtheta, int32_t ptr_kind);

/*
 * dode_last_totals -- the multi-year objective of Sec. 2.7 as the sum of the
 * independent days' objectives: FP64 sums, in day order, of the per-day
 * results of the context's last dode_loss or dode_loss_grad call, formed on
 * the device.
 *   loss_total    sum_d loss_d (host)
 *   dtheta_total  sum_d dL_d/dtheta (host), may be NULL; needs dode_loss_grad
 *                 as the last of the two calls
 * Errors: DODE_ERR_STATE (no such call since the days were loaded, or
 * dtheta_total after dode_loss), DODE_ERR_ARG, DODE_ERR_CUDA.
 */
int dode_last_totals(dode_ctx *ctx, double *loss_total, double *dtheta_total);

/*
 * dode_dense_nnls -- the paper's efficiency experiment (Sec. 5, "Algorithm
 * efficiency": a dense random B, y = B x with x >= 0, NNLS(B, y)) solved by
 * Algorithm 1 with full-row updates, for m right-hand sides sharing B:
 * per column j, r = B x_j - y_j, g = B^T r (no factor 2, as Algorithm 1
 * prints it), G += g^2, x_j = max(x_j - step g / (sqrt(G) + eps), 0).
 * Standalone: no context is needed.
 *   B          [n_rows][n_cols] FP32, row-major
 *   Y          [n_rows][m] FP32
 *   X          [n_cols][m] FP32, in: the starting point, out: the iterate after `iters` steps
 *   G          [n_cols][m] FP32 Adagrad accumulator in/out, or NULL to start from 0
 *   loss       [m] FP64 out: ||B x_j - y_j||^2 of the final iterate
 *   method     0 = automatic, 1 = one pass over B per iteration (rows of B are
 *              streamed into shared memory by bulk asynchronous copies and used
 *              for both products; all iterations run in one cooperative launch
 *              with a grid-wide step between passes; needs m = 1,
 *              n_cols % 4 == 0, n_cols <= 8192, a 16-byte aligned B and a device
 *              that supports cooperative launches, else DODE_ERR_UNSUPPORTED),
 *              2 = two passes (one per product), 3 = tensor cores: the m
 *              right-hand sides stacked into two GEMMs per iteration (R = B X - Y,
 *              then B^T R) with TF32 operands and FP32 accumulation, split-K
 *              partials summed in a fixed order, the iterations replayed as a
 *              CUDA graph; needs m a multiple of 16 in 16..256, n_rows and
 *              n_cols multiples of 4 and, for device pointers, 16-byte aligned
 *              B and Y, else DODE_ERR_UNSUPPORTED.  TF32 keeps 10 mantissa bits
 *              of each operand, so the iterates differ from those of the FP32
 *              methods by up to about 1e-2 relative.  Automatic takes one pass
 *              when it applies, else two.
 *   kernel_ms  out (may be NULL): GPU time of the iterations and the final residual
 * All arrays are host or device pointers per ptr_kind; stream is a cudaStream_t
 * (NULL = default stream); the call returns when its work is complete.
 * Limits: methods 0-2: 1 <= m <= 8 and n_cols * m <= 51200 (x is staged in
 * shared memory); method 3: 16 <= m <= 256.
 * Errors: DODE_ERR_ARG, DODE_ERR_UNSUPPORTED (the limits), DODE_ERR_OOM, DODE_ERR_CUDA,
 * DODE_ERR_DEVICE_TIMEOUT (a bounded device wait of the one-pass kernel ran out: a
 * row copy, or the grid-wide step); the message goes to stderr.  After a timeout
 * the library stays usable: the kernel lets its copies in flight land before it
 * returns.
 */
int dode_dense_nnls(int32_t n_rows, int32_t n_cols, int32_t m, const float *B, const float *Y, int32_t iters,
                    float step, float eps, int32_t method, float *X, float *G, double *loss, double *kernel_ms,
                    int32_t ptr_kind, void *stream);

/*
 * dode_dense_set_wait_limit -- how many times a bounded wait of the one-pass
 * dense kernel (method 1) polls for a row copy before it gives up with
 * DODE_ERR_DEVICE_TIMEOUT (default 2^26; process-wide).  0 makes every such
 * wait give up at once, which exercises the failure path without a fault; the
 * kernel's final wait for its own copies in flight keeps its fixed limit.
 * Errors: DODE_ERR_ARG (polls < 0).
 */
int dode_dense_set_wait_limit(int64_t polls);

/*
 * dode_set_patterns -- traffic patterns of the loaded days (Step 2-3 of the
 * framework, Sec. 4; Eq. (logit) computes a pattern's route choice from the
 * mean travel time of each path over the pattern's days).
 *   pattern  [D] host: pattern label of each loaded day (>= 0), or -1 for a day
 *            whose route choice uses its own travel times; NULL clears all
 *            labels (every day uses its own, the default)
 * From then on every call (solve, forward, loss, gradients) takes the route
 * choice of day d from the mean, over the days with d's label, of the route
 * times C_k(h) (FP64 sums in day order); dL/dtheta differentiates that route
 * choice.  Labels are cleared by dode_set_days.  Clustering the days is the
 * caller's (Sec. 3.1).  Errors: DODE_ERR_STATE, DODE_ERR_ARG (a label < -1),
 * DODE_ERR_CUDA / DODE_ERR_OOM.
 */
int dode_set_patterns(dode_ctx *ctx, const int32_t *pattern);

/*
 * dode_r2 -- goodness of fit of Step 6 ("Quality check", Sec. 4; the case study
 * reports the average R-square between observed and estimated link flow,
 * Sec. 5): per day, R^2 = 1 - SS_res / SS_tot over the observed cells, with
 * SS_res = sum m (xhat - x)^2 for OD flows q and logit dispersion theta, and
 * SS_tot = sum m (x - xbar)^2 about the day's masked mean count xbar.
 *   q   [D][N][n_od] FP32 (ptr_kind)
 *   r2  [D] FP64 (ptr_kind); NaN for a day with no observed cell or constant
 *       observed counts (SS_tot = 0)
 * Errors: DODE_ERR_STATE, DODE_ERR_ARG, DODE_ERR_CUDA / DODE_ERR_OOM.
 */
int dode_r2(dode_ctx *ctx, const float *q, float theta, double *r2, int32_t ptr_kind);

/*
 * dode_dar_distance -- stability of the DAR across days (Sec. 5: the l2
 * distance between each day's DAR matrix of Eq. (dar) and the average DAR
 * matrix, whose histogram the paper plots).  The DAR of a day holds rho for
 * every (route, link position, departure interval h1, arrival interval h2)
 * with h2 before the end of the day; the mean is taken over the loaded days.
 *   dist     [D] ||rho_d - mean rho||_F, FP64, host
 *   mean_sq  ||mean rho||_F^2, FP64, host, may be NULL
 * Shares are computed in FP32, sums in FP64 in a fixed order.  Works on the
 * loaded days' speeds only; the solver state is untouched.
 * Errors: DODE_ERR_STATE, DODE_ERR_ARG, DODE_ERR_CUDA / DODE_ERR_OOM.
 */
int dode_dar_distance(dode_ctx *ctx, double *dist, double *mean_sq);

/*
 * dode_loss_static_scratch -- the per-day loss of dode_loss for the loaded days,
 * computed without allocating any device memory.  The paper has no counterpart:
 * this serves callers that cannot call cudaMalloc once running (a real-time or
 * certified loop that forbids allocation after start-up, a process whose GPU
 * memory is owned by another allocator, a latency-critical path that cannot
 * afford cudaMalloc's implicit device synchronisation).
 *   q     [D][N][n_od] OD flows, FP32, DEVICE pointer
 *   theta logit dispersion per minute
 *   loss  [D] per-day loss, FP64, DEVICE pointer (written by the kernel)
 * All per-call scratch (q in the kernel layout, the route-choice table, the
 * residual slots and accumulator words of the resident CTAs, the work-queue
 * counter) comes from one 32 MiB file-scope device array that every GPU that
 * loads this library holds until the process exits; the day data and route
 * tables are the context's, loaded earlier.  If the days need more scratch
 * than that for even one CTA the call returns DODE_ERR_ARG and says how much;
 * otherwise it runs as many resident CTAs as fit (dode_last_grid reports how
 * many).  Each call looks up the array's device address on the context's
 * device (cudaGetSymbolAddress; host code only holds a stand-in under the
 * array's name), so a device reset between calls leaves no stale address.  The
 * call synchronises the context's stream, so it cannot be made while that
 * stream is being captured.  Every call shares the array and leaves its
 * contents behind: calls that overlap on the GPU (on different streams or
 * contexts of the same device) race and must not be made.  Returns after the
 * loss is written.
 */
int dode_loss_static_scratch(dode_ctx *ctx, const float *q, float theta, double *loss);

/* ---- inspection (host outputs; for checks and debugging) --------------------- */

/* Tick table of one day: out[h][a] = travel time of link a entered in interval h. */
int dode_get_ticks(dode_ctx *ctx, int32_t day, int32_t *out);
/* Route times of one day in minutes: out[h][k] (Eq. (cost)), leading vehicle of t^h. */
int dode_get_route_times(dode_ctx *ctx, int32_t day, float *out);
/* FIFO repairs applied on one day and the largest trip offset in intervals. */
int dode_get_day_info(dode_ctx *ctx, int32_t day, int64_t *n_repairs, int32_t *max_offset);
/*
 * DAR entries of one day for every (route k, link position j, departure h1)
 * (Eq. (dar)), as built by the plain form's DAR builder.  Call with kjh = rho =
 * NULL to get the count in *n; then with arrays of that size:
 *   kjh [n][4] = (k, j, h1, h2), rho [n] FP32, ordered by (k, j, h1, h2).
 */
int dode_get_dar(dode_ctx *ctx, int32_t day, int64_t *n, int32_t *kjh, float *rho);

/* ---- timing and launch shape --------------------------------------------------- */

/* Device time in ms of the hot-path kernel(s) of the last solve / forward / loss
 * call, measured with CUDA events on the context's stream. */
double dode_last_kernel_ms(const dode_ctx *ctx);
/* Number of hot-path kernel launches the last solve / forward / loss call made. */
int64_t dode_last_launches(const dode_ctx *ctx);
/* CTAs of the last call's fused-kernel launch (0 if that call ran no fused kernel). */
int32_t dode_last_grid(const dode_ctx *ctx);

/* Epoch slices per day of the last fused solve (1 = whole days; see
 * dode_options.epoch_slices); 0 before any fused solve.                      */
int32_t dode_last_slices(const dode_ctx *ctx);
/* CUDA device ordinal the context runs on (-1 for a NULL context). */
int32_t dode_device(const dode_ctx *ctx);
/* Number of kernel launches (all kernels, all calls) made by this context so far. */
int64_t dode_total_launches(const dode_ctx *ctx);
/* Override the fused kernel launch shape (autotuner); 0 = tuned default. */
int dode_set_launch(dode_ctx *ctx, int32_t block_threads, int32_t ctas_per_sm);
/* Cap the fused kernel's resident CTAs (0 = as many as fit); results do not
 * depend on it (each day is solved by one CTA, sums are exact). */
int dode_set_max_ctas(dode_ctx *ctx, int32_t max_ctas);
/* Switch stream (cudaStream_t); the context's previous work must be complete. */
int dode_set_stream(dode_ctx *ctx, void *stream);

const char *dode_last_error(const dode_ctx *ctx);
void dode_destroy(dode_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DODE_H */
