/*
 * spamm.h -- C ABI of the GB300 SpAMM / Newton-Schulz library (libspamm.so).
 *
 * The method is from Challacombe, Haut & Bock, "A N-Body Solver for Square
 * Root Iteration":
 *   - SpAMM product A (x)_tau B, Eq. (newspamm): both operands are held as a
 *     quadtree of Frobenius norms; a sub-product a^i . b^i is culled when
 *     ||a^i|| ||b^i|| < tau ||A|| ||B|| (relative criterion, root norms of the
 *     whole operands), and only the surviving leaf-tile products are formed.
 *   - Dual-channel Newton-Schulz iteration, Eq. (cannonical), with the NS map
 *     h[x] = (3 - x)/2 (alpha = 1, Sec. 4.2; opts->map selects the damped,
 *     stabilised h_alpha of Sec. 4.2 "Mapping"): from S scaled into (0,1],
 *     X0 = Y0 = S, Z0 = I;  T = h[X];  Y <- T (x)_{tau_s} Y;  Z <- Z (x)_tau T;
 *     X <- Y (x)_tau Z;  Y -> S^{1/2}, Z -> S^{-1/2}.  tau_s is the tighter
 *     threshold of the "sensitive" y channel (Sec. 4.1, tau_s ~ 0.01 tau).
 *   - Trace error t_k = (n - tr X_k)/n monitors convergence (Sec. 4.2).
 *
 * Conventions for every entry point:
 *   - Matrices are dense, row-major, n x n, double precision.
 *   - A matrix pointer may address host memory or device memory of the
 *     current CUDA device; the library tells them apart with
 *     cudaPointerGetAttributes.  Device memory of another GPU is rejected
 *     with SPAMM_ERR_ARG.  Page-locked host memory is read and written
 *     in place by the kernels (through its device mapping); pageable host
 *     data is staged through the library's own device buffers.  The caller owns every pointer it passes; inputs are not
 *     modified; the call returns after the results are written.
 *   - The library owns its scratch space (tile buffers, norm trees, task
 *     lists), cached per problem size and released by spamm_release().
 *   - Work runs on opts->stream (a cudaStream_t; NULL is the legacy default
 *     stream).  Calls are thread safe; concurrent calls use separate scratch.
 *   - Leaf tiles are N_b x N_b with N_b in {32, 64, 128}.  The tile grid has
 *     m = ceil(n / N_b) tiles per side; edge tiles are zero padded and
 *     quadtree nodes that cover no tile do not exist.
 *   - Return value: SPAMM_OK (0) or a negative SPAMM_ERR_* code; no C++
 *     exception crosses this interface.  spamm_last_error() gives a message
 *     for the calling thread's most recent failure.
 */
#ifndef SPAMM_H
#define SPAMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SPAMM_OK 0
#define SPAMM_ERR_ARG (-1)           /* bad size, tau < 0 or NaN, bad option    */
#define SPAMM_ERR_NOMEM (-2)         /* device allocation failed                 */
#define SPAMM_ERR_DIVERGED (-3)      /* t_k not finite or |t_k| >= 1: the
                                        iteration left its basin of stability
                                        (Sec. 3, Sec. 5.1); or, when the
                                        residual is computed, |t_k| < 1e-8 with
                                        ||ZSZ - I||_F >= 1: culling errors
                                        carried Y and Z off the roots while
                                        X = YZ looks converged;
                                        outputs are still written              */
#define SPAMM_ERR_NOTCONVERGED (-4)  /* tol_t > 0 and maxit reached with
                                        |t_k| > tol_t; outputs are written      */
#define SPAMM_ERR_TIMEOUT (-5)       /* a bounded device-side wait expired
                                        (every wait inside the kernels gives
                                        up after a fixed number of polls; see
                                        spamm_test_expire_next_wait)           */
#define SPAMM_ERR_ADMIT (-6)         /* server: request footprint exceeds the
                                        memory budget                          */
#define SPAMM_ERR_CUDA (-7)          /* a CUDA runtime call failed              */
#define SPAMM_ERR_UNSUPPORTED (-8)   /* option or size this build does not do   */
#define SPAMM_ERR_NOTFOUND (-9)      /* server: unknown request id              */

/* ---- arithmetic of the leaf-tile products ------------------------------ */
#define SPAMM_FP64 0   /* FP64 tiles, FP64 fused multiply-add                  */
#define SPAMM_EMU64 1  /* FP64 tiles split into six 8-bit digit slices (FP16) on
                          the tensor cores with exact FP32 partial sums and
                          64-bit accumulation (FP64-class result)              */

/* ---- NS map T = h_alpha[eps I + (1 - 2 eps) X] (Sec. 4.2 "Mapping") ----- */
#define SPAMM_MAP_NS 0      /* alpha = 1, eps = 0: T = (3 I - X) / 2             */
#define SPAMM_MAP_SCALED 1  /* the logistic h_alpha[u] = (sqrt(alpha)/2)(3 - alpha u)
                               after the stabilising shift-and-scale
                               u = eps + (1 - 2 eps) x of [0,1] onto [eps, 1-eps],
                               with alpha(t) = 1 + 1.85/(1 + exp(-50 (t - .35)))
                               and eps(t) = .1/(1 + exp(-75 (t - .30))) taken
                               from the trace error t of the X being mapped
                               (t_0 from S / c): scaling for the early steps,
                               switched off towards convergence.  The
                               stabiliser leaves a fixed point with
                               t ~ -eps(0) ~ -1.7e-11 (ZSZ ~ (1 + 1.7e-11) I). */

/* ---- instance of the square-root iteration ------------------------------ */
#define SPAMM_CHANNEL_DUAL 0    /* Eq. (cannonical): Y and Z channels, X = Y Z      */
#define SPAMM_CHANNEL_SINGLE 1  /* Eq. (single): Z <- Z (x)_tau h[X],
                                   W = s (x)_{tau_s} Z, X <- Z^T (x)_tau W
                                   (Y = W unscaled, which tends to S^{1/2});
                                   paper order only                            */

/* ---- schedule of one solve's iteration on the device -------------------- */
#define SPAMM_SCHED_BRANCHES 0  /* the y and z products of an iteration on two
                                   streams, each product its own cull, leaf-
                                   product, slicing and quadtree launches      */
#define SPAMM_SCHED_STAGES 1    /* the batched engine with one problem: the y and
                                   z products share one launch of each kernel,
                                   then the x product (dual channel, map
                                   SPAMM_MAP_NS, device or page-locked S, Y, Z,
                                   no residual and no profile; otherwise as
                                   SPAMM_SCHED_BRANCHES)                       */
#define SPAMM_SCHED_AUTO 2      /* chosen per device, n, arithmetic, leaf and
                                   decade of tau by timing the call's own
                                   input: three solves with each, alternating,
                                   the faster minimum kept (cached)            */

/* ---- order of the two channel products --------------------------------- */
#define SPAMM_ORDER_PAPER 0       /* Y <- T Y, Z <- Z T, X <- Y Z (as printed)  */
#define SPAMM_ORDER_TRANSPOSED 1  /* Y <- Y T, Z <- T Z, X <- Z Y: the exact
                                     transpose of the printed iteration        */

typedef struct spamm_opts {
    int leaf;          /* N_b: 32, 64 or 128; 0 = chosen by spamm_autotune_leaf
                          on the call's own input                               */
    int precision;     /* SPAMM_FP64 or SPAMM_EMU64                             */
    double tau_s;      /* y-channel threshold; < 0 selects 0.01 * tau           */
    double mu_rel;     /* Tikhonov shift S + mu I (Sec. 6) with
                          mu = mu_rel * Gershgorin bound of S; 0 = none        */
    double tol_t;      /* stop once |t_k| <= tol_t; 0 runs exactly maxit steps  */
    int order;         /* SPAMM_ORDER_PAPER or SPAMM_ORDER_TRANSPOSED           */
    int residual;      /* nonzero: also compute ||Z S Z - I||_F (FP64, dense)   */
    int profile;       /* nonzero: time every leaf-product, cull, quadtree
                          and slicing kernel of the products with CUDA events
                          on the call's stream (stats->gemm_ms, cull_ms,
                          tree_ms, slice_ms); the two branches of an
                          iteration then run one after the other            */
    void* stream;      /* cudaStream_t; NULL = legacy default stream            */
    int map;           /* SPAMM_MAP_NS or SPAMM_MAP_SCALED                      */
    int channel;       /* SPAMM_CHANNEL_DUAL or SPAMM_CHANNEL_SINGLE            */
    int schedule;      /* SPAMM_SCHED_BRANCHES, _STAGES or _AUTO (solves)       */
} spamm_opts;

typedef struct spamm_stats {
    int iters;                 /* iterations run                                */
    double t_final;            /* t_k of the last iteration                     */
    double resid_F;            /* ||Z S Z - I||_F if opts->residual, else -1    */
    double scale_c;            /* Gershgorin bound c used to scale S into (0,1] */
    long long tasks_total;     /* surviving leaf products over the whole call   */
    long long tasks_dense;     /* leaf products without culling (m^3 per product) */
    double flops;              /* 2 N_b^3 per surviving leaf product            */
    double* t_hist;            /* in: NULL or caller array of maxit doubles      */
    long long* task_hist;      /* in: NULL or caller array of 3*maxit counts
                                  (y, z, x products of each iteration)          */
    double gemm_ms;            /* opts->profile: summed duration of the
                                  leaf-product kernels (CUDA events), else 0    */
    long long gemm_launches;   /* leaf-product kernel launches of the call       */
    long long* lens_hist;      /* in: NULL, or a caller array of
                                  maxit * 3 * 3 * lens_bins counts: the plane-
                                  diagonal profile ("lensing", Sec. 7.2) of
                                  every product's surviving tile triples
                                  (i, j, k).  Entry ((k * 3 + p) * 3 + q) *
                                  lens_bins + d counts the triples of product p
                                  (task_hist order) of iteration k at distance d
                                  tiles from plane q: q = 0 |i - j|, 1 |j - k|,
                                  2 |i - k|; the last bin takes every d >=
                                  lens_bins - 1.  Filled for the iterations run */
    int lens_bins;             /* in: bins per plane, 1 .. 4096 (with lens_hist) */
    long long tensor_units;    /* SPAMM_EMU64: tensor-core work issued, counted
                                  by the leaf-product kernel in units of one
                                  128 x 64 x 64 FP16 product (2*128*64*64
                                  flops): 12 per leaf product                   */
    double cull_ms;            /* opts->profile: summed duration of the cull
                                  kernels of the products (CUDA events), else 0 */
    long long cull_launches;   /* opts->profile: cull launches timed            */
    double tree_ms;            /* opts->profile: summed duration of the products'
                                  quadtree (upper norm levels) passes           */
    long long tree_launches;
    double slice_ms;           /* opts->profile, SPAMM_EMU64: summed duration of
                                  the products' digit-slicing passes            */
    long long slice_launches;
    int schedule;              /* the schedule the solve ran with (after AUTO)  */
} spamm_stats;

/* Fill *opts with defaults: leaf 64, SPAMM_FP64, tau_s = 0.01 tau, no shift,
 * fixed iteration count, paper order, no residual, default stream,
 * SPAMM_MAP_NS, SPAMM_CHANNEL_DUAL, SPAMM_SCHED_BRANCHES. */
void spamm_opts_init(spamm_opts* opts);

/*
 * Leaf-tile size for problems like S: times one SpAMM product S (x)_tau S
 * at every leaf size the arithmetic supports (32, 64 and 128 for
 * SPAMM_FP64; SPAMM_EMU64 runs on 64 only) and returns the fastest in
 * *leaf.  The choice is cached per device, n, arithmetic and decade of tau,
 * so later calls return at once; entry points given opts->leaf = 0 use it.
 * S is n x n row-major FP64, host or device; opts may be NULL (its leaf is
 * ignored).  The trial products run on opts->stream and are synchronised.
 * Errors: SPAMM_ERR_ARG (n, tau, null pointer), SPAMM_ERR_NOMEM, SPAMM_ERR_CUDA.
 */
int spamm_autotune_leaf(const double* S, int n, double tau, const spamm_opts* opts, int* leaf);

/*
 * C = A (x)_tau B, Eq. (newspamm), with the relative criterion
 * ||A_ij||_F ||B_jk||_F < tau ||A||_F ||B||_F (evaluated squared, in FP64;
 * strict "<" culls).  tau = 0 gives the dense product.  Per output tile the
 * surviving products are summed with j ascending.  opts may be NULL
 * (defaults); stats may be NULL.
 * Errors: SPAMM_ERR_ARG for n <= 0, tau < 0 or NaN, or a bad leaf size.
 */
int spamm_multiply(const double* A, const double* B, double* C, int n, double tau,
                   const spamm_opts* opts, spamm_stats* stats);

/*
 * Y ~ S^{1/2} and Z ~ S^{-1/2} for symmetric positive definite S by the
 * dual-channel iteration of Eq. (cannonical) (see the top of this file), or
 * with opts->channel = SPAMM_CHANNEL_SINGLE the single channel of
 * Eq. (single); SPAMM_ERR_ARG for the single channel with
 * SPAMM_ORDER_TRANSPOSED.
 * S is scaled by its Gershgorin bound c (plus mu, Sec. 6) into (0,1]; the
 * results are unscaled as Y * sqrt(c), Z / sqrt(c).  Both divisions are
 * products with the once-rounded reciprocals 1/c and 1/sqrt(c), computed
 * once per solve.  Runs maxit iterations,
 * or fewer when opts->tol_t > 0.  Y and Z are written even when the status
 * is SPAMM_ERR_DIVERGED or SPAMM_ERR_NOTCONVERGED.
 */
int spamm_sqrt_invsqrt(const double* S, int n, double tau, int maxit, double* Y, double* Z,
                       const spamm_opts* opts, spamm_stats* stats);

/*
 * `count` independent problems of (possibly) different sizes, each exactly
 * as spamm_sqrt_invsqrt(S[q], n[q], tau[q], maxit, Y[q], Z[q], opts, ...).
 * The problems run concurrently on the device; every result is the one a
 * single call gives (the leaf size and arithmetic depend only on the
 * request, never on what it is batched with).  stats may be NULL or an array
 * of `count` entries.  Returns the first nonzero per-problem status, or 0.
 */
int spamm_sqrt_invsqrt_batched(int count, const double* const* S, const int* n, const double* tau,
                               int maxit, double* const* Y, double* const* Z, const spamm_opts* opts,
                               spamm_stats* stats);

/*
 * Product representation of the regularised inverse factor, Sec. 6
 * (Eq. (spammsandwich) with the iterative regularisation of
 * Eq. (product_rep)): a telescoping product of SpAMM "slices".
 *   z_0 = (S + mu[0] c0 I)^{-1/2} by spamm_sqrt_invsqrt at tau0 (the
 *         most-approximate-yet-effective slice), Z = z_0; then for
 *   l = 1 .. levels-1:
 *     R_l = Z^T (x)_{tau1} ((S + mu[l] c0 I) (x)_{tau1} Z)   (the residual)
 *     z_l = R_l^{-1/2} by spamm_sqrt_invsqrt at tau0 (no shift)
 *     Z  <- Z (x)_{tau1} z_l
 * so that Z^T (S + mu[levels-1] c0 I) Z ~ I.  c0 is the Gershgorin bound
 * of S; the shifts mu[] (levels of them, >= 0, typically decreasing) are
 * relative to it like opts->mu_rel.  Every slice runs maxit iterations (or
 * stops at opts->tol_t) with opts' leaf, precision, map, channel, order
 * and tau_s rule (opts->mu_rel is ignored).  S, Z: n x n row-major, host or
 * device.  iters: NULL or `levels` ints, the NS iterations of each slice.
 * Device scratch: six n x n matrices for the call, plus the cached plans.
 * Returns SPAMM_OK, an argument or resource error, or the first non-OK
 * status of a slice's solve (SPAMM_ERR_DIVERGED, SPAMM_ERR_NOTCONVERGED:
 * Z is still written).
 */
int spamm_invsqrt_product(const double* S, int n, int levels, const double* mu, double tau0, double tau1,
                          int maxit, double* Z, int* iters, const spamm_opts* opts);

/*
 * Norm tree of A for parity checks: nu_leaf[i*m + j] = ||A_ij||_F^2 for the
 * m x m leaf tiles (m = ceil(n/leaf)), accumulated in FP64, and *root =
 * ||A||_F^2 summed up the quadtree (Sec. 1, norm recursion).
 */
int spamm_norm_tree(const double* A, int n, int leaf, double* nu_leaf, double* root, void* stream);

/*
 * Task list of A (x)_tau B for parity checks: for output tile (i,k),
 * counts[i*m + k] surviving j, listed ascending in jlist[(i*m + k)*m + 0 ..].
 * counts holds m*m ints and jlist m*m*m ints (host or device).  *thr gets
 * the squared threshold tau^2 ||A||^2 ||B||^2 and *total the task count.
 */
int spamm_cull(const double* A, const double* B, int n, double tau, int leaf, int* counts, int* jlist,
               double* thr, long long* total, void* stream);

/*
 * C = A (x)_tau B like spamm_multiply, for callers that cannot allocate
 * device memory.  The paper has no counterpart; this is an interface for
 * programs that reserve all device memory up front and must not see a
 * library allocate once they run.  No call here allocates: no cudaMalloc,
 * cudaFree or allocating library routine.  The scratch is one fixed device
 * array of about 6.3 MB, held on every GPU that loads the library until the
 * process exits.
 *   - A, B, C: device pointers of the current device, or managed memory
 *     (row-major n x n doubles, caller-owned).  Host pointers and device
 *     memory of another GPU are rejected with SPAMM_ERR_ARG.
 *   - n <= SPAMM_NOALLOC_MAX_N; larger n returns SPAMM_ERR_UNSUPPORTED.
 *   - leaf: 32, 64 or 128 (0 selects 64).  stream: cudaStream_t or NULL.
 *   - The work is enqueued on `stream` and the call returns without waiting;
 *     synchronise the stream before reading C.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - CUDA loads device code lazily by default: the array and the kernels
 *     of each leaf size are placed in device memory by the first call that
 *     uses them.  So make one call per device, for every leaf size the
 *     program will use, before it reserves the rest of the device memory;
 *     after that no call needs device memory beyond what it was given.
 *   - Every call shares the one array.  Calls ordered on one stream are safe;
 *     calls that overlap on the GPU (other streams or threads) race.
 * Same arithmetic and task lists as spamm_multiply with SPAMM_FP64.
 */
#define SPAMM_NOALLOC_MAX_N 512
int spamm_multiply_noalloc(const double* A, const double* B, double* C, int n, double tau, int leaf,
                           void* stream);

/* ---- serving: a request loop over spamm_sqrt_invsqrt ------------------
 * Requests of any size arrive at any time and are admitted in arrival order
 * as soon as one of `max_active` workers is free and the request's device
 * footprint (the scratch spamm_sqrt_invsqrt needs for its size, leaf and
 * arithmetic, plus staging when its matrices are in host memory) fits in
 * `bytes_budget` next to the requests already running.  Each worker has its
 * own CUDA stream, so admitted requests overlap on the device.  Y and Z of a
 * request are written exactly as spamm_sqrt_invsqrt(S, n, tau, maxit, Y, Z,
 * opts) writes them: a result does not depend on the other requests.  Work
 * runs on the device that is current when the server is created, on the
 * workers' own streams: S must hold its final values when it is submitted
 * (finish the work that writes it first).  The caller keeps S, Y and Z
 * valid until the request is waited for.  When the options are ones the
 * batched solve covers (dual channel, alpha = 1 map, leaf != 0) and a
 * request's matrices are device or page-locked memory, a free worker takes
 * the head of the queue together with the requests queued behind it (same
 * maxit, at most 64, within budget / max_active of device memory) and
 * solves them as one batch, sharing every kernel launch of their
 * iterations; each result is still the one a single call gives.
 */
typedef struct spamm_server spamm_server;

#define SPAMM_REQ_QUEUED 0
#define SPAMM_REQ_RUNNING 1
#define SPAMM_REQ_DONE 2

/* Create a server; opts as for spamm_sqrt_invsqrt (residual unsupported,
 * stream ignored).  SPAMM_ERR_ARG for a zero budget or max_active outside
 * 1..64. */
int spamm_server_create(size_t bytes_budget, int max_active, const spamm_opts* opts, spamm_server** server);

/* Queue a request; *id identifies it.  SPAMM_ERR_ADMIT when its footprint
 * alone exceeds the budget (it could never run); SPAMM_ERR_ARG as for
 * spamm_sqrt_invsqrt. */
int spamm_server_submit(spamm_server* server, const double* S, int n, double tau, int maxit, double* Y,
                        double* Z, long long* id);

/* *state = SPAMM_REQ_QUEUED, _RUNNING or _DONE; SPAMM_ERR_NOTFOUND for an
 * unknown (or already waited-for) id. */
int spamm_server_poll(spamm_server* server, long long id, int* state);

/* Wait up to timeout_s seconds (< 0: no limit) for a request, then return
 * its status (as spamm_sqrt_invsqrt would) and forget it.  stats (may be
 * NULL; its t_hist/task_hist are not filled) and *latency_s (submit to
 * completion, may be NULL) are written.  SPAMM_ERR_TIMEOUT if the request is
 * still pending (it stays queued), SPAMM_ERR_NOTFOUND for an unknown id. */
int spamm_server_wait(spamm_server* server, long long id, double timeout_s, spamm_stats* stats,
                      double* latency_s);

/* Finish every queued and running request, then free the server. */
int spamm_server_destroy(spamm_server* server);

/*
 * Failure-path check of the bounded device waits.  The next spamm_multiply
 * with SPAMM_EMU64 on the calling thread makes every CTA of its tensor-core
 * leaf-product kernel first wait on an mbarrier that nothing arrives at, for
 * at most `polls` polls.  The wait expires, as any internal wait of the kernel
 * does after its own limit, before the CTA has issued a copy or a product:
 * the kernel records the error, frees its tensor memory and exits, and the
 * call returns SPAMM_ERR_TIMEOUT (C is not valid).  Later calls run normally.
 * polls = 0 clears a pending request.  SPAMM_ERR_ARG for polls < 0.
 */
int spamm_test_expire_next_wait(long long polls);

/*
 * Layout check of the tensor-core leaf product (SPAMM_EMU64).  A product
 * whose output tile holds more than one accumulator chunk of tasks can run with
 * the chunks at alternating tensor-memory columns, so that the next chunk's
 * products start while part of this chunk's accumulator is still being read
 * out.  Both layouts give the same result bits.  mode = -1: the library's
 * choice (alternating from 128 tiles per side, single products only);
 * 0: never; 1: always.  Process-wide; affects products enqueued (or graphs
 * captured) after the call, so release cached plans (spamm_release) before
 * comparing.  SPAMM_ERR_ARG for mode outside -1..1.
 */
int spamm_test_emu_alternate(int mode);

/* Message for the calling thread's last failure ("" if none). */
const char* spamm_last_error(void);

/* Short name of a status code. */
const char* spamm_strerror(int status);

/* Free every cached scratch buffer (call with no work in flight). */
int spamm_release(void);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all threads).  A diagnostic for counting device work per call. */
long long spamm_kernel_launches(void);

/* Library version string. */
const char* spamm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPAMM_H */
