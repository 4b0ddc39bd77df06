/*
 * snect.h -- C ABI of the GB300 SNeCT library.
 *
 * SNeCT (Choi & Sael, arXiv 1711.08095) fits a Tucker model X ~ G x1 U1 x2 U2 x3 U3
 * (Eq. 2) to the observed cells of a sparse patient x gene x platform tensor, with an L2
 * term (Eq. 3, in the per-entry form of Sec. 2.3.2) and a gene-network term
 * lambda_g * f_g (graph regulariser of Sec. 2.3.1), by the stochastic gradient sweep of
 * Alg. 1.  This library runs that sweep, the network pass, the objective, fold-in of new
 * patients (Eq. 9) and top-k patient search (Sec. 3.2.1) on one GPU.
 *
 * Conventions for every entry point:
 *   - Return value: SNECT_OK (0) or a negative SNECT_E* code; no C++ exception crosses the
 *     ABI.  snect_last_error() returns a message for the last failing call on a context.
 *   - Pointers marked "any" may point to host memory (pageable or pinned) or to device
 *     memory of the context's GPU; the library copies from them during the call and keeps no
 *     reference afterwards.  Pointers marked "host" must be host memory.
 *   - Indices are 0-based (the paper counts from 1).  An entry is (i, j, k) =
 *     (patient, gene, platform), stored as 3 consecutive int32.
 *   - The core G is J1*J2*J3 floats, g(p,q,r) at (p*J2 + q)*J3 + r; factor U_n is I_n*J_n
 *     floats, row-major.
 *   - All device work runs on the stream given at snect_init (the caller's stream, e.g.
 *     PyTorch's current stream; NULL means the default stream).  Calls that return results on
 *     the host synchronise that stream.
 *   - A context is not thread-safe: one host thread at a time.
 */
#ifndef SNECT_H
#define SNECT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SNECT_OK 0
#define SNECT_EINVAL (-1)   /* bad argument: size, index out of range, NaN, self loop ... */
#define SNECT_ENOMEM (-2)   /* a device allocation failed */
#define SNECT_ECUDA (-3)    /* a CUDA call failed; see snect_last_error */
#define SNECT_ETIMEDOUT (-4)
#define SNECT_EBUSY (-5)

#define SNECT_FP32 0
#define SNECT_BF16 1
#define SNECT_BF16_TC 2

typedef struct snect_ctx snect_ctx;

/* Hyper-parameters of Alg. 1 (inputs "core size (J1..JN), learning rate eta, regularisation
 * factors lambda and lambda_g"; the network constrains mode 2, the genes). */
typedef struct {
    int32_t I[3];      /* tensor dims I1 (patients), I2 (genes), I3 (platforms) */
    int32_t J[3];      /* core ranks J1, J2, J3; each in [1, 32], J1*J2*J3 <= 5120 */
    float lambda;      /* L2 weight lambda */
    float lambda_g;    /* network weight lambda_g */
    float lr;          /* learning rate eta */
    int32_t batch;     /* > 0: deterministic mode, fixed-order mini-batches of this many
                          entries (<= 4096); 0: fast mode (lock-free sweep) */
    int32_t wave;      /* fast mode: entries between two updates of the core and the
                          platform factor (0 = library default) */
    int32_t precision; /* SNECT_FP32; SNECT_BF16: fast mode with J1, J2 in {16, 32}, the sweep
                          gathers rows in BF16 (at 16 x 16 x 5 from a BF16 copy of the gene
                          factor kept beside the FP32 one, arithmetic FP32; at the other ranks
                          through the tensor-core form below); SNECT_BF16_TC: the same ranks,
                          the dense per-entry contractions on the tensor cores with BF16
                          operands and FP32 accumulation.  Every factor stays FP32. */
    uint64_t seed;     /* reserved; the caller supplies the visit order and the init */
} snect_config;

/* Objective terms after the last update (Eq. 3 + Sec. 2.3.2 + graph regulariser), FP64. */
typedef struct {
    double data;       /* 1/2 sum over training entries of (x - x~)^2 */
    double reg;        /* lambda/2 (||G||^2 + sum_n sum_{i observed} ||u_i^(n)||^2) */
    double graph;      /* f_g = 1/2 sum_edges y ||u^(2)_k1 - u^(2)_k2||^2 */
    double total;      /* data + reg + lambda_g * graph  (f_opt) */
    double rmse_train; /* sqrt(mean (x - x~)^2) over the training entries */
    double rmse_test;  /* same over the test entries passed to snect_loss (0 if none) */
} snect_loss_t;

/* Creates a context and copies the problem to the GPU (Alg. 1 inputs: tensor X, network Y,
 * hyper-parameters; line 1's initial G and U are supplied by the caller).
 *   idx   any, nnz*3 int32 training entries, in the order the sweep visits them
 *         (deterministic mode cuts this order into consecutive batches)
 *   val   any, nnz float
 *   edges any, m*2 int32 undirected gene pairs, each edge once, no self loops
 *   w     any, m float edge weights y > 0
 *   G0, U1, U2, U3  any, initial core and factors (layouts above)
 *   stream  a cudaStream_t, or NULL for the default stream
 * Validates ranges (indices, sizes, finite values, self loops); computes the counts
 * |Omega^{n,i}| and the per-batch row grouping on the GPU.  In fast mode one kernel packs,
 * validates, counts and orders the entries into waves; it reads idx and val in place when
 * they are device memory or pinned (page-locked) host memory, and pageable memory is copied
 * first.  Inside a wave the entries are grouped by platform and patient; the order among one
 * patient's entries of one platform is not fixed (every gradient of a wave is taken at the
 * wave-start parameters).  On failure *out is NULL.
 * Temporary set-up memory (staging, ordering buffers) comes from a memory pool the library
 * owns on each device; memory freed back to that pool stays reserved (its high-water mark,
 * about 40 bytes per training entry) until the process exits, so later set-ups reuse it. */
int snect_init(snect_ctx **out, const snect_config *cfg, const int32_t *idx, const float *val,
               int64_t nnz, const int32_t *edges, const float *w, int64_t m, const float *G0,
               const float *U1, const float *U2, const float *U3, void *stream);

/* Runs n_epochs epochs of Alg. 1 lines 2-14: the entry sweep (every batch in order, or the
 * fast sweep) followed by one network pass over the gene factor, each epoch one launch of a
 * CUDA graph that snect_init captured (captured again after a change of timing mode).
 * Asynchronous. */
int snect_epoch(snect_ctx *ctx, int32_t n_epochs);

/* Deterministic mode only: runs mini-batches [first, first+count) of the visit order
 * (Alg. 1 lines 4-8, each batch evaluated at its start parameters, contributions summed).
 * Asynchronous. */
int snect_batches(snect_ctx *ctx, int64_t first, int64_t count);

/* One network pass over the gene factor (Alg. 1 line 10, every edge applied to both of its
 * endpoints; each gene row walks its neighbours in ascending order against the snapshot of
 * the factor taken when the pass starts).  Asynchronous. */
int snect_edge_pass(snect_ctx *ctx);

/* Objective terms and RMSE (Eq. 3, Sec. 2.3.2, graph regulariser; f_opt = f + lambda_g f_g).
 * test_idx/test_val: any, n_test held-out entries (may be 0); read in place from device
 * memory, copied otherwise.  Predictions are FP32, squared residuals summed in compensated
 * FP32 per thread and in FP64 beyond.  Synchronises.  Errors: SNECT_EINVAL for a test entry
 * with an index outside the tensor or a non-finite value (the context stays usable);
 * SNECT_ETIMEDOUT when a completion wait of an earlier fast-mode sweep gave up. */
int snect_loss(snect_ctx *ctx, const int32_t *test_idx, const float *test_val, int64_t n_test,
               snect_loss_t *out);

/* Copies the current core and factors out to / in from any memory (layouts above). */
int snect_get_factors(snect_ctx *ctx, float *G, float *U1, float *U2, float *U3);
int snect_set_factors(snect_ctx *ctx, const float *G, const float *U1, const float *U2,
                      const float *U3);

/* Fold-in of one new patient (Eq. 9), holding G, U2, U3 fixed: with w_jk = G x2 u2_j x3 u3_k,
 * u = (sum w w^T + lambda I)^{-1} sum x w over the query's n observed (gene, platform) cells.
 * The J1 x J1 Gram and right-hand side are summed in FP32 on the GPU in a fixed order and
 * solved by an FP64 Cholesky factorisation.  jk: any, n*2 int32; val: any, n float;
 * u_out: any, J1 floats.  Returns SNECT_EINVAL if n < 1, a cell lies outside the I2 x I3
 * table or a value is not finite (checked as the Gram kernel stages the cells), or the system
 * is not positive definite.  Synchronises. */
int snect_foldin(snect_ctx *ctx, const int32_t *jk, const float *val, int64_t n, float *u_out);

/* Top-k search (Sec. 3.2.1): the k rows of U1 with the largest cosine similarity to u
 * (J1 floats, any), descending, ties to the lower row index, a zero-norm row scores 0.
 * idx_out (int32) / score_out (float): any, k each.  1 <= k <= min(I1, 64).  Synchronises. */
int snect_topk(snect_ctx *ctx, const float *u, int32_t k, int32_t *idx_out, float *score_out);

/* Continuous-batching service of fold-in + top-k queries (Eq. 9 and Sec. 3.2.1 on a stream
 * of new patients).  snect_serve_start builds the (gene, platform) table of the frozen factors,
 * one device arena of exactly mem_budget_bytes, and n_slots slots (a CUDA stream, pinned host
 * staging for max_cells cells, and small fixed device buffers: the fold-in row, I1 scores and
 * flags, the top-k).  A scheduler thread admits queued requests oldest first whenever a slot
 * is free and the request's device memory -- its cells and its Gram partials, 256-byte aligned:
 * about 12 n + 4 ceil(n / 256) (J1^2 + J1) bytes for n cells -- can be carved out of the arena;
 * so the requests in flight never hold more device memory than the budget.  Admitted requests
 * run concurrently on their slots' streams; a host callback on each slot's stream hands the
 * finished request back to the scheduler.  A request's result does not depend on what else is
 * running.  While a server runs, the context must not be trained or have its factors set.
 * Errors: SNECT_EINVAL (sizes, budget below one largest request), SNECT_ENOMEM. */
typedef struct snect_server snect_server;
int snect_serve_start(snect_ctx *ctx, int32_t n_slots, int64_t mem_budget_bytes, int32_t max_cells,
                      snect_server **out);
/* Queues one query: jk (host, n*2 int32 (gene, platform)), val (host, n floats) are copied
 * into a pinned buffer from the server's pool (four per slot); when all are in use the call
 * waits for one to come back, up to 100 ms (SNECT_SERVE_PIN_WAIT_MS in the environment at
 * snect_serve_start), then keeps its own copy.  1 <= n <= max_cells, 1 <= k <= min(I1, 64).
 * Thread-safe.  *ticket identifies the result. */
int snect_serve_submit(snect_server *srv, const int32_t *jk, const float *val, int64_t n, int32_t k,
                       int64_t *ticket);
/* Result of a ticket: u_out (J1 floats), idx_out / score_out (k each), latency_ms (submit to
 * completion, host clock); any output pointer may be NULL.  wait = 0 returns SNECT_EBUSY if
 * the request has not finished.  Each ticket's result is returned once.  Thread-safe. */
int snect_serve_poll(snect_server *srv, int64_t ticket, int32_t wait, float *u_out, int32_t *idx_out,
                     float *score_out, double *latency_ms);
/* Counters: requests admitted and completed so far, and the most requests in flight at once. */
int snect_serve_stats(snect_server *srv, int64_t *admitted, int64_t *completed, int64_t *max_concurrent);
/* Finishes every queued request, stops the scheduler and frees the slots. */
int snect_serve_stop(snect_server *srv);

/* QR orthogonalisation post-pass (Alg. 1, the step after the sweeps): for each mode n with
 * J_n <= I_n, U^(n) = Q R (thin QR, R with a positive diagonal), U^(n) <- Q, G <- G x_n R, so
 * every prediction x~ is unchanged.  Computed as Cholesky-QR applied twice with FP64 Gram
 * matrices.  A mode with J_n > I_n keeps its factor; its bit (1 << n) is set in
 * *skipped_modes (may be NULL).  Synchronous.  Errors: SNECT_EINVAL (null context, or a
 * rank-deficient factor: its Gram matrix is not positive definite), SNECT_ECUDA. */
int snect_qr_post(snect_ctx *ctx, int32_t *skipped_modes);

/* Batched form: several independent decompositions (e.g. per-cohort sub-tensors, each fitted
 * for several lambda_g) stepped together.  ctxs: n fast-mode contexts with the same core ranks,
 * the same number of waves and the same sweep (SNECT_FP32, or SNECT_BF16 at 16 x 16 x 5; not
 * the tensor-core form); a batch does not own them, they must outlive it.  One epoch of the
 * batch is one CUDA graph: per wave, one sweep launch over every problem (each CTA serves one
 * problem, the CTAs allotted in proportion to the problems' entries) and one launch of every
 * problem's wave-end steps, then every problem's network pass.  The first snect_batch_epoch
 * autotunes the sweep launch (CTAs per SM, CTAs per resident slot, fewest entries per warp) by
 * timing wave 0 of every
 * candidate at the current parameters, then clears what those trial sweeps accumulated and
 * puts back the curvature state their pre-work rewrote, so the batch steps every problem as
 * its own epochs would.  Each context then holds its own updated factors (snect_loss,
 * snect_get_factors).
 * stream: a cudaStream_t or NULL (default stream); snect_batch_epoch is asynchronous.
 * Errors: SNECT_EINVAL (mismatched contexts), SNECT_ECUDA; messages through
 * snect_batch_last_error (NULL: the last failing snect_batch_create). */
typedef struct snect_batch snect_batch;
int snect_batch_create(snect_batch **out, snect_ctx *const *ctxs, int32_t n, void *stream);
int snect_batch_epoch(snect_batch *batch, int32_t n_epochs);
/* The autotuner's choice (zeros before the first epoch): resident tile CTAs per SM, tile CTAs
 * launched per resident slot (above 1, each CTA takes a smaller share and fewer problems are
 * in flight at once), fewest entries per warp (0: no floor), and that configuration's sweep
 * time on wave 0 in ms.  Host pointers, each may be NULL. */
int snect_batch_tuning(const snect_batch *batch, int32_t *ctas_per_sm, int32_t *oversubscription,
                       int32_t *min_entries_per_warp, double *sweep_ms);
/* kernels the batch has launched so far (its graphs' kernel nodes) */
int64_t snect_batch_launch_count(const snect_batch *batch);
const char *snect_batch_last_error(const snect_batch *batch);
void snect_batch_destroy(snect_batch *batch);

/* Fold-in that allocates nothing, for callers that cannot call cudaMalloc (a process that
 * lives inside another framework's memory budget or allocator, a serving loop that must not
 * stall on the allocator, code that keeps every device buffer pre-reserved).  The paper has
 * no counterpart: this is snect_foldin's computation without a context.
 *   G, U2, U3  device, the frozen core and gene / platform factors (layouts above)
 *   jk, val    device, the query's n cells ((gene, platform) int32 pairs) and values
 *   u_out      device, J1 floats
 *   stream     a cudaStream_t, or NULL for the default stream; the call synchronises it.
 * Its only working memory is a fixed device array inside the library (about 1 MiB, reserved
 * on every GPU that loads the library until the process exits), which bounds the query at
 * n <= 1,048,576 cells; larger queries return SNECT_EINVAL before any work is queued.  The
 * first call on each device does a one-time set-up with that device current (it looks up the
 * array's address and raises one kernel's shared-memory limit so that every core up to
 * J1*J2*J3 = 5,120 fits).  Each call ends by copying two status words to the host and
 * synchronising the stream, so no call can be captured into a CUDA graph.  Calls share
 * the array, so two calls whose work overlaps on the GPU (from different streams or threads)
 * race; serialise them.  Errors: SNECT_EINVAL for bad sizes, an out-of-range cell, a
 * non-finite value or a system that is not positive definite; on those two device-side
 * errors u_out holds J1 zeros.  Messages through snect_last_error(NULL). */
int snect_foldin_static(const float *G, const float *U2, const float *U3, int32_t I2, int32_t I3,
                        int32_t J1, int32_t J2, int32_t J3, const int32_t *jk, const float *val,
                        int64_t n, float lambda, float *u_out, void *stream);

/* Personalised subtype analysis (Sec. 3.3) of n patient profiles u (any, n*J1 floats, e.g.
 * rows of U1 or fold-in results): per profile the subtype matrix S = G x1 u (J2 x J3),
 * S[q][r] = sum_p g_pqr u_p; row_norm[q] = ||S[q][:]|| (the weight of gene-mode subtype q);
 * platform_norm[k] = the norm of column k of S x3 U3, (S x3 U3)[q][k] = sum_r S[q][r] U3[k][r]
 * (the weight of platform k).  S: any, n*J2*J3 floats; row_norm: any, n*J2; platform_norm: any,
 * n*I3; each may be NULL.  FP32, fixed summation order.  All profiles in one launch.
 * Synchronises.  Errors: SNECT_EINVAL, SNECT_ECUDA. */
int snect_subtype(snect_ctx *ctx, const float *u, int64_t n, float *S, float *row_norm, float *platform_norm);

/* Stratification of the patients (Sec. 3.1.1): k-means with Euclidean distance on the rows of
 * U1, by Lloyd's iterations from the initial centroids init (any, k*J1 doubles).  A pass assigns
 * each row to its nearest centroid (squared distance, ties to the lower index); a pass that
 * changes no assignment ends the run; otherwise each centroid with rows moves to their mean
 * (one without rows stays).  At most max_iter passes.  The assignment is decided in FP64 with a
 * fixed operation order (per centroid, coordinates in order, no fused multiply-add) and each
 * centroid is its rows' sum in ascending row order divided by their count, so the result is
 * the one a sequential FP64 program with that order computes.
 *   assign     any, I1 int32: the last pass's clusters (or NULL)
 *   centroids  any, k*J1 doubles: the final centroids (or NULL)
 *   n_updates  host: centroid updates made (or NULL); inertia  host: sum over the rows of the
 *              squared distance to their assigned final centroid (or NULL)
 * 1 <= k <= min(I1, 128), max_iter >= 1.  Synchronises.  Errors: SNECT_EINVAL, SNECT_ECUDA. */
int snect_kmeans(snect_ctx *ctx, int32_t k, const double *init, int32_t max_iter, int32_t *assign,
                 double *centroids, int32_t *n_updates, double *inertia);

/* The lock-free form of Alg. 1 as the paper states it (Sec. 2.3.3), for comparison with the
 * fast mode: P workers walk one interleaved order of entries and network edges (order: any,
 * n_items int32; a value t < nnz is entry t of the visit order, t >= nnz is edge t - nnz);
 * worker w takes items w, w + P, w + 2P, ...  An entry updates its three rows by the per-entry
 * gradients of Sec. 2.3.2, read and applied without locks (atomic adds); only worker 0 steps
 * the core, with step lr * P (Alg. 1 line 8).  An edge moves both gene rows towards each other
 * (line 10).  With P = 1 this is Alg. 1 with one worker.  Runs n_epochs passes over the order
 * (no separate network pass).  Needs a deterministic-mode context (batch > 0), which keeps the
 * entries in the visit order.  Asynchronous after the order is checked.  Errors: SNECT_EINVAL
 * (mode, P < 1, an item out of range), SNECT_ECUDA. */
int snect_hogwild_epoch(snect_ctx *ctx, const int32_t *order, int64_t n_items, int32_t P, int32_t n_epochs);

/* Which entry-sweep launches of an epoch carry CUDA timing events (fast mode: one sweep
 * launch per wave; deterministic mode: the gradient kernel of each batch).  mode 0 (the
 * default): none; 1: one launch per epoch, the middle one; -1: every launch; 2: every launch
 * of every kernel of the epoch (the sweeps, the wave ends or deterministic apply kernels, the
 * network pass; read with snect_kernel_times).  Each timed launch adds two event nodes to
 * the epoch's CUDA graph, which cost the epoch several microseconds each, so timing is off
 * unless asked for.  A change takes effect at the next snect_epoch (the epoch graph is
 * captured again).  Errors: SNECT_EINVAL for another mode. */
int snect_set_sweep_timing(snect_ctx *ctx, int32_t mode);

/* Per-kernel device time of the most recent epoch under timing mode 2: ms[0] / n[0] the
 * entry-sweep launches, ms[1] / n[1] the wave-end steps (fast mode) or the apply kernels
 * (deterministic mode), ms[2] / n[2] the network pass; each the summed milliseconds between
 * CUDA events recorded on the context's stream immediately before and after each launch.
 * ms and n: host, 3 each.  All zero unless an epoch ran with mode 2.  Synchronises. */
int snect_kernel_times(snect_ctx *ctx, double *ms, int64_t *n);

/* Device time of the timed entry-sweep launches (snect_set_sweep_timing) of the most recent
 * epoch, measured with CUDA events recorded on the context's stream immediately before and
 * after each of them.  *ms_total = summed milliseconds, *n_launches = launches timed,
 * *n_entries (may be NULL) = training entries those launches processed.  All zero when no
 * epoch has run with timing on.  Synchronises. */
int snect_sweep_times(snect_ctx *ctx, double *ms_total, int64_t *n_launches, int64_t *n_entries);

/* Diagnostic of the fast sweep: what one wave's entry sweep accumulates before its end step.
 * Runs the sweep kernel of wave w alone, at the current parameters, in the launch
 * configuration an epoch uses, and copies out its accumulators: the summed data-term part of
 * the gradient equation (Sec. 2.3.2, as Alg. 1 lines 5-8 evaluate it per entry), all terms at
 * the wave-start parameters:
 *   gA  any, I1*J1 floats (or NULL): per patient row i, sum over the wave's entries of i of
 *       r (G x2 b_j x3 c_k), r = x~ - x
 *   gB  any, I2*J2 floats (or NULL): per gene row j, sum of r (G x1 a_i x3 c_k)
 *   M   any, I3*J1*J2 floats (or NULL): per platform k, M_k[p][q] = sum over the wave's entries
 *       of platform k of r a_p b_q; the core's data-term gradient is sum_k M_k o c_k and
 *       platform row k's is G_(3) vec(M_k)
 *   nA  any, I1*I3 floats (or NULL): the wave's entries per (patient, platform); nB likewise
 *       I2*I3 per (gene, platform)
 *   first, count  (host, may be NULL): the wave's entries are positions [first, first+count)
 *       of the visit order given at snect_init
 * The factors and core are not changed, and the accumulators are cleared again afterwards;
 * the fast mode's curvature state (platform systems, eigenbases) is refreshed as the wave's
 * own sweep refreshes it.  Fast mode only.  Synchronises.  Errors: SNECT_EINVAL (mode, wave
 * index), SNECT_ETIMEDOUT (a completion wait of the sweep gave up), SNECT_ECUDA. */
int snect_wave_grads(snect_ctx *ctx, int64_t w, float *gA, float *gB, float *M, float *nA, float *nB,
                     int64_t *first, int64_t *count);

/* Number of kernel launches the context has issued so far (for launch accounting). */
int64_t snect_launch_count(const snect_ctx *ctx);

/* Message for the last failing call on ctx (or for the last failing snect_init if ctx is
 * NULL).  The string stays valid until the next call on the context. */
const char *snect_last_error(const snect_ctx *ctx);

/* Frees the context's device memory and graphs.  NULL is a no-op. */
void snect_destroy(snect_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SNECT_H */
