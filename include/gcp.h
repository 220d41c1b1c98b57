/*
 * gcp.h -- C ABI of the GB300 stochastic GCP gradient library (libgcp.so).
 *
 * The library computes the stochastic gradient of Generalized CP tensor
 * decomposition (Myers & Phipps, "Synchronous and Asynchronous Parallelism
 * Approaches for GCP Tensor Decomposition with GenTen"):
 *   1. stratified sampling of p nonzeros and q zeros (Sec. 3.1.1),
 *   2. the CP model entry m = sum_r prod_k A_k(i_k, r) at each sample (Eq. cp),
 *   3. the loss f(x, m) and its derivative f'(x, m) (Eq. gcp-model),
 *   4. the all-mode sampled MTTKRP G_n(i_n,:) += w f' prod_{k!=n} A_k(i_k,:)
 *      (Eq. gcp-gradient, fused with sampling as in Sec. 3.1.2),
 * plus the Adam update of Algorithm 1 and the epoch loop of Algorithm 2.
 * Everything runs on one GPU; there are no collectives.
 *
 * Conventions
 *  - Plain pointers and sizes only.  "device" pointers are CUDA device (or
 *    managed) memory of the current device; "host" pointers are CPU memory;
 *    "host or device" pointers are classified with unified addressing.
 *  - Input arrays are copied at creation; the caller keeps ownership of every
 *    pointer it passes.  The context owns its internal buffers.
 *  - All GPU work of a context runs on the stream given in gcp_options
 *    (a cudaStream_t passed as void*; NULL = the legacy default stream).
 *    Calls that return a host value synchronise that stream; the others are
 *    asynchronous and report device-side errors at the next synchronising
 *    call (gcp_sync, gcp_loss, or gcp_grad with a host loss pointer).
 *  - No exception crosses the ABI; every call returns a gcp_status and
 *    gcp_last_error() describes the last failure of a context.
 *  - Indices are 0-based.  Factor matrices and gradients are passed as one
 *    flat FP32 array: mode 0's I_0 x R matrix (row-major), then mode 1's, ...
 *    (the single contiguous array of Sec. 3.1.3).
 *  - The linear index of (i_0..i_{d-1}) is row-major, last mode fastest.
 *  - Samples are deterministic functions of (seed, iteration, p, q): sample
 *    j of a draw class uses Philox4x64-10 with key (seed, stream) and counter
 *    (j, sub, iteration, 0); stream 0 = nonzeros (word 0 mapped onto [0, N)),
 *    stream 1 = zero candidates (attempt a, modes 4b..4b+3 at sub = 4a + b),
 *    stream 2 = dense uniform cells, stream 3 = semi-stratified zero
 *    candidates; a 64-bit word u maps onto [0, n) as floor(u n / 2^64).
 */
#ifndef GCP_H
#define GCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GCP_MAX_NDIM 8
#define GCP_MAX_RANK 128
/* Iteration number whose sample set is the fixed objective-estimate set
 * used by gcp_fit (Sec. 5.1: a fixed number of objective samples). */
#define GCP_ITER_OBJECTIVE 0xFFFFFFFFFFFFFFFFull

typedef enum {
    GCP_OK = 0,
    GCP_ERR_ARG = 1,               /* invalid argument (checked on the host)        */
    GCP_ERR_OOM = 2,               /* device allocation failed                      */
    GCP_ERR_CUDA = 3,              /* a CUDA runtime call failed                    */
    GCP_ERR_DUPLICATE = 4,         /* two nonzeros share one coordinate tuple       */
    GCP_ERR_HASH_FULL = 5,         /* nonzero hash set could not place a key        */
    GCP_ERR_SAMPLER_EXHAUSTED = 6, /* a zero draw hit nonzeros max_attempts times   */
    GCP_ERR_NONFINITE = 7,         /* loss or gradient became NaN/Inf               */
    GCP_ERR_DOMAIN = 8,            /* data outside the loss's domain                */
    GCP_ERR_STATE = 9              /* call not valid for this context               */
} gcp_status;

typedef enum {
    GCP_GAUSSIAN = 0,        /* f = (x-m)^2,               f' = 2(m-x)                 */
    GCP_POISSON = 1,         /* f = m - x log(m+eps),      f' = 1 - x/(m+eps)          */
    GCP_BERNOULLI_LOGIT = 2, /* f = log(1+e^m) - x m,      f' = e^m/(1+e^m) - x        */
    GCP_GAMMA = 3            /* f = x/(m+eps) + log(m+eps), f' = 1/(m+eps) - x/(m+eps)^2 */
} gcp_loss_t;                /* eps = 1e-10; losses of the GCP source the paper cites */

typedef enum { GCP_FP32 = 0, GCP_BF16 = 1 } gcp_factor_dtype;

typedef enum {
    GCP_MTTKRP_ATOMIC = 0,       /* fused scatter with FP32 vector atomics (Sec. 3.1.2) */
    GCP_MTTKRP_DETERMINISTIC = 1, /* sort by row + segmented sums, bit-stable run to run;
                                     grows a scratch buffer for the largest sample count
                                     S = p + q seen: a 16, 32 or 64 B record per sample, 16 B
                                     per sample and mode for the modes sorted side by side
                                     (as many as fit 1 GiB, at least one), 8 x padded rank B
                                     per 64 samples, and small counts; GCP_ERR_OOM if it
                                     cannot.  It also creates a second stream for its sort
                                     on first use, so make the first call with the largest
                                     sample count outside stream capture */
    GCP_MTTKRP_NONFUSED = 2       /* sampling writes the gradient tensor, then a separate
                                     atomic MTTKRP reads it (the unfused form of Sec. 3.1.2) */
} gcp_mttkrp_t;

typedef enum {
    GCP_SAMPLING_STRATIFIED = 0,      /* zeros by rejection against the nonzeros (Sec. 3.1.1) */
    GCP_SAMPLING_SEMI_STRATIFIED = 1, /* zeros without search, nonzero value f'(x,m)-f'(0,m)  */
    GCP_SAMPLING_UNIFORM = 2          /* dense tensors: p uniform cells, weight M/p          */
} gcp_sampling_t;

typedef struct {
    int32_t factor_dtype; /* gcp_factor_dtype: storage of the factors the kernels read     */
    int32_t mttkrp;       /* gcp_mttkrp_t                                                  */
    int32_t sampling;     /* gcp_sampling_t (sparse: stratified or semi; dense: uniform)   */
    int32_t max_attempts; /* zero-draw rejection cap; 0 selects 64                        */
    uint64_t seed;        /* Philox key word 0                                             */
    void *stream;         /* cudaStream_t for all work of the context; NULL = default     */
    double hash_max_load; /* nonzero hash set load bound in (0, 0.5]; 0 selects 0.3        */
    int32_t lane_cols;    /* factor columns per GPU lane: 4 or 8; 0 picks 4 for rank <= 32 */
    int32_t reserved;
} gcp_options;

typedef struct {
    double lr;     /* alpha                                   */
    double beta1;  /* beta_1                                  */
    double beta2;  /* beta_2                                  */
    double eps;    /* epsilon inside the square root (Alg. 1) */
    double lower;  /* lower bound l; -INFINITY for none       */
} gcp_adam_params;

typedef struct {
    gcp_adam_params adam;
    int64_t p, q;          /* gradient samples per iteration (nonzero, zero)           */
    int64_t p_obj, q_obj;  /* objective-estimate samples (fixed set)                   */
    int32_t iters;         /* iterations per epoch                                     */
    int32_t max_epochs;
    int32_t max_fails;     /* stop after this many epochs that failed to decrease F    */
    int32_t reserved;
    double decay;          /* lr *= decay after a failed epoch (state restored)        */
    uint64_t iter0;        /* iteration number of the first gradient                   */
} gcp_fit_params;

#define GCP_FIT_TRACE 256
typedef struct {
    int32_t epochs;             /* epochs run                                   */
    int32_t fails;              /* failed epochs                                */
    int64_t iterations;         /* accepted gradient steps (Adam t)             */
    double objective0;          /* objective estimate before the first epoch    */
    double objective;           /* final objective estimate                     */
    double lr;                  /* final learning rate                          */
    double seconds;             /* wall time of the fit                         */
    double grad_samples_per_s;  /* (p+q) x iterations / seconds                 */
    double attempts_per_zero;   /* mean rejection attempts per zero sample       */
    double trace[GCP_FIT_TRACE];/* objective after each epoch                   */
} gcp_fit_report;

typedef struct gcp_ctx gcp_ctx;
typedef struct gcp_batch gcp_batch;

/* Fill *opt with the defaults: FP32 factors, atomic MTTKRP, stratified
 * sampling, 64 attempts, seed 0, default stream, load 0.3, lane_cols 0. */
void gcp_options_default(gcp_options *opt);

/* Create a context for a sparse tensor (Sec. 3.1.1: COO list of N tuples and
 * N values).  dims[ndim] (host) are the mode sizes, prod(dims) < 2^63;
 * coords (host, nnz x ndim int32, row-major) and vals (host, nnz float) are
 * the nonzeros, which must be distinct and in range.  rank in 1..128.  The
 * context copies the nonzeros into packed device records and a device hash
 * set of their linear indices.  Factors start at zero; set them with
 * gcp_set_factors.  Errors: GCP_ERR_ARG (bad sizes, coordinate out of range,
 * non-finite value, unknown loss), GCP_ERR_DOMAIN (negative value for the
 * Poisson/Gamma losses, value not 0/1 for Bernoulli), GCP_ERR_DUPLICATE,
 * GCP_ERR_HASH_FULL, GCP_ERR_OOM, GCP_ERR_CUDA.  On error *out is NULL. */
gcp_status gcp_create(int32_t ndim, const int64_t *dims, int64_t nnz, const int32_t *coords,
                      const float *vals, int32_t rank, int32_t loss, const gcp_options *opt,
                      gcp_ctx **out);

/* Create a context for a dense tensor X (host or device, prod(dims) floats,
 * row-major, last mode fastest).  Sampling is uniform over all cells with
 * weight M/p (the stochastic gradient of Sec. 3.1.1 with Y sampled
 * uniformly); q must be 0 in the sampling calls.  X is copied, and its
 * values are checked on the device as gcp_create checks nonzeros:
 * GCP_ERR_ARG for a non-finite value, GCP_ERR_DOMAIN for a value outside
 * the loss's domain; also GCP_ERR_OOM, GCP_ERR_CUDA.  On error *out is NULL. */
gcp_status gcp_create_dense(int32_t ndim, const int64_t *dims, const float *X, int32_t rank,
                            int32_t loss, const gcp_options *opt, gcp_ctx **out);

/* Release every resource of the context (synchronises its stream). NULL ok. */
void gcp_destroy(gcp_ctx *ctx);

/* Last error message of the context (or, when ctx is NULL, of the last
 * failed call of this thread that has no context); never NULL; valid until
 * the next call on that context. */
const char *gcp_last_error(const gcp_ctx *ctx);

/* Shape queries. */
int32_t gcp_ndim(const gcp_ctx *ctx);
int32_t gcp_rank(const gcp_ctx *ctx);
int64_t gcp_nnz(const gcp_ctx *ctx);
/* Number of factor entries sum_k I_k * R (the flat length of A and G). */
int64_t gcp_num_params(const gcp_ctx *ctx);

/* Set all factors from A (host or device, flat FP32, see Conventions).  With
 * BF16 storage the BF16 copy the kernels read is refreshed (round to nearest
 * even) from the FP32 master.  Adam moments are not touched. */
gcp_status gcp_set_factors(gcp_ctx *ctx, const float *A);
/* Set one mode's factor matrix (host or device, I_mode x R FP32). */
gcp_status gcp_set_factor(gcp_ctx *ctx, int32_t mode, const float *A_mode);
/* Set every mode's factor matrix in one call: A_modes (host array of ndim
 * pointers) points to the per-mode matrices (host or device, I_k x R FP32,
 * row-major, each contiguous).  Asynchronous on the context's stream: the
 * matrices must stay valid until the stream has consumed them; the pointer
 * array itself is read before the call returns.  With BF16 storage the BF16
 * copy is refreshed once.  The paper has no counterpart (the autograd
 * binding stages its factor tensors with it). */
gcp_status gcp_set_factor_list(gcp_ctx *ctx, const float *const *A_modes);
/* Copy the FP32 master factors out (host or device, flat). Synchronises. */
gcp_status gcp_get_factors(gcp_ctx *ctx, float *A_out);
/* Zero the Adam moments. */
gcp_status gcp_reset_adam(gcp_ctx *ctx);

/* Draw the sample set of iteration `iter` (Sec. 3.1.1) without evaluating
 * anything: samples 0..p-1 are nonzeros (weight N/p), p..p+q-1 zeros
 * (weight (M-N)/q; semi-stratified: M/q; dense: p uniform cells, weight
 * M/p).  idx_out (device, (p+q) x ndim int32), x_out (device, p+q float)
 * and w_out (device, p+q float) may each be NULL.  Asynchronous; an
 * exhausted zero draw sets GCP_ERR_SAMPLER_EXHAUSTED, reported by gcp_sync,
 * and leaves that sample's coordinates at the last candidate. */
gcp_status gcp_sample(gcp_ctx *ctx, uint64_t iter, int64_t p, int64_t q, int32_t *idx_out,
                      float *x_out, float *w_out);
/* All sampling calls take p, q >= 0 with p + q < 2^31 (GCP_ERR_ARG otherwise). */

/* Sampled loss estimate F~ = sum_s w_s f(x_s, m_s) of iteration `iter`
 * (Eq. gcp-model on the stratified sample), reduced in FP64, written to the
 * host double *loss_out.  Synchronises; returns any pending device error. */
gcp_status gcp_loss(gcp_ctx *ctx, uint64_t iter, int64_t p, int64_t q, double *loss_out);

/* Same as gcp_loss, asynchronously, into device memory dloss_out[0]. */
gcp_status gcp_loss_async(gcp_ctx *ctx, uint64_t iter, int64_t p, int64_t q, double *dloss_out);

/* Sampled gradient of iteration `iter`: the context's gradient buffer is
 * zeroed and receives G_n(i_n,:) += w f'(x,m) prod_{k!=n} A_k(i_k,:) for all
 * modes in one fused pass (Sec. 3.1.2).  If G_out (device, flat FP32) is not
 * NULL the gradient is also copied there.  If loss_out (host) is not NULL
 * the sampled loss is written there and the call synchronises. */
gcp_status gcp_grad(gcp_ctx *ctx, uint64_t iter, int64_t p, int64_t q, float *G_out,
                    double *loss_out);

/* Asynchronous gradient: as gcp_grad, but the gradient is multiplied by
 * dscale[0] (device float, NULL = 1) and the loss goes to device memory
 * dloss_out[0] (NULL = not computed).  Used by the autograd binding. */
gcp_status gcp_grad_async(gcp_ctx *ctx, uint64_t iter, int64_t p, int64_t q, const float *dscale,
                          float *G_out, double *dloss_out);

/* Stage every mode's factor matrix and run the fused pass, in one call (the
 * autograd binding's forward evaluation; the paper has no counterpart).
 * A_modes (host array of ndim pointers) points to the per-mode matrices,
 * I_k x R FP32 row-major, each contiguous, in device memory of the
 * context's device or in managed memory (GCP_ERR_ARG otherwise); they are
 * copied into the context by one kernel
 * (with the BF16 copy refreshed), asynchronously on the context's stream,
 * so they must stay valid until the stream has consumed them.  Then, as
 * gcp_grad_async with dscale NULL: the sampled loss of iteration `iter` to
 * dloss_out[0] (device, nullable) and, if G_out (device, flat FP32) is not
 * NULL, the sampled gradient there; with G_out NULL only the loss is formed
 * (as gcp_loss_async).  Asynchronous. */
gcp_status gcp_grad_factors_async(gcp_ctx *ctx, const float *const *A_modes, uint64_t iter, int64_t p, int64_t q,
                                  float *G_out, double *dloss_out);

/* y[i] = (float)dscale[0] * x[i] for i < n, on the context's stream.
 * dscale (one FP64 value, as the FP64 loss's incoming gradient is), x and y
 * are device pointers (y may equal x); nothing is allocated.  The paper has
 * no counterpart: the autograd binding computes the loss and the gradient
 * in one fused pass in the forward evaluation and applies the incoming
 * gradient in the backward evaluation with this call.
 * GCP_ERR_ARG for a NULL pointer or n < 0. */
gcp_status gcp_scale_async(gcp_ctx *ctx, const double *dscale, const float *x, float *y, int64_t n);

/* Frobenius norm of the gradient the context holds (after gcp_grad or
 * gcp_grad_async; zero after gcp_step, which clears it), summed in FP64 on
 * the device in a fixed order, so that repeated calls agree bit for bit;
 * *norm_out (host) receives it.  GCP_ERR_NONFINITE if the gradient holds a
 * NaN or an infinity.  Synchronises the context's stream.  The paper has no
 * counterpart: it is the FP64 check kept beside the FP32 / BF16 path. */
gcp_status gcp_grad_norm(gcp_ctx *ctx, double *norm_out);

/* One Adam step (Algorithm 1, one kernel over the flat parameter vector,
 * Sec. 3.1.3) with the gradient held by the context, t >= 1. */
gcp_status gcp_adam_step(gcp_ctx *ctx, const gcp_adam_params *prm, int64_t t);

/* One training step (Algorithm 2's iteration on one GPU): the sampled
 * gradient of iteration `iter` (as gcp_grad) followed by Adam step t (as
 * gcp_adam_step).  With the atomic MTTKRP the step is two launches: the
 * fused pass, then one epilogue that finishes the loss, folds the hot-row
 * replicas, applies Adam and clears the gradient for the next step -- so
 * after gcp_step the context's gradient buffer is zero, not the step's G.
 * dloss_out (device, nullable) receives the sampled loss.  Asynchronous. */
gcp_status gcp_step(gcp_ctx *ctx, uint64_t iter, int64_t p, int64_t q, const gcp_adam_params *prm, int64_t t,
                    double *dloss_out);

/* Wait for the context's stream and return (and clear) any device error. */
gcp_status gcp_sync(gcp_ctx *ctx);

/* GCP-Adam (Algorithm 2 on one GPU): epochs of `iters` gradient + Adam
 * steps, each followed by the objective estimate on the fixed sample set
 * GCP_ITER_OBJECTIVE; an epoch that does not decrease it is undone (factors,
 * moments and t restored) and lr *= decay; stop after max_fails such epochs
 * or max_epochs.  report may be NULL. */
gcp_status gcp_fit(gcp_ctx *ctx, const gcp_fit_params *prm, gcp_fit_report *report);

/* Kernel timing (the per-phase runtime breakdown of Sec. 5.1, on one GPU).
 * While enabled, every launch of the fused sampling/model/loss/MTTKRP kernel
 * on the context's stream is bracketed by CUDA events on that stream.
 * gcp_profile_read synchronises, returns the summed kernel milliseconds and
 * the launch count since the last read, and clears them.  Disabled by
 * default; enabling costs two event records per launch. */
gcp_status gcp_profile(gcp_ctx *ctx, int32_t enable);
gcp_status gcp_profile_read(gcp_ctx *ctx, double *kernel_ms, int64_t *launches);

/* ---- Batched independent subproblems (the client shards of the federated
 * schemes, Alg. 3 and Alg. 4, simulated on one GPU) ----
 * A batch advances many contexts ("clients") together: one local step runs,
 * for every client c, the sampled gradient of p[c] nonzero and q[c] zero
 * samples followed by its own Adam update, with one multi-client launch per
 * kernel; tau local steps are captured once in a CUDA graph and replayed. */

/* Create a batch over nclients existing sparse contexts (kept by the caller,
 * who must not destroy them before the batch).  They must share order, rank,
 * loss, factor dtype, device and stream, use the atomic MTTKRP and
 * stratified or semi-stratified sampling.  p, q (host, nclients): samples per
 * local step of each client, p[c] + q[c] < 2^31.  The batch works on its own
 * stream, ordered after and before the clients' stream with events. */
gcp_status gcp_batch_create(int32_t nclients, gcp_ctx *const *clients, const int64_t *p, const int64_t *q,
                            gcp_batch **out);
void gcp_batch_destroy(gcp_batch *batch);
const char *gcp_batch_last_error(const gcp_batch *batch);

/* Tuning knobs of the multi-client fused kernel: factor columns per lane (4
 * or 8; 0 = the clients' choice) and the number of thread blocks of the
 * persistent grid (0 = all that fit on the GPU at once).  A change rebuilds
 * the graph at the next gcp_batch_local_steps. */
gcp_status gcp_batch_tune(gcp_batch *batch, int32_t lane_cols, int32_t blocks);

/* Tuning knob of the multi-client fused kernel: samples per warp tile (16,
 * 32 or 64; 0 = 32).  A warp stages a tile's samples (one, or for 64 two,
 * per lane; for 16 only half its lanes) and then evaluates them; smaller
 * tiles spread a step over more warps, larger ones keep more sample loads
 * in flight per warp.  The grid size follows the new tile size's occupancy
 * unless gcp_batch_tune set it explicitly.  A change rebuilds the graph at
 * the next gcp_batch_local_steps; results do not depend on the tile size
 * beyond the FP32 summation order.  GCP_ERR_ARG for other sizes. */
gcp_status gcp_batch_tune_tile(gcp_batch *batch, int32_t samples_per_warp);

/* tau local steps of every client: step k (0-based) samples iteration
 * iter0 + k and applies Adam step t0 + k + 1 (Alg. 1) with prm.  Each client
 * ends with the same state as tau rounds of gcp_grad + gcp_adam_step on its
 * own context, up to the summation order of the atomic MTTKRP.  A step is
 * four launches in the graph: gradients cleared, the multi-client fused
 * pass, one epilogue (loss finish, replica fold, Adam) and a counter advance.
 * Asynchronous on the clients' stream; back-to-back calls need no sync. */
gcp_status gcp_batch_local_steps(gcp_batch *batch, int32_t tau, const gcp_adam_params *prm, uint64_t iter0,
                                 int64_t t0);

/* Sampled loss of every client's last local step (host, nclients doubles).
 * Synchronises; returns any pending device error of a client. */
gcp_status gcp_batch_losses(gcp_batch *batch, double *loss_out);

/* GCP-FedAdam reconciliation (Alg. 4) for a batch whose clients are shards
 * of one model (identical mode sizes).  The batch keeps the server model U
 * and its Adam moments.
 * gcp_batch_server_init: U = client 0's factors, server moments cleared,
 *   every client's factors set to U.
 * gcp_batch_server_step: the pseudo-gradient D = U - M_c, all-reduced as the
 *   mean over clients (summed in client order), updates U with Adam
 *   (Algorithm 1, hyperparameters prm -- its lr is the meta-rate -- and
 *   server step t >= 1); then every client's factors are set to U (M <- U).
 *   The clients' own Adam moments are kept.
 * Both are asynchronous on the clients' stream; GCP_ERR_STATE before init,
 * GCP_ERR_ARG for clients of different shapes. */
gcp_status gcp_batch_server_init(gcp_batch *batch);
gcp_status gcp_batch_server_step(gcp_batch *batch, const gcp_adam_params *prm, int64_t t);

/* Sampled loss and gradient of a caller-supplied sample list, allocating
 * nothing.  The paper has no counterpart: it exists for callers that cannot
 * allocate device memory -- code that runs under a device-memory budget
 * fixed at start-up, such as a host framework that owns every allocation
 * through its own pool, or a long-running service that must not grow its
 * footprint.  The caller passes every input and output; the only scratch
 * (one loss partial per block of 2048 samples) is a file-scope device array
 * of the library, 128 KB, held by every GPU that loads the library until the
 * process exits.  No cudaMalloc, cudaFree or allocating library routine is
 * called.
 *   dims[ndim] (host) mode sizes; rank 1..128; loss a gcp_loss_t;
 *   idx (device, nsamples x ndim int32 row-major), x and w (device, nsamples
 *   floats): sample s is cell idx[s], value x[s], weight w[s];
 *   A (device, flat FP32 factors, see Conventions, unpadded rank columns);
 *   G (device, same layout, overwritten) receives
 *     sum_s w_s f'(x_s, m_s) prod_{k!=n} A_k(i_k,:) in each mode's rows;
 *   loss_out (device, 2 doubles): [0] = sum_s w_s f(x_s, m_s) (FP64, fixed
 *   order), [1] = samples skipped because a coordinate was out of range;
 *   stream a cudaStream_t (NULL = default stream).
 * nsamples may be at most GCP_NOALLOC_MAX_SAMPLES; larger counts are
 * rejected with GCP_ERR_ARG (message from gcp_last_error(NULL)) and must be
 * split over several calls.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Every call on a device
 * shares the array: calls whose kernels overlap on the GPU race and must be
 * ordered by the caller (one stream, or events).  Asynchronous: the call
 * returns before any result exists, so a NaN or infinite loss is not a
 * status code here; the caller reads loss_out[0] after the stream. */
#define GCP_NOALLOC_MAX_SAMPLES 16777216LL
gcp_status gcp_grad_samples_noalloc(int32_t ndim, const int64_t *dims, int32_t rank, int32_t loss,
                                    int64_t nsamples, const int32_t *idx, const float *x, const float *w,
                                    const float *A, float *G, double *loss_out, void *stream);

/* Measured ceiling of the L2-resident row traffic (measurement support; the
 * paper has no counterpart).  The fused pass's factor gathers and gradient
 * reductions hit rows that stay in L2, so its binding limit is the SM -> L2
 * path.  This call moves rows of buf in the same pattern and nothing else:
 * ops operations, each by one group of row_floats/4 lanes, on rows_per_op
 * uniformly random rows (splitmix64 of the op index):
 *   GCP_PROBE_RED  adds a 16-byte slice per lane to each row
 *                  (red.global.add.v4.f32, the atomic MTTKRP's scatter);
 *   GCP_PROBE_LOAD reads each row with 16-byte vector loads (the gathers);
 *   GCP_PROBE_BOTH reads rows_per_op rows, then adds to rows_per_op others.
 * buf (device, caller-owned, 16-byte aligned, rows x row_floats floats,
 * finite values) is modified by the RED and BOTH kinds with additions below
 * 1e-29 per element.  row_floats a power of two in 4..128; rows_per_op in
 * 1..8.  The caller times the call with events on `stream`.  GCP_ERR_ARG for
 * bad sizes (message from gcp_last_error(NULL)).  Asynchronous. */
#define GCP_PROBE_RED 0
#define GCP_PROBE_LOAD 1
#define GCP_PROBE_BOTH 2
gcp_status gcp_probe_l2(int32_t kind, int32_t row_floats, int32_t rows_per_op, float *buf, int64_t rows,
                        int64_t ops, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GCP_H */
