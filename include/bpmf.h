/*
 * bpmf.h -- C ABI of the GB300 BPMF Gibbs sampler (one chain on one GPU).
 *
 * The method is Bayesian Probabilistic Matrix Factorization by Gibbs sampling
 * as laid out in Alg. 1 of arXiv:1705.10633 (Sec. 2): per sweep, sample the
 * movie hyper-parameters from V, update every movie, sample the user
 * hyper-parameters from U, update every user, then predict the test points and
 * compute the RMSE.  The per-item update (Sec. 2; Sec. 3.1) forms the K x K
 * precision from the other side's vectors of the item's ratings, factors it by
 * Cholesky instead of inverting it, and draws the item's new vector.
 *
 * Conventions shared by every entry point:
 *   - Return value: BPMF_OK (0) or a negative BPMF_E* code; bpmf_strerror()
 *     names it.  No entry point aborts the process.
 *   - Pointers named host_* or documented as host memory are read (or written)
 *     only during the call; the caller keeps ownership.  Device memory the
 *     library needs is owned by the handle and released by bpmf_destroy().
 *   - A handle is not thread-safe.  Work is ordered on the CUDA stream given to
 *     bpmf_create(); calls that return host values synchronise that stream.
 *   - Matrices are row-major.  U is M x K (users = rows of R), V is N x K
 *     (movies = columns of R); K <= 64.
 *   - Ratings: CSR (users) with int64 row pointers, int32 column indices and
 *     FP32 values.  Columns inside a row may be in any order.
 */
#ifndef BPMF_H
#define BPMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------- */
#define BPMF_OK 0
#define BPMF_EINVAL -1   /* bad argument: dims, K > 64, malformed CSR/CSC, ... */
#define BPMF_ENOMEM -2   /* device or host allocation failed                  */
#define BPMF_ECUDA -3    /* a CUDA runtime call failed                        */
#define BPMF_ENOTPD -4   /* a precision matrix had a non-positive pivot       */
#define BPMF_ETIMEOUT -5 /* a bounded device wait gave up                     */
#define BPMF_ENAN -6     /* a NaN/Inf was produced                            */
#define BPMF_EGAMMA -7   /* the gamma sampler exhausted its attempts          */

/* ---- flags (bpmf_params.flags) ----------------------------------------- */
#define BPMF_BF16_GRAM 0x1u   /* tensor-core Gram from BF16 copies of the other side's
                                 rows (one 128-B row per rating instead of the FP16 hi/lo
                                 pair): half the gathered bytes, ~2^-8 relative error in
                                 the Gram; needs K in 49..64 without BPMF_CUDA_CORE_GRAM,
                                 else bpmf_create returns BPMF_EINVAL                     */
#define BPMF_CLIP 0x2u        /* clip predictions to [clip_lo, clip_hi]                   */
#define BPMF_DEBUG_MEANS 0x4u /* keep each row's conditional mean (bpmf_debug_means)      */
#define BPMF_NO_CENTER 0x8u   /* do not subtract the training mean from the ratings       */
#define BPMF_CUDA_CORE_GRAM 0x10u /* every row on the CUDA-core (FP32 FMA) kernel         */
#define BPMF_TEST_STALL 0x100u /* test only: the tensor-core kernel's gather producers never
                                  signal, so its bounded waits run out and the sweep reports
                                  BPMF_ETIMEOUT (exercises failure detection without a fault) */

/* ---- sides and phases --------------------------------------------------- */
#define BPMF_USER 0  /* rows of R, factors U, CSR */
#define BPMF_MOVIE 1 /* columns of R, factors V, CSC */

#define BPMF_PHASE_HYPER_USER 0  /* statistics of U, Normal-Wishart draw of (mu_U, Lambda_U) */
#define BPMF_PHASE_HYPER_MOVIE 1 /* same for V                                              */
#define BPMF_PHASE_ROWS_USER 2   /* every user row given V                                  */
#define BPMF_PHASE_ROWS_MOVIE 3  /* every movie column given U                              */
#define BPMF_PHASE_PREDICT 4     /* test predictions, running averages, RMSE                */
#define BPMF_PHASE_ADVANCE 5     /* sweep counter += 1                                      */

typedef struct bpmf_ctx* bpmf_handle;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns device memory of at least `bytes` bytes usable on `stream`, or NULL. */
typedef void* (*bpmf_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*bpmf_free_fn)(void* ptr, void* stream, void* ctx);

typedef struct {
    double alpha;       /* rating precision (BPMF observation noise precision)         */
    double beta0;       /* Normal-Wishart prior: mean precision scale                   */
    double nu0;         /* Normal-Wishart prior: degrees of freedom, must be >= K       */
    const double* mu0;  /* K prior mean, NULL = zeros (host, copied)                    */
    const double* W0;   /* K x K SPD prior scale, NULL = identity (host, copied)        */
    uint64_t seed;      /* Philox key                                                   */
    uint32_t job_id;    /* goes into the Philox counter (tag | job_id << 8)             */
    int32_t burn_in;    /* sweeps before predictions enter the running average          */
    int32_t order;      /* 0 = movies first (Alg. 1), 1 = users first                   */
    uint32_t flags;     /* BPMF_* flags                                                  */
    double clip_lo, clip_hi;
    int32_t long_min_degree; /* rows with at least this many ratings use the tensor-core
                                kernel (K in 49..64); <= 0 = library default (16;
                                48 with BPMF_BF16_GRAM)                               */
    int32_t wait_timeout_ms; /* limit of every device-side wait, <= 0 = 2000 ms         */
    int32_t split_degree; /* rows on the CUDA-core kernel with at least this many ratings
                             are split into runs of split_degree / 2 ratings done by
                             separate warps (Sec. 3.2), the partial Gram matrices summed
                             in run order by the last warp; <= 0 = default (1024)      */
    int32_t rank_one_degree; /* rows on the CUDA-core kernel with fewer ratings than this
                                take the rank-one route (Sec. 3.1): chol(Lambda_X) from the
                                hyper step updated once per rating, no Gram and no
                                factorization; 1 = empty rows only, 0 = default (1),
                                < 0 = none                                             */
    bpmf_alloc_fn alloc; /* NULL = cudaMalloc / cudaFree */
    bpmf_free_fn free;
    void* alloc_ctx;
} bpmf_params;

/* Fill *p with the defaults: alpha 2, beta0 2, nu0 = K (set at create when 0),
 * mu0 0, W0 I, seed 0, burn_in 0, order 0, no flags, clip [1, 5]. */
int bpmf_default_params(bpmf_params* p);

/*
 * Create a chain: the state Alg. 1 (Sec. 2) iterates on, for the M x N rating
 * matrix R ~ U V^T of Sec. 1 (users = rows, movies = columns).  Copies the ratings
 * (host arrays) to the device, builds the column view (the ratings of each movie,
 * which the movie loop of Alg. 1 walks), bins the rows by degree (Sec. 4.2's
 * per-item cost) and draws the initial factors U, V ~ N(0, 1) from the Philox
 * init streams (the paper does not state an initial state).
 *   csr_*        : M + 1 row pointers (csr_ptr[0] = 0), nnz column indices in
 *                  [0, N), nnz values.  Host memory.
 *   csc_*        : the same ratings by column (rows ascending inside each column),
 *                  or all three NULL.  The library always builds the column view
 *                  itself; one passed here must equal it entry by entry, else
 *                  BPMF_EINVAL.  Host memory.
 *   test_*       : T held-out points (row, column, value), T may be 0.  Host.
 *   cuda_stream  : cudaStream_t for all work of this handle (NULL = default).
 * Errors: BPMF_EINVAL for bad sizes, K outside [1, 64], nu0 < K, pointers out
 * of order, indices out of range or a column view that is not the transpose of
 * the rows; BPMF_ENOMEM; BPMF_ECUDA.
 */
int bpmf_create(bpmf_handle* out, int64_t M, int64_t N, int32_t K, const int64_t* csr_ptr,
                const int32_t* csr_col, const float* csr_val, const int64_t* csc_ptr,
                const int32_t* csc_row, const float* csc_val, int64_t T, const int32_t* test_i,
                const int32_t* test_j, const float* test_r, const bpmf_params* p,
                void* cuda_stream);

/*
 * Run n_sweeps full Gibbs sweeps (Alg. 1): hyper(V), movies, hyper(U), users,
 * predict (order 0; order 1 swaps the sides).  Each hyper step runs on a second
 * stream of the handle beside the other side's row update (each depends only on
 * its own side's factors), and sweeps after the first replay a CUDA graph of the
 * launches when the handle's stream can be captured (not the legacy default
 * stream); results are bit-identical to running the phases one by one.  If either
 * RMSE pointer is non-NULL, the call waits for the sweeps and writes the RMSE of
 * the last sweep's sample and of the running-average prediction (NaN before
 * burn-in; both NaN when T = 0).  Host pointers.  A sticky device error from any
 * kernel is returned as its code.
 */
int bpmf_sweep(bpmf_handle h, int32_t n_sweeps, double* rmse_sample, double* rmse_avg);

/*
 * n_sweeps sweeps of each of n independent chains, issued sweep by sweep and
 * chain by chain, so chains created on different streams run concurrently on the
 * device (small jobs do not fill the GPU alone).  hs: host array of n handles,
 * borrowed.  Each chain's result equals bpmf_sweep(hs[k], n_sweeps) alone.  Does
 * not wait; read RMSEs with bpmf_sweep(h, 0, ...).  BPMF_EINVAL for a NULL handle
 * or negative counts; the first launch error stops the batch.
 */
int bpmf_sweep_batch(bpmf_handle* hs, int32_t n, int32_t n_sweeps);

/*
 * Batched sweeps of many independent chains with the launches shared: each step of
 * Alg. 1's sweep (hyper-parameters of one side, its rows, the other side's, the
 * prediction loop) runs for all chains of the batch in one launch per kernel variant
 * (per K class where kernels are compiled per K), over a table of (chain, blocks) in
 * which every chain gets the blocks its own launch would have and the heaviest chains
 * come first -- the work queue in longest-processing-time order of Sec. 4.2's cost
 * model, c0 + c1 d per item, served by the device's block dispatch.  The chains'
 * tensor-core launches (K = 64 rows of the long bin) fork over eight streams.  One
 * sweep is captured as one CUDA graph when `cuda_stream` can be captured.
 *
 * bpmf_batch_create: hs is a host array of n >= 1 distinct handles, borrowed (they must
 * outlive the batch and keep their bins: after bpmf_set_tuning or bpmf_set_shard on one
 * of them, bpmf_batch_sweep returns BPMF_EINVAL; make a new batch).  All on one device, with the
 * same sweep order and no shard restriction, else BPMF_EINVAL.  cuda_stream: the
 * stream the batch's launches go to (NULL: the legacy default stream, not captured).
 * The tables live in one device allocation of the batch (cudaMalloc), freed by
 * bpmf_batch_destroy.
 *
 * bpmf_batch_sweep: n_sweeps sweeps of every chain, ordered after the work already
 * queued on each chain's own stream, and before work queued there later.  Each
 * chain's result equals bpmf_sweep(hs[k], n_sweeps) alone, bit for bit.  Does not
 * wait; read RMSEs with bpmf_sweep(h, 0, ...).  bpmf_batch_launch_count: kernels
 * launched by the batch's sweeps so far.  bpmf_batch_destroy waits for the batch's
 * stream, then frees it (NULL is a no-op).
 */
typedef struct bpmf_batch_ctx* bpmf_batch;
int bpmf_batch_create(bpmf_handle* hs, int32_t n, void* cuda_stream, bpmf_batch* out);
int bpmf_batch_sweep(bpmf_batch b, int32_t n_sweeps);
int bpmf_batch_launch_count(bpmf_batch b, int64_t* launches);
int bpmf_batch_destroy(bpmf_batch b);

/*
 * Change the tuning thresholds of a live handle (long_min_degree, split_degree and
 * rank_one_degree of bpmf_params, each with its meaning of 0 and of negative values
 * there): the rows of both sides
 * are binned and split again (host sort of the degrees kept from bpmf_create,
 * host-to-device copies waited for; the segment arrays grow when a smaller
 * split_degree needs more, the old ones held until bpmf_destroy).  The chain state
 * is untouched; rows may move between the CUDA-core and tensor-core kernels or
 * between split and whole or between the Gram and rank-one routes, whose results agree
 * within the FP32 tolerance, not bit for bit.  For autotuning.  BPMF_ENOMEM / BPMF_ECUDA leave the handle unusable.
 */
int bpmf_set_tuning(bpmf_handle h, int32_t long_min_degree, int32_t split_degree,
                    int32_t rank_one_degree);

/* Run one BPMF_PHASE_* step of a sweep (for checking the steps one by one). */
int bpmf_step(bpmf_handle h, int32_t phase);

/*
 * Predictions r_bar + u_i . v_j of the current sample for n points (clipped
 * under BPMF_CLIP): the "predict rating" step of Alg. 1's last loop (Sec. 2), on
 * points the caller names.  where = 0: i, j, out are host arrays; where = 1:
 * device arrays valid on the handle's stream.  BPMF_EINVAL for indices out of
 * range (checked on the host for where = 0; device indices are the caller's
 * responsibility).
 */
int bpmf_predict(bpmf_handle h, int64_t n, const int32_t* i, const int32_t* j, float* out,
                 int32_t where);

/*
 * Chain state, host buffers: the variables Alg. 1 (Sec. 2) carries from one
 * sampling iteration to the next -- U (M x K), V (N x K) FP32 and the sampled
 * hyper-parameters in FP64, laid out as [mu_U (K), Lambda_U (K x K), mu_V (K),
 * Lambda_V (K x K)] -- and sweep = number of completed sweeps.  Any pointer may be
 * NULL to skip that part.  The paper has no checkpoint step; because every random
 * number here is a function of (seed, sweep, row), restoring a state and
 * continuing reproduces an uninterrupted chain.
 */
int bpmf_get_state(bpmf_handle h, float* U, float* V, double* hyper, uint64_t* sweep);
int bpmf_set_state(bpmf_handle h, const float* U, const float* V, const double* hyper,
                   uint64_t sweep);

/* Running prediction sums (T doubles) and the number of sweeps they hold. */
int bpmf_get_accum(bpmf_handle h, double* psum, int64_t* n_avg);
int bpmf_set_accum(bpmf_handle h, const double* psum, int64_t n_avg);

/* Statistics of the last hyper step of `side`: row count, mean (K) and scatter
 * S = (1/n) sum (x - mean)(x - mean)^T (K x K), FP64 host buffers. */
int bpmf_get_stats(bpmf_handle h, int32_t side, int64_t* n, double* mean, double* S);

/* Conditional means of the last row update of `side` (rows x K FP32, host): each
 * row's update of Alg. 1 (Sec. 2) draws the new vector as this mean "plus randomly
 * sampled noise"; kept for checking the update against a reference.  Needs
 * BPMF_DEBUG_MEANS at create, else BPMF_EINVAL. */
int bpmf_debug_means(bpmf_handle h, int32_t side, float* out);

/* Sticky device status: BPMF_OK, BPMF_ETIMEOUT (reported first: later launches may
 * report what a timed-out one left behind), BPMF_ENOTPD (a precision matrix of Sec.
 * 3.1's factorisation was not positive definite in FP32), BPMF_ENAN or BPMF_EGAMMA.
 * The paper has no counterpart; kernels record failures here instead of trapping.
 * Syncs the handle's stream. */
int bpmf_status(bpmf_handle h);

/*
 * Sharded sweeps (one process per GPU; Sec. 4.2 and 4.3 of the paper spread the items
 * over nodes by a per-item cost of a fixed part plus a part per rating, and send the
 * updated items to the nodes that need them after each half-sweep):
 *
 * bpmf_set_shard restricts the row phases of `side` to rows [row_begin, row_end)
 * (every row again with [0, rows)); the rows are binned and planned again (host sort
 * of the degrees kept from bpmf_create, host-to-device copies waited for).  The hyper
 * step still reduces over every row of the side and the prediction step over every
 * test point, so every shard must hold the whole side before them: a caller exchanges
 * the rows each shard updated after every row phase (bpmf_get_rows, a collective of its
 * own, bpmf_put_rows).  A row's update depends only on the other side, the side's
 * hyper-parameters and (seed, sweep, row), so shards that exchange this way run the
 * same chain, bit for bit, as one handle over all rows.  BPMF_EINVAL for a bad side or
 * range.
 *
 * bpmf_get_rows copies rows [row_begin, row_end) of U (side 0) or V (side 1) to out,
 * packed (K floats a row); bpmf_put_rows overwrites them from in and refreshes their
 * 16-bit copies for the tensor-core Gram.  where = 0: host buffer (the call waits for
 * the copy); where = 1: device buffer, the copy ordered on the handle's stream.  The
 * paper's exchange uses MPI or GASPI between nodes; here the caller's collective (NCCL,
 * or gloo on host copies) moves the rows.
 */
int bpmf_set_shard(bpmf_handle h, int32_t side, int64_t row_begin, int64_t row_end);
int bpmf_get_rows(bpmf_handle h, int32_t side, int64_t row_begin, int64_t row_end, float* out,
                  int32_t where);
int bpmf_put_rows(bpmf_handle h, int32_t side, int64_t row_begin, int64_t row_end,
                  const float* in, int32_t where);

/* Host only (no handle, no device work): the device bytes bpmf_create would hold for
 * this problem (the figure bpmf_info then reports as device_bytes), for admission of
 * jobs against a memory budget before any allocation.  Arguments as for bpmf_create:
 * M x N ratings in CSR (csr_ptr: M + 1 offsets; csr_col: the column of each rating,
 * used for the column view's degrees), K latent dimensions, n_test test points, params
 * (NULL: defaults; the flags, long_min_degree and split_degree change the bins and the
 * buffers).  num_sms: SM count of the device the handle will run on (<= 0: the current
 * device, read with cudaDeviceGetAttribute).  *out_bytes receives the sum of
 * bpmf_create's allocations, each rounded up to 256 bytes as it rounds them (scratch
 * that bpmf_create frees before returning is not counted).  BPMF_EINVAL for a NULL
 * pointer, sizes outside bpmf_create's limits or a column index outside [0, N);
 * BPMF_ECUDA if the SM count cannot be read; BPMF_ENOMEM if the host cannot allocate. */
int bpmf_device_bytes(int64_t M, int64_t N, int32_t K, const int64_t* csr_ptr,
                      const int32_t* csr_col, int64_t n_test, const bpmf_params* params,
                      int32_t num_sms, int64_t* out_bytes);

/* Host only (no device work, no handle): the degree bins bpmf_create makes for one
 * side.  ptr: rows + 1 offsets of the side's ratings (ptr[0] = 0, non-decreasing);
 * rows with at least long_min ratings form the tensor-core bin (long_min <= 0: no such
 * bin).  order_out (rows entries) receives the short bin, then the long bin, each
 * longest first with equal degrees in ascending row order (a counting sort, Sec. 4.2's
 * ordering of items by cost); *n_short the size of the short bin.  BPMF_EINVAL on
 * rows < 1 or above INT32_MAX, a row with more than INT32_MAX ratings, a NULL pointer
 * or malformed offsets; BPMF_ENOMEM if the host sort cannot allocate. */
int bpmf_bin_rows(int64_t rows, const int64_t* ptr, int64_t long_min, int32_t* order_out,
                  int64_t* n_short);

/* Host only (no device work, no handle): the balanced plan bpmf_create makes for
 * the tensor-core rows of a launch of `grid` CTAs.  degree[k] (n entries, >= 0) are
 * the rows' rating counts in the order the kernel deals them (longest first); a row
 * costs its 64-rating stages plus two (Sec. 4.2's fixed-plus-per-rating cost of an
 * item).  When round-robin (row k to CTA k mod grid) would leave the busiest CTA
 * more than 5% above the mean cost and there are more rows than CTAs, *planned = 1,
 * order_out[p] (n entries) is the row placed at p and CTA c takes places
 * first_out[c] .. first_out[c + 1] - 1 (first_out: min(n, grid) + 1 entries), each
 * row, longest first, given to the CTA with the least cost so far (ties: lowest
 * CTA); else *planned = 0 and the outputs are not written.  BPMF_EINVAL on n or a
 * degree outside [0, INT32_MAX], grid < 1, or a NULL pointer that is needed;
 * BPMF_ENOMEM if the host plan cannot allocate. */
int bpmf_balance_rows(int64_t n, const int64_t* degree, int64_t grid, int32_t* order_out,
                      int64_t* first_out, int32_t* planned);

/* Diagnostics: number of rows of `side` on the CUDA-core kernel and on the
 * tensor-core kernel, how many of the former are split and into how many
 * segments, the centring mean, device bytes held, and `balanced`: bit 0 (bit 1)
 * set when the tensor-core rows are dealt to the CTAs of a Gram launch on every SM
 * (on all SMs but one, as bpmf_sweep launches; two CTAs per SM) by the balanced
 * plan -- each row, longest first, to the CTA with the least work so far, made
 * where the plain round-robin order would leave one CTA over 5% above the mean --
 * instead of round-robin.  NULL outputs are skipped. */
int bpmf_info(bpmf_handle h, int32_t side, int64_t* n_short, int64_t* n_long, int64_t* n_split,
              int64_t* n_segments, double* rbar, int64_t* device_bytes, int32_t* balanced);

/* Number of kernels this handle has launched so far (all phases, all sweeps). */
int bpmf_launch_count(bpmf_handle h, int64_t* launches);

/*
 * Launch timing of the row phases run by bpmf_step (not inside bpmf_sweep, whose sweeps
 * may be a captured CUDA graph).  on != 0: each row phase records CUDA events on the
 * handle's stream around its CUDA-core launches and around each of the two launches
 * of the tensor-core route (the Gram kernel, then the factorisation kernel).
 * bpmf_row_launch_ms waits for the last timed row phase and returns each part's
 * milliseconds (host pointers, all three required), -1 for a part that did not
 * launch (or when timing is off).
 */
int bpmf_set_row_timing(bpmf_handle h, int32_t on);
int bpmf_row_launch_ms(bpmf_handle h, float* cuda_core_ms, float* gram_ms, float* chol_ms);

/*
 * Row statistics of a device matrix, computed without allocating any memory.
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory when they need the reduction (for example a
 * serving process whose pool has already reserved the whole GPU, or a
 * latency-critical loop where cudaMalloc/cudaFree would synchronise the
 * device).  It runs the same reduction as the hyper step of a handle and
 * writes the same quantities bpmf_get_stats returns:
 *   mean = (1/rows) sum_r x_r,  S = (1/rows) sum_r (x_r - mean)(x_r - mean)^T.
 *   X      : device, rows x ld FP32 with ld = K rounded up to a multiple of 16
 *            (16, 32, 48 or 64), 16-byte aligned; columns K..ld-1 are ignored.
 *   shift  : device, K doubles (8-byte aligned) subtracted before summing for
 *            accuracy (any value near the mean does; a handle's hyper step uses
 *            the FP64 mean of the first 256 rows, summed in row order), or NULL
 *            for zero.
 *   mean   : device, K doubles (written).   S : device, K x K doubles (written);
 *            both 8-byte aligned.
 *   stream : cudaStream_t; the call only enqueues work and returns.
 * Scratch lives in a fixed file-scope device array (about 5.4 MB, held on every
 * GPU that loads the library until the process exits); K > 64, rows outside
 * [1, 2^31 - 1] or a misaligned pointer is rejected with BPMF_EINVAL before any
 * launch.  The first call on each device looks up the array's device address
 * (with that device current) and keeps it, so make that first call before any
 * stream capture, and do not call this entry point after cudaDeviceReset in the
 * same process (the array may then sit elsewhere).  All calls share the one
 * array: calls that overlap on the GPU (other streams, other threads) race and
 * must be serialised by the caller.  Nothing in the array needs to start at zero.
 */
int bpmf_row_stats_noalloc(const float* X, int64_t rows, int32_t K, const double* shift,
                           double* mean, double* S, void* stream);

/* Human-readable name of a return code (static string). */
const char* bpmf_strerror(int code);

/* Release everything the handle owns (waits for its streams first).  NULL-safe.  The
 * paper has no counterpart. */
int bpmf_destroy(bpmf_handle h);

#ifdef __cplusplus
}
#endif

#endif /* BPMF_H */
