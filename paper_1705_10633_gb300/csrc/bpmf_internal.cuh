// bpmf_internal.cuh -- device-side structures and kernel launchers shared by the
// translation units of the GB300 BPMF library.  Not part of the public ABI.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bpmf {

constexpr int kMaxK = 64;

// Per-handle scalars that live on the device so that a whole sweep can be
// replayed (CUDA graph) without host involvement.
struct Control {
    unsigned long long sweep;  // completed sweeps (Philox counter field c2)
    long long n_avg;           // sweeps held in the running prediction sums
    unsigned int status;       // sticky error bits (kStatus*)
    unsigned int pad;
    double rmse_sample;
    double rmse_avg;
};

enum : unsigned int { kStatusNotPD = 1u, kStatusNaN = 2u, kStatusGamma = 4u };

// One segment of a long row on the CUDA-core kernel: ratings [lo, hi) of `row`, the
// `slot`-th split row, whose segments are first .. first + count - 1 (Sec. 3.2: an
// item with many ratings is cut into smaller tasks that run in parallel).
struct Segment {
    int64_t lo, hi;
    int32_t row, slot, first, count;
};

// Arguments of one row-update launch (one side, one degree bin).
struct RowArgs {
    const int64_t* ptr;    // rows + 1 offsets into idx/val
    const int32_t* idx;    // other-side index of each rating
    const float* val;      // centred rating
    const float* Y;        // other side's factors, ldy floats per row
    float* X;              // this side's factors (written), ldx floats per row
    float* means;          // conditional means (ldx per row) or nullptr
    __half* Xh;            // FP16 split of X (hi, lo), ldx per row, or nullptr
    __half* Xl;
    const __half* Yh;      // FP16 split of Y (tensor-core kernel only)
    const __half* Yl;
    const int32_t* rows;   // rows of this bin, longest first
    int64_t nrows;
    // tensor-core kernel: a balanced assignment of the rows to the CTAs of a launch of
    // exactly plan_grid CTAs -- CTA b takes rows[cta_first[b]] .. rows[cta_first[b + 1] - 1]
    // (its rows longest first).  Without one (nullptr, or another grid) CTA b takes
    // rows[b], rows[b + grid], ...
    const int64_t* cta_first;
    int64_t plan_grid;
    // CUDA-core kernel only: the first nsplit rows are done as nsegs segments, each
    // writing its partial Gram rows and right-hand side to part; the last segment of
    // a row to finish (counted in seg_done, which it resets) sums them in segment
    // order and samples the row
    const Segment* segs;
    int64_t nsegs;
    // tensor-core route (kp == 64): the Gram kernel writes each row's precision and
    // right-hand side to slot p of `gram` (p = the row's place in `rows`), the
    // factorisation kernel reads them back
    float* gram;
    int64_t nsplit;
    float* part;
    unsigned int* seg_done;
    const float* lam;      // prior precision, kp x kp, identity beyond K
    const float* lam_ct;   // the same, chunk-transposed: float4 (i, 4c..4c+3) at c * kp + i
    const float* lammu;    // prior precision times prior mean, kp (zero beyond K)
    const float* lamchol_ct;  // chol(prior precision), lower, chunk-transposed like lam_ct
    int64_t nrank_one;     // CUDA-core kernel: the last nrank_one rows of the bin (at most
                           // the rank-one threshold's ratings) take the rank-one route
    Control* ctl;
    uint64_t seed;
    uint32_t c3;           // Philox tag word of this side's row noise
    int64_t timeout_ns;    // bound on every device wait (tensor-core kernel)
    int test_stall;        // test only: producers never signal (exercises the timeout path)
    int bf16;              // Xh / Xl / Yh hold BF16 (the tensor-core Gram takes Yh only)
    int ldx, ldy;
    int K;
    float alpha;
};

// ---- launchers (each returns the launch error) ----------------------------
cudaError_t launch_init_factors(float* X, int64_t rows, int K, int ld, uint64_t seed, uint32_t c3,
                                cudaStream_t s);
cudaError_t launch_center_values(float* val, int64_t n, double rbar, cudaStream_t s);
// Column range check and fixed-order FP64 sum of n ratings: scratch[0] = sum (scratch
// holds 1 + kCheckSumBlocks doubles), *bad = 1 if an index is outside [0, ncols).
constexpr int kCheckSumBlocks = 512;
cudaError_t launch_check_sum(const int32_t* col, const float* val, int64_t n, int32_t ncols,
                             double* scratch, unsigned int* bad, cudaStream_t s);

// Hyper step, part 1: per-block partial sums of (x - shift) and (x - shift)(x - shift)^T.
int hyper_reduce_blocks(int64_t rows, int num_sms);
__host__ __device__ inline size_t hyper_partial_doubles(int kp)
{
    return (size_t)kp + (size_t)kp * kp;
}
cudaError_t launch_hyper_reduce(const float* X, int64_t rows, int kp, const double* shift64,
                                double* partials, int nblocks, cudaStream_t s);
// part 2: fixed-order sum of the partials -> sums[kp + kp*kp]
cudaError_t launch_hyper_combine(const double* partials, int nblocks, int kp, double* sums,
                                 cudaStream_t s);

struct NWArgs {
    const double* sums;     // kp + kp*kp raw sums from the reduction
    const double* shift64;  // kp, shift used by the reduction (mean of the first rows)
    int64_t n;              // rows of this side
    int K, kp;
    double beta0, nu0;
    const double* mu0;      // K
    const double* W0inv;    // K x K
    uint64_t seed;
    uint32_t sweep_offset;  // the draw belongs to sweep ctl->sweep + sweep_offset
    uint32_t c3_normal, c3_gamma;
    Control* ctl;
    double* stats;          // out: mean (K), S (K x K)
    double* mu64;           // out: K    (also the next shift)
    double* lam64;          // out: K x K
    float* lam32;           // out: kp x kp, identity beyond K, then its chunk-transposed copy,
                            // then the chunk-transposed lower Cholesky factor (identity beyond K)
    float* lammu32;         // out: kp
    double* draws;          // K(K-1)/2 + 2K scratch: the step's random draws
    const double* partials; // nparts > 0: the reduction's block partials, combined here
    int nparts;             // (fixed order); 0: `sums` holds the combined sums
};
// Doubles of NWArgs::draws for K.
inline size_t nw_draws_doubles(int K) { return (size_t)K * (K - 1) / 2 + 2 * (size_t)K; }
// The one-CTA draw (its random numbers come from launch_hyper_stats_draws).
cudaError_t launch_nw_sample(const NWArgs& a, cudaStream_t s);
// The hyper step's first launch: the shift (FP64 mean of the first rows, computed by every
// block, published by block 0), the reduction's block partials, and in extra blocks the
// draw's random numbers.
cudaError_t launch_hyper_stats_draws(const float* X, int64_t rows, int K, int kp, double* shift64,
                                     double* partials, int nblocks, const NWArgs& a, cudaStream_t s);
// Reductions of at most this many blocks are combined inside the draw kernel.
constexpr int kFuseCombineBlocks = 8;
// Index of (i, j) in the chunk-transposed copy of a kp x kp matrix (kp a multiple
// of 4): float4 (i, 4c .. 4c + 3) sits at float4 index c * kp + i.
__host__ __device__ inline int chunk_t_index(int i, int j, int kp)
{
    return ((j >> 2) * kp + i) * 4 + (j & 3);
}
// FP32 copies of a hyper state given in FP64 (after bpmf_set_state).
cudaError_t launch_hyper_refresh(const double* mu64, const double* lam64, int K, int kp,
                                 float* lam32, float* lammu32, Control* ctl, cudaStream_t s);

// Row updates on CUDA cores: one warp per row (any degree).
cudaError_t launch_rows_warp(const RowArgs& a, int kp, int num_sms, cudaStream_t s);
// Kernel launches launch_rows_warp makes for `a` (0 to 2).
int rows_warp_launches(const RowArgs& a);
// Floats of one segment's partial in `part` (Gram rows owned by a lane, and the
// right-hand side, lane-interleaved).
int warp_partial_floats(int kp);
// ---- batched launches: one launch runs the same step for many jobs --------------
// A job's share of a batched launch: its arguments and the blocks [first, first + count)
// of the launch's grid, which run the job's work exactly as a launch of `count` blocks of
// its own would (a job's result does not depend on the other jobs in the launch).
// Tables are ordered by `first`.
template <class A>
struct BatchEntry {
    A args;
    int32_t first;
    int32_t count;
};
// The entry whose blocks hold block b.
template <class A>
__device__ __forceinline__ int batch_find(const BatchEntry<A>* t, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t[mid].first <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
// Work items of a row launch (segments and rows of the Gram route, or rank-one rows).
int64_t rows_warp_items(const RowArgs& a, bool rank_one);
// CTAs of the CUDA-core row kernel one SM holds at once for this kp.
int rows_warp_resident_blocks(int kp);
cudaError_t launch_rows_warp_batch(const BatchEntry<RowArgs>* t, int n, int64_t blocks, int kp,
                                   bool rank_one, cudaStream_t s);
// The hyper step's reduction for many jobs of one kp (blocks: nred + draw blocks each).
struct ReduceArgs {
    const float* X;
    int64_t rows;
    int shiftK;
    double* shift64;
    double* partials;
    int nred;
    NWArgs draws;
};
cudaError_t launch_hyper_reduce_batch(const BatchEntry<ReduceArgs>* t, int n, int64_t blocks,
                                      int kp, cudaStream_t s);
int hyper_draw_blocks(int K);
// The fixed-order combine for many jobs (E = kp + kp^2 doubles each, 128 per block).
struct CombineArgs {
    const double* partials;
    int nblocks, E;
    double* sums;
};
int hyper_combine_blocks(int kp);
cudaError_t launch_hyper_combine_batch(const BatchEntry<CombineArgs>* t, int n, int64_t blocks,
                                       cudaStream_t s);
// The Normal-Wishart draw for many jobs: one CTA each.
cudaError_t launch_nw_sample_batch(const NWArgs* t, int n, cudaStream_t s);
// Test-set prediction for many jobs: the blocks of each job (its own prediction block
// count), then one thread per job for its RMSEs (and, with advance, its sweep counter).
struct PredictArgs {
    const int32_t* ti;
    const int32_t* tj;
    const float* tr;
    int64_t T;
    const float* U;
    const float* V;
    int ld, kp;
    double rbar;
    int clip;
    double lo, hi;
    int burn_in;
    double* psum;
    Control* ctl;
    double* partials;
};
cudaError_t launch_predict_batch(const BatchEntry<PredictArgs>* t, int n, int64_t blocks,
                                 cudaStream_t s);
cudaError_t launch_predict_finish_batch(const BatchEntry<PredictArgs>* t, int n, bool advance,
                                        cudaStream_t s);

// Row updates with the Gram on tensor cores (kp == 64, rows of the long bin).
// Scratch device memory for one call (allocated and returned inside it).
struct TempAlloc {
    void* (*alloc_fn)(size_t bytes, void* ctx);
    void (*free_fn)(void* p, void* ctx);
    void* ctx;
    void* alloc(size_t bytes) const { return alloc_fn(bytes, ctx); }
    void free(void* p) const { free_fn(p, ctx); }
};

// CSC of the ratings from the CSR on the device (same order as a stable counting
// sort by column).  csc_ptr: N + 1, csc_row / csc_val: nnz (< 2^31).  Waits for the
// stream before returning its scratch.
cudaError_t build_csc_device(const int64_t* csr_ptr, const int32_t* csr_col, const float* csr_val,
                             int64_t M, int64_t N, int64_t nnz, int64_t* csc_ptr, int32_t* csc_row,
                             float* csc_val, const TempAlloc& tmp, cudaStream_t s);
// *same: whether a caller's column view (host arrays, raw values) equals the one built
// on the device (values centred by rbar): offsets, row indices (ascending in each
// column) and values, entry by entry.  Waits for the stream.
cudaError_t check_csc_device(const int64_t* built_ptr, const int32_t* built_row, const float* built_val,
                             const int64_t* csc_ptr, const int32_t* csc_row, const float* csc_val,
                             int64_t N, int64_t nnz, double rbar, const TempAlloc& tmp, bool* same,
                             cudaStream_t s);

// One slot of the tensor-core route's scratch (K = 64): the lower triangle of the
// row's Gram sum_c y_c y_c^T in float4 chunks, chunk column c (columns 4c .. 4c + 3)
// holding rows 4c .. 63 consecutively from float4 gram_chunk_offset(c), then
// sum_c r_c y_c (64 floats); Lambda_i = Lambda_X + alpha Gram and b_i =
// Lambda_X mu_X + alpha sum_c r_c y_c are formed from it by the factorisation kernel.
constexpr int kGramChunks = 544;
constexpr int kGramSlotFloats = 4 * kGramChunks + 64;
__host__ __device__ constexpr int gram_chunk_offset(int c) { return c * (66 - 2 * c); }
// Gram kernel (A3 on tensor cores): Lambda_i and b_i of the rows in a.rows into a.gram.
// It runs kGramCtasPerSm persistent CTAs per SM (grid = that many times num_sms, at
// most one CTA per row); a balanced plan of the rows must be made for that grid.
constexpr int kGramCtasPerSm = 2;
cudaError_t launch_rows_gram(const RowArgs& a, int num_sms, cudaStream_t s);
// Factorisation kernel (A4, A5): reads a.gram, writes the rows' new factors.
cudaError_t launch_rows_chol(const RowArgs& a, int num_sms, cudaStream_t s);
// FP16 hi/lo split of a factor matrix (after init or set_state).
cudaError_t launch_split_factors(const float* X, int64_t rows, int ld, __half* Xh, __half* Xl,
                                 int bf16, cudaStream_t s);

enum : unsigned int { kStatusTimeout = 8u };

// Test predictions.
int predict_blocks(int64_t T, int num_sms);
cudaError_t launch_predict(const int32_t* ti, const int32_t* tj, const float* tr, int64_t T,
                           const float* U, const float* V, int ld, int kp, double rbar, int clip,
                           double lo, double hi, int burn_in, double* psum, Control* ctl,
                           double* partials, int nblocks, cudaStream_t s);
cudaError_t launch_predict_finish(const double* partials, int nblocks, int64_t T, int burn_in,
                                  Control* ctl, cudaStream_t s);
cudaError_t launch_predict_points(const int32_t* i, const int32_t* j, int64_t n, const float* U,
                                  const float* V, int ld, int kp, double rbar, int clip, double lo,
                                  double hi, float* out, cudaStream_t s);
cudaError_t launch_advance(Control* ctl, cudaStream_t s);

}  // namespace bpmf
