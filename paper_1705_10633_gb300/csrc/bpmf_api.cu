// bpmf_api.cu -- the C ABI of include/bpmf.h: handle lifetime, host-side
// validation and preprocessing (column view, degree bins), and the order of
// the device phases of one Gibbs sweep (Alg. 1).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <new>
#include <numeric>
#include <queue>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bpmf.h"
#include "bpmf_internal.cuh"
#include "philox.cuh"

using namespace bpmf;

namespace {

// Default threshold of the tensor-core route.  With the BF16 Gram (8-bit mantissas) the
// rows keep to 48 ratings and more: a row of few ratings has a precision dominated by a
// handful of rank-one terms, and its conditional mean then carries the inputs' 2^-9
// error at up to 1.7% (a 16-rating movie of the 480k x 18k workload); the FP32-class
// Gram has no such limit.
constexpr int kDefaultLongMinDegree = 16;
constexpr int kDefaultLongMinDegreeBf16 = 48;
int64_t default_long_min(uint32_t flags)
{
    return (flags & BPMF_BF16_GRAM) ? kDefaultLongMinDegreeBf16 : kDefaultLongMinDegree;
}
constexpr int kDefaultSplitDegree = 1024;
constexpr int kDefaultRankOneDegree = 1;
constexpr int kDefaultWaitTimeoutMs = 2000;

struct DevSide {
    int64_t rows = 0;
    // rows this handle updates in its row phases: [shard_lo, shard_hi) (all rows unless
    // bpmf_set_shard restricted them); the hyper step always reduces over every row
    int64_t shard_lo = 0, shard_hi = 0;
    int64_t* ptr = nullptr;
    int32_t* idx = nullptr;
    float* val = nullptr;
    float* X = nullptr;
    __half* Xh = nullptr;  // FP16 split of X, kept when the tensor-core kernel is on
    __half* Xl = nullptr;
    float* means = nullptr;
    int32_t* bin_rows = nullptr;  // short bin first, then long bin, each longest first
    int64_t n_short = 0, n_long = 0;
    int64_t long_ratings = 0;  // ratings of the long bin's rows
    std::vector<int64_t> ptr_h;  // host copy of ptr, for binning again (bpmf_set_tuning)
    // long rows of the CUDA-core kernel, cut into segments (first n_split rows of
    // the short bin); capacities grow when bpmf_set_tuning asks for more
    Segment* segs = nullptr;
    int64_t n_segs = 0, seg_cap = 0;
    int64_t n_split = 0, split_cap = 0;
    int64_t n_rank_one = 0;  // last rows of the short bin, on the rank-one route
    float* part = nullptr;           // seg_cap partials
    unsigned int* seg_done = nullptr;  // split_cap counters, zero between launches
    // balanced plans of the long bin for the two grids a tensor-core launch can have
    // (every SM, or one left to the hyper steps): rows grouped by CTA, per-CTA offsets;
    // plan_grid 0 when round-robin is kept
    int32_t* plan_rows[2] = {nullptr, nullptr};
    int64_t* plan_first[2] = {nullptr, nullptr};
    int64_t plan_grid[2] = {0, 0};
    int64_t plan_cap[2] = {0, 0};
    double* mu64 = nullptr;
    double* shift64 = nullptr;  // kp: shift of the hyper statistics
    double* lam64 = nullptr;
    double* nw_draws = nullptr;  // the hyper step's random draws (scratch)
    float* lam32 = nullptr;
    float* lammu32 = nullptr;
    double* partials = nullptr;
    int red_blocks = 1;
    double* sums = nullptr;
    double* stats = nullptr;
    uint32_t tag_init = 0, tag_row = 0, tag_hyper = 0, tag_gamma = 0;
};

}  // namespace

struct bpmf_ctx {
    int device = 0;
    int num_sms = 1;
    int64_t long_min = 48;           // binning threshold of the tensor-core kernel
    int64_t split_degree = 1024;  // CUDA-core rows with this many ratings are split
    int rank_one_max = 0;  // CUDA-core rows with at most this many ratings: rank-one route
    int row_sms = 1;  // CTAs of the row kernels: all SMs, or all but one while the
                      // next hyper step runs beside them (bpmf_sweep)
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr;  // hyper steps overlapped with row phases
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // the steady-state overlapped sweep as a CUDA graph (0: not tried, 1: ready,
    // -1: the stream cannot be captured)
    int graph_state = 0;
    cudaGraphExec_t sweep_graph = nullptr;
    int64_t graph_launches = 0;
    int64_t M = 0, N = 0, nnz = 0, T = 0;
    int K = 0, kp = 0;
    bool tc = false;  // long rows on the tensor-core kernel
    bpmf_params p{};
    std::vector<double> mu0, W0;
    double rbar = 0.0;
    DevSide side[2];
    double* mu0_d = nullptr;
    double* W0inv_d = nullptr;
    int32_t* ti = nullptr;
    int32_t* tj = nullptr;
    float* tr = nullptr;
    double* psum = nullptr;
    double* pred_partials = nullptr;
    int pred_blocks = 1;
    Control* ctl = nullptr;
    std::vector<void*> allocs;
    std::vector<size_t> alloc_bytes;
    int64_t bytes = 0;
    int64_t launches = 0;  // kernels launched by the phases
    uint64_t bins_version = 0;  // moves whenever a side is binned again (a batch checks it)
    // bpmf_set_row_timing: events around the row kernels of phases run by bpmf_step
    bool row_timing = false;
    cudaEvent_t tev[4] = {nullptr, nullptr, nullptr, nullptr};
    int timed_parts = 0;  // bit 0: CUDA-core launches recorded, bit 1: tensor-core launches
    // scratch of the tensor-core route: one slot (precision and right-hand side) per row
    // of the larger long bin
    float* gram = nullptr;
    int64_t gram_cap = 0;
};

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? BPMF_OK : BPMF_ECUDA; }

void* dalloc(bpmf_ctx* h, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (h->p.alloc) {
        p = h->p.alloc(bytes, (void*)h->stream, h->p.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        h->allocs.push_back(p);
        h->alloc_bytes.push_back(bytes);
        h->bytes += (int64_t)bytes;
    }
    return p;
}

// Scratch for one call: through the caller's hook when there is one, not kept.
void* temp_alloc(size_t bytes, void* ctx)
{
    bpmf_ctx* h = static_cast<bpmf_ctx*>(ctx);
    bytes = (bytes + 255) & ~(size_t)255;
    if (h->p.alloc) return h->p.alloc(bytes, (void*)h->stream, h->p.alloc_ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void temp_free(void* p, void* ctx)
{
    bpmf_ctx* h = static_cast<bpmf_ctx*>(ctx);
    if (!p) return;
    if (h->p.free) h->p.free(p, (void*)h->stream, h->p.alloc_ctx);
    else cudaFree(p);
}

// Release one allocation made by dalloc before the handle is destroyed.
void dfree(bpmf_ctx* h, void* p)
{
    if (!p) return;
    for (size_t k = 0; k < h->allocs.size(); ++k) {
        if (h->allocs[k] != p) continue;
        h->allocs.erase(h->allocs.begin() + (std::ptrdiff_t)k);
        h->bytes -= (int64_t)h->alloc_bytes[k];
        h->alloc_bytes.erase(h->alloc_bytes.begin() + (std::ptrdiff_t)k);
        if (h->p.free) h->p.free(p, (void*)h->stream, h->p.alloc_ctx);
        else cudaFree(p);
        return;
    }
}

template <class T>
bool alloc_n(bpmf_ctx* h, T** out, size_t n)
{
    *out = static_cast<T*>(dalloc(h, sizeof(T) * n));
    return *out != nullptr;
}

// Host FP64 Cholesky (lower) used to validate W0 and to invert it.
bool host_cholesky(int K, const double* A, std::vector<double>& L)
{
    L.assign((size_t)K * K, 0.0);
    for (int j = 0; j < K; ++j) {
        double d = A[j * K + j];
        for (int k = 0; k < j; ++k) d -= L[j * K + k] * L[j * K + k];
        if (!(d > 0.0)) return false;
        L[j * K + j] = sqrt(d);
        for (int i = j + 1; i < K; ++i) {
            double s = A[i * K + j];
            for (int k = 0; k < j; ++k) s -= L[i * K + k] * L[j * K + k];
            L[i * K + j] = s / L[j * K + j];
        }
    }
    return true;
}

bool host_spd_inverse(int K, const double* A, std::vector<double>& inv)
{
    std::vector<double> L;
    if (!host_cholesky(K, A, L)) return false;
    inv.assign((size_t)K * K, 0.0);
    std::vector<double> y(K), x(K);
    for (int c = 0; c < K; ++c) {
        for (int i = 0; i < K; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * K + k] * y[k];
            y[i] = s / L[i * K + i];
        }
        for (int i = K - 1; i >= 0; --i) {
            double s = y[i];
            for (int k = i + 1; k < K; ++k) s -= L[k * K + i] * x[k];
            x[i] = s / L[i * K + i];
        }
        for (int i = 0; i < K; ++i) inv[i * K + c] = x[i];
    }
    return true;
}

bool valid_ptr(int64_t rows, const int64_t* ptr)
{
    if (ptr[0] != 0) return false;
    for (int64_t r = 0; r < rows; ++r)
        if (ptr[r + 1] < ptr[r]) return false;
    return true;
}

bool valid_csr(int64_t rows, int64_t cols, const int64_t* ptr, const int32_t* idx)
{
    if (!valid_ptr(rows, ptr)) return false;
    const int64_t nnz = ptr[rows];
    for (int64_t t = 0; t < nnz; ++t)
        if (idx[t] < 0 || (int64_t)idx[t] >= cols) return false;
    return true;
}

// Column view by counting sort; rows ascend inside each column.
void build_csc(int64_t M, int64_t N, const int64_t* rp, const int32_t* ci, const float* v,
               std::vector<int64_t>& cp, std::vector<int32_t>& ri, std::vector<float>& cv)
{
    const int64_t nnz = rp[M];
    cp.assign((size_t)N + 1, 0);
    for (int64_t t = 0; t < nnz; ++t) cp[(size_t)ci[t] + 1] += 1;
    for (int64_t j = 0; j < N; ++j) cp[j + 1] += cp[j];
    std::vector<int64_t> fill(cp.begin(), cp.end() - 1);
    ri.resize((size_t)nnz);
    cv.resize((size_t)nnz);
    for (int64_t i = 0; i < M; ++i)
        for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
            const int64_t q = fill[ci[t]]++;
            ri[q] = (int32_t)i;
            cv[q] = v[t];
        }
}

// Degree bins: rows below `long_min` (short bin) then the rest (long bin), each
// ordered by decreasing degree so that a grid-stride loop hands the longest
// rows out first (the per-item cost model of Sec. 4.2: fixed + per-rating cost).
void bin_rows(int64_t rows, const int64_t* ptr, int64_t long_min, std::vector<int32_t>& order,
              int64_t* n_short, int64_t* n_long, int64_t* long_ratings)
{
    // counting sort by degree (stable: equal degrees keep ascending row order)
    int64_t dmax = 0;
    for (int64_t r = 0; r < rows; ++r) dmax = std::max(dmax, ptr[r + 1] - ptr[r]);
    std::vector<int64_t> start((size_t)dmax + 2, 0);
    for (int64_t r = 0; r < rows; ++r) ++start[(size_t)(ptr[r + 1] - ptr[r])];
    // bucket offsets: short-bin degrees (below long_min) first, each bin from its
    // largest degree down
    const int64_t split = std::min(long_min, dmax + 1);  // degrees >= split are long
    int64_t off = 0, ns = 0, nl_ratings = 0;
    std::vector<int64_t> pos((size_t)dmax + 1, 0);
    for (int64_t d = split - 1; d >= 0; --d) {
        pos[(size_t)d] = off;
        off += start[(size_t)d];
    }
    ns = off;
    for (int64_t d = dmax; d >= split; --d) {
        pos[(size_t)d] = off;
        off += start[(size_t)d];
        nl_ratings += d * start[(size_t)d];
    }
    order.resize((size_t)rows);
    for (int64_t r = 0; r < rows; ++r) order[(size_t)pos[(size_t)(ptr[r + 1] - ptr[r])]++] = (int32_t)r;
    *n_short = ns;
    *n_long = rows - ns;
    *long_ratings = nl_ratings;
}

// rank_one_degree of bpmf_params (rows with fewer ratings take the rank-one route; 0
// the default, < 0 none) as the largest degree on that route (-1: none).
int rank_one_from(int32_t v) { return (v > 0 ? v : (v == 0 ? kDefaultRankOneDegree : 0)) - 1; }

// Segments of the CUDA-core kernel's long rows (Sec. 3.2's split of items with many
// ratings into smaller parallel tasks): the rows at the head of the short bin (longest
// first) with at least split_degree ratings are cut into ceil(d / (split_degree / 2))
// near-equal runs of consecutive ratings.  Uploads the list (waited for) and zeroes
// the rows' counters; grows the device arrays when the list outgrows them.
// The segment list itself (host only); returns the number of rows split.
int64_t build_segments(const int64_t* ptr, const std::vector<int32_t>& order, int64_t n_short,
                       int64_t split_degree, std::vector<Segment>& segs)
{
    segs.clear();
    int64_t nsplit = 0;
    const int64_t seg_len = split_degree / 2 > 0 ? split_degree / 2 : 1;
    for (int64_t r = 0; r < n_short; ++r) {
        const int32_t row = order[(size_t)r];
        const int64_t p0 = ptr[row], deg = ptr[row + 1] - p0;
        if (deg < split_degree || deg < 2) break;  // the bin is ordered longest first
        const int64_t n = (deg + seg_len - 1) / seg_len;
        const int32_t first = (int32_t)segs.size();
        for (int64_t t = 0; t < n; ++t)
            segs.push_back(Segment{p0 + t * deg / n, p0 + (t + 1) * deg / n, row, (int32_t)nsplit,
                                   first, (int32_t)n});
        ++nsplit;
    }
    return nsplit;
}

int plan_segments(bpmf_ctx* h, DevSide& d, const std::vector<int32_t>& order)
{
    std::vector<Segment> segs;
    const int64_t nsplit = build_segments(d.ptr_h.data(), order, d.n_short, h->split_degree, segs);
    const int64_t nsegs = (int64_t)segs.size();
    if (nsegs > d.seg_cap) {
        if (!alloc_n(h, &d.segs, (size_t)nsegs) ||
            !alloc_n(h, &d.part, (size_t)nsegs * warp_partial_floats(h->kp)))
            return BPMF_ENOMEM;
        d.seg_cap = nsegs;
    }
    if (nsplit > d.split_cap) {
        if (!alloc_n(h, &d.seg_done, (size_t)nsplit)) return BPMF_ENOMEM;
        d.split_cap = nsplit;
    }
    cudaError_t e = cudaSuccess;
    if (nsegs)
        e = cudaMemcpyAsync(d.segs, segs.data(), sizeof(Segment) * nsegs, cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess && nsplit)
        e = cudaMemsetAsync(d.seg_done, 0, sizeof(unsigned int) * nsplit, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // `segs` goes out of scope
    if (e != cudaSuccess) return BPMF_ECUDA;
    d.n_segs = nsegs;
    d.n_split = nsplit;
    // the shortest rows (the bin's tail) with at most rank_one_max ratings, never a split row
    int64_t nr1 = 0;
    while (nr1 < d.n_short - nsplit) {
        const int32_t row = order[(size_t)(d.n_short - 1 - nr1)];
        if (d.ptr_h[(size_t)row + 1] - d.ptr_h[(size_t)row] > h->rank_one_max) break;
        ++nr1;
    }
    d.n_rank_one = nr1;
    return BPMF_OK;
}

// Balanced assignment of the tensor-core bin's rows to the CTAs of a launch (the
// paper's workload model, Sec. 4.2: an item costs a fixed part plus a part per rating).
// A row's work is its 64-rating stages plus two; rows go, longest first, each to the CTA
// with the least work so far (longest-processing-time list scheduling).  Made for the two
// grids a launch can have, and only where the plain order (row j to CTA j mod G) would
// leave the busiest CTA more than kPlanImbalance above the mean: a few capped columns of
// 2.7e5 ratings among ten thousand shorter ones put 26% more on some CTAs of the
// 480k x 18k workload's movie launch, while its users are within 2%.
constexpr double kPlanImbalance = 1.05;

int64_t plan_cost(int64_t degree) { return (degree + 63) / 64 + 2; }

// The plan for n items of the given costs (in the order they would be dealt) over G CTAs:
// false when round-robin is kept; else pos[p] = the item at place p, CTA c's items at
// places first[c] .. first[c + 1] - 1 in dealing order.
bool balance_plan(const std::vector<int64_t>& cost, int64_t G, std::vector<int32_t>& pos,
                  std::vector<int64_t>& first)
{
    const int64_t n = (int64_t)cost.size();
    if (G < 1 || n <= G) return false;  // one item per CTA at most: nothing to balance
    int64_t total = 0;
    std::vector<int64_t> rr((size_t)G, 0);
    for (int64_t k = 0; k < n; ++k) {
        rr[(size_t)(k % G)] += cost[(size_t)k];
        total += cost[(size_t)k];
    }
    const int64_t rr_max = *std::max_element(rr.begin(), rr.end());
    if ((double)rr_max * (double)G <= kPlanImbalance * (double)total) return false;
    using Load = std::pair<int64_t, int64_t>;  // (work so far, CTA): ties by CTA index
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> least;
    for (int64_t c = 0; c < G; ++c) least.push({0, c});
    std::vector<int32_t> owner((size_t)n);
    for (int64_t k = 0; k < n; ++k) {
        Load l = least.top();
        least.pop();
        owner[(size_t)k] = (int32_t)l.second;
        l.first += cost[(size_t)k];
        least.push(l);
    }
    first.assign((size_t)G + 1, 0);
    for (int64_t k = 0; k < n; ++k) ++first[(size_t)owner[(size_t)k] + 1];
    for (int64_t c = 0; c < G; ++c) first[(size_t)c + 1] += first[(size_t)c];
    std::vector<int64_t> fill(first.begin(), first.end() - 1);
    pos.resize((size_t)n);
    for (int64_t k = 0; k < n; ++k) pos[(size_t)fill[(size_t)owner[(size_t)k]]++] = (int32_t)k;
    return true;
}

// Plan costs of the long bin's rows (order[n_short ..]), longest first.
void long_bin_costs(const int64_t* ptr, const std::vector<int32_t>& order, int64_t n_short,
                    int64_t n_long, std::vector<int64_t>& cost)
{
    cost.resize((size_t)n_long);
    for (int64_t k = 0; k < n_long; ++k) {
        const int32_t row = order[(size_t)(n_short + k)];
        cost[(size_t)k] = plan_cost(ptr[row + 1] - ptr[row]);
    }
}

int plan_long_bin(bpmf_ctx* h, DevSide& d, const std::vector<int32_t>& order)
{
    d.plan_grid[0] = d.plan_grid[1] = 0;
    const int64_t n = d.n_long;
    if (!h->tc || n == 0) return BPMF_OK;
    std::vector<int64_t> cost;
    long_bin_costs(d.ptr_h.data(), order, d.n_short, n, cost);
    std::vector<int32_t> pos, plan((size_t)n);
    std::vector<int64_t> first;
    for (int q = 0; q < 2; ++q) {
        const int64_t G = std::min<int64_t>(n, (int64_t)kGramCtasPerSm * (h->num_sms - q));
        if (!balance_plan(cost, G, pos, first)) continue;
        for (int64_t p = 0; p < n; ++p) plan[(size_t)p] = order[(size_t)(d.n_short + pos[(size_t)p])];
        if (n > d.plan_cap[q]) {
            if (!alloc_n(h, &d.plan_rows[q], (size_t)n)) return BPMF_ENOMEM;
            d.plan_cap[q] = n;
        }
        // CTA offsets for the largest grid a Gram launch can have
        if (!d.plan_first[q] && !alloc_n(h, &d.plan_first[q], (size_t)kGramCtasPerSm * h->num_sms + 1))
            return BPMF_ENOMEM;
        cudaError_t e = cudaMemcpyAsync(d.plan_rows[q], plan.data(), sizeof(int32_t) * n,
                                        cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d.plan_first[q], first.data(), sizeof(int64_t) * (G + 1),
                                cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // host vectors are reused
        if (e != cudaSuccess) return BPMF_ECUDA;
        d.plan_grid[q] = G;
    }
    return BPMF_OK;
}

// Bins of one side (every row in the short bin when the tensor-core kernel is off),
// the split of its long CUDA-core rows and the balanced plan of its tensor-core rows.
int bin_side(bpmf_ctx* h, DevSide& d, std::vector<int32_t>& order)
{
    ++h->bins_version;
    // the rows of this handle's shard (every row unless restricted), as global row ids
    bin_rows(d.shard_hi - d.shard_lo, d.ptr_h.data() + d.shard_lo, h->tc ? h->long_min : INT64_MAX,
             order, &d.n_short, &d.n_long, &d.long_ratings);
    if (d.shard_lo)
        for (int32_t& r : order) r += (int32_t)d.shard_lo;
    if (h->tc && d.n_long > h->gram_cap) {
        // the scratch grows to the longest long bin; the old one is no longer referenced
        // (the stream is idle here: binning waits for it)
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return BPMF_ECUDA;
        dfree(h, h->gram);
        h->gram = nullptr;
        h->gram_cap = 0;
        if (!alloc_n(h, &h->gram, (size_t)d.n_long * kGramSlotFloats)) return BPMF_ENOMEM;
        h->gram_cap = d.n_long;
    }
    cudaError_t e = cudaMemcpyAsync(d.bin_rows, order.data(), sizeof(int32_t) * order.size(),
                                    cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return BPMF_ECUDA;
    const int rc = plan_segments(h, d, order);  // waits for the stream: `order` may be reused
    if (rc != BPMF_OK) return rc;
    return plan_long_bin(h, d, order);
}

int sync_status(bpmf_ctx* h)
{
    Control c;
    cudaError_t e = cudaMemcpyAsync(&c, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return BPMF_ECUDA;
    // a timed-out wait comes first: the launches after it may report what it left behind
    if (c.status & kStatusTimeout) return BPMF_ETIMEOUT;
    if (c.status & kStatusNotPD) return BPMF_ENOTPD;
    if (c.status & kStatusNaN) return BPMF_ENAN;
    if (c.status & kStatusGamma) return BPMF_EGAMMA;
    return BPMF_OK;
}

// Hyper step of side s on `st`; sweep_offset = 1 draws the next sweep's
// hyper-parameters (the device sweep counter has not advanced yet).
// The Normal-Wishart draw's arguments for side s (also the reduction's draw blocks).
NWArgs nw_args(bpmf_ctx* h, int s, uint32_t sweep_offset)
{
    DevSide& d = h->side[s];
    NWArgs a;
    memset(&a, 0, sizeof(a));
    a.sums = d.sums;
    a.shift64 = d.shift64;
    a.n = d.rows;
    a.K = h->K;
    a.kp = h->kp;
    a.beta0 = h->p.beta0;
    a.nu0 = h->p.nu0;
    a.mu0 = h->mu0_d;
    a.W0inv = h->W0inv_d;
    a.seed = h->p.seed;
    a.sweep_offset = sweep_offset;
    a.c3_normal = d.tag_hyper;
    a.c3_gamma = d.tag_gamma;
    a.ctl = h->ctl;
    a.stats = d.stats;
    a.mu64 = d.mu64;
    a.lam64 = d.lam64;
    a.lam32 = d.lam32;
    a.lammu32 = d.lammu32;
    a.draws = d.nw_draws;
    // a few partials are combined by the draw kernel itself, more by their own launch
    a.partials = d.partials;
    a.nparts = d.red_blocks <= kFuseCombineBlocks ? d.red_blocks : 0;
    return a;
}

int phase_hyper(bpmf_ctx* h, int s, cudaStream_t st, uint32_t sweep_offset)
{
    DevSide& d = h->side[s];
    // shift + partials + random draws in one launch, then the combine when the draw
    // kernel does not do it, then the draw
    const NWArgs a = nw_args(h, s, sweep_offset);
    const bool fuse = a.nparts > 0;
    cudaError_t e = launch_hyper_stats_draws(d.X, d.rows, h->K, h->kp, d.shift64, d.partials,
                                             d.red_blocks, a, st);
    if (e == cudaSuccess && !fuse) e = launch_hyper_combine(d.partials, d.red_blocks, h->kp, d.sums, st);
    if (e != cudaSuccess) return BPMF_ECUDA;
    h->launches += fuse ? 2 : 3;
    return cuda_rc(launch_nw_sample(a, st));
}

// The row kernels' arguments for side s, set for the short bin (the CUDA-core kernel).
RowArgs row_args(bpmf_ctx* h, int s)
{
    DevSide& d = h->side[s];
    const DevSide& o = h->side[1 - s];
    RowArgs a;
    memset(&a, 0, sizeof(a));
    a.ptr = d.ptr;
    a.idx = d.idx;
    a.val = d.val;
    a.Y = o.X;
    a.ldy = h->kp;
    a.X = d.X;
    a.Xh = d.Xh;
    a.Xl = d.Xl;
    a.Yh = o.Xh;
    a.Yl = o.Xl;
    a.ldx = h->kp;
    a.means = d.means;
    a.lam = d.lam32;
    a.lam_ct = d.lam32 + (size_t)h->kp * h->kp;
    a.lamchol_ct = d.lam32 + (size_t)2 * h->kp * h->kp;
    a.lammu = d.lammu32;
    a.ctl = h->ctl;
    a.seed = h->p.seed;
    a.c3 = d.tag_row;
    a.K = h->K;
    a.alpha = (float)h->p.alpha;
    a.timeout_ns = (int64_t)(h->p.wait_timeout_ms > 0 ? h->p.wait_timeout_ms : kDefaultWaitTimeoutMs) *
                   1000000LL;
    a.test_stall = (h->p.flags & BPMF_TEST_STALL) ? 1 : 0;
    a.bf16 = (h->p.flags & BPMF_BF16_GRAM) ? 1 : 0;
    // the short bin (every row when the tensor-core kernel is off) on the CUDA-core
    // kernel, its longest rows as segments
    a.rows = d.bin_rows;
    a.nrows = d.n_short;
    a.segs = d.segs;
    a.nsegs = d.n_segs;
    a.nsplit = d.n_split;
    a.part = d.part;
    a.seg_done = d.seg_done;
    a.nrank_one = d.n_rank_one;
    return a;
}

// The same arguments turned to the long bin (the tensor-core route) for a Gram launch
// over row_sms SMs: the balanced plan made for that grid, when there is one.
void long_bin_args(bpmf_ctx* h, int s, RowArgs& a)
{
    const DevSide& d = h->side[s];
    a.nsegs = a.nsplit = a.nrank_one = 0;
    a.rows = d.bin_rows + d.n_short;
    a.nrows = d.n_long;
    const int64_t grid = std::min<int64_t>(d.n_long, (int64_t)kGramCtasPerSm * h->row_sms);  // the Gram launch's CTAs
    for (int q = 0; q < 2; ++q)
        if (d.plan_grid[q] > 0 && d.plan_grid[q] == grid) {
            a.rows = d.plan_rows[q];
            a.cta_first = d.plan_first[q];
            a.plan_grid = grid;
        }
    a.gram = h->gram;
}

// timed: record events around the CUDA-core and tensor-core launches (bpmf_step only,
// never inside a captured sweep)
int phase_rows(bpmf_ctx* h, int s, bool timed = false)
{
    const DevSide& d = h->side[s];
    RowArgs a = row_args(h, s);
    cudaError_t e = cudaSuccess;
    timed = timed && h->row_timing;
    if (timed) {
        h->timed_parts = (a.nrows > 0 ? 1 : 0) | (d.n_long > 0 ? 2 : 0);
        e = cudaEventRecord(h->tev[0], h->stream);
    }
    if (e == cudaSuccess && a.nrows > 0) {
        h->launches += rows_warp_launches(a);
        e = launch_rows_warp(a, h->kp, h->row_sms, h->stream);
    }
    if (e == cudaSuccess && timed) e = cudaEventRecord(h->tev[1], h->stream);
    long_bin_args(h, s, a);
    if (e == cudaSuccess && a.nrows > 0) {
        h->launches += 1;
        e = launch_rows_gram(a, h->row_sms, h->stream);
    }
    if (e == cudaSuccess && timed) e = cudaEventRecord(h->tev[2], h->stream);
    if (e == cudaSuccess && a.nrows > 0) {
        h->launches += 1;
        e = launch_rows_chol(a, h->row_sms, h->stream);
    }
    if (e == cudaSuccess && timed) e = cudaEventRecord(h->tev[3], h->stream);
    return cuda_rc(e);
}

PredictArgs pred_args(bpmf_ctx* h)
{
    PredictArgs p;
    memset(&p, 0, sizeof(p));
    p.ti = h->ti;
    p.tj = h->tj;
    p.tr = h->tr;
    p.T = h->T;
    p.U = h->side[BPMF_USER].X;
    p.V = h->side[BPMF_MOVIE].X;
    p.ld = p.kp = h->kp;
    p.rbar = h->rbar;
    p.clip = (h->p.flags & BPMF_CLIP) ? 1 : 0;
    p.lo = h->p.clip_lo;
    p.hi = h->p.clip_hi;
    p.burn_in = h->p.burn_in;
    p.psum = h->psum;
    p.ctl = h->ctl;
    p.partials = h->pred_partials;
    return p;
}

int phase_predict(bpmf_ctx* h)
{
    const DevSide& u = h->side[BPMF_USER];
    const DevSide& v = h->side[BPMF_MOVIE];
    cudaError_t e = cudaSuccess;
    if (h->T > 0)
        e = launch_predict(h->ti, h->tj, h->tr, h->T, u.X, v.X, h->kp, h->kp, h->rbar,
                           (h->p.flags & BPMF_CLIP) ? 1 : 0, h->p.clip_lo, h->p.clip_hi,
                           h->p.burn_in, h->psum, h->ctl, h->pred_partials, h->pred_blocks,
                           h->stream);
    if (e == cudaSuccess)
        e = launch_predict_finish(h->pred_partials, h->T > 0 ? h->pred_blocks : 0, h->T,
                                  h->p.burn_in, h->ctl, h->stream);
    h->launches += h->T > 0 ? 2 : 1;
    return cuda_rc(e);
}

// Host-side NVTX range for the lifetime of a scope (annotates the enqueue of a phase or a
// sweep call for a profiler's timeline; a no-op without a tool attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

const char* phase_name(int phase)
{
    switch (phase) {
    case BPMF_PHASE_HYPER_USER: return "bpmf hyper users";
    case BPMF_PHASE_HYPER_MOVIE: return "bpmf hyper movies";
    case BPMF_PHASE_ROWS_USER: return "bpmf rows users";
    case BPMF_PHASE_ROWS_MOVIE: return "bpmf rows movies";
    case BPMF_PHASE_PREDICT: return "bpmf predict";
    default: return "bpmf advance";
    }
}

// timed: bpmf_step's call (row phases may record their launch events)
int run_phase(bpmf_ctx* h, int phase, bool timed = false)
{
    const NvtxRange range(phase_name(phase));
    switch (phase) {
    case BPMF_PHASE_HYPER_USER: return phase_hyper(h, BPMF_USER, h->stream, 0);
    case BPMF_PHASE_HYPER_MOVIE: return phase_hyper(h, BPMF_MOVIE, h->stream, 0);
    case BPMF_PHASE_ROWS_USER: return phase_rows(h, BPMF_USER, timed);
    case BPMF_PHASE_ROWS_MOVIE: return phase_rows(h, BPMF_MOVIE, timed);
    case BPMF_PHASE_PREDICT: return phase_predict(h);
    case BPMF_PHASE_ADVANCE: h->launches += 1; return cuda_rc(launch_advance(h->ctl, h->stream));
    default: return BPMF_EINVAL;
    }
}

int copy_packed_d2h(const float* dev, int64_t rows, int K, int ld, float* host, cudaStream_t s)
{
    if (rows == 0) return BPMF_OK;
    return cuda_rc(cudaMemcpy2DAsync(host, sizeof(float) * K, dev, sizeof(float) * ld,
                                     sizeof(float) * K, (size_t)rows, cudaMemcpyDeviceToHost, s));
}

}  // namespace

extern "C" {

int bpmf_default_params(bpmf_params* p)
{
    if (!p) return BPMF_EINVAL;
    memset(p, 0, sizeof(*p));
    p->alpha = 2.0;
    p->beta0 = 2.0;
    p->nu0 = 0.0;  // 0 = K
    p->clip_lo = 1.0;
    p->clip_hi = 5.0;
    return BPMF_OK;
}

const char* bpmf_strerror(int code)
{
    switch (code) {
    case BPMF_OK: return "ok";
    case BPMF_EINVAL: return "invalid argument";
    case BPMF_ENOMEM: return "out of memory";
    case BPMF_ECUDA: return "CUDA runtime error";
    case BPMF_ENOTPD: return "precision matrix not positive definite";
    case BPMF_ETIMEOUT: return "device wait timed out";
    case BPMF_ENAN: return "NaN or Inf produced";
    case BPMF_EGAMMA: return "gamma sampler exhausted its attempts";
    default: return "unknown error";
    }
}

int bpmf_destroy(bpmf_handle h)
{
    if (!h) return BPMF_OK;
    cudaStreamSynchronize(h->stream);
    if (h->aux) {
        cudaStreamSynchronize(h->aux);
        cudaStreamDestroy(h->aux);
    }
    if (h->sweep_graph) cudaGraphExecDestroy(h->sweep_graph);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->tev)
        if (e) cudaEventDestroy(e);
    for (void* ptr : h->allocs) {
        if (h->p.free) h->p.free(ptr, (void*)h->stream, h->p.alloc_ctx);
        else cudaFree(ptr);
    }
    delete h;
    return BPMF_OK;
}

int bpmf_create(bpmf_handle* out, int64_t M, int64_t N, int32_t K, const int64_t* csr_ptr,
                const int32_t* csr_col, const float* csr_val, const int64_t* csc_ptr,
                const int32_t* csc_row, const float* csc_val, int64_t T, const int32_t* test_i,
                const int32_t* test_j, const float* test_r, const bpmf_params* p,
                void* cuda_stream)
{
    if (!out) return BPMF_EINVAL;
    *out = nullptr;
    if (M <= 0 || N <= 0 || M > INT32_MAX || N > INT32_MAX || K < 1 || K > kMaxK || T < 0)
        return BPMF_EINVAL;
    if (!csr_ptr || (!csr_col && csr_ptr[M] > 0) || (!csr_val && csr_ptr[M] > 0)) return BPMF_EINVAL;
    if (T > 0 && (!test_i || !test_j || !test_r)) return BPMF_EINVAL;
    const bool have_csc = csc_ptr || csc_row || csc_val;
    if (have_csc && !(csc_ptr && (csc_ptr[N] == 0 || (csc_row && csc_val)))) return BPMF_EINVAL;
    bpmf_params prm;
    if (p) prm = *p;
    else bpmf_default_params(&prm);
    if (prm.nu0 == 0.0) prm.nu0 = (double)K;
    if (!(prm.alpha > 0.0) || !(prm.beta0 > 0.0) || !(prm.nu0 >= (double)K)) return BPMF_EINVAL;
    if (prm.order != 0 && prm.order != 1) return BPMF_EINVAL;
    // The column view is always built by the library from the row view: on the device
    // when the ratings fit 32-bit positions (the column indices of the row view are then
    // checked there, in one pass with the mean), else on the host.  A column view the
    // caller passes must equal it entry by entry (rows ascending in each column), else
    // BPMF_EINVAL: the same ratings in two views that disagree would give a chain of
    // another matrix.
    if (!valid_ptr(M, csr_ptr)) return BPMF_EINVAL;
    const bool device_csc = csr_ptr[M] > 0 && csr_ptr[M] < INT32_MAX;
    if (!device_csc && !valid_csr(M, N, csr_ptr, csr_col)) return BPMF_EINVAL;
    if (have_csc) {
        if (!valid_csr(N, M, csc_ptr, csc_row) || csc_ptr[N] != csr_ptr[M]) return BPMF_EINVAL;
    }
    for (int64_t t = 0; t < T; ++t)
        if (test_i[t] < 0 || test_i[t] >= M || test_j[t] < 0 || test_j[t] >= N) return BPMF_EINVAL;

    bpmf_ctx* h = new (std::nothrow) bpmf_ctx();
    if (!h) return BPMF_ENOMEM;
    h->p = prm;
    h->M = M;
    h->N = N;
    h->K = K;
    h->kp = (K + 15) / 16 * 16;
    h->tc = h->kp == 64 && !(prm.flags & BPMF_CUDA_CORE_GRAM);
    // the BF16 Gram is a mode of the tensor-core kernel
    if ((prm.flags & BPMF_BF16_GRAM) && !h->tc) {
        delete h;
        return BPMF_EINVAL;
    }
    h->T = T;
    h->nnz = csr_ptr[M];
    h->stream = (cudaStream_t)cuda_stream;
    h->mu0.assign(K, 0.0);
    h->W0.assign((size_t)K * K, 0.0);
    for (int k = 0; k < K; ++k) h->mu0[k] = prm.mu0 ? prm.mu0[k] : 0.0;
    for (int i = 0; i < K * K; ++i) h->W0[i] = prm.W0 ? prm.W0[i] : (i / K == i % K ? 1.0 : 0.0);
    h->p.mu0 = nullptr;
    h->p.W0 = nullptr;
    std::vector<double> W0inv;
    if (!host_spd_inverse(K, h->W0.data(), W0inv)) {
        delete h;
        return BPMF_EINVAL;
    }
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return BPMF_ECUDA;
    }
    h->row_sms = h->num_sms;
    for (cudaEvent_t& e : h->ev) {
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            bpmf_destroy(h);
            return BPMF_ECUDA;
        }
    }
    std::vector<int64_t> cp;
    std::vector<int32_t> ri;
    std::vector<float> cv;
    // the column view built on the host when it is not built on the device (same order
    // as the device build); a caller's view is compared with it here
    if (!device_csc) {
        build_csc(M, N, csr_ptr, csr_col, csr_val, cp, ri, cv);
        if (have_csc) {
            const int64_t nz = csr_ptr[M];
            const bool same = std::equal(cp.begin(), cp.end(), csc_ptr) &&
                              std::equal(ri.begin(), ri.end(), csc_row) &&
                              std::equal(cv.begin(), cv.end(), csc_val, [](float a, float b) {
                                  return memcmp(&a, &b, sizeof(float)) == 0;
                              }) && (int64_t)ri.size() == nz;
            if (!same) {
                bpmf_destroy(h);
                return BPMF_EINVAL;
            }
        }
    }
    const int64_t* user_csc_ptr = csc_ptr;
    const int32_t* user_csc_row = csc_row;
    const float* user_csc_val = csc_val;
    if (!device_csc) {
        csc_ptr = cp.data();
        csc_row = ri.data();
        csc_val = cv.data();
    }
    const int64_t long_min = prm.long_min_degree > 0 ? prm.long_min_degree : default_long_min(prm.flags);
    h->long_min = long_min;
    h->split_degree = prm.split_degree > 0 ? prm.split_degree : kDefaultSplitDegree;
    h->rank_one_max = rank_one_from(prm.rank_one_degree);
    const int64_t* hp[2] = {csr_ptr, device_csc ? nullptr : csc_ptr};
    const int32_t* hi[2] = {csr_col, csc_row};
    const float* hv[2] = {csr_val, csc_val};
    const int64_t rows[2] = {M, N};
    int rc = BPMF_OK;
    const int kp = h->kp;
    cudaStream_t st = h->stream;
    std::vector<int32_t> order;
    for (int s = 0; s < 2 && rc == BPMF_OK; ++s) {
        DevSide& d = h->side[s];
        d.rows = rows[s];
        d.shard_lo = 0;
        d.shard_hi = d.rows;
        d.tag_init = tag_word(s == 0 ? kTagInitU : kTagInitV, prm.job_id);
        d.tag_row = tag_word(s == 0 ? kTagRowU : kTagRowV, prm.job_id);
        d.tag_hyper = tag_word(s == 0 ? kTagHyperU : kTagHyperV, prm.job_id);
        d.tag_gamma = tag_word(s == 0 ? kTagGammaU : kTagGammaV, prm.job_id);
        d.red_blocks = hyper_reduce_blocks(d.rows, h->num_sms);
        bool ok = alloc_n(h, &d.ptr, d.rows + 1) && alloc_n(h, &d.idx, h->nnz) &&
                  alloc_n(h, &d.val, h->nnz) && alloc_n(h, &d.X, (size_t)d.rows * kp) &&
                  alloc_n(h, &d.bin_rows, d.rows) && alloc_n(h, &d.mu64, K) && alloc_n(h, &d.shift64, kp) &&
                  alloc_n(h, &d.lam64, (size_t)K * K) && alloc_n(h, &d.nw_draws, nw_draws_doubles(K)) &&
                  alloc_n(h, &d.lam32, (size_t)3 * kp * kp) &&
                  alloc_n(h, &d.lammu32, kp) &&
                  alloc_n(h, &d.partials, (size_t)d.red_blocks * hyper_partial_doubles(kp)) &&
                  alloc_n(h, &d.sums, hyper_partial_doubles(kp)) &&
                  alloc_n(h, &d.stats, (size_t)K + (size_t)K * K);
        if (ok && (prm.flags & BPMF_DEBUG_MEANS)) ok = alloc_n(h, &d.means, (size_t)d.rows * kp);
        if (ok && h->tc)
            ok = alloc_n(h, &d.Xh, (size_t)d.rows * kp) && alloc_n(h, &d.Xl, (size_t)d.rows * kp);
        if (!ok) {
            rc = BPMF_ENOMEM;
            break;
        }
        cudaError_t e = cudaSuccess;
        const bool built = s == 1 && device_csc;
        if (built) {
            // from the user side's arrays, whose values are already centred (centring
            // is per entry, so gathering centred values equals centring gathered ones)
            const DevSide& u = h->side[0];
            const TempAlloc tmp{temp_alloc, temp_free, h};
            e = build_csc_device(u.ptr, u.idx, u.val, M, N, h->nnz, d.ptr, d.idx, d.val, tmp, st);
            if (e == cudaSuccess && have_csc) {
                bool same = false;
                e = check_csc_device(d.ptr, d.idx, d.val, user_csc_ptr, user_csc_row, user_csc_val,
                                     N, h->nnz, h->rbar, tmp, &same, st);
                if (e == cudaSuccess && !same) {
                    rc = BPMF_EINVAL;
                    break;
                }
            }
            cp.resize((size_t)N + 1);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(cp.data(), d.ptr, sizeof(int64_t) * (N + 1),
                                    cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            hp[1] = cp.data();
        } else {
            e = cudaMemcpyAsync(d.ptr, hp[s], sizeof(int64_t) * (d.rows + 1), cudaMemcpyHostToDevice,
                                st);
            if (e == cudaSuccess && h->nnz)
                e = cudaMemcpyAsync(d.idx, hi[s], sizeof(int32_t) * h->nnz, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess && h->nnz)
                e = cudaMemcpyAsync(d.val, hv[s], sizeof(float) * h->nnz, cudaMemcpyHostToDevice, st);
        }
        if (e != cudaSuccess) {
            rc = BPMF_ECUDA;
            break;
        }
        if (s == 0) {
            // training mean (FP64, fixed summation order) and the column range check
            double* scratch = nullptr;
            unsigned int* bad = nullptr;
            double sum = 0.0;
            unsigned int bad_h = 0;
            if (!alloc_n(h, &scratch, 1 + (size_t)kCheckSumBlocks) || !alloc_n(h, &bad, 1)) {
                rc = BPMF_ENOMEM;
                break;
            }
            e = launch_check_sum(d.idx, d.val, h->nnz, (int32_t)N, scratch, bad, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&sum, scratch, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&bad_h, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                rc = BPMF_ECUDA;
                break;
            }
            if (bad_h) {
                rc = BPMF_EINVAL;
                break;
            }
            h->rbar = ((prm.flags & BPMF_NO_CENTER) || h->nnz == 0) ? 0.0 : sum / (double)h->nnz;
        }
        d.ptr_h.assign(hp[s], hp[s] + d.rows + 1);
        rc = bin_side(h, d, order);
        if (rc != BPMF_OK) break;
        if (e == cudaSuccess && !built) e = launch_center_values(d.val, h->nnz, h->rbar, st);
        if (e == cudaSuccess) e = launch_init_factors(d.X, d.rows, K, kp, prm.seed, d.tag_init, st);
        if (e == cudaSuccess && d.Xh) e = launch_split_factors(d.X, d.rows, kp, d.Xh, d.Xl, (h->p.flags & BPMF_BF16_GRAM) ? 1 : 0, st);
        if (e == cudaSuccess && d.means) e = cudaMemsetAsync(d.means, 0, sizeof(float) * d.rows * kp, st);
        // initial hyper state: mu = 0, Lambda = I
        std::vector<double> I((size_t)K * K, 0.0);
        for (int k = 0; k < K; ++k) I[(size_t)k * K + k] = 1.0;
        if (e == cudaSuccess) e = cudaMemsetAsync(d.mu64, 0, sizeof(double) * K, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d.lam64, I.data(), sizeof(double) * K * K, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = launch_hyper_refresh(d.mu64, d.lam64, K, kp, d.lam32, d.lammu32, nullptr, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host vectors go out of scope
        if (e != cudaSuccess) rc = BPMF_ECUDA;
    }
    if (rc == BPMF_OK) {
        h->pred_blocks = predict_blocks(T, h->num_sms);
        bool ok = alloc_n(h, &h->mu0_d, K) && alloc_n(h, &h->W0inv_d, (size_t)K * K) &&
                  alloc_n(h, &h->ti, T) && alloc_n(h, &h->tj, T) && alloc_n(h, &h->tr, T) &&
                  alloc_n(h, &h->psum, T) && alloc_n(h, &h->pred_partials, 2 * (size_t)h->pred_blocks) &&
                  alloc_n(h, &h->ctl, 1);
        if (!ok) rc = BPMF_ENOMEM;
    }
    if (rc == BPMF_OK) {
        cudaError_t e = cudaMemcpyAsync(h->mu0_d, h->mu0.data(), sizeof(double) * K,
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->W0inv_d, W0inv.data(), sizeof(double) * K * K,
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && T) e = cudaMemcpyAsync(h->ti, test_i, 4 * T, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && T) e = cudaMemcpyAsync(h->tj, test_j, 4 * T, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && T) e = cudaMemcpyAsync(h->tr, test_r, 4 * T, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && T) e = cudaMemsetAsync(h->psum, 0, sizeof(double) * T, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->ctl, 0, sizeof(Control), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = BPMF_ECUDA;
    }
    if (rc != BPMF_OK) {
        cudaGetLastError();
        bpmf_destroy(h);
        return rc;
    }
    *out = h;
    return BPMF_OK;
}

int bpmf_set_tuning(bpmf_handle h, int32_t long_min_degree, int32_t split_degree,
                    int32_t rank_one_degree)
{
    if (!h) return BPMF_EINVAL;
    h->rank_one_max = rank_one_from(rank_one_degree);
    h->long_min = long_min_degree > 0 ? long_min_degree : default_long_min(h->p.flags);
    h->split_degree = split_degree > 0 ? split_degree : kDefaultSplitDegree;
    std::vector<int32_t> order;
    for (int s = 0; s < 2; ++s) {
        const int rc = bin_side(h, h->side[s], order);
        if (rc != BPMF_OK) return rc;
    }
    // the captured sweep holds the old bins' launch shapes
    if (h->sweep_graph) cudaGraphExecDestroy(h->sweep_graph);
    h->sweep_graph = nullptr;
    h->graph_state = 0;
    return BPMF_OK;
}

int bpmf_step(bpmf_handle h, int32_t phase)
{
    if (!h) return BPMF_EINVAL;
    return run_phase(h, phase, true);
}

namespace {

// Overlapped sweeps: each hyper step runs on the aux stream beside a row phase
// (Alg. 1's data dependencies: the second side's hyper step needs that side's rows
// of the previous sweep only, the first side's needs this sweep's first-side rows):
//   main: [hyper(1st) s0] | rows(1st) | wait H2 | rows(2nd) | predict | wait H1 | advance
//   aux:    wait A: hyper(2nd) s -> H2 | wait R1: hyper(1st) s+1 -> H1
// The row kernels leave one SM to the aux stream.  advance waits for the aux stream, so
// the device sweep counter never moves under a hyper step.

// Start: the first side's hyper step of the first sweep, row kernels on one SM fewer.
int sweep_begin(bpmf_ctx* h, int first)
{
    const int rc = phase_hyper(h, first, h->stream, 0);
    h->row_sms = h->num_sms - 1;
    return rc;
}

void sweep_end(bpmf_ctx* h) { h->row_sms = h->num_sms; }

// One sweep; with next_hyper, also the following sweep's first-side hyper step.
int sweep_body(bpmf_ctx* h, int first, bool next_hyper)
{
    const int second = 1 - first;
    const int rowp[2] = {BPMF_PHASE_ROWS_USER, BPMF_PHASE_ROWS_MOVIE};
    cudaEvent_t evA = h->ev[0], evR1 = h->ev[1], evH2 = h->ev[2], evH1 = h->ev[3];
    int rc = BPMF_OK;
    cudaError_t e = cudaEventRecord(evA, h->stream);
    if (e == cudaSuccess) rc = run_phase(h, rowp[first]);
    if (e == cudaSuccess && rc == BPMF_OK) e = cudaEventRecord(evR1, h->stream);
    if (e == cudaSuccess && rc == BPMF_OK) e = cudaStreamWaitEvent(h->aux, evA, 0);
    if (e == cudaSuccess && rc == BPMF_OK) rc = phase_hyper(h, second, h->aux, 0);
    if (e == cudaSuccess && rc == BPMF_OK) e = cudaEventRecord(evH2, h->aux);
    if (e == cudaSuccess && rc == BPMF_OK && next_hyper) {
        e = cudaStreamWaitEvent(h->aux, evR1, 0);
        if (e == cudaSuccess) rc = phase_hyper(h, first, h->aux, 1);
        if (e == cudaSuccess && rc == BPMF_OK) e = cudaEventRecord(evH1, h->aux);
    }
    if (e == cudaSuccess && rc == BPMF_OK) e = cudaStreamWaitEvent(h->stream, evH2, 0);
    if (e == cudaSuccess && rc == BPMF_OK) rc = run_phase(h, rowp[second]);
    if (e == cudaSuccess && rc == BPMF_OK) rc = run_phase(h, BPMF_PHASE_PREDICT);
    if (e == cudaSuccess && rc == BPMF_OK && next_hyper) e = cudaStreamWaitEvent(h->stream, evH1, 0);
    if (e == cudaSuccess && rc == BPMF_OK) rc = run_phase(h, BPMF_PHASE_ADVANCE);
    if (e != cudaSuccess) rc = BPMF_ECUDA;
    return rc;  // the main stream has waited for everything the aux stream was given
}

// The sweep that is followed by another, captured once per handle into a CUDA graph
// (kernel arguments are fixed per handle; counters are read from device memory).
// Returns false when the stream cannot be captured (the legacy default stream).
bool ensure_sweep_graph(bpmf_ctx* h, int first)
{
    if (h->graph_state != 0) return h->graph_state > 0;
    h->graph_state = -1;
    if (!h->stream) return false;
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int64_t l0 = h->launches;
    const int rc = sweep_body(h, first, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    const int64_t captured = h->launches - l0;
    h->launches = l0;
    if (rc != BPMF_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return false;
    }
    const cudaError_t ei = cudaGraphInstantiate(&h->sweep_graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        h->sweep_graph = nullptr;
        return false;
    }
    h->graph_launches = captured;
    h->graph_state = 1;
    return true;
}

// One sweep of a run that began with sweep_begin; the last one leaves the next
// sweep's hyper step undrawn, so the state after a run is the phase-by-phase one.
int sweep_next(bpmf_ctx* h, int first, bool last)
{
    if (!last && ensure_sweep_graph(h, first)) {
        h->launches += h->graph_launches;
        return cuda_rc(cudaGraphLaunch(h->sweep_graph, h->stream));
    }
    return sweep_body(h, first, !last);
}

int sweep_plain(bpmf_ctx* h, int n_sweeps)
{
    const int first = h->p.order == 0 ? BPMF_MOVIE : BPMF_USER;
    const int second = 1 - first;
    const int hyp[2] = {BPMF_PHASE_HYPER_USER, BPMF_PHASE_HYPER_MOVIE};
    const int rowp[2] = {BPMF_PHASE_ROWS_USER, BPMF_PHASE_ROWS_MOVIE};
    for (int it = 0; it < n_sweeps; ++it) {
        const int seq[6] = {hyp[first], rowp[first], hyp[second], rowp[second], BPMF_PHASE_PREDICT,
                            BPMF_PHASE_ADVANCE};
        for (int ph : seq) {
            const int rc = run_phase(h, ph);
            if (rc) return rc;
        }
    }
    return BPMF_OK;
}

int read_rmse(bpmf_ctx* h, double* rmse_sample, double* rmse_avg)
{
    Control c;
    cudaError_t e = cudaMemcpyAsync(&c, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return BPMF_ECUDA;
    if (rmse_sample) *rmse_sample = c.rmse_sample;
    if (rmse_avg) *rmse_avg = c.rmse_avg;
    // a timed-out wait comes first: the launches after it may report what it left behind
    if (c.status & kStatusTimeout) return BPMF_ETIMEOUT;
    if (c.status & kStatusNotPD) return BPMF_ENOTPD;
    if (c.status & kStatusNaN) return BPMF_ENAN;
    if (c.status & kStatusGamma) return BPMF_EGAMMA;
    return BPMF_OK;
}

}  // namespace

int bpmf_sweep(bpmf_handle h, int32_t n_sweeps, double* rmse_sample, double* rmse_avg)
{
    if (!h || n_sweeps < 0) return BPMF_EINVAL;
    const NvtxRange range("bpmf_sweep");
    if (n_sweeps > 0 && h->num_sms >= 8) {
        const int first = h->p.order == 0 ? BPMF_MOVIE : BPMF_USER;
        int rc = sweep_begin(h, first);
        for (int it = 0; it < n_sweeps && rc == BPMF_OK; ++it) rc = sweep_next(h, first, it + 1 == n_sweeps);
        sweep_end(h);
        if (rc) return rc;
    } else {
        const int rc = sweep_plain(h, n_sweeps);
        if (rc) return rc;
    }
    if (rmse_sample || rmse_avg) return read_rmse(h, rmse_sample, rmse_avg);
    return BPMF_OK;
}

int bpmf_sweep_batch(bpmf_handle* hs, int32_t n, int32_t n_sweeps)
{
    if (n < 0 || n_sweeps < 0 || (n > 0 && !hs)) return BPMF_EINVAL;
    for (int32_t k = 0; k < n; ++k)
        if (!hs[k]) return BPMF_EINVAL;
    int rc = BPMF_OK;
    std::vector<char> overlapped((size_t)n, 0);
    for (int32_t k = 0; k < n && rc == BPMF_OK; ++k) {
        bpmf_ctx* h = hs[k];
        if (n_sweeps > 0 && h->num_sms >= 8) {
            rc = sweep_begin(h, h->p.order == 0 ? BPMF_MOVIE : BPMF_USER);
            overlapped[(size_t)k] = 1;
        }
    }
    // sweep by sweep, job by job: each job's launches go to its own streams, so
    // independent jobs overlap on the device
    for (int32_t it = 0; it < n_sweeps && rc == BPMF_OK; ++it)
        for (int32_t k = 0; k < n && rc == BPMF_OK; ++k) {
            bpmf_ctx* h = hs[k];
            if (overlapped[(size_t)k])
                rc = sweep_next(h, h->p.order == 0 ? BPMF_MOVIE : BPMF_USER, it + 1 == n_sweeps);
            else
                rc = sweep_plain(h, 1);
        }
    for (int32_t k = 0; k < n; ++k)
        if (overlapped[(size_t)k]) sweep_end(hs[k]);
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched sweeps: every step of a sweep runs for all jobs of the batch in one launch
// (per K class where the kernels are compiled per K), with each job's blocks in a table
// the CTAs search; the jobs' tensor-core launches go to forked streams.  One sweep is
// captured as one CUDA graph.
// ---------------------------------------------------------------------------
namespace {

constexpr int kBatchForks = 8;  // streams the tensor-core launches of the jobs fork to

struct BatchLaunch {
    int kind;       // 0 rows (CUDA-core), 1 reduce, 2 combine, 3 draw, 4 predict, 5 finish
    int kp;
    bool rank_one;
    const void* table;
    int n;
    int64_t blocks;
};

}  // namespace

struct bpmf_batch_ctx {
    std::vector<bpmf_ctx*> jobs;
    std::vector<uint64_t> bins_version;  // each job's when its tables were made
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr;  // hyper steps beside the row launches
    cudaEvent_t ev[4] = {};      // sweep-level fork / join
    int first = BPMF_MOVIE;
    int num_sms = 1;
    void* dev = nullptr;  // all tables, one allocation
    // hyper[s]: side s's hyper step for the current sweep; hyper_next: the first side's
    // for the next sweep, drawn before the sweep counter moves (sweep_offset 1)
    std::vector<BatchLaunch> hyper[2], hyper_next, rows[2];
    std::vector<bpmf_ctx*> tc[2];  // jobs with a tensor-core bin on the side
    BatchLaunch predict{}, finish{};
    cudaStream_t fork[kBatchForks] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kBatchForks] = {};
    cudaGraphExec_t graph = nullptr;
    int graph_state = 0;
    int64_t graph_launches = 0;
    int64_t launches = 0;
};

namespace {

// Blocks of a job's CUDA-core row launch in a batch: its share of about sixteen waves
// of the launch's resident CTAs, by the cost model c0 + c1 d of its items, at most one
// block per four items (a warp per item).  Many small blocks of about equal cost keep
// the launch's tail short (4 waves: 112, 8: 116, 16: 117 M rows/s on 256 jobs).
int64_t batch_row_blocks(int64_t items, double cost, double total_cost, int64_t waves_blocks)
{
    int64_t want = (int64_t)std::llround((double)waves_blocks * cost / std::max(total_cost, 1.0));
    want = std::max<int64_t>(want, 1);
    return std::min<int64_t>(want, (items + 3) / 4);
}

template <class A>
struct TableBuilder {
    std::vector<BatchEntry<A>> entries;
    int64_t blocks = 0;
    void add(const A& a, int64_t count)
    {
        BatchEntry<A> e;
        e.args = a;
        e.first = (int32_t)blocks;
        e.count = (int32_t)count;
        entries.push_back(e);
        blocks += count;
    }
};

// Stream order between the jobs' streams and the batch stream (outside any capture).
int batch_order(bpmf_batch_ctx* b, bool jobs_first)
{
    for (bpmf_ctx* h : b->jobs) {
        cudaEvent_t ev = h->ev[0];
        cudaStream_t from = jobs_first ? h->stream : b->stream;
        cudaStream_t to = jobs_first ? b->stream : h->stream;
        if (from == to) continue;
        if (cudaEventRecord(ev, from) != cudaSuccess || cudaStreamWaitEvent(to, ev, 0) != cudaSuccess)
            return BPMF_ECUDA;
    }
    return BPMF_OK;
}

int batch_run(bpmf_batch_ctx* b, const std::vector<BatchLaunch>& ls, cudaStream_t st)
{
    for (const BatchLaunch& l : ls) {
        cudaError_t e = cudaSuccess;
        switch (l.kind) {
        case 0:
            e = launch_rows_warp_batch(static_cast<const BatchEntry<RowArgs>*>(l.table), l.n,
                                       l.blocks, l.kp, l.rank_one, st);
            break;
        case 1:
            e = launch_hyper_reduce_batch(static_cast<const BatchEntry<ReduceArgs>*>(l.table), l.n,
                                          l.blocks, l.kp, st);
            break;
        case 2:
            e = launch_hyper_combine_batch(static_cast<const BatchEntry<CombineArgs>*>(l.table), l.n,
                                           l.blocks, st);
            break;
        case 3: e = launch_nw_sample_batch(static_cast<const NWArgs*>(l.table), l.n, st); break;
        case 4:
            e = launch_predict_batch(static_cast<const BatchEntry<PredictArgs>*>(l.table), l.n,
                                     l.blocks, st);
            break;
        default:
            e = launch_predict_finish_batch(static_cast<const BatchEntry<PredictArgs>*>(l.table), l.n,
                                            true, st);
            break;
        }
        if (e != cudaSuccess) return BPMF_ECUDA;
        b->launches += 1;
    }
    return BPMF_OK;
}

// Side s's rows, forked over the batch's streams and joined back: the CUDA-core
// launches (one per K class and route, so that one launch's tail overlaps the next)
// and the jobs' tensor-core launches, heaviest first, round-robin.
int batch_rows(bpmf_batch_ctx* b, int s)
{
    const size_t nl = b->rows[s].size() + b->tc[s].size();
    const int nf = (int)std::min<size_t>(kBatchForks, nl);
    if (nf == 0) return BPMF_OK;
    if (cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess) return BPMF_ECUDA;
    for (int f = 0; f < nf; ++f)
        if (cudaStreamWaitEvent(b->fork[f], b->ev_fork, 0) != cudaSuccess) return BPMF_ECUDA;
    int rc = BPMF_OK;
    size_t k = 0;
    for (const BatchLaunch& l : b->rows[s])
        if (rc == BPMF_OK) rc = batch_run(b, {l}, b->fork[k++ % (size_t)nf]);
    for (size_t q = 0; q < b->tc[s].size() && rc == BPMF_OK; ++q) {
        bpmf_ctx* h = b->tc[s][q];
        cudaStream_t st = b->fork[k++ % (size_t)nf];
        h->row_sms = h->num_sms;
        RowArgs a = row_args(h, s);
        long_bin_args(h, s, a);
        cudaError_t e = launch_rows_gram(a, h->num_sms, st);
        if (e == cudaSuccess) e = launch_rows_chol(a, h->num_sms, st);
        if (e != cudaSuccess) rc = BPMF_ECUDA;
        b->launches += 2;
    }
    for (int f = 0; f < nf && rc == BPMF_OK; ++f)
        if (cudaEventRecord(b->ev_join[f], b->fork[f]) != cudaSuccess ||
            cudaStreamWaitEvent(b->stream, b->ev_join[f], 0) != cudaSuccess)
            rc = BPMF_ECUDA;
    return rc;
}

// One sweep whose first-side hyper step is done (Alg. 1's data dependencies, as in
// bpmf_sweep): the second side's hyper step runs on the aux stream beside the first
// side's rows; with next, the next sweep's first-side hyper step beside the second
// side's rows; the prediction, then the sweep counters move.
int batch_sweep_body(bpmf_batch_ctx* b, bool next)
{
    const int f = b->first, sc = 1 - b->first;
    cudaEvent_t evA = b->ev[0], evR1 = b->ev[1], evH2 = b->ev[2], evH1 = b->ev[3];
    if (cudaEventRecord(evA, b->stream) != cudaSuccess ||
        cudaStreamWaitEvent(b->aux, evA, 0) != cudaSuccess)
        return BPMF_ECUDA;
    int rc = batch_run(b, b->hyper[sc], b->aux);
    if (rc == BPMF_OK && cudaEventRecord(evH2, b->aux) != cudaSuccess) rc = BPMF_ECUDA;
    if (rc == BPMF_OK) rc = batch_rows(b, f);
    if (rc == BPMF_OK && next) {
        if (cudaEventRecord(evR1, b->stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->aux, evR1, 0) != cudaSuccess)
            rc = BPMF_ECUDA;
        if (rc == BPMF_OK) rc = batch_run(b, b->hyper_next, b->aux);
        if (rc == BPMF_OK && cudaEventRecord(evH1, b->aux) != cudaSuccess) rc = BPMF_ECUDA;
    }
    if (rc == BPMF_OK && cudaStreamWaitEvent(b->stream, evH2, 0) != cudaSuccess) rc = BPMF_ECUDA;
    if (rc == BPMF_OK) rc = batch_rows(b, sc);
    if (rc == BPMF_OK && b->predict.n > 0) rc = batch_run(b, {b->predict}, b->stream);
    // the counters move once the next sweep's draw (which reads them) is done
    if (rc == BPMF_OK && next && cudaStreamWaitEvent(b->stream, evH1, 0) != cudaSuccess) rc = BPMF_ECUDA;
    if (rc == BPMF_OK) rc = batch_run(b, {b->finish}, b->stream);
    return rc;  // the batch stream has waited for everything the aux stream was given
}

void batch_free(bpmf_batch_ctx* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->aux) cudaStreamDestroy(b->aux);
    for (cudaEvent_t e : b->ev)
        if (e) cudaEventDestroy(e);
    for (int f = 0; f < kBatchForks; ++f) {
        if (b->fork[f]) cudaStreamDestroy(b->fork[f]);
        if (b->ev_join[f]) cudaEventDestroy(b->ev_join[f]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->dev) cudaFree(b->dev);
    delete b;
}

}  // namespace

extern "C" {

int bpmf_batch_create(bpmf_handle* hs, int32_t n, void* cuda_stream, bpmf_batch* out)
{
    if (!out) return BPMF_EINVAL;
    *out = nullptr;
    if (n < 1 || !hs) return BPMF_EINVAL;
    for (int32_t k = 0; k < n; ++k) {
        if (!hs[k] || hs[k]->device != hs[0]->device || hs[k]->num_sms != hs[0]->num_sms ||
            hs[k]->p.order != hs[0]->p.order)
            return BPMF_EINVAL;
        for (int32_t q = 0; q < k; ++q)
            if (hs[q] == hs[k]) return BPMF_EINVAL;
        for (int s = 0; s < 2; ++s)
            if (hs[k]->side[s].shard_lo != 0 || hs[k]->side[s].shard_hi != hs[k]->side[s].rows)
                return BPMF_EINVAL;
    }
    bpmf_batch_ctx* b = new (std::nothrow) bpmf_batch_ctx();
    if (!b) return BPMF_ENOMEM;
    try {
        b->jobs.assign(hs, hs + n);
        for (int32_t k = 0; k < n; ++k) b->bins_version.push_back(hs[k]->bins_version);
    } catch (const std::bad_alloc&) {
        delete b;
        return BPMF_ENOMEM;
    }
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->first = hs[0]->p.order == 0 ? BPMF_MOVIE : BPMF_USER;
    b->num_sms = hs[0]->num_sms;
    bool ok = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t& e : b->ev)
        ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    for (int f = 0; f < kBatchForks && ok; ++f)
        ok = cudaStreamCreateWithFlags(&b->fork[f], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->ev_join[f], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        return BPMF_ECUDA;
    }
    // host tables; each job's share is what its own launch would be, ordered heaviest
    // first (the work queue in longest-processing-time order of the cost model
    // c0 + c1 d: the CTAs of the heaviest jobs are dispatched first).  Each table is
    // staged in `image` at a 256-B aligned offset, kept in its launch until the one
    // device allocation exists.
    std::vector<char> image;
    auto place = [&](const void* p, size_t bytes) -> const void* {
        const size_t off = image.size();
        image.resize(off + ((bytes + 255) & ~(size_t)255), 0);
        memcpy(image.data() + off, p, bytes);
        return reinterpret_cast<const void*>(off);
    };
    const int kps[4] = {16, 32, 48, 64};
    auto build_hyper = [&](int s, uint32_t offset, std::vector<BatchLaunch>& out) {
        // the reductions (with the draw blocks) by kp, the combines, the draws
        for (int kp : kps) {
            std::vector<std::pair<int64_t, bpmf_ctx*>> order;
            for (bpmf_ctx* h : b->jobs)
                if (h->kp == kp) order.push_back({h->side[s].red_blocks + hyper_draw_blocks(h->K), h});
            if (order.empty()) continue;
            std::stable_sort(order.begin(), order.end(),
                             [](const auto& x, const auto& y) { return x.first > y.first; });
            TableBuilder<ReduceArgs> t;
            for (auto& o : order) {
                bpmf_ctx* h = o.second;
                const DevSide& d = h->side[s];
                ReduceArgs r;
                memset(&r, 0, sizeof(r));
                r.X = d.X;
                r.rows = d.rows;
                r.shiftK = h->K;
                r.shift64 = d.shift64;
                r.partials = d.partials;
                r.nred = d.red_blocks;
                r.draws = nw_args(h, s, offset);
                t.add(r, o.first);
            }
            out.push_back(BatchLaunch{1, kp, false, place(t.entries.data(), t.entries.size() * sizeof(t.entries[0])),
                                      (int)t.entries.size(), t.blocks});
        }
        TableBuilder<CombineArgs> tc;
        for (bpmf_ctx* h : b->jobs) {
            const DevSide& d = h->side[s];
            if (d.red_blocks <= kFuseCombineBlocks) continue;
            CombineArgs c;
            c.partials = d.partials;
            c.nblocks = d.red_blocks;
            c.E = (int)hyper_partial_doubles(h->kp);
            c.sums = d.sums;
            tc.add(c, hyper_combine_blocks(h->kp));
        }
        if (!tc.entries.empty())
            out.push_back(BatchLaunch{2, 0, false, place(tc.entries.data(), tc.entries.size() * sizeof(tc.entries[0])),
                                      (int)tc.entries.size(), tc.blocks});
        std::vector<NWArgs> tn;
        for (bpmf_ctx* h : b->jobs) tn.push_back(nw_args(h, s, offset));
        out.push_back(BatchLaunch{3, 0, false, place(tn.data(), tn.size() * sizeof(tn[0])), (int)tn.size(),
                                  (int64_t)tn.size()});
    };
    try {
        for (int s = 0; s < 2; ++s) {
            build_hyper(s, 0, b->hyper[s]);
            // the CUDA-core row launches by (kp, route); the tensor-core bins per job
            for (int kp : kps)
                for (int r1 = 0; r1 < 2; ++r1) {
                    std::vector<std::pair<double, bpmf_ctx*>> order;
                    double total = 0.0;
                    for (bpmf_ctx* h : b->jobs) {
                        if (h->kp != kp) continue;
                        const RowArgs a = row_args(h, s);
                        const int64_t items = rows_warp_items(a, r1 != 0);
                        if (items <= 0) continue;
                        const DevSide& d = h->side[s];
                        const double ratings = (double)(h->nnz - d.long_ratings);
                        const double cost = 2.0 * (double)items + (r1 ? 0.0 : ratings / 64.0);
                        order.push_back({cost, h});
                        total += cost;
                    }
                    if (order.empty()) continue;
                    std::stable_sort(order.begin(), order.end(),
                                     [](const auto& x, const auto& y) { return x.first > y.first; });
                    const int64_t waves = 16LL * b->num_sms * rows_warp_resident_blocks(kp);
                    TableBuilder<RowArgs> t;
                    for (auto& o : order) {
                        const RowArgs a = row_args(o.second, s);
                        t.add(a, batch_row_blocks(rows_warp_items(a, r1 != 0), o.first, total, waves));
                    }
                    b->rows[s].push_back(BatchLaunch{0, kp, r1 != 0,
                                                     place(t.entries.data(), t.entries.size() * sizeof(t.entries[0])),
                                                     (int)t.entries.size(), t.blocks});
                }
            std::vector<std::pair<int64_t, bpmf_ctx*>> tc;
            for (bpmf_ctx* h : b->jobs)
                if (h->tc && h->side[s].n_long > 0) tc.push_back({h->side[s].long_ratings, h});
            std::stable_sort(tc.begin(), tc.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
            for (auto& o : tc) b->tc[s].push_back(o.second);
        }
        build_hyper(b->first, 1, b->hyper_next);
        TableBuilder<PredictArgs> tp, tf;
        for (bpmf_ctx* h : b->jobs) {
            const PredictArgs p = pred_args(h);
            if (h->T > 0) tp.add(p, h->pred_blocks);
            BatchEntry<PredictArgs> e;
            e.args = p;
            e.first = 0;
            e.count = h->T > 0 ? h->pred_blocks : 0;
            tf.entries.push_back(e);
        }
        b->predict = BatchLaunch{4, 0, false, nullptr, (int)tp.entries.size(), tp.blocks};
        if (!tp.entries.empty())
            b->predict.table = place(tp.entries.data(), tp.entries.size() * sizeof(tp.entries[0]));
        b->finish = BatchLaunch{5, 0, false, place(tf.entries.data(), tf.entries.size() * sizeof(tf.entries[0])),
                                (int)tf.entries.size(), 0};
    } catch (const std::bad_alloc&) {
        batch_free(b);
        return BPMF_ENOMEM;
    }
    if (cudaMalloc(&b->dev, image.size()) != cudaSuccess ||
        cudaMemcpy(b->dev, image.data(), image.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return BPMF_ENOMEM;
    }
    // table offsets into device addresses
    auto fix = [&](BatchLaunch& l) {
        if (l.n > 0) l.table = static_cast<char*>(b->dev) + reinterpret_cast<size_t>(l.table);
    };
    for (int s = 0; s < 2; ++s) {
        for (BatchLaunch& l : b->hyper[s]) fix(l);
        for (BatchLaunch& l : b->rows[s]) fix(l);
    }
    for (BatchLaunch& l : b->hyper_next) fix(l);
    fix(b->predict);
    fix(b->finish);
    *out = b;
    return BPMF_OK;
}

int bpmf_batch_sweep(bpmf_batch b, int32_t n_sweeps)
{
    if (!b || n_sweeps < 0) return BPMF_EINVAL;
    // a job binned again since (bpmf_set_tuning, bpmf_set_shard) no longer matches the
    // tables: the batch must be made again
    for (size_t k = 0; k < b->jobs.size(); ++k)
        if (b->jobs[k]->bins_version != b->bins_version[k]) return BPMF_EINVAL;
    if (n_sweeps == 0) return BPMF_OK;
    const NvtxRange range("bpmf_batch_sweep");
    int rc = batch_order(b, true);
    // the first side's hyper step of the first sweep; the sweeps but the last draw the
    // next one's beside their own work (one captured graph, made on first use when the
    // batch stream can be captured); the last leaves it undrawn, as bpmf_sweep does
    if (rc == BPMF_OK) rc = batch_run(b, b->hyper[b->first], b->stream);
    if (rc == BPMF_OK && n_sweeps > 1 && b->graph_state == 0) {
        b->graph_state = -1;
        if (b->stream && cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const int64_t l0 = b->launches;
            const int rcb = batch_sweep_body(b, true);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
            b->graph_launches = b->launches - l0;
            b->launches = l0;
            if (rcb == BPMF_OK && e == cudaSuccess && g &&
                cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess)
                b->graph_state = 1;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();
    }
    for (int32_t it = 0; it < n_sweeps && rc == BPMF_OK; ++it) {
        const bool last = it + 1 == n_sweeps;
        if (!last && b->graph_state > 0) {
            rc = cuda_rc(cudaGraphLaunch(b->graph, b->stream));
            b->launches += b->graph_launches;
        } else {
            rc = batch_sweep_body(b, !last);
        }
    }
    if (rc == BPMF_OK) rc = batch_order(b, false);
    return rc;
}

int bpmf_batch_launch_count(bpmf_batch b, int64_t* launches)
{
    if (!b || !launches) return BPMF_EINVAL;
    *launches = b->launches;
    return BPMF_OK;
}

int bpmf_batch_destroy(bpmf_batch b)
{
    if (!b) return BPMF_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
    return BPMF_OK;
}

int bpmf_predict(bpmf_handle h, int64_t n, const int32_t* i, const int32_t* j, float* out,
                 int32_t where)
{
    if (!h || n < 0 || (n > 0 && (!i || !j || !out)) || (where != 0 && where != 1)) return BPMF_EINVAL;
    if (n == 0) return BPMF_OK;
    const int clip = (h->p.flags & BPMF_CLIP) ? 1 : 0;
    const DevSide& u = h->side[BPMF_USER];
    const DevSide& v = h->side[BPMF_MOVIE];
    if (where == 1)
        return cuda_rc(launch_predict_points(i, j, n, u.X, v.X, h->kp, h->kp, h->rbar, clip,
                                             h->p.clip_lo, h->p.clip_hi, out, h->stream));
    for (int64_t t = 0; t < n; ++t)
        if (i[t] < 0 || i[t] >= h->M || j[t] < 0 || j[t] >= h->N) return BPMF_EINVAL;
    int32_t *di = nullptr, *dj = nullptr;
    float* dout = nullptr;
    cudaError_t e = cudaMallocAsync(&di, 4 * n, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&dj, 4 * n, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync(&dout, 4 * n, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(di, i, 4 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dj, j, 4 * n, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = launch_predict_points(di, dj, n, u.X, v.X, h->kp, h->kp, h->rbar, clip, h->p.clip_lo,
                                  h->p.clip_hi, dout, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, 4 * n, cudaMemcpyDeviceToHost, h->stream);
    if (di) cudaFreeAsync(di, h->stream);
    if (dj) cudaFreeAsync(dj, h->stream);
    if (dout) cudaFreeAsync(dout, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return BPMF_ECUDA;
    }
    return BPMF_OK;
}

int bpmf_get_state(bpmf_handle h, float* U, float* V, double* hyper, uint64_t* sweep)
{
    if (!h) return BPMF_EINVAL;
    const int K = h->K;
    int rc = BPMF_OK;
    if (U) rc = copy_packed_d2h(h->side[0].X, h->M, K, h->kp, U, h->stream);
    if (!rc && V) rc = copy_packed_d2h(h->side[1].X, h->N, K, h->kp, V, h->stream);
    if (!rc && hyper) {
        double* o = hyper;
        for (int s = 0; s < 2 && !rc; ++s) {
            rc = cuda_rc(cudaMemcpyAsync(o, h->side[s].mu64, sizeof(double) * K,
                                         cudaMemcpyDeviceToHost, h->stream));
            if (!rc)
                rc = cuda_rc(cudaMemcpyAsync(o + K, h->side[s].lam64, sizeof(double) * K * K,
                                             cudaMemcpyDeviceToHost, h->stream));
            o += K + K * K;
        }
    }
    Control c;
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(&c, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, h->stream));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(h->stream));
    if (!rc && sweep) *sweep = c.sweep;
    return rc;
}

int bpmf_set_state(bpmf_handle h, const float* U, const float* V, const double* hyper,
                   uint64_t sweep)
{
    if (!h) return BPMF_EINVAL;
    const int K = h->K, kp = h->kp;
    cudaStream_t st = h->stream;
    const float* src[2] = {U, V};
    int rc = BPMF_OK;
    for (int s = 0; s < 2 && !rc; ++s) {
        if (!src[s]) continue;
        DevSide& d = h->side[s];
        rc = cuda_rc(cudaMemsetAsync(d.X, 0, sizeof(float) * d.rows * kp, st));
        if (!rc)
            rc = cuda_rc(cudaMemcpy2DAsync(d.X, sizeof(float) * kp, src[s], sizeof(float) * K,
                                           sizeof(float) * K, (size_t)d.rows,
                                           cudaMemcpyHostToDevice, st));
        if (!rc && d.Xh) rc = cuda_rc(launch_split_factors(d.X, d.rows, kp, d.Xh, d.Xl, (h->p.flags & BPMF_BF16_GRAM) ? 1 : 0, st));
    }
    if (!rc && hyper) {
        const double* in = hyper;
        for (int s = 0; s < 2 && !rc; ++s) {
            DevSide& d = h->side[s];
            rc = cuda_rc(cudaMemcpyAsync(d.mu64, in, sizeof(double) * K, cudaMemcpyHostToDevice, st));
            if (!rc)
                rc = cuda_rc(cudaMemcpyAsync(d.lam64, in + K, sizeof(double) * K * K,
                                             cudaMemcpyHostToDevice, st));
            if (!rc)
                rc = cuda_rc(launch_hyper_refresh(d.mu64, d.lam64, K, kp, d.lam32, d.lammu32, h->ctl, st));
            in += K + K * K;
        }
    }
    if (!rc) {
        unsigned long long sw = sweep;
        rc = cuda_rc(cudaMemcpyAsync(&h->ctl->sweep, &sw, sizeof(sw), cudaMemcpyHostToDevice, st));
    }
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(st));
    return rc;
}

int bpmf_get_accum(bpmf_handle h, double* psum, int64_t* n_avg)
{
    if (!h) return BPMF_EINVAL;
    int rc = BPMF_OK;
    if (psum && h->T)
        rc = cuda_rc(cudaMemcpyAsync(psum, h->psum, sizeof(double) * h->T, cudaMemcpyDeviceToHost,
                                     h->stream));
    Control c;
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(&c, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, h->stream));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(h->stream));
    if (!rc && n_avg) *n_avg = c.n_avg;
    return rc;
}

int bpmf_set_accum(bpmf_handle h, const double* psum, int64_t n_avg)
{
    if (!h || n_avg < 0) return BPMF_EINVAL;
    int rc = BPMF_OK;
    if (psum && h->T)
        rc = cuda_rc(cudaMemcpyAsync(h->psum, psum, sizeof(double) * h->T, cudaMemcpyHostToDevice,
                                     h->stream));
    long long na = n_avg;
    if (!rc)
        rc = cuda_rc(cudaMemcpyAsync(&h->ctl->n_avg, &na, sizeof(na), cudaMemcpyHostToDevice, h->stream));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(h->stream));
    return rc;
}

int bpmf_get_stats(bpmf_handle h, int32_t side, int64_t* n, double* mean, double* S)
{
    if (!h || (side != 0 && side != 1)) return BPMF_EINVAL;
    const int K = h->K;
    const DevSide& d = h->side[side];
    int rc = BPMF_OK;
    if (mean) rc = cuda_rc(cudaMemcpyAsync(mean, d.stats, sizeof(double) * K, cudaMemcpyDeviceToHost, h->stream));
    if (!rc && S)
        rc = cuda_rc(cudaMemcpyAsync(S, d.stats + K, sizeof(double) * K * K, cudaMemcpyDeviceToHost,
                                     h->stream));
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(h->stream));
    if (!rc && n) *n = d.rows;
    return rc;
}

int bpmf_debug_means(bpmf_handle h, int32_t side, float* out)
{
    if (!h || (side != 0 && side != 1) || !out) return BPMF_EINVAL;
    const DevSide& d = h->side[side];
    if (!d.means) return BPMF_EINVAL;
    int rc = copy_packed_d2h(d.means, d.rows, h->K, h->kp, out, h->stream);
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(h->stream));
    return rc;
}

int bpmf_status(bpmf_handle h)
{
    if (!h) return BPMF_EINVAL;
    return sync_status(h);
}

int bpmf_set_row_timing(bpmf_handle h, int32_t on)
{
    if (!h) return BPMF_EINVAL;
    if (on && !h->tev[0]) {
        for (cudaEvent_t& e : h->tev) {
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return BPMF_ECUDA;
            }
        }
    }
    h->row_timing = on != 0;
    h->timed_parts = 0;
    return BPMF_OK;
}

int bpmf_row_launch_ms(bpmf_handle h, float* cuda_core_ms, float* gram_ms, float* chol_ms)
{
    if (!h || !cuda_core_ms || !gram_ms || !chol_ms) return BPMF_EINVAL;
    *cuda_core_ms = *gram_ms = *chol_ms = -1.f;
    if (!h->row_timing || !h->timed_parts) return BPMF_OK;
    if (cudaEventSynchronize(h->tev[3]) != cudaSuccess) return BPMF_ECUDA;
    float a = 0.f, b = 0.f, c = 0.f;
    if (cudaEventElapsedTime(&a, h->tev[0], h->tev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&b, h->tev[1], h->tev[2]) != cudaSuccess ||
        cudaEventElapsedTime(&c, h->tev[2], h->tev[3]) != cudaSuccess) {
        cudaGetLastError();
        return BPMF_ECUDA;
    }
    if (h->timed_parts & 1) *cuda_core_ms = a;
    if (h->timed_parts & 2) {
        *gram_ms = b;
        *chol_ms = c;
    }
    return BPMF_OK;
}

int bpmf_launch_count(bpmf_handle h, int64_t* launches)
{
    if (!h || !launches) return BPMF_EINVAL;
    *launches = h->launches;
    return BPMF_OK;
}

int bpmf_set_shard(bpmf_handle h, int32_t side, int64_t row_begin, int64_t row_end)
{
    if (!h || (side != 0 && side != 1)) return BPMF_EINVAL;
    DevSide& d = h->side[side];
    if (row_begin < 0 || row_end < row_begin || row_end > d.rows) return BPMF_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {  // no launch may use the old bins
        cudaGetLastError();
        return BPMF_ECUDA;
    }
    d.shard_lo = row_begin;
    d.shard_hi = row_end;
    std::vector<int32_t> order;
    const int rc = bin_side(h, d, order);
    // the captured sweep holds the old bins' launch shapes
    if (h->sweep_graph) cudaGraphExecDestroy(h->sweep_graph);
    h->sweep_graph = nullptr;
    h->graph_state = 0;
    return rc;
}

int bpmf_get_rows(bpmf_handle h, int32_t side, int64_t row_begin, int64_t row_end, float* out,
                  int32_t where)
{
    if (!h || (side != 0 && side != 1) || (where != 0 && where != 1)) return BPMF_EINVAL;
    const DevSide& d = h->side[side];
    if (row_begin < 0 || row_end < row_begin || row_end > d.rows) return BPMF_EINVAL;
    const int64_t n = row_end - row_begin;
    if (n == 0) return BPMF_OK;
    if (!out) return BPMF_EINVAL;
    cudaError_t e = cudaMemcpy2DAsync(out, sizeof(float) * h->K, d.X + row_begin * h->kp,
                                      sizeof(float) * h->kp, sizeof(float) * h->K, (size_t)n,
                                      where ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                      h->stream);
    if (e == cudaSuccess && where == 0) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_rc(e);
}

int bpmf_put_rows(bpmf_handle h, int32_t side, int64_t row_begin, int64_t row_end, const float* in,
                  int32_t where)
{
    if (!h || (side != 0 && side != 1) || (where != 0 && where != 1)) return BPMF_EINVAL;
    DevSide& d = h->side[side];
    if (row_begin < 0 || row_end < row_begin || row_end > d.rows) return BPMF_EINVAL;
    const int64_t n = row_end - row_begin;
    if (n == 0) return BPMF_OK;
    if (!in) return BPMF_EINVAL;
    // the padding columns K .. kp-1 stay zero; the 16-bit split the other side's Gram
    // gathers follows the new rows
    cudaError_t e = cudaMemcpy2DAsync(d.X + row_begin * h->kp, sizeof(float) * h->kp, in,
                                      sizeof(float) * h->K, sizeof(float) * h->K, (size_t)n,
                                      where ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                      h->stream);
    if (e == cudaSuccess && d.Xh)
        e = launch_split_factors(d.X + row_begin * h->kp, n, h->kp, d.Xh + row_begin * h->kp,
                                 d.Xl + row_begin * h->kp, (h->p.flags & BPMF_BF16_GRAM) ? 1 : 0,
                                 h->stream);
    if (e == cudaSuccess && where == 0) e = cudaStreamSynchronize(h->stream);  // host buffer
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_rc(e);
}

int bpmf_device_bytes(int64_t M, int64_t N, int32_t K, const int64_t* csr_ptr,
                      const int32_t* csr_col, int64_t n_test, const bpmf_params* params,
                      int32_t num_sms, int64_t* out_bytes)
{
    if (!out_bytes || M <= 0 || N <= 0 || K < 1 || K > kMaxK || n_test < 0 || !csr_ptr ||
        M > INT32_MAX || N > INT32_MAX || !valid_ptr(M, csr_ptr))
        return BPMF_EINVAL;
    const int64_t nnz = csr_ptr[M];
    if (nnz > 0 && !csr_col) return BPMF_EINVAL;
    if (num_sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return BPMF_ECUDA;
        }
    }
    bpmf_params prm;
    if (params) prm = *params;
    else bpmf_default_params(&prm);
    // every size below is one allocation of bpmf_create, rounded as it rounds them
    auto rb = [](size_t b) -> int64_t {
        if (b == 0) b = 16;
        return (int64_t)((b + 255) & ~(size_t)255);
    };
    const int kp = (K + 15) / 16 * 16;
    const bool tc = kp == 64 && !(prm.flags & BPMF_CUDA_CORE_GRAM);
    const int64_t long_min = prm.long_min_degree > 0 ? prm.long_min_degree : default_long_min(prm.flags);
    const int64_t split = prm.split_degree > 0 ? prm.split_degree : kDefaultSplitDegree;
    std::vector<int64_t> cptr;
    try {
        // the column view's offsets, from the column counts
        cptr.assign((size_t)N + 1, 0);
        for (int64_t e = 0; e < nnz; ++e) {
            const int32_t c = csr_col[e];
            if (c < 0 || c >= N) return BPMF_EINVAL;
            ++cptr[(size_t)c + 1];
        }
        for (int64_t c = 0; c < N; ++c) cptr[(size_t)c + 1] += cptr[(size_t)c];
        int64_t bytes = 0, gram_rows = 0;
        std::vector<int32_t> order, pos;
        std::vector<Segment> segs;
        std::vector<int64_t> cost, first;
        for (int s = 0; s < 2; ++s) {
            const int64_t rows = s == 0 ? M : N;
            const int64_t* ptr = s == 0 ? csr_ptr : cptr.data();
            const size_t r = (size_t)rows;
            bytes += rb(8 * (r + 1)) + 2 * rb(4 * (size_t)nnz) + rb(4 * r * kp) + rb(4 * r) +
                     rb(8 * (size_t)K) + rb(8 * (size_t)kp) + rb(8 * (size_t)K * K) +
                     rb(8 * nw_draws_doubles(K)) + rb(4 * 3 * (size_t)kp * kp) + rb(4 * (size_t)kp) +
                     rb(8 * (size_t)hyper_reduce_blocks(rows, num_sms) * hyper_partial_doubles(kp)) +
                     rb(8 * hyper_partial_doubles(kp)) + rb(8 * ((size_t)K + (size_t)K * K));
            if (prm.flags & BPMF_DEBUG_MEANS) bytes += rb(4 * r * kp);
            if (tc) bytes += 2 * rb(2 * r * kp);
            int64_t n_short = 0, n_long = 0, long_ratings = 0;
            bin_rows(rows, ptr, tc ? long_min : INT64_MAX, order, &n_short, &n_long, &long_ratings);
            const int64_t nsplit = build_segments(ptr, order, n_short, split, segs);
            if (!segs.empty())
                bytes += rb(sizeof(Segment) * segs.size()) +
                         rb(4 * segs.size() * warp_partial_floats(kp));
            if (nsplit > 0) bytes += rb(sizeof(unsigned int) * (size_t)nsplit);
            if (tc && n_long > 0) {
                long_bin_costs(ptr, order, n_short, n_long, cost);
                for (int q = 0; q < 2; ++q) {
                    const int64_t G = std::min<int64_t>(n_long, (int64_t)kGramCtasPerSm * (num_sms - q));
                    if (!balance_plan(cost, G, pos, first)) continue;
                    bytes += rb(4 * (size_t)n_long) + rb(8 * ((size_t)kGramCtasPerSm * num_sms + 1));
                }
                gram_rows = std::max(gram_rows, n_long);
            }
            if (s == 0) bytes += rb(8 * (1 + (size_t)kCheckSumBlocks)) + rb(4);
        }
        if (gram_rows > 0) bytes += rb(4 * (size_t)gram_rows * kGramSlotFloats);
        const size_t T = (size_t)n_test;
        bytes += rb(8 * (size_t)K) + rb(8 * (size_t)K * K) + 3 * rb(4 * T) + rb(8 * T) +
                 rb(16 * (size_t)predict_blocks(n_test, num_sms)) + rb(sizeof(Control));
        *out_bytes = bytes;
    } catch (const std::bad_alloc&) {
        return BPMF_ENOMEM;
    }
    return BPMF_OK;
}

int bpmf_bin_rows(int64_t rows, const int64_t* ptr, int64_t long_min, int32_t* order_out,
                  int64_t* n_short)
{
    if (rows < 1 || rows > (int64_t)INT32_MAX || !ptr || !order_out || !n_short) return BPMF_EINVAL;
    if (!valid_ptr(rows, ptr)) return BPMF_EINVAL;
    // the counting sort keeps one counter per degree: a row's degree is bounded like a
    // row index (the device kernels count ratings of a row in 32 bits too)
    for (int64_t r = 0; r < rows; ++r)
        if (ptr[r + 1] - ptr[r] > (int64_t)INT32_MAX) return BPMF_EINVAL;
    try {
        std::vector<int32_t> order;
        int64_t nl = 0, lr = 0;
        bin_rows(rows, ptr, long_min > 0 ? long_min : INT64_MAX, order, n_short, &nl, &lr);
        std::copy(order.begin(), order.end(), order_out);
    } catch (const std::bad_alloc&) {
        return BPMF_ENOMEM;
    }
    return BPMF_OK;
}

int bpmf_balance_rows(int64_t n, const int64_t* degree, int64_t grid, int32_t* order_out,
                      int64_t* first_out, int32_t* planned)
{
    if (n < 0 || n > (int64_t)INT32_MAX || grid < 1 || !planned ||
        (n > 0 && (!degree || !order_out || !first_out)))
        return BPMF_EINVAL;
    try {
        std::vector<int64_t> cost((size_t)n);
        for (int64_t k = 0; k < n; ++k) {
            if (degree[k] < 0 || degree[k] > (int64_t)INT32_MAX) return BPMF_EINVAL;
            cost[(size_t)k] = plan_cost(degree[k]);
        }
        std::vector<int32_t> pos;
        std::vector<int64_t> first;
        *planned = balance_plan(cost, std::min<int64_t>(n, grid), pos, first) ? 1 : 0;
        if (*planned) {
            std::copy(pos.begin(), pos.end(), order_out);
            std::copy(first.begin(), first.end(), first_out);
        }
    } catch (const std::bad_alloc&) {
        return BPMF_ENOMEM;
    }
    return BPMF_OK;
}

int bpmf_info(bpmf_handle h, int32_t side, int64_t* n_short, int64_t* n_long, int64_t* n_split,
              int64_t* n_segments, double* rbar, int64_t* device_bytes, int32_t* balanced)
{
    if (!h || (side != 0 && side != 1)) return BPMF_EINVAL;
    if (balanced) *balanced = (h->side[side].plan_grid[0] > 0 ? 1 : 0) | (h->side[side].plan_grid[1] > 0 ? 2 : 0);
    if (n_short) *n_short = h->side[side].n_short;
    if (n_long) *n_long = h->side[side].n_long;
    if (n_split) *n_split = h->side[side].n_split;
    if (n_segments) *n_segments = h->side[side].n_segs;
    if (rbar) *rbar = h->rbar;
    if (device_bytes) *device_bytes = h->bytes;
    return BPMF_OK;
}

}  // extern "C"
