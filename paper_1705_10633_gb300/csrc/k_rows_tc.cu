// k_rows_tc.cu -- per-row conditional update with the Gram on the 5th-generation
// tensor cores (tcgen05, accumulators in TMEM), for rows with many ratings.
//
// The Gram sum_c y_c y_c^T of a row is a dense contraction over its ratings
// (the "K x K outer product" of Sec. 3.1).  The other side's factors are kept
// as an FP16 split y = h + l (|l| <= 2^-11 |h|) and the ratings as r = r_hi +
// r_lo; one M = 128, N = 144 MMA per 16 ratings computes
//     D = [H^T ; L^T] . [H | L | R]
// whose column blocks 0..63 and 64..127, summed over both row halves, give
// (H + L)^T (H + L) (FP32-class accuracy at the FP16 tensor rate), and whose
// columns 128, 129 give (H + L)^T r.  A and B are the same three 64-wide
// 128B-swizzled atoms of a stage (h rows, l rows, and the ratings in the first
// two columns of an otherwise zero atom), so each k-block reads them once.
//
// One CTA per SM, persistent over the rows of the long bin (12 or 16 warps, by shape).
// The rows, longest first, are dealt round-robin to the CTAs, or by the host's balanced
// plan (each row to the CTA with the least work so far) where round-robin would leave
// one CTA well above the mean (a few rows of 2.7e5 ratings among thousands of shorter
// ones).  Warp roles:
//   warp 0       MMA issuer (one lane) and TMEM owner (512 columns)
//   warp 1       prefetch: row descriptors (row, first, last rating) into a
//                ring, and every stage's rating indices and values into a
//                second ring, far ahead of use (cp.async, mbarrier completion)
//   warps 2-3    gather (with warps 8-9 in the long-row shape): cp.async of the
//                128-B h and l rows of each rating into 128B-swizzled tiles
//                (MN-major operand layout); they never wait for their copies,
//                the stage barrier completes when they land
//   warps 4-7    drain: TMEM -> shared Lambda_i += alpha Gram (the buffer starts
//                from Lambda_X), b_i
//   the rest     one row each: Cholesky, solves, Philox noise, store
// Stages of 64 ratings flow producer -> MMA through mbarriers; accumulators
// (3 TMEM slots of 144 columns) MMA -> drain; Lambda buffers (one per Cholesky warp) drain ->
// Cholesky.  A long row is accumulated in chunks of 16 stages, each in a fresh
// TMEM accumulator that the drain adds into the row's FP32 buffer: the tensor
// core's accumulation rounding then grows with the chunk length only, not with
// the row's degree (rows here reach 2.7e5 ratings).  Every wait is bounded in time; a timeout sets a status bit, the
// CTA stops its loops, waits for its own copies and MMAs, frees TMEM and exits.
#include "bpmf_internal.cuh"
#include "philox.cuh"
#include "rows_common.cuh"

namespace bpmf {
namespace {

constexpr int kKT = 64;
constexpr int kStageRatings = 64;
constexpr int kNAcc = 3;
constexpr int kChunkStages = 16;  // stages per TMEM accumulation before it is flushed
constexpr int kRowRing = 32;   // row descriptors in flight
constexpr int kIdxRing = 8;    // stages of rating indices / values in flight
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kAccStride = 160;  // 144 columns used

constexpr uint32_t kTileBytes = kStageRatings * 128;        // 64 ratings x 64 halves
constexpr uint32_t kRBytes = kTileBytes;                    // ratings atom (2 of 64 columns)
constexpr uint32_t kStageBytes = 2 * kTileBytes + kRBytes;  // 24 KB (1 KB multiple)
// A Lambda buffer: the lower triangle of the 64 x 64 precision in the XOR-swizzled
// layout sw64 (row stride 64, 16-B chunks permuted by row & 7), then b (64 floats).
constexpr uint32_t kLamFloats = 64 * 64 + 64;
constexpr uint32_t kCholScratchFloats = 2 * 64 + 64 + 64;

// Two shapes of the CTA, chosen per launch by the rows' mean degree:
//   NCHOL Cholesky warps (and Lambda buffers), NSTAGE gather stages and EXTRA gather
//   warps beside warps 2-3.
// Rows of a few hundred ratings need many rows in factorisation at once (8, 3, 0);
// rows of thousands of ratings, whose gathered rows come partly from HBM, need
// more copies in flight and more threads issuing them, and few rows in factorisation
// (2, 7, 2).  Warps: 0 MMA, 1 prefetch, 2-3 gather, 4-7 drain (TMEM lane quarters
// 0-3), 8 .. 7 + EXTRA gather, then the Cholesky warps.  Registers after setmaxnreg:
// producers kProdRegs, drain kDrainRegs, Cholesky kCholRegs.
template <int NCHOL, int NSTAGE, int EXTRA>
struct TcShape {
    static constexpr int kNChol = NCHOL;
    static constexpr int kNStage = NSTAGE;
    static constexpr int kGather = 64 + 32 * EXTRA;  // gather threads
    static constexpr int kCholWarp0 = 8 + EXTRA;
    static constexpr int kThreads = (8 + EXTRA + NCHOL) * 32;
    static_assert(kGather == 64 || kGather == 128, "gather threads");
    static constexpr uint32_t kOffStages = 0;
    static constexpr uint32_t kOffLam = kOffStages + NSTAGE * kStageBytes;
    static constexpr uint32_t kOffChol = kOffLam + NCHOL * kLamFloats * 4;
    static constexpr uint32_t kOffRtmp = kOffChol + NCHOL * kCholScratchFloats * 4;
    static constexpr uint32_t kOffRowRing = kOffRtmp + 64 * 4;          // kRowRing x 32 B
    static constexpr uint32_t kOffIdxRing = kOffRowRing + kRowRing * 32;  // kIdxRing x (64 idx + 64 val)
    static constexpr uint32_t kOffBars = kOffIdxRing + kIdxRing * 512;
    static constexpr int kNumBars = 2 * NSTAGE + 2 * kNAcc + 2 * NCHOL + 2 * kRowRing + 2 * kIdxRing + 1;
    static constexpr uint32_t kOffMisc = kOffBars + kNumBars * 8;
    static constexpr uint32_t kSmemBytes = kOffMisc + 16 + 1024;  // + alignment slack
    // the launch gives 65536 / kThreads registers a thread (128 or 168)
    static constexpr int kProdRegs = NCHOL == 8 ? 72 : 96;
    static constexpr int kDrainRegs = NCHOL == 8 ? 96 : 128;
    static constexpr int kCholRegs = NCHOL == 8 ? 168 : 176;
    static_assert(kSmemBytes <= 232448, "shared memory");
    static_assert(32 * ((4 + EXTRA) * kProdRegs + 4 * kDrainRegs + NCHOL * kCholRegs) <=
                      kThreads * (65536 / kThreads / 8 * 8),
                  "registers");
};
using ShapeShortRows = TcShape<8, 3, 0>;
using ShapeLongRows = TcShape<2, 7, 2>;
// The BF16 Gram gathers half the bytes (h rows only): its long rows run better with
// four factorisation warps and 64 gather threads (measured: movie launch 5.00 against
// 5.73 ms with the shape above, which takes the FP16 split's from 6.08 to 5.87 ms).
using ShapeLongRowsBf16 = TcShape<4, 6, 0>;

// Instruction descriptor of kind::f16: D = F32, A = B = F16, both MN-major.
constexpr uint32_t make_idesc(int M, int N)
{
    return (1u << 4) | (0u << 7) | (0u << 10) | (1u << 15) | (1u << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t kIdesc = make_idesc(128, 144);
constexpr uint32_t kIdescBf16 = kIdesc | (1u << 7) | (1u << 10);  // A and B in BF16

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start, leading / stride byte
// offsets (>> 4), descriptor version 1, layout (0 none, 2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)(layout & 7u) << 61);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

struct WaitCtx {
    volatile int* abort_flag;
    int64_t timeout_ns;
    Control* ctl;
};

// Wait for the phase of `bar` with parity `parity`; false after the time limit
// (which also raises the CTA's abort flag and the status bit) or once aborted.
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, const WaitCtx& w)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31u) == 0) {
            if (*w.abort_flag) return false;
            if ((int64_t)(globaltimer_ns() - t0) > w.timeout_ns) {
                *w.abort_flag = 1;
                atomicOr(&w.ctl->status, kStatusTimeout);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
// Arrive on `bar` once every cp.async this thread issued so far has landed.
__device__ __forceinline__ void cp_async_arrive(uint32_t bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void named_bar(uint32_t id, uint32_t nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// Named barrier that also returns the OR of `pred` over its participants, so a
// decision taken after it is the same in every participating thread.
__device__ __forceinline__ bool bar_any(uint32_t id, uint32_t nthreads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

#define TMEM_LD16(taddr, r)                                                                      \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "                                       \
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"               \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),       \
                   "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),     \
                   "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])                            \
                 : "r"(taddr))

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t& a, uint32_t& b)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
                 : "=r"(a), "=r"(b)
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace

// One drain thread's share of a TMEM accumulator: row m of the Gram is the sum of
// accumulator columns c and 64 + c; 16 of each per round, added into the row's
// lower-triangle chunks (the buffer starts from the prior precision).  Warps
// whose rows end before column 32 stop after two rounds; the trip count is
// warp-uniform, as the collective loads require.
__device__ __forceinline__ void drain_rows(uint32_t taddr, float* L, int m, int quarter, float alpha)
{
    const int ngroups = (quarter & 1) ? 4 : 2;
#pragma unroll 1
    for (int h = 0; h < ngroups; ++h) {
        uint32_t g[16], e[16];
        TMEM_LD16(taddr + 16 * h, g);
        TMEM_LD16(taddr + 64 + 16 * h, e);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int cc = 4 * h + q;
            if (4 * cc <= m) {
                float4* p = chunk_ptr(L, m, cc);
                float4 v = *p;
                v.x = fmaf(alpha, __uint_as_float(g[4 * q + 0]) + __uint_as_float(e[4 * q + 0]), v.x);
                v.y = fmaf(alpha, __uint_as_float(g[4 * q + 1]) + __uint_as_float(e[4 * q + 1]), v.y);
                v.z = fmaf(alpha, __uint_as_float(g[4 * q + 2]) + __uint_as_float(e[4 * q + 2]), v.z);
                v.w = fmaf(alpha, __uint_as_float(g[4 * q + 3]) + __uint_as_float(e[4 * q + 3]), v.w);
                *p = v;
            }
        }
    }
}

template <class Shape, bool kBf16>
__global__ void __launch_bounds__(Shape::kThreads, 1) rows_tc_kernel(RowArgs a)
{
    constexpr int kNChol = Shape::kNChol, kNStage = Shape::kNStage, kThreads = Shape::kThreads;
    constexpr uint32_t kOffStages = Shape::kOffStages, kOffLam = Shape::kOffLam;
    constexpr uint32_t kOffChol = Shape::kOffChol, kOffRtmp = Shape::kOffRtmp;
    constexpr uint32_t kOffRowRing = Shape::kOffRowRing, kOffIdxRing = Shape::kOffIdxRing;
    constexpr uint32_t kOffBars = Shape::kOffBars, kOffMisc = Shape::kOffMisc;
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    float* lam_bufs = reinterpret_cast<float*>(sm + kOffLam);
    float* chol_scratch = reinterpret_cast<float*>(sm + kOffChol);
    float* rtmp = reinterpret_cast<float*>(sm + kOffRtmp);
    long long* row_ring = reinterpret_cast<long long*>(sm + kOffRowRing);  // [row, p0, p1, -]
    const int* idx_ring = reinterpret_cast<const int*>(sm + kOffIdxRing);
    const float* val_ring = reinterpret_cast<const float*>(sm + kOffIdxRing + 256);
    const uint32_t bars = sbase + kOffBars;
    const uint32_t bar_stage_full = bars;
    const uint32_t bar_stage_empty = bar_stage_full + 8 * kNStage;
    const uint32_t bar_acc_full = bar_stage_empty + 8 * kNStage;
    const uint32_t bar_acc_empty = bar_acc_full + 8 * kNAcc;
    const uint32_t bar_lam_full = bar_acc_empty + 8 * kNAcc;
    const uint32_t bar_lam_empty = bar_lam_full + 8 * kNChol;
    const uint32_t bar_row_full = bar_lam_empty + 8 * kNChol;
    const uint32_t bar_row_empty = bar_row_full + 8 * kRowRing;
    const uint32_t bar_idx_full = bar_row_empty + 8 * kRowRing;
    const uint32_t bar_idx_empty = bar_idx_full + 8 * kIdxRing;
    const uint32_t bar_final = bar_idx_empty + 8 * kIdxRing;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffMisc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kOffMisc + 4);
    volatile int* never_set = reinterpret_cast<volatile int*>(sm + kOffMisc + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    // rows of this CTA, longest first: a.rows[first + j] for j < nj under a balanced
    // plan made for this grid, else a.rows[blockIdx.x + j * G]
    const bool planned = a.cta_first != nullptr && a.plan_grid == (int64_t)G;
    const int64_t first = planned ? __ldg(a.cta_first + blockIdx.x) : 0;
    const int64_t nj = planned ? __ldg(a.cta_first + blockIdx.x + 1) - first
                               : (a.nrows > blockIdx.x ? (a.nrows - blockIdx.x + G - 1) / G : 0);
    const WaitCtx wc{abort_flag, a.timeout_ns, a.ctl};

    // ---- set-up: zero the ratings atoms (and the l atoms, which the BF16 Gram leaves
    // unused), barriers, TMEM
    for (uint32_t e = tid; e < kNStage * kRBytes / 16; e += kThreads) {
        const uint32_t s = e / (kRBytes / 16), o = e % (kRBytes / 16);
        *reinterpret_cast<uint4*>(sm + kOffStages + s * kStageBytes + 2 * kTileBytes + 16 * o) =
            make_uint4(0u, 0u, 0u, 0u);
        if (kBf16)
            *reinterpret_cast<uint4*>(sm + kOffStages + s * kStageBytes + kTileBytes + 16 * o) =
                make_uint4(0u, 0u, 0u, 0u);
    }
    // every precision buffer starts from the prior precision
    for (int b = 0; b < kNChol; ++b)
        fill_lower_sw64(lam_bufs + b * kLamFloats, reinterpret_cast<const float4*>(a.lam_ct), tid,
                        kThreads);
    if (tid == 0) {
        for (int s = 0; s < kNStage; ++s) {
            mbar_init(bar_stage_full + 8 * s, Shape::kGather);
            mbar_init(bar_stage_empty + 8 * s, 1);
        }
        for (int s = 0; s < kNAcc; ++s) {
            mbar_init(bar_acc_full + 8 * s, 1);
            mbar_init(bar_acc_empty + 8 * s, 128);
        }
        for (int s = 0; s < kNChol; ++s) {
            mbar_init(bar_lam_full + 8 * s, 128);
            mbar_init(bar_lam_empty + 8 * s, 32);
        }
        for (int s = 0; s < kRowRing; ++s) {
            mbar_init(bar_row_full + 8 * s, 1);
            mbar_init(bar_row_empty + 8 * s, 1);
        }
        for (int s = 0; s < kIdxRing; ++s) {
            mbar_init(bar_idx_full + 8 * s, 32);
            mbar_init(bar_idx_empty + 8 * s, Shape::kGather);
        }
        mbar_init(bar_final, 1);
        *abort_flag = 0;
        *never_set = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    constexpr int64_t kChunkRatings = (int64_t)kChunkStages * kStageRatings;

    // ======================= gather (warps 2-3 and the extra gather warps) ==========
    // gt: this thread's index among the kGather gather threads
    constexpr int kGatherN = Shape::kGather;
    constexpr int kRps = kGatherN / 16, kRpsB = kGatherN / 8;  // ratings per copy round
    constexpr int kCopies = kBf16 ? 512 / kGatherN : 1024 / kGatherN;
    auto gather_role = [&](const int gt) {
        uint32_t g = 0;
        bool ok = true;
        for (int64_t j = 0; j < nj && ok; ++j) {
            const int rs = (int)(j % kRowRing);
            if (!wait_bounded(bar_row_full + 8 * rs, (uint32_t)((j / kRowRing) & 1), wc)) break;
            const int64_t p0 = row_ring[4 * rs + 1], p1 = row_ring[4 * rs + 2];
            for (int64_t base = p0; base < p1; base += kStageRatings, ++g) {
                const uint32_t is = g % kIdxRing, s = g % kNStage;
                if (!wait_bounded(bar_idx_full + 8 * is, (g / kIdxRing) & 1u, wc) ||
                    !wait_bounded(bar_stage_empty + 8 * s, ((g / kNStage) & 1u) ^ 1u, wc)) {
                    ok = false;
                    break;
                }
                const int cnt = (int)min((int64_t)kStageRatings, p1 - base);
                // this thread's rows (-1 past the row's end), read before the slot is
                // released: FP16 split, rating (gt >> 4) + kRps k, 16-B chunk gt & 15 of
                // its h and l rows; BF16, rating (gt >> 3) + kRpsB k, chunk gt & 7 of its
                // h row (kRps = gather threads / 16 ratings per round)
                int cols[kCopies];
                if constexpr (!kBf16) {
#pragma unroll
                    for (int k = 0; k < kCopies; ++k) {
                        const int qq = (gt >> 4) + kRps * k;
                        cols[k] = qq < cnt ? idx_ring[is * 128 + qq] : -1;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < kCopies; ++k) {
                        const int qq = (gt >> 3) + kRpsB * k;
                        cols[k] = qq < cnt ? idx_ring[is * 128 + qq] : -1;
                    }
                }
                // the first 64 threads also carry the stage's 64 rating values
                const float rv = gt < 64 && gt < cnt ? val_ring[is * 128 + gt] : 0.f;
                mbar_arrive(bar_idx_empty + 8 * is);
                const uint32_t sH = sbase + kOffStages + s * kStageBytes;
                const uint32_t sL = sH + kTileBytes;
                const uint32_t sR = sL + kTileBytes;
                if constexpr (!kBf16) {
                    const int c = gt & 15, ch = c & 7;
                    const __half* Ysrc = (c >> 3) ? a.Yl : a.Yh;
                    const uint32_t tile = (c >> 3) ? sL : sH;
#pragma unroll
                    for (int k = 0; k < kCopies; ++k) {
                        const int qq = (gt >> 4) + kRps * k;
                        const uint32_t dst = tile + qq * 128 + ((ch ^ (qq & 7)) << 4);
                        if (cols[k] >= 0)
                            cp_async16(dst, Ysrc + (int64_t)cols[k] * kKT + ch * 8, 16);
                        else
                            cp_async16(dst, a.Yh, 0);  // zero fill past the row's end
                    }
                } else {
                    // h rows only; the l atom stays zero
                    const int ch = gt & 7;
#pragma unroll
                    for (int k = 0; k < kCopies; ++k) {
                        const int qq = (gt >> 3) + kRpsB * k;
                        const uint32_t dst = sH + qq * 128 + ((ch ^ (qq & 7)) << 4);
                        if (cols[k] >= 0)
                            cp_async16(dst, a.Yh + (int64_t)cols[k] * kKT + ch * 8, 16);
                        else
                            cp_async16(dst, a.Yh, 0);
                    }
                }
                if (gt < 64) {
                    __half hi, lo;
                    split16(rv, kBf16, hi, lo);
                    const uint32_t packed = (uint32_t)__half_as_ushort(hi) |
                                            ((uint32_t)__half_as_ushort(lo) << 16);
                    asm volatile("st.shared.b32 [%0], %1;" ::"r"(sR + gt * 128 + ((gt & 7) << 4)),
                                 "r"(packed)
                                 : "memory");
                }
                fence_proxy_async();
                if (!a.test_stall) cp_async_arrive(bar_stage_full + 8 * s);
            }
        }
        cp_async_wait_all();
    };

    if (warp < 4) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(Shape::kProdRegs) : "memory");
        if (warp == 0) {
            // ======================= MMA issuer =======================
            if (lane == 0) {
                constexpr uint32_t idesc = kBf16 ? kIdescBf16 : kIdesc;
                uint32_t g = 0, u = 0;  // stages consumed, accumulation chunks issued
                bool ok = true;
                for (int64_t j = 0; j < nj && ok; ++j) {
                    const int rs = (int)(j % kRowRing);
                    if (!wait_bounded(bar_row_full + 8 * rs, (uint32_t)((j / kRowRing) & 1), wc)) break;
                    const int64_t p0 = row_ring[4 * rs + 1], p1 = row_ring[4 * rs + 2];
                    // a long row is summed in chunks of kChunkStages stages, each in a
                    // fresh TMEM accumulator that the drain adds into the row's buffer
                    for (int64_t c0 = p0; c0 < p1 && ok; c0 += kChunkRatings, ++u) {
                        const uint32_t slot = u % kNAcc;
                        if (!wait_bounded(bar_acc_empty + 8 * slot, ((u / kNAcc) & 1u) ^ 1u, wc)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t dgram = tmem_base + slot * kAccStride;
                        const int64_t c1 = min(p1, c0 + kChunkRatings);
                        for (int64_t base = c0; base < c1; base += kStageRatings, ++g) {
                            const uint32_t s = g % kNStage;
                            if (!wait_bounded(bar_stage_full + 8 * s, (g / kNStage) & 1u, wc)) {
                                ok = false;
                                break;
                            }
                            // the stage was written through the generic proxy (cp.async and
                            // stores) and is read by the tensor core through the async proxy
                            fence_proxy_async();
                            tc_fence_after();
                            const int cnt = (int)min((int64_t)kStageRatings, p1 - base);
                            const uint32_t sH = sbase + kOffStages + s * kStageBytes;
                            for (int kb = 0; kb < (cnt + 15) / 16; ++kb) {
                                // A = [H^T; L^T] (M = 128: atoms 0, 1), B = [H | L | R]
                                // (N = 144: atoms 0, 1 and the first 16 columns of 2):
                                // one descriptor, atoms kTileBytes apart, 16 ratings
                                // (16 x 128 B rows) per k-block
                                const uint64_t desc = sdesc(sH + kb * 2048, kTileBytes, 1024, 2);
                                const uint32_t acc = (base > c0 || kb > 0) ? 1u : 0u;
                                tc_mma(dgram, desc, desc, idesc, acc);
                            }
                            tc_commit(bar_stage_empty + 8 * s);
                        }
                        if (ok) tc_commit(bar_acc_full + 8 * slot);
                    }
                }
                // all MMAs this thread issued complete before TMEM is released; this wait
                // ignores the abort flag and ends only by completion or its time limit
                tc_commit(bar_final);
                const WaitCtx wfinal{never_set, a.timeout_ns, a.ctl};
                (void)wait_bounded(bar_final, 0u, wfinal);
            }
            __syncwarp();
        } else if (warp == 1) {
            // ======================= prefetch =======================
            uint32_t g = 0;  // stages whose indices were prefetched
            bool ok = true;
            for (int64_t j0 = 0; j0 < nj && ok; j0 += 32) {
                // descriptors of the next 32 rows, one row per lane (independent loads)
                const int64_t jj = j0 + lane;
                int my_row = -1;
                long long my_p0 = 0, my_p1 = 0;
                if (jj < nj) {
                    my_row = __ldg(a.rows + (planned ? first + jj : blockIdx.x + jj * G));
                    my_p0 = __ldg(a.ptr + my_row);
                    my_p1 = __ldg(a.ptr + my_row + 1);
                }
                const int nb = (int)min((int64_t)32, nj - j0);
                for (int r = 0; r < nb && ok; ++r) {
                    const int64_t j = j0 + r;
                    const int row = __shfl_sync(kFullMask, my_row, r);
                    const long long p0 = __shfl_sync(kFullMask, my_p0, r);
                    const long long p1 = __shfl_sync(kFullMask, my_p1, r);
                    const int rs = (int)(j % kRowRing);
                    bool w = wait_bounded(bar_row_empty + 8 * rs, (uint32_t)((j / kRowRing) & 1) ^ 1u, wc);
                    if (!__all_sync(kFullMask, w)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        row_ring[4 * rs + 0] = row;
                        row_ring[4 * rs + 1] = p0;
                        row_ring[4 * rs + 2] = p1;
                        mbar_arrive(bar_row_full + 8 * rs);
                    }
                    for (long long base = p0; base < p1; base += kStageRatings, ++g) {
                        const uint32_t is = g % kIdxRing;
                        w = wait_bounded(bar_idx_empty + 8 * is, ((g / kIdxRing) & 1u) ^ 1u, wc);
                        if (!__all_sync(kFullMask, w)) {
                            ok = false;
                            break;
                        }
                        const int cnt = (int)min((long long)kStageRatings, p1 - base);
                        const uint32_t dst = sbase + kOffIdxRing + is * 512;
                        for (int e = lane; e < cnt; e += 32) {
                            cp_async4(dst + 4 * e, a.idx + base + e);
                            cp_async4(dst + 256 + 4 * e, a.val + base + e);
                        }
                        cp_async_arrive(bar_idx_full + 8 * is);
                    }
                }
            }
            cp_async_wait_all();
        } else {
            gather_role(tid - 64);
        }
    } else if (warp < 8) {
        // ======================= TMEM drain =======================
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(Shape::kDrainRegs) : "memory");
        const int quarter = warp & 3;
        const int m = 32 * (quarter & 1) + lane;  // row of Lambda this thread serves
        const float alpha = a.alpha;
        uint32_t u = 0;  // accumulation chunks drained
        bool live = true;
        for (int64_t j = 0; j < nj && live; ++j) {
            const int rs = (int)(j % kRowRing);
            const int b = (int)(j % kNChol);
            bool ok = wait_bounded(bar_row_full + 8 * rs, (uint32_t)((j / kRowRing) & 1), wc);
            if (bar_any(1, 128, !ok || *abort_flag != 0)) {
                *abort_flag = 1;
                break;
            }
            const int64_t p0 = row_ring[4 * rs + 1], p1 = row_ring[4 * rs + 2];
            float* L = lam_bufs + b * kLamFloats;
            float rsum = 0.f;
            for (int64_t c0 = p0; c0 < p1; c0 += kChunkRatings, ++u) {
                const uint32_t slot = u % kNAcc;
                const bool first = c0 == p0;
                // wait outcomes are made uniform over the 128 drain threads before any
                // warp-collective (tcgen05.ld) or group barrier depends on them
                ok = wait_bounded(bar_acc_full + 8 * slot, (u / kNAcc) & 1u, wc);
                if (bar_any(1, 128, !ok)) {
                    *abort_flag = 1;
                    live = false;
                    break;
                }
                if (first) {
                    ok = wait_bounded(bar_lam_empty + 8 * b, (uint32_t)((j / kNChol) & 1) ^ 1u, wc);
                    if (bar_any(1, 128, !ok)) {
                        *abort_flag = 1;
                        live = false;
                        break;
                    }
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + ((uint32_t)(32 * quarter) << 16) + slot * kAccStride;
                // The accumulator holds H^T (H + L) in its top 64 lanes and L^T (H + L) in
                // its bottom 64; their sum is the chunk's Gram (H + L is the FP16 split of
                // the other side's rows).  Both halves add into the row's buffer, which
                // starts from the prior precision, the bottom first; only chunks on or
                // below the diagonal are formed.
                uint32_t r0, r1;
                tmem_ld2(taddr + 128, r0, r1);
                if (quarter >= 2) drain_rows(taddr, L, m, quarter, alpha);
                named_bar(1, 128);
                if (quarter < 2) drain_rows(taddr, L, m, quarter, alpha);
                tmem_wait_ld();
                tc_fence_before();
                mbar_arrive(bar_acc_empty + 8 * slot);
                rsum += __uint_as_float(r0) + __uint_as_float(r1);
                named_bar(1, 128);
            }
            if (!live) break;
            if (quarter >= 2) rtmp[m] = rsum;
            named_bar(1, 128);
            if (quarter < 2) L[4096 + m] = fmaf(alpha, rsum + rtmp[m], __ldg(a.lammu + m));
            mbar_arrive(bar_lam_full + 8 * b);
            named_bar(1, 128);  // rtmp is reused by the next row
        }
    } else if (warp < Shape::kCholWarp0) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(Shape::kProdRegs) : "memory");
        gather_role(64 + tid - 256);
    } else {
        // ======================= Cholesky, solve, sample =======================
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(Shape::kCholRegs) : "memory");
        const int cw = warp - Shape::kCholWarp0;
        float* scratch = chol_scratch + cw * kCholScratchFloats;
        float* colbuf = scratch;
        float* dinv = scratch + 128;
        float* zb = scratch + 192;
        bool bad = false;
        for (int64_t j = cw; j < nj; j += kNChol) {
            if (__any_sync(kFullMask, *abort_flag != 0)) break;  // warp-uniform
            const bool ok = wait_bounded(bar_lam_full + 8 * cw, (uint32_t)((j / kNChol) & 1), wc);
            if (!__all_sync(kFullMask, ok)) break;
            // the row descriptor was published before this row's stages existed
            const int rs = (int)(j % kRowRing);
            const int row = (int)row_ring[4 * rs + 0];
            float* L = lam_bufs + cw * kLamFloats;
            float x1, x2, m1, m2;
            factor_solve_sample_rl64(L, L + 4096, colbuf, dinv, zb, lane, a.K, a.seed, (uint32_t)row,
                                     sweep, a.c3, a.means != nullptr, x1, x2, m1, m2, bad);
            store_row_panels(a, row, lane, x1, x2, m1, m2);
            __syncwarp();  // every lane is done reading L
            // the buffer goes back holding the prior precision, which the drain
            // accumulates into
            fill_lower_sw64(L, reinterpret_cast<const float4*>(a.lam_ct), lane, 32);
            __syncwarp();
            mbar_arrive(bar_lam_empty + 8 * cw);
            if (lane == 0) mbar_arrive(bar_row_empty + 8 * rs);
        }
        if (bad && lane == 0) atomicOr(&a.ctl->status, kStatusNotPD);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                     "r"(kTmemCols)
                     : "memory");
    }
}

template <class Shape, bool kBf16>
cudaError_t launch_shape(const RowArgs& a, int num_sms, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(rows_tc_kernel<Shape, kBf16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Shape::kSmemBytes);
    if (e != cudaSuccess) return e;
    // setmaxnreg.inc takes registers that other warps released from what the CTA was
    // launched with (the compiled count times the threads): if the split's total were
    // above that, the Cholesky warps' increase would never be granted.  Refuse the
    // launch instead (the compiled count can sit below the launch bound).
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, rows_tc_kernel<Shape, kBf16>);
    if (e != cudaSuccess) return e;
    const long split = 32L * ((4 + Shape::kCholWarp0 - 8) * Shape::kProdRegs +
                              4 * Shape::kDrainRegs + Shape::kNChol * Shape::kCholRegs);
    if (split > (long)fa.numRegs * Shape::kThreads) return cudaErrorInvalidConfiguration;
    int64_t grid = a.nrows < num_sms ? a.nrows : num_sms;
    rows_tc_kernel<Shape, kBf16><<<(unsigned)grid, Shape::kThreads, Shape::kSmemBytes, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rows_tc(const RowArgs& a, int64_t nratings, int64_t shape_degree, int num_sms,
                           cudaStream_t s)
{
    if (a.nrows <= 0) return cudaSuccess;
    const bool longrows = nratings >= shape_degree * a.nrows;
    if (a.bf16)
        return longrows ? launch_shape<ShapeLongRowsBf16, true>(a, num_sms, s)
                        : launch_shape<ShapeShortRows, true>(a, num_sms, s);
    return longrows ? launch_shape<ShapeLongRows, false>(a, num_sms, s)
                    : launch_shape<ShapeShortRows, false>(a, num_sms, s);
}

__global__ void split_factors_kernel(const float* __restrict__ X, int64_t n, __half* __restrict__ Xh,
                                     __half* __restrict__ Xl, int bf16)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        __half h, l;
        split16(X[e], bf16 != 0, h, l);
        Xh[e] = h;
        Xl[e] = l;
    }
}

cudaError_t launch_split_factors(const float* X, int64_t rows, int ld, __half* Xh, __half* Xl,
                                 int bf16, cudaStream_t s)
{
    const int64_t n = rows * ld;
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    split_factors_kernel<<<(int)(want < 8192 ? want : 8192), 256, 0, s>>>(X, n, Xh, Xl, bf16);
    return cudaGetLastError();
}

}  // namespace bpmf
