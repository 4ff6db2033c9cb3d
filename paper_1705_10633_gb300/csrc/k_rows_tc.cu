// k_rows_tc.cu -- the Gram and right-hand side of each long row on the
// 5th-generation tensor cores (tcgen05, accumulators in TMEM).
//
// The Gram sum_c y_c y_c^T of a row is a dense contraction over its ratings
// (the "K x K outer product" of Sec. 3.1).  The other side's factors are kept as
// an FP16 split y = h + l (|l| <= 2^-11 |h|) and the ratings as r = r_hi + r_lo.
// One M = 128, N = 80 MMA per 16 ratings computes
//     D = [L^T ; H^T] . [H | R]
// (A = the l and h rows, B = the h rows and the split ratings), so TMEM lanes
// 0..63 hold L^T H and L^T r, lanes 64..127 hold H^T H and H^T r, and
//     (H + L)^T (H + L) = H^T H + L^T H + (L^T H)^T + L^T L,
// where the last term (2^-22 relative) is dropped.  A stage is three 64-wide
// 128B-swizzled MN-major atoms (l rows, h rows, ratings in the first two columns
// of an otherwise zero atom); A starts at the l atom, B at the h atom.
//
// This kernel only forms the Gram (H + L)^T (H + L) and (H + L)^T r of each row and
// writes them to the row's slot of the scratch (layout in bpmf_internal.cuh);
// k_rows_chol.cu forms Lambda_i = Lambda_X + alpha Gram and b_i = Lambda_X mu_X +
// alpha (H + L)^T r as it loads the slot, and factors them.  Keeping the factorisation out
// of this kernel leaves the SM's issue slots and shared memory to the gather and
// the tensor core, and the factorisation kernel runs with every warp of the SM.
//
// Two CTAs per SM (each with half of the SM's TMEM and shared memory), persistent
// over the rows (dealt round-robin, or by the host's balanced plan where round-robin
// would be uneven).  Each CTA is one pipeline; two of them keep the tensor core busy
// while one MMA issuer waits for a stage or commits.  Warp roles (12 warps):
//   warp 0        MMA issuer (one lane) and TMEM owner (2 accumulators)
//   warp 1        prefetch: row descriptors (row, first, last rating, slot) into a
//                 ring, and every stage's rating indices and values into a second
//                 ring, far ahead of use (cp.async, mbarrier completion)
//   warps 2-3, 8-9  gather: cp.async of the 128-B h and l rows of each rating into the
//                 swizzled atoms; the stage barrier completes when they land
//   warps 10-11   idle (the last warpgroup's spare warps give their registers away)
//   warps 4-7     drain (TMEM lane quarters 0-3): TMEM -> registers, summed over the
//                 row's accumulation chunks; at the row's end the L^T H rows go
//                 through a shared staging buffer so the H^T H rows can add L^T H and
//                 its transpose and store the packed lower triangle of the Gram (the
//                 factorisation kernel scales it by alpha and adds Lambda_X as it loads
//                 it)
// Stages of 64 ratings flow producer -> MMA through mbarriers; accumulators MMA ->
// drain.  A long row is accumulated in chunks of 16 stages, each in a fresh
// accumulator that the drain adds into its registers: the tensor core's accumulation
// rounding grows with the chunk length only, not with the row's degree (rows here
// reach 2.7e5 ratings).  Every wait is bounded in time; a timeout sets a status bit,
// the CTA stops its loops, waits for its own copies and MMAs, frees TMEM and exits.
#include "bpmf_internal.cuh"
#include "philox.cuh"
#include "rows_common.cuh"

namespace bpmf {
namespace {

constexpr int kKT = 64;
constexpr int kStageRatings = 64;
constexpr int kChunkStages = 16;   // stages per TMEM accumulation before it is drained
constexpr int kRowRing = 32;       // row descriptors in flight
constexpr int kIdxRing = 8;        // stages of rating indices / values in flight
constexpr int kGroups = 1;         // drain groups of a CTA
constexpr int kSlotsPerGroup = 2;  // TMEM accumulators per drain group
constexpr int kNumAcc = kGroups * kSlotsPerGroup;
constexpr uint32_t kTmemCols = 256;  // half of the SM's TMEM: two CTAs share an SM
constexpr uint32_t kAccStride = 128;  // 80 columns used
constexpr int kN = 80;                // MMA N: 64 h columns + the ratings atom's first 16

constexpr uint32_t kTileBytes = kStageRatings * 128;  // one atom: 64 ratings x 64 halves
constexpr uint32_t kStageBytes = 3 * kTileBytes;      // l, h, ratings (24 KB)
constexpr int kNStage = 3;
constexpr int kGatherWarps = 4;
constexpr int kGather = 32 * kGatherWarps;
constexpr int kWarps = 12;
// setmaxnreg is executed by whole warpgroups (four consecutive warps): the CTA is made of
// full ones, and each warpgroup takes one register share
static_assert(kWarps % 4 == 0, "whole warpgroups");
constexpr int kThreads = kWarps * 32;
constexpr uint32_t kStagingFloats = 64 * 64 + 64;  // L^T H rows (sw64 layout) and L^T r

constexpr uint32_t kOffStages = 0;
constexpr uint32_t kOffStaging = kOffStages + kNStage * kStageBytes;
constexpr uint32_t kOffRowRing = kOffStaging + kGroups * kStagingFloats * 4;  // kRowRing x 32 B
constexpr uint32_t kOffIdxRing = kOffRowRing + kRowRing * 32;                // kIdxRing x (64 idx + 64 val)
constexpr uint32_t kOffBars = kOffIdxRing + kIdxRing * 512;
constexpr int kNumBars = 2 * kNStage + 2 * kNumAcc + 2 * kRowRing + 2 * kIdxRing + 1;
constexpr uint32_t kOffMisc = kOffBars + kNumBars * 8;
constexpr uint32_t kSmemBytes = kOffMisc + 16 + 1024;  // + alignment slack
static_assert(kGramCtasPerSm * (kSmemBytes + 1024) <= 233472, "shared memory of the SM's CTAs");
static_assert(kNumAcc * kAccStride <= kTmemCols, "TMEM columns");
// Registers: the launch gives 80 a thread (two CTAs of 384 threads within the register
// file).  A warpgroup puts one warp on each SM sub-partition, so a sub-partition holds, of
// each CTA, two producer or idle warps (warpgroups 0 and 2) and one drain warp (warpgroup 1),
// and setmaxnreg moves registers between them within it: producers and idle warps drop to
// kProdRegs, drain warps rise to kDrainRegs.
constexpr int kLaunchRegs = 80;
constexpr int kProdRegs = 48;
constexpr int kDrainRegs = 144;
static_assert(2 * kProdRegs + kDrainRegs <= 3 * kLaunchRegs, "registers per sub-partition");

// Instruction descriptor of kind::f16: D = F32, A = B = F16 (or BF16), both MN-major.
constexpr uint32_t make_idesc(int M, int N)
{
    return (1u << 4) | (0u << 7) | (0u << 10) | (1u << 15) | (1u << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t kIdesc = make_idesc(128, kN);
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
// kBackoff: a role that tolerates latency (the drain, the producers) sleeps briefly
// between polls, so its spinning does not take issue slots from the MMA issuer that
// shares its SM sub-partition.
template <bool kBackoff = false>
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity, const WaitCtx& w)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (kBackoff) __nanosleep(64);
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
// L2 policy for data read or written once (the streamed ratings, the scratch slots):
// evicted first, so that it does not push the other side's gathered 16-bit rows,
// which every CTA re-reads, out of L2.
__device__ __forceinline__ uint64_t l2_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void cp_async4_once(uint32_t dst, const void* src, uint64_t pol)
{
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, 4, %2;" ::"r"(dst),
                 "l"(src), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_once(float4* p, float4 v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x),
                 "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
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

template <bool kBf16>
__global__ void __launch_bounds__(kThreads, kGramCtasPerSm) rows_gram_kernel(RowArgs a)
{
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(sm);
    float* staging = reinterpret_cast<float*>(sm + kOffStaging);
    long long* row_ring = reinterpret_cast<long long*>(sm + kOffRowRing);  // [row, p0, p1, slot]
    const int* idx_ring = reinterpret_cast<const int*>(sm + kOffIdxRing);
    const float* val_ring = reinterpret_cast<const float*>(sm + kOffIdxRing + 256);
    const uint32_t bars = sbase + kOffBars;
    const uint32_t bar_stage_full = bars;
    const uint32_t bar_stage_empty = bar_stage_full + 8 * kNStage;
    const uint32_t bar_acc_full = bar_stage_empty + 8 * kNStage;
    const uint32_t bar_acc_empty = bar_acc_full + 8 * kNumAcc;
    const uint32_t bar_row_full = bar_acc_empty + 8 * kNumAcc;
    const uint32_t bar_row_empty = bar_row_full + 8 * kRowRing;
    const uint32_t bar_idx_full = bar_row_empty + 8 * kRowRing;
    const uint32_t bar_idx_empty = bar_idx_full + 8 * kIdxRing;
    const uint32_t bar_final = bar_idx_empty + 8 * kIdxRing;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffMisc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kOffMisc + 4);
    volatile int* never_set = reinterpret_cast<volatile int*>(sm + kOffMisc + 8);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = gridDim.x;
    // rows of this CTA, longest first: places first .. first + nj - 1 of a.rows under a
    // balanced plan made for this grid, else places blockIdx.x + j * G
    const bool planned = a.cta_first != nullptr && a.plan_grid == (int64_t)G;
    const int64_t first = planned ? __ldg(a.cta_first + blockIdx.x) : 0;
    const int64_t nj = planned ? __ldg(a.cta_first + blockIdx.x + 1) - first
                               : (a.nrows > blockIdx.x ? (a.nrows - blockIdx.x + G - 1) / G : 0);
    const WaitCtx wc{abort_flag, a.timeout_ns, a.ctl};

    // ---- set-up: zero the ratings atoms (and the l atoms, which the BF16 Gram leaves
    // unused), barriers, TMEM
    for (uint32_t e = tid; e < kNStage * kTileBytes / 16; e += kThreads) {
        const uint32_t s = e / (kTileBytes / 16), o = e % (kTileBytes / 16);
        *reinterpret_cast<uint4*>(sm + kOffStages + s * kStageBytes + 2 * kTileBytes + 16 * o) =
            make_uint4(0u, 0u, 0u, 0u);
        if (kBf16)
            *reinterpret_cast<uint4*>(sm + kOffStages + s * kStageBytes + 16 * o) =
                make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        for (int s = 0; s < kNStage; ++s) {
            mbar_init(bar_stage_full + 8 * s, kGather);
            mbar_init(bar_stage_empty + 8 * s, 1);
        }
        for (int s = 0; s < kNumAcc; ++s) {
            mbar_init(bar_acc_full + 8 * s, 1);
            mbar_init(bar_acc_empty + 8 * s, 128);
        }
        for (int s = 0; s < kRowRing; ++s) {
            mbar_init(bar_row_full + 8 * s, 1);
            mbar_init(bar_row_empty + 8 * s, 1);
        }
        for (int s = 0; s < kIdxRing; ++s) {
            mbar_init(bar_idx_full + 8 * s, 32);
            mbar_init(bar_idx_empty + 8 * s, kGather);
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
    constexpr int64_t kChunkRatings = (int64_t)kChunkStages * kStageRatings;

    // ======================= gather (warps 2-3, 8-9) =======================
    // gt: this thread's index among the kGather gather threads
    constexpr int kRps = kGather / 16, kRpsB = kGather / 8;  // ratings per copy round
    constexpr int kCopies = kBf16 ? 512 / kGather : 1024 / kGather;
    auto gather_role = [&](const int gt) {
        uint32_t g = 0;
        bool ok = true;
        for (int64_t j = 0; j < nj && ok; ++j) {
            const int rs = (int)(j % kRowRing);
            if (!wait_bounded<true>(bar_row_full + 8 * rs, (uint32_t)((j / kRowRing) & 1), wc)) break;
            const int64_t p0 = row_ring[4 * rs + 1], p1 = row_ring[4 * rs + 2];
            for (int64_t base = p0; base < p1; base += kStageRatings, ++g) {
                const uint32_t is = g % kIdxRing, s = g % kNStage;
                if (!wait_bounded<true>(bar_idx_full + 8 * is, (g / kIdxRing) & 1u, wc) ||
                    !wait_bounded<true>(bar_stage_empty + 8 * s, ((g / kNStage) & 1u) ^ 1u, wc)) {
                    ok = false;
                    break;
                }
                const int cnt = (int)min((int64_t)kStageRatings, p1 - base);
                // this thread's rows (-1 past the row's end), read before the slot is
                // released: FP16 split, rating (gt >> 4) + kRps k, 16-B chunk gt & 15 of
                // its l and h rows; BF16, rating (gt >> 3) + kRpsB k, chunk gt & 7 of its
                // h row
                int cols[kCopies];
#pragma unroll
                for (int k = 0; k < kCopies; ++k) {
                    const int qq = kBf16 ? (gt >> 3) + kRpsB * k : (gt >> 4) + kRps * k;
                    cols[k] = qq < cnt ? idx_ring[is * 128 + qq] : -1;
                }
                // the first 64 threads also carry the stage's 64 rating values
                const float rv = gt < 64 && gt < cnt ? val_ring[is * 128 + gt] : 0.f;
                mbar_arrive(bar_idx_empty + 8 * is);
                const uint32_t sL = sbase + kOffStages + s * kStageBytes;
                const uint32_t sH = sL + kTileBytes;
                const uint32_t sR = sH + kTileBytes;
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

    if (warp < 4 || warp >= 8) {
        asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kProdRegs) : "memory");
        if (warp == 0) {
            // ======================= MMA issuer =======================
            if (lane == 0) {
                constexpr uint32_t idesc = kBf16 ? kIdescBf16 : kIdesc;
                // stage ring position and phase kept as counters (no division in the loop)
                uint32_t st = 0, st_phase = 0;
                uint32_t uc0 = 0, uc1 = 0;  // accumulation chunks issued per drain group
                const uint32_t stage0 = sbase + kOffStages;
                const uint64_t adesc0 = sdesc(stage0, kTileBytes, 1024, 2);
                const uint64_t bdesc0 = sdesc(stage0 + kTileBytes, kTileBytes, 1024, 2);
                bool ok = true;
                for (int64_t j = 0; j < nj && ok; ++j) {
                    const int rs = (int)(j % kRowRing);
                    if (!wait_bounded(bar_row_full + 8 * rs, (uint32_t)((j / kRowRing) & 1), wc)) break;
                    const int64_t p0 = row_ring[4 * rs + 1];
                    const int32_t n = (int32_t)(row_ring[4 * rs + 2] - p0);  // ratings of the row
                    const int grp = (int)(j % kGroups);
                    // a long row is summed in chunks of kChunkStages stages, each in a
                    // fresh accumulator of the row's drain group
                    for (int32_t c0 = 0; c0 < n && ok; c0 += (int32_t)kChunkRatings) {
                        const uint32_t u = grp ? uc1++ : uc0++;
                        const uint32_t slot = grp * kSlotsPerGroup + u % kSlotsPerGroup;
                        if (!wait_bounded(bar_acc_empty + 8 * slot,
                                          ((u / kSlotsPerGroup) & 1u) ^ 1u, wc)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t dgram = tmem_base + slot * kAccStride;
                        const int32_t c1 = min(n, c0 + (int32_t)kChunkRatings);
                        for (int32_t base = c0; base < c1; base += kStageRatings) {
                            if (!wait_bounded(bar_stage_full + 8 * st, st_phase, wc)) {
                                ok = false;
                                break;
                            }
                            // the stage was written through the generic proxy (cp.async and
                            // stores) and is read by the tensor core through the async proxy
                            fence_proxy_async();
                            tc_fence_after();
                            // A = [L^T; H^T] (M = 128: the l and h atoms), B = [H | R]
                            // (N = 80: the h atom and the ratings atom's first 16
                            // columns); 16 ratings (16 x 128-B rows) per k-block, a k-block
                            // 2048 B further (128 in the descriptor's address field)
                            const uint64_t soff = (uint64_t)((st * kStageBytes) >> 4);
                            const int nkb = (min(kStageRatings, c1 - base) + 15) >> 4;
                            const uint32_t acc0 = base > c0 ? 1u : 0u;
                            tc_mma(dgram, adesc0 + soff, bdesc0 + soff, idesc, acc0);
                            for (int kb = 1; kb < nkb; ++kb)
                                tc_mma(dgram, adesc0 + soff + 128 * kb, bdesc0 + soff + 128 * kb, idesc, 1u);
                            tc_commit(bar_stage_empty + 8 * st);
                            if (++st == kNStage) {
                                st = 0;
                                st_phase ^= 1u;
                            }
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
            const uint64_t once = l2_evict_first();
            bool ok = true;
            for (int64_t j0 = 0; j0 < nj && ok; j0 += 32) {
                // descriptors of the next 32 rows, one row per lane (independent loads)
                const int64_t jj = j0 + lane;
                int my_row = -1;
                long long my_p0 = 0, my_p1 = 0, my_slot = 0;
                if (jj < nj) {
                    my_slot = planned ? first + jj : blockIdx.x + jj * G;
                    my_row = __ldg(a.rows + my_slot);
                    my_p0 = __ldg(a.ptr + my_row);
                    my_p1 = __ldg(a.ptr + my_row + 1);
                }
                const int nb = (int)min((int64_t)32, nj - j0);
                for (int r = 0; r < nb && ok; ++r) {
                    const int64_t j = j0 + r;
                    const int row = __shfl_sync(kFullMask, my_row, r);
                    const long long p0 = __shfl_sync(kFullMask, my_p0, r);
                    const long long p1 = __shfl_sync(kFullMask, my_p1, r);
                    const long long slot = __shfl_sync(kFullMask, my_slot, r);
                    const int rs = (int)(j % kRowRing);
                    bool w = wait_bounded<true>(bar_row_empty + 8 * rs, (uint32_t)((j / kRowRing) & 1) ^ 1u, wc);
                    if (!__all_sync(kFullMask, w)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        row_ring[4 * rs + 0] = row;
                        row_ring[4 * rs + 1] = p0;
                        row_ring[4 * rs + 2] = p1;
                        row_ring[4 * rs + 3] = slot;
                        mbar_arrive(bar_row_full + 8 * rs);
                    }
                    for (long long base = p0; base < p1; base += kStageRatings, ++g) {
                        const uint32_t is = g % kIdxRing;
                        w = wait_bounded<true>(bar_idx_empty + 8 * is, ((g / kIdxRing) & 1u) ^ 1u, wc);
                        if (!__all_sync(kFullMask, w)) {
                            ok = false;
                            break;
                        }
                        const int cnt = (int)min((long long)kStageRatings, p1 - base);
                        const uint32_t dst = sbase + kOffIdxRing + is * 512;
                        for (int e = lane; e < cnt; e += 32) {
                            cp_async4_once(dst + 4 * e, a.idx + base + e, once);
                            cp_async4_once(dst + 256 + 4 * e, a.val + base + e, once);
                        }
                        cp_async_arrive(bar_idx_full + 8 * is);
                    }
                }
            }
            cp_async_wait_all();
        } else if (warp < 10) {
            gather_role(warp < 4 ? tid - 64 : 64 + tid - 256);
        }
    } else {
        // ======================= TMEM drain (warps 4-7) =======================
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kDrainRegs) : "memory");
        const int grp = (warp - 4) >> 2;
        const int q = warp & 3;       // TMEM lane quarter: lanes 32q .. 32q + 31
        const bool hh = q >= 2;       // H^T [H | R] rows (else L^T [H | R] rows)
        const int m = 32 * (q & 1) + lane;  // row of the Gram this thread serves
        const uint32_t bar_id = 1 + grp;
        float* T = staging + grp * kStagingFloats;
        const uint64_t once = l2_evict_first();
        uint32_t u = 0;  // accumulation chunks drained by this group
        for (int64_t j = grp; j < nj; j += kGroups) {
            const int rs = (int)(j % kRowRing);
            bool ok = wait_bounded<true>(bar_row_full + 8 * rs, (uint32_t)((j / kRowRing) & 1), wc);
            if (bar_any(bar_id, 128, !ok || *abort_flag != 0)) {
                *abort_flag = 1;
                break;
            }
            const int64_t p0 = row_ring[4 * rs + 1], p1 = row_ring[4 * rs + 2];
            const int64_t slot_out = row_ring[4 * rs + 3];
            float acc[64];
#pragma unroll
            for (int i = 0; i < 64; ++i) acc[i] = 0.f;
            float rsum = 0.f;
            bool live = true;
            for (int64_t c0 = p0; c0 < p1; c0 += kChunkRatings, ++u) {
                const uint32_t slot = grp * kSlotsPerGroup + u % kSlotsPerGroup;
                // wait outcomes are made uniform over the group's 128 threads before any
                // warp-collective (tcgen05.ld) or group barrier depends on them
                ok = wait_bounded<true>(bar_acc_full + 8 * slot, (u / kSlotsPerGroup) & 1u, wc);
                if (bar_any(bar_id, 128, !ok)) {
                    *abort_flag = 1;
                    live = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + ((uint32_t)(32 * q) << 16) + slot * kAccStride;
                // H^T H rows below 32 need columns 0..31 only (their lower triangle); the
                // L^T H rows need all 64 (their transpose fills the H^T H rows' triangle)
                const int ngroups = (hh && (q & 1) == 0) ? 1 : 2;
#pragma unroll
                for (int hgrp = 0; hgrp < 2; ++hgrp) {
                    if (hgrp < ngroups) {  // warp-uniform
                        uint32_t v0[16], v1[16];
                        TMEM_LD16(taddr + 32 * hgrp, v0);
                        TMEM_LD16(taddr + 32 * hgrp + 16, v1);
                        tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            acc[32 * hgrp + i] += __uint_as_float(v0[i]);
                            acc[32 * hgrp + 16 + i] += __uint_as_float(v1[i]);
                        }
                    }
                }
                uint32_t r0, r1;
                tmem_ld2(taddr + 64, r0, r1);
                tmem_wait_ld();
                rsum += __uint_as_float(r0) + __uint_as_float(r1);
                tc_fence_before();
                mbar_arrive(bar_acc_empty + 8 * slot);
            }
            if (!live) break;
            // ---- the row's end: L^T H rows to the staging buffer, then each H^T H row
            // m adds (L^T H)[m][c] + (L^T H)[c][m] over its lower triangle
            if (!hh) {
#pragma unroll
                for (int c = 0; c < 16; ++c)
                    *chunk_ptr(T, m, c) = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
                T[4096 + m] = rsum;
            }
            named_bar(bar_id, 128);
            if (hh) {
                float4* out = reinterpret_cast<float4*>(a.gram + slot_out * kGramSlotFloats);
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    if (4 * c <= m) {
                        const float4 t = ld_chunk(T, m, c);
                        float4 o;
                        o.x = acc[4 * c + 0] + t.x + T[sw64(4 * c + 0, m)];
                        o.y = acc[4 * c + 1] + t.y + T[sw64(4 * c + 1, m)];
                        o.z = acc[4 * c + 2] + t.z + T[sw64(4 * c + 2, m)];
                        o.w = acc[4 * c + 3] + t.w + T[sw64(4 * c + 3, m)];
                        st_once(out + gram_chunk_offset(c) + m - 4 * c, o, once);
                    }
                }
                reinterpret_cast<float*>(out)[4 * kGramChunks + m] = rsum + T[4096 + m];
            }
            named_bar(bar_id, 128);  // the staging buffer is reused by the group's next row
            if (q == 0 && lane == 0) mbar_arrive(bar_row_empty + 8 * rs);
        }
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

template <bool kBf16>
static cudaError_t launch_gram(const RowArgs& a, int num_sms, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(rows_gram_kernel<kBf16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    // setmaxnreg.inc takes registers that other warps released from what the CTA was
    // launched with (the compiled count times the threads): if the split's total were
    // above that, the drain warps' increase would never be granted.  Refuse the launch
    // instead (the compiled count can sit below the launch bound).
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, rows_gram_kernel<kBf16>);
    if (e != cudaSuccess) return e;
    const long split = 32L * (8 * kProdRegs + 4 * kDrainRegs);
    if (split > (long)fa.numRegs * kThreads) return cudaErrorInvalidConfiguration;
    const int64_t ctas = (int64_t)kGramCtasPerSm * num_sms;
    const int64_t grid = a.nrows < ctas ? a.nrows : ctas;
    rows_gram_kernel<kBf16><<<(unsigned)grid, kThreads, kSmemBytes, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rows_gram(const RowArgs& a, int num_sms, cudaStream_t s)
{
    if (a.nrows <= 0) return cudaSuccess;
    return a.bf16 ? launch_gram<true>(a, num_sms, s) : launch_gram<false>(a, num_sms, s);
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
