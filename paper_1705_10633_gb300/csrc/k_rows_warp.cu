// k_rows_warp.cu -- per-row conditional update on CUDA cores, one warp per row.
//
// For row i of one side (Alg. 1 inner loops; Sec. 2 and Sec. 3.1):
//   Lambda_i = Lambda_X + alpha sum_c y_c y_c^T      (Gram of gathered rows)
//   b_i      = alpha sum_c r_c y_c + Lambda_X mu_X
//   L L^T = Lambda_i (Cholesky instead of an inverse, Sec. 3.1)
//   x_i = L^{-T} (L^{-1} b_i + z),  z ~ N(0, I) from the row's Philox stream
// which equals mean + L^{-T} z with mean = Lambda_i^{-1} b_i.
//
// Layout inside the warp (KT = K rounded up to 16, K <= 64):
//   gather : 32 ratings per chunk, each lane loads float4 pieces of the
//            gathered rows into a shared-memory stage (coalesced 16-B loads);
//   Gram   : lane owns rows i1 = lane and i2 = 63 - lane of Lambda_i (65
//            lower-triangle entries for KT = 64, balanced) and adds
//            y[i] * y[0..KT) per rating, y read as shared-memory broadcasts;
//   Cholesky: on the same registers; column k of L is published through
//            shared memory each step and every lane updates its own rows.
//   solves : forward substitution with the pivot broadcast by shuffle, back
//            substitution reading L from shared memory.
//
// Long rows (Sec. 3.2: items with many ratings are split into smaller tasks so that
// one item does not hold up the rest): the launch's work items are first the
// segments of its split rows, then its other rows.  A segment's warp accumulates
// the Gram rows and right-hand side of its ratings only and writes them to global
// memory; the warp that finishes a row's last segment (a counter per row, taken
// after a device-wide fence) adds the row's partials in segment order -- the sum
// is the same whichever warp comes last -- and factors and samples the row.  No
// warp waits for another.
#include "bpmf_internal.cuh"
#include "philox.cuh"
#include "rows_common.cuh"

namespace bpmf {

constexpr int kWarpsPerCta = 4;
constexpr int kChunk = 32;

template <int KT>
struct WarpLayout {
    static constexpr int NR1 = KT < 32 ? KT : 32;  // rows owned as i1 = lane
    static constexpr bool TWO = KT > 32;           // rows owned as i2 = 63 - lane
    static constexpr int LD = KT + 1;              // row stride of the square buffer
    static constexpr int F4 = KT / 4;              // float4 per gathered row
    static constexpr int RPI = 32 / F4;            // gathered rows per warp load
    static constexpr int STAGE = kChunk * KT;
    static constexpr int SQ = KT * LD;
    static constexpr int PER_WARP = STAGE + SQ + 2 * KT + KT + KT + kChunk;  // floats
    static constexpr int PER_WARP_ALIGNED = (PER_WARP + 3) & ~3;
    // a segment's partial: NR1 + (TWO ? KT : 0) Gram rows' entries and two right-hand
    // side entries per lane, entry-major (32 consecutive floats per entry)
    static constexpr int NA = TWO ? KT : 0;
    static constexpr int PART = (NR1 + NA + 2) * 32;
};

// One chunk of up to 32 ratings starting at `base`: index and value loads, the
// gathered rows of Y into the stage (rows >= cnt zero), values into rb.
template <int KT>
__device__ __forceinline__ void gather_chunk(const RowArgs& a, int64_t base, int cnt, float* stage,
                                             float* rb, int lane)
{
    using W = WarpLayout<KT>;
    int c = 0;
    float r = 0.f;
    if (lane < cnt) {
        c = __ldg(a.idx + base + lane);
        r = __ldg(a.val + base + lane);
    }
    rb[lane] = r;
    const int f = lane % W::F4, sub = lane / W::F4;
#pragma unroll 4
    for (int it = 0; it < kChunk / W::RPI; ++it) {
        const int qq = it * W::RPI + sub;
        const int cq = __shfl_sync(kFullMask, c, qq & 31);
        if (sub < W::RPI) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (qq < cnt) v = __ldg(reinterpret_cast<const float4*>(a.Y + (int64_t)cq * a.ldy) + f);
            reinterpret_cast<float4*>(stage + qq * KT)[f] = v;
        }
    }
    __syncwarp();
}

// Gram rows i1, i2 and right-hand side entries of ratings [p0, p1), added to the
// registers (the stage holds 32 gathered rows of Y at a time).
template <int KT>
__device__ __forceinline__ void accumulate_ratings(const RowArgs& a, int64_t p0, int64_t p1,
                                                   float* stage, float* rb, int lane, bool v1,
                                                   bool v2, float (&a1)[RowRegs<KT>::NR1],
                                                   float (&a2)[RowRegs<KT>::NA2], float& rhs1,
                                                   float& rhs2)
{
    using W = WarpLayout<KT>;
    const int i1 = lane, i2 = 63 - lane;
    for (int64_t base = p0; base < p1; base += kChunk) {
        const int cnt = (int)min((int64_t)kChunk, p1 - base);
        gather_chunk<KT>(a, base, cnt, stage, rb, lane);
        // one rating at a time: row i of the Gram += y[i] * y (lower part used)
#pragma unroll 2
        for (int qq = 0; qq < cnt; ++qq) {
            const float* srow = stage + qq * KT;
            const float rq = rb[qq];
            const float x1 = v1 ? srow[i1] : 0.f;
            const float x2 = v2 ? srow[i2] : 0.f;
            rhs1 = fmaf(rq, x1, rhs1);
            rhs2 = fmaf(rq, x2, rhs2);
#pragma unroll
            for (int j4 = 0; j4 < KT; j4 += 4) {
                const float4 y4 = *reinterpret_cast<const float4*>(srow + j4);
                const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j4 + u;
                    if (j < W::NR1) a1[j < W::NR1 ? j : 0] = fmaf(x1, yv[u], a1[j < W::NR1 ? j : 0]);
                    if (W::TWO) a2[W::TWO ? j : 0] = fmaf(x2, yv[u], a2[W::TWO ? j : 0]);
                }
            }
        }
        __syncwarp();
    }
}

// Rank-one route (Sec. 3.1, Sec. 3.2: cheaper for items with few ratings): a1 / a2
// start as the lane's rows of chol(Lambda_X) and take one rank-one update with
// sqrt(alpha) y per rating of [p0, p1); the right-hand side accumulates as on the
// Gram route.
template <int KT>
__device__ __forceinline__ void rank_one_ratings(const RowArgs& a, int64_t p0, int64_t p1,
                                                 float* stage, float* rb, int lane, bool v1,
                                                 bool v2, float (&a1)[RowRegs<KT>::NR1],
                                                 float (&a2)[RowRegs<KT>::NA2], float& rhs1,
                                                 float& rhs2, bool& bad)
{
    const int i1 = lane, i2 = 63 - lane;
    const float sqa = sqrtf(a.alpha);
    for (int64_t base = p0; base < p1; base += kChunk) {
        const int cnt = (int)min((int64_t)kChunk, p1 - base);
        gather_chunk<KT>(a, base, cnt, stage, rb, lane);
#pragma unroll 1
        for (int qq = 0; qq < cnt; ++qq) {
            const float* srow = stage + qq * KT;
            const float rq = rb[qq];
            const float y1 = v1 ? srow[i1] : 0.f;
            const float y2 = v2 ? srow[i2] : 0.f;
            rhs1 = fmaf(rq, y1, rhs1);
            rhs2 = fmaf(rq, y2, rhs2);
            warp_rank_one<KT>(a1, a2, sqa * y1, sqa * y2, lane, bad);
        }
        __syncwarp();
    }
}

template <int KT>
__device__ __forceinline__ void store_partial(float* pp, int lane, const float (&a1)[RowRegs<KT>::NR1],
                                              const float (&a2)[RowRegs<KT>::NA2], float rhs1,
                                              float rhs2)
{
    using W = WarpLayout<KT>;
#pragma unroll
    for (int j = 0; j < W::NR1; ++j) __stcg(pp + j * 32 + lane, a1[j]);
#pragma unroll
    for (int j = 0; j < W::NA; ++j) __stcg(pp + (W::NR1 + j) * 32 + lane, a2[W::TWO ? j : 0]);
    __stcg(pp + (W::NR1 + W::NA) * 32 + lane, rhs1);
    __stcg(pp + (W::NR1 + W::NA + 1) * 32 + lane, rhs2);
}

// L2 loads: the partials were written by other SMs during this launch.
template <int KT>
__device__ __forceinline__ void add_partial(const float* pp, int lane, float (&a1)[RowRegs<KT>::NR1],
                                            float (&a2)[RowRegs<KT>::NA2], float& rhs1, float& rhs2)
{
    using W = WarpLayout<KT>;
#pragma unroll
    for (int j = 0; j < W::NR1; ++j) a1[j] += __ldcg(pp + j * 32 + lane);
#pragma unroll
    for (int j = 0; j < W::NA; ++j) a2[W::TWO ? j : 0] += __ldcg(pp + (W::NR1 + j) * 32 + lane);
    rhs1 += __ldcg(pp + (W::NR1 + W::NA) * 32 + lane);
    rhs2 += __ldcg(pp + (W::NR1 + W::NA + 1) * 32 + lane);
}

// kR1 = false: the segments of the split rows, then rows nsplit .. nrows - nrank_one - 1
// of the bin on the Gram route; kR1 = true: the last nrank_one rows (the shortest) on
// the rank-one route.  Two instantiations keep each route's register budget its own.
// The kernel's work for one job: this CTA is block `bid` of the `nblocks` blocks the
// job's items are dealt over (items q = bid * 4 + warp, step 4 nblocks).
template <int KT, bool kR1>
__device__ __forceinline__ void rows_warp_body(const RowArgs& a, int64_t bid, int64_t nblocks)
{
    using W = WarpLayout<KT>;
    extern __shared__ float4 dyn_smem4[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    float* sm = reinterpret_cast<float*>(dyn_smem4) + wib * W::PER_WARP_ALIGNED;
    float* stage = sm;
    float* sq = stage + W::STAGE;
    float* colbuf = sq + W::SQ;
    float* dinv = colbuf + 2 * KT;
    float* zb = dinv + KT;
    float* rb = zb + KT;

    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    const int i1 = lane;
    const int i2 = 63 - lane;
    const bool v1 = i1 < KT;
    const bool v2 = W::TWO && i2 < KT;
    const int64_t nwarps = nblocks * kWarpsPerCta;
    bool bad = false;

    const int64_t nitems = kR1 ? a.nrank_one : a.nsegs + a.nrows - a.nsplit - a.nrank_one;
    for (int64_t q = bid * kWarpsPerCta + wib; q < nitems; q += nwarps) {
        // Gram rows i1, i2 accumulate in the registers the Cholesky works on
        float a1[RowRegs<KT>::NR1];
        float a2[RowRegs<KT>::NA2];
#pragma unroll
        for (int j = 0; j < W::NR1; ++j) a1[j] = 0.f;
#pragma unroll
        for (int j = 0; j < (W::TWO ? KT : 1); ++j) a2[j] = 0.f;
        float rhs1 = 0.f, rhs2 = 0.f;
        const bool is_seg = !kR1 && q < a.nsegs;
        int row = 0;
        int64_t p0, p1;
        if (is_seg) {
            p0 = __ldg(&a.segs[q].lo);
            p1 = __ldg(&a.segs[q].hi);
        } else {
            row = kR1 ? a.rows[a.nrows - a.nrank_one + q] : a.rows[a.nsplit + (q - a.nsegs)];
            p0 = a.ptr[row];
            p1 = a.ptr[row + 1];
        }
        constexpr bool rank_one = kR1;
        const float4* lct = reinterpret_cast<const float4*>(rank_one ? a.lamchol_ct : a.lam_ct);
        if constexpr (rank_one) {
            // the lane's rows of chol(Lambda_X) (chunk-transposed: coalesced float4 loads)
#pragma unroll
            for (int c = 0; c < W::NR1 / 4; ++c) {
                const float4 l4 = v1 ? __ldg(lct + c * KT + (v1 ? i1 : 0)) : make_float4(0.f, 0.f, 0.f, 0.f);
                a1[4 * c + 0] = v1 ? l4.x : (4 * c == 0 ? 1.f : 0.f);
                a1[4 * c + 1] = l4.y;
                a1[4 * c + 2] = l4.z;
                a1[4 * c + 3] = l4.w;
            }
            if (W::TWO) {
#pragma unroll
                for (int c = 0; c < KT / 4; ++c) {
                    const float4 l4 =
                        v2 ? __ldg(lct + c * KT + (v2 ? i2 : 0)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) a2[W::TWO ? 4 * c + u : 0] = lv[u];
                }
            }
            rank_one_ratings<KT>(a, p0, p1, stage, rb, lane, v1, v2, a1, a2, rhs1, rhs2, bad);
        } else {
            accumulate_ratings<KT>(a, p0, p1, stage, rb, lane, v1, v2, a1, a2, rhs1, rhs2);
        }
        if (is_seg) {
            store_partial<KT>(a.part + q * W::PART, lane, a1, a2, rhs1, rhs2);
            const Segment* sg = a.segs + q;
            const int slot = __ldg(&sg->slot), first = __ldg(&sg->first), count = __ldg(&sg->count);
            __threadfence();
            __syncwarp();
            unsigned int prev = 0;
            if (lane == 0) prev = atomicAdd(a.seg_done + slot, 1u);
            prev = __shfl_sync(kFullMask, prev, 0);
            if (prev + 1 != (unsigned int)count) continue;  // another warp finishes the row
            __threadfence();
#pragma unroll
            for (int j = 0; j < W::NR1; ++j) a1[j] = 0.f;
#pragma unroll
            for (int j = 0; j < (W::TWO ? KT : 1); ++j) a2[j] = 0.f;
            rhs1 = rhs2 = 0.f;
            for (int g = 0; g < count; ++g)
                add_partial<KT>(a.part + (int64_t)(first + g) * W::PART, lane, a1, a2, rhs1, rhs2);
            if (lane == 0) a.seg_done[slot] = 0u;  // ready for the next launch
            row = __ldg(&sg->row);
        }
        // Gram route: Lambda_i rows = Lambda_X rows + alpha * Gram rows.  Lambda_X comes
        // from its chunk-transposed copy (float4 (i, 4c..4c+3) at c * KT + i): the lanes'
        // loads of one chunk are consecutive 16-B words, not 32 rows apart.
        if constexpr (!rank_one) {
#pragma unroll
            for (int c = 0; c < W::NR1 / 4; ++c) {
                const float4 l4 = v1 ? __ldg(lct + c * KT + (v1 ? i1 : 0)) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = 4 * c + u;
                    a1[j] = v1 ? fmaf(a.alpha, a1[j], lv[u]) : (j == 0 ? 1.f : 0.f);
                }
            }
            if (W::TWO) {
#pragma unroll
                for (int c = 0; c < KT / 4; ++c) {
                    const float4 l4 =
                        v2 ? __ldg(lct + c * KT + (v2 ? i2 : 0)) : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = W::TWO ? 4 * c + u : 0;
                        a2[j] = v2 ? fmaf(a.alpha, a2[j], lv[u]) : 0.f;
                    }
                }
            }
        }
        // b = alpha * rhs + Lambda_X mu_X
        float b1 = v1 ? fmaf(a.alpha, rhs1, __ldg(a.lammu + i1)) : 0.f;
        float b2 = v2 ? fmaf(a.alpha, rhs2, __ldg(a.lammu + i2)) : 0.f;

        if constexpr (rank_one) warp_forward<KT>(a1, a2, b1, b2, dinv, lane);
        else warp_factor<KT>(a1, a2, b1, b2, colbuf, dinv, lane, bad);
        float x1, x2, m1, m2;
        warp_sample_tail<KT>(a1, a2, b1, b2, dinv, zb, sq, lane, a.K, a.seed, (uint32_t)row, sweep,
                             a.c3, a.means != nullptr, x1, x2, m1, m2);
        store_row<KT>(a, row, lane, x1, x2, m1, m2);
        __syncwarp();
    }
    if (bad && lane == 0) atomicOr(&a.ctl->status, kStatusNotPD);
}

template <int KT, bool kR1>
__global__ void __launch_bounds__(kWarpsPerCta * 32) rows_warp_kernel(RowArgs a)
{
    rows_warp_body<KT, kR1>(a, blockIdx.x, gridDim.x);
}

// Many jobs in one launch: each CTA finds its job's entry and runs the job's work as
// block bid of the job's count (the same per-row arithmetic as a launch of its own).
// The job's arguments are staged in shared memory: the body reads them where it needs
// them, as a launch of its own reads its parameters, instead of holding a copy of the
// whole struct in registers (which cost the K = 16 kernel half its occupancy and the
// K = 64 one spills).
template <int KT, bool kR1>
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    rows_warp_batch_kernel(const BatchEntry<RowArgs>* __restrict__ t, int n)
{
    __shared__ __align__(16) unsigned char args_raw[sizeof(RowArgs)];
    __shared__ int64_t span[2];
    if (threadIdx.x == 0) {
        const int j = batch_find(t, n, (int)blockIdx.x);
        span[0] = (int64_t)blockIdx.x - t[j].first;
        span[1] = t[j].count;
        // the whole struct, 4 bytes at a time (RowArgs is 8-byte aligned)
        const unsigned int* src = reinterpret_cast<const unsigned int*>(&t[j].args);
        unsigned int* dst = reinterpret_cast<unsigned int*>(args_raw);
        for (int w = 0; w < (int)(sizeof(RowArgs) / 4); ++w) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    rows_warp_body<KT, kR1>(*reinterpret_cast<const RowArgs*>(args_raw), span[0], span[1]);
}

template <int KT, bool kR1>
static cudaError_t warp_kernel_attrs(size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(rows_warp_kernel<KT, kR1>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rows_warp_kernel<KT, kR1>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rows_warp_batch_kernel<KT, kR1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(rows_warp_batch_kernel<KT, kR1>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int KT, bool kR1>
static cudaError_t launch_route(const RowArgs& a, int num_sms, cudaStream_t s)
{
    using W = WarpLayout<KT>;
    const int64_t nitems = kR1 ? a.nrank_one : a.nsegs + a.nrows - a.nsplit - a.nrank_one;
    if (nitems <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * (size_t)W::PER_WARP_ALIGNED * kWarpsPerCta;
    // all of the unified L1 / shared memory as shared, so residency is set by registers
    cudaError_t e = warp_kernel_attrs<KT, kR1>(smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_warp_kernel<KT, kR1>,
                                                      kWarpsPerCta * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t need = (nitems + kWarpsPerCta - 1) / kWarpsPerCta;
    int64_t grid = (int64_t)num_sms * per_sm;
    if (need < grid) grid = need;
    if (grid < 1) return cudaSuccess;
    rows_warp_kernel<KT, kR1><<<(unsigned)grid, kWarpsPerCta * 32, smem, s>>>(a);
    return cudaGetLastError();
}

int warp_partial_floats(int kp)
{
    switch (kp) {
    case 16: return WarpLayout<16>::PART;
    case 32: return WarpLayout<32>::PART;
    case 48: return WarpLayout<48>::PART;
    default: return WarpLayout<64>::PART;
    }
}

// The Gram-route launch, then the rank-one launch (each skipped when it has no work).
template <int KT>
static cudaError_t launch_kt(const RowArgs& a, int num_sms, cudaStream_t s)
{
    cudaError_t e = launch_route<KT, false>(a, num_sms, s);
    if (e == cudaSuccess) e = launch_route<KT, true>(a, num_sms, s);
    return e;
}

cudaError_t launch_rows_warp(const RowArgs& a, int kp, int num_sms, cudaStream_t s)
{
    switch (kp) {
    case 16: return launch_kt<16>(a, num_sms, s);
    case 32: return launch_kt<32>(a, num_sms, s);
    case 48: return launch_kt<48>(a, num_sms, s);
    case 64: return launch_kt<64>(a, num_sms, s);
    default: return cudaErrorInvalidValue;
    }
}

int rows_warp_launches(const RowArgs& a)
{
    return (a.nsegs + a.nrows - a.nsplit - a.nrank_one > 0 ? 1 : 0) + (a.nrank_one > 0 ? 1 : 0);
}

int64_t rows_warp_items(const RowArgs& a, bool rank_one)
{
    return rank_one ? a.nrank_one : a.nsegs + a.nrows - a.nsplit - a.nrank_one;
}

template <int KT, bool kR1>
static cudaError_t launch_batch_kt(const BatchEntry<RowArgs>* t, int n, int64_t blocks,
                                   cudaStream_t s)
{
    using W = WarpLayout<KT>;
    const size_t smem = sizeof(float) * (size_t)W::PER_WARP_ALIGNED * kWarpsPerCta;
    cudaError_t e = warp_kernel_attrs<KT, kR1>(smem);
    if (e != cudaSuccess) return e;
    rows_warp_batch_kernel<KT, kR1><<<(unsigned)blocks, kWarpsPerCta * 32, smem, s>>>(t, n);
    return cudaGetLastError();
}

cudaError_t launch_rows_warp_batch(const BatchEntry<RowArgs>* t, int n, int64_t blocks, int kp,
                                   bool rank_one, cudaStream_t s)
{
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    switch (kp * 2 + (rank_one ? 1 : 0)) {
    case 32: return launch_batch_kt<16, false>(t, n, blocks, s);
    case 33: return launch_batch_kt<16, true>(t, n, blocks, s);
    case 64: return launch_batch_kt<32, false>(t, n, blocks, s);
    case 65: return launch_batch_kt<32, true>(t, n, blocks, s);
    case 96: return launch_batch_kt<48, false>(t, n, blocks, s);
    case 97: return launch_batch_kt<48, true>(t, n, blocks, s);
    case 128: return launch_batch_kt<64, false>(t, n, blocks, s);
    case 129: return launch_batch_kt<64, true>(t, n, blocks, s);
    default: return cudaErrorInvalidValue;
    }
}

int rows_warp_resident_blocks(int kp)
{
    int per_sm = 1;
    auto occ = [&](auto kernel, size_t smem) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWarpsPerCta * 32, smem) !=
            cudaSuccess) {
            cudaGetLastError();
            per_sm = 1;
        }
    };
    switch (kp) {
    case 16: warp_kernel_attrs<16, false>(sizeof(float) * WarpLayout<16>::PER_WARP_ALIGNED * kWarpsPerCta);
             occ(rows_warp_batch_kernel<16, false>, sizeof(float) * WarpLayout<16>::PER_WARP_ALIGNED * kWarpsPerCta); break;
    case 32: warp_kernel_attrs<32, false>(sizeof(float) * WarpLayout<32>::PER_WARP_ALIGNED * kWarpsPerCta);
             occ(rows_warp_batch_kernel<32, false>, sizeof(float) * WarpLayout<32>::PER_WARP_ALIGNED * kWarpsPerCta); break;
    case 48: warp_kernel_attrs<48, false>(sizeof(float) * WarpLayout<48>::PER_WARP_ALIGNED * kWarpsPerCta);
             occ(rows_warp_batch_kernel<48, false>, sizeof(float) * WarpLayout<48>::PER_WARP_ALIGNED * kWarpsPerCta); break;
    default: warp_kernel_attrs<64, false>(sizeof(float) * WarpLayout<64>::PER_WARP_ALIGNED * kWarpsPerCta);
             occ(rows_warp_batch_kernel<64, false>, sizeof(float) * WarpLayout<64>::PER_WARP_ALIGNED * kWarpsPerCta); break;
    }
    return per_sm < 1 ? 1 : per_sm;
}

}  // namespace bpmf
