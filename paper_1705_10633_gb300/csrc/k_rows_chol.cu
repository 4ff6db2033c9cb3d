// k_rows_chol.cu -- factor, solve and sample the long rows whose precision and
// right-hand side the Gram kernel (k_rows_tc.cu) left in the scratch (Sec. 3.1: a
// Cholesky factorisation instead of an inverse; Alg. 1: the new vector is the
// conditional mean plus randomly sampled noise).
//
// One warp per row, eight warps per CTA, one CTA per SM, rows dealt round-robin
// over all warps of the grid (every row costs the same at K = 64).  Eight warps (two
// per SM sub-partition) already reach the SM's throughput on this code, which is bound
// by the shared-memory broadcasts and shuffles of the column steps: twelve were no
// faster, and eight leave each warp the registers to keep its rows without spills.
// Lane l loads rows l and 32 + l of Lambda_i from the row's scratch slot straight into
// registers (coalesced 16-B loads: the slot stores each float4 column chunk's rows
// consecutively), then runs the shifted right-looking factorisation with the forward
// solve fused (two columns a step, with paired FMAs), Philox noise and the back solve
// (rows_common.cuh), and stores the FP32 row and its 16-bit split.
#include "bpmf_internal.cuh"
#include "philox.cuh"
#include "rows_common.cuh"

namespace bpmf {
namespace {

constexpr int kCholWarps = 8;
// per warp: L^T (64 x kLtLd), 1 / diag (64), noise (64); per CTA: Lambda_X packed like
// a slot and Lambda_X mu_X
constexpr int kCholWarpFloats = 64 * kLtLd + 64 + 64;
constexpr size_t kCholSmemBytes = ((size_t)kCholWarps * kCholWarpFloats + kGramSlotFloats) * 4;
static_assert(kCholSmemBytes <= 232448, "shared memory");

}  // namespace

__global__ void __launch_bounds__(kCholWarps * 32, 1) rows_chol_kernel(RowArgs a)
{
    extern __shared__ __align__(16) float chol_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4* prior4 = reinterpret_cast<float4*>(chol_smem + kCholWarps * kCholWarpFloats);
    const float* prior_mu = chol_smem + kCholWarps * kCholWarpFloats + 4 * kGramChunks;
    {
        // Lambda_X comes chunk-transposed (float4 (i, 4c..4c+3) at c * 64 + i); packed
        // here like a slot, so that a lane's prior chunks sit where its Gram chunks do
        const float4* lam_ct = reinterpret_cast<const float4*>(a.lam_ct);
        for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
            const int i = e & 63, c = e >> 6;
            if (4 * c <= i) prior4[gram_chunk_offset(c) + i - 4 * c] = __ldg(lam_ct + c * 64 + i);
        }
        for (int e = threadIdx.x; e < 64; e += blockDim.x)
            const_cast<float*>(prior_mu)[e] = __ldg(a.lammu + e);
        __syncthreads();
    }
    float* M = chol_smem + warp * kCholWarpFloats;
    float* dinv = M + 64 * kLtLd;
    float* zb = dinv + 64;
    const uint32_t sweep = (uint32_t)a.ctl->sweep;
    // a Gram launch that gave up on a wait left its slots unfinished: nothing to factor
    if (*reinterpret_cast<volatile unsigned int*>(&a.ctl->status) & kStatusTimeout) return;
    bool bad = false;
    const int64_t W = (int64_t)gridDim.x * kCholWarps;
    for (int64_t p = (int64_t)blockIdx.x * kCholWarps + warp; p < a.nrows; p += W) {
        const int row = __ldg(a.rows + p);
        const float4* src = reinterpret_cast<const float4*>(a.gram + p * kGramSlotFloats);
        float2 a1[16], a2[32];  // column pairs
        // Lambda_i = Lambda_X + alpha Gram, b_i = Lambda_X mu_X + alpha (H + L)^T r.
        // Row lane: chunk columns c <= lane / 4; row 32 + lane: c <= 8 + lane / 4 (the
        // rest of each row lies above the diagonal and is never used)
        const float alpha = a.alpha;
        auto lambda4 = [&](int at) {
            const float4 g = __ldg(src + at), px = prior4[at];
            return make_float4(fmaf(alpha, g.x, px.x), fmaf(alpha, g.y, px.y),
                               fmaf(alpha, g.z, px.z), fmaf(alpha, g.w, px.w));
        };
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * c <= lane) v = lambda4(gram_chunk_offset(c) + lane - 4 * c);
            a1[2 * c + 0] = make_float2(v.x, v.y);
            a1[2 * c + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * c <= 32 + lane) v = lambda4(gram_chunk_offset(c) + 32 + lane - 4 * c);
            a2[2 * c + 0] = make_float2(v.x, v.y);
            a2[2 * c + 1] = make_float2(v.z, v.w);
        }
        const float* bsrc = a.gram + p * kGramSlotFloats + 4 * kGramChunks;
        const float b1 = fmaf(alpha, __ldg(bsrc + lane), prior_mu[lane]);
        const float b2 = fmaf(alpha, __ldg(bsrc + 32 + lane), prior_mu[32 + lane]);
        __syncwarp();  // every lane's back solve of the previous row is done with M
        float x1, x2, m1, m2;
        factor_solve_sample_rl64(a1, a2, b1, b2, M, dinv, zb, lane, a.K, a.seed,
                                 (uint32_t)row, sweep, a.c3, a.means != nullptr, x1, x2, m1, m2,
                                 bad);
        store_row_panels(a, row, lane, x1, x2, m1, m2);
    }
    if (bad && lane == 0) atomicOr(&a.ctl->status, kStatusNotPD);
}

cudaError_t launch_rows_chol(const RowArgs& a, int num_sms, cudaStream_t s)
{
    if (a.nrows <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(rows_chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kCholSmemBytes);
    if (e != cudaSuccess) return e;
    const int64_t need = (a.nrows + kCholWarps - 1) / kCholWarps;
    const int64_t grid = need < num_sms ? need : num_sms;
    rows_chol_kernel<<<(unsigned)grid, kCholWarps * 32, kCholSmemBytes, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bpmf
