// rows_common.cuh -- the per-row factor / solve / sample step shared by the
// row-update kernels (Sec. 3.1: Cholesky instead of an inverse; Alg. 1: the new
// vector is the conditional mean plus randomly sampled noise).
//
// One warp holds one K x K precision (K padded to KT, identity in the padding):
// lane l owns row i1 = l (columns 0..31) and row i2 = 63 - l (columns 0..KT-1),
// 65 lower-triangle entries per lane at KT = 64.  On return the lane holds its
// entries of x = L^{-T}(L^{-1} b + z) (and of the mean L^{-T} L^{-1} b).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "bpmf_internal.cuh"
#include "philox.cuh"

namespace bpmf {

constexpr unsigned kFullMask = 0xffffffffu;

// FP16 hi/lo split of an FP32 value: x = hi + lo + O(2^-22 |x|).
__device__ __forceinline__ void split_f16(float x, __half& hi, __half& lo)
{
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

// The 16-bit copies of a factor entry the tensor-core kernel gathers: the FP16 split
// (hi, lo), or with bf16 set the BF16 rounding of x (hi) and of the remainder (lo).
__device__ __forceinline__ void split16(float x, bool bf16, __half& hi, __half& lo)
{
    if (bf16) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi = __ushort_as_half(__bfloat16_as_ushort(h));
        lo = __ushort_as_half(__bfloat16_as_ushort(__float2bfloat16_rn(x - __bfloat162float(h))));
    } else {
        split_f16(x, hi, lo);
    }
}

template <int KT>
struct RowRegs {
    static constexpr int NR1 = KT < 32 ? KT : 32;  // columns of row i1 kept in registers
    static constexpr bool TWO = KT > 32;           // a second row i2 = 63 - lane exists
    static constexpr int NA2 = TWO ? KT : 1;
    static constexpr int LD = KT + 1;              // row stride of the square buffer
};

// Pivot work of column k (a compile-time index once the caller's loop is unrolled)
// for the warp layout (rows i1 = lane, i2 = 63 - lane): scales the lane's entries of
// column k into L[r][k] (the diagonal owner gets L[k][k]), returns them in l1 / l2
// (zero above the diagonal), applies y_k to the right-hand side (forward solve
// fused: b_k becomes y_k, rows below lose L[r][k] y_k), writes 1 / L[k][k] to dinv
// and publishes the column in the buffer of k's parity.  Selects, not branches.
template <int KT>
__device__ __forceinline__ void warp_pivot(int k, float (&a1)[RowRegs<KT>::NR1],
                                           float (&a2)[RowRegs<KT>::NA2], float& b1, float& b2,
                                           float& l1, float& l2, float* colbuf, float* dinv,
                                           int lane, bool v1, bool v2, bool& bad)
{
    using R = RowRegs<KT>;
    const int i1 = lane, i2 = 63 - lane;
    float* cb = colbuf + (k & 1) * KT;
    const int owner = k < 32 ? k : 63 - k;
    const float pv = k < R::NR1 ? a1[k < R::NR1 ? k : 0] : a2[R::TWO ? k : 0];
    float piv = __shfl_sync(kFullMask, pv, owner);
    const float bk = __shfl_sync(kFullMask, k < 32 ? b1 : b2, owner);
    if (!(piv > 0.f && piv < INFINITY)) {  // also catches NaN
        bad = true;
        piv = 1.f;
    }
    const float rinv = rsqrtf(piv);
    const float yk = bk * rinv;
    if (lane == 0) dinv[k] = rinv;
    l1 = l2 = 0.f;
    if (k < R::NR1) {
        const int kk = k < R::NR1 ? k : 0;
        const bool below = i1 > k;
        a1[kk] = below ? a1[kk] * rinv : (i1 == k ? piv * rinv : a1[kk]);
        l1 = below ? a1[kk] : 0.f;
        b1 = below ? fmaf(-l1, yk, b1) : (i1 == k ? yk : b1);
        if (below && v1) cb[i1] = l1;
    }
    if (R::TWO) {
        const int kk = R::TWO ? k : 0;
        const bool below = i2 > k;
        a2[kk] = below ? a2[kk] * rinv : (i2 == k ? piv * rinv : a2[kk]);
        l2 = below ? a2[kk] : 0.f;
        b2 = below ? fmaf(-l2, yk, b2) : (i2 == k ? yk : b2);
        if (below && v2) cb[i2] = l2;
    }
}

// Right-looking Cholesky of the lane's two register rows (rows i1 = lane, i2 = 63 -
// lane of Lambda_i) with the forward solve fused: on return a1 / a2 hold the rows of
// L, b1 / b2 the entries of y = L^{-1} b, dinv the inverse diagonal.  Step k first
// updates column k + 1 and does its pivot work, then the rest of its update (the
// next pivot's latency overlaps this step's FMAs).  colbuf: 2*KT floats.
template <int KT>
__device__ __forceinline__ void warp_factor(float (&a1)[RowRegs<KT>::NR1],
                                            float (&a2)[RowRegs<KT>::NA2], float& b1, float& b2,
                                            float* colbuf, float* dinv, int lane, bool& bad)
{
    using R = RowRegs<KT>;
    const bool v1 = lane < KT;
    const bool v2 = R::TWO && 63 - lane < KT;
    float l1, l2;
    warp_pivot<KT>(0, a1, a2, b1, b2, l1, l2, colbuf, dinv, lane, v1, v2, bad);
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        __syncwarp();  // column k of L is in its buffer
        const float* cb = colbuf + (k & 1) * KT;
        float nl1 = 0.f, nl2 = 0.f;
        if (k + 1 < KT) {
            const int j = k + 1;
            const float c = cb[j];
            if (j < R::NR1) a1[j < R::NR1 ? j : 0] = fmaf(-l1, c, a1[j < R::NR1 ? j : 0]);
            if (R::TWO) a2[R::TWO ? j : 0] = fmaf(-l2, c, a2[R::TWO ? j : 0]);
            warp_pivot<KT>(j, a1, a2, b1, b2, nl1, nl2, colbuf, dinv, lane, v1, v2, bad);
        }
#pragma unroll
        for (int j4 = ((k + 2) / 4) * 4; j4 < KT; j4 += 4) {
            const float4 cv = *reinterpret_cast<const float4*>(cb + j4);
            const float cj[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j4 + u;
                if (j > k + 1) {
                    if (j < R::NR1) a1[j < R::NR1 ? j : 0] = fmaf(-l1, cj[u], a1[j < R::NR1 ? j : 0]);
                    if (R::TWO) a2[R::TWO ? j : 0] = fmaf(-l2, cj[u], a2[R::TWO ? j : 0]);
                }
            }
        }
        l1 = nl1;
        l2 = nl2;
    }

}

// Rank-one update (Sec. 3.1: for few ratings the factor of the prior precision is
// updated instead of factoring the Gram): L L^T + x x^T = L' L'^T for lower L with a
// positive diagonal, one Givens rotation per column (the classical LINPACK-style
// update): r = sqrt(L_kk^2 + x_k^2), c = L_kk / r, s = x_k / r, L'_kk = r and for rows
// i > k  L'_ik = c L_ik + s x_i,  x_i <- c x_i - s L_ik.  Rows as in warp_factor; x1 / x2
// are the lane's entries of x (consumed).
template <int KT>
__device__ __forceinline__ void warp_rank_one(float (&a1)[RowRegs<KT>::NR1],
                                              float (&a2)[RowRegs<KT>::NA2], float x1, float x2,
                                              int lane, bool& bad)
{
    using R = RowRegs<KT>;
    const int i1 = lane, i2 = 63 - lane;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const int owner = k < 32 ? k : 63 - k;
        const float lk = k < R::NR1 ? a1[k < R::NR1 ? k : 0] : a2[R::TWO ? k : 0];
        float lkk = __shfl_sync(kFullMask, lk, owner);
        const float xk = __shfl_sync(kFullMask, k < 32 ? x1 : x2, owner);
        if (!(lkk > 0.f && lkk < INFINITY)) {  // also catches NaN
            bad = true;
            lkk = 1.f;
        }
        const float q = fmaf(lkk, lkk, xk * xk);
        const float rinv = rsqrtf(q);
        const float c = lkk * rinv, sn = xk * rinv, r = q * rinv;
        if (k < R::NR1) {
            const int kk = k < R::NR1 ? k : 0;
            const float t = a1[kk];
            const bool below = i1 > k;
            a1[kk] = below ? fmaf(c, t, sn * x1) : (i1 == k ? r : t);
            x1 = below ? fmaf(c, x1, -sn * t) : x1;
        }
        if (R::TWO) {
            const int kk = R::TWO ? k : 0;
            const float t = a2[kk];
            const bool below = i2 > k;
            a2[kk] = below ? fmaf(c, t, sn * x2) : (i2 == k ? r : t);
            x2 = below ? fmaf(c, x2, -sn * t) : x2;
        }
    }
}

// Forward solve y = L^{-1} b on the lane's register rows of L (b1 / b2 become y),
// writing the inverse diagonal to dinv.
template <int KT>
__device__ __forceinline__ void warp_forward(const float (&a1)[RowRegs<KT>::NR1],
                                             const float (&a2)[RowRegs<KT>::NA2], float& b1,
                                             float& b2, float* dinv, int lane)
{
    using R = RowRegs<KT>;
    const int i1 = lane, i2 = 63 - lane;
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const int owner = k < 32 ? k : 63 - k;
        const float lk = k < R::NR1 ? a1[k < R::NR1 ? k : 0] : a2[R::TWO ? k : 0];
        const float lkk = __shfl_sync(kFullMask, lk, owner);
        const float bk = __shfl_sync(kFullMask, k < 32 ? b1 : b2, owner);
        const float rinv = __frcp_rn(lkk);
        const float yk = bk * rinv;
        if (lane == 0) dinv[k] = rinv;
        if (k < R::NR1) {
            const float l = a1[k < R::NR1 ? k : 0];
            b1 = i1 > k ? fmaf(-l, yk, b1) : (i1 == k ? yk : b1);
        }
        if (R::TWO) {
            const float l = a2[R::TWO ? k : 0];
            b2 = i2 > k ? fmaf(-l, yk, b2) : (i2 == k ? yk : b2);
        }
    }
}

// After the factor and forward solve (a1 / a2 = rows of L, b1 / b2 = y, dinv):
// x = L^{-T} (y + z) with z ~ N(0, I) from the row's Philox stream, and the
// conditional mean L^{-T} y.  zb: KT floats, sq: KT x LD (L is written here for the
// back solve).
template <int KT>
__device__ __forceinline__ void warp_sample_tail(const float (&a1)[RowRegs<KT>::NR1],
                                                 const float (&a2)[RowRegs<KT>::NA2], float b1,
                                                 float b2, const float* dinv, float* zb,
                                                 float* sq, int lane, int K, uint64_t seed,
                                                 uint32_t row, uint32_t sweep, uint32_t c3,
                                                 bool want_means, float& x1, float& x2,
                                                 float& m1, float& m2)
{
    using R = RowRegs<KT>;
    const int i1 = lane, i2 = 63 - lane;
    const bool v1 = i1 < KT;
    const bool v2 = R::TWO && i2 < KT;
    // ---- noise z (zero beyond K) and L into the square buffer for the back solve
    if (lane < KT / 4) {
        const float4 z4 = normals4_f32(seed, (uint32_t)lane, row, sweep, c3);
        const int kk = 4 * lane;
        zb[kk + 0] = kk + 0 < K ? z4.x : 0.f;
        zb[kk + 1] = kk + 1 < K ? z4.y : 0.f;
        zb[kk + 2] = kk + 2 < K ? z4.z : 0.f;
        zb[kk + 3] = kk + 3 < K ? z4.w : 0.f;
    }
#pragma unroll
    for (int j = 0; j < R::NR1; ++j)
        if (v1 && j <= i1) sq[i1 * R::LD + j] = a1[j];
    if (R::TWO) {
#pragma unroll
        for (int j = 0; j < KT; ++j)
            if (v2 && j <= i2) sq[i2 * R::LD + j] = a2[R::TWO ? j : 0];
    }
    __syncwarp();
    float t1 = b1 + (v1 ? zb[i1] : 0.f);
    float t2 = b2 + (v2 ? zb[i2] : 0.f);
    float n1 = b1, n2 = b2;

    // ---- back substitution x = L^{-T} t (and the mean from y alone); no register
    // indexing here, so the loop is only partly unrolled (keeps register pressure low).
    // Selects, not branches: the update of a row on or below i is computed and
    // dropped (its L entry is read from a clamped in-range index).
    const bool u1 = v1, u2 = v2;
#pragma unroll 4
    for (int i = KT - 1; i >= 0; --i) {
        const int owner = i < 32 ? i : 63 - i;
        const float di = dinv[i];
        const float ui = __shfl_sync(kFullMask, i < 32 ? t1 : t2, owner) * di;
        const float* Lrow = sq + i * R::LD;
        const bool lo1 = u1 && i1 < i;
        const float la = Lrow[lo1 ? i1 : 0];
        t1 = i1 == i ? ui : (lo1 ? fmaf(-la, ui, t1) : t1);
        float lb = 0.f;
        bool lo2 = false;
        if (R::TWO) {
            lo2 = u2 && i2 < i;
            lb = Lrow[lo2 ? i2 : 0];
            t2 = i2 == i ? ui : (lo2 ? fmaf(-lb, ui, t2) : t2);
        }
        if (want_means) {
            const float mi = __shfl_sync(kFullMask, i < 32 ? n1 : n2, owner) * di;
            n1 = i1 == i ? mi : (lo1 ? fmaf(-la, mi, n1) : n1);
            if (R::TWO) n2 = i2 == i ? mi : (lo2 ? fmaf(-lb, mi, n2) : n2);
        }
    }
    x1 = t1;
    x2 = t2;
    m1 = n1;
    m2 = n2;
}

// Factor, forward solve and sample (the Gram route): colbuf 2*KT floats, dinv KT,
// zb KT, sq KT x LD.
template <int KT>
__device__ __forceinline__ void factor_solve_sample(float (&a1)[RowRegs<KT>::NR1],
                                                    float (&a2)[RowRegs<KT>::NA2], float b1,
                                                    float b2, float* colbuf, float* dinv,
                                                    float* zb, float* sq, int lane, int K,
                                                    uint64_t seed, uint32_t row, uint32_t sweep,
                                                    uint32_t c3, bool want_means, float& x1,
                                                    float& x2, float& m1, float& m2, bool& bad)
{
    warp_factor<KT>(a1, a2, b1, b2, colbuf, dinv, lane, bad);
    warp_sample_tail<KT>(a1, a2, b1, b2, dinv, zb, sq, lane, K, seed, row, sweep, c3, want_means,
                         x1, x2, m1, m2);
}

// ---------------------------------------------------------------------------
// K = 64 matrices in shared memory.  Element (i, j) sits at sw64(i, j): row-major
// with stride 64 and the 16-B chunk index XOR-ed with (i & 7).  Eight lanes that
// access the same chunk of eight consecutive rows (float4), and 32 lanes that
// access 32 consecutive columns of one row, both hit distinct banks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int sw64(int i, int j)
{
    return i * 64 + (((j >> 2) ^ (i & 7)) << 2) + (j & 3);
}

__device__ __forceinline__ float4* chunk_ptr(float* M, int i, int c)
{
    return reinterpret_cast<float4*>(M + i * 64 + ((c ^ (i & 7)) << 2));
}

__device__ __forceinline__ float4 ld_chunk(const float* M, int i, int c)
{
    return *reinterpret_cast<const float4*>(M + i * 64 + ((c ^ (i & 7)) << 2));
}


// The K = 64 factor's transpose L^T in a warp's buffer: row j holds column j of L,
// L[r][j] at j * kLtLd + r - (j & ~1) (chol_pivot).  The padded row (68 floats) keeps
// the row stores conflict-free and spreads the back solve's loads of 32 different rows
// over the banks.
constexpr int kLtLd = 68;

// Pivot work of column j of a right-looking Cholesky with the forward solve fused,
// for K = 64 with lane l owning rows r1 = l and r2 = 32 + l; p1 / p2 are the lane's
// entries A[r1][j] / A[r2][j] after the updates of columns 0 .. j-1.  Gives the
// lane's L[r][j] in l1 / l2 (zero on and above the diagonal), applies y_j to the
// right-hand side (b_j becomes y_j = b_j / L[j][j], rows below lose L[r][j] y_j),
// writes 1 / L[j][j] to dinv and column j of L transposed into row j of M, L[r][j]
// at position r - (j & ~1) (a conflict-free row store): in a step over the columns
// k, k + 1 (k even) both columns' entries of row k + 2 + t then sit at position t + 2,
// in aligned pairs, and the row is both the columns' broadcast source and the back
// solve's copy of L.  Branch-free apart from the predicated stores.  HAS1 = false once the rows r1 are finished.
// A pivot that is not positive and finite is not caught here: 1 / L[j][j] then comes
// out non-positive, infinite or NaN, which the caller checks once per row.
template <bool HAS1>
__device__ __forceinline__ void chol_pivot(int j, float p1, float p2, float& b1, float& b2,
                                           float& l1, float& l2, float* M, float* dinv, int lane)
{
    const int r1 = lane, r2 = 32 + lane;
    const int owner = j & 31;
    const float piv = __shfl_sync(kFullMask, (HAS1 && j < 32) ? p1 : p2, owner);
    const float bk = __shfl_sync(kFullMask, (HAS1 && j < 32) ? b1 : b2, owner);
    const float rinv = rsqrtf(piv);
    const float yk = bk * rinv;
    if (lane == 0) dinv[j] = rinv;
    float* cb = M + j * kLtLd - (j & ~1);
    l1 = 0.f;
    if (HAS1) {
        const bool below = r1 > j;
        l1 = below ? p1 * rinv : 0.f;
        b1 = below ? fmaf(-l1, yk, b1) : (r1 == j ? yk : b1);
        if (below) cb[r1] = l1;
    }
    const bool below2 = r2 > j;
    l2 = below2 ? p2 * rinv : 0.f;
    b2 = below2 ? fmaf(-l2, yk, b2) : (r2 == j ? yk : b2);
    if (below2) cb[r2] = l2;
}

// Column pairs (k, k + 1), k = k0, k0 + 2, .. < k1, all even (the pivot work of
// column k0 already done: l1 / l2 hold the lane's L[r][k0] and row k0 of M its
// column).  The rows are kept in registers as pairs, "shifted": at pair k,
// (a[s].x, a[s].y) = (A[r][k + 2s], A[r][k + 2s + 1]).  A pair updates column k + 1
// by column k and does its pivot work, then the rest of each row twice,
//   A[r][c] -= L[r][k] L[c][k],  then  A[r][c] -= L[r][k + 1] L[c][k + 1]   (c >= k + 2),
// the same two roundings in the same order as two single-column steps, each with
// paired FMAs; reading a[s + 1] into a[s] slides the rows by two, so every register
// index stays static in a rolled loop.  Lookahead: the second update does column
// k + 2 first, then that column's pivot work, then the rest, so the pivot's latency
// overlaps the bulk of the FMAs.  P1 / P2: pairs of a1 / a2 still inside the matrix
// (P1 = 0 once the rows r1 are finished); pairs past the matrix are stale and only
// ever reach pairs past the matrix.
template <int P1, int P2>
__device__ __forceinline__ void chol_pair_steps(float2 (&a1)[16], float2 (&a2)[32], float& b1,
                                                float& b2, float& l1, float& l2, int k0, int k1,
                                                float* M, float* dinv, int lane)
{
    static_assert(P1 % 2 == 0 && P2 % 2 == 0 && P2 > 0, "step shape");
#pragma unroll 1
    for (int k = k0; k < k1; k += 2) {
        __syncwarp();  // column k is in row k of M
        const float4* ce = reinterpret_cast<const float4*>(M + k * kLtLd);
        const float4* co = reinterpret_cast<const float4*>(M + (k + 1) * kLtLd);
        const float4 e0 = ce[0];  // e0.y = L[k + 1][k]
        float m1 = 0.f, m2 = 0.f;
        {
            const float n1 = P1 > 0 ? fmaf(-l1, e0.y, a1[0].y) : 0.f;
            const float n2 = fmaf(-l2, e0.y, a2[0].y);
            chol_pivot<(P1 > 0)>(k + 1, n1, n2, b1, b2, m1, m2, M, dinv, lane);
        }
        const float2 nl1 = make_float2(-l1, -l1), nl2 = make_float2(-l2, -l2);
#pragma unroll
        for (int s = 0; s + 1 < P2; ++s) {
            const int q = (s + 1) >> 1;  // column k's entries of rows k + 2s + 2, k + 2s + 3
            const float4 c4 = q == 0 ? e0 : ce[q];
            const float2 c = ((s + 1) & 1) ? make_float2(c4.z, c4.w) : make_float2(c4.x, c4.y);
            a2[s] = __ffma2_rn(nl2, c, a2[s + 1]);
            if (s + 1 < P1) a1[s] = __ffma2_rn(nl1, c, a1[s + 1]);
        }
        __syncwarp();  // column k + 1 is in row k + 1 of M
        const float2 ml1 = make_float2(-m1, -m1), ml2 = make_float2(-m2, -m2);
        float q1 = 0.f, q2 = 0.f;
#pragma unroll
        for (int s = 0; s + 1 < P2; ++s) {
            const int q = (s + 1) >> 1;
            const float4 c4 = co[q];
            const float2 c = ((s + 1) & 1) ? make_float2(c4.z, c4.w) : make_float2(c4.x, c4.y);
            a2[s] = __ffma2_rn(ml2, c, a2[s]);
            if (s + 1 < P1) a1[s] = __ffma2_rn(ml1, c, a1[s]);
            if (s == 0 && k + 2 < 64)
                chol_pivot<(P1 > 0)>(k + 2, a1[0].x, a2[0].x, b1, b2, q1, q2, M, dinv, lane);
        }
        l1 = q1;
        l2 = q2;
    }
}

// Factor / solve / sample for K = 64.  Lane l holds rows r1 = l (a1: columns 0..31)
// and r2 = 32 + l (a2: columns 0..63) of Lambda_i in registers, as pairs of columns
// -- entries above the diagonal are never used -- and its entries b1 = b_i[r1],
// b2 = b_i[r2].  M is the warp's 64 x kLtLd buffer; it receives the strictly lower
// part of L, transposed and shifted (chol_pivot), for the column steps and the back
// solve (its previous contents are ignored).
// bad is set when a pivot was not positive and finite (Lambda_i not positive
// definite in FP32).  The factorisation runs in eight spans of 8 columns so the
// register rows shrink as they finish, then x = L^{-T}(y + z).
__device__ __forceinline__ void factor_solve_sample_rl64(float2 (&a1)[16], float2 (&a2)[32], float b1,
                                                         float b2, float* M, float* dinv,
                                                         float* zb, int lane, int K,
                                                         uint64_t seed, uint32_t row,
                                                         uint32_t sweep, uint32_t c3,
                                                         bool want_means, float& x1, float& x2,
                                                         float& m1, float& m2, bool& bad)
{
    const int r1 = lane, r2 = 32 + lane;
    float l1, l2;
    chol_pivot<true>(0, a1[0].x, a2[0].x, b1, b2, l1, l2, M, dinv, lane);
    chol_pair_steps<16, 32>(a1, a2, b1, b2, l1, l2, 0, 8, M, dinv, lane);
    chol_pair_steps<12, 28>(a1, a2, b1, b2, l1, l2, 8, 16, M, dinv, lane);
    chol_pair_steps<8, 24>(a1, a2, b1, b2, l1, l2, 16, 24, M, dinv, lane);
    chol_pair_steps<4, 20>(a1, a2, b1, b2, l1, l2, 24, 32, M, dinv, lane);
    chol_pair_steps<0, 16>(a1, a2, b1, b2, l1, l2, 32, 40, M, dinv, lane);
    chol_pair_steps<0, 12>(a1, a2, b1, b2, l1, l2, 40, 48, M, dinv, lane);
    chol_pair_steps<0, 8>(a1, a2, b1, b2, l1, l2, 48, 56, M, dinv, lane);
    chol_pair_steps<0, 4>(a1, a2, b1, b2, l1, l2, 56, 64, M, dinv, lane);
    // every pivot's 1 / L[j][j] is in dinv (the last step began with a warp sync): it is
    // positive and finite exactly when the pivot was
    {
        const float d1 = dinv[r1], d2 = dinv[r2];
        if (!(d1 > 0.f && d1 < INFINITY && d2 > 0.f && d2 < INFINITY)) bad = true;  // and NaN
    }
    // ---- noise z (zero beyond K)
    if (lane < 16) {
        const float4 z4 = normals4_f32(seed, (uint32_t)lane, row, sweep, c3);
        const int kk = 4 * lane;
        zb[kk + 0] = kk + 0 < K ? z4.x : 0.f;
        zb[kk + 1] = kk + 1 < K ? z4.y : 0.f;
        zb[kk + 2] = kk + 2 < K ? z4.z : 0.f;
        zb[kk + 3] = kk + 3 < K ? z4.w : 0.f;
    }
    __syncwarp();
    float t1 = b1 + zb[r1];
    float t2 = b2 + zb[r2];
    float n1 = b1, n2 = b2;
    // ---- back substitution x = L^{-T} t: step i broadcasts x_i and every lane
    // updates its rows r < i with L[i][r], which sits in row r of M at position
    // i - (r & ~1); four of them (two aligned pairs) serve four steps.  Steps i >= 32
    // update every row r1 < 32 and, with selects, the rows r2 = 32 + lane; steps i < 32
    // leave the rows r2 (all past i) alone and update the rows r1 with selects.
#pragma unroll 1
    for (int g = 15; g >= 8; --g) {
        const float* q1 = M + r1 * kLtLd + 4 * g - (r1 & ~1);
        const float* q2 = M + r2 * kLtLd + 4 * g - (r2 & ~1);
        const float2 x1 = *reinterpret_cast<const float2*>(q1), y1 = *reinterpret_cast<const float2*>(q1 + 2);
        const float2 x2 = *reinterpret_cast<const float2*>(q2), y2 = *reinterpret_cast<const float2*>(q2 + 2);
        const float4 D = *reinterpret_cast<const float4*>(dinv + 4 * g);
        const float l1v[4] = {x1.x, x1.y, y1.x, y1.y};
        const float l2v[4] = {x2.x, x2.y, y2.x, y2.y};
        const float dv[4] = {D.x, D.y, D.z, D.w};
#pragma unroll
        for (int u = 3; u >= 0; --u) {
            const int i = 4 * g + u;
            const float ui = __shfl_sync(kFullMask, t2, i & 31) * dv[u];
            const float f2 = fmaf(-l2v[u], ui, t2);
            t1 = fmaf(-l1v[u], ui, t1);
            t2 = r2 == i ? ui : (r2 < i ? f2 : t2);
            if (want_means) {
                const float mi = __shfl_sync(kFullMask, n2, i & 31) * dv[u];
                const float g2 = fmaf(-l2v[u], mi, n2);
                n1 = fmaf(-l1v[u], mi, n1);
                n2 = r2 == i ? mi : (r2 < i ? g2 : n2);
            }
        }
    }
#pragma unroll 1
    for (int g = 7; g >= 0; --g) {
        const float* q1 = M + r1 * kLtLd + 4 * g - (r1 & ~1);
        const float2 x1 = *reinterpret_cast<const float2*>(q1), y1 = *reinterpret_cast<const float2*>(q1 + 2);
        const float4 D = *reinterpret_cast<const float4*>(dinv + 4 * g);
        const float l1v[4] = {x1.x, x1.y, y1.x, y1.y};
        const float dv[4] = {D.x, D.y, D.z, D.w};
#pragma unroll
        for (int u = 3; u >= 0; --u) {
            const int i = 4 * g + u;
            const float ui = __shfl_sync(kFullMask, t1, i) * dv[u];
            const float f1 = fmaf(-l1v[u], ui, t1);
            t1 = r1 == i ? ui : (r1 < i ? f1 : t1);
            if (want_means) {
                const float mi = __shfl_sync(kFullMask, n1, i) * dv[u];
                const float g1 = fmaf(-l1v[u], mi, n1);
                n1 = r1 == i ? mi : (r1 < i ? g1 : n1);
            }
        }
    }
    x1 = t1;
    x2 = t2;
    m1 = n1;
    m2 = n2;
}

// Store for the two-panel ownership (rows l and 32 + l).
__device__ __forceinline__ void store_row_panels(const RowArgs& a, int row, int lane, float x1,
                                                 float x2, float m1, float m2)
{
    const int r1 = lane, r2 = 32 + lane;
    const bool v2 = true;
    const int64_t off = (int64_t)row * a.ldx;
    a.X[off + r1] = x1;
    if (v2) a.X[off + r2] = x2;
    if (a.Xh) {
        __half h, l;
        split16(x1, a.bf16, h, l);
        a.Xh[off + r1] = h;
        a.Xl[off + r1] = l;
        if (v2) {
            split16(x2, a.bf16, h, l);
            a.Xh[off + r2] = h;
            a.Xl[off + r2] = l;
        }
    }
    if (a.means) {
        a.means[off + r1] = m1;
        if (v2) a.means[off + r2] = m2;
    }
}


// Write the lane's entries of one row: FP32 factors, their FP16 split (when the
// other side's tensor-core kernel gathers them) and the conditional mean.
template <int KT>
__device__ __forceinline__ void store_row(const RowArgs& a, int row, int lane, float x1, float x2,
                                          float m1, float m2)
{
    using R = RowRegs<KT>;
    const int i1 = lane, i2 = 63 - lane;
    const bool v1 = i1 < KT;
    const bool v2 = R::TWO && i2 < KT;
    const int64_t off = (int64_t)row * a.ldx;
    if (v1) a.X[off + i1] = x1;
    if (v2) a.X[off + i2] = x2;
    if (a.Xh) {
        __half h, l;
        if (v1) {
            split16(x1, a.bf16, h, l);
            a.Xh[off + i1] = h;
            a.Xl[off + i1] = l;
        }
        if (v2) {
            split16(x2, a.bf16, h, l);
            a.Xh[off + i2] = h;
            a.Xl[off + i2] = l;
        }
    }
    if (a.means) {
        if (v1) a.means[off + i1] = m1;
        if (v2) a.means[off + i2] = m2;
    }
}

}  // namespace bpmf
