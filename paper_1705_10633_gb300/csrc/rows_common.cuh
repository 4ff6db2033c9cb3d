// rows_common.cuh -- the per-row factor / solve / sample step shared by the
// row-update kernels (Sec. 3.1: Cholesky instead of an inverse; Alg. 1: the new
// vector is the conditional mean plus randomly sampled noise).
//
// One warp holds one K x K precision (K padded to KT, identity in the padding):
// lane l owns row i1 = l (columns 0..31) and row i2 = 63 - l (columns 0..KT-1),
// 65 lower-triangle entries per lane at KT = 64.  On return the lane holds its
// entries of x = L^{-T}(L^{-1} b + z) (and of the mean L^{-T} L^{-1} b).
#pragma once
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

template <int KT>
struct RowRegs {
    static constexpr int NR1 = KT < 32 ? KT : 32;  // columns of row i1 kept in registers
    static constexpr bool TWO = KT > 32;           // a second row i2 = 63 - lane exists
    static constexpr int NA2 = TWO ? KT : 1;
    static constexpr int LD = KT + 1;              // row stride of the square buffer
};

// colbuf: 2*KT floats, dinv: KT, zb: KT, sq: KT x LD (L is written here for the back solve).
template <int KT>
__device__ __forceinline__ void factor_solve_sample(float (&a1)[RowRegs<KT>::NR1],
                                                    float (&a2)[RowRegs<KT>::NA2], float b1,
                                                    float b2, float* colbuf, float* dinv,
                                                    float* zb, float* sq, int lane, int K,
                                                    uint64_t seed, uint32_t row, uint32_t sweep,
                                                    uint32_t c3, bool want_means, float& x1,
                                                    float& x2, float& m1, float& m2, bool& bad)
{
    using R = RowRegs<KT>;
    const int i1 = lane, i2 = 63 - lane;
    const bool v1 = i1 < KT;
    const bool v2 = R::TWO && i2 < KT;

    // ---- right-looking Cholesky; column k is published through shared memory
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        float* cb = colbuf + (k & 1) * KT;
        const int owner = k < 32 ? k : 63 - k;
        float pv;
        if (k < R::NR1) pv = a1[k < R::NR1 ? k : 0];
        else pv = a2[R::TWO ? k : 0];
        float piv = __shfl_sync(kFullMask, pv, owner);
        if (!(piv > 0.f && piv < INFINITY)) {  // also catches NaN
            bad = true;
            piv = 1.f;
        }
        const float rinv = rsqrtf(piv);
        if (lane == 0) dinv[k] = rinv;
        float l1 = 0.f, l2 = 0.f;
        if (k < R::NR1) {
            const int kk = k < R::NR1 ? k : 0;
            if (i1 > k) a1[kk] *= rinv;
            else if (i1 == k) a1[kk] = piv * rinv;
            l1 = a1[kk];
            if (i1 > k && v1) cb[i1] = l1;
        }
        if (R::TWO) {
            const int kk = R::TWO ? k : 0;
            if (i2 > k) a2[kk] *= rinv;
            else if (i2 == k) a2[kk] = piv * rinv;
            l2 = a2[kk];
            if (i2 > k && v2) cb[i2] = l2;
        }
        __syncwarp();
#pragma unroll
        for (int j4 = ((k + 1) / 4) * 4; j4 < KT; j4 += 4) {
            const float4 cv = *reinterpret_cast<const float4*>(cb + j4);
            const float cj[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j4 + u;
                if (j > k) {
                    if (j < R::NR1) a1[j < R::NR1 ? j : 0] = fmaf(-l1, cj[u], a1[j < R::NR1 ? j : 0]);
                    if (R::TWO) a2[R::TWO ? j : 0] = fmaf(-l2, cj[u], a2[R::TWO ? j : 0]);
                }
            }
        }
    }

    // ---- forward substitution y = L^{-1} b (in place in b1, b2)
#pragma unroll
    for (int k = 0; k < KT; ++k) {
        const int owner = k < 32 ? k : 63 - k;
        const float bk = __shfl_sync(kFullMask, k < 32 ? b1 : b2, owner);
        const float yk = bk * dinv[k];
        if (k < R::NR1) {
            if (i1 == k) b1 = yk;
            else if (i1 > k) b1 = fmaf(-a1[k < R::NR1 ? k : 0], yk, b1);
        }
        if (R::TWO) {
            if (i2 == k) b2 = yk;
            else if (i2 > k) b2 = fmaf(-a2[R::TWO ? k : 0], yk, b2);
        }
    }
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
    // indexing here, so the loop is only partly unrolled (keeps register pressure low)
#pragma unroll 4
    for (int i = KT - 1; i >= 0; --i) {
        const int owner = i < 32 ? i : 63 - i;
        const float di = dinv[i];
        const float ui = __shfl_sync(kFullMask, i < 32 ? t1 : t2, owner) * di;
        float mi = 0.f;
        if (want_means) mi = __shfl_sync(kFullMask, i < 32 ? n1 : n2, owner) * di;
        const float* Lrow = sq + i * R::LD;
        if (i1 == i) {
            t1 = ui;
            n1 = mi;
        } else if (i1 < i && v1) {
            const float l = Lrow[i1];
            t1 = fmaf(-l, ui, t1);
            n1 = fmaf(-l, mi, n1);
        }
        if (R::TWO) {
            if (i2 == i) {
                t2 = ui;
                n2 = mi;
            } else if (i2 < i && v2) {
                const float l = Lrow[i2];
                t2 = fmaf(-l, ui, t2);
                n2 = fmaf(-l, mi, n2);
            }
        }
    }
    x1 = t1;
    x2 = t2;
    m1 = n1;
    m2 = n2;
}

// Same step for a matrix that sits in shared memory (KT = 48 or 64), in two
// column panels so that at most two 32-entry row pieces are live in registers
// (no spills under a 128-register budget).  sq holds Lambda_i row-major with
// stride KT + 1 (lower triangle valid) and b_i in column KT; it is overwritten
// with L.  Lane l owns rows r1 = l and r2 = 32 + l (the latter if l < KT - 32).
//   panel 1: right-looking Cholesky of columns 0..31 on rows r1 (L11) and r2 (L21)
//   update : A22 -= L21 L21^T, with L21 transposed through the unused upper block
//   panel 2: Cholesky of the updated A22 (one row per lane)
template <int KT>
__device__ __forceinline__ void factor_solve_sample_smem(float* sq, float* colbuf, float* dinv,
                                                         float* zb, int lane, int K, uint64_t seed,
                                                         uint32_t row, uint32_t sweep, uint32_t c3,
                                                         bool want_means, float& x1, float& x2,
                                                         float& m1, float& m2, bool& bad)
{
    static_assert(KT == 48 || KT == 64, "two-panel factor needs 32 < KT <= 64");
    constexpr int Q = KT - 32;
    constexpr int LD = KT + 1;
    const int r1 = lane, r2 = 32 + lane;
    const bool v2 = lane < Q;
    float a1[32], a2[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        a1[j] = sq[r1 * LD + j];
        a2[j] = v2 ? sq[r2 * LD + j] : 0.f;
    }
    float b1 = sq[r1 * LD + KT];
    float b2 = v2 ? sq[r2 * LD + KT] : 0.f;
    __syncwarp();

    // ---- panel 1: columns 0..31
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        float* cb = colbuf + (k & 1) * 32;
        float piv = __shfl_sync(kFullMask, a1[k], k);
        if (!(piv > 0.f && piv < INFINITY)) {
            bad = true;
            piv = 1.f;
        }
        const float rinv = rsqrtf(piv);
        if (lane == 0) dinv[k] = rinv;
        if (r1 > k) a1[k] *= rinv;
        else if (r1 == k) a1[k] = piv * rinv;
        a2[k] *= rinv;
        if (r1 > k) cb[r1] = a1[k];
        __syncwarp();
        const float l1 = a1[k], l2 = a2[k];
#pragma unroll
        for (int j4 = ((k + 1) / 4) * 4; j4 < 32; j4 += 4) {
            const float4 cv = *reinterpret_cast<const float4*>(cb + j4);
            const float cj[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j4 + u;
                if (j > k) {
                    a1[j] = fmaf(-l1, cj[u], a1[j]);
                    a2[j] = fmaf(-l2, cj[u], a2[j]);
                }
            }
        }
    }
    // ---- forward substitution, columns 0..31 (L11 and L21)
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const float yk = __shfl_sync(kFullMask, b1, k) * dinv[k];
        if (r1 == k) b1 = yk;
        else if (r1 > k) b1 = fmaf(-a1[k], yk, b1);
        b2 = fmaf(-a2[k], yk, b2);
    }
    // L11 and L21 into sq; L21 also transposed into the unused upper block
    // (row k, columns 32..KT-1) for the trailing update
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (j <= r1) sq[r1 * LD + j] = a1[j];
        if (v2) {
            sq[r2 * LD + j] = a2[j];
            sq[j * LD + 32 + lane] = a2[j];
        }
    }
    __syncwarp();
    // ---- trailing update of row r2: A22[r2][32 + j] -= L21[r2] . L21[32 + j]
    float a3[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) a3[j] = v2 ? sq[r2 * LD + 32 + j] : 0.f;
#pragma unroll 2
    for (int k = 0; k < 32; ++k) {
        const float lk = v2 ? sq[r2 * LD + k] : 0.f;  // L21[r2][k], already stored
        const float* Trow = sq + k * LD + 32;
#pragma unroll
        for (int j = 0; j < Q; ++j) a3[j] = fmaf(-lk, Trow[j], a3[j]);
    }
    // ---- panel 2: Cholesky of the updated A22, row r2 on lane l
#pragma unroll 32
    for (int k = 0; k < Q; ++k) {
        float* cb = colbuf + (k & 1) * 32;
        float piv = __shfl_sync(kFullMask, a3[k], k);
        if (!(piv > 0.f && piv < INFINITY)) {
            bad = true;
            piv = 1.f;
        }
        const float rinv = rsqrtf(piv);
        if (lane == 0) dinv[32 + k] = rinv;
        if (lane > k) a3[k] *= rinv;
        else if (lane == k) a3[k] = piv * rinv;
        if (lane > k && v2) cb[lane] = a3[k];
        __syncwarp();
        const float l3 = a3[k];
#pragma unroll 8
        for (int j4 = ((k + 1) / 4) * 4; j4 < Q; j4 += 4) {
            const float4 cv = *reinterpret_cast<const float4*>(cb + j4);
            const float cj[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j4 + u;
                if (j > k) a3[j] = fmaf(-l3, cj[u], a3[j]);
            }
        }
    }
    // ---- forward substitution, columns 32..KT-1 (L22)
#pragma unroll 32
    for (int k = 0; k < Q; ++k) {
        const float yk = __shfl_sync(kFullMask, b2, k) * dinv[32 + k];
        if (lane == k) b2 = yk;
        else if (lane > k) b2 = fmaf(-a3[k], yk, b2);
    }
#pragma unroll 32
    for (int j = 0; j < Q; ++j)
        if (v2 && j <= lane) sq[r2 * LD + 32 + j] = a3[j];
    // ---- noise z (zero beyond K)
    if (lane < KT / 4) {
        const float4 z4 = normals4_f32(seed, (uint32_t)lane, row, sweep, c3);
        const int kk = 4 * lane;
        zb[kk + 0] = kk + 0 < K ? z4.x : 0.f;
        zb[kk + 1] = kk + 1 < K ? z4.y : 0.f;
        zb[kk + 2] = kk + 2 < K ? z4.z : 0.f;
        zb[kk + 3] = kk + 3 < K ? z4.w : 0.f;
    }
    __syncwarp();
    float t1 = b1 + zb[r1];
    float t2 = b2 + (v2 ? zb[r2] : 0.f);
    float n1 = b1, n2 = b2;
    // ---- back substitution x = L^{-T} t (rows r1 = l, r2 = 32 + l)
#pragma unroll 4
    for (int i = KT - 1; i >= 0; --i) {
        const int owner = i < 32 ? i : i - 32;
        const float di = dinv[i];
        const float ui = __shfl_sync(kFullMask, i < 32 ? t1 : t2, owner) * di;
        float mi = 0.f;
        if (want_means) mi = __shfl_sync(kFullMask, i < 32 ? n1 : n2, owner) * di;
        const float* Lrow = sq + i * LD;
        if (r1 == i) {
            t1 = ui;
            n1 = mi;
        } else if (r1 < i) {
            const float l = Lrow[r1];
            t1 = fmaf(-l, ui, t1);
            n1 = fmaf(-l, mi, n1);
        }
        if (v2) {
            if (r2 == i) {
                t2 = ui;
                n2 = mi;
            } else if (r2 < i) {
                const float l = Lrow[r2];
                t2 = fmaf(-l, ui, t2);
                n2 = fmaf(-l, mi, n2);
            }
        }
    }
    x1 = t1;
    x2 = t2;
    m1 = n1;
    m2 = n2;
}

// Store for the two-panel ownership (rows l and 32 + l).
template <int KT>
__device__ __forceinline__ void store_row_panels(const RowArgs& a, int row, int lane, float x1,
                                                 float x2, float m1, float m2)
{
    const int r1 = lane, r2 = 32 + lane;
    const bool v2 = lane < KT - 32;
    const int64_t off = (int64_t)row * a.ldx;
    a.X[off + r1] = x1;
    if (v2) a.X[off + r2] = x2;
    if (a.Xh) {
        __half h, l;
        split_f16(x1, h, l);
        a.Xh[off + r1] = h;
        a.Xl[off + r1] = l;
        if (v2) {
            split_f16(x2, h, l);
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
            split_f16(x1, h, l);
            a.Xh[off + i1] = h;
            a.Xl[off + i1] = l;
        }
        if (v2) {
            split_f16(x2, h, l);
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
