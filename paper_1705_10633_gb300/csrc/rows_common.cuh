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

// Column steps k0 .. k1 - 1 of a right-looking Cholesky with the forward solve
// fused, for K = 64 with lane l owning rows r1 = l and r2 = 32 + l.  The rows are
// kept in registers "shifted": a1[t] = A[r1][k + t] and a2[t] = A[r2][k + t] at step
// k, so the update  A[r][k+1+t] -= L[r][k] L[k+1+t][k]  also slides each row by
// one (a[t] = a[t+1] - l c[t]) and every register index stays static in a rolled
// loop.  N1 / N2: entries of a1 / a2 still inside the matrix (N1 = 0 once the
// rows r1 are finished).  The strictly lower part of L is written transposed into
// M (row k of M receives column k of L: a conflict-free row store), the inverse
// diagonal into dinv; the pivot column is broadcast through cbuf (two 64-float
// buffers, by step parity).
template <int N1, int N2>
__device__ __forceinline__ void chol_shifted_steps(float (&a1)[32], float (&a2)[64], float& b1,
                                                   float& b2, int k0, int k1, float* M,
                                                   float* cbuf, float* dinv, int lane, bool& bad)
{
    static_assert(N1 % 4 == 0 && N2 % 4 == 0 && N2 > 0, "step shape");
    const int r1 = lane, r2 = 32 + lane;
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
        const int owner = k & 31;
        float piv = __shfl_sync(kFullMask, N1 > 0 ? a1[0] : a2[0], owner);
        const float bk = __shfl_sync(kFullMask, N1 > 0 ? b1 : b2, owner);
        if (!(piv > 0.f && piv < INFINITY)) {  // also catches NaN
            bad = true;
            piv = 1.f;
        }
        const float rinv = rsqrtf(piv);
        const float yk = bk * rinv;
        if (lane == 0) dinv[k] = rinv;
        float* cb = cbuf + (k & 1) * 64;
        float l1 = 0.f, l2 = 0.f;
        if (N1 > 0) {
            if (r1 == k) {
                b1 = yk;
            } else if (r1 > k) {
                l1 = a1[0] * rinv;
                M[sw64(k, r1)] = l1;
                b1 = fmaf(-l1, yk, b1);
                cb[r1 - k - 1] = l1;
            }
        }
        if (r2 == k) {
            b2 = yk;
        } else if (r2 > k) {
            l2 = a2[0] * rinv;
            M[sw64(k, r2)] = l2;
            b2 = fmaf(-l2, yk, b2);
            cb[r2 - k - 1] = l2;
        }
        __syncwarp();
        // cb[t] = L[k + 1 + t][k]; entries past the matrix are stale and only ever
        // reach register entries past the matrix
#pragma unroll
        for (int t4 = 0; t4 < N2; t4 += 4) {
            const float4 c = *reinterpret_cast<const float4*>(cb + t4);
            const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = t4 + u;
                if (t + 1 < N2) a2[t] = fmaf(-l2, cv[u], a2[t + 1]);
                if (t + 1 < N1) a1[t] = fmaf(-l1, cv[u], a1[t + 1]);
            }
        }
    }
}

// Lower-triangle chunks (4c <= i) of a sw64 matrix set from a chunk-transposed copy
// in global memory (float4 (i, 4c..4c+3) at c * 64 + i) by `nthreads` threads:
// consecutive threads take consecutive rows, so the loads coalesce and the stores
// are conflict-free.
__device__ __forceinline__ void fill_lower_sw64(float* M, const float4* src_ct, int t, int nthreads)
{
#pragma unroll 4
    for (int e = t; e < 1024; e += nthreads) {
        const int i = e & 63, c = e >> 6;
        if (4 * c <= i) *chunk_ptr(M, i, c) = __ldg(src_ct + c * 64 + i);
    }
}

// Factor / solve / sample for K = 64: Lambda_i in shared memory (sw64 layout, lower
// triangle valid, the rest scratch; overwritten with the strictly lower part of L,
// transposed), b_i in bv.  Lane l owns
// rows r1 = l and r2 = 32 + l; the factorization runs in four spans of 16 columns
// so the register rows shrink as they finish, then x = L^{-T}(y + z).
__device__ __forceinline__ void factor_solve_sample_rl64(float* M, const float* bv, float* cbuf,
                                                         float* dinv, float* zb, int lane, int K,
                                                         uint64_t seed, uint32_t row,
                                                         uint32_t sweep, uint32_t c3,
                                                         bool want_means, float& x1, float& x2,
                                                         float& m1, float& m2, bool& bad)
{
    const int r1 = lane, r2 = 32 + lane;
    float a1[32], a2[64];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float4 u = ld_chunk(M, r1, c);
        a1[4 * c + 0] = u.x; a1[4 * c + 1] = u.y; a1[4 * c + 2] = u.z; a1[4 * c + 3] = u.w;
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const float4 v = ld_chunk(M, r2, c);
        a2[4 * c + 0] = v.x; a2[4 * c + 1] = v.y; a2[4 * c + 2] = v.z; a2[4 * c + 3] = v.w;
    }
    float b1 = bv[r1];
    float b2 = bv[r2];
    __syncwarp();  // every lane has its rows before L overwrites them
    chol_shifted_steps<32, 64>(a1, a2, b1, b2, 0, 16, M, cbuf, dinv, lane, bad);
    chol_shifted_steps<16, 48>(a1, a2, b1, b2, 16, 32, M, cbuf, dinv, lane, bad);
    chol_shifted_steps<0, 32>(a1, a2, b1, b2, 32, 48, M, cbuf, dinv, lane, bad);
    chol_shifted_steps<0, 16>(a1, a2, b1, b2, 48, 64, M, cbuf, dinv, lane, bad);
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
    // updates its rows r < i with L[i][r], which sits in row r of M (L^T); one
    // float4 of that row serves four steps
#pragma unroll 1
    for (int g = 15; g >= 0; --g) {
        const float4 A1 = ld_chunk(M, r1, g), A2 = ld_chunk(M, r2, g);
        const float4 D = *reinterpret_cast<const float4*>(dinv + 4 * g);
        const float l1v[4] = {A1.x, A1.y, A1.z, A1.w};
        const float l2v[4] = {A2.x, A2.y, A2.z, A2.w};
        const float dv[4] = {D.x, D.y, D.z, D.w};
#pragma unroll
        for (int u = 3; u >= 0; --u) {
            const int i = 4 * g + u;
            const int owner = i & 31;
            const float ui = __shfl_sync(kFullMask, i < 32 ? t1 : t2, owner) * dv[u];
            float mi = 0.f;
            if (want_means) mi = __shfl_sync(kFullMask, i < 32 ? n1 : n2, owner) * dv[u];
            if (r1 == i) {
                t1 = ui;
                n1 = mi;
            } else if (r1 < i) {
                t1 = fmaf(-l1v[u], ui, t1);
                n1 = fmaf(-l1v[u], mi, n1);
            }
            if (r2 == i) {
                t2 = ui;
                n2 = mi;
            } else if (r2 < i) {
                t2 = fmaf(-l2v[u], ui, t2);
                n2 = fmaf(-l2v[u], mi, n2);
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
