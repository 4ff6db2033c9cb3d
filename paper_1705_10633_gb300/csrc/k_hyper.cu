// k_hyper.cu -- the hyper-parameter step of Alg. 1 ("sample hyper-parameters
// movies/users based on V/U", Sec. 2): sufficient statistics of a factor matrix
// and the Normal-Wishart draw of (mu, Lambda).
//
//   reduce : every block takes the shift s (FP64 mean of the first rows, fixed
//            order), then streams a contiguous slab of rows once, the next 64-row
//            chunk in flight while the current one is summed, accumulating (x - s)
//            and the lower triangle of (x - s)(x - s)^T in FP32 registers over each
//            chunk and folding it into FP64 accumulators, so the sums stay small.
//   combine: fixed-order FP64 sum of the block partials (deterministic).
//   nw     : one CTA in FP64 -- posterior parameters, chol(W*) through the
//            reversed factorisation of its inverse, Bartlett Wishart draw with
//            Marsaglia-Tsang gammas, chol(Lambda), mean draw.
#include <string.h>

#include <algorithm>

#include "bpmf_internal.cuh"
#include "philox.cuh"

namespace bpmf {

// ---------------------------------------------------------------------------
// reduction
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedChunk = 64;
constexpr int64_t kShiftRows = 256;  // rows whose FP64 mean is the statistics' shift
constexpr int kGammaMaxAttempts = 64;

// One thread's share of the Normal-Wishart step's random draws, which depend only on
// (seed, sweep, side) and the posterior degrees of freedom (nu0 + rows, fixed per side):
// draws[q] for q < K(K-1)/2 the Bartlett factor's off-diagonal normals (stream 0), then K
// normals of the mean draw (stream 1), then the Bartlett diagonal sqrt(chi^2(nu* - k)) =
// sqrt(2 Gamma((nu* - k) / 2)) by Marsaglia-Tsang.  Thread q takes one Philox call (four
// normals) or one gamma; they run as extra blocks of the reduction launch, spread over
// SMs (FP64 is slow on this GPU, and the one-CTA draw kernel only reads them).
__device__ void nw_draws_thread(const NWArgs& a, int q)
{
    const int K = a.K, noff = K * (K - 1) / 2;
    const int ncall0 = (noff + 3) / 4, ncall1 = (K + 3) / 4;
    const uint32_t sweep = (uint32_t)a.ctl->sweep + a.sweep_offset;
    if (q < ncall0 + ncall1) {
        const bool mean = q >= ncall0;
        const uint32_t c = mean ? (uint32_t)(q - ncall0) : (uint32_t)q;
        const uint4 w = philox_call(a.seed, c, mean ? 1u : 0u, sweep, a.c3_normal);
        const double2 z0 = box_muller_f64(w.x, w.y), z1 = box_muller_f64(w.z, w.w);
        const double z[4] = {z0.x, z0.y, z1.x, z1.y};
        const int base = mean ? noff : 0, lim = mean ? K : noff;
        for (int u = 0; u < 4; ++u)
            if ((int)(4 * c) + u < lim) a.draws[base + 4 * c + u] = z[u];
    } else if (q < ncall0 + ncall1 + K) {
        const int k = q - ncall0 - ncall1;
        const double nu_s = a.nu0 + (double)a.n;
        const double shape = 0.5 * (nu_s - (double)k);
        const double d = shape - 1.0 / 3.0;
        const double c = 1.0 / sqrt(9.0 * d);
        double g = -1.0;
        for (int att = 0; att < kGammaMaxAttempts; ++att) {
            const uint4 wd = philox_call(a.seed, (uint32_t)att, (uint32_t)k, sweep, a.c3_gamma);
            const double x = box_muller_f64(wd.x, wd.y).x;
            const double sx = 1.0 + c * x;
            if (sx <= 0.0) continue;
            const double v = sx * sx * sx;
            const double u = (double)((wd.z >> 8) + 1u) * 0x1p-24;
            if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) {
                g = d * v;
                break;
            }
        }
        if (g < 0.0) {
            atomicOr(&a.ctl->status, kStatusGamma);
            g = shape;
        }
        a.draws[noff + K + k] = sqrt(2.0 * g);
    }
}

int nw_draws_threads(int K) { return (K * (K - 1) / 2 + 3) / 4 + (K + 3) / 4 + K; }

int hyper_reduce_blocks(int64_t rows, int num_sms)
{
    int64_t want = (rows + 1023) / 1024;  // at least ~1k rows per block
    // a small side: up to the blocks the draw kernel combines itself, of at least 128
    // rows each, so that no block walks through more than a few chunks in sequence
    if (want < kFuseCombineBlocks) want = std::min<int64_t>(kFuseCombineBlocks, (rows + 127) / 128);
    int64_t cap = (int64_t)num_sms * 2;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

// Block `bid` of one side's reduction launch (nred reduction blocks, then draw blocks).
template <int KT>
__device__ __forceinline__ void hyper_reduce_body(const float* __restrict__ X, int64_t rows,
                                                  int shiftK, double* __restrict__ shift64,
                                                  double* __restrict__ partials, int nred,
                                                  const NWArgs& draws, int bid)
{
    // blocks past the reduction's draw the Normal-Wishart step's random numbers
    if (bid >= nred) {
        nw_draws_thread(draws, (bid - nred) * kRedThreads + (int)threadIdx.x);
        return;
    }
    // The scatter is a 16 x 16 grid of TT x TT tiles; threads 0..135 own the tiles on
    // and below the diagonal (t = ty (ty + 1) / 2 + tx, tx <= ty) and also write their
    // mirror images; the other threads only stage rows.
    constexpr int TT = KT / 16;
    constexpr int kLowerTiles = 16 * 17 / 2;
    constexpr int F4 = KT / 4;
    constexpr int NPF = kRedChunk * F4 / kRedThreads;  // float4 a thread stages per chunk
    static_assert(NPF * kRedThreads == kRedChunk * F4, "chunk staging");
    __shared__ __align__(16) float xs[kRedChunk][KT];
    __shared__ float sh[KT];
    const int t = threadIdx.x;
    const bool tile_on = t < kLowerTiles;
    int ty = 0;
    while (tile_on && (ty + 1) * (ty + 2) / 2 <= t) ++ty;
    const int tx = tile_on ? t - ty * (ty + 1) / 2 : 0;
    if (shiftK > 0) {
        // the shift: FP64 mean of the first kShiftRows rows, zero beyond shiftK columns,
        // taken by every block in the same fixed order (column c = t mod 64 of rows
        // t / 64 (mod 4), four partial sums); block 0 publishes it for the draw.
        // Subtracting a value near the mean keeps the FP32 chunk sums of (x - s)(x - s)^T
        // from cancelling against d d^T; taken from the data (not the last drawn mu, which
        // on a side with few rows can sit far from the sample mean) and in a fixed order,
        // it keeps resumed chains bit-identical.
        __shared__ double part[4][64];
        const int c = t & 63, g = t >> 6;
        const int64_t n = rows < kShiftRows ? rows : kShiftRows;
        double s = 0.0;
        if (c < shiftK)
            for (int64_t r = g; r < n; r += 4) s += (double)X[r * KT + c];
        part[g][c] = s;
        __syncthreads();
        if (t < KT) {
            const double tot = (part[0][t] + part[1][t]) + (part[2][t] + part[3][t]);
            const double v = (t < shiftK && n > 0) ? tot / (double)n : 0.0;
            sh[t] = (float)v;
            if (bid == 0) shift64[t] = v;
        }
    } else if (t < KT) {
        sh[t] = (float)shift64[t];
    }
    const int64_t r0 = rows * bid / nred;
    const int64_t r1 = rows * (bid + 1) / nred;
    // a chunk's rows in registers (rows past the slab's end zero)
    float4 pf[NPF];
    auto load_chunk = [&](int64_t base) {
        const int cnt = (int)min((int64_t)kRedChunk, r1 - base);
#pragma unroll
        for (int i = 0; i < NPF; ++i) {
            const int e = t + i * kRedThreads, r = e / F4, f = e % F4;
            pf[i] = r < cnt ? __ldg(reinterpret_cast<const float4*>(X + (base + r) * KT) + f)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    if (r0 < r1) load_chunk(r0);
    double acc64[TT][TT];
    double s64 = 0.0;
#pragma unroll
    for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) acc64[i][j] = 0.0;
    __syncthreads();
    for (int64_t base = r0; base < r1; base += kRedChunk) {
        const int cnt = (int)min((int64_t)kRedChunk, r1 - base);
        // stage (x - s) for the chunk; rows past the end stay zero
#pragma unroll
        for (int i = 0; i < NPF; ++i) {
            const int e = t + i * kRedThreads, r = e / F4, f = e % F4;
            float4 v = pf[i];
            if (r < cnt) {
                v.x -= sh[4 * f + 0];
                v.y -= sh[4 * f + 1];
                v.z -= sh[4 * f + 2];
                v.w -= sh[4 * f + 3];
            }
            *reinterpret_cast<float4*>(&xs[r][4 * f]) = v;
        }
        __syncthreads();
        // the next chunk's loads are in flight while this one is summed
        if (base + kRedChunk < r1) load_chunk(base + kRedChunk);
        float s32 = 0.f;
        if (t < KT)
#pragma unroll 8
            for (int r = 0; r < kRedChunk; ++r) s32 += xs[r][t];
        s64 += (double)s32;
        if (tile_on) {
            float acc[TT][TT];
#pragma unroll
            for (int i = 0; i < TT; ++i)
#pragma unroll
                for (int j = 0; j < TT; ++j) acc[i][j] = 0.f;
#pragma unroll 4
            for (int r = 0; r < kRedChunk; ++r) {
                float a[TT], b[TT];
#pragma unroll
                for (int i = 0; i < TT; ++i) {
                    a[i] = xs[r][ty * TT + i];
                    b[i] = xs[r][tx * TT + i];
                }
#pragma unroll
                for (int i = 0; i < TT; ++i)
#pragma unroll
                    for (int j = 0; j < TT; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < TT; ++i)
#pragma unroll
                for (int j = 0; j < TT; ++j) acc64[i][j] += (double)acc[i][j];
        }
        __syncthreads();
    }
    double* out = partials + (size_t)bid * hyper_partial_doubles(KT);
    if (t < KT) out[t] = s64;
    if (tile_on) {
        // entry (p, q) and its mirror (q, p): fmaf(x_p, x_q, .) equals fmaf(x_q, x_p, .),
        // so the mirror is the value the upper tile's own sum would give
#pragma unroll
        for (int i = 0; i < TT; ++i)
#pragma unroll
            for (int j = 0; j < TT; ++j) {
                out[KT + (ty * TT + i) * KT + tx * TT + j] = acc64[i][j];
                out[KT + (tx * TT + j) * KT + ty * TT + i] = acc64[i][j];
            }
    }
}

template <int KT>
__global__ void __launch_bounds__(kRedThreads) hyper_reduce_kernel(const float* __restrict__ X,
                                                                   int64_t rows, int shiftK,
                                                                   double* __restrict__ shift64,
                                                                   double* __restrict__ partials,
                                                                   int nred, NWArgs draws)
{
    hyper_reduce_body<KT>(X, rows, shiftK, shift64, partials, nred, draws, (int)blockIdx.x);
}

template <int KT>
__global__ void __launch_bounds__(kRedThreads)
    hyper_reduce_batch_kernel(const BatchEntry<ReduceArgs>* __restrict__ t, int n)
{
    const int j = batch_find(t, n, (int)blockIdx.x);
    const ReduceArgs r = t[j].args;
    hyper_reduce_body<KT>(r.X, r.rows, r.shiftK, r.shift64, r.partials, r.nred, r.draws,
                          (int)blockIdx.x - t[j].first);
}

cudaError_t launch_hyper_reduce_batch(const BatchEntry<ReduceArgs>* t, int n, int64_t blocks,
                                      int kp, cudaStream_t s)
{
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    const unsigned g = (unsigned)blocks;
    switch (kp) {
    case 16: hyper_reduce_batch_kernel<16><<<g, kRedThreads, 0, s>>>(t, n); break;
    case 32: hyper_reduce_batch_kernel<32><<<g, kRedThreads, 0, s>>>(t, n); break;
    case 48: hyper_reduce_batch_kernel<48><<<g, kRedThreads, 0, s>>>(t, n); break;
    case 64: hyper_reduce_batch_kernel<64><<<g, kRedThreads, 0, s>>>(t, n); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int hyper_draw_blocks(int K) { return (nw_draws_threads(K) + kRedThreads - 1) / kRedThreads; }

static cudaError_t reduce_launch(const float* X, int64_t rows, int kp, int shiftK, double* shift64,
                                 double* partials, int nblocks, int ndraw, const NWArgs& draws,
                                 cudaStream_t s)
{
    const int grid = nblocks + ndraw;
    switch (kp) {
    case 16: hyper_reduce_kernel<16><<<grid, kRedThreads, 0, s>>>(X, rows, shiftK, shift64, partials, nblocks, draws); break;
    case 32: hyper_reduce_kernel<32><<<grid, kRedThreads, 0, s>>>(X, rows, shiftK, shift64, partials, nblocks, draws); break;
    case 48: hyper_reduce_kernel<48><<<grid, kRedThreads, 0, s>>>(X, rows, shiftK, shift64, partials, nblocks, draws); break;
    case 64: hyper_reduce_kernel<64><<<grid, kRedThreads, 0, s>>>(X, rows, shiftK, shift64, partials, nblocks, draws); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_hyper_reduce(const float* X, int64_t rows, int kp, const double* shift64,
                                double* partials, int nblocks, cudaStream_t s)
{
    NWArgs none;
    memset(&none, 0, sizeof(none));
    return reduce_launch(X, rows, kp, 0, const_cast<double*>(shift64), partials, nblocks, 0, none, s);
}

cudaError_t launch_hyper_stats_draws(const float* X, int64_t rows, int K, int kp, double* shift64,
                                     double* partials, int nblocks, const NWArgs& a, cudaStream_t s)
{
    return reduce_launch(X, rows, kp, K, shift64, partials, nblocks, hyper_draw_blocks(K), a, s);
}

__device__ __forceinline__ void hyper_combine_body(const double* __restrict__ partials,
                                                   int nblocks, int E, double* __restrict__ sums,
                                                   int e)
{
    if (e >= E) return;
    // four interleaved accumulators (more loads in flight), added in a fixed order
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = 0;
    for (; b + 3 < nblocks; b += 4) {
        a0 += partials[(size_t)b * E + e];
        a1 += partials[(size_t)(b + 1) * E + e];
        a2 += partials[(size_t)(b + 2) * E + e];
        a3 += partials[(size_t)(b + 3) * E + e];
    }
    for (; b < nblocks; ++b) a0 += partials[(size_t)b * E + e];
    sums[e] = (a0 + a1) + (a2 + a3);
}

__global__ void hyper_combine_kernel(const double* __restrict__ partials, int nblocks, int E,
                                     double* __restrict__ sums)
{
    hyper_combine_body(partials, nblocks, E, sums, (int)(blockIdx.x * blockDim.x + threadIdx.x));
}

__global__ void hyper_combine_batch_kernel(const BatchEntry<CombineArgs>* __restrict__ t, int n)
{
    const int j = batch_find(t, n, (int)blockIdx.x);
    const CombineArgs c = t[j].args;
    hyper_combine_body(c.partials, c.nblocks, c.E, c.sums,
                       ((int)blockIdx.x - t[j].first) * (int)blockDim.x + (int)threadIdx.x);
}

int hyper_combine_blocks(int kp) { return ((int)hyper_partial_doubles(kp) + 127) / 128; }

cudaError_t launch_hyper_combine(const double* partials, int nblocks, int kp, double* sums,
                                 cudaStream_t s)
{
    const int E = (int)hyper_partial_doubles(kp);
    hyper_combine_kernel<<<hyper_combine_blocks(kp), 128, 0, s>>>(partials, nblocks, E, sums);
    return cudaGetLastError();
}

cudaError_t launch_hyper_combine_batch(const BatchEntry<CombineArgs>* t, int n, int64_t blocks,
                                       cudaStream_t s)
{
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    hyper_combine_batch_kernel<<<(unsigned)blocks, 128, 0, s>>>(t, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Normal-Wishart draw, one CTA, FP64.  Matrices are K x K row-major in smem.
// ---------------------------------------------------------------------------
constexpr int kNWThreads = 256;
// 1 / sqrt(p) for p > 0 in FP64: an FP32 estimate refined by two steps of Newton's
// iteration for the reciprocal square root, y <- y (3 - p y^2) / 2, whose relative error
// squares each step (2^-23 -> 2^-45 -> FP64 rounding).  A handful of FP64 operations
// instead of a square root and a division (FP64 issues slowly on this GPU, and the
// factorisations below take one of these per column, serially).  Outside FP32's
// normal range: the FP64 square root and division.
__device__ __forceinline__ double rsqrt_newton(double p)
{
    if (p > 1e-30 && p < 1e30) {
        double y = (double)rsqrtf((float)p);
        y = y * fma(-0.5 * p * y, y, 1.5);
        y = y * fma(-0.5 * p * y, y, 1.5);
        return y;
    }
    return 1.0 / sqrt(p);
}

// In-place right-looking Cholesky of the lower triangle of A (K x K row-major in shared
// memory; the upper triangle is set to 0), by a block of kNWThreads = 256 threads.  Per
// column: one thread takes the pivot's reciprocal square root, the column is scaled by
// it, and the trailing lower triangle is updated on a 16 x 16 thread grid.  *bad is set
// on a non-positive pivot (which is replaced by 1).
__device__ void nw_cholesky(double* A, int K, int* bad)
{
    __shared__ double s_rinv;
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    for (int k = 0; k < K; ++k) {
        if (t == 0) {
            double p = A[k * K + k];
            if (!(p > 0.0)) {
                *bad = 1;
                p = 1.0;
            }
            const double r = rsqrt_newton(p);
            s_rinv = r;
            A[k * K + k] = p * r;
        }
        __syncthreads();
        const double rinv = s_rinv;
        for (int i = k + 1 + t; i < K; i += kNWThreads) A[i * K + k] *= rinv;
        __syncthreads();
        for (int i = k + 1 + ty; i < K; i += 16) {
            const double lik = A[i * K + k];
            for (int j = k + 1 + tx; j <= i; j += 16) A[i * K + j] = fma(-lik, A[j * K + k], A[i * K + j]);
        }
        __syncthreads();
    }
    for (int e = t; e < K * K; e += kNWThreads)
        if (e % K > e / K) A[e] = 0.0;
    __syncthreads();
}

// Dot product of x[0..n) and y[0..n) (strides sx, sy) with four interleaved FP64
// accumulators added in a fixed order: a quarter of the dependent chain.
__device__ __forceinline__ double dot4(const double* x, int sx, const double* y, int sy, int n)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = 0;
    for (; k + 3 < n; k += 4) {
        s0 = fma(x[k * sx], y[k * sy], s0);
        s1 = fma(x[(k + 1) * sx], y[(k + 1) * sy], s1);
        s2 = fma(x[(k + 2) * sx], y[(k + 2) * sy], s2);
        s3 = fma(x[(k + 3) * sx], y[(k + 3) * sy], s3);
    }
    for (; k < n; ++k) s0 = fma(x[k * sx], y[k * sy], s0);
    return (s0 + s1) + (s2 + s3);
}

// Entry e of the reduction's sums: from `sums`, or (nparts > 0) the fixed-order sum of the
// block partials, in the combine kernel's order (four interleaved accumulators).
__device__ double nw_sum(const NWArgs& a, int e)
{
    if (a.nparts == 0) return a.sums[e];
    const int E = (int)hyper_partial_doubles(a.kp);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = 0;
    for (; b + 3 < a.nparts; b += 4) {
        a0 += a.partials[(size_t)b * E + e];
        a1 += a.partials[(size_t)(b + 1) * E + e];
        a2 += a.partials[(size_t)(b + 2) * E + e];
        a3 += a.partials[(size_t)(b + 3) * E + e];
    }
    for (; b < a.nparts; ++b) a0 += a.partials[(size_t)b * E + e];
    return (a0 + a1) + (a2 + a3);
}

__device__ __forceinline__ void nw_sample_body(const NWArgs& a)
{
    extern __shared__ double nw_sm[];
    const int K = a.K, KK = K * K, t = threadIdx.x;
    double* M0 = nw_sm;
    double* M1 = M0 + KK;
    double* M2 = M1 + KK;
    double* mean = M2 + KK;
    double* dvec = mean + K;
    double* mustar = dvec + K;
    double* w = mustar + K;
    double* z = w + K;
    __shared__ int bad;
    const double n = (double)a.n;
    if (t == 0) bad = 0;
    // ---- statistics: mean = s + S1/n, S = S2/n - d d^T with d = S1/n ----
    for (int k = t; k < K; k += blockDim.x) {
        const double s = (double)(float)a.shift64[k];
        const double d = nw_sum(a, k) / n;
        dvec[k] = d;
        mean[k] = s + d;
    }
    __syncthreads();
    for (int e = t; e < KK; e += blockDim.x) {
        const int i = e / K, j = e % K;
        const double S = nw_sum(a, a.kp + i * a.kp + j) / n - dvec[i] * dvec[j];
        M1[e] = S;
        a.stats[K + e] = S;
    }
    for (int k = t; k < K; k += blockDim.x) a.stats[k] = mean[k];
    __syncthreads();
    // ---- posterior parameters ----
    const double beta_s = a.beta0 + n;
    const double cross = a.beta0 * n / (a.beta0 + n);
    for (int k = t; k < K; k += blockDim.x) mustar[k] = (a.beta0 * a.mu0[k] + n * mean[k]) / (a.beta0 + n);
    for (int e = t; e < KK; e += blockDim.x) {
        const int i = e / K, j = e % K;
        M0[e] = a.W0inv[e] + n * M1[e] + cross * (a.mu0[i] - mean[i]) * (a.mu0[j] - mean[j]);
    }
    __syncthreads();
    // ---- L_W = chol(W*), W* = P^{-1}.  With J the reversal (J_ij = [i + j = K - 1]) and
    // G = chol(J P J):  P^{-1} = J G^{-T} G^{-1} J, and J G^{-T} J is lower with a positive
    // diagonal, so it is the Cholesky factor of W* (one factorisation and one triangular
    // inverse instead of inverse, product and a second factorisation) ----
    for (int e = t; e < KK; e += kNWThreads) {
        const int i = e / K, j = e % K;
        M1[e] = M0[(K - 1 - i) * K + (K - 1 - j)];
    }
    __syncthreads();
    nw_cholesky(M1, K, &bad);  // G
    for (int k = t; k < K; k += kNWThreads) dvec[k] = 1.0 / M1[k * K + k];
    __syncthreads();
    // G^{-1} into M2 by forward substitution, four lanes per column: lane q of column j
    // sums the terms k = q (mod 4) and writes the rows i = q (mod 4), so it only reads
    // entries it wrote; the four partial sums meet by butterfly shuffles (every lane of a
    // warp runs every row, so the shuffles are uniform)
    {
        const int j = t >> 2, q = t & 3;
        const bool col = j < K;
        if (col && (j & 3) == q) M2[j * K + j] = dvec[j];
        for (int i = 1; i < K; ++i) {
            double part = 0.0;
            if (col && i > j)
                for (int k = j + ((q - j) & 3); k < i; k += 4) part = fma(M1[i * K + k], M2[k * K + j], part);
            part += __shfl_xor_sync(0xffffffffu, part, 1);
            part += __shfl_xor_sync(0xffffffffu, part, 2);
            if (col && i > j && (i & 3) == q) M2[i * K + j] = -part * dvec[i];
        }
        if (col)
            for (int i = q; i < j; i += 4) M2[i * K + j] = 0.0;
    }
    __syncthreads();
    // L_W[i][j] = G^{-1}[K-1-j][K-1-i] into M0 (lower)
    for (int e = t; e < KK; e += kNWThreads) {
        const int i = e / K, j = e % K;
        M0[e] = (j <= i) ? M2[(K - 1 - j) * K + (K - 1 - i)] : 0.0;
    }
    // ---- Bartlett factor A in M1 (its normals and chi^2 square roots from the draws
    // kernel) ----
    const int noff = K * (K - 1) / 2;
    for (int e = t; e < KK; e += kNWThreads) {
        const int i = e / K, j = e % K;
        M1[e] = j < i ? a.draws[i * (i - 1) / 2 + j] : (i == j ? a.draws[noff + K + i] : 0.0);
    }
    __syncthreads();
    // B = L_W A (lower times lower: lower) into M2
    for (int e = t; e < KK; e += kNWThreads) {
        const int i = e / K, j = e % K;
        M2[e] = (j <= i) ? dot4(M0 + i * K + j, 1, M1 + j * K + j, K, i - j + 1) : 0.0;
    }
    __syncthreads();
    // Lambda = B B^T into M1: the lower triangle, mirrored (the products are the same
    // either way round, so the matrix is exactly symmetric)
    for (int e = t; e < KK; e += kNWThreads) {
        const int i = e / K, j = e % K;
        if (j <= i) {
            const double v = dot4(M2 + i * K, 1, M2 + j * K, 1, j + 1);
            M1[i * K + j] = v;
            M1[j * K + i] = v;
        }
    }
    __syncthreads();
    // ---- C = chol(Lambda) by the same routine that bpmf_set_state's refresh uses on the
    // stored Lambda (so a resumed chain's rank-one route sees identical factors), and
    // mu = mu* + chol(beta* Lambda)^{-T} z = mu* + C^{-T} z / sqrt(beta*) ----
    for (int e = t; e < KK; e += kNWThreads) M0[e] = M1[e];
    for (int k = t; k < K; k += kNWThreads) z[k] = a.draws[noff + k];
    __syncthreads();
    nw_cholesky(M0, K, &bad);
    if (t < 32) {
        // back substitution C^T w = z / sqrt(beta*) in one warp: lane l keeps the residuals
        // of rows l and 32 + l; step i takes w_i from its owner and every lane removes
        // C[i][r] w_i from its rows r < i
        const double rb = 1.0 / sqrt(beta_s);
        double r1 = t < K ? z[t] * rb : 0.0, r2 = 32 + t < K ? z[32 + t] * rb : 0.0;
        for (int i = K - 1; i >= 0; --i) {
            const double own = i < 32 ? r1 : r2;
            const double wi = __shfl_sync(0xffffffffu, own, i & 31) / M0[i * K + i];
            if (t == 0) w[i] = wi;
            if (t < i) r1 = fma(-M0[i * K + t], wi, r1);
            if (32 + t < i) r2 = fma(-M0[i * K + 32 + t], wi, r2);
        }
    }
    __syncthreads();
    // ---- outputs ----
    for (int k = t; k < K; k += blockDim.x) a.mu64[k] = mustar[k] + w[k];
    for (int e = t; e < KK; e += blockDim.x) a.lam64[e] = M1[e];
    const int kp = a.kp;
    for (int e = t; e < kp * kp; e += blockDim.x) {
        const int i = e / kp, j = e % kp;
        const bool in = i < K && j < K;
        const float v = in ? (float)M1[i * K + j] : (i == j ? 1.f : 0.f);
        a.lam32[e] = v;
        a.lam32[kp * kp + chunk_t_index(i, j, kp)] = v;
        // chol(Lambda) for the rank-one route
        const float c = in ? (float)M0[i * K + j] : (i == j ? 1.f : 0.f);
        a.lam32[2 * kp * kp + chunk_t_index(i, j, kp)] = c;
    }
    for (int i = t; i < kp; i += blockDim.x) {
        double s = 0.0;
        if (i < K)
            for (int j = 0; j < K; ++j) s += M1[i * K + j] * (mustar[j] + w[j]);
        a.lammu32[i] = (float)s;
    }
    if (t == 0) {
        unsigned int st = 0;
        if (bad) st |= kStatusNotPD;
        if (st) atomicOr(&a.ctl->status, st);
    }
}

__global__ void __launch_bounds__(kNWThreads) nw_sample_kernel(NWArgs a) { nw_sample_body(a); }

// One CTA per job.
__global__ void __launch_bounds__(kNWThreads) nw_sample_batch_kernel(const NWArgs* __restrict__ t)
{
    const NWArgs a = t[blockIdx.x];
    nw_sample_body(a);
}

static size_t nw_smem(int K) { return sizeof(double) * (3 * (size_t)K * K + 5 * (size_t)K); }

cudaError_t launch_nw_sample(const NWArgs& a, cudaStream_t s)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(nw_sample_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)nw_smem(64));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    nw_sample_kernel<<<1, kNWThreads, nw_smem(a.K), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_nw_sample_batch(const NWArgs* t, int n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(nw_sample_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)nw_smem(64));
    if (e != cudaSuccess) return e;
    nw_sample_batch_kernel<<<(unsigned)n, kNWThreads, nw_smem(64), s>>>(t);
    return cudaGetLastError();
}

__global__ void hyper_refresh_kernel(const double* mu64, const double* lam64, int K, int kp,
                                     float* lam32, float* lammu32, Control* ctl)
{
    extern __shared__ double rf_sm[];  // K x K: chol(Lambda) for the rank-one route
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) rf_sm[e] = lam64[e];
    __syncthreads();
    nw_cholesky(rf_sm, K, &bad);
    for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) {
        const int i = e / kp, j = e % kp;
        const bool in = i < K && j < K;
        const float v = in ? (float)lam64[i * K + j] : (i == j ? 1.f : 0.f);
        lam32[e] = v;
        lam32[kp * kp + chunk_t_index(i, j, kp)] = v;
        const float c = in ? (float)rf_sm[i * K + j] : (i == j ? 1.f : 0.f);
        lam32[2 * kp * kp + chunk_t_index(i, j, kp)] = c;
    }
    if (threadIdx.x == 0 && bad && ctl) atomicOr(&ctl->status, kStatusNotPD);
    for (int i = threadIdx.x; i < kp; i += blockDim.x) {
        double s = 0.0;
        if (i < K)
            for (int j = 0; j < K; ++j) s += lam64[i * K + j] * mu64[j];
        lammu32[i] = (float)s;
    }
}

cudaError_t launch_hyper_refresh(const double* mu64, const double* lam64, int K, int kp,
                                 float* lam32, float* lammu32, Control* ctl, cudaStream_t s)
{
    hyper_refresh_kernel<<<1, 256, sizeof(double) * K * K, s>>>(mu64, lam64, K, kp, lam32,
                                                                 lammu32, ctl);
    return cudaGetLastError();
}

}  // namespace bpmf
