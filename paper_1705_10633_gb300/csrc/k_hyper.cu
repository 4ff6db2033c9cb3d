// k_hyper.cu -- the hyper-parameter step of Alg. 1 ("sample hyper-parameters
// movies/users based on V/U", Sec. 2): sufficient statistics of a factor matrix
// and the Normal-Wishart draw of (mu, Lambda).
//
//   reduce : every block streams a contiguous slab of rows once (HBM bound),
//            accumulating (x - s) and (x - s)(x - s)^T in FP32 registers over
//            64-row chunks and folding each chunk into FP64 accumulators; s is
//            the side's current hyper mean, so the sums stay small.
//   combine: fixed-order FP64 sum of the block partials (deterministic).
//   nw     : one CTA in FP64 -- posterior parameters, Cholesky, inverse,
//            Bartlett Wishart draw with Marsaglia-Tsang gammas, mean draw.
#include "bpmf_internal.cuh"
#include "philox.cuh"

namespace bpmf {

// ---------------------------------------------------------------------------
// reduction
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedChunk = 64;

int hyper_reduce_blocks(int64_t rows, int num_sms)
{
    int64_t want = (rows + 1023) / 1024;  // at least ~1k rows per block
    int64_t cap = (int64_t)num_sms * 2;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

template <int KT>
__global__ void __launch_bounds__(kRedThreads) hyper_reduce_kernel(const float* __restrict__ X,
                                                                   int64_t rows,
                                                                   const double* __restrict__ shift64,
                                                                   double* __restrict__ partials)
{
    constexpr int TT = KT / 16;  // each thread owns a TT x TT tile of the scatter
    __shared__ __align__(16) float xs[kRedChunk][KT];
    __shared__ float sh[KT];
    const int t = threadIdx.x;
    const int ty = t / 16, tx = t % 16;
    if (t < KT) sh[t] = (float)shift64[t];
    const int64_t r0 = rows * blockIdx.x / gridDim.x;
    const int64_t r1 = rows * (blockIdx.x + 1) / gridDim.x;
    double acc64[TT][TT];
    double s64 = 0.0;
#pragma unroll
    for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) acc64[i][j] = 0.0;
    __syncthreads();
    for (int64_t base = r0; base < r1; base += kRedChunk) {
        const int cnt = (int)min((int64_t)kRedChunk, r1 - base);
        // stage (x - s) for the chunk; rows past the end are zero
        constexpr int F4 = KT / 4;
        for (int e = t; e < kRedChunk * F4; e += kRedThreads) {
            const int r = e / F4, f = e % F4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < cnt) {
                v = __ldg(reinterpret_cast<const float4*>(X + (base + r) * KT) + f);
                v.x -= sh[4 * f + 0];
                v.y -= sh[4 * f + 1];
                v.z -= sh[4 * f + 2];
                v.w -= sh[4 * f + 3];
            }
            *reinterpret_cast<float4*>(&xs[r][4 * f]) = v;
        }
        __syncthreads();
        float acc[TT][TT];
        float s32 = 0.f;
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
            if (t < KT) s32 += xs[r][t];
        }
#pragma unroll
        for (int i = 0; i < TT; ++i)
#pragma unroll
            for (int j = 0; j < TT; ++j) acc64[i][j] += (double)acc[i][j];
        s64 += (double)s32;
        __syncthreads();
    }
    double* out = partials + (size_t)blockIdx.x * hyper_partial_doubles(KT);
    if (t < KT) out[t] = s64;
#pragma unroll
    for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) out[KT + (ty * TT + i) * KT + tx * TT + j] = acc64[i][j];
}

// Shift for the statistics: the FP64 mean of the first rows (at most kShiftRows),
// zero beyond K.  Subtracting a value near the mean keeps the FP32 chunk sums of
// (x - s)(x - s)^T from cancelling against d d^T; a shift taken from the data itself
// (rather than from the last drawn mu, which can sit far from the sample mean when a
// side has few rows) and computed in a fixed order keeps resumed chains bit-identical.
constexpr int64_t kShiftRows = 256;

__global__ void hyper_shift_kernel(const float* __restrict__ X, int64_t rows, int K, int kp,
                                   double* __restrict__ shift64)
{
    const int t = threadIdx.x;
    if (t >= kp) return;
    const int64_t n = rows < kShiftRows ? rows : kShiftRows;
    double s = 0.0;
    if (t < K)
        for (int64_t r = 0; r < n; ++r) s += (double)X[r * kp + t];
    shift64[t] = (t < K && n > 0) ? s / (double)n : 0.0;
}

cudaError_t launch_hyper_shift(const float* X, int64_t rows, int K, int kp, double* shift64,
                               cudaStream_t s)
{
    hyper_shift_kernel<<<1, 64, 0, s>>>(X, rows, K, kp, shift64);
    return cudaGetLastError();
}

cudaError_t launch_hyper_reduce(const float* X, int64_t rows, int kp, const double* shift64,
                                double* partials, int nblocks, cudaStream_t s)
{
    switch (kp) {
    case 16: hyper_reduce_kernel<16><<<nblocks, kRedThreads, 0, s>>>(X, rows, shift64, partials); break;
    case 32: hyper_reduce_kernel<32><<<nblocks, kRedThreads, 0, s>>>(X, rows, shift64, partials); break;
    case 48: hyper_reduce_kernel<48><<<nblocks, kRedThreads, 0, s>>>(X, rows, shift64, partials); break;
    case 64: hyper_reduce_kernel<64><<<nblocks, kRedThreads, 0, s>>>(X, rows, shift64, partials); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

__global__ void hyper_combine_kernel(const double* __restrict__ partials, int nblocks, int E,
                                     double* __restrict__ sums)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double acc = 0.0;
    for (int b = 0; b < nblocks; ++b) acc += partials[(size_t)b * E + e];
    sums[e] = acc;
}

cudaError_t launch_hyper_combine(const double* partials, int nblocks, int kp, double* sums,
                                 cudaStream_t s)
{
    const int E = (int)hyper_partial_doubles(kp);
    hyper_combine_kernel<<<(E + 127) / 128, 128, 0, s>>>(partials, nblocks, E, sums);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Normal-Wishart draw, one CTA, FP64.  Matrices are K x K row-major in smem.
// ---------------------------------------------------------------------------
constexpr int kNWThreads = 256;
constexpr int kGammaMaxAttempts = 64;

// In-place right-looking Cholesky of the lower triangle of A (upper set to 0).
// Returns false (in every thread) if a pivot is not positive.
__device__ bool nw_cholesky(double* A, int K, int* bad)
{
    const int t = threadIdx.x;
    for (int k = 0; k < K; ++k) {
        if (t == 0) {
            const double p = A[k * K + k];
            if (!(p > 0.0)) *bad = 1;
            A[k * K + k] = sqrt(p > 0.0 ? p : 1.0);
        }
        __syncthreads();
        const double lkk = A[k * K + k];
        for (int i = k + 1 + t; i < K; i += blockDim.x) A[i * K + k] /= lkk;
        __syncthreads();
        // trailing update of the lower triangle, j in (k, i]
        const int m = K - k - 1;
        for (int e = t; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) A[i * K + j] -= A[i * K + k] * A[j * K + k];
        }
        __syncthreads();
    }
    for (int e = t; e < K * K; e += blockDim.x)
        if (e % K > e / K) A[e] = 0.0;
    __syncthreads();
    return *bad == 0;
}

__global__ void __launch_bounds__(kNWThreads) nw_sample_kernel(NWArgs a)
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
    __shared__ int bad, gbad;
    const uint32_t sweep = (uint32_t)a.ctl->sweep + a.sweep_offset;
    const double n = (double)a.n;
    if (t == 0) { bad = 0; gbad = 0; }
    // ---- statistics: mean = s + S1/n, S = S2/n - d d^T with d = S1/n ----
    for (int k = t; k < K; k += blockDim.x) {
        const double s = (double)(float)a.shift64[k];
        const double d = a.sums[k] / n;
        dvec[k] = d;
        mean[k] = s + d;
    }
    __syncthreads();
    for (int e = t; e < KK; e += blockDim.x) {
        const int i = e / K, j = e % K;
        const double S = a.sums[a.kp + i * a.kp + j] / n - dvec[i] * dvec[j];
        M1[e] = S;
        a.stats[K + e] = S;
    }
    for (int k = t; k < K; k += blockDim.x) a.stats[k] = mean[k];
    __syncthreads();
    // ---- posterior parameters ----
    const double beta_s = a.beta0 + n, nu_s = a.nu0 + n;
    const double cross = a.beta0 * n / (a.beta0 + n);
    for (int k = t; k < K; k += blockDim.x) mustar[k] = (a.beta0 * a.mu0[k] + n * mean[k]) / (a.beta0 + n);
    for (int e = t; e < KK; e += blockDim.x) {
        const int i = e / K, j = e % K;
        M0[e] = a.W0inv[e] + n * M1[e] + cross * (a.mu0[i] - mean[i]) * (a.mu0[j] - mean[j]);
    }
    __syncthreads();
    // ---- W* = P^{-1}: chol(P) = L, Linv by forward substitution per column ----
    nw_cholesky(M0, K, &bad);
    for (int j = t; j < K; j += blockDim.x) {
        for (int i = 0; i < K; ++i) {
            double v;
            if (i < j) v = 0.0;
            else {
                double s = (i == j) ? 1.0 : 0.0;
                for (int k = j; k < i; ++k) s -= M0[i * K + k] * M1[k * K + j];
                v = s / M0[i * K + i];
            }
            M1[i * K + j] = v;  // column j is private to this thread
        }
    }
    __syncthreads();
    // W = Linv^T Linv
    for (int e = t; e < KK; e += blockDim.x) {
        const int i = e / K, j = e % K;
        const int k0 = i > j ? i : j;
        double s = 0.0;
        for (int k = k0; k < K; ++k) s += M1[k * K + i] * M1[k * K + j];
        M2[e] = s;
    }
    __syncthreads();
    // L_W = chol(W) in M2
    nw_cholesky(M2, K, &bad);
    // ---- Bartlett factor A in M1 ----
    for (int e = t; e < KK; e += blockDim.x) M1[e] = 0.0;
    __syncthreads();
    for (int k = t; k < K; k += blockDim.x) {
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
            if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) { g = d * v; break; }
        }
        if (g < 0.0) { gbad = 1; g = shape; }
        M1[k * K + k] = sqrt(2.0 * g);
    }
    const int noff = K * (K - 1) / 2;
    for (int q = t; q < noff; q += blockDim.x) {
        // q = k(k-1)/2 + l, k > l
        int k = (int)((1.0 + sqrt(1.0 + 8.0 * (double)q)) * 0.5);
        while (k * (k - 1) / 2 > q) --k;
        while ((k + 1) * k / 2 <= q) ++k;
        const int l = q - k * (k - 1) / 2;
        M1[k * K + l] = normal_f64(a.seed, (uint32_t)q, 0u, sweep, a.c3_normal);
    }
    __syncthreads();
    // B = L_W A (lower) into M0
    for (int e = t; e < KK; e += blockDim.x) {
        const int i = e / K, j = e % K;
        double s = 0.0;
        for (int k = j; k <= i; ++k) s += M2[i * K + k] * M1[k * K + j];
        M0[e] = (j <= i) ? s : 0.0;
    }
    __syncthreads();
    // Lambda = B B^T into M1
    for (int e = t; e < KK; e += blockDim.x) {
        const int i = e / K, j = e % K;
        const int kmax = i < j ? i : j;
        double s = 0.0;
        for (int k = 0; k <= kmax; ++k) s += M0[i * K + k] * M0[j * K + k];
        M1[e] = s;
    }
    __syncthreads();
    // ---- C = chol(Lambda) by the same routine that bpmf_set_state's refresh uses on the
    // stored Lambda (so a resumed chain's rank-one route sees identical factors), and
    // mu = mu* + chol(beta* Lambda)^{-T} z = mu* + C^{-T} z / sqrt(beta*) ----
    for (int e = t; e < KK; e += blockDim.x) M2[e] = M1[e];
    for (int k = t; k < K; k += blockDim.x) z[k] = normal_f64(a.seed, (uint32_t)k, 1u, sweep, a.c3_normal);
    __syncthreads();
    nw_cholesky(M2, K, &bad);
    if (t == 0) {
        const double rb = 1.0 / sqrt(beta_s);
        for (int i = K - 1; i >= 0; --i) {
            double s = z[i] * rb;
            for (int k = i + 1; k < K; ++k) s -= M2[k * K + i] * w[k];
            w[i] = s / M2[i * K + i];
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
        const float c = in ? (float)M2[i * K + j] : (i == j ? 1.f : 0.f);
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
        if (gbad) st |= kStatusGamma;
        if (st) atomicOr(&a.ctl->status, st);
    }
}

cudaError_t launch_nw_sample(const NWArgs& a, cudaStream_t s)
{
    const size_t smem = sizeof(double) * (3 * (size_t)a.K * a.K + 5 * (size_t)a.K);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(nw_sample_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(sizeof(double) * (3 * 64 * 64 + 5 * 64)));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    nw_sample_kernel<<<1, kNWThreads, smem, s>>>(a);
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
