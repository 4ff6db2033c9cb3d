// k_misc.cu -- initial factors, rating centring, test-set prediction and RMSE
// (Alg. 1, last inner loop: "for all test points: predict rating and compute
// RMSE"), and the sweep counter.
#include <math.h>

#include "bpmf_internal.cuh"
#include "philox.cuh"

namespace bpmf {

// U or V ~ N(0, 1): row r takes normals 0..K-1 of its init stream (c1 = r,
// c2 = 0); one thread per Philox call (four normals); padding columns are 0.
__global__ void init_factors_kernel(float* X, int64_t rows, int K, int ld, uint64_t seed, uint32_t c3)
{
    const int calls = ld / 4;
    const int64_t n = rows * calls;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / calls;
        const int c = (int)(e % calls);
        float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        if (4 * c < K) z = normals4_f32(seed, (uint32_t)c, (uint32_t)r, 0u, c3);
        const int k = 4 * c;
        if (k + 0 >= K) z.x = 0.f;
        if (k + 1 >= K) z.y = 0.f;
        if (k + 2 >= K) z.z = 0.f;
        if (k + 3 >= K) z.w = 0.f;
        reinterpret_cast<float4*>(X + r * ld)[c] = z;
    }
}

cudaError_t launch_init_factors(float* X, int64_t rows, int K, int ld, uint64_t seed, uint32_t c3,
                                cudaStream_t s)
{
    const int64_t n = rows * (ld / 4);
    const int blocks = (int)((n + 255) / 256 < 65535 * 8 ? (n + 255) / 256 : 65535 * 8);
    if (blocks < 1) return cudaSuccess;
    init_factors_kernel<<<blocks, 256, 0, s>>>(X, rows, K, ld, seed, c3);
    return cudaGetLastError();
}

// Ratings check and FP64 sum in a fixed order (the result does not depend on timing):
// block b takes the contiguous range [b n / B, (b + 1) n / B), thread t its elements
// t, t + 256, ... in order, then a fixed tree; the finishing block adds the B partials
// the same way.  Column indices outside [0, ncols) set *bad.
constexpr int kSumThreads = 256;

__device__ double block_tree_sum(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = kSumThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    return sh[0];
}

__global__ void __launch_bounds__(kSumThreads) check_sum_kernel(const int32_t* __restrict__ col,
                                                               const float* __restrict__ val,
                                                               int64_t n, int32_t ncols,
                                                               double* __restrict__ partials,
                                                               unsigned int* bad)
{
    __shared__ double sh[kSumThreads];
    const int64_t lo = n * blockIdx.x / gridDim.x, hi = n * (blockIdx.x + 1) / gridDim.x;
    double acc = 0.0;
    bool ok = true;
    for (int64_t e = lo + threadIdx.x; e < hi; e += kSumThreads) {
        const int32_t c = col[e];
        ok &= c >= 0 && c < ncols;
        acc += (double)val[e];
    }
    if (!ok) atomicOr(bad, 1u);
    const double t = block_tree_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kSumThreads) sum_finish_kernel(const double* __restrict__ partials,
                                                                int nparts, double* out)
{
    __shared__ double sh[kSumThreads];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nparts; b += kSumThreads) acc += partials[b];
    const double t = block_tree_sum(acc, sh);
    if (threadIdx.x == 0) *out = t;
}

cudaError_t launch_check_sum(const int32_t* col, const float* val, int64_t n, int32_t ncols,
                             double* scratch, unsigned int* bad, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (n > 0) {
        check_sum_kernel<<<kCheckSumBlocks, kSumThreads, 0, s>>>(col, val, n, ncols, scratch + 1, bad);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        sum_finish_kernel<<<1, kSumThreads, 0, s>>>(scratch + 1, kCheckSumBlocks, scratch);
        return cudaGetLastError();
    }
    return cudaMemsetAsync(scratch, 0, sizeof(double), s);
}

__global__ void center_values_kernel(float* val, int64_t n, double rbar)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        val[e] = (float)((double)val[e] - rbar);
}

cudaError_t launch_center_values(float* val, int64_t n, double rbar, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const int blocks = (int)(want < 4096 ? want : 4096);
    center_values_kernel<<<blocks, 256, 0, s>>>(val, n, rbar);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// prediction / RMSE
// ---------------------------------------------------------------------------
constexpr int kPredThreads = 256;

int predict_blocks(int64_t T, int num_sms)
{
    int64_t want = (T + kPredThreads - 1) / kPredThreads;
    int64_t cap = (int64_t)num_sms * 4;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

__device__ __forceinline__ float dot_row(const float* __restrict__ u, const float* __restrict__ v,
                                         int kp)
{
    float s = 0.f;
    for (int k = 0; k < kp; k += 4) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(u + k));
        const float4 b = __ldg(reinterpret_cast<const float4*>(v + k));
        s = fmaf(a.x, b.x, s);
        s = fmaf(a.y, b.y, s);
        s = fmaf(a.z, b.z, s);
        s = fmaf(a.w, b.w, s);
    }
    return s;
}

__device__ __forceinline__ double block_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;
}

// Block `bid` of `nblocks` of one job's prediction launch.
__device__ __forceinline__ void predict_body(
    const int32_t* __restrict__ ti, const int32_t* __restrict__ tj, const float* __restrict__ tr,
    int64_t T, const float* __restrict__ U, const float* __restrict__ V, int ld, int kp,
    double rbar, int clip, double lo, double hi, int burn_in, double* __restrict__ psum,
    const Control* __restrict__ ctl, double* __restrict__ partials, int64_t bid, int64_t nblocks)
{
    __shared__ double red[kPredThreads / 32];
    const int acc = (long long)ctl->sweep >= (long long)burn_in ? 1 : 0;
    const long long n_new = ctl->n_avg + acc;
    double se = 0.0, sa = 0.0;
    for (int64_t t = bid * blockDim.x + threadIdx.x; t < T; t += nblocks * blockDim.x) {
        const int i = ti[t], j = tj[t];
        double p = rbar + (double)dot_row(U + (int64_t)i * ld, V + (int64_t)j * ld, kp);
        if (clip) p = fmin(fmax(p, lo), hi);
        const double r = (double)tr[t];
        se += (p - r) * (p - r);
        double ps = psum[t];
        if (acc) {
            ps += p;
            psum[t] = ps;
        }
        if (n_new > 0) {
            const double pa = ps / (double)n_new;
            sa += (pa - r) * (pa - r);
        }
    }
    const double bse = block_sum(se, red);
    const double bsa = block_sum(sa, red);
    if (threadIdx.x == 0) {
        partials[2 * bid] = bse;
        partials[2 * bid + 1] = bsa;
    }
}

__global__ void __launch_bounds__(kPredThreads) predict_kernel(
    const int32_t* __restrict__ ti, const int32_t* __restrict__ tj, const float* __restrict__ tr,
    int64_t T, const float* __restrict__ U, const float* __restrict__ V, int ld, int kp,
    double rbar, int clip, double lo, double hi, int burn_in, double* __restrict__ psum,
    const Control* __restrict__ ctl, double* __restrict__ partials)
{
    predict_body(ti, tj, tr, T, U, V, ld, kp, rbar, clip, lo, hi, burn_in, psum, ctl, partials,
                 blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(kPredThreads)
    predict_batch_kernel(const BatchEntry<PredictArgs>* __restrict__ tab, int n)
{
    const int j = batch_find(tab, n, (int)blockIdx.x);
    const PredictArgs p = tab[j].args;
    predict_body(p.ti, p.tj, p.tr, p.T, p.U, p.V, p.ld, p.kp, p.rbar, p.clip, p.lo, p.hi,
                 p.burn_in, p.psum, p.ctl, p.partials, (int64_t)blockIdx.x - tab[j].first,
                 tab[j].count);
}

cudaError_t launch_predict(const int32_t* ti, const int32_t* tj, const float* tr, int64_t T,
                           const float* U, const float* V, int ld, int kp, double rbar, int clip,
                           double lo, double hi, int burn_in, double* psum, Control* ctl,
                           double* partials, int nblocks, cudaStream_t s)
{
    predict_kernel<<<nblocks, kPredThreads, 0, s>>>(ti, tj, tr, T, U, V, ld, kp, rbar, clip, lo,
                                                    hi, burn_in, psum, ctl, partials);
    return cudaGetLastError();
}

__device__ __forceinline__ void predict_finish_body(const double* partials, int nblocks,
                                                    int64_t T, int burn_in, Control* ctl)
{
    const int acc = (long long)ctl->sweep >= (long long)burn_in ? 1 : 0;
    const long long n_new = ctl->n_avg + acc;
    double se = 0.0, sa = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        se += partials[2 * b];
        sa += partials[2 * b + 1];
    }
    ctl->n_avg = n_new;
    if (T > 0) {
        ctl->rmse_sample = sqrt(se / (double)T);
        ctl->rmse_avg = n_new > 0 ? sqrt(sa / (double)T) : (double)NAN;
    } else {
        ctl->rmse_sample = (double)NAN;
        ctl->rmse_avg = (double)NAN;
    }
}

__global__ void predict_finish_kernel(const double* partials, int nblocks, int64_t T, int burn_in,
                                      Control* ctl)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    predict_finish_body(partials, nblocks, T, burn_in, ctl);
}

// One thread per job: the job's RMSEs from its prediction partials (its `count` blocks;
// none without test points), then, with advance, its sweep counter moved on.
__global__ void predict_finish_batch_kernel(const BatchEntry<PredictArgs>* __restrict__ tab, int n,
                                            int advance)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const PredictArgs p = tab[j].args;
    predict_finish_body(p.partials, p.T > 0 ? tab[j].count : 0, p.T, p.burn_in, p.ctl);
    if (advance) p.ctl->sweep += 1ull;
}

cudaError_t launch_predict_batch(const BatchEntry<PredictArgs>* t, int n, int64_t blocks,
                                 cudaStream_t s)
{
    if (n <= 0 || blocks <= 0) return cudaSuccess;
    predict_batch_kernel<<<(unsigned)blocks, kPredThreads, 0, s>>>(t, n);
    return cudaGetLastError();
}

cudaError_t launch_predict_finish_batch(const BatchEntry<PredictArgs>* t, int n, bool advance,
                                        cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    predict_finish_batch_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(t, n, advance ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_predict_finish(const double* partials, int nblocks, int64_t T, int burn_in,
                                  Control* ctl, cudaStream_t s)
{
    predict_finish_kernel<<<1, 32, 0, s>>>(partials, nblocks, T, burn_in, ctl);
    return cudaGetLastError();
}

__global__ void predict_points_kernel(const int32_t* __restrict__ pi, const int32_t* __restrict__ pj,
                                      int64_t n, const float* __restrict__ U,
                                      const float* __restrict__ V, int ld, int kp, double rbar,
                                      int clip, double lo, double hi, float* __restrict__ out)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x) {
        double p = rbar + (double)dot_row(U + (int64_t)pi[t] * ld, V + (int64_t)pj[t] * ld, kp);
        if (clip) p = fmin(fmax(p, lo), hi);
        out[t] = (float)p;
    }
}

cudaError_t launch_predict_points(const int32_t* i, const int32_t* j, int64_t n, const float* U,
                                  const float* V, int ld, int kp, double rbar, int clip, double lo,
                                  double hi, float* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t want = (n + 255) / 256;
    const int blocks = (int)(want < 4096 ? want : 4096);
    predict_points_kernel<<<blocks, 256, 0, s>>>(i, j, n, U, V, ld, kp, rbar, clip, lo, hi, out);
    return cudaGetLastError();
}

__global__ void advance_kernel(Control* ctl)
{
    if (threadIdx.x == 0) ctl->sweep += 1ull;
}

cudaError_t launch_advance(Control* ctl, cudaStream_t s)
{
    advance_kernel<<<1, 32, 0, s>>>(ctl);
    return cudaGetLastError();
}

}  // namespace bpmf
