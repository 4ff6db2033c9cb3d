// bpmf_noalloc.cu -- row statistics of a device matrix without allocating.
//
// Some callers cannot allocate device memory at the moment they need this
// reduction: a serving process whose memory pool has already reserved the
// whole GPU (cudaMalloc would fail), or a latency-critical loop where
// cudaMalloc/cudaFree would synchronise the device and stall the other
// streams.  This entry point runs the same two reduction kernels as the hyper
// step of a handle (block partial sums, then their fixed-order combine), but
// keeps their scratch in a file-scope __device__ array of fixed size instead
// of memory owned by a handle.
//
// The array is part of the library's device image: every GPU on which the
// library is loaded holds it (kScratchDoubles doubles, about 5.4 MB) until the
// process exits.  Host code cannot use the array's name as a device address,
// so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.  The cached
// address belongs to the device context of that first call: after a
// cudaDeviceReset in the same process the module is loaded again and the array
// may move, so the entry point must not be called after a reset.
#include <stdint.h>

#include <mutex>

#include "bpmf.h"
#include "bpmf_internal.cuh"

namespace {

constexpr int kNoAllocMaxK = 64;       // largest K the scratch is sized for
constexpr int kNoAllocMaxBlocks = 160; // reduction blocks the scratch holds
constexpr size_t kEntries = (size_t)kNoAllocMaxK + (size_t)kNoAllocMaxK * kNoAllocMaxK;
// layout: [padded shift: 64] [combined sums: kEntries] [block partials: blocks x kEntries]
constexpr size_t kShiftOff = 0;
constexpr size_t kSumsOff = kNoAllocMaxK;
constexpr size_t kPartialsOff = kSumsOff + kEntries;
constexpr size_t kScratchDoubles = kPartialsOff + (size_t)kNoAllocMaxBlocks * kEntries;

__device__ __align__(256) double g_row_stats_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_lookup_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int scratch_on_current_device(double** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return BPMF_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return BPMF_EINVAL;
    std::lock_guard<std::mutex> lock(g_lookup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_row_stats_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return BPMF_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return BPMF_OK;
}

// Shift padded with zeros to the kernel width; a null shift means zero.
__global__ void stage_shift_kernel(const double* __restrict__ shift, int K, int kp,
                                   double* __restrict__ dst)
{
    for (int k = threadIdx.x; k < kp; k += blockDim.x) dst[k] = (shift && k < K) ? shift[k] : 0.0;
}

// mean = s + S1 / n and S = S2 / n - d d^T with d = S1 / n (the same formulas the
// hyper step applies before its Normal-Wishart draw).
__global__ void stats_finalize_kernel(const double* __restrict__ sums,
                                      const double* __restrict__ shift_padded, int64_t n, int K,
                                      int kp, double* __restrict__ mean, double* __restrict__ S)
{
    const double nd = (double)n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += gridDim.x * blockDim.x) {
        const int i = e / K, j = e % K;
        const double di = sums[i] / nd, dj = sums[j] / nd;
        S[e] = sums[kp + i * kp + j] / nd - di * dj;
        if (j == 0) mean[i] = (double)(float)shift_padded[i] + di;
    }
}

}  // namespace

extern "C" int bpmf_row_stats_noalloc(const float* X, int64_t rows, int32_t K, const double* shift,
                                      double* mean, double* S, void* cuda_stream)
{
    if (!X || !mean || !S) return BPMF_EINVAL;
    // the reduction reads X a float4 at a time; the FP64 buffers are read and written
    // as doubles: misaligned pointers are refused here, before any launch
    if ((reinterpret_cast<uintptr_t>(X) & 15u) != 0 || (reinterpret_cast<uintptr_t>(mean) & 7u) != 0 ||
        (reinterpret_cast<uintptr_t>(S) & 7u) != 0 || (reinterpret_cast<uintptr_t>(shift) & 7u) != 0)
        return BPMF_EINVAL;
    if (K < 1 || K > kNoAllocMaxK) return BPMF_EINVAL;  // beyond the static scratch
    if (rows < 1 || rows > (int64_t)INT32_MAX) return BPMF_EINVAL;
    const int kp = (K + 15) / 16 * 16;
    double* scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc != BPMF_OK) return rc;
    int dev = 0, num_sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return BPMF_ECUDA;
    }
    int nblocks = bpmf::hyper_reduce_blocks(rows, num_sms);
    if (nblocks > kNoAllocMaxBlocks) nblocks = kNoAllocMaxBlocks;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    double* shift_padded = scratch + kShiftOff;
    double* sums = scratch + kSumsOff;
    double* partials = scratch + kPartialsOff;
    stage_shift_kernel<<<1, 64, 0, s>>>(shift, K, kp, shift_padded);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = bpmf::launch_hyper_reduce(X, rows, kp, shift_padded, partials, nblocks, s);
    if (e == cudaSuccess) e = bpmf::launch_hyper_combine(partials, nblocks, kp, sums, s);
    if (e == cudaSuccess) {
        stats_finalize_kernel<<<(K * K + 255) / 256, 256, 0, s>>>(sums, shift_padded, rows, K, kp,
                                                                  mean, S);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? BPMF_OK : BPMF_ECUDA;
}
