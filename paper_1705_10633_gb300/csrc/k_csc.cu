// k_csc.cu -- column view (CSC) of the ratings built on the device from the CSR
// already uploaded, in the same order as a host counting sort: inside each column
// the entries keep their row-major order (a stable sort by column).
//
//   counts per column (atomics) -> exclusive scan -> column pointers
//   stable radix sort of (column, position) pairs over the bits the columns need
//   gather: row of each position (binary search in the row pointers) and its value
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "bpmf_internal.cuh"

namespace bpmf {
namespace {

__global__ void col_count_kernel(const int32_t* __restrict__ col, int64_t nnz,
                                 unsigned long long* __restrict__ counts)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + col[e], 1ull);
}

__global__ void iota_kernel(int32_t* __restrict__ v, int64_t n)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        v[e] = (int32_t)e;
}

// rows[k] = the row holding position perm[k] (last r with ptr[r] <= perm[k]),
// vals[k] = val[perm[k]]
__global__ void csc_gather_kernel(const int32_t* __restrict__ perm, int64_t nnz,
                                  const int64_t* __restrict__ ptr, int64_t M,
                                  const float* __restrict__ val, int32_t* __restrict__ rows,
                                  float* __restrict__ vals)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = perm[k];
        int64_t lo = 0, hi = M;  // ptr[lo] <= e < ptr[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (ptr[mid] <= e) lo = mid;
            else hi = mid;
        }
        rows[k] = (int32_t)lo;
        vals[k] = val[e];
    }
}

int grid_for(int64_t n) { return (int)(n / 256 + 1 < 16384 ? n / 256 + 1 : 16384); }

}  // namespace

cudaError_t build_csc_device(const int64_t* csr_ptr, const int32_t* csr_col, const float* csr_val,
                             int64_t M, int64_t N, int64_t nnz, int64_t* csc_ptr, int32_t* csc_row,
                             float* csc_val, const TempAlloc& tmp, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(csc_ptr, 0, sizeof(int64_t) * (N + 1), s);
    if (e != cudaSuccess || nnz == 0) return e;
    // column pointers: counts into csc_ptr[1..N], then an inclusive scan in place
    col_count_kernel<<<grid_for(nnz), 256, 0, s>>>(
        csr_col, nnz, reinterpret_cast<unsigned long long*>(csc_ptr + 1));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    size_t scan_bytes = 0, sort_bytes = 0;
    int end_bit = 1;
    while (end_bit < 31 && (int64_t(1) << end_bit) < N) ++end_bit;
    const uint32_t* keys = reinterpret_cast<const uint32_t*>(csr_col);
    e = cub::DeviceScan::InclusiveSum(nullptr, scan_bytes, csc_ptr + 1, csc_ptr + 1, N, s);
    if (e == cudaSuccess)
        e = cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, keys, (uint32_t*)nullptr,
                                            (const int32_t*)nullptr, (int32_t*)nullptr, nnz, 0,
                                            end_bit, s);
    if (e != cudaSuccess) return e;
    const size_t temp_bytes = scan_bytes > sort_bytes ? scan_bytes : sort_bytes;
    // scratch: positions in, sorted keys (discarded), positions out, CUB temp
    char* pool = static_cast<char*>(tmp.alloc(3 * sizeof(int32_t) * (size_t)nnz + temp_bytes + 768));
    if (!pool) return cudaErrorMemoryAllocation;
    auto carve = [&](size_t bytes) {
        char* p = pool;
        pool += (bytes + 255) & ~(size_t)255;
        return p;
    };
    char* base = pool;
    int32_t* pos_in = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * nnz));
    uint32_t* keys_out = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * nnz));
    int32_t* pos_out = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * nnz));
    void* temp = carve(temp_bytes);
    size_t bytes = temp_bytes;
    e = cub::DeviceScan::InclusiveSum(temp, bytes, csc_ptr + 1, csc_ptr + 1, N, s);
    if (e == cudaSuccess) {
        iota_kernel<<<grid_for(nnz), 256, 0, s>>>(pos_in, nnz);
        e = cudaGetLastError();
    }
    bytes = temp_bytes;
    if (e == cudaSuccess)
        e = cub::DeviceRadixSort::SortPairs(temp, bytes, keys, keys_out, pos_in, pos_out, nnz, 0,
                                            end_bit, s);
    if (e == cudaSuccess) {
        csc_gather_kernel<<<grid_for(nnz), 256, 0, s>>>(pos_out, nnz, csr_ptr, M, csr_val,
                                                        csc_row, csc_val);
        e = cudaGetLastError();
    }
    const cudaError_t es = cudaStreamSynchronize(s);  // the scratch is returned below
    tmp.free(base);
    return e != cudaSuccess ? e : es;
}

namespace {

// *bad = 1 where a caller's column view (cp, ci, cv: raw values) differs from the built
// one (bp, bi, bv: values centred by rbar): the offsets, a row index, or a value once
// centred the way the built values were
__global__ void csc_compare_kernel(const int64_t* __restrict__ bp, const int32_t* __restrict__ bi,
                                   const float* __restrict__ bv, const int64_t* __restrict__ cp,
                                   const int32_t* __restrict__ ci, const float* __restrict__ cv,
                                   int64_t N, int64_t nnz, double rbar, unsigned int* bad)
{
    const int64_t n = nnz > N + 1 ? nnz : N + 1;
    bool diff = false;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e <= N && bp[e] != cp[e]) diff = true;
        if (e < nnz && (bi[e] != ci[e] || bv[e] != (float)((double)cv[e] - rbar))) diff = true;
    }
    if (diff) *bad = 1u;
}

}  // namespace

cudaError_t check_csc_device(const int64_t* built_ptr, const int32_t* built_row, const float* built_val,
                             const int64_t* csc_ptr, const int32_t* csc_row, const float* csc_val,
                             int64_t N, int64_t nnz, double rbar, const TempAlloc& tmp, bool* same,
                             cudaStream_t s)
{
    *same = false;
    const size_t ptr_bytes = ((sizeof(int64_t) * (size_t)(N + 1)) + 255) & ~(size_t)255;
    const size_t idx_bytes = ((sizeof(int32_t) * (size_t)nnz) + 255) & ~(size_t)255;
    char* pool = static_cast<char*>(tmp.alloc(ptr_bytes + 2 * idx_bytes + 256));
    if (!pool) return cudaErrorMemoryAllocation;
    int64_t* cp = reinterpret_cast<int64_t*>(pool);
    int32_t* ci = reinterpret_cast<int32_t*>(pool + ptr_bytes);
    float* cv = reinterpret_cast<float*>(pool + ptr_bytes + idx_bytes);
    unsigned int* bad = reinterpret_cast<unsigned int*>(pool + ptr_bytes + 2 * idx_bytes);
    unsigned int bad_h = 0;
    cudaError_t e = cudaMemcpyAsync(cp, csc_ptr, sizeof(int64_t) * (N + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nnz)
        e = cudaMemcpyAsync(ci, csc_row, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nnz)
        e = cudaMemcpyAsync(cv, csc_val, sizeof(float) * nnz, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        csc_compare_kernel<<<grid_for(nnz > N + 1 ? nnz : N + 1), 256, 0, s>>>(
            built_ptr, built_row, built_val, cp, ci, cv, N, nnz, rbar, bad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
    const cudaError_t es = cudaStreamSynchronize(s);  // the scratch is returned below
    tmp.free(pool);
    if (e == cudaSuccess) e = es;
    if (e == cudaSuccess) *same = bad_h == 0;
    return e;
}

}  // namespace bpmf
