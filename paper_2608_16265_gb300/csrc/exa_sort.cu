// exa_sort.cu -- setup-time device sorts and scans (CUB), used only by exa_create.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <cstdint>

// Stable sort of (key, value) pairs by key over bits [0, end_bit).
cudaError_t exa_sort_pairs_u64(const unsigned long long *kin, unsigned long long *kout, const int *vin,
                               int *vout, int n, int end_bit, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    size_t bytes = 0;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, bytes, kin, kout, vin, vout, n, 0, end_bit, s);
    if (e != cudaSuccess) return e;
    void *tmp = nullptr;
    e = cudaMalloc(&tmp, bytes);
    if (e != cudaSuccess) return e;
    e = cub::DeviceRadixSort::SortPairs(tmp, bytes, kin, kout, vin, vout, n, 0, end_bit, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(tmp);
    return e != cudaSuccess ? e : e2;
}

// out[i] = in[0] + ... + in[i]
cudaError_t exa_inclusive_sum_i32(const int *in, int *out, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    size_t bytes = 0;
    cudaError_t e = cub::DeviceScan::InclusiveSum(nullptr, bytes, in, out, n, s);
    if (e != cudaSuccess) return e;
    void *tmp = nullptr;
    e = cudaMalloc(&tmp, bytes);
    if (e != cudaSuccess) return e;
    e = cub::DeviceScan::InclusiveSum(tmp, bytes, in, out, n, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(tmp);
    return e != cudaSuccess ? e : e2;
}
