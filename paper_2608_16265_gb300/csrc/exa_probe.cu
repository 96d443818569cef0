// exa_probe.cu -- FP64 FMA throughput probe (include/exa_probe.h).
//
// Every thread runs EXA_PROBE_CHAINS independent chains a <- fma(a, b, c); within a chain each FMA
// depends on the previous one, so the compiler can neither fold nor reorder them, and the chains
// give the scheduler enough independent FMAs to keep the FP64 pipe full.  b is just below one and
// c tiny, so the values stay bounded and normal.  The result is stored only if it equals an
// impossible value, which keeps the chains live without any memory traffic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "../../include/exa_probe.h"

namespace {

#define EXA_PROBE_CHAINS 8
#define EXA_PROBE_UNROLL 16

__global__ void __launch_bounds__(256) k_dfma_chains(int iters, double b, double c, double *sink) {
    double a[EXA_PROBE_CHAINS];
#pragma unroll
    for (int j = 0; j < EXA_PROBE_CHAINS; j++) a[j] = 1.0 + 1e-3 * (threadIdx.x + 37 * j);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < EXA_PROBE_UNROLL; u++)
#pragma unroll
            for (int j = 0; j < EXA_PROBE_CHAINS; j++) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < EXA_PROBE_CHAINS; j++) s += a[j];
    if (s == -1.0) sink[0] = s;
}

}  // namespace

extern "C" exa_status exa_probe_fp64_fma(int32_t device, double target_ms, double *inst_per_s, double *ms,
                                         int32_t *sms_out) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return EXA_E_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return EXA_E_CUDA;
    target_ms = std::min(2000.0, std::max(10.0, target_ms));
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return EXA_E_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dfma_chains, 256, 0) != cudaSuccess) return EXA_E_CUDA;
    const int blocks = sms * std::max(occ, 1);
    double *sink = nullptr;
    if (cudaMalloc((void **)&sink, sizeof(double)) != cudaSuccess) return EXA_E_CUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    exa_status st = EXA_OK;
    float t = 0.0f;
    int iters = 64;
    auto timed = [&](int it) -> bool {
        if (cudaEventRecord(e0) != cudaSuccess) return false;
        k_dfma_chains<<<blocks, 256>>>(it, 0.9999999999999, 1e-13, sink);
        if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1) != cudaSuccess) return false;
        if (cudaEventSynchronize(e1) != cudaSuccess) return false;
        return cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess || !timed(iters)) {
        st = EXA_E_CUDA;
    } else {
        // grow the work until one launch takes a tenth of the target, then size it to the target
        while (t < 0.1f * (float)target_ms && iters < (1 << 24)) {
            iters *= 4;
            if (!timed(iters)) { st = EXA_E_CUDA; break; }
        }
        if (st == EXA_OK) {
            iters = (int)std::min<double>(1 << 26, std::max(1.0, iters * target_ms / std::max(t, 1e-3f)));
            if (!timed(iters)) st = EXA_E_CUDA;
        }
    }
    if (st == EXA_OK) {
        const double n = (double)blocks * 256.0 * (double)iters * EXA_PROBE_UNROLL * EXA_PROBE_CHAINS;
        if (inst_per_s) *inst_per_s = n / (t * 1e-3);
        if (ms) *ms = t;
        if (sms_out) *sms_out = sms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}

extern "C" exa_status exa_probe_host_link(int32_t device, int64_t bytes, double *h2d_bytes_per_s,
                                          double *d2h_bytes_per_s) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return EXA_E_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return EXA_E_CUDA;
    bytes = std::min<int64_t>(4LL << 30, std::max<int64_t>(64LL << 20, bytes));
    void *h = nullptr, *d = nullptr;
    if (cudaHostAlloc(&h, (size_t)bytes, cudaHostAllocDefault) != cudaSuccess) return EXA_E_OOM;
    if (cudaMalloc(&d, (size_t)bytes) != cudaSuccess) {
        cudaFreeHost(h);
        return EXA_E_OOM;
    }
    std::memset(h, 0, (size_t)bytes);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    exa_status st = EXA_OK;
    double best[2] = {0.0, 0.0};
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = EXA_E_CUDA;
    for (int dir = 0; dir < 2 && st == EXA_OK; dir++) {
        void *dst = dir == 0 ? d : h;
        const void *src = dir == 0 ? h : d;
        const cudaMemcpyKind kind = dir == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
        for (int r = 0; r < 4 && st == EXA_OK; r++) {  // the first copy warms up
            float t = 0.0f;
            if (cudaEventRecord(e0) != cudaSuccess || cudaMemcpyAsync(dst, src, (size_t)bytes, kind, 0) != cudaSuccess ||
                cudaEventRecord(e1) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                st = EXA_E_CUDA;
                break;
            }
            if (r > 0 && t > 0.0f) best[dir] = std::max(best[dir], (double)bytes / (t * 1e-3));
        }
    }
    if (st == EXA_OK) {
        if (h2d_bytes_per_s) *h2d_bytes_per_s = best[0];
        if (d2h_bytes_per_s) *d2h_bytes_per_s = best[1];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    cudaFreeHost(h);
    return st;
}
