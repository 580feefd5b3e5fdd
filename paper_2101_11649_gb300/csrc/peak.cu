// Measured FP64 fused-multiply-add throughput of the current device, the
// denominator of the FP64-pipe roofline of the solve-phase kernels (their
// products issue one FMA per stored entry).  Every thread runs CHAINS
// independent FMA recurrences in registers; the grid fills every SM to its
// occupancy limit, so the FP64 pipes, not latency, bound the launch.
#include <cuda_runtime.h>

#include "../../include/mgr_gb300.h"
#include "common.cuh"

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int CHAINS = 8;

__device__ double g_fma_sink;

__global__ void __launch_bounds__(PEAK_THREADS) k_fma_chains(int iters, double m, double c) {
    double a[CHAINS];
#pragma unroll
    for (int q = 0; q < CHAINS; q++) a[q] = 1.0 + 1e-3 * q + 1e-9 * threadIdx.x;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int q = 0; q < CHAINS; q++) a[q] = fma(a[q], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < CHAINS; q++) s += a[q];
    // keeps the chains live; the recurrences stay near 1, so this never stores
    if (s == 12345.678) g_fma_sink = s;
}

}  // namespace

extern "C" mgr_status mgr_measure_fp64_fma(void *stream, int32_t reps, double *fma_per_s) {
    if (!fma_per_s || reps < 1) return MGR_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains, PEAK_THREADS, 0) !=
            cudaSuccess)
        return MGR_ERR_CUDA;
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 2048;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return MGR_ERR_CUDA;
    float best = 0.f;
    for (int r = 0; r <= reps; r++) {  // the first launch warms up, untimed
        cudaEventRecord(e0, s);
        k_fma_chains<<<grid, PEAK_THREADS, 0, s>>>(iters, 0.9999999, 1e-7);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess || best <= 0.f) return MGR_ERR_CUDA;
    const double fmas = (double)grid * PEAK_THREADS * CHAINS * iters;
    *fma_per_s = fmas / (best * 1e-3);
    return MGR_OK;
}
