// Residual and residual norm without any device allocation.
//
// Some callers cannot call cudaMalloc when they need a residual check:
// plug-ins whose host application owns all device memory through its own
// pool and forbids allocations behind its back, and latency-critical loops
// that must never enter the allocator (a cudaMalloc can block on the device
// or fail when memory is exhausted).  This entry point serves them: the
// caller passes the matrix, the vectors and the outputs, and the only
// scratch the reduction needs (one partial sum per block and the ticket that
// elects the last block) lives in the file-scope static device array below.
//
// The array holds MGR_NOALLOC_MAX_BLOCKS partial sums plus one slot for the
// ticket: 32 KiB, held by every GPU that loads this library until the process
// exits.  One block reduces NOALLOC_SPAN consecutive entries, so n = nb * b
// may be at most MGR_NOALLOC_MAX_BLOCKS * NOALLOC_SPAN = 16,777,216.
//
// Host code cannot use the array's name as a device address: on the host the
// symbol is a stand-in, and a kernel handed it would fault (or, where the GPU
// can reach host memory, silently use the wrong memory).  The first call on
// each device therefore looks the device address up with
// cudaGetSymbolAddress, with that device current, and caches it; that first
// call should come before any stream capture.  Every call shares the array
// and overwrites the previous contents: the ticket is cleared at the start of
// each call, every partial is rewritten, and calls that overlap on the GPU
// (different streams, different host threads) race on it.
#include <cuda_runtime.h>
#include <stdio.h>

#include <mutex>

#include "../../include/mgr_gb300.h"
#include "common.cuh"

namespace {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_SPAN = 4096;  // entries reduced by one block

static __device__ __align__(256) double g_noalloc_scratch[MGR_NOALLOC_MAX_BLOCKS + 1];

std::mutex g_mtx;
double *g_addr[64] = {};

// Block b sums r[i]^2 for i in [b*SPAN, (b+1)*SPAN) into partial[b]; the last
// block to finish (ticket) adds the partials in block order and writes the
// square root.  Fixed order: repeated calls give identical bits.
__global__ void __launch_bounds__(NOALLOC_THREADS) k_norm_static(const double *r, long long n,
                                                                 double *scratch, int nblocks,
                                                                 double *norm_out) {
    unsigned *ticket = reinterpret_cast<unsigned *>(scratch + MGR_NOALLOC_MAX_BLOCKS);
    __shared__ double sh[NOALLOC_THREADS / 32];
    __shared__ bool last;
    const long long base = (long long)blockIdx.x * NOALLOC_SPAN;
    double s = 0.0;
    for (int t = threadIdx.x; t < NOALLOC_SPAN; t += NOALLOC_THREADS) {
        long long i = base + t;
        if (i < n) s += r[i] * r[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NOALLOC_THREADS / 32; w++) t += sh[w];
        scratch[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)(nblocks - 1);
    }
    __syncthreads();
    if (last && threadIdx.x < 32) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += 32) t += __ldcg(scratch + b);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) *norm_out = sqrt(t);
    }
}

}  // namespace

extern "C" mgr_status mgr_residual_norm_noalloc(int32_t nb, int32_t b, const int32_t *row_ptr,
                                                const int32_t *col_idx, const double *val,
                                                const double *x, const double *bvec, double *r,
                                                double *norm_out, void *stream) {
    if (b < 1 || b > 4 || nb < 1 || !row_ptr || !col_idx || !val || !x || !bvec || !r || !norm_out)
        return MGR_ERR_INVALID;
    const long long n = (long long)nb * b;
    const long long nblocks = (n + NOALLOC_SPAN - 1) / NOALLOC_SPAN;
    if (nblocks > MGR_NOALLOC_MAX_BLOCKS) return MGR_ERR_UNSUPPORTED;  // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MGR_ERR_CUDA;
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mtx);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return MGR_ERR_CUDA;
            }
            g_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the ticket must start at zero
    if (cudaMemsetAsync(scratch + MGR_NOALLOC_MAX_BLOCKS, 0, sizeof(double), s) != cudaSuccess)
        return MGR_ERR_CUDA;
    mgr::launch_bsr_residual(nb, b, row_ptr, col_idx, val, x, bvec, r, s);
    k_norm_static<<<(unsigned)nblocks, NOALLOC_THREADS, 0, s>>>(r, n, scratch, (int)nblocks, norm_out);
    return cudaGetLastError() == cudaSuccess ? MGR_OK : MGR_ERR_CUDA;
}
