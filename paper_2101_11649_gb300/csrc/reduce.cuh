// Fixed-order reductions shared by the Krylov kernels and their batched
// forms: each block accumulates a fixed element set, writes its partial, and
// the last block to finish (ticket) sums the partials in block order, one
// warp per output.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "spmv.cuh"

namespace mgr {

static const int RED_THREADS = 256;
static const int RED_EPT = 2;

__host__ __device__ constexpr int pow2_at_least(int k) { return k <= 1 ? 1 : 2 * pow2_at_least((k + 1) / 2); }
__host__ __device__ constexpr int log2_of(int p) { return p <= 1 ? 0 : 1 + log2_of(p / 2); }

// Warp sum of K values per lane by recursive halving: at the level with
// lane distance o, a lane keeps half of its values and adds the partner's
// copies of them, so after log2 K' levels (K' = K rounded up to a power of
// two) each lane holds one partial sum, of value index lane >> (5 - log2 K'),
// and plain shuffle levels finish it.  K' - 1 + 5 - log2 K' adds per lane
// instead of 5 K; the order is fixed, so results are reproducible.
template <int K>
__device__ __forceinline__ double warp_sum_many(const double (&acc)[K], int lane, int &index) {
    constexpr int KP = pow2_at_least(K);
    constexpr int LK = log2_of(KP);
    static_assert(KP <= 32, "at most 32 values");
    double v[KP];
#pragma unroll
    for (int i = 0; i < KP; i++) v[i] = i < K ? acc[i] : 0.0;
#pragma unroll
    for (int lev = 0; lev < LK; lev++) {
        const int o = 16 >> lev, m = KP >> (lev + 1);
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < m; i++) {
            const double send = upper ? v[i] : v[i + m];
            const double keep = upper ? v[i + m] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    double t = v[0];
#pragma unroll
    for (int o = (16 >> LK); o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    index = lane >> (5 - LK);
    return t;
}

template <int K>
__device__ __forceinline__ void block_partials(double (&acc)[K], double *partial) {
    __shared__ double sh[RED_THREADS / 32][K > 0 ? K : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int LK = log2_of(pow2_at_least(K));
    int idx;
    const double t0 = warp_sum_many<K>(acc, lane, idx);
    if ((lane & ((1 << (5 - LK)) - 1)) == 0 && idx < K) sh[w][idx] = t0;
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
#pragma unroll
        for (int ww = 0; ww < RED_THREADS / 32; ww++) t += sh[ww][threadIdx.x];
        partial[(long long)blockIdx.x * K + threadIdx.x] = t;
    }
}

// true in the last block to arrive (all partials visible to it)
__device__ __forceinline__ bool last_block(unsigned *ticket) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    return am_last;
}

// out[i] = sum over blocks of partial[b*K + i], warp per output, fixed tree
template <int K>
__device__ __forceinline__ void sum_partials(const double *partial, double *out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = w; i < K; i += RED_THREADS / 32) {
        double t = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(partial + (long long)b * K + i);
        t = group_sum<32, double>(t);
        if (lane == 0) out[i] = t;
    }
}

// Classical Gram-Schmidt with a rescue pass: the second projection runs
// only when the first removed more than 99% of |w| (|w'| < 0.1 |w|), the
// cancellation that costs orthogonality (a DGKS-type test with eta = 0.1).
static constexpr double REORTH_ETA2 = 1e-2;

#define K_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) \
    X(15) X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) \
    X(30) X(31) X(32)

}  // namespace mgr
