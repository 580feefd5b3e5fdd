// SELL-C-sigma row products shared by the solve-phase kernels (spmv.cuh)
// and the fused coarse-level kernel (tail.cu): one routine, so a row's sum
// has the same operation order, and the same bits, wherever it is formed.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace mgr {

template <int G, class T>
__device__ __forceinline__ T group_sum(T s) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
    return s;
}

// ---------------------------------------------------------- SELL-C-sigma
// One warp per slice of C = 32/G rows, G lanes per row.  Each step of the
// slice is 32 contiguous entries (coalesced value and column loads); a lane
// runs one FMA chain over its entries t*G + g and the row's G partial sums
// meet in a fixed shuffle tree.  The slice width L is warp-uniform, so each
// round issues U independent value/column loads, then U gathers, then U
// FMAs without divergence: the longest slice costs ceil(L/U) dependent
// load-gather rounds.  Padding entries carry zero values and a column of
// the same row.
//
// Per precision (fitted to GB300 timings of every AMG level's products):
// FP64 issues U = 4 loads per round and loads the epilogue's row values
// after the products, so registers go to more resident warps; FP32 issues
// U = 8 and (PF) starts the epilogue's row loads and the next slice's
// offsets before the products, so they overlap them.  Both stay within 48
// registers (5 blocks, 40 warps per SM).
template <class T>
struct SellCfg { static constexpr int U = 4, PF = 0, BP = 0; };
template <>
struct SellCfg<float> { static constexpr int U = 6, PF = 1, BP = 1; };

// one bulk request that brings [p, p + bytes) into L2 (16-byte aligned
// address, size a multiple of 16; no completion to wait for)
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
constexpr int SELL_BLOCKS = 5;

template <class T>
__host__ __device__ inline const T *sell_vals(const DCSR &M);
template <>
inline const double *sell_vals<double>(const DCSR &M) { return M.sv; }
template <>
inline const float *sell_vals<float>(const DCSR &M) { return M.sv32; }


// Loads of the matrix stream (values and column indices, each read once per
// product) bypass L1 allocation, so L1 keeps the lines of the gathered
// vector, which neighbouring rows reuse.  Measured on GB300: 3-7% shorter
// V-cycles than plain read-only loads, the same bits.
__device__ __forceinline__ float ld_stream(const float *p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_stream(const double *p) {
    double v;
    asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_stream(const int *p) {
    int v;
    asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// The calling lane's share of a slice row: lane r*G + g runs the FMA chain
// over the row's entries t*G + g, t ascending, U loads in flight per round.
// The chain does not depend on G (the layout places the entries).
template <class T, class XF>
__device__ __forceinline__ T sell_chain(int L, long long base, const int *__restrict__ sci,
                                        const T *__restrict__ sv, const XF &xf) {
    constexpr int U = SellCfg<T>::U;
    T acc = (T)0;
    for (int t = 0; t < L; t += U) {
        T vv[U], xx[U];
        int cc[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (t + u < L) {
                const long long o = base + (long long)(t + u) * 32;
                vv[u] = ld_stream(sv + o);
                cc[u] = ld_stream(sci + o);
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (t + u < L) xx[u] = xf(cc[u]);
#pragma unroll
        for (int u = 0; u < U; u++)
            if (t + u < L) acc = fma(vv[u], xx[u], acc);
    }
    return acc;
}

// The same chain with the next round's values and columns loaded before
// this round's FMAs, so that the loads overlap the FMAs (the FMA order, and
// so the bits, are those of sell_chain).  It holds one more round of values
// and columns in registers (64 per thread for FP64, SELL_BLOCKS_PIPE blocks
// per SM).  On GB300 it shortens the FP64 products of long rows, where the
// FP64 FMAs and the loads would otherwise take turns, and lengthens those of
// short rows (fewer resident warps, nothing to overlap): the setup times both
// per matrix (DCSR::sched bit 1).
constexpr int SELL_BLOCKS_PIPE = 4;
template <class T, class XF>
__device__ __forceinline__ T sell_chain_pipe(int L, long long base, const int *__restrict__ sci,
                                             const T *__restrict__ sv, const XF &xf) {
    constexpr int U = SellCfg<T>::U;
    T acc = (T)0, vv[U];
    int cc[U];
#pragma unroll
    for (int u = 0; u < U; u++)
        if (u < L) {
            const long long o = base + (long long)u * 32;
            vv[u] = ld_stream(sv + o);
            cc[u] = ld_stream(sci + o);
        }
    for (int t = 0; t < L; t += U) {
        T xx[U], vn[U];
        int cn[U];
#pragma unroll
        for (int u = 0; u < U; u++)
            if (t + u < L) xx[u] = xf(cc[u]);
#pragma unroll
        for (int u = 0; u < U; u++)
            if (t + U + u < L) {
                const long long o = base + (long long)(t + U + u) * 32;
                vn[u] = ld_stream(sv + o);
                cn[u] = ld_stream(sci + o);
            }
#pragma unroll
        for (int u = 0; u < U; u++)
            if (t + u < L) acc = fma(vv[u], xx[u], acc);
#pragma unroll
        for (int u = 0; u < U; u++) {
            vv[u] = vn[u];
            cc[u] = cn[u];
        }
    }
    return acc;
}

// The G partial sums of a row meet in a fixed shuffle tree (lane distances
// G/2, G/4, .., 1); every lane of the group ends with the row's sum.  The
// run-time-G form performs the same additions in the same order.
template <int G, class T, class XF, int PIPE = 0>
__device__ __forceinline__ T sell_rows(int L, long long base, const int *__restrict__ sci,
                                       const T *__restrict__ sv, const XF &xf) {
    T acc;
    if constexpr (PIPE) acc = sell_chain_pipe<T>(L, base, sci, sv, xf);
    else acc = sell_chain<T>(L, base, sci, sv, xf);
    if (G > 1) acc = group_sum<G, T>(acc);
    return acc;
}

template <class T>
__device__ __forceinline__ T group_sum_rt(T s, int G) {
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
    return s;
}

}  // namespace mgr
