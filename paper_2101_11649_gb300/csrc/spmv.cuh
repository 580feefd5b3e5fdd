// Row-product engines shared by the solve-phase translation units: the
// chunk engine (batched form and the handle-free BSR product), the SELL-C-sigma
// kernel with its launch shapes, and the gather and epilogue functors every
// cycle step is built from.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "sell.cuh"

namespace mgr {

#define GRIDN(n, t) (unsigned)((((long long)(n)) + (t)-1) / (t) > 0 ? (((long long)(n)) + (t)-1) / (t) : 1)

static const int NUM_SMS = 152;

// ----------------------------------------------------------- chunk engine
// A warp owns R consecutive rows (R a power of two, ~192 nonzeros per
// chunk).  Phase 1 stages the chunk's values and column indices in shared
// memory with CU independent coalesced loads per lane.  Phase 2 gives each
// row G = 32/R lanes; lane j of a group runs one fused multiply-add chain
// over a contiguous slice of its row, and the group combines its G partial
// sums with a fixed shuffle tree.  This keeps the FP64 work at one FMA per
// nonzero plus log2(G) adds per row (FP64 issue rate, not HBM, bounds FP64
// sparse products on this part).
constexpr int CCAP = 384;      // nonzeros a warp stages in shared memory
constexpr int CWARPS = 8;      // warps per block

static inline int rows_per_warp(long long nnz, int n) {
    double avg = n > 0 ? (double)nnz / n : 1.0;
    if (avg < 1.0) avg = 1.0;
    int r = 1;
    while (r < 32 && (r * 2) * avg <= 192.0) r *= 2;
    return r;
}

template <int G, class T>
__device__ __forceinline__ T group_tree(T s) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, G);
    return s;
}

template <int R, class T, class XF, class EPI>
__device__ __forceinline__ void chunk_rows(int r0, int r1, int p0, int cnt, const int *__restrict__ rp,
                                           const int *__restrict__ ci, const T *__restrict__ v,
                                           const XF &xf, const EPI &epi, T *sv, int *sc, int lane) {
    constexpr int G = 32 / R;
    // phase 1: stage values and columns
#pragma unroll
    for (int t = 0; t < CCAP / 32; t++) {
        const int q = lane + 32 * t;
        if (q < cnt) { sv[q] = __ldg(v + p0 + q); sc[q] = __ldg(ci + p0 + q); }
    }
    __syncwarp();
    // phase 2: G lanes per row, contiguous slices
    const int grp = lane / G, j = lane % G;
    const int row = r0 + grp;
    T s = (T)0;
    if (row < r1) {
        const int a = __ldg(rp + row) - p0, b = __ldg(rp + row + 1) - p0;
        const int len = b - a, Lr = (len + G - 1) / G;
        const int q0 = a + j * Lr, q1 = min(q0 + Lr, b);
        for (int q = q0; q < q1; q++) s = fma(sv[q], xf(sc[q]), s);
    }
    s = group_tree<G, T>(s);
    if (row < r1 && j == 0) epi(row, s);
    __syncwarp();
}

template <int R, class T, class XF, class EPI>
__global__ void __launch_bounds__(CWARPS * 32) k_csr_chunk(int n, const int *__restrict__ rp,
                                                           const int *__restrict__ ci,
                                                           const T *__restrict__ v, XF xf, EPI epi) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ T sv[CWARPS][CCAP];
    __shared__ int sc[CWARPS][CCAP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchunk = (n + R - 1) / R;
    for (int c = blockIdx.x * CWARPS + warp; c < nchunk; c += gridDim.x * CWARPS) {
        const int r0 = c * R, r1 = min(r0 + R, n);
        const int p0 = __ldg(rp + r0), p1 = __ldg(rp + r1);
        const int cnt = p1 - p0;
        if (cnt <= CCAP) {
            chunk_rows<R, T, XF, EPI>(r0, r1, p0, cnt, rp, ci, v, xf, epi, sv[warp], sc[warp], lane);
        } else {
            for (int row = r0; row < r1; row++) {
                const int a = __ldg(rp + row), b = __ldg(rp + row + 1);
                T s = (T)0;
                for (int p = a + lane; p < b; p += 32) s = fma(__ldg(v + p), xf(__ldg(ci + p)), s);
                s = group_tree<32, T>(s);
                if (lane == 0) epi(row, s);
            }
        }
    }
}

template <class T, class XF, class EPI>
static void csr_chunk(int n, long long nnz, const int *rp, const int *ci, const T *v, XF xf, EPI epi,
                      cudaStream_t s) {
    if (n <= 0) return;
    int R = rows_per_warp(nnz, n);
    long long nchunk = (n + R - 1) / R;
    long long blocks = (nchunk + CWARPS - 1) / CWARPS;
    if (blocks > NUM_SMS * 8) blocks = NUM_SMS * 8;
    if (blocks < 1) blocks = 1;
    unsigned g = (unsigned)blocks;
    switch (R) {
        case 1: launch_k(k_csr_chunk<1, T, XF, EPI>, dim3(g), dim3(CWARPS * 32), s, n, rp, ci, v, xf, epi); break;
        case 2: launch_k(k_csr_chunk<2, T, XF, EPI>, dim3(g), dim3(CWARPS * 32), s, n, rp, ci, v, xf, epi); break;
        case 4: launch_k(k_csr_chunk<4, T, XF, EPI>, dim3(g), dim3(CWARPS * 32), s, n, rp, ci, v, xf, epi); break;
        case 8: launch_k(k_csr_chunk<8, T, XF, EPI>, dim3(g), dim3(CWARPS * 32), s, n, rp, ci, v, xf, epi); break;
        case 16: launch_k(k_csr_chunk<16, T, XF, EPI>, dim3(g), dim3(CWARPS * 32), s, n, rp, ci, v, xf, epi); break;
        default: launch_k(k_csr_chunk<32, T, XF, EPI>, dim3(g), dim3(CWARPS * 32), s, n, rp, ci, v, xf, epi); break;
    }
}

// ---------------------------------------------------------- SELL-C-sigma
// k_sell: one warp per slice (layout and row sums in sell.cuh); FP32 (PF)
// starts a slice's epilogue loads and the next slice's offsets before the
// slice's products.  Slices reach the warps in one of two orders, chosen per
// matrix at setup by timing both (DCSR::sched): grid-stride over all slices
// (CONTIG = 0), or a contiguous range of slices per block whose warps
// interleave inside it (CONTIG = 1), so that the warps of an SM gather from
// neighbouring rows and L1 keeps the vector lines they share (a structured
// stencil's neighbouring grid lines).  Every row's sum is the same either way,
// and with the pipelined chain (PIPE, FP64; sell.cuh).
template <int G, class T, class XF, class EPI, int CONTIG, int PIPE>
__global__ void __launch_bounds__(256, PIPE ? SELL_BLOCKS_PIPE : SELL_BLOCKS)
    k_sell(int nsl, const long long *__restrict__ sptr, const int *__restrict__ slen,
           const int *__restrict__ perm, const int *__restrict__ sci, const T *__restrict__ sv, XF xf,
           EPI epi) {
    constexpr int PF = SellCfg<T>::PF, BP = SellCfg<T>::BP;
    constexpr int C = 32 / G;
    const int lane = threadIdx.x & 31;
    int nw, sl;
    if (CONTIG) {
        const int per = (nsl + gridDim.x - 1) / gridDim.x;
        const int s0 = blockIdx.x * per;
        nsl = min(nsl, s0 + per);
        nw = blockDim.x >> 5;
        sl = s0 + (threadIdx.x >> 5);
    } else {
        nw = (gridDim.x * blockDim.x) >> 5;
        sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    }
    if (sl >= nsl) return;
    if (BP) {
        // the next slice's header two slices ahead, so that its values and
        // columns can be prefetched to L2 (one bulk request each, from lane
        // 0) while this slice is summed
        int L = __ldg(slen + sl);
        long long base = __ldg(sptr + sl) + lane;
        int row = __ldg(perm + (long long)sl * C + lane / G);
        int nx = sl + nw, L2 = 0, row2 = -1;
        long long s2 = 0;
        if (nx < nsl) {
            L2 = __ldg(slen + nx);
            s2 = __ldg(sptr + nx);
            row2 = __ldg(perm + (long long)nx * C + lane / G);
        }
        pdl_wait();  // slice offsets and rows above are read-only
        pdl_launch_dependents();
        for (;;) {
            const bool own = (lane % G == 0) && row >= 0;
            typename EPI::Pre pre{};
            if (own) pre = epi.pre(row);
            const int nx2 = nx + nw;
            int L3 = 0, row3 = -1;
            long long s3 = 0;
            if (nx2 < nsl) {
                L3 = __ldg(slen + nx2);
                s3 = __ldg(sptr + nx2);
                row3 = __ldg(perm + (long long)nx2 * C + lane / G);
            }
            if (lane == 0 && nx < nsl && L2 > 0) {
                prefetch_l2(sv + s2, (unsigned)(L2 * 32 * (int)sizeof(T)));
                prefetch_l2(sci + s2, (unsigned)(L2 * 32 * 4));
            }
            const T acc = sell_rows<G, T>(L, base, sci, sv, xf);
            if (own) epi.put(row, acc, pre);
            if (nx >= nsl) break;
            sl = nx; L = L2; base = s2 + lane; row = row2;
            nx = nx2; L2 = L3; s2 = s3; row2 = row3;
        }
        return;
    }
    int L = __ldg(slen + sl);
    long long base = __ldg(sptr + sl) + lane;
    int row = __ldg(perm + (long long)sl * C + lane / G);
    pdl_wait();  // slice offsets and rows above are read-only
    pdl_launch_dependents();
    for (;;) {
        const bool own = (lane % G == 0) && row >= 0;
        typename EPI::Pre pre{};
        if (PF && own) pre = epi.pre(row);
        const int nx = sl + nw;
        int L2 = 0, row2 = -1;
        long long base2 = 0;
        if (PF && nx < nsl) {
            L2 = __ldg(slen + nx);
            base2 = __ldg(sptr + nx) + lane;
            row2 = __ldg(perm + (long long)nx * C + lane / G);
        }
        const T acc = sell_rows<G, T, XF, PIPE>(L, base, sci, sv, xf);
        if (own) epi.put(row, acc, PF ? pre : epi.pre(row));
        if (nx >= nsl) break;
        sl = nx;
        if (PF) {
            L = L2; base = base2; row = row2;
        } else {
            L = __ldg(slen + sl);
            base = __ldg(sptr + sl) + lane;
            row = __ldg(perm + (long long)sl * C + lane / G);
        }
    }
}

// grid: two waves of resident blocks for the grid-stride order, one for the
// contiguous order (each block's range is its whole share)
template <int G, class T, class XF, class EPI>
static void sell_launch(const DCSR &M, const T *vals, XF xf, EPI epi, cudaStream_t s) {
    const int contig = M.sched & 1;
    const bool pipe = sizeof(T) == 8 && (M.sched & 2);
    long long blocks = ((long long)M.nsl * 32 + 255) / 256;
    const long long cap = (long long)NUM_SMS * (pipe ? SELL_BLOCKS_PIPE : SELL_BLOCKS) * (contig ? 1 : 2);
    if (blocks > cap) blocks = cap;
    const dim3 grid((unsigned)(blocks < 1 ? 1 : blocks));
#define SELL_GO(C, P) \
    launch_k(k_sell<G, T, XF, EPI, C, P>, grid, dim3(256), s, M.nsl, M.sptr, M.slen, M.perm, M.sci, vals, xf, epi)
    if constexpr (sizeof(T) == 8) {
        if (pipe) {
            if (contig) SELL_GO(1, 1);
            else SELL_GO(0, 1);
            return;
        }
    }
    if (contig) SELL_GO(1, 0);
    else SELL_GO(0, 0);
#undef SELL_GO
}

// Row products over a matrix: SELL-C-sigma when built, else the chunk engine.
template <class T, class XF, class EPI>
static void spmv_rows(const DCSR &M, const T *csr_vals, XF xf, EPI epi, cudaStream_t s) {
    if (M.n <= 0) return;
    const T *sv = sell_vals<T>(M);
    if (M.sptr && sv) {
        switch (M.sg) {
            case 1: sell_launch<1, T>(M, sv, xf, epi, s); break;
            case 2: sell_launch<2, T>(M, sv, xf, epi, s); break;
            case 4: sell_launch<4, T>(M, sv, xf, epi, s); break;
            case 8: sell_launch<8, T>(M, sv, xf, epi, s); break;
            case 16: sell_launch<16, T>(M, sv, xf, epi, s); break;
            default: sell_launch<32, T>(M, sv, xf, epi, s); break;
        }
        return;
    }
    csr_chunk<T>(M.n, M.nnz, M.rp, M.ci, csr_vals, xf, epi, s);
}

// gathers
template <class T, class XT>
struct XPlain {
    const XT *x;
    __device__ __forceinline__ T operator()(int j) const { return (T)__ldg(x + j); }
};

// epilogues.  pre(row) issues the loads an epilogue needs from its row
// alone (so the SELL kernel can start them before the row's products);
// put(row, s, p) finishes the row.  Every row is finished by one lane and
// no epilogue reads what another row writes.
#define EPI_CALL \
    __device__ __forceinline__ void operator()(int row, T s) const { put(row, s, pre(row)); }
struct PreNone {};
template <class T, class TO>
struct EStore {
    TO *y;
    using Pre = PreNone;
    __device__ __forceinline__ Pre pre(int) const { return {}; }
    __device__ __forceinline__ void put(int row, T s, const Pre &) const { y[row] = (TO)s; }
    EPI_CALL
};
template <class T>
struct EAdd {
    T *y;
    struct Pre { T y; };
    __device__ __forceinline__ Pre pre(int row) const { return {y[row]}; }
    __device__ __forceinline__ void put(int row, T s, const Pre &p) const { y[row] = p.y + s; }
    EPI_CALL
};
struct EAxpby {
    double alpha, beta;
    const double *b;  // residual mode when non-null: y = b - s
    double *y;
    using T = double;
    struct Pre { double u; };
    __device__ __forceinline__ Pre pre(int row) const {
        return {b ? b[row] : (beta == 0.0 ? 0.0 : y[row])};
    }
    __device__ __forceinline__ void put(int row, double s, const Pre &p) const {
        if (b) y[row] = p.u - s;
        else y[row] = beta == 0.0 ? alpha * s : alpha * s + beta * p.u;
    }
    EPI_CALL
};
template <class T>
struct EStoreScaled {  // y = s ; x = d s  (restriction that also seeds the next pre-smoothing)
    T *y;
    const T *d;
    T *x;
    struct Pre { T d; };
    __device__ __forceinline__ Pre pre(int row) const { return {d[row]}; }
    __device__ __forceinline__ void put(int row, T s, const Pre &p) const {
        y[row] = s;
        x[row] = p.d * s;
    }
    EPI_CALL
};
template <class T, class TV>
struct EGatherMinusScaled {  // y = b[idx] - s ; x = d y
    const int *idx;
    const TV *b;
    T *y;
    const T *d;
    T *x;
    struct Pre { T b, d; };
    __device__ __forceinline__ Pre pre(int row) const { return {(T)b[idx[row]], d[row]}; }
    __device__ __forceinline__ void put(int row, T s, const Pre &p) const {
        T t = p.b - s;
        y[row] = t;
        x[row] = p.d * t;
    }
    EPI_CALL
};
template <class T, class TV>
struct EResid {  // res = r - s
    const TV *r;
    T *res;
    struct Pre { T r; };
    __device__ __forceinline__ Pre pre(int row) const { return {(T)r[row]}; }
    __device__ __forceinline__ void put(int row, T s, const Pre &p) const { res[row] = p.r - s; }
    EPI_CALL
};
template <class T, class TV>
struct EPost {  // xout = x + d (r - A x)
    const TV *r;
    const T *d;
    const T *x;
    TV *xout;
    struct Pre { T r, d, x; };
    __device__ __forceinline__ Pre pre(int row) const { return {(T)r[row], d[row], x[row]}; }
    __device__ __forceinline__ void put(int row, T s, const Pre &p) const {
        xout[row] = (TV)fma(p.d, p.r - s, p.x);
    }
    EPI_CALL
};
template <class T, class TV>
struct EGatherMinus {  // y = b[idx[row]] + sign * s
    const int *idx;
    const TV *b;
    T sign;
    T *y;
    struct Pre { T b; };
    __device__ __forceinline__ Pre pre(int row) const { return {(T)b[idx[row]]}; }
    __device__ __forceinline__ void put(int row, T s, const Pre &p) const { y[row] = p.b + sign * s; }
    EPI_CALL
};
template <class T, class TV>
struct EInterp {  // z[fidx] = zF + s
    const int *fidx;
    const T *zF;
    TV *z;
    struct Pre { int f; T zF; };
    __device__ __forceinline__ Pre pre(int row) const { return {fidx[row], zF[row]}; }
    __device__ __forceinline__ void put(int, T s, const Pre &p) const { z[p.f] = (TV)(p.zF + s); }
    EPI_CALL
};
#undef EPI_CALL

}  // namespace mgr
