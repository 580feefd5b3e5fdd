// Solve-phase cycle steps: the outer operator product (SELL-C-sigma for
// b = 1, one thread per scalar row of a block row for b = 2..4), the MGR
// level steps (F-relaxation, injection restriction, interpolation) and the
// AMG level steps (residual, restriction, prolongation, post-smoothing,
// coarsest dense solve).  Each step is one pass over its matrix with a gather
// functor and a fused epilogue (spmv.cuh); every reduction has a fixed
// order, so repeated runs give identical bits.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include "common.cuh"
#include "sell.cuh"
#include "spmv.cuh"

namespace mgr {

bool pdl_on() {
    static const bool on = [] {
        const char *e = getenv("MGR_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

// --------------------------------------------------------------- CSR y = A x
template <class T>
void launch_csr_spmv(const DCSR &A, const T *vals, const T *x, T *y, cudaStream_t s) {
    spmv_rows<T>(A, vals, XPlain<T, T>{x}, EStore<T, T>{y}, s);
}

template <class T>
void launch_csr_spmv_add(const DCSR &A, const T *vals, const T *x, T *y, cudaStream_t s) {
    spmv_rows<T>(A, vals, XPlain<T, T>{x}, EAdd<T>{y}, s);
}

void launch_csr_residual(const DCSR &A, const double *x, const double *bvec, double *y,
                         cudaStream_t s) {
    spmv_rows<double>(A, A.v, XPlain<double, double>{x}, EAxpby{1.0, 0.0, bvec, y}, s);
}

// -------------------------------------------------------------- BSR (FP64)
// b == 1 without a handle is CSR (chunk engine).  b > 1: one thread per scalar row (I, r);
// the b values of row r of each block are contiguous.
template <int B>
__global__ void k_bsrB(int nb, const int *__restrict__ rp, const int *__restrict__ ci,
                       const double *__restrict__ val, const double *__restrict__ x,
                       const double *bvec, double *y, double alpha, double beta, int mode) {
    pdl_wait();
    pdl_launch_dependents();
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nb * B) return;
    int I = (int)(t / B), r = (int)(t % B);
    double s = 0.0;
    int p1 = __ldg(rp + I + 1);
    for (int p = __ldg(rp + I); p < p1; p++) {
        int J = __ldg(ci + p);
        const double *blk = val + ((long long)p * B + r) * B;
        const double *xj = x + (long long)J * B;
#pragma unroll
        for (int c = 0; c < B; c++) s += __ldg(blk + c) * __ldg(xj + c);
    }
    if (mode == 1) y[t] = bvec[t] - s;
    else y[t] = beta == 0.0 ? alpha * s : alpha * s + beta * y[t];
}

static void bsr_dispatch(int nb, int b, long long nnzb, const int *rp, const int *ci,
                         const double *val, const double *x, const double *bvec, double *y,
                         double alpha, double beta, int mode, cudaStream_t s) {
    if (nb <= 0) return;
    if (b == 1) {
        csr_chunk<double>(nb, nnzb > 0 ? nnzb : 8LL * nb, rp, ci, val, XPlain<double, double>{x},
                          EAxpby{alpha, beta, mode == 1 ? bvec : nullptr, y}, s);
        return;
    }
    long long n = (long long)nb * b;
    unsigned grid = GRIDN(n, 256);
    switch (b) {
        case 2: launch_k(k_bsrB<2>, dim3(grid), dim3(256), s, nb, rp, ci, val, x, bvec, y, alpha, beta, mode); break;
        case 3: launch_k(k_bsrB<3>, dim3(grid), dim3(256), s, nb, rp, ci, val, x, bvec, y, alpha, beta, mode); break;
        default: launch_k(k_bsrB<4>, dim3(grid), dim3(256), s, nb, rp, ci, val, x, bvec, y, alpha, beta, mode); break;
    }
}

void launch_bsr_spmv(int nb, int b, const int *rp, const int *ci, const double *val,
                     const double *x, double *y, double alpha, double beta, cudaStream_t s,
                     long long nnzb) {
    bsr_dispatch(nb, b, nnzb, rp, ci, val, x, nullptr, y, alpha, beta, 0, s);
}

void launch_bsr_residual(int nb, int b, const int *rp, const int *ci, const double *val,
                         const double *x, const double *bvec, double *y, cudaStream_t s,
                         long long nnzb) {
    bsr_dispatch(nb, b, nnzb, rp, ci, val, x, bvec, y, 1.0, 0.0, bvec ? 1 : 0, s);
}

// ---------------------------------------------------------------- MGR level
// F-relaxation, first sweep from z_F = 0: z_F = omega D^{-1} v_F
template <class T, class TV>
__global__ void k_frelax_first(int nF, const int *fidx, const int *gstart, const int *gsize,
                               const T *dinv, T omega, const TV *v, T *zF) {
    pdl_wait();
    pdl_launch_dependents();
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nF) return;
    int g = gstart[f], k = gsize[f];
    T s = (T)0;
    for (int q = 0; q < k; q++) s += dinv[(long long)f * 4 + q] * (T)v[fidx[g + q]];
    zF[f] = omega * s;
}

template <class T, class TV>
void launch_frelax_first(int nF, const int *fidx, const int *gstart, const int *gsize,
                         const T *dinv, T omega, const TV *v, T *zF, cudaStream_t s) {
    if (nF == 0) return;
    launch_k(k_frelax_first<T, TV>, dim3(GRIDN(nF, 256)), dim3(256), s, nF, fidx, gstart, gsize, dinv, omega, v, zF);
}

// r_F = v_F - A_FF z_F
template <class T, class TV>
void launch_frelax_residual(const DCSR &AFF, const T *vals, const int *fidx, const TV *v,
                            const T *zF, T *rF, cudaStream_t s) {
    spmv_rows<T>(AFF, vals, XPlain<T, T>{zF}, EGatherMinus<T, TV>{fidx, v, (T)-1, rF}, s);
}

// z_F += omega D^{-1} r_F (transpose: D^{-T})
template <class T>
__global__ void k_frelax_update(int nF, const int *gstart, const int *gsize, const T *dinv, T omega,
                                const T *rF, T *zF, int transpose) {
    pdl_wait();
    pdl_launch_dependents();
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nF) return;
    int g = gstart[f], k = gsize[f], r = f - g;
    T s = (T)0;
    for (int q = 0; q < k; q++) {
        T d = transpose ? dinv[(long long)(g + q) * 4 + r] : dinv[(long long)f * 4 + q];
        s += d * rF[g + q];
    }
    zF[f] += omega * s;
}

template <class T>
void launch_frelax_update(int nF, const int *gstart, const int *gsize, const T *dinv, T omega,
                          const T *rF, T *zF, int transpose, cudaStream_t s) {
    if (nF == 0) return;
    launch_k(k_frelax_update<T>, dim3(GRIDN(nF, 256)), dim3(256), s, nF, gstart, gsize, dinv, omega, rF, zF, transpose);
}

// AMG F-relaxation step: t = omega * (V-cycle output), rounded, then
// z_F = t (first sweep) or z_F = z_F + t (no fused multiply-add, so the
// two roundings match a plain multiply and add)
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

template <class T>
__global__ void k_frelax_scale(int nF, T omega, const T *t, T *zF, int accumulate) {
    pdl_wait();
    pdl_launch_dependents();
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nF) return;
    const T w = mul_rn(omega, t[f]);
    zF[f] = accumulate ? zF[f] + w : w;
}

template <class T>
void launch_frelax_scale(int nF, T omega, const T *t, T *zF, int accumulate, cudaStream_t s) {
    if (nF == 0) return;
    launch_k(k_frelax_scale<T>, dim3(GRIDN(nF, 256)), dim3(256), s, nF, omega, t, zF, accumulate);
}

// injection restriction of the residual: v_C = v[C] - A_CF z_F
template <class T, class TV>
void launch_mgr_restrict(const DCSR &ACF, const T *vals, const int *cidx, const TV *v,
                         const T *zF, T *vC, cudaStream_t s) {
    spmv_rows<T>(ACF, vals, XPlain<T, T>{zF}, EGatherMinus<T, TV>{cidx, v, (T)-1, vC}, s);
}

template <class T, class TV>
__global__ void k_scatter_c(int nC, const int *cidx, const T *eC, TV *z) {
    pdl_wait();
    pdl_launch_dependents();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nC) z[cidx[i]] = (TV)eC[i];
}

// interpolation + correction: z[F] = z_F + W e_C, z[C] = e_C
template <class T, class TV>
void launch_mgr_interp(const DCSR &W, const T *wvals, int nC, const int *fidx, const int *cidx,
                       const T *zF, const T *eC, TV *z, cudaStream_t s) {
    spmv_rows<T>(W, wvals, XPlain<T, T>{eC}, EInterp<T, TV>{fidx, zF, z}, s);
    if (nC > 0) launch_k(k_scatter_c<T, TV>, dim3(GRIDN(nC, 256)), dim3(256), s, nC, cidx, eC, z);
}

// transposed-cycle pieces
template <class T, class TV>
__global__ void k_gather(const int *idx, int n, const TV *v, T *out) {
    pdl_wait();
    pdl_launch_dependents();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (T)v[idx[i]];
}

template <class T, class TV>
void launch_gather(const int *idx, int n, const TV *v, T *out, cudaStream_t s) {
    if (n == 0) return;
    launch_k(k_gather<T, TV>, dim3(GRIDN(n, 256)), dim3(256), s, idx, n, v, out);
}

// y[i] = bsrc[idx_b[i]] + sign * (M x)_i
template <class T, class TV>
void launch_csr_axpy_gather(const DCSR &M, const T *vals, const T *x, const int *idx_b,
                            const TV *bsrc, T sign, T *y, cudaStream_t s) {
    spmv_rows<T>(M, vals, XPlain<T, T>{x}, EGatherMinus<T, TV>{idx_b, bsrc, sign, y}, s);
}

template <class T, class TV>
__global__ void k_scatter2(int nF, int nC, const int *fidx, const int *cidx, const T *zF,
                           const T *eC, TV *z) {
    pdl_wait();
    pdl_launch_dependents();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nF) z[fidx[i]] = (TV)zF[i];
    else if (i < nF + nC) z[cidx[i - nF]] = (TV)eC[i - nF];
}

template <class T, class TV>
void launch_scatter2(int nF, int nC, const int *fidx, const int *cidx, const T *zF, const T *eC,
                     TV *z, cudaStream_t s) {
    launch_k(k_scatter2<T, TV>, dim3(GRIDN(nF + nC, 256)), dim3(256), s, nF, nC, fidx, cidx, zF, eC, z);
}

// ---------------------------------------------------------------- AMG level
// pre-smoothing from x = 0 fused with the residual:
//   x_i = dinv_i r_i ;  res_i = r_i - sum_j a_ij dinv_j r_j

// residual of the pre-smoothed iterate x = D r computed by the producer of r:
//   res_i = r_i - sum_j a_ij x_j
template <class T, class TV>
void launch_amg_residual(const DCSR &A, const T *vals, const T *x, const TV *r, T *res,
                         cudaStream_t s) {
    spmv_rows<T>(A, vals, XPlain<T, T>{x}, EResid<T, TV>{r, res}, s);
}

// restriction r_c = R res that also writes x_c = D_c r_c for the next level
template <class T>
void launch_restrict_scaled(const DCSR &R, const T *vals, const T *res, T *rc, const T *dc, T *xc,
                            cudaStream_t s) {
    spmv_rows<T>(R, vals, XPlain<T, T>{res}, EStoreScaled<T>{rc, dc, xc}, s);
}

// MGR injection restriction that also writes x = D v_C for the AMG below
template <class T, class TV>
void launch_mgr_restrict_scaled(const DCSR &ACF, const T *vals, const int *cidx, const TV *v,
                                const T *zF, T *vC, const T *d, T *x, cudaStream_t s) {
    spmv_rows<T>(ACF, vals, XPlain<T, T>{zF}, EGatherMinusScaled<T, TV>{cidx, v, vC, d, x}, s);
}

template <class T, class TV>
__global__ void k_scale(int n, const T *d, const TV *r, T *x) {
    pdl_wait();
    pdl_launch_dependents();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = d[i] * (T)r[i];
}

template <class T, class TV>
void launch_scale(int n, const T *d, const TV *r, T *x, cudaStream_t s) {
    if (n > 0) launch_k(k_scale<T, TV>, dim3(GRIDN(n, 256)), dim3(256), s, n, d, r, x);
}

// post-smoothing: xout_i = x_i + dinv_i (r_i - sum_j a_ij x_j)
template <class T, class TV>
void launch_amg_post_smooth(const DCSR &A, const T *vals, const T *dinv, const TV *r, const T *x,
                            TV *xout, cudaStream_t s) {
    spmv_rows<T>(A, vals, XPlain<T, T>{x}, EPost<T, TV>{r, dinv, x, xout}, s);
}

// coarsest grid: x = A^{-1} r with the explicit FP64 inverse; one warp per row
template <class TV>
__global__ void k_dense_matvec(int n, const double *inv, const TV *r, TV *x) {
    pdl_wait();
    pdl_launch_dependents();
    int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int c = lane; c < n; c += 32) s = fma(inv[(long long)row * n + c], (double)r[c], s);
    s = group_sum<32, double>(s);
    if (lane == 0) x[row] = (TV)s;
}

template <class TV>
void launch_dense_matvec(int n, const double *inv, const TV *r, TV *x, cudaStream_t s) {
    if (n == 0) return;
    launch_k(k_dense_matvec<TV>, dim3(GRIDN((long long)n * 32, 256)), dim3(256), s, n, inv, r, x);
}


// ------------------------------------------------------------ SELL tuning
// Time y = M x in both slice orders of k_sell (grid-stride, contiguous per
// block) and keep the faster one in M.sched.  Each timed launch follows a
// write of the flush buffer (larger than L2), so the matrix streams from
// HBM as it does inside a V-cycle; the orders alternate and each keeps its
// best of two launches; the contiguous order must win by 5%.  The choice
// only changes which warp sums which row, never a result.
template <class T>
static int sell_tune_t(DCSR &M, const T *vals, cudaStream_t s, Arena &ar, const SellTune &tn) {
    T *x = ar.alloc<T>((size_t)(M.m > 0 ? M.m : 1));
    T *y = ar.alloc<T>((size_t)(M.n > 0 ? M.n : 1));
    if (!x || !y) return ST_NOMEM;
    cudaMemsetAsync(x, 0, sizeof(T) * (M.m > 0 ? M.m : 1), s);
    // the forms: both slice orders; FP64 also with the pipelined chain, when
    // a lane's chain averages two load rounds or more (with fewer there is no
    // next round to load early)
    const double lane_len = (double)M.sell_stored / (32.0 * M.nsl);
    const int nform = (sizeof(T) == 8 && lane_len >= 2.0 * SellCfg<T>::U) ? 4 : 2;
    const int nround = 2 * nform;  // <= SELL_TUNE_ROUNDS
    for (int round = 0; round < nround; round++) {
        M.sched = round % nform;
        cudaMemsetAsync(tn.flush, round, tn.flush_bytes, s);
        cudaEventRecord(tn.ev[2 * round], s);
        spmv_rows<T>(M, vals, XPlain<T, T>{x}, EStore<T, T>{y}, s);
        cudaEventRecord(tn.ev[2 * round + 1], s);
    }
    float best[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    if (cudaEventSynchronize(tn.ev[2 * nround - 1]) == cudaSuccess)
        for (int round = 0; round < nround; round++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, tn.ev[2 * round], tn.ev[2 * round + 1]) == cudaSuccess &&
                ms < best[round % nform])
                best[round % nform] = ms;
        }
    ar.release(x);
    ar.release(y);
    // another form only when it is at least 5% faster than the first
    int pick = 0;
    for (int f = 1; f < nform; f++)
        if (best[f] < 0.95f * best[0] && best[f] < best[pick]) pick = f;
    M.sched = pick;
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// MGR_SELL_ORDER=grid, contig, grid_pipe or contig_pipe puts every SELL
// product of a setup into that form instead of timing it (a test knob: all
// forms must give the same bits; FP32 products ignore _pipe); anything else,
// or unset, times each product.
static int forced_order() {
    static const int f = [] {
        const char *e = getenv("MGR_SELL_ORDER");
        if (!e) return -1;
        if (!strcmp(e, "grid")) return 0;
        if (!strcmp(e, "contig")) return 1;
        if (!strcmp(e, "grid_pipe")) return 2;
        if (!strcmp(e, "contig_pipe")) return 3;
        return -1;
    }();
    return f;
}

int sell_tune(DCSR &M, const SellTune &tn, cudaStream_t s, Arena &ar) {
    M.sched = 0;
    if (forced_order() >= 0) {
        if (M.sptr) M.sched = tn.fp32 ? (forced_order() & 1) : forced_order();
        return ST_OK;
    }
    // a product of fewer slices than one wave of warps runs the same in every form
    if (!M.sptr || M.nsl < SELL_TUNE_MIN_SLICES || !tn.flush) return ST_OK;
    if (tn.fp32) return M.sv32 ? sell_tune_t<float>(M, M.sv32, s, ar, tn) : ST_OK;
    return M.sv ? sell_tune_t<double>(M, M.sv, s, ar, tn) : ST_OK;
}

// ------------------------------------------------------- instantiations
#define INST_T_TV(T, TV)                                                                          \
    template void launch_frelax_first<T, TV>(int, const int *, const int *, const int *,          \
                                             const T *, T, const TV *, T *, cudaStream_t);        \
    template void launch_frelax_residual<T, TV>(const DCSR &, const T *, const int *, const TV *, \
                                                const T *, T *, cudaStream_t);                    \
    template void launch_mgr_restrict<T, TV>(const DCSR &, const T *, const int *, const TV *,    \
                                             const T *, T *, cudaStream_t);                       \
    template void launch_mgr_interp<T, TV>(const DCSR &, const T *, int, const int *, const int *,\
                                           const T *, const T *, TV *, cudaStream_t);             \
    template void launch_gather<T, TV>(const int *, int, const TV *, T *, cudaStream_t);          \
    template void launch_csr_axpy_gather<T, TV>(const DCSR &, const T *, const T *, const int *,  \
                                                const TV *, T, T *, cudaStream_t);                \
    template void launch_scatter2<T, TV>(int, int, const int *, const int *, const T *, const T *,\
                                         TV *, cudaStream_t);                                     \
    template void launch_amg_post_smooth<T, TV>(const DCSR &, const T *, const T *, const TV *,   \
                                                const T *, TV *, cudaStream_t);                   \
    template void launch_amg_residual<T, TV>(const DCSR &, const T *, const T *, const TV *, T *, \
                                             cudaStream_t);                                       \
    template void launch_mgr_restrict_scaled<T, TV>(const DCSR &, const T *, const int *,         \
                                                    const TV *, const T *, T *, const T *, T *,   \
                                                    cudaStream_t);                                \
    template void launch_scale<T, TV>(int, const T *, const TV *, T *, cudaStream_t);

INST_T_TV(double, double)
INST_T_TV(float, float)
INST_T_TV(float, double)

template void launch_frelax_update<double>(int, const int *, const int *, const double *, double,
                                           const double *, double *, int, cudaStream_t);
template void launch_frelax_update<float>(int, const int *, const int *, const float *, float,
                                          const float *, float *, int, cudaStream_t);
template void launch_frelax_scale<double>(int, double, const double *, double *, int, cudaStream_t);
template void launch_frelax_scale<float>(int, float, const float *, float *, int, cudaStream_t);
template void launch_csr_spmv<double>(const DCSR &, const double *, const double *, double *,
                                      cudaStream_t);
template void launch_csr_spmv<float>(const DCSR &, const float *, const float *, float *,
                                     cudaStream_t);
template void launch_restrict_scaled<double>(const DCSR &, const double *, const double *, double *,
                                             const double *, double *, cudaStream_t);
template void launch_restrict_scaled<float>(const DCSR &, const float *, const float *, float *,
                                            const float *, float *, cudaStream_t);
template void launch_csr_spmv_add<double>(const DCSR &, const double *, const double *, double *,
                                          cudaStream_t);
template void launch_csr_spmv_add<float>(const DCSR &, const float *, const float *, float *,
                                         cudaStream_t);
template void launch_dense_matvec<double>(int, const double *, const double *, double *,
                                          cudaStream_t);
template void launch_dense_matvec<float>(int, const double *, const float *, float *, cudaStream_t);

}  // namespace mgr
