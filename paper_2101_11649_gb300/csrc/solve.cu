// Solve-phase kernels: sparse products, the MGR and AMG cycle steps, and
// the FGMRES reductions.  All are HBM-bandwidth-bound.
//
// CSR rows are processed by a chunk engine: a warp owns R consecutive rows
// (R chosen per matrix so that a chunk holds ~192 nonzeros), loads the
// chunk's nonzeros with CU independent coalesced loads per lane, keeps the
// products in shared memory, and each lane then sums one row in order.
// Gathers and epilogues are functors, so every cycle step (residual,
// smoothing, restriction, interpolation) is one pass over its matrix.
// Every reduction uses a fixed order, so repeated runs give identical bits.
#include <cuda_runtime.h>
#include <stdlib.h>

#include "common.cuh"
#include "sell.cuh"

namespace mgr {

#define GRIDN(n, t) (unsigned)((((long long)(n)) + (t)-1) / (t) > 0 ? (((long long)(n)) + (t)-1) / (t) : 1)

static const int NUM_SMS = 152;

bool pdl_on() {
    static const bool on = [] {
        const char *e = getenv("MGR_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

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
// k_sell: one warp per slice (layout and row sums in sell.cuh), grid-stride
// over slices; FP32 (PF) starts a slice's epilogue loads and the next
// slice's offsets before the slice's products.
template <int G, class T, class XF, class EPI>
__global__ void __launch_bounds__(256, SELL_BLOCKS)
    k_sell(int nsl, const long long *__restrict__ sptr, const int *__restrict__ slen,
           const int *__restrict__ perm, const int *__restrict__ sci, const T *__restrict__ sv, XF xf,
           EPI epi) {
    constexpr int PF = SellCfg<T>::PF;
    constexpr int C = 32 / G;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int sl = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sl >= nsl) return;
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
        const T acc = sell_rows<G, T>(L, base, sci, sv, xf);
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

template <int G, class T, class XF, class EPI>
static void sell_launch(const DCSR &M, const T *vals, XF xf, EPI epi, cudaStream_t s) {
    long long blocks = ((long long)M.nsl * 32 + 255) / 256;
    const long long cap = (long long)NUM_SMS * SELL_BLOCKS * 2;
    if (blocks > cap) blocks = cap;
    launch_k(k_sell<G, T, XF, EPI>, dim3((unsigned)(blocks < 1 ? 1 : blocks)), dim3(256), s, M.nsl, M.sptr,
             M.slen, M.perm, M.sci, vals, xf, epi);
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
template <class T, class TV>
struct XScaled {  // x_j = d_j r_j (pre-smoothing from zero)
    const T *d;
    const TV *r;
    __device__ __forceinline__ T operator()(int j) const { return __ldg(d + j) * (T)__ldg(r + j); }
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
struct ESmooth0 {  // x = d r ; res = r - A (d r)
    const TV *r;
    const T *d;
    T *x, *res;
    struct Pre { T r, d; };
    __device__ __forceinline__ Pre pre(int row) const { return {(T)r[row], d[row]}; }
    __device__ __forceinline__ void put(int row, T s, const Pre &p) const {
        x[row] = p.d * p.r;
        res[row] = p.r - s;
    }
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
// b == 1 is CSR (chunk engine).  b > 1: one thread per scalar row (I, r);
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
template <class T, class TV>
void launch_amg_smooth0_residual(const DCSR &A, const T *vals, const T *dinv, const TV *r, T *x,
                                 T *res, cudaStream_t s) {
    spmv_rows<T>(A, vals, XScaled<T, TV>{dinv, r}, ESmooth0<T, TV>{r, dinv, x, res}, s);
}

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

template <class TV>
__global__ void k_copy_cast(const TV *in, double *out, int n) {
    pdl_wait();
    pdl_launch_dependents();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

template <class TV>
void launch_copy_cast(const TV *in, double *out, int n, cudaStream_t s) {
    if (n == 0) return;
    launch_k(k_copy_cast<TV>, dim3(GRIDN(n, 256)), dim3(256), s, in, out, n);
}

// ------------------------------------------------------------- Krylov (FP64)
// Reductions over n with a fixed grid: each block accumulates a fixed
// element set, writes its partial, and the last block to finish (ticket)
// sums the partials in block order, one warp per output.
static const int RED_THREADS = 256;
static const int RED_EPT = 2;

int multidot_blocks(int n) {
    long long b = ((long long)n + RED_THREADS * RED_EPT - 1) / (RED_THREADS * RED_EPT);
    if (b > NUM_SMS * 2) b = NUM_SMS * 2;
    return (int)(b < 1 ? 1 : b);
}

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

// h[i] = V_i . w for i < K (w may be V_{K-1} itself).  Skipped when
// *flag == 0 (flag != nullptr): the conditional reorthogonalisation pass.
// The K basis vectors are read in chunks of KB: a chunk's loads are all
// issued before its FMAs, so every thread keeps 2 KB loads in flight
// whatever schedule the compiler picks for a given K.
template <int K>
__global__ void __launch_bounds__(RED_THREADS, 2) k_dots(const double *__restrict__ V, long long ldv,
                                                         const double *__restrict__ w, int n,
                                                         double *partial, double *h, unsigned *ticket,
                                                         const int *flag) {
    pdl_wait();
    pdl_launch_dependents();
    if (flag && *flag == 0) return;
    constexpr int KB = K < 8 ? K : 8;
    double acc[K];
#pragma unroll
    for (int i = 0; i < K; i++) acc[i] = 0.0;
    const long long stride = (long long)gridDim.x * RED_THREADS * RED_EPT;
    for (long long e0 = (long long)blockIdx.x * RED_THREADS * RED_EPT + threadIdx.x; e0 < n; e0 += stride) {
        double wv[RED_EPT];
#pragma unroll
        for (int u = 0; u < RED_EPT; u++) {
            const long long e = e0 + (long long)u * RED_THREADS;
            wv[u] = e < n ? __ldg(w + e) : 0.0;
        }
#pragma unroll
        for (int i0 = 0; i0 < K; i0 += KB) {
            double vv[KB][RED_EPT];
#pragma unroll
            for (int i = 0; i < KB; i++)
#pragma unroll
                for (int u = 0; u < RED_EPT; u++) {
                    const long long e = e0 + (long long)u * RED_THREADS;
                    vv[i][u] = (i0 + i < K && e < n) ? __ldg(V + (i0 + i) * ldv + e) : 0.0;
                }
#pragma unroll
            for (int i = 0; i < KB; i++)
                if (i0 + i < K)
#pragma unroll
                    for (int u = 0; u < RED_EPT; u++) acc[i0 + i] = fma(vv[i][u], wv[u], acc[i0 + i]);
        }
    }
    block_partials<K>(acc, partial);
    if (last_block(ticket)) {
        sum_partials<K>(partial, h);
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

// Classical Gram-Schmidt with a rescue pass: the second projection runs
// only when the first removed more than 99% of |w| (|w'| < 0.1 |w|), the
// cancellation that costs orthogonality (a DGKS-type test with eta = 0.1).
static constexpr double REORTH_ETA2 = 1e-2;

// w <- w - sum_{i<K} V_i h_i ; nrm2 = |w|^2.  mode 1 (first pass) also
// decides reorthogonalisation (|w'|^2 < eta^2 |w|^2, with |w|^2 = h[K]) and
// writes it to *flag; mode 2 (the second pass) is skipped when *flag == 0.
// Chunked loads as in k_dots; h is read from shared memory.
template <int K>
__global__ void __launch_bounds__(RED_THREADS, 2) k_update_norm(const double *__restrict__ V, long long ldv,
                                                                const double *__restrict__ h, double *w,
                                                                int n, double *partial, double *nrm2,
                                                                unsigned *ticket, int *flag, int mode) {
    pdl_wait();
    pdl_launch_dependents();
    if (mode == 2 && *flag == 0) return;
    constexpr int KB = K < 16 ? K : 16;
    __shared__ double hs[K];
    if (threadIdx.x < K) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * RED_THREADS * RED_EPT;
    for (long long e0 = (long long)blockIdx.x * RED_THREADS * RED_EPT + threadIdx.x; e0 < n; e0 += stride) {
        double wv[RED_EPT];
#pragma unroll
        for (int u = 0; u < RED_EPT; u++) {
            const long long e = e0 + (long long)u * RED_THREADS;
            wv[u] = e < n ? w[e] : 0.0;
        }
#pragma unroll
        for (int i0 = 0; i0 < K; i0 += KB) {
            double vv[KB][RED_EPT];
#pragma unroll
            for (int i = 0; i < KB; i++)
#pragma unroll
                for (int u = 0; u < RED_EPT; u++) {
                    const long long e = e0 + (long long)u * RED_THREADS;
                    vv[i][u] = (i0 + i < K && e < n) ? __ldg(V + (i0 + i) * ldv + e) : 0.0;
                }
#pragma unroll
            for (int i = 0; i < KB; i++)
                if (i0 + i < K) {
                    const double hi = hs[i0 + i];
#pragma unroll
                    for (int u = 0; u < RED_EPT; u++) wv[u] = fma(-vv[i][u], hi, wv[u]);
                }
        }
#pragma unroll
        for (int u = 0; u < RED_EPT; u++) {
            const long long e = e0 + (long long)u * RED_THREADS;
            if (e < n) { w[e] = wv[u]; acc[0] = fma(wv[u], wv[u], acc[0]); }
        }
    }
    block_partials<1>(acc, partial);
    if (last_block(ticket)) {
        sum_partials<1>(partial, nrm2);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (mode == 1) *flag = (*nrm2 < REORTH_ETA2 * h[K]) ? 1 : 0;
            *ticket = 0u;
        }
    }
}

#define K_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) \
    X(15) X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) X(25) X(26) X(27) X(28) X(29) \
    X(30) X(31) X(32)

void launch_dots(const double *V, long long ldv, int k, const double *w, int n, double *partial,
                 double *h, unsigned *ticket, const int *flag, int nblk, cudaStream_t s) {
    switch (k) {
#define X(K) case K: launch_k(k_dots<K>, dim3(nblk), dim3(RED_THREADS), s, V, ldv, w, n, partial, h, ticket, flag); break;
        K_CASES(X)
#undef X
        default: break;
    }
}

void launch_update_norm(const double *V, long long ldv, int k, const double *h, double *w, int n,
                        double *partial, double *nrm2, unsigned *ticket, int *flag, int mode,
                        int nblk, cudaStream_t s) {
    switch (k) {
#define X(K) case K: launch_k(k_update_norm<K>, dim3(nblk), dim3(RED_THREADS), s, V, ldv, h, w, n, partial, nrm2, ticket, flag, mode); break;
        K_CASES(X)
#undef X
        default: break;
    }
}

// x . y (sqrt when asked) with the ticketed reduction
__global__ void __launch_bounds__(RED_THREADS) k_dot2(const double *x, const double *y, int n,
                                                      double *partial, double *out, unsigned *ticket,
                                                      int sqrt_out) {
    pdl_wait();
    pdl_launch_dependents();
    double acc[1] = {0.0};
    const long long stride = (long long)gridDim.x * RED_THREADS;
    for (long long e = (long long)blockIdx.x * RED_THREADS + threadIdx.x; e < n; e += stride)
        acc[0] += x[e] * y[e];
    block_partials<1>(acc, partial);
    if (last_block(ticket)) {
        sum_partials<1>(partial, out);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sqrt_out) *out = sqrt(*out);
            *ticket = 0u;
        }
    }
}

void launch_dot(const double *x, const double *y, int n, double *partial, double *out,
                unsigned *ticket, int sqrt_out, int nblk, cudaStream_t s) {
    launch_k(k_dot2, dim3(nblk), dim3(RED_THREADS), s, x, y, n, partial, out, ticket, sqrt_out);
}

// y = x * s  or  y = x / s  (s a device scalar)
__global__ void k_vec_scale(const double *x, double *y, const double *sc, int invert, int n) {
    pdl_wait();
    pdl_launch_dependents();
    const double f = invert ? 1.0 / *sc : *sc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        y[e] = x[e] * f;
}

void launch_vec_scale(const double *x, double *y, const double *scale_num, const double *,
                      int invert, int n, cudaStream_t s) {
    unsigned g = GRIDN(n, 256);
    launch_k(k_vec_scale, dim3(g > NUM_SMS * 8 ? NUM_SMS * 8 : g), dim3(256), s, x, y, scale_num, invert, n);
}

// x += sum_i y_i Z_i
__global__ void k_multi_axpy(const double *__restrict__ Z, long long ldz, int k,
                             const double *__restrict__ y, double *x, int n) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ double ys[32];
    if (threadIdx.x < k) ys[threadIdx.x] = y[threadIdx.x];
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        double s = x[e];
        for (int i = 0; i < k; i++) s += ys[i] * __ldg(Z + i * ldz + e);
        x[e] = s;
    }
}

void launch_multi_axpy(const double *Z, long long ldz, int k, const double *y, double *x, int n,
                       cudaStream_t s) {
    unsigned g = GRIDN(n, 256);
    launch_k(k_multi_axpy, dim3(g > NUM_SMS * 8 ? NUM_SMS * 8 : g), dim3(256), s, Z, ldz, k, y, x, n);
}

// dA[p, r, c] = -lam[I*b + r] * x[J*b + c]
__global__ void k_grad_values(int nb, int b, const int *rp, const int *ci, const double *lam,
                              const double *x, double *dA) {
    pdl_wait();
    pdl_launch_dependents();
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nb * b) return;
    int I = (int)(t / b), r = (int)(t % b);
    double l = lam[t];
    for (int p = rp[I]; p < rp[I + 1]; p++) {
        int J = ci[p];
        for (int c = 0; c < b; c++) dA[((long long)p * b + r) * b + c] = -l * x[(long long)J * b + c];
    }
}

void launch_grad_values(int nb, int b, const int *rp, const int *ci, const double *lam,
                        const double *x, double *dA, cudaStream_t s) {
    launch_k(k_grad_values, dim3(GRIDN((long long)nb * b, 256)), dim3(256), s, nb, b, rp, ci, lam, x, dA);
}

// ------------------------------------------------------------- misc
// input validation of a block-CSR matrix: bit 2 malformed pattern, bit 8 a
// non-finite value, bit 16 a missing diagonal block
__global__ void k_validate_bsr(int nb, int b, const int *rp, const int *ci, const double *val,
                               int *err) {
    pdl_wait();
    pdl_launch_dependents();
    int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nb) return;
    int p0 = rp[I], p1 = rp[I + 1];
    if (I == 0 && p0 != 0) atomicOr(err, 2);
    if (p1 < p0) { atomicOr(err, 2); return; }
    bool diag = false;
    for (int p = p0; p < p1; p++) {
        int J = ci[p];
        if (J < 0 || J >= nb || (p > p0 && ci[p - 1] >= J)) atomicOr(err, 2);
        if (J == I) diag = true;
        for (int t = 0; t < b * b; t++)
            if (!isfinite(val[(long long)p * b * b + t])) { atomicOr(err, 8); break; }
    }
    if (!diag) atomicOr(err, 16);
}

void launch_validate_bsr(int nb, int b, const int *rp, const int *ci, const double *val, int *err,
                         cudaStream_t s) {
    launch_k(k_validate_bsr, dim3(GRIDN(nb, 256)), dim3(256), s, nb, b, rp, ci, val, err);
}

__global__ void k_transpose_dense(int n, const double *in, double *out) {
    pdl_wait();
    pdl_launch_dependents();
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)n * n) return;
    int r = (int)(e / n), c = (int)(e % n);
    out[(long long)c * n + r] = in[e];
}

void launch_transpose_dense(int n, const double *in, double *out, cudaStream_t s) {
    if (n == 0) return;
    launch_k(k_transpose_dense, dim3(GRIDN((long long)n * n, 256)), dim3(256), s, n, in, out);
}

// H is (m+1) x m row-major.  h1[0..j] first-pass projections and h1[j+1] =
// |w|^2 before orthogonalisation; when *flag (reorthogonalised) h2 holds the
// second-pass projections and nrmB the final |w|^2, else nrmA.  Applies the
// previous Givens rotations to column j, forms the new one, and writes
// stat = {|g_{j+1}|, converged, breakdown, h_{j+1,j}}.
__global__ void k_arnoldi_finish(int j, int m, const double *h1, const double *h2,
                                 const double *nrmA, const double *nrmB, const int *flag,
                                 double *H, double *cs, double *sn, double *g, double *hn_out,
                                 double *stat, const double *tol) {
    pdl_wait();
    pdl_launch_dependents();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double tol_abs = *tol;
    const int re = *flag;
    double w0 = sqrt(h1[j + 1]);
    for (int i = 0; i <= j; i++) H[i * m + j] = re ? h1[i] + h2[i] : h1[i];
    double hn = sqrt(re ? *nrmB : *nrmA);
    for (int i = 0; i < j; i++) {
        double a = H[i * m + j], b = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * b;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
    }
    double a = H[j * m + j], b = hn;
    double rho = sqrt(a * a + b * b);
    cs[j] = a / rho;
    sn[j] = b / rho;
    H[j * m + j] = rho;
    H[(j + 1) * m + j] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = cs[j] * g[j];
    double est = fabs(g[j + 1]);
    *hn_out = hn;
    stat[0] = est;
    stat[1] = est <= tol_abs ? 1.0 : 0.0;
    stat[2] = hn <= 1e-14 * w0 ? 1.0 : 0.0;
    stat[3] = hn;
    stat[4] = re;
}

void launch_arnoldi_finish(int j, int m, const double *h1, const double *h2, const double *nrmA,
                           const double *nrmB, const int *flag, double *H, double *cs, double *sn,
                           double *g, double *hn, double *stat, const double *tol, cudaStream_t s) {
    launch_k(k_arnoldi_finish, dim3(1), dim3(32), s, j, m, h1, h2, nrmA, nrmB, flag, H, cs, sn, g, hn, stat, tol);
}

__global__ void k_init_g(double *g, int m, const double *beta) {
    pdl_wait();
    pdl_launch_dependents();
    int i = threadIdx.x;
    if (i <= m) g[i] = i == 0 ? *beta : 0.0;
}

void launch_init_g(double *g, int m, const double *beta, cudaStream_t s) {
    launch_k(k_init_g, dim3(1), dim3(64), s, g, m, beta);
}

__global__ void k_solve_upper(int k, int m, const double *H, const double *g, double *y) {
    pdl_wait();
    pdl_launch_dependents();
    if (threadIdx.x != 0) return;
    for (int i = k - 1; i >= 0; i--) {
        double s = g[i];
        for (int t = i + 1; t < k; t++) s -= H[i * m + t] * y[t];
        y[i] = s / H[i * m + i];
    }
}

void launch_solve_upper(int k, int m, const double *H, const double *g, double *y, cudaStream_t s) {
    launch_k(k_solve_upper, dim3(1), dim3(32), s, k, m, H, g, y);
}

__global__ void k_iota(int *a, int n) {
    pdl_wait();
    pdl_launch_dependents();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = i;
}

void launch_iota(int *a, int n, cudaStream_t s) {
    if (n > 0) launch_k(k_iota, dim3(GRIDN(n, 256)), dim3(256), s, a, n);
}

__global__ void k_gather_int(const int *idx, int n, const int *v, int *out) {
    pdl_wait();
    pdl_launch_dependents();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v[idx[i]];
}

void launch_gather_int(const int *idx, int n, const int *v, int *out, cudaStream_t s) {
    if (n > 0) launch_k(k_gather_int, dim3(GRIDN(n, 256)), dim3(256), s, idx, n, v, out);
}


// ================================================================ batched
// One launch per kernel class over every system of a batch: the grid walks
// a flattened list of work items (warp-chunks, elements or blocks) whose
// per-system start offsets are in `prefix`; each item finds its system by
// binary search and runs the single-system code on that system's operands.
__device__ __forceinline__ int find_job(const long long *prefix, int njobs, long long g) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool job_off(const BJob &J) { return J.active && *J.active == 0; }

template <class T>
struct EStoreMaybeScaled {  // y = s ; x = d s when d
    T *y;
    const T *d;
    T *x;
    __device__ __forceinline__ void operator()(int row, T s) const {
        y[row] = s;
        if (d) x[row] = d[row] * s;
    }
};
template <class T, class TV>
struct EGatherMinusMaybeScaled {  // y = b[idx] - s ; x = d y when d
    const int *idx;
    const TV *b;
    T *y;
    const T *d;
    T *x;
    __device__ __forceinline__ void operator()(int row, T s) const {
        T t = (T)b[idx[row]] - s;
        y[row] = t;
        if (d) x[row] = d[row] * t;
    }
};
struct EOuter {  // y = s, or y = b - s (residual)
    const double *b;
    double *y;
    __device__ __forceinline__ void operator()(int row, double s) const { y[row] = b ? b[row] - s : s; }
};

template <class T, class TV, int OP> struct BOpT;
template <class T, class TV> struct BOpT<T, TV, BOP_RESID> {
    __device__ static XPlain<T, T> xf(const BJob &J, int) { return {(const T *)J.x}; }
    __device__ static EResid<T, TV> epi(const BJob &J, int js) { return {(const TV *)J.r + js * J.sr, (T *)J.o1}; }
};
template <class T, class TV> struct BOpT<T, TV, BOP_RESTRICT> {
    __device__ static XPlain<T, T> xf(const BJob &J, int) { return {(const T *)J.x}; }
    __device__ static EStoreMaybeScaled<T> epi(const BJob &J, int) { return {(T *)J.o1, (const T *)J.d, (T *)J.o2}; }
};
template <class T, class TV> struct BOpT<T, TV, BOP_PROLONG> {
    __device__ static XPlain<T, T> xf(const BJob &J, int) { return {(const T *)J.x}; }
    __device__ static EAdd<T> epi(const BJob &J, int) { return {(T *)J.o1}; }
};
template <class T, class TV> struct BOpT<T, TV, BOP_POST> {
    __device__ static XPlain<T, T> xf(const BJob &J, int) { return {(const T *)J.x}; }
    __device__ static EPost<T, TV> epi(const BJob &J, int js) {
        return {(const TV *)J.r + js * J.sr, (const T *)J.d, (const T *)J.x, (TV *)J.o1 + js * J.so1};
    }
};
template <class T, class TV> struct BOpT<T, TV, BOP_MGR_RESTRICT> {
    __device__ static XPlain<T, T> xf(const BJob &J, int) { return {(const T *)J.x}; }
    __device__ static EGatherMinusMaybeScaled<T, TV> epi(const BJob &J, int js) {
        return {J.idx, (const TV *)J.r + js * J.sr, (T *)J.o1, (const T *)J.d, (T *)J.o2};
    }
};
template <class T, class TV> struct BOpT<T, TV, BOP_MGR_INTERP> {
    __device__ static XPlain<T, T> xf(const BJob &J, int) { return {(const T *)J.x}; }
    __device__ static EInterp<T, TV> epi(const BJob &J, int js) {
        return {J.idx, (const T *)J.zF, (TV *)J.o1 + js * J.so1};
    }
};
template <class T, class TV> struct BOpT<T, TV, BOP_OUTER_CSR> {
    __device__ static XPlain<double, double> xf(const BJob &J, int js) { return {(const double *)J.x + js * J.sx}; }
    __device__ static EOuter epi(const BJob &J, int js) { return {(const double *)J.r, (double *)J.o1 + js * J.so1}; }
};

template <int R, class T, class TV, int OP>
__global__ void __launch_bounds__(CWARPS * 32) k_bchunk(const BJob *__restrict__ jobs,
                                                        const long long *__restrict__ prefix,
                                                        int njobs, int js) {
    pdl_wait();
    pdl_launch_dependents();
    __shared__ T sv[CWARPS][CCAP];
    __shared__ int sc[CWARPS][CCAP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long total = prefix[njobs];
    for (long long g = (long long)blockIdx.x * CWARPS + warp; g < total; g += (long long)gridDim.x * CWARPS) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const int c = (int)(g - prefix[j]);
        const int n = J.n;
        const int r0 = c * R, r1 = min(r0 + R, n);
        const int *rp = J.rp, *ci = J.ci;
        const T *v = (const T *)J.v;
        const auto xf = BOpT<T, TV, OP>::xf(J, js);
        const auto epi = BOpT<T, TV, OP>::epi(J, js);
        const int p0 = __ldg(rp + r0), p1 = __ldg(rp + r1);
        const int cnt = p1 - p0;
        if (cnt <= CCAP) {
            chunk_rows<R>(r0, r1, p0, cnt, rp, ci, v, xf, epi, sv[warp], sc[warp], lane);
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

template <class T, class TV, int OP>
static void bchunk_dispatch(const BJob *jobs, const long long *prefix, int njobs, long long total,
                            int R, int js, cudaStream_t s) {
    if (total <= 0) return;
    long long blocks = (total + CWARPS - 1) / CWARPS;
    if (blocks > NUM_SMS * 8) blocks = NUM_SMS * 8;
    unsigned g = (unsigned)(blocks < 1 ? 1 : blocks);
    switch (R) {
        case 1: launch_plain(k_bchunk<1, T, TV, OP>, dim3(g), dim3(CWARPS * 32), s, jobs, prefix, njobs, js); break;
        case 2: launch_plain(k_bchunk<2, T, TV, OP>, dim3(g), dim3(CWARPS * 32), s, jobs, prefix, njobs, js); break;
        case 4: launch_plain(k_bchunk<4, T, TV, OP>, dim3(g), dim3(CWARPS * 32), s, jobs, prefix, njobs, js); break;
        case 8: launch_plain(k_bchunk<8, T, TV, OP>, dim3(g), dim3(CWARPS * 32), s, jobs, prefix, njobs, js); break;
        case 16: launch_plain(k_bchunk<16, T, TV, OP>, dim3(g), dim3(CWARPS * 32), s, jobs, prefix, njobs, js); break;
        default: launch_plain(k_bchunk<32, T, TV, OP>, dim3(g), dim3(CWARPS * 32), s, jobs, prefix, njobs, js); break;
    }
}

template <class T, class TV>
void launch_bchunk(int op, const BJob *jobs, const long long *prefix, int njobs, long long total,
                   int R, int js, cudaStream_t s) {
    switch (op) {
        case BOP_RESID: bchunk_dispatch<T, TV, BOP_RESID>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_RESTRICT: bchunk_dispatch<T, TV, BOP_RESTRICT>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_PROLONG: bchunk_dispatch<T, TV, BOP_PROLONG>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_POST: bchunk_dispatch<T, TV, BOP_POST>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_MGR_RESTRICT: bchunk_dispatch<T, TV, BOP_MGR_RESTRICT>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_MGR_INTERP: bchunk_dispatch<T, TV, BOP_MGR_INTERP>(jobs, prefix, njobs, total, R, js, s); break;
        default: break;
    }
}

template <>
void launch_bchunk<double, double>(int op, const BJob *jobs, const long long *prefix, int njobs,
                                   long long total, int R, int js, cudaStream_t s) {
    switch (op) {
        case BOP_RESID: bchunk_dispatch<double, double, BOP_RESID>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_RESTRICT: bchunk_dispatch<double, double, BOP_RESTRICT>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_PROLONG: bchunk_dispatch<double, double, BOP_PROLONG>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_POST: bchunk_dispatch<double, double, BOP_POST>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_MGR_RESTRICT: bchunk_dispatch<double, double, BOP_MGR_RESTRICT>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_MGR_INTERP: bchunk_dispatch<double, double, BOP_MGR_INTERP>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_OUTER_CSR: bchunk_dispatch<double, double, BOP_OUTER_CSR>(jobs, prefix, njobs, total, R, js, s); break;
        default: break;
    }
}

static inline unsigned elem_grid(long long total) {
    long long g = (total + 255) / 256;
    if (g > NUM_SMS * 8) g = NUM_SMS * 8;
    return (unsigned)(g < 1 ? 1 : g);
}

// z_F = omega D^{-1} v_F (first F-relaxation sweep), per system
template <class T, class TV>
__global__ void k_bfrelax_first(const BJob *jobs, const long long *prefix, int njobs, T omega, int js) {
    pdl_wait();
    pdl_launch_dependents();
    const long long total = prefix[njobs];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const int f = (int)(g - prefix[j]);
        const TV *v = (const TV *)J.r + js * J.sr;
        const T *dinv = (const T *)J.d;
        const int gst = J.gs[f], k = J.gz[f];
        T s = (T)0;
        for (int q = 0; q < k; q++) s += dinv[(long long)f * 4 + q] * (T)v[J.idx[gst + q]];
        ((T *)J.o1)[f] = omega * s;
    }
}

template <class T, class TV>
void launch_bfrelax_first(const BJob *jobs, const long long *prefix, int njobs, long long total,
                          T omega, int js, cudaStream_t s) {
    if (total > 0) launch_plain(k_bfrelax_first<T, TV>, dim3(elem_grid(total)), dim3(256), s, jobs, prefix, njobs, omega, js);
}

// z[cidx[i]] = e_C[i], per system
template <class T, class TV>
__global__ void k_bscatter(const BJob *jobs, const long long *prefix, int njobs, int js) {
    pdl_wait();
    pdl_launch_dependents();
    const long long total = prefix[njobs];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const int i = (int)(g - prefix[j]);
        ((TV *)J.o1 + js * J.so1)[J.idx[i]] = (TV)((const T *)J.x)[i];
    }
}

template <class T, class TV>
void launch_bscatter(const BJob *jobs, const long long *prefix, int njobs, long long total, int js,
                     cudaStream_t s) {
    if (total > 0) launch_plain(k_bscatter<T, TV>, dim3(elem_grid(total)), dim3(256), s, jobs, prefix, njobs, js);
}

// coarsest dense solves: one warp per row over every system's coarsest grid
template <class TV>
__global__ void k_bdense(const BJob *jobs, const long long *prefix, int njobs, int js) {
    pdl_wait();
    pdl_launch_dependents();
    const long long total = prefix[njobs];
    const int lane = threadIdx.x & 31;
    for (long long g = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; g < total;
         g += ((long long)gridDim.x * blockDim.x) >> 5) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const int row = (int)(g - prefix[j]), n = J.n;
        const double *inv = (const double *)J.v;
        const TV *r = (const TV *)J.r;
        double s = 0.0;
        for (int c = lane; c < n; c += 32) s = fma(inv[(long long)row * n + c], (double)r[c], s);
        s = group_sum<32, double>(s);
        if (lane == 0) ((TV *)J.o1)[row] = (TV)s;
    }
}

template <class TV>
void launch_bdense(const BJob *jobs, const long long *prefix, int njobs, long long total, int js,
                   cudaStream_t s) {
    if (total <= 0) return;
    long long g = (total * 32 + 255) / 256;
    if (g > NUM_SMS * 8) g = NUM_SMS * 8;
    launch_plain(k_bdense<TV>, dim3((unsigned)(g < 1 ? 1 : g)), dim3(256), s, jobs, prefix, njobs, js);
}

// outer block-CSR product (b > 1), one thread per scalar row; r != null: residual
template <int B>
__global__ void k_bbsr(const BJob *jobs, const long long *prefix, int njobs, int js) {
    pdl_wait();
    pdl_launch_dependents();
    const long long total = prefix[njobs];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const long long t = g - prefix[j];
        const int I = (int)(t / B), r = (int)(t % B);
        const double *x = (const double *)J.x + js * J.sx;
        const double *val = (const double *)J.v;
        double s = 0.0;
        const int p1 = __ldg(J.rp + I + 1);
        for (int p = __ldg(J.rp + I); p < p1; p++) {
            const int Jc = __ldg(J.ci + p);
            const double *blk = val + ((long long)p * B + r) * B;
#pragma unroll
            for (int c = 0; c < B; c++) s = fma(__ldg(blk + c), __ldg(x + (long long)Jc * B + c), s);
        }
        double *y = (double *)J.o1 + js * J.so1;
        y[t] = J.r ? ((const double *)J.r)[t] - s : s;
    }
}

void launch_bbsr(int b, const BJob *jobs, const long long *prefix, int njobs, long long total, int js,
                 cudaStream_t s) {
    if (total <= 0) return;
    unsigned g = elem_grid(total);
    switch (b) {
        case 2: launch_plain(k_bbsr<2>, dim3(g), dim3(256), s, jobs, prefix, njobs, js); break;
        case 3: launch_plain(k_bbsr<3>, dim3(g), dim3(256), s, jobs, prefix, njobs, js); break;
        default: launch_plain(k_bbsr<4>, dim3(g), dim3(256), s, jobs, prefix, njobs, js); break;
    }
}

// y = x / scale or x * scale, per system (scale a device scalar in J.d)
__global__ void k_bscale(const BJob *jobs, const long long *prefix, int njobs, int js, int invert) {
    pdl_wait();
    pdl_launch_dependents();
    const long long total = prefix[njobs];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const long long e = g - prefix[j];
        const double sc = *(const double *)J.d;
        const double f = invert ? 1.0 / sc : sc;
        ((double *)J.o1 + js * J.so1)[e] = ((const double *)J.x + js * J.sx)[e] * f;
    }
}

void launch_bscale(const BJob *jobs, const long long *prefix, int njobs, long long total, int js,
                   int invert, cudaStream_t s) {
    if (total > 0) launch_plain(k_bscale, dim3(elem_grid(total)), dim3(256), s, jobs, prefix, njobs, js, invert);
}

// x += sum_{i < k} y_i Z_i per system (k in *J.gz, y in J.r, Z in J.v, x in J.o1)
__global__ void k_bmulti_axpy(const BJob *jobs, const long long *prefix, int njobs) {
    pdl_wait();
    pdl_launch_dependents();
    const long long total = prefix[njobs];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        const long long e = g - prefix[j];
        const int k = *J.gz;
        const double *Z = (const double *)J.v, *y = (const double *)J.r;
        double s = ((double *)J.o1)[e];
        for (int i = 0; i < k; i++) s += y[i] * Z[(long long)i * J.n + e];
        ((double *)J.o1)[e] = s;
    }
}

void launch_bmulti_axpy(const BJob *jobs, const long long *prefix, int njobs, long long total,
                        cudaStream_t s) {
    if (total > 0) launch_plain(k_bmulti_axpy, dim3(elem_grid(total)), dim3(256), s, jobs, prefix, njobs);
}

// Segmented Arnoldi projections: the blocks of system j are blocks
// bprefix[j] .. bprefix[j+1]-1; h_j[i] = V_j,i . w_j for i < K, reduced by
// the system's own last block.  conditional: skip systems with *flag == 0.
template <int K>
__global__ void __launch_bounds__(RED_THREADS) k_bdots(const BJob *jobs, const long long *bprefix,
                                                       int njobs, int js, int conditional,
                                                       int sqrt_out) {
    pdl_wait();
    pdl_launch_dependents();
    const int j = find_job(bprefix, njobs, blockIdx.x);
    const BJob &J = jobs[j];
    if (job_off(J)) return;
    if (conditional && *J.flag == 0) return;
    const int b = (int)(blockIdx.x - bprefix[j]), nblk = J.nblk;
    const long long n = J.n;
    const double *V = (const double *)J.v;
    const double *w = (const double *)J.x + js * J.sx;
    double acc[K];
#pragma unroll
    for (int i = 0; i < K; i++) acc[i] = 0.0;
    const long long stride = (long long)nblk * RED_THREADS * RED_EPT;
    for (long long e0 = (long long)b * RED_THREADS * RED_EPT + threadIdx.x; e0 < n; e0 += stride) {
        double wv[RED_EPT];
#pragma unroll
        for (int u = 0; u < RED_EPT; u++) {
            long long e = e0 + (long long)u * RED_THREADS;
            wv[u] = e < n ? __ldg(w + e) : 0.0;
        }
#pragma unroll
        for (int i = 0; i < K; i++)
#pragma unroll
            for (int u = 0; u < RED_EPT; u++) {
                long long e = e0 + (long long)u * RED_THREADS;
                if (e < n) acc[i] = fma(__ldg(V + i * n + e), wv[u], acc[i]);
            }
    }
    // block partial
    __shared__ double sh[RED_THREADS / 32][K];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < K; i++) {
        double v = group_sum<32, double>(acc[i]);
        if (lane == 0) sh[wq][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int ww = 0; ww < RED_THREADS / 32; ww++) t += sh[ww][threadIdx.x];
        J.partial[(long long)b * K + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(J.ticket, 1u) == (unsigned)(nblk - 1);
    __syncthreads();
    if (!last) return;
    double *h = (double *)J.o1;
    for (int i = wq; i < K; i += RED_THREADS / 32) {
        double t = 0.0;
        for (int bb = lane; bb < nblk; bb += 32) t += __ldcg(J.partial + (long long)bb * K + i);
        t = group_sum<32, double>(t);
        if (lane == 0) h[i] = sqrt_out ? sqrt(t) : t;
    }
    __syncthreads();
    if (threadIdx.x == 0) *J.ticket = 0u;
}

// Segmented w <- w - V h ; |w|^2 (mode 1 decides *flag, mode 2 skipped when
// *flag == 0).  h in J.r, nrm2 out in J.o2.
template <int K>
__global__ void __launch_bounds__(RED_THREADS) k_bupdate_norm(const BJob *jobs, const long long *bprefix,
                                                              int njobs, int js, int mode) {
    pdl_wait();
    pdl_launch_dependents();
    const int j = find_job(bprefix, njobs, blockIdx.x);
    const BJob &J = jobs[j];
    if (job_off(J)) return;
    if (mode == 2 && *J.flag == 0) return;
    const int b = (int)(blockIdx.x - bprefix[j]), nblk = J.nblk;
    const long long n = J.n;
    const double *V = (const double *)J.v;
    double *w = (double *)J.x + js * J.sx;
    const double *h = (const double *)J.r;
    double hs[K];
#pragma unroll
    for (int i = 0; i < K; i++) hs[i] = h[i];
    double acc = 0.0;
    const long long stride = (long long)nblk * RED_THREADS * RED_EPT;
    for (long long e0 = (long long)b * RED_THREADS * RED_EPT + threadIdx.x; e0 < n; e0 += stride) {
        double wv[RED_EPT];
#pragma unroll
        for (int u = 0; u < RED_EPT; u++) {
            long long e = e0 + (long long)u * RED_THREADS;
            wv[u] = e < n ? w[e] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < K; i++)
#pragma unroll
            for (int u = 0; u < RED_EPT; u++) {
                long long e = e0 + (long long)u * RED_THREADS;
                if (e < n) wv[u] = fma(-__ldg(V + i * n + e), hs[i], wv[u]);
            }
#pragma unroll
        for (int u = 0; u < RED_EPT; u++) {
            long long e = e0 + (long long)u * RED_THREADS;
            if (e < n) { w[e] = wv[u]; acc = fma(wv[u], wv[u], acc); }
        }
    }
    __shared__ double sh[RED_THREADS / 32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    acc = group_sum<32, double>(acc);
    if (lane == 0) sh[wq] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int ww = 0; ww < RED_THREADS / 32; ww++) t += sh[ww];
        J.partial[b] = t;
        __threadfence();
        last = atomicAdd(J.ticket, 1u) == (unsigned)(nblk - 1);
    }
    __syncthreads();
    if (!last || wq != 0) return;
    double t = 0.0;
    for (int bb = lane; bb < nblk; bb += 32) t += __ldcg(J.partial + bb);
    t = group_sum<32, double>(t);
    if (lane == 0) {
        double *nrm2 = (double *)J.o2;
        *nrm2 = t;
        if (mode == 1) *J.flag = (t < REORTH_ETA2 * h[K]) ? 1 : 0;
        *J.ticket = 0u;
    }
}

void launch_bdots(int k, const BJob *jobs, const long long *bprefix, int njobs, long long nblocks,
                  int js, int conditional, int sqrt_out, cudaStream_t s) {
    if (nblocks <= 0) return;
    unsigned g = (unsigned)nblocks;
    switch (k) {
#define X(K) case K: launch_plain(k_bdots<K>, dim3(g), dim3(RED_THREADS), s, jobs, bprefix, njobs, js, conditional, sqrt_out); break;
        K_CASES(X)
#undef X
        default: break;
    }
}

void launch_bupdate_norm(int k, const BJob *jobs, const long long *bprefix, int njobs,
                         long long nblocks, int js, int mode, cudaStream_t s) {
    if (nblocks <= 0) return;
    unsigned g = (unsigned)nblocks;
    switch (k) {
#define X(K) case K: launch_plain(k_bupdate_norm<K>, dim3(g), dim3(RED_THREADS), s, jobs, bprefix, njobs, js, mode); break;
        K_CASES(X)
#undef X
        default: break;
    }
}

template void launch_bchunk<float, float>(int, const BJob *, const long long *, int, long long, int, int, cudaStream_t);
template void launch_bchunk<float, double>(int, const BJob *, const long long *, int, long long, int, int, cudaStream_t);
template void launch_bfrelax_first<double, double>(const BJob *, const long long *, int, long long, double, int, cudaStream_t);
template void launch_bfrelax_first<float, double>(const BJob *, const long long *, int, long long, float, int, cudaStream_t);
template void launch_bfrelax_first<float, float>(const BJob *, const long long *, int, long long, float, int, cudaStream_t);
template void launch_bscatter<double, double>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bscatter<float, double>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bscatter<float, float>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bdense<double>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bdense<float>(const BJob *, const long long *, int, long long, int, cudaStream_t);

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
    template void launch_amg_smooth0_residual<T, TV>(const DCSR &, const T *, const T *,          \
                                                     const TV *, T *, T *, cudaStream_t);         \
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
template void launch_copy_cast<double>(const double *, double *, int, cudaStream_t);
template void launch_copy_cast<float>(const float *, double *, int, cudaStream_t);

}  // namespace mgr
