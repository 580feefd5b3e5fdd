// Batched form: one launch per kernel class over every system of a batch.
#include <cuda_runtime.h>

#include "common.cuh"
#include "reduce.cuh"
#include "spmv.cuh"

namespace mgr {

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
template <class T, class TV> struct BOpT<T, TV, BOP_FRELAX_RESID> {  // r_F = v[fidx] - A_FF z_F
    __device__ static XPlain<T, T> xf(const BJob &J, int) { return {(const T *)J.x}; }
    __device__ static EGatherMinus<T, TV> epi(const BJob &J, int js) {
        return {J.idx, (const TV *)J.r + js * J.sr, (T)-1, (T *)J.o1};
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
        case BOP_FRELAX_RESID: bchunk_dispatch<T, TV, BOP_FRELAX_RESID>(jobs, prefix, njobs, total, R, js, s); break;
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
        case BOP_FRELAX_RESID: bchunk_dispatch<double, double, BOP_FRELAX_RESID>(jobs, prefix, njobs, total, R, js, s); break;
        case BOP_OUTER_CSR: bchunk_dispatch<double, double, BOP_OUTER_CSR>(jobs, prefix, njobs, total, R, js, s); break;
        default: break;
    }
}

// SELL row products of a batch: work item g is one slice of one member's
// matrix; each member keeps its own lanes per row (sg) and layout, and a
// row's sum is the chain and tree of the single-system kernel (sell.cuh), so
// a member's products give the bits its own handle gives.
template <class T, class TV, int OP>
__global__ void __launch_bounds__(256) k_bsell(const BJob *__restrict__ jobs,
                                               const long long *__restrict__ prefix, int njobs,
                                               int js) {
    pdl_wait();
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long total = prefix[njobs];
    for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < total; g += nwarps) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const int sl = (int)(g - prefix[j]);
        const int G = J.sg, C = 32 / G;
        const int L = __ldg(J.slen + sl);
        const long long base = __ldg(J.sptr + sl) + lane;
        const int row = __ldg(J.perm + (long long)sl * C + lane / G);
        const auto xf = BOpT<T, TV, OP>::xf(J, js);
        const auto epi = BOpT<T, TV, OP>::epi(J, js);
        T acc = sell_chain<T>(L, base, J.sci, (const T *)J.sv, xf);
        if (G > 1) acc = group_sum_rt<T>(acc, G);
        if (lane % G == 0 && row >= 0) epi(row, acc);
    }
}

template <class T, class TV, int OP>
static void bsell_dispatch(const BJob *jobs, const long long *prefix, int njobs, long long total, int js,
                           cudaStream_t s) {
    if (total <= 0) return;
    long long blocks = (total + 7) / 8;
    if (blocks > NUM_SMS * 16) blocks = NUM_SMS * 16;
    launch_plain(k_bsell<T, TV, OP>, dim3((unsigned)(blocks < 1 ? 1 : blocks)), dim3(256), s, jobs, prefix,
                 njobs, js);
}

template <class T, class TV>
void launch_bsell(int op, const BJob *jobs, const long long *prefix, int njobs, long long total, int js,
                  cudaStream_t s) {
    switch (op) {
        case BOP_RESID: bsell_dispatch<T, TV, BOP_RESID>(jobs, prefix, njobs, total, js, s); break;
        case BOP_RESTRICT: bsell_dispatch<T, TV, BOP_RESTRICT>(jobs, prefix, njobs, total, js, s); break;
        case BOP_PROLONG: bsell_dispatch<T, TV, BOP_PROLONG>(jobs, prefix, njobs, total, js, s); break;
        case BOP_POST: bsell_dispatch<T, TV, BOP_POST>(jobs, prefix, njobs, total, js, s); break;
        case BOP_MGR_RESTRICT: bsell_dispatch<T, TV, BOP_MGR_RESTRICT>(jobs, prefix, njobs, total, js, s); break;
        case BOP_MGR_INTERP: bsell_dispatch<T, TV, BOP_MGR_INTERP>(jobs, prefix, njobs, total, js, s); break;
        case BOP_FRELAX_RESID: bsell_dispatch<T, TV, BOP_FRELAX_RESID>(jobs, prefix, njobs, total, js, s); break;
        default: break;
    }
}

template <>
void launch_bsell<double, double>(int op, const BJob *jobs, const long long *prefix, int njobs,
                                  long long total, int js, cudaStream_t s) {
    switch (op) {
        case BOP_RESID: bsell_dispatch<double, double, BOP_RESID>(jobs, prefix, njobs, total, js, s); break;
        case BOP_RESTRICT: bsell_dispatch<double, double, BOP_RESTRICT>(jobs, prefix, njobs, total, js, s); break;
        case BOP_PROLONG: bsell_dispatch<double, double, BOP_PROLONG>(jobs, prefix, njobs, total, js, s); break;
        case BOP_POST: bsell_dispatch<double, double, BOP_POST>(jobs, prefix, njobs, total, js, s); break;
        case BOP_MGR_RESTRICT: bsell_dispatch<double, double, BOP_MGR_RESTRICT>(jobs, prefix, njobs, total, js, s); break;
        case BOP_MGR_INTERP: bsell_dispatch<double, double, BOP_MGR_INTERP>(jobs, prefix, njobs, total, js, s); break;
        case BOP_FRELAX_RESID: bsell_dispatch<double, double, BOP_FRELAX_RESID>(jobs, prefix, njobs, total, js, s); break;
        case BOP_OUTER_CSR: bsell_dispatch<double, double, BOP_OUTER_CSR>(jobs, prefix, njobs, total, js, s); break;
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

// gather of the F-relaxation input v_F (o1 = r[idx]) with the seed of the
// F hierarchy's pre-smoothing (o2 = d .* v_F); idx null reads r itself, o1
// null skips the store (the seed of the final AMG after the Z product)
template <class T, class TV>
__global__ void k_bgather(const BJob *jobs, const long long *prefix, int njobs, int js) {
    pdl_wait();
    pdl_launch_dependents();
    const long long total = prefix[njobs];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const int i = (int)(g - prefix[j]);
        const TV *r = (const TV *)J.r + js * J.sr;
        const T v = (T)r[J.idx ? J.idx[i] : i];
        if (J.o1) ((T *)J.o1)[i] = v;
        if (J.d) ((T *)J.o2)[i] = ((const T *)J.d)[i] * v;
    }
}

template <class T, class TV>
void launch_bgather(const BJob *jobs, const long long *prefix, int njobs, long long total, int js,
                    cudaStream_t s) {
    if (total > 0) launch_plain(k_bgather<T, TV>, dim3(elem_grid(total)), dim3(256), s, jobs, prefix, njobs, js);
}

__device__ __forceinline__ double bmul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float bmul_rn(float a, float b) { return __fmul_rn(a, b); }

template <class T>
__global__ void k_bomega(const BJob *jobs, const long long *prefix, int njobs, T omega) {
    pdl_wait();
    pdl_launch_dependents();
    const long long total = prefix[njobs];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const int i = (int)(g - prefix[j]);
        ((T *)J.o1)[i] = bmul_rn(omega, ((const T *)J.x)[i]);
    }
}

template <class T>
void launch_bomega(const BJob *jobs, const long long *prefix, int njobs, long long total, T omega,
                   cudaStream_t s) {
    if (total > 0) launch_plain(k_bomega<T>, dim3(elem_grid(total)), dim3(256), s, jobs, prefix, njobs, omega);
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

// y = x * (1/scale) or x * scale, per system (scale a device scalar in J.d).
// Each block forms the systems' factors once (up to BSCALE_CACHE systems):
// an FP64 division per element would cost more FP64 issue than the pass.
static constexpr int BSCALE_CACHE = 1024;
__global__ void k_bscale(const BJob *jobs, const long long *prefix, int njobs, int js, int invert) {
    __shared__ double fs[BSCALE_CACHE];
    pdl_wait();
    pdl_launch_dependents();
    const bool cached = njobs <= BSCALE_CACHE;
    if (cached)
        for (int j = threadIdx.x; j < njobs; j += blockDim.x) {
            const BJob &J = jobs[j];
            if (job_off(J)) continue;
            const double sc = *(const double *)J.d;
            fs[j] = invert ? 1.0 / sc : sc;
        }
    __syncthreads();
    const long long total = prefix[njobs];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        const int j = find_job(prefix, njobs, g);
        const BJob &J = jobs[j];
        if (job_off(J)) continue;
        const long long e = g - prefix[j];
        double f;
        if (cached) f = fs[j];
        else {
            const double sc = *(const double *)J.d;
            f = invert ? 1.0 / sc : sc;
        }
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
template void launch_bsell<float, float>(int, const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bsell<float, double>(int, const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bfrelax_first<double, double>(const BJob *, const long long *, int, long long, double, int, cudaStream_t);
template void launch_bfrelax_first<float, double>(const BJob *, const long long *, int, long long, float, int, cudaStream_t);
template void launch_bfrelax_first<float, float>(const BJob *, const long long *, int, long long, float, int, cudaStream_t);
template void launch_bscatter<double, double>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bscatter<float, double>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bscatter<float, float>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bgather<double, double>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bgather<float, double>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bgather<float, float>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bomega<double>(const BJob *, const long long *, int, long long, double, cudaStream_t);
template void launch_bomega<float>(const BJob *, const long long *, int, long long, float, cudaStream_t);
template void launch_bdense<double>(const BJob *, const long long *, int, long long, int, cudaStream_t);
template void launch_bdense<float>(const BJob *, const long long *, int, long long, int, cudaStream_t);

}  // namespace mgr
