// Fused AMG tail: the small coarse levels of the AMG V(1,1) cycle and the
// coarsest dense solve in one cooperative launch over the whole GPU.
//
// On the small levels every separate kernel costs a launch, a ramp and a
// drain for a few microseconds of work.  Here the grid's warps stride over
// each phase's SELL slices and the phases meet at grid-wide barriers (all
// CTAs are co-resident by the cooperative launch; a barrier's wait is bounded
// and a wait that runs out sets an error word and ends the launch).  The
// phase list lives in device memory (built at setup).  Vectors written inside
// the launch are read through L2 (ld.global.cg), so no SM sees a stale L1
// line of another SM's result; matrices and diagonals are read-only.  Each
// row sum and each epilogue is the same operation sequence as in the
// per-level kernels (sell.cuh and the epilogues of spmv.cuh), so the result
// is bitwise the one the per-level kernels give.
#include <cuda_runtime.h>

#include "common.cuh"
#include "sell.cuh"

namespace mgr {

static constexpr int TAIL_THREADS = 512;
static constexpr long long TAIL_SPIN = 1LL << 23;  // ~0.5 s of 32 ns sleeps

template <class T>
struct XCg {
    const T *x;
    __device__ __forceinline__ T operator()(int j) const { return __ldcg(x + j); }
};

// Grid-wide barrier.  sync[0]: arrivals, sync[1]: generation, sync[2]: error.
// Each CTA reads the generation before it arrives (it cannot move before
// this CTA's arrival); the last arrival resets the count and advances the
// generation; the others poll it.  false: this CTA must stop (a wait ran out
// here or elsewhere).
__device__ __forceinline__ bool grid_barrier(unsigned *sync, long long spin) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = sync + 1;
        volatile unsigned *err = sync + 2;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(sync, 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x) {
            atomicExch(sync, 0u);
            __threadfence();
            atomicAdd(sync + 1, 1u);
        } else {
            long long i = 0;
            while (*gen == g) {
                if (++i > spin || *err) {
                    ok = 0;
                    atomicOr(sync + 2, 1u);
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok_s = ok && *err == 0;
    }
    __syncthreads();
    return ok_s != 0;
}

// one phase: every slice of M, the grid's warps striding over them.  G is
// a run-time value here (one loop per phase kind instead of one per lane
// count); the chain and the tree are those of sell_rows.
template <class T, class F>
__device__ __forceinline__ void tail_phase(const SellView &M, const T *x, const F &fin, int gw, int W,
                                           int lane) {
    const XCg<T> xf{x};
    const T *sv = (const T *)M.sv;
    const int G = M.sg, C = 32 / G;
    for (int sl = gw; sl < M.nsl; sl += W) {
        const int L = __ldg(M.slen + sl);
        const long long base = __ldg(M.sptr + sl) + lane;
        T acc = sell_chain<T>(L, base, M.sci, sv, xf);
        if (G > 1) acc = group_sum_rt<T>(acc, G);
        const int row = __ldg(M.perm + (long long)sl * C + lane / G);
        if (lane % G == 0 && row >= 0) fin(row, acc);
    }
}

// phase epilogues: the operation sequences of EResid, EStoreScaled, EStore,
// EAdd and EPost in spmv.cuh
template <class T>
struct FResid {  // res = r - s
    const T *r;
    T *res;
    __device__ __forceinline__ void operator()(int row, T s) const { res[row] = __ldcg(r + row) - s; }
};
template <class T>
struct FRestrictScaled {  // r_c = s ; xw_c = d_c s
    T *rc, *xwc;
    const T *dc;
    __device__ __forceinline__ void operator()(int row, T s) const {
        rc[row] = s;
        xwc[row] = __ldg(dc + row) * s;
    }
};
template <class T>
struct FStore {
    T *y;
    __device__ __forceinline__ void operator()(int row, T s) const { y[row] = s; }
};
template <class T>
struct FAdd {  // xw += s
    T *y;
    __device__ __forceinline__ void operator()(int row, T s) const { y[row] = __ldcg(y + row) + s; }
};
template <class T>
struct FPost {  // x = xw + d (r - s)
    const T *r, *d, *xw;
    T *x;
    __device__ __forceinline__ void operator()(int row, T s) const {
        x[row] = fma(__ldg(d + row), __ldcg(r + row) - s, __ldcg(xw + row));
    }
};

template <class T>
__global__ void __launch_bounds__(TAIL_THREADS, 1) k_amg_tail(const TailPlan *__restrict__ plan, unsigned *sync) {
    const int lane = threadIdx.x & 31;
    const int gw = (int)blockIdx.x * (TAIL_THREADS / 32) + (int)(threadIdx.x >> 5);
    const int W = (int)gridDim.x * (TAIL_THREADS / 32);
    const int np = plan->nphase;
    const long long spin = plan->spin > 0 ? plan->spin : TAIL_SPIN;
    for (int p = 0; p < np; p++) {
        const TailPhase &P = plan->ph[p];
        const int kind = P.kind;
        if (kind == TAIL_DENSE) {
            // coarsest: x = A^{-1} r, one warp per row (the order of k_dense_matvec)
            const int n = P.n;
            const double *inv = P.inv;
            const T *r = (const T *)P.x;
            T *x = (T *)P.y;
            for (int row = gw; row < n; row += W) {
                double s = 0.0;
                for (int c = lane; c < n; c += 32) s = fma(__ldg(inv + (long long)row * n + c), (double)__ldcg(r + c), s);
                s = group_sum<32, double>(s);
                if (lane == 0) x[row] = (T)s;
            }
        } else {
            const SellView M = P.M;
            const T *x = (const T *)P.x;
            switch (kind) {
                case TAIL_RESID: tail_phase<T>(M, x, FResid<T>{(const T *)P.r, (T *)P.y}, gw, W, lane); break;
                case TAIL_RESTRICT_SCALED:
                    tail_phase<T>(M, x, FRestrictScaled<T>{(T *)P.y, (T *)P.y2, (const T *)P.d}, gw, W, lane);
                    break;
                case TAIL_RESTRICT: tail_phase<T>(M, x, FStore<T>{(T *)P.y}, gw, W, lane); break;
                case TAIL_PROLONG: tail_phase<T>(M, x, FAdd<T>{(T *)P.y}, gw, W, lane); break;
                default:
                    tail_phase<T>(M, x, FPost<T>{(const T *)P.r, (const T *)P.d, x, (T *)P.y}, gw, W, lane);
                    break;
            }
        }
        if (p + 1 < np && !grid_barrier(sync, spin)) return;
    }
}

template <class T>
int launch_amg_tail(const TailPlan *plan, int grid, unsigned *sync, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(TAIL_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, k_amg_tail<T>, plan, sync);
}

int amg_tail_grid(void) {
    static int cached[64];
    static bool known[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!known[dev]) {
        int coop = 0, sms = 0, b64 = 0, b32 = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_amg_tail<double>, TAIL_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_amg_tail<float>, TAIL_THREADS, 0);
        cudaGetLastError();
        const int b = b64 < b32 ? b64 : b32;
        cached[dev] = (coop && b >= 1) ? sms * b : 0;
        known[dev] = true;
    }
    return cached[dev];
}

template int launch_amg_tail<double>(const TailPlan *, int, unsigned *, cudaStream_t);
template int launch_amg_tail<float>(const TailPlan *, int, unsigned *, cudaStream_t);

}  // namespace mgr
