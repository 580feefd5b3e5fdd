// Fused AMG tail: the small coarse levels of the AMG V(1,1) cycle and the
// coarsest dense solve in one launch of a single thread-block cluster.
//
// On the small levels every separate kernel costs a launch, a ramp and a
// drain for a few microseconds of work.  Here the cluster's warps stride over
// each phase's SELL slices and the phases meet at hardware cluster barriers
// (release/acquire, no spin waits).  The phase list lives in device memory
// (built at setup).  Vectors written inside the launch are
// read through L2 (ld.global.cg), so no SM sees a stale L1 line of another
// SM's result; matrices and diagonals are read-only.  Each row sum and each
// epilogue is the same operation sequence as in the per-level kernels
// (sell.cuh and the epilogues of solve.cu), so the result is bitwise the
// one the per-level kernels give.
#include <cuda_runtime.h>

#include "common.cuh"
#include "sell.cuh"

namespace mgr {

static constexpr int TAIL_THREADS = 512;

template <class T>
struct XCg {
    const T *x;
    __device__ __forceinline__ T operator()(int j) const { return __ldcg(x + j); }
};

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ int cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
__device__ __forceinline__ int cluster_ctas() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return (int)r;
}

// one phase: every slice of M, the cluster's warps striding over them.  G is
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
// EAdd and EPost in solve.cu
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
__global__ void __launch_bounds__(TAIL_THREADS, 1) k_amg_tail(const TailPlan *__restrict__ plan) {
    pdl_wait();
    pdl_launch_dependents();
    const int lane = threadIdx.x & 31;
    const int gw = cluster_rank() * (TAIL_THREADS / 32) + (int)(threadIdx.x >> 5);
    const int W = cluster_ctas() * (TAIL_THREADS / 32);
    const int np = plan->nphase;
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
        if (p + 1 < np) cluster_barrier();
    }
}

template <class T>
int launch_amg_tail(const TailPlan *plan, int cluster, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster);
    cfg.blockDim = dim3(TAIL_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_on() ? 2 : 1;
    return (int)cudaLaunchKernelEx(&cfg, k_amg_tail<T>, plan);
}

template <class T>
static bool tail_fits(int cl) {
    if (cl > 8 && cudaFuncSetAttribute(k_amg_tail<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess)
        return false;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl);
    cfg.blockDim = dim3(TAIL_THREADS);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_amg_tail<T>, &cfg) != cudaSuccess) return false;
    return nc >= 1;
}

int amg_tail_cluster(void) {
    static int cached[64];
    static bool known[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!known[dev]) {
        int cl = 0;
        for (int c : {16, 8})
            if (tail_fits<double>(c) && tail_fits<float>(c)) {
                cl = c;
                break;
            }
        cudaGetLastError();  // a refused size leaves no error behind
        cached[dev] = cl;
        known[dev] = true;
    }
    return cached[dev];
}

template int launch_amg_tail<double>(const TailPlan *, int, cudaStream_t);
template int launch_amg_tail<float>(const TailPlan *, int, cudaStream_t);

}  // namespace mgr
