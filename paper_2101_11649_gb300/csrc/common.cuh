// Internal declarations shared by the CUDA translation units of the MGR
// library.  Nothing here is part of the public C ABI (include/mgr_gb300.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

namespace mgr {

// Scalar CSR on the device.  Columns strictly ascending per row.  v32 is an
// optional FP32 copy of the values (FP32 V-cycle).
struct DCSR {
    int n = 0, m = 0;
    int nnz = 0;
    int *rp = nullptr, *ci = nullptr;
    double *v = nullptr;
    float *v32 = nullptr;
    // SELL-C-sigma copy for the solve phase (null when not built): rows
    // sorted by length inside windows of 1024, cut into slices of C = 32/sg
    // rows; each row gets sg lanes of a warp.  A slice is stored as steps of
    // 32 contiguous entries: entry t*sg + g of the slice's row r sits at
    // step t, position r*sg + g; rows are padded with zero values to the
    // slice's longest row.
    int nsl = 0;
    int sg = 1;                  // lanes per row (power of two, <= 32)
    long long *sptr = nullptr;   // [nsl+1] slice offsets
    int *slen = nullptr;         // [nsl] slice widths in steps of 32 entries
    int *perm = nullptr;         // [nsl*32/sg] row of each slice row (-1: none)
    int *sci = nullptr;          // padded column indices
    double *sv = nullptr;        // padded values (FP64)
    float *sv32 = nullptr;       // padded values (FP32)
    long long sell_stored = 0;   // stored entries including padding
    int sched = 0;               // SELL product form: bit 0 slice order (0 grid-stride, 1 contiguous per
                                 // block), bit 1 the pipelined FP64 chain
};


// Programmatic dependent launch.  Solve-phase kernels are launched with
// programmatic stream serialisation: a kernel may be scheduled while its
// predecessor drains; it waits (griddepcontrol.wait) before it reads or
// writes memory that earlier kernels touch, then lets its own successor be
// scheduled.  A kernel started without the attribute passes both at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
bool pdl_on();  // false when the environment sets MGR_PDL=0
// The batched form's kernels are launched in plain stream order: with many
// systems per launch, early scheduling of the successor measured slower.
template <class... KArgs, class... Args>
inline void launch_plain(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
template <class... KArgs, class... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_on() ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Status codes mirror mgr_status.
enum { ST_OK = 0, ST_INVALID = 1, ST_NOMEM = 2, ST_CUDA = 3, ST_SINGULAR = 4,
       ST_NOT_CONVERGED = 5, ST_TIMEOUT = 6, ST_UNSUPPORTED = 7 };

// Device error word bits written by setup kernels.
enum { ERRW_SINGULAR = 1, ERRW_INVALID = 2, ERRW_OVERFLOW = 4 };

// Device memory of one owner.  Released blocks stay in a pool and serve
// later requests of about the same size (all work of an owner runs on one
// stream, so stream order protects a reused block); recycle() returns every
// block to the pool, trim() frees the pooled blocks (cudaFree).
struct Arena {
    std::vector<std::pair<void *, size_t>> blocks;  // live
    std::multimap<size_t, void *> pool;             // released, kept for reuse
    size_t bytes = 0;
    int status = ST_OK;
    void *get(size_t nbytes);
    template <class T> T *alloc(size_t count) { return (T *)get(count * sizeof(T)); }
    void release(void *p);
    void recycle();
    void trim();
    void free_all();
};

// A SELL-C-sigma matrix as the fused coarse-level kernel reads it (values of
// that kernel's precision).
struct SellView {
    int nsl = 0, sg = 1;
    const long long *sptr = nullptr;
    const int *slen = nullptr, *perm = nullptr, *sci = nullptr;
    const void *sv = nullptr;
};

// Fused AMG tail: levels k_t .. k_c - 1 of an AMG V(1,1) cycle (residual,
// restriction, then after the coarsest solve prolongation and post-smoothing)
// plus the coarsest dense solve, in one cooperative launch over the GPU.
// The launch walks a list of phases built at setup; consecutive phases meet
// at a grid-wide barrier.  Vectors are of the kernel's precision T (void here).
enum { TAIL_RESID = 0, TAIL_RESTRICT_SCALED = 1, TAIL_RESTRICT = 2, TAIL_DENSE = 3, TAIL_PROLONG = 4,
       TAIL_POST = 5 };
constexpr int TAIL_MAX_PHASES = 64;
struct TailPhase {
    int kind = 0;
    int n = 0;                  // TAIL_DENSE: order of the coarsest inverse
    SellView M;                 // the phase's matrix (not TAIL_DENSE)
    const void *x = nullptr;    // gathered vector (TAIL_DENSE: r of the coarsest level)
    void *y = nullptr;          // output: res, r_c, xw (read-modify-write), x
    void *y2 = nullptr;         // TAIL_RESTRICT_SCALED: xw_c = d_c r_c
    const void *r = nullptr;    // TAIL_RESID, TAIL_POST: the level's right-hand side
    const void *d = nullptr;    // TAIL_RESTRICT_SCALED: d_c; TAIL_POST: d
    const double *inv = nullptr;  // TAIL_DENSE: coarsest inverse, row-major
};
struct TailPlan {
    int nphase = 0;
    long long spin = 0;  // polls before a barrier wait gives up (0: the default)
    TailPhase ph[TAIL_MAX_PHASES];
};
// sync: 3 device words (arrivals, generation, error), zero before the first
// launch; the error word is nonzero after a barrier wait ran out.
template <class T>
int launch_amg_tail(const TailPlan *plan_device, int grid, unsigned *sync, cudaStream_t s);
// CTAs of a cooperative tail launch (SMs x resident CTAs per SM); 0 when the
// device cannot run it (the cycle then launches the levels one at a time).
int amg_tail_grid(void);

// Slice-order tuning of a SELL product: the values' precision, a flush
// buffer larger than L2 and an event pair (owned by the caller)
constexpr int SELL_TUNE_ROUNDS = 8;  // timed launches per product (2 per form)
struct SellTune {
    int fp32 = 0;
    void *flush = nullptr;
    size_t flush_bytes = 0;
    cudaEvent_t ev[2 * SELL_TUNE_ROUNDS] = {};  // a pair around each timed launch
};
constexpr int SELL_TUNE_MIN_SLICES = 4096;
constexpr size_t SELL_TUNE_FLUSH_BYTES = 192u << 20;
// SELL-C-sigma build from the CSR arrays (values of both precisions when
// present); with tn, the product is then timed in each form (both slice
// orders; FP64 also with the pipelined chain) with the values of tn's
// precision and the fastest kept (sell_tune)
int build_sell(DCSR &M, cudaStream_t s, Arena &ar, const SellTune *tn = nullptr);
int sell_tune(DCSR &M, const SellTune &tn, cudaStream_t s, Arena &ar);
// re-copy the values of a built SELL layout after the CSR values changed
void refresh_sell(DCSR &M, cudaStream_t s);

// ------------------------------------------------------------- utilities
int scan_exclusive(const int *in, int *out, int n, cudaStream_t s, Arena &ar, int *total);
int scan_exclusive_ll(const int *in, long long *out, int n, cudaStream_t s, Arena &ar,
                      long long *total);

// ------------------------------------------------------------- setup (bit-exact with the CPU reading)
void launch_bsr_to_csr(int nb, int b, const int *rp, const int *ci, const double *val, DCSR &A,
                       cudaStream_t s);
// flags: per local row of level l, 0 = F, 1 = C, 2 = invalid (level < l)
void launch_level_flags(const int8_t *dof_level_g, const int *gdof, int n, int level, int *isF,
                        int *isC, int *err, cudaStream_t s);
void launch_index_maps(const int *isF, const int *isC, const int *fpos_ex, const int *cpos_ex,
                       int n, int *fidx, int *cidx, int *fmap, int *cmap, cudaStream_t s);
// Submatrix of A: rows ridx[0..nr), columns remapped through cmap (-1 drops).
int extract_submatrix(const DCSR &A, const int *ridx, int nr, const int *cmap, int ncols, DCSR &out,
                      cudaStream_t s, Arena &ar);
int mgr_dinv(const DCSR &AFF, const int *fidx, const int *gdof, int b, int relax, int *gstart,
             int *gsize, double *dinv, int *errw, cudaStream_t s);
int mgr_build_w(const DCSR &AFC, const int *gstart, const int *gsize, const double *dinv, DCSR &W,
                cudaStream_t s, Arena &ar);
// C = A*B (+E added last), accumulation order of the CPU reading.
int spgemm(const DCSR &A, const DCSR &B, const DCSR *E, DCSR &C, cudaStream_t s, Arena &ar);
int transpose(const DCSR &A, DCSR &T, cudaStream_t s, Arena &ar);
int amg_strength(const DCSR &A, const int *func, double theta, uint8_t *sflag, DCSR &S,
                 cudaStream_t s, Arena &ar);
int amg_pmis(const DCSR &S, const DCSR &ST, int level, int *cf, cudaStream_t s, Arena &ar);
int amg_extpi(const DCSR &A, const uint8_t *sflag, const int *cf, const int *func, int pmax,
              DCSR &P, int *nc, cudaStream_t s, Arena &ar);
int l1_inverse(const DCSR &A, double *dinv, float *dinv32, int *errw, cudaStream_t s);
void launch_coarse_func(const int *cf, const int *func, const DCSR &P, int *cfunc, int n,
                        cudaStream_t s);
void launch_iota_mod(int *func, int n, int nf, cudaStream_t s);
int dense_inverse(const DCSR &A, double *inv, int *errw, cudaStream_t s, Arena &ar);
void launch_cast_f32(const double *in, float *out, long long n, cudaStream_t s);
// src[q] = index into the BSR value array of entry q of the scalar transpose
int transpose_sources(int nb, int b, const int *brp, const int *bci, long long nnzb, int *src,
                      cudaStream_t s);
void launch_gather_f64(const int *src, const double *in, double *out, long long n, cudaStream_t s);
// structure checks (check.cu): violations are added to *bad (device)
int check_csr(const DCSR &M, unsigned long long *bad, cudaStream_t s, Arena &ar);
int check_split(int n, const int *fidx, int nF, const int *cidx, int nC, const int *gstart,
                const int *gsize, unsigned long long *bad, cudaStream_t s, Arena &ar);
int check_add(unsigned long long *bad, unsigned long long v, cudaStream_t s);
int check_iota(const int *a, int n, unsigned long long *bad, cudaStream_t s);
// 1 when the n values of a and b are bitwise equal, 0 when not, -1 on error
int same_bits(const double *a, const double *b, long long n, cudaStream_t s, Arena &ar);

// ------------------------------------------------------------- solve phase
// BSR y = alpha A x + beta y (b in 1..4) on FP64
void launch_bsr_spmv(int nb, int b, const int *rp, const int *ci, const double *val,
                     const double *x, double *y, double alpha, double beta, cudaStream_t s,
                     long long nnzb = 0);
// y = bvec - A x  (residual) or y = A x when bvec == nullptr
void launch_bsr_residual(int nb, int b, const int *rp, const int *ci, const double *val,
                         const double *x, const double *bvec, double *y, cudaStream_t s,
                         long long nnzb = 0);

// MGR level kernels, T = value/arith type, TV = type of the level's in/out vectors
template <class T, class TV>
void launch_frelax_first(int nF, const int *fidx, const int *gstart, const int *gsize,
                         const T *dinv, T omega, const TV *v, T *zF, cudaStream_t s);
template <class T, class TV>
void launch_frelax_residual(const DCSR &AFF, const T *vals, const int *fidx, const TV *v,
                            const T *zF, T *rF, cudaStream_t s);
template <class T>
void launch_frelax_update(int nF, const int *gstart, const int *gsize, const T *dinv, T omega,
                          const T *rF, T *zF, int transpose, cudaStream_t s);
template <class T, class TV>
void launch_mgr_restrict(const DCSR &ACF, const T *vals, const int *cidx, const TV *v,
                         const T *zF, T *vC, cudaStream_t s);
template <class T, class TV>
void launch_mgr_interp(const DCSR &W, const T *wvals, int nC, const int *fidx, const int *cidx,
                       const T *zF, const T *eC, TV *z, cudaStream_t s);
// transposed-cycle pieces
template <class T, class TV>
void launch_gather(const int *idx, int n, const TV *v, T *out, cudaStream_t s);
template <class T, class TV>
void launch_csr_axpy_gather(const DCSR &M, const T *vals, const T *x, const int *idx_b,
                            const TV *bsrc, T sign, T *y, cudaStream_t s);
template <class T, class TV>
void launch_scatter2(int nF, int nC, const int *fidx, const int *cidx, const T *zF, const T *eC,
                     TV *z, cudaStream_t s);

// AMG level kernels
template <class T>
void launch_csr_spmv(const DCSR &A, const T *vals, const T *x, T *y, cudaStream_t s);
template <class T>
void launch_csr_spmv_add(const DCSR &A, const T *vals, const T *x, T *y, cudaStream_t s);
template <class T, class TV>
void launch_amg_post_smooth(const DCSR &A, const T *vals, const T *dinv, const TV *r, const T *x,
                            TV *xout, cudaStream_t s);
template <class T, class TV>
void launch_amg_residual(const DCSR &A, const T *vals, const T *x, const TV *r, T *res,
                         cudaStream_t s);
template <class T>
void launch_restrict_scaled(const DCSR &R, const T *vals, const T *res, T *rc, const T *dc, T *xc,
                            cudaStream_t s);
template <class T, class TV>
void launch_mgr_restrict_scaled(const DCSR &ACF, const T *vals, const int *cidx, const TV *v,
                                const T *zF, T *vC, const T *d, T *x, cudaStream_t s);
template <class T, class TV>
void launch_scale(int n, const T *d, const TV *r, T *x, cudaStream_t s);
template <class TV>
void launch_dense_matvec(int n, const double *inv, const TV *r, TV *x, cudaStream_t s);

// Krylov pieces (FP64); reductions finish in their last block (ticket)
void launch_vec_scale(const double *x, double *y, const double *scale_num, const double *scale_den,
                      int invert, int n, cudaStream_t s);
void launch_dot(const double *x, const double *y, int n, double *partial, double *out,
                unsigned *ticket, int sqrt_out, int nblk, cudaStream_t s);
void launch_dots(const double *V, long long ldv, int k, const double *w, int n, double *partial,
                 double *h, unsigned *ticket, const int *flag, int nblk, cudaStream_t s);
void launch_update_norm(const double *V, long long ldv, int k, const double *h, double *w, int n,
                        double *partial, double *nrm2, unsigned *ticket, int *flag, int mode,
                        int nblk, cudaStream_t s);
void launch_multi_axpy(const double *Z, long long ldz, int k, const double *y, double *x, int n,
                       cudaStream_t s);
int multidot_blocks(int n);

// ---------------------------------------------------------------- batched
// One system's operands for one kernel class.  Vectors that walk the Krylov
// basis (the top-level input/output of the V-cycle, the outer product's
// operands) are addressed as base + jsel * stride, jsel a launch argument.
struct BJob {
    int n = 0;                       // rows / elements / block rows
    const int *rp = nullptr, *ci = nullptr;
    const void *v = nullptr;         // matrix values (or dense inverse)
    const void *x = nullptr;         // gathered vector
    const void *r = nullptr;         // per-row input
    const void *d = nullptr;         // per-row diagonal inverse (may be null)
    void *o1 = nullptr, *o2 = nullptr;
    const int *idx = nullptr;        // index map
    const int *gs = nullptr, *gz = nullptr;  // block-Jacobi group start / size
    const void *zF = nullptr;
    const int *active = nullptr;     // system still iterating (null = always)
    long long sx = 0, sr = 0, so1 = 0;  // strides per jsel
    // Krylov reductions
    double *partial = nullptr;
    unsigned *ticket = nullptr;
    int *flag = nullptr;
    int nblk = 0;
    // the matrix's SELL-C-sigma copy (row products of the SELL table kind)
    const long long *sptr = nullptr;
    const int *slen = nullptr, *perm = nullptr, *sci = nullptr;
    const void *sv = nullptr;
    int nsl = 0, sg = 1;
};

// batched table launches (T = value type, TV = top-level vector type)
enum BOp { BOP_RESID, BOP_RESTRICT, BOP_PROLONG, BOP_POST, BOP_MGR_RESTRICT, BOP_MGR_INTERP,
           BOP_OUTER_CSR, BOP_FRELAX_RESID };
template <class T, class TV>
void launch_bchunk(int op, const BJob *jobs, const long long *prefix, int njobs, long long total,
                   int R, int jsel, cudaStream_t s);
// the same row products over the members' SELL copies: one work item per slice
template <class T, class TV>
void launch_bsell(int op, const BJob *jobs, const long long *prefix, int njobs, long long total,
                  int jsel, cudaStream_t s);
template <class T, class TV>
void launch_bfrelax_first(const BJob *jobs, const long long *prefix, int njobs, long long total,
                          T omega, int jsel, cudaStream_t s);
template <class T, class TV>
void launch_bscatter(const BJob *jobs, const long long *prefix, int njobs, long long total,
                     int jsel, cudaStream_t s);
// element jobs of the AMG F-relaxation and the restriction of Eq. 5:
// o1 = r[idx] (idx null: r) when o1 is set, o2 = d .* that value when d is set
template <class T, class TV>
void launch_bgather(const BJob *jobs, const long long *prefix, int njobs, long long total, int jsel,
                    cudaStream_t s);
// o1 = omega * x, rounded as one multiplication (a weighted first F sweep)
template <class T>
void launch_bomega(const BJob *jobs, const long long *prefix, int njobs, long long total, T omega,
                   cudaStream_t s);
template <class TV>
void launch_bdense(const BJob *jobs, const long long *prefix, int njobs, long long total, int jsel,
                   cudaStream_t s);
void launch_bbsr(int b, const BJob *jobs, const long long *prefix, int njobs, long long total,
                 int jsel, cudaStream_t s);
void launch_bdots(int k, const BJob *jobs, const long long *bprefix, int njobs, long long nblocks,
                  int jsel, int conditional, int sqrt_out, cudaStream_t s);
void launch_bupdate_norm(int k, const BJob *jobs, const long long *bprefix, int njobs,
                         long long nblocks, int jsel, int mode, cudaStream_t s);
void launch_bscale(const BJob *jobs, const long long *prefix, int njobs, long long total, int jsel,
                   int invert, cudaStream_t s);
void launch_bmulti_axpy(const BJob *jobs, const long long *prefix, int njobs, long long total,
                        cudaStream_t s);

void launch_grad_values(int nb, int b, const int *rp, const int *ci, const double *lam,
                        const double *x, double *dA, cudaStream_t s);

}  // namespace mgr
