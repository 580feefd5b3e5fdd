// C ABI of the MGR library (include/mgr_gb300.h): handle, setup
// orchestration, the V-cycle driver and flexible GMRES.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <type_traits>
#include <chrono>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mgr_gb300.h"
#include "common.cuh"
#include "sell.cuh"

namespace mgr {

void launch_validate_bsr(int nb, int b, const int *rp, const int *ci, const double *val, int *err,
                         cudaStream_t s);
void launch_csr_residual(const DCSR &A, const double *x, const double *bvec, double *y,
                         cudaStream_t s);
void launch_transpose_dense(int n, const double *in, double *out, cudaStream_t s);
void launch_arnoldi_finish(int j, int m, const double *h1, const double *h2, const double *nrmA,
                           const double *nrmB, const int *flag, double *H, double *cs, double *sn,
                           double *g, double *hn, double *stat, const double *tol, cudaStream_t s);
void launch_init_g(double *g, int m, const double *beta, cudaStream_t s);
void launch_solve_upper(int k, int m, const double *H, const double *g, double *y, cudaStream_t s);
void launch_iota(int *a, int n, cudaStream_t s);
void launch_gather_int(const int *idx, int n, const int *v, int *out, cudaStream_t s);
template <class T>
void launch_frelax_scale(int nF, T omega, const T *t, T *zF, int accumulate, cudaStream_t s);

struct MgrLevel {
    int n = 0, nF = 0, nC = 0;
    int *fidx = nullptr, *cidx = nullptr, *gdof = nullptr, *fiota = nullptr;
    DCSR A, AFF, AFC, ACF, W, AFFT, ACFT, WT;
    int relax = 0, sweeps = 1;
    double omega = 1.0;
    int *gstart = nullptr, *gsize = nullptr;
    double *dinv = nullptr;
    float *dinv32 = nullptr;
    // work vectors (FP64 and FP32 variants)
    double *zF = nullptr, *rF = nullptr, *vC = nullptr, *eC = nullptr;
    float *zF32 = nullptr, *rF32 = nullptr, *vC32 = nullptr, *eC32 = nullptr;
    // AMG F-relaxation (MGR_RELAX_AMG): the hierarchy of A_FF and the
    // V-cycle output of a weighted or repeated sweep
    struct AmgH *famg = nullptr;
    bool fshared = false;  // A_FF, A_FF^T are famg's level 0 (not after a refresh)
    double *tF = nullptr;
    float *tF32 = nullptr;
    // restriction of Eq. 5 (MGR_RESTRICT_JACOBI): Z = -A_CF D^{-1} and Z^T;
    // q_F = Z^T e_C and y_F of the transposed cycle
    int rtype = MGR_RESTRICT_INJECTION;
    DCSR Z, ZT;
    double *qF = nullptr, *yF = nullptr;
    float *qF32 = nullptr, *yF32 = nullptr;
};

struct AmgLevel {
    DCSR A, P, R, AT;
    double *dinv = nullptr;
    float *dinv32 = nullptr;
    int *cf = nullptr, *func = nullptr;
    int nc = 0;
    double *r = nullptr, *x = nullptr, *xw = nullptr, *res = nullptr;
    float *r32 = nullptr, *x32 = nullptr, *xw32 = nullptr, *res32 = nullptr;
};

// One AMG hierarchy: the final coarse block's, or the one an AMG
// F-relaxation (MGR_U, Sec. 4.3) builds on A_FF of its MGR level.
struct AmgH {
    int namg = 0;
    AmgLevel amg[32];
    int nco = 0;
    double *coinv = nullptr, *coinvT = nullptr;
    // fused AMG tail (levels tail_k .. namg-1 in one cooperative launch), -1: off
    int tail_k = -1, tail_grid = 0;
    unsigned *tail_sync = nullptr;  // grid barrier words (arrivals, generation, error)
    TailPlan *tail_plan[2] = {nullptr, nullptr};  // device phase lists [trans]
    int frelax = 0;                 // 1: an F-relaxation hierarchy (profile names)
    Arena ar;                       // F-relaxation hierarchies own their memory
    bool sell = false;              // SELL copies built
};

struct Krylov {
    int m = 0, n = 0, nblk = 0;
    double *V = nullptr, *Z = nullptr, *r = nullptr;
    double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double *h1 = nullptr, *h2 = nullptr, *nrm2 = nullptr, *hn = nullptr, *beta = nullptr;
    double *partial = nullptr, *stat = nullptr, *nrmB = nullptr;
    unsigned *ticket = nullptr;
    int *flag = nullptr;
    double *tol = nullptr;     // device copy of rtol * |b|
    long long graph_kernels[2][32] = {};
    std::vector<double> hist;  // relative residuals of the last solve (mgr_solve_history)
    double *hstat = nullptr;  // pinned host mirror of stat
    std::vector<cudaGraphExec_t> graphs[2];
};

// Per-kernel-class timing: a CUDA event pair around each launch on the
// handle's stream, tagged with the algorithmic bytes that launch moves
// (every array read or written once).
struct Prof {
    int on = 0;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<int> ptag;
    std::vector<std::string> names;
    std::vector<double> ms, bytes, fma;
    std::vector<long long> cnt;
};

static std::atomic<long long> g_launches{0};

// NVTX range over a phase (setup, each MGR level, each AMG hierarchy, solve,
// refresh); free unless a profiler is attached.
struct Nvtx {
    explicit Nvtx(const char *name) { nvtxRangePushA(name); }
    ~Nvtx() { nvtxRangePop(); }
};

}  // namespace mgr

using namespace mgr;

struct mgr_ctx {
    int dev = 0;
    cudaStream_t s = nullptr;
    bool own_stream = false;  // created here when the caller passed the legacy default stream
    Arena ar;
    mgr_options opt;
    int nb = 0, b = 0, n = 0;
    long long nnzb = 0;
    int *brp = nullptr, *bci = nullptr;
    double *bval = nullptr;
    DCSR A0T;  // scalar transpose of A (adjoint outer products)
    int *a0t_src = nullptr;  // BSR value index of each A0T entry (value updates)
    DCSR Aout; // CSR view of A when b == 1 (the outer product runs on its SELL copy)
    int8_t *dlevel = nullptr;
    int nlev = 0;
    MgrLevel lev[MGR_MAX_LEVELS];
    AmgH H;  // the final coarse block's AMG hierarchy
    // the hierarchy below (MGR levels, H, their SELL copies and the fused
    // tail) lives in its own arena so that mgr_refresh can rebuild it
    Arena lar;
    DCSR A0;  // level-0 scalar CSR (in lar)
    bool ready = false, in_batch = false;
    int *errw = nullptr;
    Krylov kr;
    Prof prof;
    double setup_ms = 0.0;
    std::string err;
};

static thread_local std::string g_last_error;

// Setup of the members of a batch skips the slice-order timing (the batched
// solve does not use SELL products; the members keep the grid-stride order).
static thread_local bool g_no_tune = false;

// Resources of the timing of SELL product forms (sell_tune): a flush buffer
// larger than L2 and an event pair, held only while a setup builds its SELL
// copies.  nullptr when tuning is off or a resource is missing (every product
// then keeps the plain grid-stride form).
static const SellTune *tune_begin(SellTune &t) {
    if (g_no_tune) return nullptr;
    t.flush_bytes = SELL_TUNE_FLUSH_BYTES;
    if (cudaMalloc(&t.flush, t.flush_bytes) != cudaSuccess) {
        cudaGetLastError();
        t.flush = nullptr;
        return nullptr;
    }
    for (cudaEvent_t &e : t.ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
    return &t;
}

static void tune_end(SellTune &t) {
    if (t.flush) cudaFree(t.flush);
    for (cudaEvent_t e : t.ev)
        if (e) cudaEventDestroy(e);
    t = SellTune();
}

static int setup_tail(mgr_handle h, AmgH &G, int tail_nnz, cudaStream_t s, Arena &ar);

static mgr_status fail(mgr_handle h, mgr_status st, const std::string &msg) {
    if (h) h->err = msg;
    g_last_error = msg;
    return st;
}

static mgr_status cuda_fail(mgr_handle h, const char *where) {
    cudaError_t e = cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
    return fail(h, e == cudaErrorMemoryAllocation ? MGR_ERR_NOMEM : MGR_ERR_CUDA, buf);
}

// RAII scope around one kernel launch: counts it, and when profiling is on
// records an event pair tagged by name and algorithmic bytes.
struct KScope {
    mgr_handle h;
    long long idx = -1;
    KScope(mgr_handle hh, const char *name, int level, double bytes, double fma64 = 0.0) : h(hh) {
        g_launches.fetch_add(1, std::memory_order_relaxed);
        Prof &P = h->prof;
        if (!P.on) return;
        char buf[96];
        if (level >= 0) snprintf(buf, sizeof buf, "%s[L%d]", name, level);
        else snprintf(buf, sizeof buf, "%s", name);
        int tag = -1;
        for (size_t t = 0; t < P.names.size(); t++)
            if (P.names[t] == buf) { tag = (int)t; break; }
        if (tag < 0) {
            tag = (int)P.names.size();
            P.names.push_back(buf); P.ms.push_back(0.0); P.bytes.push_back(0.0); P.cnt.push_back(0);
            P.fma.push_back(0.0);
        }
        P.bytes[tag] += bytes;
        P.fma[tag] += fma64;
        if (P.pool.size() < 2 * (P.used + 1)) {
            cudaEvent_t a, b;
            cudaEventCreate(&a); cudaEventCreate(&b);
            P.pool.push_back(a); P.pool.push_back(b);
        }
        idx = (long long)P.used++;
        P.ptag.resize(P.used);
        P.ptag[idx] = tag;
        cudaEventRecord(P.pool[2 * idx], h->s);
    }
    ~KScope() {
        if (idx >= 0) cudaEventRecord(h->prof.pool[2 * idx + 1], h->s);
    }
};

static void prof_resolve(mgr_handle h) {
    Prof &P = h->prof;
    if (!P.used) return;
    cudaStreamSynchronize(h->s);
    for (size_t i = 0; i < P.used; i++) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, P.pool[2 * i], P.pool[2 * i + 1]);
        P.ms[P.ptag[i]] += ms;
        P.cnt[P.ptag[i]] += 1;
    }
    P.used = 0;
}

extern "C" void mgr_options_default(mgr_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    for (int l = 0; l < MGR_MAX_LEVELS; l++) {
        o->relax_type[l] = MGR_RELAX_JACOBI;
        o->relax_sweeps[l] = 1;
        o->relax_weight[l] = 1.0;
    }
    o->amg_theta = 0.25;
    o->amg_max_levels = 25;
    o->amg_max_coarse = 1024;
    o->amg_pmax = 4;
    o->amg_num_functions = 1;
    o->precision = MGR_PREC_FP64;
    o->restart = 30;
    o->use_graphs = 1;
    o->amg_tail_nnz = 0;
    for (int l = 0; l < MGR_MAX_LEVELS; l++) {
        o->relax_functions[l] = 1;
        o->restrict_type[l] = MGR_RESTRICT_INJECTION;
    }
    o->spin_limit = 0;
}

// ---------------------------------------------------------------- helpers
static int read_errw(mgr_handle h) {
    int e = 0;
    cudaMemcpyAsync(&e, h->errw, sizeof(int), cudaMemcpyDeviceToHost, h->s);
    cudaStreamSynchronize(h->s);
    cudaMemsetAsync(h->errw, 0, sizeof(int), h->s);
    return e;
}

// The fused AMG tail's error word (nonzero once one of its grid-barrier
// waits ran out).  Synchronises the stream to read it; a set word is cleared
// with the barrier's other words so that later launches start clean.
static bool tail_timed_out(mgr_handle h) {
    if (!h->H.tail_sync) return false;
    unsigned terr = 0;
    cudaMemcpyAsync(&terr, h->H.tail_sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, h->s);
    cudaStreamSynchronize(h->s);
    if (!terr) return false;
    cudaMemsetAsync(h->H.tail_sync, 0, 4 * sizeof(unsigned), h->s);
    cudaStreamSynchronize(h->s);
    return true;
}

static int to_f32(Arena &ar, DCSR &M, cudaStream_t s) {
    if (M.nnz == 0) { M.v32 = ar.alloc<float>(1); return M.v32 ? 0 : ST_NOMEM; }
    M.v32 = ar.alloc<float>(M.nnz);
    if (!M.v32) return ST_NOMEM;
    launch_cast_f32(M.v, M.v32, M.nnz, s);
    return 0;
}

// Deep copy of a CSR matrix (pattern and FP64 values) into ar.
static int copy_csr(const DCSR &A, DCSR &out, Arena &ar, cudaStream_t s) {
    out = DCSR();
    out.n = A.n; out.m = A.m; out.nnz = A.nnz;
    out.rp = ar.alloc<int>(A.n + 1);
    out.ci = ar.alloc<int>(A.nnz + 1);
    out.v = ar.alloc<double>(A.nnz + 1);
    if (!out.rp || !out.ci || !out.v) return ST_NOMEM;
    cudaMemcpyAsync(out.rp, A.rp, sizeof(int) * (A.n + 1), cudaMemcpyDeviceToDevice, s);
    if (A.nnz) {
        cudaMemcpyAsync(out.ci, A.ci, sizeof(int) * A.nnz, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(out.v, A.v, sizeof(double) * A.nnz, cudaMemcpyDeviceToDevice, s);
    }
    return ST_OK;
}

// AMG setup of hierarchy G on A0 (strength, PMIS, extended+i, Galerkin
// products, l1 smoother scaling, dense inverse of the coarsest grid) with
// nfunc functions of the unknown approach, allocated from ar.  own_copy:
// level 0 holds a copy of A0 (a hierarchy that outlives A0's arena).
static mgr_status setup_amg(mgr_handle h, AmgH &G, DCSR A0, int nfunc, Arena &ar, bool own_copy) {
    Nvtx nv(G.frelax ? "mgr AMG setup (F-relaxation)" : "mgr AMG setup (coarse block)");
    cudaStream_t s = h->s;
    const mgr_options &o = h->opt;
    int maxl = o.amg_max_levels < 1 ? 1 : (o.amg_max_levels > 32 ? 32 : o.amg_max_levels);
    if (own_copy) {
        if (copy_csr(A0, G.amg[0].A, ar, s)) return fail(h, MGR_ERR_NOMEM, "amg level 0");
    } else {
        G.amg[0].A = A0;
    }
    A0 = G.amg[0].A;
    G.amg[0].func = ar.alloc<int>(A0.n + 1);
    if (!G.amg[0].func) return fail(h, MGR_ERR_NOMEM, "amg func");
    launch_iota_mod(G.amg[0].func, A0.n, nfunc < 1 ? 1 : nfunc, s);
    int k = 0;
    for (;;) {
        AmgLevel &L = G.amg[k];
        int n = L.A.n;
        G.namg = k + 1;
        if (transpose(L.A, L.AT, s, ar)) return fail(h, MGR_ERR_NOMEM, "amg transpose");
        if (n <= o.amg_max_coarse || k + 1 >= maxl) break;
        uint8_t *sflag = ar.alloc<uint8_t>(L.A.nnz + 1);
        if (!sflag) return fail(h, MGR_ERR_NOMEM, "strength");
        DCSR S, ST;
        int rc = amg_strength(L.A, L.func, o.amg_theta, sflag, S, s, ar);
        if (!rc) rc = transpose(S, ST, s, ar);
        L.cf = ar.alloc<int>(n + 1);
        if (rc || !L.cf) return fail(h, MGR_ERR_NOMEM, "strength/transpose");
        rc = amg_pmis(S, ST, k, L.cf, s, ar);
        if (rc) return fail(h, rc == ST_TIMEOUT ? MGR_ERR_TIMEOUT : MGR_ERR_CUDA, "pmis");
        int nc = 0;
        rc = amg_extpi(L.A, sflag, L.cf, L.func, o.amg_pmax, L.P, &nc, s, ar);
        if (rc) return fail(h, MGR_ERR_NOMEM, "extended+i interpolation");
        ar.release(sflag); ar.release(S.rp); ar.release(S.ci); ar.release(ST.rp); ar.release(ST.ci);
        if (nc == 0 || nc == n) {
            ar.release(L.P.rp); ar.release(L.P.ci); ar.release(L.P.v);
            L.P = DCSR();
            break;
        }
        L.nc = nc;
        if (transpose(L.P, L.R, s, ar)) return fail(h, MGR_ERR_NOMEM, "P^T");
        DCSR AP;
        if (spgemm(L.A, L.P, nullptr, AP, s, ar)) return fail(h, MGR_ERR_NOMEM, "A P");
        AmgLevel &C = G.amg[k + 1];
        if (spgemm(L.R, AP, nullptr, C.A, s, ar)) return fail(h, MGR_ERR_NOMEM, "P^T A P");
        ar.release(AP.rp); ar.release(AP.ci); ar.release(AP.v);
        C.func = ar.alloc<int>(nc + 1);
        L.dinv = ar.alloc<double>(n + 1);
        L.dinv32 = ar.alloc<float>(n + 1);
        if (!C.func || !L.dinv || !L.dinv32) return fail(h, MGR_ERR_NOMEM, "amg level");
        launch_coarse_func(L.cf, L.func, L.P, C.func, n, s);
        l1_inverse(L.A, L.dinv, L.dinv32, h->errw, s);
        if (read_errw(h) & ERRW_SINGULAR) return fail(h, MGR_ERR_SINGULAR, "zero l1 row scaling in AMG smoother");
        k++;
    }
    AmgLevel &Lc = G.amg[G.namg - 1];
    G.nco = Lc.A.n;
    if (G.nco > 4096) return fail(h, MGR_ERR_UNSUPPORTED, "AMG coarsening stalled above 4096 rows");
    G.coinv = ar.alloc<double>((size_t)G.nco * G.nco + 1);
    G.coinvT = ar.alloc<double>((size_t)G.nco * G.nco + 1);
    if (!G.coinv || !G.coinvT) return fail(h, MGR_ERR_NOMEM, "coarsest inverse");
    if (G.nco > 0) {
        if (dense_inverse(Lc.A, G.coinv, h->errw, s, ar)) return fail(h, MGR_ERR_NOMEM, "coarsest");
        if (read_errw(h) & ERRW_SINGULAR) return fail(h, MGR_ERR_SINGULAR, "singular coarsest AMG grid");
        launch_transpose_dense(G.nco, G.coinv, G.coinvT, s);
    }
    // FP32 copies and work vectors
    for (int q = 0; q < G.namg; q++) {
        AmgLevel &L = G.amg[q];
        int n = L.A.n;
        if (to_f32(ar, L.A, s) || to_f32(ar, L.AT, s)) return fail(h, MGR_ERR_NOMEM, "fp32 copies");
        if (q < G.namg - 1 && (to_f32(ar, L.P, s) || to_f32(ar, L.R, s))) return fail(h, MGR_ERR_NOMEM, "fp32 copies");
        L.r = ar.alloc<double>(n + 1); L.x = ar.alloc<double>(n + 1);
        L.xw = ar.alloc<double>(n + 1); L.res = ar.alloc<double>(n + 1);
        L.r32 = ar.alloc<float>(n + 1); L.x32 = ar.alloc<float>(n + 1);
        L.xw32 = ar.alloc<float>(n + 1); L.res32 = ar.alloc<float>(n + 1);
        if (!L.r || !L.x || !L.xw || !L.res || !L.r32 || !L.x32 || !L.xw32 || !L.res32)
            return fail(h, MGR_ERR_NOMEM, "amg vectors");
    }
    return MGR_OK;
}

// The MGR hierarchy below the outer operator (Sec. 3): the level-0 scalar
// CSR, every MGR level (split, D_FF, W, Z, coarse operator, F-relaxation
// AMG), the final coarse block's AMG hierarchy, their SELL copies and the
// fused AMG tail, all in h->lar (F-relaxation hierarchies in their own
// arenas).  reuse: keep the AMG F-relaxation hierarchies a previous build
// left (mgr_refresh).  On failure the handle is not usable (ready stays
// false).
static mgr_status build_levels(mgr_handle h, bool reuse) {
    Nvtx nv(reuse ? "mgr hierarchy (refresh)" : "mgr hierarchy");
    Arena &ar = h->lar;
    cudaStream_t s = h->s;
    const int nb = h->nb, b = h->b, n = h->n;
    const long long nnzb = h->nnzb;
    // level-0 scalar CSR
    DCSR A0;
    A0.n = A0.m = n;
    A0.nnz = (int)(nnzb * b * b);
    A0.rp = ar.alloc<int>(n + 1);
    A0.ci = ar.alloc<int>(A0.nnz);
    A0.v = ar.alloc<double>(A0.nnz);
    if (!A0.rp || !A0.ci || !A0.v) return fail(h, MGR_ERR_NOMEM, "scalar copy");
    launch_bsr_to_csr(nb, b, h->brp, h->bci, h->bval, A0, s);
    h->A0 = A0;
    DCSR cur = A0;
    int *gdof = nullptr;
    for (int l = 0; l < h->nlev; l++) {
        MgrLevel &L = h->lev[l];
        char nvn[32];
        snprintf(nvn, sizeof nvn, "mgr level %d", l);
        Nvtx nvl(nvn);
        L.A = cur; L.gdof = gdof; L.n = cur.n;
        L.relax = h->opt.relax_type[l];
        L.sweeps = h->opt.relax_sweeps[l] < 1 ? 1 : h->opt.relax_sweeps[l];
        L.omega = h->opt.relax_weight[l];
        if (L.relax < MGR_RELAX_JACOBI || L.relax > MGR_RELAX_AMG) { return fail(h, MGR_ERR_INVALID, "relax type"); }
        L.rtype = h->opt.restrict_type[l];
        if (L.rtype < MGR_RESTRICT_INJECTION || L.rtype > MGR_RESTRICT_JACOBI) {
            return fail(h, MGR_ERR_INVALID, "restriction type");
        }
        if (L.rtype == MGR_RESTRICT_JACOBI && L.relax == MGR_RELAX_BLOCK_JACOBI) {
            return fail(h, MGR_ERR_UNSUPPORTED, "the restriction of Eq. 5 takes a diagonal D_FF");
        }
        int nl = L.n;
        int *isF = ar.alloc<int>(nl + 1), *isC = ar.alloc<int>(nl + 1);
        int *fpos = ar.alloc<int>(nl + 1), *cpos = ar.alloc<int>(nl + 1);
        int *fmap = ar.alloc<int>(nl + 1), *cmap = ar.alloc<int>(nl + 1);
        L.fidx = ar.alloc<int>(nl + 1); L.cidx = ar.alloc<int>(nl + 1);
        if (!isF || !isC || !fpos || !cpos || !fmap || !cmap || !L.fidx || !L.cidx) {
            return fail(h, MGR_ERR_NOMEM, "level maps");
        }
        launch_level_flags(h->dlevel, gdof, nl, l, isF, isC, h->errw, s);
        int nF = 0, nC = 0;
        scan_exclusive(isF, fpos, nl, s, ar, &nF);
        scan_exclusive(isC, cpos, nl, s, ar, &nC);
        if (read_errw(h)) { return fail(h, MGR_ERR_INVALID, "labels: a dof eliminated twice"); }
        if (nF == 0 || nC == 0) {
            char buf[128];
            snprintf(buf, sizeof buf, "MGR level %d has an empty %s set", l, nF == 0 ? "F" : "C");
            return fail(h, MGR_ERR_INVALID, buf);
        }
        L.nF = nF; L.nC = nC;
        launch_index_maps(isF, isC, fpos, cpos, nl, L.fidx, L.cidx, fmap, cmap, s);
        DCSR ACC;
        int rc = extract_submatrix(cur, L.fidx, nF, fmap, nF, L.AFF, s, ar);
        if (!rc) rc = extract_submatrix(cur, L.fidx, nF, cmap, nC, L.AFC, s, ar);
        if (!rc) rc = extract_submatrix(cur, L.cidx, nC, fmap, nF, L.ACF, s, ar);
        if (!rc) rc = extract_submatrix(cur, L.cidx, nC, cmap, nC, ACC, s, ar);
        L.gstart = ar.alloc<int>(nF + 1); L.gsize = ar.alloc<int>(nF + 1);
        L.dinv = ar.alloc<double>((size_t)nF * 4 + 4); L.dinv32 = ar.alloc<float>((size_t)nF * 4 + 4);
        if (rc || !L.gstart || !L.gsize || !L.dinv || !L.dinv32) { return fail(h, MGR_ERR_NOMEM, "level blocks"); }
        {
            const int none = 0x7fffffff;  // errw[1]: the first singular F point
            cudaMemcpyAsync(h->errw + 1, &none, sizeof(int), cudaMemcpyHostToDevice, s);
        }
        mgr_dinv(L.AFF, L.fidx, gdof, b, L.relax, L.gstart, L.gsize, L.dinv, h->errw, s);
        if (read_errw(h) & ERRW_SINGULAR) {
            int f = -1, loc = -1, dof = -1;
            cudaMemcpy(&f, h->errw + 1, sizeof(int), cudaMemcpyDeviceToHost);
            if (f >= 0 && f < nF) {
                cudaMemcpy(&loc, L.fidx + f, sizeof(int), cudaMemcpyDeviceToHost);
                dof = loc;
                if (gdof && loc >= 0) cudaMemcpy(&dof, gdof + loc, sizeof(int), cudaMemcpyDeviceToHost);
            }
            char buf[192];
            snprintf(buf, sizeof buf,
                     "singular D_FF (zero diagonal or singular block) at MGR level %d, first at F point %d (dof %d)",
                     l, f, dof);
            return fail(h, MGR_ERR_SINGULAR, buf);
        }
        launch_cast_f32(L.dinv, L.dinv32, (long long)nF * 4, s);
        if (mgr_build_w(L.AFC, L.gstart, L.gsize, L.dinv, L.W, s, ar)) { return fail(h, MGR_ERR_NOMEM, "W"); }
        DCSR next;
        if (transpose(L.ACF, L.ACFT, s, ar)) { return fail(h, MGR_ERR_NOMEM, "level transposes"); }
        if (L.rtype == MGR_RESTRICT_JACOBI) {
            // R~ A P~ = Z (A_FF W + A_FC) + (A_CF W + A_CC), Z^T = -D^{-1} A_CF^T
            DCSR T1, U;
            if (mgr_build_w(L.ACFT, L.gstart, L.gsize, L.dinv, L.ZT, s, ar) || transpose(L.ZT, L.Z, s, ar) ||
                spgemm(L.AFF, L.W, &L.AFC, T1, s, ar) || spgemm(L.ACF, L.W, &ACC, U, s, ar) ||
                spgemm(L.Z, T1, &U, next, s, ar)) {
                return fail(h, MGR_ERR_NOMEM, "coarse operator");
            }
            ar.release(T1.rp); ar.release(T1.ci); ar.release(T1.v);
            ar.release(U.rp); ar.release(U.ci); ar.release(U.v);
        } else if (spgemm(L.ACF, L.W, &ACC, next, s, ar)) {
            return fail(h, MGR_ERR_NOMEM, "coarse operator");
        }
        ar.release(ACC.rp); ar.release(ACC.ci); ar.release(ACC.v);
        const bool keep = reuse && L.relax == MGR_RELAX_AMG && L.famg && L.famg->namg > 0 &&
                          L.famg->amg[0].A.n == nF && L.famg->amg[0].A.nnz == L.AFF.nnz;
        if (!keep && L.famg) {
            L.famg->ar.free_all();
            delete L.famg;
            L.famg = nullptr;
        }
        L.fshared = false;
        if (keep) {
            // an unchanged A_FF is shared with the kept hierarchy's level 0
            // (no second transpose, FP32 or SELL copy)
            const int same = same_bits(L.AFF.v, L.famg->amg[0].A.v, L.AFF.nnz, s, ar);
            if (same < 0) return fail(h, MGR_ERR_CUDA, "A_FF comparison");
            if (same) {
                ar.release(L.AFF.rp); ar.release(L.AFF.ci); ar.release(L.AFF.v);
                L.AFF = L.famg->amg[0].A;
                L.AFFT = L.famg->amg[0].AT;
                L.fshared = true;
            }
        }
        if (L.relax == MGR_RELAX_AMG && !keep) {
            // the F-relaxation's AMG hierarchy on A_FF (same AMG parameters as
            // the final coarse block), in an arena of its own so that a
            // refresh can keep it; its level 0 holds a copy of A_FF, A_FF^T
            // and their FP32 copies, which the level shares
            L.famg = new (std::nothrow) AmgH();
            if (!L.famg) return fail(h, MGR_ERR_NOMEM, "F-relaxation AMG");
            L.famg->frelax = 1;
            mgr_status fst = setup_amg(h, *L.famg, L.AFF, h->opt.relax_functions[l], L.famg->ar, true);
            if (fst != MGR_OK) {
                std::string m = "F-relaxation AMG at MGR level " + std::to_string(l) + ": " + h->err;
                return fail(h, fst, m);
            }
            L.AFF = L.famg->amg[0].A;
            L.AFFT = L.famg->amg[0].AT;
            L.fshared = true;
        } else if (!L.fshared && transpose(L.AFF, L.AFFT, s, ar)) {
            // (a kept hierarchy relaxes with the A_FF it was built from; the
            // level's own residuals use the new A_FF)
            return fail(h, MGR_ERR_NOMEM, "level transposes");
        }
        if (transpose(L.W, L.WT, s, ar)) {
            return fail(h, MGR_ERR_NOMEM, "level transposes");
        }
        if ((!L.fshared && (to_f32(ar, L.AFF, s) || to_f32(ar, L.AFFT, s))) || to_f32(ar, L.ACF, s) ||
            to_f32(ar, L.W, s) || to_f32(ar, L.ACFT, s) || to_f32(ar, L.WT, s) ||
            (L.rtype == MGR_RESTRICT_JACOBI && (to_f32(ar, L.Z, s) || to_f32(ar, L.ZT, s)))) {
            return fail(h, MGR_ERR_NOMEM, "fp32");
        }
        L.fiota = ar.alloc<int>(nF + 1);
        L.zF = ar.alloc<double>(nF + 1); L.rF = ar.alloc<double>(nF + 1);
        L.vC = ar.alloc<double>(nC + 1); L.eC = ar.alloc<double>(nC + 1);
        L.zF32 = ar.alloc<float>(nF + 1); L.rF32 = ar.alloc<float>(nF + 1);
        L.vC32 = ar.alloc<float>(nC + 1); L.eC32 = ar.alloc<float>(nC + 1);
        if (L.famg) {
            L.tF = ar.alloc<double>(nF + 1); L.tF32 = ar.alloc<float>(nF + 1);
            if (!L.tF || !L.tF32) { return fail(h, MGR_ERR_NOMEM, "level vectors"); }
        }
        if (L.rtype == MGR_RESTRICT_JACOBI) {
            L.qF = ar.alloc<double>(nF + 1); L.qF32 = ar.alloc<float>(nF + 1);
            L.yF = ar.alloc<double>(nF + 1); L.yF32 = ar.alloc<float>(nF + 1);
            if (!L.qF || !L.qF32 || !L.yF || !L.yF32) { return fail(h, MGR_ERR_NOMEM, "level vectors"); }
        }
        int *g2 = ar.alloc<int>(nC + 1);
        if (!L.fiota || !L.zF || !L.rF || !L.vC || !L.eC || !L.zF32 || !L.rF32 || !L.vC32 || !L.eC32 || !g2) {
            return fail(h, MGR_ERR_NOMEM, "level vectors");
        }
        launch_iota(L.fiota, nF, s);
        // original dof of each C point (the next level's rows)
        if (gdof) launch_gather_int(L.cidx, nC, gdof, g2, s);
        else cudaMemcpyAsync(g2, L.cidx, sizeof(int) * nC, cudaMemcpyDeviceToDevice, s);
        ar.release(isF); ar.release(isC); ar.release(fpos); ar.release(cpos); ar.release(fmap); ar.release(cmap);
        gdof = g2;
        cur = next;
    }
    mgr_status st = setup_amg(h, h->H, cur, h->opt.amg_num_functions, ar, false);
    if (st != MGR_OK) return st;
    // SELL-C-sigma copies of every matrix the solve phase multiplies with,
    // each with the slice order its product runs fastest in (timed here)
    {
        SellTune tune;
        tune.fp32 = h->opt.precision == MGR_PREC_FP32 ? 1 : 0;
        const SellTune *prec = tune_begin(tune);
        int rc2 = 0;
        auto sell_amg = [&](AmgH &G, Arena &gar) {
            if (G.sell) return;
            for (int k = 0; k + 1 < G.namg && !rc2; k++) {
                AmgLevel &A = G.amg[k];
                DCSR *ms[] = {&A.A, &A.AT, &A.P, &A.R};
                for (DCSR *m : ms) rc2 |= build_sell(*m, s, gar, prec);
            }
            G.sell = !rc2;
        };
        for (int l = 0; l < h->nlev && !rc2; l++) {
            MgrLevel &L = h->lev[l];
            if (L.famg) sell_amg(*L.famg, L.famg->ar);
            if (L.fshared && L.famg->namg > 1) {
                // A_FF and A_FF^T are the F hierarchy's level 0: one SELL copy
                L.AFF = L.famg->amg[0].A;
                L.AFFT = L.famg->amg[0].AT;
                DCSR *ms[] = {&L.ACF, &L.W, &L.ACFT, &L.WT};
                for (DCSR *m : ms) rc2 |= build_sell(*m, s, ar, prec);
            } else {
                DCSR *ms[] = {&L.AFF, &L.ACF, &L.W, &L.AFFT, &L.ACFT, &L.WT};
                for (DCSR *m : ms) rc2 |= build_sell(*m, s, ar, prec);
            }
            if (L.rtype == MGR_RESTRICT_JACOBI) rc2 |= build_sell(L.Z, s, ar, prec) | build_sell(L.ZT, s, ar, prec);
        }
        sell_amg(h->H, ar);
        tune_end(tune);
        if (rc2) return fail(h, MGR_ERR_NOMEM, "SELL copies");
    }
    {
        const int rc3 = setup_tail(h, h->H, h->opt.amg_tail_nnz, s, ar);
        if (rc3) return fail(h, rc3 == ST_NOMEM ? MGR_ERR_NOMEM : MGR_ERR_CUDA, "fused AMG tail");
    }
    return MGR_OK;
}

extern "C" mgr_status mgr_setup(const mgr_bsr *Ain, const mgr_labels *cf, const mgr_options *opt,
                                void *stream, mgr_handle *out) {
    if (!out) return fail(nullptr, MGR_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!Ain || !cf || !cf->dof_level) return fail(nullptr, MGR_ERR_INVALID, "NULL argument");
    if (Ain->b < 1 || Ain->b > 4 || Ain->nb < 1 || Ain->nnzb < 1 || !Ain->row_ptr || !Ain->col_idx || !Ain->val)
        return fail(nullptr, MGR_ERR_INVALID, "bad block matrix sizes (b must be 1..4)");
    if ((long long)Ain->nnzb * Ain->b * Ain->b > 2000000000LL || (long long)Ain->nb * Ain->b > 2000000000LL)
        return fail(nullptr, MGR_ERR_UNSUPPORTED, "matrix too large for 32-bit scalar indices");
    if (cf->num_levels < 0 || cf->num_levels > MGR_MAX_LEVELS)
        return fail(nullptr, MGR_ERR_INVALID, "num_levels out of range");
    Nvtx nv("mgr_setup");
    auto t0 = std::chrono::steady_clock::now();
    mgr_handle h = new mgr_ctx();
    cudaGetDevice(&h->dev);
    h->s = (cudaStream_t)stream;
    if (!h->s) {
        // the legacy default stream cannot be captured into graphs: use a
        // blocking stream of our own, which it orders against implicitly
        if (cudaStreamCreate(&h->s) != cudaSuccess) { delete h; return cuda_fail(nullptr, "stream"); }
        h->own_stream = true;
    }
    if (opt) h->opt = *opt; else mgr_options_default(&h->opt);
    if (h->opt.restart < 1) h->opt.restart = 1;
    if (h->opt.restart > 30) h->opt.restart = 30;
    Arena &ar = h->ar;
    cudaStream_t s = h->s;
    h->nb = Ain->nb; h->b = Ain->b; h->nnzb = Ain->nnzb; h->n = Ain->nb * Ain->b;
    int nb = h->nb, b = h->b, n = h->n;
    long long nnzb = h->nnzb;
    h->errw = ar.alloc<int>(4);
    h->brp = ar.alloc<int>(nb + 1);
    h->bci = ar.alloc<int>(nnzb);
    h->bval = ar.alloc<double>(nnzb * b * b);
    h->dlevel = ar.alloc<int8_t>(n + 1);
    if (!h->errw || !h->brp || !h->bci || !h->bval || !h->dlevel) {
        mgr_free(h);
        return fail(nullptr, MGR_ERR_NOMEM, "device allocation of the matrix copy");
    }
    cudaMemsetAsync(h->errw, 0, 4 * sizeof(int), s);
    cudaMemcpyKind kind = Ain->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaMemcpyAsync(h->brp, Ain->row_ptr, sizeof(int) * (nb + 1), kind, s);
    cudaMemcpyAsync(h->bci, Ain->col_idx, sizeof(int) * nnzb, kind, s);
    cudaMemcpyAsync(h->bval, Ain->val, sizeof(double) * nnzb * b * b, kind, s);
    cudaMemcpyAsync(h->dlevel, cf->dof_level, n, cudaMemcpyHostToDevice, s);
    // host-side row_ptr check: every later device read goes through it
    {
        std::vector<int> hrp(nb + 1);
        if (Ain->on_device) cudaMemcpy(hrp.data(), Ain->row_ptr, sizeof(int) * (nb + 1), cudaMemcpyDeviceToHost);
        else memcpy(hrp.data(), Ain->row_ptr, sizeof(int) * (nb + 1));
        bool ok = hrp[0] == 0 && (long long)hrp[nb] == nnzb;
        for (int I = 0; ok && I < nb; I++) ok = hrp[I + 1] >= hrp[I];
        if (!ok) {
            mgr_free(h);
            return fail(nullptr, MGR_ERR_INVALID, "row_ptr must start at 0, be non-decreasing and end at nnzb");
        }
    }
    // host-side label check
    for (int i = 0; i < n; i++)
        if (cf->dof_level[i] < 0 || cf->dof_level[i] > cf->num_levels) {
            mgr_free(h);
            return fail(nullptr, MGR_ERR_INVALID, "dof_level value out of range");
        }
    launch_validate_bsr(nb, b, h->brp, h->bci, h->bval, h->errw, s);
    int ew = read_errw(h);
    if (cudaGetLastError() != cudaSuccess) { mgr_free(h); return cuda_fail(nullptr, "copy/validate"); }
    if (ew) {
        mgr_free(h);
        return fail(nullptr, MGR_ERR_INVALID,
                    (ew & 8) ? "non-finite matrix value"
                    : (ew & 16) ? "missing diagonal block"
                    : "row_ptr/col_idx malformed (unsorted, duplicate or out-of-range column)");
    }
    h->nlev = cf->num_levels;
    {
        mgr_status st = build_levels(h, false);
        if (st != MGR_OK) { std::string m = h->err; mgr_free(h); return fail(nullptr, st, m); }
    }
    if (transpose(h->A0, h->A0T, s, ar)) { mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "A^T"); }
    h->a0t_src = ar.alloc<int>((size_t)h->A0T.nnz + 1);
    if (!h->a0t_src || transpose_sources(nb, b, h->brp, h->bci, nnzb, h->a0t_src, s)) {
        mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "A^T sources");
    }
    // Krylov workspace
    Krylov &K = h->kr;
    K.m = h->opt.restart; K.n = n; K.nblk = multidot_blocks(n);
    K.V = ar.alloc<double>((size_t)(K.m + 1) * n);
    K.Z = ar.alloc<double>((size_t)K.m * n);
    K.r = ar.alloc<double>(n);
    K.H = ar.alloc<double>((K.m + 1) * K.m);
    K.cs = ar.alloc<double>(K.m + 1); K.sn = ar.alloc<double>(K.m + 1);
    K.g = ar.alloc<double>(K.m + 2); K.y = ar.alloc<double>(K.m + 1);
    K.h1 = ar.alloc<double>(40); K.h2 = ar.alloc<double>(40);
    K.nrm2 = ar.alloc<double>(4); K.hn = ar.alloc<double>(4); K.beta = ar.alloc<double>(4);
    K.partial = ar.alloc<double>((size_t)K.nblk * 33 + 33);
    K.stat = ar.alloc<double>(8);
    K.nrmB = ar.alloc<double>(4);
    K.ticket = ar.alloc<unsigned>(4);
    K.flag = ar.alloc<int>(4);
    K.tol = ar.alloc<double>(2);
    if (!K.nrmB || !K.ticket || !K.flag || !K.tol) { mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "Krylov workspace"); }
    cudaMemsetAsync(K.ticket, 0, 4 * sizeof(unsigned), s);
    cudaMemsetAsync(K.flag, 0, 4 * sizeof(int), s);
    cudaMallocHost(&K.hstat, 8 * sizeof(double));
    if (!K.V || !K.Z || !K.r || !K.H || !K.partial || !K.stat || !K.hstat) {
        mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "Krylov workspace");
    }
    // SELL-C-sigma copies of the outer operator and its transpose
    {
        SellTune tune;  // the outer products are FP64 in both forms
        const SellTune *tp = tune_begin(tune);
        int rc2 = 0;
        if (b == 1) {
            h->Aout.n = h->Aout.m = n;
            h->Aout.nnz = (int)nnzb;
            h->Aout.rp = h->brp; h->Aout.ci = h->bci; h->Aout.v = h->bval;
            rc2 |= build_sell(h->Aout, s, ar, tp);
        }
        rc2 |= build_sell(h->A0T, s, ar, tp);
        tune_end(tune);
        if (rc2) { mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "SELL copies"); }
    }
    cudaStreamSynchronize(s);
    if (cudaGetLastError() != cudaSuccess) { mgr_free(h); return cuda_fail(nullptr, "setup"); }
    // setup temporaries are freed (cudaFree)
    h->ar.trim();
    h->lar.trim();
    for (int l = 0; l < h->nlev; l++)
        if (h->lev[l].famg) h->lev[l].famg->ar.trim();
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    h->ready = true;
    *out = h;
    return MGR_OK;
}

// -------------------------------------------------------------- V-cycle
template <class T> struct Sel;
template <> struct Sel<double> {
    static const double *v(const DCSR &M) { return M.v; }
    static double *zF(MgrLevel &L) { return L.zF; }
    static double *rF(MgrLevel &L) { return L.rF; }
    static double *vC(MgrLevel &L) { return L.vC; }
    static double *eC(MgrLevel &L) { return L.eC; }
    static double *tF(MgrLevel &L) { return L.tF; }
    static double *qF(MgrLevel &L) { return L.qF; }
    static double *yF(MgrLevel &L) { return L.yF; }
    static const double *dinv(MgrLevel &L) { return L.dinv; }
    static const double *dinv(AmgLevel &L) { return L.dinv; }
    static double *r(AmgLevel &L) { return L.r; }
    static double *x(AmgLevel &L) { return L.x; }
    static double *xw(AmgLevel &L) { return L.xw; }
    static double *res(AmgLevel &L) { return L.res; }
};
template <> struct Sel<float> {
    static const float *v(const DCSR &M) { return M.v32; }
    static float *zF(MgrLevel &L) { return L.zF32; }
    static float *rF(MgrLevel &L) { return L.rF32; }
    static float *vC(MgrLevel &L) { return L.vC32; }
    static float *eC(MgrLevel &L) { return L.eC32; }
    static float *tF(MgrLevel &L) { return L.tF32; }
    static float *qF(MgrLevel &L) { return L.qF32; }
    static float *yF(MgrLevel &L) { return L.yF32; }
    static const float *dinv(MgrLevel &L) { return L.dinv32; }
    static const float *dinv(AmgLevel &L) { return L.dinv32; }
    static float *r(AmgLevel &L) { return L.r32; }
    static float *x(AmgLevel &L) { return L.x32; }
    static float *xw(AmgLevel &L) { return L.xw32; }
    static float *res(AmgLevel &L) { return L.res32; }
};

// ------------------------------------------------------- fused AMG tail
template <class T>
static SellView sell_view(const DCSR &M) {
    SellView v;
    v.nsl = M.nsl;
    v.sg = M.sg;
    v.sptr = M.sptr;
    v.slen = M.slen;
    v.perm = M.perm;
    v.sci = M.sci;
    v.sv = sell_vals<T>(M);
    return v;
}

// The phase list of levels tail_k .. namg-1 (the order of amg_cycle below).
// false when a matrix of the tail has no SELL copy of this precision.
template <class T>
static bool build_tail_plan(AmgH &G, int trans, TailPlan &P) {
    const int kt = G.tail_k, kc = G.namg - 1;
    P.nphase = 0;
    auto add = [&](int kind) -> TailPhase & {
        TailPhase &q = P.ph[P.nphase++];
        q = TailPhase();
        q.kind = kind;
        return q;
    };
    for (int k = kt; k < kc; k++) {
        AmgLevel &L = G.amg[k];
        const DCSR &A = trans ? L.AT : L.A;
        if (!A.sptr || !sell_vals<T>(A) || !L.R.sptr || !sell_vals<T>(L.R) || !L.P.sptr || !sell_vals<T>(L.P))
            return false;
        TailPhase &q = add(TAIL_RESID);
        q.M = sell_view<T>(A);
        q.x = Sel<T>::xw(L);
        q.r = Sel<T>::r(L);
        q.y = Sel<T>::res(L);
        AmgLevel &C = G.amg[k + 1];
        TailPhase &q2 = add(k + 1 < kc ? TAIL_RESTRICT_SCALED : TAIL_RESTRICT);
        q2.M = sell_view<T>(L.R);
        q2.x = Sel<T>::res(L);
        q2.y = Sel<T>::r(C);
        if (k + 1 < kc) {
            q2.y2 = Sel<T>::xw(C);
            q2.d = Sel<T>::dinv(C);
        }
    }
    TailPhase &qd = add(TAIL_DENSE);
    qd.n = G.nco;
    qd.inv = trans ? G.coinvT : G.coinv;
    qd.x = Sel<T>::r(G.amg[kc]);
    qd.y = Sel<T>::x(G.amg[kc]);
    for (int k = kc - 1; k >= kt; k--) {
        AmgLevel &L = G.amg[k];
        const DCSR &A = trans ? L.AT : L.A;
        TailPhase &q = add(TAIL_PROLONG);
        q.M = sell_view<T>(L.P);
        q.x = Sel<T>::x(G.amg[k + 1]);
        q.y = Sel<T>::xw(L);
        TailPhase &q2 = add(TAIL_POST);
        q2.M = sell_view<T>(A);
        q2.x = Sel<T>::xw(L);
        q2.r = Sel<T>::r(L);
        q2.d = Sel<T>::dinv(L);
        q2.y = Sel<T>::x(L);
    }
    return true;
}

// Choose the tail's first level and upload its phase lists (both
// orientations).  Leaves the tail off when the option, the hierarchy or the
// device does not allow it.
static int setup_tail(mgr_handle h, AmgH &G, int tail_nnz, cudaStream_t s, Arena &ar) {
    G.tail_k = -1;
    if (tail_nnz <= 0 || G.namg < 3) return ST_OK;
    int kt = -1;
    for (int k = 1; k < G.namg - 1; k++)
        if (G.amg[k].A.nnz <= tail_nnz) {
            kt = k;
            break;
        }
    if (kt < 0) return ST_OK;
    if (G.namg - 1 - kt > TAIL_MAX_PHASES / 4 - 1) kt = G.namg - 1 - (TAIL_MAX_PHASES / 4 - 1);
    const int grid = amg_tail_grid();
    if (grid <= 0) return ST_OK;
    G.tail_k = kt;
    for (int trans = 0; trans < 2; trans++) {
        TailPlan plan;
        plan.spin = h->opt.spin_limit > 0 ? h->opt.spin_limit : 0;
        const bool ok = h->opt.precision == MGR_PREC_FP32 ? build_tail_plan<float>(G, trans, plan)
                                                          : build_tail_plan<double>(G, trans, plan);
        if (!ok) {
            G.tail_k = -1;
            return ST_OK;
        }
        G.tail_plan[trans] = ar.alloc<TailPlan>(1);
        if (!G.tail_plan[trans]) return ST_NOMEM;
        if (cudaMemcpyAsync(G.tail_plan[trans], &plan, sizeof(TailPlan), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return ST_CUDA;
    }
    G.tail_sync = ar.alloc<unsigned>(4);
    if (!G.tail_sync) return ST_NOMEM;
    if (cudaMemsetAsync(G.tail_sync, 0, 4 * sizeof(unsigned), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return ST_CUDA;
    G.tail_grid = grid;
    return ST_OK;
}

// Algorithmic bytes and FP64 FMAs of one tail launch: the sums of the
// per-step kernel classes it replaces.
static void tail_cost(const AmgH &G, double ts, double &bytes, double &fma) {
    const int kt = G.tail_k, kc = G.namg - 1;
    const double f64 = ts == 8 ? 1.0 : 0.0;
    bytes = 0;
    fma = 0;
    for (int k = kt; k < kc; k++) {
        const AmgLevel &L = G.amg[k];
        const double an = L.A.n, annz = L.A.nnz, nc = G.amg[k + 1].A.n;
        const bool cc = (k + 1 == kc);
        bytes += annz * (ts + 4) + (an + 1) * 4 + an * (3 * ts);
        bytes += (double)L.R.nnz * (ts + 4) + (nc + 1) * 4 + an * ts + nc * ts * (cc ? 1 : 3);
        bytes += (double)L.P.nnz * (ts + 4) + (an + 1) * 4 + nc * ts + 2 * an * ts;
        bytes += annz * (ts + 4) + (an + 1) * 4 + an * (4 * ts);
        fma += f64 * (2 * annz + L.R.nnz + L.P.nnz + an);
    }
    bytes += (double)G.nco * G.nco * 8 + 2.0 * G.nco * ts;
    fma += (double)G.nco * G.nco;
}

// Profile names of the AMG steps: [0] the final coarse block's hierarchy,
// [1] an F-relaxation hierarchy.
enum { NM_COARSE, NM_RESID, NM_RESTRICT, NM_PROLONG, NM_POST, NM_SCALE };
static const char *const AMG_NAMES[2][6] = {
    {"coarsest_dense_solve", "amg_residual", "amg_restrict", "amg_prolong", "amg_post_smooth", "amg_scale"},
    {"frelax_coarsest_dense_solve", "frelax_amg_residual", "frelax_amg_restrict", "frelax_amg_prolong",
     "frelax_amg_post_smooth", "frelax_amg_scale"}};

// AMG V(1,1) on level k: r (TV) -> x (TV).  On entry L.xw already holds the
// pre-smoothed iterate D_k r (l1-Jacobi from zero), written by whoever
// produced r.  trans uses A_k^T and the transposed coarsest inverse (the
// exact transpose of the cycle).
template <class T, class TV>
static void amg_cycle(mgr_handle h, AmgH &G, int k, const TV *r, TV *x, int trans) {
    cudaStream_t s = h->s;
    AmgLevel &L = G.amg[k];
    if constexpr (std::is_same<T, TV>::value) {
        if (k == G.tail_k && G.tail_grid > 0 && (const void *)r == (const void *)Sel<T>::r(L) &&
            (void *)x == (void *)Sel<T>::x(L)) {
            double by, fm;
            tail_cost(G, sizeof(T), by, fm);
            int rc;
            {
                KScope ks(h, "amg_tail", k, by, fm);
                rc = launch_amg_tail<T>(G.tail_plan[trans ? 1 : 0], G.tail_grid, G.tail_sync, s);
            }
            if (rc == cudaSuccess) return;
            // a refused cooperative launch: clear it, keep to one launch per step
            cudaGetLastError();
            G.tail_grid = 0;
        }
    }
    if (k == G.namg - 1) {
        KScope ks(h, AMG_NAMES[G.frelax][NM_COARSE], k, (double)G.nco * G.nco * 8 + 2.0 * G.nco * sizeof(TV),
                  (double)G.nco * G.nco);
        launch_dense_matvec<TV>(G.nco, trans ? G.coinvT : G.coinv, r, x, s);
        return;
    }
    const DCSR &A = trans ? L.AT : L.A;
    const T *av = Sel<T>::v(A);
    const T *d = Sel<T>::dinv(L);
    T *xw = Sel<T>::xw(L), *res = Sel<T>::res(L);
    AmgLevel &C = G.amg[k + 1];
    const bool c_coarsest = (k + 1 == G.namg - 1);
    const double ts = sizeof(T), tv = sizeof(TV);
    const double f64 = sizeof(T) == 8 ? 1.0 : 0.0;  // FP64 FMAs only in the FP64 form
    double an = A.n, annz = A.nnz, nc = C.A.n;
    {
        KScope ks(h, AMG_NAMES[G.frelax][NM_RESID], k, annz * (ts + 4) + (an + 1) * 4 + an * (2 * ts + tv), f64 * annz);
        launch_amg_residual<T, TV>(A, av, xw, r, res, s);
    }
    {
        KScope ks(h, AMG_NAMES[G.frelax][NM_RESTRICT], k, (double)L.R.nnz * (ts + 4) + (nc + 1) * 4 + an * ts + nc * ts * (c_coarsest ? 1 : 3),
                  f64 * L.R.nnz);
        if (c_coarsest) launch_csr_spmv<T>(L.R, Sel<T>::v(L.R), res, Sel<T>::r(C), s);
        else launch_restrict_scaled<T>(L.R, Sel<T>::v(L.R), res, Sel<T>::r(C), Sel<T>::dinv(C), Sel<T>::xw(C), s);
    }
    amg_cycle<T, T>(h, G, k + 1, Sel<T>::r(C), Sel<T>::x(C), trans);
    {
        KScope ks(h, AMG_NAMES[G.frelax][NM_PROLONG], k, (double)L.P.nnz * (ts + 4) + (an + 1) * 4 + nc * ts + 2 * an * ts, f64 * L.P.nnz);
        launch_csr_spmv_add<T>(L.P, Sel<T>::v(L.P), Sel<T>::x(C), xw, s);
    }
    {
        KScope ks(h, AMG_NAMES[G.frelax][NM_POST], k, annz * (ts + 4) + (an + 1) * 4 + an * (2 * ts + 2 * tv), f64 * (annz + an));
        launch_amg_post_smooth<T, TV>(A, av, d, r, xw, x, s);
    }
}

// x_0 = D_0 r for the AMG entry when r is not produced by a fused epilogue
template <class T, class TV>
static void amg_prepare(mgr_handle h, AmgH &G, const TV *r) {
    if (G.namg < 2) return;
    AmgLevel &L = G.amg[0];
    KScope ks(h, AMG_NAMES[G.frelax][NM_SCALE], 0, (double)L.A.n * (2 * sizeof(T) + sizeof(TV)));
    launch_scale<T, TV>(L.A.n, Sel<T>::dinv(L), r, Sel<T>::xw(L), h->s);
}

// Transposed cycle, sweeps after the first: r_F = y_F - A_FF^T z_F.  y_F is
// v_F - A_CF^T e_C, rebuilt from v for injection, or kept in y_F (it also
// holds - A_FF^T Z^T e_C) for the restriction of Eq. 5.
template <class T, class TV>
static void t_sweep_residual(mgr_handle h, int l, const TV *v) {
    cudaStream_t s = h->s;
    MgrLevel &L = h->lev[l];
    T *zF = Sel<T>::zF(L), *rF = Sel<T>::rF(L), *eC = Sel<T>::eC(L);
    const double ts = sizeof(T), tv = sizeof(TV), nF = L.nF, nC = L.nC;
    if (L.rtype == MGR_RESTRICT_JACOBI) {
        KScope ks(h, "mgrT_frelax_residual", l, (double)L.AFFT.nnz * (ts + 4) + (nF + 1) * 4 + nF * (4 + 3 * ts));
        launch_csr_axpy_gather<T, T>(L.AFFT, Sel<T>::v(L.AFFT), zF, L.fiota, Sel<T>::yF(L), (T)-1, rF, s);
        return;
    }
    { KScope ks(h, "mgrT_interp", l, (double)L.ACFT.nnz * (ts + 4) + (nF + 1) * 4 + nC * ts + nF * (4 + tv + ts));
      launch_csr_axpy_gather<T, TV>(L.ACFT, Sel<T>::v(L.ACFT), eC, L.fidx, v, (T)-1, rF, s); }
    { KScope ks(h, "mgrT_frelax_residual", l, (double)L.AFFT.nnz * (ts + 4) + (nF + 1) * 4 + nF * (4 + 3 * ts));
      launch_csr_axpy_gather<T, T>(L.AFFT, Sel<T>::v(L.AFFT), zF, L.fiota, rF, (T)-1, rF, s); }
}

// AMG F-relaxation of MGR level l (MGR_U, Sec. 4.3): s sweeps of
// z_F += omega B (y_F - A_FF z_F) from z_F = 0, B one AMG V(1,1) cycle on A_FF
// (trans: the transposed cycle on A_FF^T).  Forward: y_F = v_F, gathered
// here; transposed: y_F is already in r_F and is rebuilt for later sweeps.
template <class T, class TV>
static void frelax_amg(mgr_handle h, int l, const TV *v, int trans) {
    cudaStream_t s = h->s;
    MgrLevel &L = h->lev[l];
    AmgH &G = *L.famg;
    T *zF = Sel<T>::zF(L), *rF = Sel<T>::rF(L), *tF = Sel<T>::tF(L);
    const T om = (T)L.omega;
    const double ts = sizeof(T), tv = sizeof(TV), nF = L.nF;
    if (!trans) {
        KScope ks(h, "mgr_frelax_gather", l, nF * (4 + tv + ts));
        launch_gather<T, TV>(L.fidx, L.nF, v, rF, s);
    }
    for (int sw = 0; sw < L.sweeps; sw++) {
        if (sw > 0) {
            if (!trans) {
                KScope ks(h, "mgr_frelax_residual", l, (double)L.AFF.nnz * (ts + 4) + (nF + 1) * 4 + nF * (4 + tv + 2 * ts));
                launch_frelax_residual<T, TV>(L.AFF, Sel<T>::v(L.AFF), L.fidx, v, zF, rF, s);
            } else {
                t_sweep_residual<T, TV>(h, l, v);
            }
        }
        amg_prepare<T, T>(h, G, rF);
        if (sw == 0 && L.omega == 1.0) {
            amg_cycle<T, T>(h, G, 0, rF, zF, trans);  // z_F = 1 * B y_F
            continue;
        }
        amg_cycle<T, T>(h, G, 0, rF, tF, trans);
        KScope ks(h, "mgr_frelax_scale", l, nF * (sw > 0 ? 3 : 2) * ts);
        launch_frelax_scale<T>(L.nF, om, tF, zF, sw > 0, s);
    }
}

// MGR level l forward cycle (Algorithm 1): v (TV) -> z (TV)
template <class T, class TV>
static void mgr_cycle(mgr_handle h, int l, const TV *v, TV *z) {
    cudaStream_t s = h->s;
    if (l == h->nlev) {
        if (l == 0) amg_prepare<T, TV>(h, h->H, v);
        amg_cycle<T, TV>(h, h->H, 0, v, z, 0);
        return;
    }
    MgrLevel &L = h->lev[l];
    T *zF = Sel<T>::zF(L), *rF = Sel<T>::rF(L), *vC = Sel<T>::vC(L), *eC = Sel<T>::eC(L);
    const T *dinv = Sel<T>::dinv(L);
    T om = (T)L.omega;
    const double ts = sizeof(T), tv = sizeof(TV);
    const double f64 = sizeof(T) == 8 ? 1.0 : 0.0;
    double nF = L.nF, nC = L.nC, gs = L.relax == 2 ? 4.0 : 1.0;
    if (L.famg) {
        frelax_amg<T, TV>(h, l, v, 0);
    } else {
        KScope ks(h, "mgr_frelax_first", l, nF * (gs * ts + 4 + tv + ts + (L.relax == 2 ? 8 : 0)));
        launch_frelax_first<T, TV>(L.nF, L.fidx, L.gstart, L.gsize, dinv, om, v, zF, s);
    }
    for (int sw = 1; sw < L.sweeps && !L.famg; sw++) {
        {
            KScope ks(h, "mgr_frelax_residual", l, (double)L.AFF.nnz * (ts + 4) + (nF + 1) * 4 + nF * (4 + tv + 2 * ts));
            launch_frelax_residual<T, TV>(L.AFF, Sel<T>::v(L.AFF), L.fidx, v, zF, rF, s);
        }
        KScope ks(h, "mgr_frelax_update", l, nF * (gs * ts + 3 * ts + 8));
        launch_frelax_update<T>(L.nF, L.gstart, L.gsize, dinv, om, rF, zF, 0, s);
    }
    if (L.rtype == MGR_RESTRICT_JACOBI) {
        // r_F = v_F - A_FF z_F for the restricted residual of Eq. 5
        KScope ks(h, "mgr_frelax_residual", l, (double)L.AFF.nnz * (ts + 4) + (nF + 1) * 4 + nF * (4 + tv + 2 * ts));
        launch_frelax_residual<T, TV>(L.AFF, Sel<T>::v(L.AFF), L.fidx, v, zF, rF, s);
    }
    {
        const bool fuse = (l + 1 == h->nlev) && h->H.namg > 1 && L.rtype == MGR_RESTRICT_INJECTION;
        KScope ks(h, "mgr_restrict", l, (double)L.ACF.nnz * (ts + 4) + (nC + 1) * 4 + nF * ts + nC * (4 + tv + ts + (fuse ? 2 * ts : 0)),
                  f64 * L.ACF.nnz);
        if (fuse) launch_mgr_restrict_scaled<T, TV>(L.ACF, Sel<T>::v(L.ACF), L.cidx, v, zF, vC,
                                                    Sel<T>::dinv(h->H.amg[0]), Sel<T>::xw(h->H.amg[0]), s);
        else launch_mgr_restrict<T, TV>(L.ACF, Sel<T>::v(L.ACF), L.cidx, v, zF, vC, s);
    }
    if (L.rtype == MGR_RESTRICT_JACOBI) {
        {
            KScope ks(h, "mgr_restrict_z", l, (double)L.Z.nnz * (ts + 4) + (nC + 1) * 4 + nF * ts + 2 * nC * ts,
                      f64 * L.Z.nnz);
            launch_csr_spmv_add<T>(L.Z, Sel<T>::v(L.Z), rF, vC, s);  // r_C += Z r_F
        }
        if (l + 1 == h->nlev) amg_prepare<T, T>(h, h->H, vC);
    }
    mgr_cycle<T, T>(h, l + 1, vC, eC);
    {
        KScope ks(h, "mgr_interp", l, (double)L.W.nnz * (ts + 4) + (nF + 1) * 4 + nC * (ts + 4 + tv) + nF * (ts + 4 + tv),
                  f64 * L.W.nnz);
        launch_mgr_interp<T, TV>(L.W, Sel<T>::v(L.W), L.nC, L.fidx, L.cidx, zF, eC, z, s);
    }
}

// exact transpose of mgr_cycle:
//   r_C = v_C + W^T v_F; e_C = B^T r_C; z_C = e_C; z_F = K^T (v_F - A_CF^T e_C)
template <class T, class TV>
static void mgr_cycle_t(mgr_handle h, int l, const TV *v, TV *z) {
    cudaStream_t s = h->s;
    if (l == h->nlev) {
        amg_prepare<T, TV>(h, h->H, v);
        amg_cycle<T, TV>(h, h->H, 0, v, z, 1);
        return;
    }
    MgrLevel &L = h->lev[l];
    T *zF = Sel<T>::zF(L), *rF = Sel<T>::rF(L), *vC = Sel<T>::vC(L), *eC = Sel<T>::eC(L);
    const T *dinv = Sel<T>::dinv(L);
    T om = (T)L.omega;
    const double ts = sizeof(T), tv = sizeof(TV);
    double nF = L.nF, nC = L.nC, gs = L.relax == 2 ? 4.0 : 1.0;
    { KScope ks(h, "mgrT_gather", l, nF * (4 + tv + ts));
      launch_gather<T, TV>(L.fidx, L.nF, v, zF, s); }               // zF <- v_F (scratch)
    { KScope ks(h, "mgrT_restrict", l, (double)L.WT.nnz * (ts + 4) + (nC + 1) * 4 + nF * ts + nC * (4 + tv + ts));
      launch_csr_axpy_gather<T, TV>(L.WT, Sel<T>::v(L.WT), zF, L.cidx, v, (T)1, vC, s); }
    mgr_cycle_t<T, T>(h, l + 1, vC, eC);
    { KScope ks(h, "mgrT_interp", l, (double)L.ACFT.nnz * (ts + 4) + (nF + 1) * 4 + nC * ts + nF * (4 + tv + ts));
      launch_csr_axpy_gather<T, TV>(L.ACFT, Sel<T>::v(L.ACFT), eC, L.fidx, v, (T)-1, rF, s); }  // y_F
    T *qF = Sel<T>::qF(L);
    if (L.rtype == MGR_RESTRICT_JACOBI) {
        // q_F = Z^T e_C;  y_F -= A_FF^T q_F (kept in y_F for later sweeps)
        { KScope ks(h, "mgrT_restrict_z", l, (double)L.ZT.nnz * (ts + 4) + (nF + 1) * 4 + nC * ts + nF * ts,
                    (sizeof(T) == 8 ? 1.0 : 0.0) * L.ZT.nnz);
          launch_csr_spmv<T>(L.ZT, Sel<T>::v(L.ZT), eC, qF, s); }
        { KScope ks(h, "mgrT_frelax_residual", l, (double)L.AFFT.nnz * (ts + 4) + (nF + 1) * 4 + nF * (4 + 3 * ts));
          launch_csr_axpy_gather<T, T>(L.AFFT, Sel<T>::v(L.AFFT), qF, L.fiota, rF, (T)-1, rF, s); }
        if (L.sweeps > 1) cudaMemcpyAsync(Sel<T>::yF(L), rF, sizeof(T) * L.nF, cudaMemcpyDeviceToDevice, s);
    }
    auto finish = [&]() {
        if (L.rtype == MGR_RESTRICT_JACOBI) {
            KScope ks(h, "mgr_frelax_scale", l, nF * 3 * ts);
            launch_frelax_scale<T>(L.nF, (T)1, qF, zF, 1, s);  // z_F = K^T y_F + q_F
        }
        KScope ks(h, "mgrT_scatter", l, (nF + nC) * (4 + ts + tv));
        launch_scatter2<T, TV>(L.nF, L.nC, L.fidx, L.cidx, zF, eC, z, s);
    };
    if (L.famg) {
        frelax_amg<T, TV>(h, l, v, 1);
        finish();
        return;
    }
    // K^T y_F: sweeps of z += omega D^{-T} (y - A_FF^T z) from z = 0
    cudaMemsetAsync(zF, 0, sizeof(T) * L.nF, s);
    { KScope ks(h, "mgrT_frelax_update", l, nF * (gs * ts + 3 * ts + 8));
      launch_frelax_update<T>(L.nF, L.gstart, L.gsize, dinv, om, rF, zF, 1, s); }
    for (int sw = 1; sw < L.sweeps; sw++) {
        t_sweep_residual<T, TV>(h, l, v);  // r_F = y_F - A_FF^T z_F
        KScope ks(h, "mgrT_frelax_update", l, nF * (gs * ts + 3 * ts + 8));
        launch_frelax_update<T>(L.nF, L.gstart, L.gsize, dinv, om, rF, zF, 1, s);
    }
    finish();
}

static void vcycle(mgr_handle h, const double *v, double *z, int trans) {
    if (h->opt.precision == MGR_PREC_FP32) {
        if (trans) mgr_cycle_t<float, double>(h, 0, v, z);
        else mgr_cycle<float, double>(h, 0, v, z);
    } else {
        if (trans) mgr_cycle_t<double, double>(h, 0, v, z);
        else mgr_cycle<double, double>(h, 0, v, z);
    }
}

static double outer_bytes(mgr_handle h) {
    double b = h->b;
    return (double)h->nnzb * (b * b * 8 + 4) + (h->nb + 1.0) * 4 + 2.0 * h->n * 8;
}

static void outer_spmv(mgr_handle h, const double *x, double *y, int trans) {
    KScope ks(h, trans ? "spmv_AT" : "spmv_A", -1, outer_bytes(h), (double)h->nnzb * h->b * h->b);
    if (trans) launch_csr_spmv<double>(h->A0T, h->A0T.v, x, y, h->s);
    else if (h->b == 1) launch_csr_spmv<double>(h->Aout, h->Aout.v, x, y, h->s);
    else launch_bsr_spmv(h->nb, h->b, h->brp, h->bci, h->bval, x, y, 1.0, 0.0, h->s, h->nnzb);
}

static void outer_residual(mgr_handle h, const double *x, const double *bvec, double *y, int trans) {
    KScope ks(h, trans ? "residual_AT" : "residual_A", -1, outer_bytes(h) + h->n * 8.0, (double)h->nnzb * h->b * h->b);
    if (trans) launch_csr_residual(h->A0T, x, bvec, y, h->s);
    else if (h->b == 1) launch_csr_residual(h->Aout, x, bvec, y, h->s);
    else launch_bsr_residual(h->nb, h->b, h->brp, h->bci, h->bval, x, bvec, y, h->s, h->nnzb);
}

extern "C" mgr_status mgr_apply(mgr_handle h, const double *v, double *z) {
    if (!h || !v || !z) return fail(h, MGR_ERR_INVALID, "NULL argument");
    if (!h->ready) return fail(h, MGR_ERR_INVALID, "no hierarchy (a refresh failed)");
    vcycle(h, v, z, 0);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_apply");
    if (tail_timed_out(h))
        return fail(h, MGR_ERR_TIMEOUT, "a grid barrier of the fused AMG tail ran out of time");
    return MGR_OK;
}

extern "C" mgr_status mgr_apply_transpose(mgr_handle h, const double *v, double *z) {
    if (!h || !v || !z) return fail(h, MGR_ERR_INVALID, "NULL argument");
    if (!h->ready) return fail(h, MGR_ERR_INVALID, "no hierarchy (a refresh failed)");
    vcycle(h, v, z, 1);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_apply_transpose");
    if (tail_timed_out(h))
        return fail(h, MGR_ERR_TIMEOUT, "a grid barrier of the fused AMG tail ran out of time");
    return MGR_OK;
}

extern "C" mgr_status mgr_spmv(mgr_handle h, const double *x, double *y) {
    if (!h || !x || !y) return fail(h, MGR_ERR_INVALID, "NULL argument");
    outer_spmv(h, x, y, 0);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_spmv");
    return MGR_OK;
}

// ----------------------------------------------------------------- FGMRES
// One Arnoldi step j: z_j = M^{-1} v_j, w = A z_j (stored in V_{j+1}),
// classical Gram-Schmidt against V_0..V_j with the norm of w taken in the
// same pass and a conditional second pass, Givens update, status to the
// pinned host mirror, then v_{j+1} = w / h_{j+1,j}.
static void arnoldi_step(mgr_handle h, int j, int trans) {
    Krylov &K = h->kr;
    cudaStream_t s = h->s;
    long long n = K.n;
    double *vj = K.V + j * n, *zj = K.Z + j * n, *w = K.V + (j + 1) * n;
    vcycle(h, vj, zj, trans);
    outer_spmv(h, zj, w, trans);
    double nd = (double)n;
    int k = j + 1;
    // first pass: projections on V_0..V_j and |w|^2 (w = V_{j+1} itself)
    { KScope ks(h, "arnoldi_dots", -1, (k + 1) * nd * 8, (k + 1) * nd);
      launch_dots(K.V, n, k + 1, w, (int)n, K.partial, K.h1, K.ticket, nullptr, K.nblk, s); }
    { KScope ks(h, "arnoldi_update_norm", -1, k * nd * 8 + 2 * nd * 8, (k + 1) * nd);
      launch_update_norm(K.V, n, k, K.h1, w, (int)n, K.partial, K.nrm2, K.ticket, K.flag, 1, K.nblk, s); }
    // second pass only when the first cancelled most of w (device flag)
    { KScope ks(h, "arnoldi_reorth", -1, 0.0);
      launch_dots(K.V, n, k, w, (int)n, K.partial, K.h2, K.ticket, K.flag, K.nblk, s); }
    { KScope ks(h, "arnoldi_reorth", -1, 0.0);
      launch_update_norm(K.V, n, k, K.h2, w, (int)n, K.partial, K.nrmB, K.ticket, K.flag, 2, K.nblk, s); }
    { KScope ks(h, "givens", -1, 0.0);
      launch_arnoldi_finish(j, K.m, K.h1, K.h2, K.nrm2, K.nrmB, K.flag, K.H, K.cs, K.sn, K.g, K.hn, K.stat, K.tol, s); }
    cudaMemcpyAsync(K.hstat, K.stat, 5 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (h->H.tail_sync)  // the fused tail's error word, read after every step
        cudaMemcpyAsync(K.hstat + 6, h->H.tail_sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    { KScope ks(h, "vec_scale", -1, nd * 16);
      launch_vec_scale(w, w, K.hn, nullptr, 1, (int)n, s); }
}

// Run step j, from a captured CUDA graph when enabled (one graph per
// (direction, j), captured on first use and replayed afterwards; the
// kernels read every per-solve scalar from device memory).
static cudaError_t run_step(mgr_handle h, int j, int trans) {
    Krylov &K = h->kr;
    if (!h->opt.use_graphs || h->prof.on) {
        arnoldi_step(h, j, trans);
        return cudaGetLastError();
    }
    auto &gv = K.graphs[trans];
    if ((int)gv.size() < K.m) gv.resize(K.m, nullptr);
    if (!gv[j]) {
        cudaGraph_t g = nullptr;
        long long before = g_launches.load();
        cudaError_t e = cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        arnoldi_step(h, j, trans);
        e = cudaStreamEndCapture(h->s, &g);
        if (e != cudaSuccess) return e;
        // the launches recorded during capture execute at replay time
        K.graph_kernels[trans][j] = g_launches.load() - before;
        g_launches.fetch_sub(K.graph_kernels[trans][j]);
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        gv[j] = ex;
    }
    g_launches.fetch_add(K.graph_kernels[trans][j]);
    return cudaGraphLaunch(gv[j], h->s);
}

static mgr_status fgmres(mgr_handle h, const double *b, double *x, double rtol, int maxit, int trans,
                         mgr_solve_info *info) {
    if (!h || !b || !x) return fail(h, MGR_ERR_INVALID, "NULL argument");
    if (!h->ready) return fail(h, MGR_ERR_INVALID, "no hierarchy (a refresh failed)");
    if (!(rtol >= 0.0)) return fail(h, MGR_ERR_INVALID, "rtol must be >= 0");
    Nvtx nv(trans ? "mgr_solve_transpose" : "mgr_solve");
    auto t0 = std::chrono::steady_clock::now();
    Krylov &K = h->kr;
    cudaStream_t s = h->s;
    long long n = K.n;
    int m = K.m;
    { KScope ks(h, "norm", -1, n * 8.0);
      launch_dot(b, b, (int)n, K.partial, K.beta, K.ticket, 1, K.nblk, s); }
    double bn = 0.0;
    cudaMemcpyAsync(&bn, K.beta, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "solve");
    if (!isfinite(bn)) return fail(h, MGR_ERR_INVALID, "right-hand side is not finite");
    int it = 0, reorth = 0;
    double relres = 0.0;
    mgr_status st = MGR_ERR_NOT_CONVERGED;
    if (bn == 0.0) {
        K.hist.assign(1, 0.0);
        cudaMemsetAsync(x, 0, sizeof(double) * n, s);
        cudaStreamSynchronize(s);
        relres = 0.0;
        st = MGR_OK;
    } else {
        double tol_abs = rtol * bn;
        cudaMemcpyAsync(K.tol, &tol_abs, sizeof(double), cudaMemcpyHostToDevice, s);
        K.hist.clear();
        K.hstat[6] = 0.0;
        for (;;) {
            outer_residual(h, x, b, K.r, trans);
            { KScope ks(h, "norm", -1, n * 8.0);
              launch_dot(K.r, K.r, (int)n, K.partial, K.beta, K.ticket, 1, K.nblk, s); }
            double beta = 0.0;
            cudaMemcpyAsync(&beta, K.beta, sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "solve residual");
            relres = beta / bn;
            if (it == 0) K.hist.push_back(relres);
            if (!isfinite(beta)) { st = MGR_ERR_INVALID; h->err = "residual is not finite"; break; }
            if (beta <= tol_abs) { st = MGR_OK; break; }
            if (it >= maxit) break;
            { KScope ks(h, "vec_scale", -1, n * 16.0);
              launch_vec_scale(K.r, K.V, K.beta, nullptr, 1, (int)n, s); }
            { KScope ks(h, "givens", -1, 0.0);
              launch_init_g(K.g, m, K.beta, s); }
            int k = 0;
            for (int j = 0; j < m && it < maxit; j++) {
                cudaError_t ge = run_step(h, j, trans);
                cudaStreamSynchronize(s);
                if (ge != cudaSuccess || cudaGetLastError() != cudaSuccess) return cuda_fail(h, "Arnoldi step");
                it++;
                k = j + 1;
                double est = K.hstat[0];
                K.hist.push_back(est / bn);
                int conv = K.hstat[1] != 0.0, brk = K.hstat[2] != 0.0;
                if (!isfinite(est)) { st = MGR_ERR_INVALID; break; }
                if (K.hstat[4] != 0.0) reorth++;
                unsigned tail_err = 0;
                memcpy(&tail_err, K.hstat + 6, sizeof(unsigned));
                if (tail_err) { st = MGR_ERR_TIMEOUT; break; }
                if (conv || brk) break;
            }
            if (st == MGR_ERR_INVALID) { h->err = "preconditioned residual is not finite"; break; }
            // a preconditioner that left its tail early is not applied to x
            if (st == MGR_ERR_TIMEOUT) break;
            { KScope ks(h, "givens", -1, 0.0);
              launch_solve_upper(k, m, K.H, K.g, K.y, s); }
            { KScope ks(h, "update_x", -1, (k + 2.0) * n * 8, (double)k * n);
              launch_multi_axpy(K.Z, n, k, K.y, x, (int)n, s); }
        }
    }
    cudaStreamSynchronize(s);
    if (tail_timed_out(h) || st == MGR_ERR_TIMEOUT) {
        st = MGR_ERR_TIMEOUT;
        h->err = "a grid barrier of the fused AMG tail ran out of time";
    }
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iterations = it;
        info->rel_residual = relres;
        info->setup_ms = h->setup_ms;
        info->solve_ms = ms;
        info->mgr_levels = h->nlev;
        info->amg_levels = h->H.namg;
        int q = 0;
        double tot = 0, base = 0;
        for (int l = 0; l < h->nlev && q < 40; l++, q++) { info->level_rows[q] = h->lev[l].n; info->level_nnz[q] = h->lev[l].A.nnz; }
        for (int k = 0; k < h->H.namg && q < 40; k++, q++) {
            info->level_rows[q] = h->H.amg[k].A.n; info->level_nnz[q] = h->H.amg[k].A.nnz;
            tot += h->H.amg[k].A.nnz;
            if (k == 0) base = h->H.amg[k].A.nnz;
        }
        info->operator_complexity = base > 0 ? tot / base : 0.0;
        info->reorth_steps = reorth;
    }
    if (st == MGR_ERR_NOT_CONVERGED) return fail(h, st, "maximum iterations reached");
    if (st != MGR_OK) return fail(h, st, h->err);
    return MGR_OK;
}

extern "C" mgr_status mgr_solve(mgr_handle h, const double *b, double *x, double rtol,
                                int32_t maxit, mgr_solve_info *info) {
    return fgmres(h, b, x, rtol, maxit, 0, info);
}

extern "C" mgr_status mgr_solve_transpose(mgr_handle h, const double *g, double *lam, double rtol,
                                          int32_t maxit, mgr_solve_info *info) {
    return fgmres(h, g, lam, rtol, maxit, 1, info);
}

extern "C" mgr_status mgr_update_values(mgr_handle h, const double *val, int32_t on_device) {
    if (!h || !val) return fail(h, MGR_ERR_INVALID, "NULL argument");
    cudaStream_t s = h->s;
    const long long nv = h->nnzb * h->b * h->b;
    Arena tmp;
    // validated in a scratch copy first: invalid values leave the handle as it was
    double *nvv = tmp.alloc<double>(nv + 1);
    if (!nvv) return fail(h, MGR_ERR_NOMEM, "update scratch");
    cudaMemcpyAsync(nvv, val, sizeof(double) * nv, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    launch_validate_bsr(h->nb, h->b, h->brp, h->bci, nvv, h->errw, s);
    if (read_errw(h)) { tmp.free_all(); return fail(h, MGR_ERR_INVALID, "non-finite matrix value"); }
    cudaMemcpyAsync(h->bval, nvv, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s);
    // the transposed outer operator: same pattern, one gather of the new values
    launch_gather_f64(h->a0t_src, h->bval, h->A0T.v, h->A0T.nnz, s);
    if (h->Aout.sptr) refresh_sell(h->Aout, s);
    if (h->A0T.sptr) refresh_sell(h->A0T, s);
    cudaStreamSynchronize(s);
    tmp.free_all();
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_update_values");
    return MGR_OK;
}

extern "C" mgr_status mgr_refresh(mgr_handle h, const double *val, int32_t on_device) {
    if (!h || !val) return fail(h, MGR_ERR_INVALID, "NULL argument");
    if (h->in_batch) return fail(h, MGR_ERR_UNSUPPORTED, "handles of a batch are not refreshed one by one");
    Nvtx nv("mgr_refresh");
    auto t0 = std::chrono::steady_clock::now();
    mgr_status st = mgr_update_values(h, val, on_device);
    if (st != MGR_OK) return st;
    cudaStream_t s = h->s;
    cudaStreamSynchronize(s);
    // captured graphs and the fused tail point into the old hierarchy
    for (int d = 0; d < 2; d++) {
        for (auto g : h->kr.graphs[d]) if (g) cudaGraphExecDestroy(g);
        h->kr.graphs[d].clear();
    }
    h->ready = false;
    // the slice order each product was timed into at setup: the pattern is
    // the same, so the rebuilt copies keep it instead of being timed again
    std::vector<int> sched_lev, sched_amg;
    auto lev_mats = [](MgrLevel &L) {
        return std::vector<DCSR *>{&L.AFF, &L.ACF, &L.W, &L.AFFT, &L.ACFT, &L.WT, &L.Z, &L.ZT};
    };
    for (int l = 0; l < h->nlev; l++)
        for (DCSR *m : lev_mats(h->lev[l])) sched_lev.push_back(m->sched);
    const int old_namg = h->H.namg;
    for (int k = 0; k < old_namg; k++)
        for (DCSR *m : {&h->H.amg[k].A, &h->H.amg[k].AT, &h->H.amg[k].P, &h->H.amg[k].R})
            sched_amg.push_back(m->sched);
    for (int l = 0; l < MGR_MAX_LEVELS; l++) {
        AmgH *keep = h->lev[l].famg;
        h->lev[l] = MgrLevel();
        h->lev[l].famg = keep;
    }
    h->H = AmgH();
    h->lar.recycle();  // the new hierarchy has the old one's sizes: reuse its blocks
    const bool no_tune = g_no_tune;
    g_no_tune = true;
    st = build_levels(h, true);
    g_no_tune = no_tune;
    if (st == MGR_OK) {
        size_t q = 0;
        for (int l = 0; l < h->nlev; l++)
            for (DCSR *m : lev_mats(h->lev[l])) m->sched = sched_lev[q++];
        q = 0;
        for (int k = 0; k < old_namg && k < h->H.namg; k++)
            for (DCSR *m : {&h->H.amg[k].A, &h->H.amg[k].AT, &h->H.amg[k].P, &h->H.amg[k].R})
                m->sched = sched_amg[q++];
        // A_FF shared with a kept F hierarchy carries that hierarchy's order
        for (int l = 0; l < h->nlev; l++) {
            MgrLevel &L = h->lev[l];
            if (L.fshared && L.famg && L.famg->namg > 1) {
                L.AFF.sched = L.famg->amg[0].A.sched;
                L.AFFT.sched = L.famg->amg[0].AT.sched;
            }
        }
    }
    if (st != MGR_OK) {
        // a partly built F-relaxation hierarchy must not be kept by a later refresh
        for (int l = 0; l < MGR_MAX_LEVELS; l++) {
            if (h->lev[l].famg) h->lev[l].famg->ar.free_all();
            delete h->lev[l].famg;
            h->lev[l].famg = nullptr;
        }
        h->lar.trim();
        return st;
    }
    cudaStreamSynchronize(s);
    h->lar.trim();
    for (int l = 0; l < h->nlev; l++)
        if (h->lev[l].famg) h->lev[l].famg->ar.trim();
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_refresh");
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    h->ready = true;
    return MGR_OK;
}

extern "C" mgr_status mgr_grad_values(mgr_handle h, const double *lam, const double *x,
                                      double *dA_val) {
    if (!h || !lam || !x || !dA_val) return fail(h, MGR_ERR_INVALID, "NULL argument");
    launch_grad_values(h->nb, h->b, h->brp, h->bci, lam, x, dA_val, h->s);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_grad_values");
    return MGR_OK;
}

extern "C" mgr_status mgr_bsr_spmv(int32_t nb, int32_t b, const int32_t *row_ptr,
                                   const int32_t *col_idx, const double *val, const double *x,
                                   double *y, double alpha, double beta, void *stream) {
    if (b < 1 || b > 4 || nb < 0 || !row_ptr || !col_idx || !val || !x || !y)
        return fail(nullptr, MGR_ERR_INVALID, "bad arguments");
    launch_bsr_spmv(nb, b, row_ptr, col_idx, val, x, y, alpha, beta, (cudaStream_t)stream);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(nullptr, "mgr_bsr_spmv");
    return MGR_OK;
}

extern "C" void mgr_free(mgr_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->s);
    for (int l = 0; l < MGR_MAX_LEVELS; l++) {
        if (h->lev[l].famg) h->lev[l].famg->ar.free_all();
        delete h->lev[l].famg;
        h->lev[l].famg = nullptr;
    }
    h->lar.free_all();
    for (int d = 0; d < 2; d++)
        for (auto g : h->kr.graphs[d]) if (g) cudaGraphExecDestroy(g);
    if (h->kr.hstat) cudaFreeHost(h->kr.hstat);
    for (auto e : h->prof.pool) cudaEventDestroy(e);
    h->ar.free_all();
    if (h->own_stream) cudaStreamDestroy(h->s);
    delete h;
}

extern "C" const char *mgr_last_error(mgr_handle h) {
    return h ? h->err.c_str() : g_last_error.c_str();
}

// -------------------------------------------------------------- inspection
// amg = 1: the final coarse block's hierarchy; 2 + l: MGR level l's AMG
// F-relaxation hierarchy (nullptr when that level has none)
static const AmgH *amg_of(mgr_handle h, int amg) {
    if (amg == 1) return &h->H;
    const int l = amg - 2;
    if (l < 0 || l >= h->nlev) return nullptr;
    return h->lev[l].famg;
}

static const DCSR *pick(mgr_handle h, int amg, int level, int which) {
    if (!amg) {
        if (level < 0 || level > h->nlev) return nullptr;
        if (level == h->nlev) return which == 0 ? &h->H.amg[0].A : nullptr;
        MgrLevel &L = h->lev[level];
        switch (which) {
            case 0: return &L.A;
            case 1: return &L.AFF;
            case 2: return &L.AFC;
            case 3: return &L.ACF;
            case 4: return &L.W;
            case 5: return L.rtype == MGR_RESTRICT_JACOBI ? &L.Z : nullptr;
        }
        return nullptr;
    }
    const AmgH *G = amg_of(h, amg);
    if (!G || level < 0 || level >= G->namg) return nullptr;
    if (which == 0) return &G->amg[level].A;
    if (which == 1) return G->amg[level].P.rp ? &G->amg[level].P : nullptr;
    return nullptr;
}

extern "C" mgr_status mgr_get_matrix(mgr_handle h, int32_t amg, int32_t level, int32_t which,
                                     int32_t *dims, int32_t *rp, int32_t *ci, double *v) {
    if (!h || !dims) return fail(h, MGR_ERR_INVALID, "NULL argument");
    const DCSR *M = pick(h, amg, level, which);
    if (!M) { dims[0] = dims[1] = dims[2] = -1; return fail(h, MGR_ERR_INVALID, "no such matrix"); }
    dims[0] = M->n; dims[1] = M->m; dims[2] = M->nnz;
    cudaStreamSynchronize(h->s);
    if (rp) cudaMemcpy(rp, M->rp, sizeof(int) * (M->n + 1), cudaMemcpyDeviceToHost);
    if (ci && M->nnz) cudaMemcpy(ci, M->ci, sizeof(int) * M->nnz, cudaMemcpyDeviceToHost);
    if (v && M->nnz) cudaMemcpy(v, M->v, sizeof(double) * M->nnz, cudaMemcpyDeviceToHost);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_get_matrix");
    return MGR_OK;
}

extern "C" mgr_status mgr_get_cf(mgr_handle h, int32_t level, int32_t *cf) {
    return mgr_get_amg_cf(h, 1, level, cf);
}

extern "C" mgr_status mgr_get_amg_cf(mgr_handle h, int32_t amg, int32_t level, int32_t *cf) {
    if (!h || !cf) return fail(h, MGR_ERR_INVALID, "NULL argument");
    const AmgH *G = amg_of(h, amg);
    if (!G || level < 0 || level >= G->namg - 1 || !G->amg[level].cf) return fail(h, MGR_ERR_INVALID, "no C/F split on that level");
    cudaStreamSynchronize(h->s);
    cudaMemcpy(cf, G->amg[level].cf, sizeof(int) * G->amg[level].A.n, cudaMemcpyDeviceToHost);
    return MGR_OK;
}

extern "C" int32_t mgr_get_amg_levels(mgr_handle h, int32_t amg) {
    if (!h) return 0;
    const AmgH *G = amg_of(h, amg);
    return G ? G->namg : 0;
}

extern "C" mgr_status mgr_get_dinv(mgr_handle h, int32_t level, double *dinv, int32_t *gsize) {
    if (!h || !dinv || !gsize) return fail(h, MGR_ERR_INVALID, "NULL argument");
    if (level < 0 || level >= h->nlev) return fail(h, MGR_ERR_INVALID, "no such MGR level");
    MgrLevel &L = h->lev[level];
    cudaStreamSynchronize(h->s);
    cudaMemcpy(dinv, L.dinv, sizeof(double) * 4 * L.nF, cudaMemcpyDeviceToHost);
    cudaMemcpy(gsize, L.gsize, sizeof(int) * L.nF, cudaMemcpyDeviceToHost);
    return MGR_OK;
}

// Every index array of the hierarchy against the size of what it indexes
// (check.cu), and the shapes of consecutive operators.
static int check_amg(const AmgH &G, unsigned long long *bad, cudaStream_t s, Arena &ar) {
    int rc = 0;
    unsigned long long hb = 0;
    for (int k = 0; k < G.namg; k++) {
        const AmgLevel &L = G.amg[k];
        rc |= check_csr(L.A, bad, s, ar);
        rc |= check_csr(L.AT, bad, s, ar);
        hb += L.A.n != L.A.m || L.AT.n != L.A.n || L.AT.nnz != L.A.nnz;
        if (k + 1 < G.namg) {
            const int nc = G.amg[k + 1].A.n;
            rc |= check_csr(L.P, bad, s, ar);
            rc |= check_csr(L.R, bad, s, ar);
            hb += L.P.n != L.A.n || L.P.m != nc || L.R.n != nc || L.R.m != L.A.n;
        }
    }
    hb += G.namg < 1 || G.nco != G.amg[G.namg - 1].A.n;
    rc |= check_add(bad, hb, s);
    return rc;
}

extern "C" mgr_status mgr_check_hierarchy(mgr_handle h, int64_t *violations) {
    if (!h || !violations) return fail(h, MGR_ERR_INVALID, "NULL argument");
    if (!h->ready) return fail(h, MGR_ERR_INVALID, "no hierarchy (a refresh failed)");
    cudaStream_t s = h->s;
    Arena tmp;
    unsigned long long *bad = tmp.alloc<unsigned long long>(1);
    if (!bad) return fail(h, MGR_ERR_NOMEM, "check scratch");
    cudaMemsetAsync(bad, 0, sizeof(*bad), s);
    int rc = 0;
    unsigned long long hb = 0;
    for (int l = 0; l < h->nlev; l++) {
        const MgrLevel &L = h->lev[l];
        const DCSR *ms[] = {&L.AFF, &L.ACF, &L.W, &L.AFFT, &L.ACFT, &L.WT};
        for (const DCSR *m : ms) rc |= check_csr(*m, bad, s, tmp);
        hb += L.AFF.n != L.nF || L.AFF.m != L.nF || L.ACF.n != L.nC || L.ACF.m != L.nF ||
              L.W.n != L.nF || L.W.m != L.nC;
        if (L.rtype == MGR_RESTRICT_JACOBI) {
            rc |= check_csr(L.Z, bad, s, tmp) | check_csr(L.ZT, bad, s, tmp);
            hb += L.Z.n != L.nC || L.Z.m != L.nF || L.ZT.n != L.nF || L.ZT.m != L.nC;
        }
        const int nnext = l + 1 < h->nlev ? h->lev[l + 1].n : h->H.amg[0].A.n;
        hb += nnext != L.nC;
        rc |= check_split(L.n, L.fidx, L.nF, L.cidx, L.nC, L.gstart, L.gsize, bad, s, tmp);
        rc |= check_iota(L.fiota, L.nF, bad, s);
        if (L.famg) {
            rc |= check_amg(*L.famg, bad, s, tmp);
            hb += L.famg->amg[0].A.n != L.nF;
        }
    }
    rc |= check_amg(h->H, bad, s, tmp);
    rc |= check_csr(h->A0T, bad, s, tmp);
    hb += h->A0T.n != h->n || h->A0T.m != h->n;
    if (h->b == 1) rc |= check_csr(h->Aout, bad, s, tmp);
    rc |= check_add(bad, hb, s);
    unsigned long long tot = 0;
    cudaMemcpyAsync(&tot, bad, sizeof(tot), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    tmp.free_all();
    if (rc == ST_NOMEM) return fail(h, MGR_ERR_NOMEM, "check scratch");
    if (rc || cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_check_hierarchy");
    *violations = (int64_t)tot;
    return MGR_OK;
}

extern "C" mgr_status mgr_get_info(mgr_handle h, int32_t *out) {
    if (!h || !out) return fail(h, MGR_ERR_INVALID, "NULL argument");
    out[0] = h->nlev; out[1] = h->H.namg; out[2] = h->n;
    return MGR_OK;
}

extern "C" int32_t mgr_solve_history(mgr_handle h, double *out, int32_t cap) {
    if (!h) return 0;
    const auto &v = h->kr.hist;
    const int32_t cnt = (int32_t)v.size();
    for (int32_t i = 0; out && i < cnt && i < cap; i++) out[i] = v[i];
    return cnt;
}

extern "C" int64_t mgr_launch_count(void) { return g_launches.load(); }

extern "C" mgr_status mgr_profile(mgr_handle h, int32_t on) {
    if (!h) return fail(h, MGR_ERR_INVALID, "NULL handle");
    prof_resolve(h);
    Prof &P = h->prof;
    P.names.clear(); P.ms.clear(); P.bytes.clear(); P.fma.clear(); P.cnt.clear(); P.ptag.clear(); P.used = 0;
    P.on = on != 0;
    return MGR_OK;
}

extern "C" int32_t mgr_profile_entries(mgr_handle h) {
    if (!h) return 0;
    prof_resolve(h);
    return (int32_t)h->prof.names.size();
}

extern "C" mgr_status mgr_profile_entry(mgr_handle h, int32_t i, char *name, int32_t name_cap,
                                        double *total_ms, int64_t *launches,
                                        double *bytes_per_launch, double *fp64_fma_per_launch) {
    if (!h) return fail(h, MGR_ERR_INVALID, "NULL handle");
    prof_resolve(h);
    Prof &P = h->prof;
    if (i < 0 || i >= (int32_t)P.names.size()) return fail(h, MGR_ERR_INVALID, "no such entry");
    if (name && name_cap > 0) { strncpy(name, P.names[i].c_str(), name_cap - 1); name[name_cap - 1] = 0; }
    if (total_ms) *total_ms = P.ms[i];
    if (launches) *launches = P.cnt[i];
    // per-launch figures averaged over the recorded launches (they vary with
    // the Arnoldi step)
    double nrec = P.cnt[i] > 0 ? (double)P.cnt[i] : 1.0;
    if (bytes_per_launch) *bytes_per_launch = P.bytes[i] / nrec;
    if (fp64_fma_per_launch) *fp64_fma_per_launch = P.fma[i] / nrec;
    return MGR_OK;
}

// ================================================================ batched
// Many systems of uneven sizes solved together: each keeps its own hierarchy
// (built by mgr_setup), and every kernel class runs as ONE launch over all
// systems through a job table (per-system operands + a prefix of work items).
// The V-cycle is level-synchronous across systems; FGMRES reductions are
// segmented per system; converged systems drop out through device flags.

namespace mgr {

struct BTable {
    BJob *jobs = nullptr;
    long long *prefix = nullptr;
    int njobs = 0;
    long long total = 0;
    int R = 1;
    // 0 chunk (warp-chunks of R rows), 1 elements, 2 reduction blocks,
    // 3 SELL slices (the same row products over the members' SELL copies)
    int kind = 0;
    bool sell_ok = false;  // every member's matrix has a SELL copy (kind 0 may become 3)
    std::vector<BJob> host;
};

struct BKry {  // one system's Krylov scalars for the per-system bookkeeping kernels
    double *h1, *h2, *nrm2, *nrmB, *H, *cs, *sn, *g, *hn, *stat, *beta, *y;
    const double *tol;
    int *flag, *active, *kk;
};

__global__ void k_bgivens(BKry *kr, int nsys, int j, int m) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    BKry K = kr[s];
    if (!*K.active) return;
    const int re = *K.flag;
    double w0 = sqrt(K.h1[j + 1]);
    for (int i = 0; i <= j; i++) K.H[i * m + j] = re ? K.h1[i] + K.h2[i] : K.h1[i];
    double hn = sqrt(re ? *K.nrmB : *K.nrm2);
    for (int i = 0; i < j; i++) {
        double a = K.H[i * m + j], b = K.H[(i + 1) * m + j];
        K.H[i * m + j] = K.cs[i] * a + K.sn[i] * b;
        K.H[(i + 1) * m + j] = -K.sn[i] * a + K.cs[i] * b;
    }
    double a = K.H[j * m + j], b = hn;
    double rho = sqrt(a * a + b * b);
    K.cs[j] = a / rho;
    K.sn[j] = b / rho;
    K.H[j * m + j] = rho;
    K.H[(j + 1) * m + j] = 0.0;
    K.g[j + 1] = -K.sn[j] * K.g[j];
    K.g[j] = K.cs[j] * K.g[j];
    double est = fabs(K.g[j + 1]);
    *K.hn = hn;
    K.stat[0] = est;
    K.stat[1] = est <= *K.tol ? 1.0 : 0.0;
    K.stat[2] = hn <= 1e-14 * w0 ? 1.0 : 0.0;
    K.stat[3] = hn;
    K.stat[4] = re;
}

__global__ void k_binit_g(BKry *kr, int nsys, int m) {
    int s = blockIdx.x;
    if (s >= nsys) return;
    BKry K = kr[s];
    if (!*K.active) return;
    for (int i = threadIdx.x; i <= m; i += blockDim.x) K.g[i] = i == 0 ? *K.beta : 0.0;
}

__global__ void k_bsolve_upper(BKry *kr, int nsys, int m) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    BKry K = kr[s];
    int k = *K.kk;
    for (int i = k - 1; i >= 0; i--) {
        double t = K.g[i];
        for (int c = i + 1; c < k; c++) t -= K.H[i * m + c] * K.y[c];
        K.y[i] = t / K.H[i * m + i];
    }
}

}  // namespace mgr

struct mgr_batch_ctx {
    int nsys = 0;
    std::vector<mgr_handle> hs;
    cudaStream_t s = nullptr;
    bool own_stream = false;
    Arena ar;
    int prec = 0, nlev = 0, kmax = 0, b = 1, m = 30;
    int *active = nullptr, *kk = nullptr;
    double *tol = nullptr, *stat = nullptr, *hstat = nullptr;
    BKry *kry = nullptr;
    // tables
    std::vector<BTable> mgr_first, mgr_restrict, mgr_interp, mgr_scatter;
    std::vector<BTable> amg_resid, amg_restrict, amg_prolong, amg_post;
    // per MGR level: the AMG F-relaxation (gather of v_F with the seed of the
    // F hierarchy's pre-smoothing, that hierarchy's cycle, the weight) and the
    // restriction of Eq. 5 (r_F = v_F - A_FF z_F, v_C += Z r_F, the seed of the
    // final AMG's pre-smoothing)
    struct BAmg {
        std::vector<BTable> resid, restr, prolong, post;
        BTable coarse;
        int kmax = 0;
    };
    std::vector<BAmg> famg;
    std::vector<BTable> fgather, fomega, frres, zres;
    BTable cprep;
    BTable coarse, outer, dots1, dots2, upd1, upd2, vnorm, rnorm, v0scale;
    BTable resid_user, xupd;
    std::vector<cudaGraphExec_t> graphs;
    std::vector<long long> graph_kernels;
    std::string err;
};

static mgr_status bfail(mgr_batch bh, mgr_status st, const std::string &msg) {
    if (bh) bh->err = msg;
    g_last_error = msg;
    return st;
}

// work items of one job: chunks of R rows, elements, or reduction blocks
static long long job_items(const BTable &t, const BJob &j, int R) {
    if (t.kind == 0) return (j.n + R - 1) / R;
    if (t.kind == 2) return j.nblk;
    if (t.kind == 3) return j.n > 0 ? j.nsl : 0;
    return j.n;
}

// the SELL copy of M (values of precision T) into job J; false when M has none
template <class T>
static bool job_sell(BJob &J, const DCSR &M) {
    const void *sv = sizeof(T) == 8 ? (const void *)M.sv : (const void *)M.sv32;
    if (M.n > 0 && (!M.sptr || !sv)) return false;
    J.sptr = M.sptr; J.slen = M.slen; J.perm = M.perm; J.sci = M.sci; J.sv = sv;
    J.nsl = M.nsl; J.sg = M.sg;
    return true;
}

static int upload_table(mgr_batch bh, BTable &t) {
    t.njobs = (int)t.host.size();
    if (!t.jobs) t.jobs = bh->ar.alloc<BJob>(t.njobs + 1);
    if (!t.prefix) t.prefix = bh->ar.alloc<long long>(t.njobs + 2);
    if (!t.jobs || !t.prefix) return ST_NOMEM;
    std::vector<long long> pre(t.njobs + 1, 0);
    for (int i = 0; i < t.njobs; i++) pre[i + 1] = pre[i] + job_items(t, t.host[i], t.R);
    t.total = pre[t.njobs];
    if (t.njobs) cudaMemcpyAsync(t.jobs, t.host.data(), sizeof(BJob) * t.njobs, cudaMemcpyHostToDevice, bh->s);
    cudaMemcpyAsync(t.prefix, pre.data(), sizeof(long long) * (t.njobs + 1), cudaMemcpyHostToDevice, bh->s);
    cudaStreamSynchronize(bh->s);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

template <class T>
static const void *vals_of(const DCSR &M) {
    return sizeof(T) == 8 ? (const void *)M.v : (const void *)M.v32;
}
template <class T>
static void *sel(double *d, float *f) { return sizeof(T) == 8 ? (void *)d : (void *)f; }

// The AMG input/output buffers of system s at AMG level k (T precision)
template <class T>
static void amg_io(mgr_handle h, int k, void **r, void **x) {
    if (k == 0) {
        MgrLevel &L = h->lev[h->nlev - 1];
        *r = sel<T>(L.vC, L.vC32);
        *x = sel<T>(L.eC, L.eC32);
    } else {
        AmgLevel &A = h->H.amg[k];
        *r = sel<T>(A.r, A.r32);
        *x = sel<T>(A.x, A.x32);
    }
}

// AMG tables of one hierarchy per member (hier(s)), level 0's input and
// output given by io0(s) and the coarser levels' by the hierarchy's own
// buffers: residual, restriction (with the next level's pre-smoothing seed),
// prolongation, post-smoothing per level, and each member's coarsest solve.
template <class T, class H, class IO>
static void build_amg_tables(mgr_batch bh, mgr_batch_ctx::BAmg &B, H hier, IO io0) {
    B.kmax = 0;
    for (int s = 0; s < bh->nsys; s++) B.kmax = std::max(B.kmax, hier(s).namg - 1);
    B.resid.assign(B.kmax, BTable()); B.restr.assign(B.kmax, BTable());
    B.prolong.assign(B.kmax, BTable()); B.post.assign(B.kmax, BTable());
    B.coarse = BTable();
    std::vector<char> ok[4];
    for (auto &v : ok) v.assign(B.kmax, 1);
    for (int s = 0; s < bh->nsys; s++) {
        AmgH &G = hier(s);
        int *act = bh->active + s;
        auto io = [&](int k, void **r, void **x) {
            if (k == 0) { io0(s, r, x); return; }
            *r = sel<T>(G.amg[k].r, G.amg[k].r32);
            *x = sel<T>(G.amg[k].x, G.amg[k].x32);
        };
        const int cl = G.namg - 1;
        for (int k = 0; k < cl; k++) {
            AmgLevel &A = G.amg[k];
            AmgLevel &C = G.amg[k + 1];
            void *rk, *xk, *rc, *xc;
            io(k, &rk, &xk);
            io(k + 1, &rc, &xc);
            BJob e; e.n = A.A.n; e.rp = A.A.rp; e.ci = A.A.ci; e.v = vals_of<T>(A.A);
            ok[0][k] &= (char)job_sell<T>(e, A.A);
            e.x = sel<T>(A.xw, A.xw32); e.r = rk; e.o1 = sel<T>(A.res, A.res32); e.active = act;
            B.resid[k].host.push_back(e);
            BJob q; q.n = A.R.n; q.rp = A.R.rp; q.ci = A.R.ci; q.v = vals_of<T>(A.R);
            ok[1][k] &= (char)job_sell<T>(q, A.R);
            q.x = sel<T>(A.res, A.res32); q.o1 = rc; q.active = act;
            if (k + 1 < cl) { q.d = sel<T>(C.dinv, C.dinv32); q.o2 = sel<T>(C.xw, C.xw32); }
            B.restr[k].host.push_back(q);
            BJob pr; pr.n = A.P.n; pr.rp = A.P.rp; pr.ci = A.P.ci; pr.v = vals_of<T>(A.P);
            ok[2][k] &= (char)job_sell<T>(pr, A.P);
            pr.x = xc; pr.o1 = sel<T>(A.xw, A.xw32); pr.active = act;
            B.prolong[k].host.push_back(pr);
            BJob po; po.n = A.A.n; po.rp = A.A.rp; po.ci = A.A.ci; po.v = vals_of<T>(A.A);
            ok[3][k] &= (char)job_sell<T>(po, A.A);
            po.x = sel<T>(A.xw, A.xw32); po.r = rk; po.d = sel<T>(A.dinv, A.dinv32); po.o1 = xk;
            po.active = act;
            B.post[k].host.push_back(po);
        }
        void *rc, *xc;
        io(cl, &rc, &xc);
        BJob c; c.n = G.nco; c.v = G.coinv; c.r = rc; c.o1 = xc; c.active = act;
        B.coarse.host.push_back(c);
    }
    for (int k = 0; k < B.kmax; k++) {
        B.resid[k].sell_ok = ok[0][k]; B.restr[k].sell_ok = ok[1][k];
        B.prolong[k].sell_ok = ok[2][k]; B.post[k].sell_ok = ok[3][k];
    }
    B.coarse.kind = 1;
}

template <class T>
static int build_tables(mgr_batch bh) {
    const int L = bh->nlev;
    bh->mgr_first.assign(L, BTable()); bh->mgr_restrict.assign(L, BTable());
    bh->mgr_interp.assign(L, BTable()); bh->mgr_scatter.assign(L, BTable());
    bh->amg_resid.assign(bh->kmax, BTable()); bh->amg_restrict.assign(bh->kmax, BTable());
    bh->amg_prolong.assign(bh->kmax, BTable()); bh->amg_post.assign(bh->kmax, BTable());
    bh->famg.assign(L, mgr_batch_ctx::BAmg());
    bh->fgather.assign(L, BTable()); bh->fomega.assign(L, BTable());
    bh->frres.assign(L, BTable()); bh->zres.assign(L, BTable());
    bh->cprep = BTable();
    std::vector<char> sell_fr(L, 1), sell_z(L, 1);
    std::vector<char> sell_all[2] = {std::vector<char>(L, 1), std::vector<char>(L, 1)};
    std::vector<char> sell_amg[4];
    for (auto &v : sell_amg) v.assign(bh->kmax, 1);
    bool sell_outer = bh->b == 1;
    for (int s = 0; s < bh->nsys; s++) {
        mgr_handle h = bh->hs[s];
        Krylov &K = h->kr;
        const int n = h->n;
        int *act = bh->active + s;
        for (int l = 0; l < L; l++) {
            MgrLevel &M = h->lev[l];
            const void *vin = l == 0 ? (const void *)K.V : sel<T>(h->lev[l - 1].vC, h->lev[l - 1].vC32);
            void *zout = l == 0 ? (void *)K.Z : sel<T>(h->lev[l - 1].eC, h->lev[l - 1].eC32);
            long long st = l == 0 ? n : 0;
            if (M.famg) {
                // v_F, and the seed D_0 v_F of the F hierarchy's pre-smoothing
                AmgH &G = *M.famg;
                BJob g; g.n = M.nF; g.r = vin; g.sr = st; g.idx = M.fidx; g.o1 = sel<T>(M.rF, M.rF32);
                if (G.namg > 1) { g.d = sel<T>(G.amg[0].dinv, G.amg[0].dinv32); g.o2 = sel<T>(G.amg[0].xw, G.amg[0].xw32); }
                g.active = act;
                bh->fgather[l].host.push_back(g);
                BJob w0; w0.n = M.nF; w0.x = sel<T>(M.tF, M.tF32); w0.o1 = sel<T>(M.zF, M.zF32); w0.active = act;
                bh->fomega[l].host.push_back(w0);
            } else {
                BJob f; f.n = M.nF; f.r = vin; f.sr = st; f.d = sel<T>(M.dinv, M.dinv32); f.gs = M.gstart;
                f.gz = M.gsize; f.idx = M.fidx; f.o1 = sel<T>(M.zF, M.zF32); f.active = act;
                bh->mgr_first[l].host.push_back(f);
            }
            if (M.rtype == MGR_RESTRICT_JACOBI) {
                // r_F = v_F - A_FF z_F, then v_C += Z r_F (Eq. 5)
                BJob fr; fr.n = M.nF; fr.rp = M.AFF.rp; fr.ci = M.AFF.ci; fr.v = vals_of<T>(M.AFF);
                sell_fr[l] &= (char)job_sell<T>(fr, M.AFF);
                fr.x = sel<T>(M.zF, M.zF32); fr.idx = M.fidx; fr.r = vin; fr.sr = st;
                fr.o1 = sel<T>(M.rF, M.rF32); fr.active = act;
                bh->frres[l].host.push_back(fr);
                BJob z; z.n = M.nC; z.rp = M.Z.rp; z.ci = M.Z.ci; z.v = vals_of<T>(M.Z);
                sell_z[l] &= (char)job_sell<T>(z, M.Z);
                z.x = sel<T>(M.rF, M.rF32); z.o1 = sel<T>(M.vC, M.vC32); z.active = act;
                bh->zres[l].host.push_back(z);
                if (l + 1 == L && h->H.namg > 1) {
                    BJob c; c.n = M.nC; c.r = sel<T>(M.vC, M.vC32); c.d = sel<T>(h->H.amg[0].dinv, h->H.amg[0].dinv32);
                    c.o2 = sel<T>(h->H.amg[0].xw, h->H.amg[0].xw32); c.active = act;
                    bh->cprep.host.push_back(c);
                }
            }
            BJob r; r.n = M.nC; r.rp = M.ACF.rp; r.ci = M.ACF.ci; r.v = vals_of<T>(M.ACF);
            sell_all[0][l] &= (char)job_sell<T>(r, M.ACF);
            r.x = sel<T>(M.zF, M.zF32); r.idx = M.cidx; r.r = vin; r.sr = st;
            r.o1 = sel<T>(M.vC, M.vC32); r.active = act;
            if (l + 1 == L && h->H.namg > 1 && M.rtype == MGR_RESTRICT_INJECTION) {
                r.d = sel<T>(h->H.amg[0].dinv, h->H.amg[0].dinv32);
                r.o2 = sel<T>(h->H.amg[0].xw, h->H.amg[0].xw32);
            }
            bh->mgr_restrict[l].host.push_back(r);
            BJob w; w.n = M.nF; w.rp = M.W.rp; w.ci = M.W.ci; w.v = vals_of<T>(M.W);
            sell_all[1][l] &= (char)job_sell<T>(w, M.W);
            w.x = sel<T>(M.eC, M.eC32); w.idx = M.fidx; w.zF = sel<T>(M.zF, M.zF32);
            w.o1 = zout; w.so1 = st; w.active = act;
            bh->mgr_interp[l].host.push_back(w);
            BJob c; c.n = M.nC; c.idx = M.cidx; c.x = sel<T>(M.eC, M.eC32); c.o1 = zout; c.so1 = st;
            c.active = act;
            bh->mgr_scatter[l].host.push_back(c);
        }
        const int cl = h->H.namg - 1;  // this system's coarsest AMG level
        for (int k = 0; k < cl; k++) {
            AmgLevel &A = h->H.amg[k];
            AmgLevel &C = h->H.amg[k + 1];
            void *rk, *xk;
            amg_io<T>(h, k, &rk, &xk);
            void *rc, *xc;
            amg_io<T>(h, k + 1, &rc, &xc);
            BJob e; e.n = A.A.n; e.rp = A.A.rp; e.ci = A.A.ci; e.v = vals_of<T>(A.A);
            sell_amg[0][k] &= (char)job_sell<T>(e, A.A);
            e.x = sel<T>(A.xw, A.xw32); e.r = rk; e.o1 = sel<T>(A.res, A.res32); e.active = act;
            bh->amg_resid[k].host.push_back(e);
            BJob q; q.n = A.R.n; q.rp = A.R.rp; q.ci = A.R.ci; q.v = vals_of<T>(A.R);
            sell_amg[1][k] &= (char)job_sell<T>(q, A.R);
            q.x = sel<T>(A.res, A.res32); q.o1 = rc; q.active = act;
            if (k + 1 < cl) { q.d = sel<T>(C.dinv, C.dinv32); q.o2 = sel<T>(C.xw, C.xw32); }
            bh->amg_restrict[k].host.push_back(q);
            BJob pr; pr.n = A.P.n; pr.rp = A.P.rp; pr.ci = A.P.ci; pr.v = vals_of<T>(A.P);
            sell_amg[2][k] &= (char)job_sell<T>(pr, A.P);
            pr.x = xc; pr.o1 = sel<T>(A.xw, A.xw32); pr.active = act;
            bh->amg_prolong[k].host.push_back(pr);
            BJob po; po.n = A.A.n; po.rp = A.A.rp; po.ci = A.A.ci; po.v = vals_of<T>(A.A);
            sell_amg[3][k] &= (char)job_sell<T>(po, A.A);
            po.x = sel<T>(A.xw, A.xw32); po.r = rk; po.d = sel<T>(A.dinv, A.dinv32); po.o1 = xk;
            po.active = act;
            bh->amg_post[k].host.push_back(po);
        }
        {
            void *rc, *xc;
            amg_io<T>(h, cl, &rc, &xc);
            BJob c; c.n = h->H.nco; c.v = h->H.coinv; c.r = rc; c.o1 = xc; c.active = act;
            bh->coarse.host.push_back(c);
        }
        // outer product w = A z_j -> V_{j+1}
        BJob o; o.n = bh->b == 1 ? n : n; o.rp = h->brp; o.ci = h->bci; o.v = h->bval;
        if (bh->b == 1) sell_outer = job_sell<double>(o, h->Aout) && sell_outer;
        o.x = K.Z; o.sx = n; o.o1 = K.V + n; o.so1 = n; o.active = act;
        bh->outer.host.push_back(o);
        // Arnoldi: w = V_{j+1} = V + n + j n
        BJob d1; d1.n = n; d1.v = K.V; d1.x = K.V + n; d1.sx = n; d1.partial = K.partial;
        d1.ticket = K.ticket; d1.flag = K.flag; d1.nblk = K.nblk; d1.o1 = K.h1; d1.active = act;
        bh->dots1.host.push_back(d1);
        BJob d2 = d1; d2.o1 = K.h2;
        bh->dots2.host.push_back(d2);
        BJob u1 = d1; u1.r = K.h1; u1.o2 = K.nrm2;
        bh->upd1.host.push_back(u1);
        BJob u2 = d1; u2.r = K.h2; u2.o2 = K.nrmB;
        bh->upd2.host.push_back(u2);
        BJob vn; vn.n = n; vn.x = K.V + n; vn.sx = n; vn.o1 = K.V + n; vn.so1 = n; vn.d = K.hn;
        vn.active = act;
        bh->vnorm.host.push_back(vn);
        BJob rn; rn.n = n; rn.v = K.r; rn.x = K.r; rn.partial = K.partial; rn.ticket = K.ticket;
        rn.flag = K.flag; rn.nblk = K.nblk; rn.o1 = K.beta; rn.active = act;
        bh->rnorm.host.push_back(rn);
        BJob v0; v0.n = n; v0.x = K.r; v0.o1 = K.V; v0.d = K.beta; v0.active = act;
        bh->v0scale.host.push_back(v0);
    }
    for (int l = 0; l < L; l++) {
        bh->mgr_restrict[l].sell_ok = sell_all[0][l];
        bh->mgr_interp[l].sell_ok = sell_all[1][l];
        bh->frres[l].sell_ok = sell_fr[l];
        bh->zres[l].sell_ok = sell_z[l];
        bh->fgather[l].kind = bh->fomega[l].kind = 1;
        bh->frres[l].kind = bh->zres[l].kind = 0;
        if (bh->hs[0]->lev[l].famg) {
            const bool w1 = bh->hs[0]->lev[l].omega == 1.0;
            build_amg_tables<T>(bh, bh->famg[l], [&](int s) -> AmgH & { return *bh->hs[s]->lev[l].famg; },
                                [&](int s, void **r, void **x) {
                                    MgrLevel &M = bh->hs[s]->lev[l];
                                    *r = sel<T>(M.rF, M.rF32);
                                    *x = w1 ? sel<T>(M.zF, M.zF32) : sel<T>(M.tF, M.tF32);
                                });
        }
    }
    bh->cprep.kind = 1;
    for (int k = 0; k < bh->kmax; k++) {
        bh->amg_resid[k].sell_ok = sell_amg[0][k];
        bh->amg_restrict[k].sell_ok = sell_amg[1][k];
        bh->amg_prolong[k].sell_ok = sell_amg[2][k];
        bh->amg_post[k].sell_ok = sell_amg[3][k];
    }
    bh->outer.sell_ok = sell_outer;
    auto setR = [](std::vector<BTable> &v, int kind) { for (auto &t : v) t.kind = kind; };
    setR(bh->mgr_first, 1); setR(bh->mgr_scatter, 1);
    setR(bh->mgr_restrict, 0); setR(bh->mgr_interp, 0);
    setR(bh->amg_resid, 0); setR(bh->amg_restrict, 0); setR(bh->amg_prolong, 0); setR(bh->amg_post, 0);
    bh->coarse.kind = 1;
    bh->outer.kind = bh->b == 1 ? 0 : 1;
    bh->dots1.kind = bh->dots2.kind = bh->upd1.kind = bh->upd2.kind = bh->rnorm.kind = 2;
    bh->vnorm.kind = bh->v0scale.kind = 1;
    if (bh->b > 1)  // one item per scalar row of the block product
        for (auto &j : bh->outer.host) j.n = j.n;
    auto initR = [](BTable &t) {
        if (t.kind != 0) { t.R = 1; return; }
        long long nnz = 0, n = 0;
        for (auto &j : t.host) { n += j.n; }
        (void)nnz;
        t.R = 1;
    };
    (void)initR;
    return ST_OK;
}

// rows-per-warp from the table's aggregate density (the autotuner refines it)
static int table_R0(mgr_batch bh, BTable &t) {
    long long n = 0, nnz = 0;
    std::vector<int> hrp;
    for (auto &j : t.host) {
        if (j.n <= 0) continue;
        int last = 0, first = 0;
        cudaMemcpyAsync(&first, j.rp, sizeof(int), cudaMemcpyDeviceToHost, bh->s);
        cudaMemcpyAsync(&last, j.rp + j.n, sizeof(int), cudaMemcpyDeviceToHost, bh->s);
        cudaStreamSynchronize(bh->s);
        n += j.n;
        nnz += last - first;
    }
    double avg = n > 0 ? (double)nnz / n : 1.0;
    if (avg < 1.0) avg = 1.0;
    int r = 1;
    while (r < 32 && (r * 2) * avg <= 192.0) r *= 2;
    return r;
}

template <class T>
static void run_chunk(mgr_batch bh, BTable &t, int op, int js, bool top) {
    if (!t.total) return;
    KScope ks(bh->hs[0], t.kind == 3 ? "batched_sell" : "batched_chunk", op, 0.0);
    if (t.kind == 3) {
        if (top) launch_bsell<T, double>(op, t.jobs, t.prefix, t.njobs, t.total, js, bh->s);
        else launch_bsell<T, T>(op, t.jobs, t.prefix, t.njobs, t.total, js, bh->s);
        return;
    }
    if (top) launch_bchunk<T, double>(op, t.jobs, t.prefix, t.njobs, t.total, t.R, js, bh->s);
    else launch_bchunk<T, T>(op, t.jobs, t.prefix, t.njobs, t.total, t.R, js, bh->s);
}

// Autotuner: for every row-product table try the members' SELL copies (one
// item per slice) and the chunk engine with R0/2, R0, 2 R0 rows per warp
// (within 1..32); time three launches of each (the first discarded) and keep
// the fastest.  The buffers hold no solve state yet, so the trial launches
// are harmless.
template <class T>
static int autotune(mgr_batch bh, BTable &t, int op, bool top) {
    if (t.kind != 0 || t.host.empty()) return upload_table(bh, t);
    int R0 = table_R0(bh, t);
    // candidates: (kind, R)
    int cands[4][2] = {{3, 1}, {0, R0 / 2}, {0, R0}, {0, R0 * 2}};
    float best = 1e30f;
    int bestK = 0, bestR = R0;
    cudaEvent_t a, b;
    cudaEventCreate(&a); cudaEventCreate(&b);
    for (int c = 0; c < 4; c++) {
        const int kind = cands[c][0], R = cands[c][1];
        if (kind == 3 && !t.sell_ok) continue;
        if (kind == 0 && (R < 1 || R > 32)) continue;
        t.kind = kind;
        t.R = R;
        if (upload_table(bh, t)) { cudaEventDestroy(a); cudaEventDestroy(b); return ST_NOMEM; }
        float ms = 0.f;
        for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(a, bh->s);
            run_chunk<T>(bh, t, op, 0, top);
            cudaEventRecord(b, bh->s);
            cudaEventSynchronize(b);
            float e = 0.f;
            cudaEventElapsedTime(&e, a, b);
            if (rep > 0) ms += e;
        }
        if (ms < best) { best = ms; bestK = kind; bestR = R; }
    }
    cudaEventDestroy(a); cudaEventDestroy(b);
    t.kind = bestK;
    t.R = bestR;
    return upload_table(bh, t);
}

template <class T>
static int finish_tables(mgr_batch bh) {
    int rc = 0;
    for (int l = 0; l < bh->nlev && !rc; l++) {
        rc |= upload_table(bh, bh->mgr_first[l]);
        rc |= upload_table(bh, bh->mgr_scatter[l]);
        rc |= upload_table(bh, bh->fgather[l]);
        rc |= upload_table(bh, bh->fomega[l]);
        if (!bh->frres[l].host.empty()) rc |= autotune<T>(bh, bh->frres[l], BOP_FRELAX_RESID, l == 0);
        if (!bh->zres[l].host.empty()) rc |= autotune<T>(bh, bh->zres[l], BOP_PROLONG, false);
        mgr_batch_ctx::BAmg &F = bh->famg[l];
        for (int k = 0; k < F.kmax && !rc; k++) {
            rc |= autotune<T>(bh, F.resid[k], BOP_RESID, false);
            rc |= autotune<T>(bh, F.restr[k], BOP_RESTRICT, false);
            rc |= autotune<T>(bh, F.prolong[k], BOP_PROLONG, false);
            rc |= autotune<T>(bh, F.post[k], BOP_POST, false);
        }
        if (!F.coarse.host.empty()) rc |= upload_table(bh, F.coarse);
        rc |= autotune<T>(bh, bh->mgr_restrict[l], BOP_MGR_RESTRICT, l == 0);
        rc |= autotune<T>(bh, bh->mgr_interp[l], BOP_MGR_INTERP, l == 0);
    }
    for (int k = 0; k < bh->kmax && !rc; k++) {
        rc |= autotune<T>(bh, bh->amg_resid[k], BOP_RESID, false);
        rc |= autotune<T>(bh, bh->amg_restrict[k], BOP_RESTRICT, false);
        rc |= autotune<T>(bh, bh->amg_prolong[k], BOP_PROLONG, false);
        rc |= autotune<T>(bh, bh->amg_post[k], BOP_POST, false);
    }
    rc |= upload_table(bh, bh->coarse);
    rc |= upload_table(bh, bh->cprep);
    if (bh->b == 1) rc |= autotune<double>(bh, bh->outer, BOP_OUTER_CSR, true);
    else rc |= upload_table(bh, bh->outer);
    rc |= upload_table(bh, bh->dots1); rc |= upload_table(bh, bh->dots2);
    rc |= upload_table(bh, bh->upd1); rc |= upload_table(bh, bh->upd2);
    rc |= upload_table(bh, bh->vnorm); rc |= upload_table(bh, bh->rnorm);
    rc |= upload_table(bh, bh->v0scale);
    return rc;
}

// One batched MGR V-cycle on V_j -> Z_j of every active system.
// One level-synchronous AMG V(1,1) over every member's hierarchy of a table set.
template <class T>
static void bamg_cycle(mgr_batch bh, mgr_batch_ctx::BAmg &B, int j) {
    for (int k = 0; k < B.kmax; k++) {
        run_chunk<T>(bh, B.resid[k], BOP_RESID, j, false);
        run_chunk<T>(bh, B.restr[k], BOP_RESTRICT, j, false);
    }
    { KScope ks(bh->hs[0], "batched_coarsest", -1, 0.0);
      launch_bdense<T>(B.coarse.jobs, B.coarse.prefix, B.coarse.njobs, B.coarse.total, j, bh->s); }
    for (int k = B.kmax - 1; k >= 0; k--) {
        run_chunk<T>(bh, B.prolong[k], BOP_PROLONG, j, false);
        run_chunk<T>(bh, B.post[k], BOP_POST, j, false);
    }
}

template <class T>
static void bvcycle(mgr_batch bh, int j) {
    cudaStream_t s = bh->s;
    const int L = bh->nlev;
    for (int l = 0; l < L; l++) {
        const MgrLevel &M0 = bh->hs[0]->lev[l];  // options are the same for every member
        if (M0.famg) {
            // AMG F-relaxation (MGR_U, Sec. 4.3): z_F = omega * B v_F
            BTable &g = bh->fgather[l];
            { KScope ks(bh->hs[0], "batched_frelax_gather", l, 0.0);
              if (l == 0) launch_bgather<T, double>(g.jobs, g.prefix, g.njobs, g.total, j, s);
              else launch_bgather<T, T>(g.jobs, g.prefix, g.njobs, g.total, j, s); }
            bamg_cycle<T>(bh, bh->famg[l], j);
            if (M0.omega != 1.0) {
                BTable &w = bh->fomega[l];
                KScope ks(bh->hs[0], "batched_frelax_scale", l, 0.0);
                launch_bomega<T>(w.jobs, w.prefix, w.njobs, w.total, (T)M0.omega, s);
            }
        } else {
            BTable &f = bh->mgr_first[l];
            KScope ks(bh->hs[0], "batched_frelax_first", l, 0.0);
            if (l == 0) launch_bfrelax_first<T, double>(f.jobs, f.prefix, f.njobs, f.total, (T)M0.omega, j, s);
            else launch_bfrelax_first<T, T>(f.jobs, f.prefix, f.njobs, f.total, (T)M0.omega, j, s);
        }
        if (M0.rtype == MGR_RESTRICT_JACOBI) run_chunk<T>(bh, bh->frres[l], BOP_FRELAX_RESID, j, l == 0);
        run_chunk<T>(bh, bh->mgr_restrict[l], BOP_MGR_RESTRICT, j, l == 0);
        if (M0.rtype == MGR_RESTRICT_JACOBI) {
            run_chunk<T>(bh, bh->zres[l], BOP_PROLONG, j, false);  // v_C += Z r_F
            if (l + 1 == L) {
                BTable &c = bh->cprep;
                KScope ks(bh->hs[0], "batched_amg_scale", -1, 0.0);
                launch_bgather<T, T>(c.jobs, c.prefix, c.njobs, c.total, j, s);
            }
        }
    }
    for (int k = 0; k < bh->kmax; k++) {
        run_chunk<T>(bh, bh->amg_resid[k], BOP_RESID, j, false);
        run_chunk<T>(bh, bh->amg_restrict[k], BOP_RESTRICT, j, false);
    }
    { KScope ks(bh->hs[0], "batched_coarsest", -1, 0.0);
      launch_bdense<T>(bh->coarse.jobs, bh->coarse.prefix, bh->coarse.njobs, bh->coarse.total, j, s); }
    for (int k = bh->kmax - 1; k >= 0; k--) {
        run_chunk<T>(bh, bh->amg_prolong[k], BOP_PROLONG, j, false);
        run_chunk<T>(bh, bh->amg_post[k], BOP_POST, j, false);
    }
    for (int l = L - 1; l >= 0; l--) {
        run_chunk<T>(bh, bh->mgr_interp[l], BOP_MGR_INTERP, j, l == 0);
        BTable &c = bh->mgr_scatter[l];
        KScope ks(bh->hs[0], "batched_scatter", l, 0.0);
        if (l == 0) launch_bscatter<T, double>(c.jobs, c.prefix, c.njobs, c.total, j, s);
        else launch_bscatter<T, T>(c.jobs, c.prefix, c.njobs, c.total, j, s);
    }
}

static void bstep(mgr_batch bh, int j) {
    cudaStream_t s = bh->s;
    if (bh->prec == MGR_PREC_FP32) bvcycle<float>(bh, j);
    else bvcycle<double>(bh, j);
    {
        KScope ks(bh->hs[0], "batched_spmv_A", -1, 0.0);
        if (bh->b == 1 && bh->outer.kind == 3)
            launch_bsell<double, double>(BOP_OUTER_CSR, bh->outer.jobs, bh->outer.prefix, bh->outer.njobs, bh->outer.total, j, s);
        else if (bh->b == 1) launch_bchunk<double, double>(BOP_OUTER_CSR, bh->outer.jobs, bh->outer.prefix, bh->outer.njobs, bh->outer.total, bh->outer.R, j, s);
        else launch_bbsr(bh->b, bh->outer.jobs, bh->outer.prefix, bh->outer.njobs, bh->outer.total, j, s);
    }
    const int k = j + 1;
    { KScope ks(bh->hs[0], "batched_arnoldi", -1, 0.0);
      launch_bdots(k + 1, bh->dots1.jobs, bh->dots1.prefix, bh->dots1.njobs, bh->dots1.total, j, 0, 0, s); }
    { KScope ks(bh->hs[0], "batched_arnoldi", -1, 0.0);
      launch_bupdate_norm(k, bh->upd1.jobs, bh->upd1.prefix, bh->upd1.njobs, bh->upd1.total, j, 1, s); }
    { KScope ks(bh->hs[0], "batched_arnoldi", -1, 0.0);
      launch_bdots(k, bh->dots2.jobs, bh->dots2.prefix, bh->dots2.njobs, bh->dots2.total, j, 1, 0, s); }
    { KScope ks(bh->hs[0], "batched_arnoldi", -1, 0.0);
      launch_bupdate_norm(k, bh->upd2.jobs, bh->upd2.prefix, bh->upd2.njobs, bh->upd2.total, j, 2, s); }
    { KScope ks(bh->hs[0], "batched_givens", -1, 0.0);
      k_bgivens<<<(bh->nsys + 31) / 32, 32, 0, s>>>(bh->kry, bh->nsys, j, bh->m); }
    cudaMemcpyAsync(bh->hstat, bh->stat, sizeof(double) * 8 * bh->nsys, cudaMemcpyDeviceToHost, s);
    { KScope ks(bh->hs[0], "batched_vec_scale", -1, 0.0);
      launch_bscale(bh->vnorm.jobs, bh->vnorm.prefix, bh->vnorm.njobs, bh->vnorm.total, j, 1, s); }
}

static cudaError_t brun_step(mgr_batch bh, int j, bool graphs) {
    if (!graphs) { bstep(bh, j); return cudaGetLastError(); }
    if ((int)bh->graphs.size() < bh->m) { bh->graphs.resize(bh->m, nullptr); bh->graph_kernels.resize(bh->m, 0); }
    if (!bh->graphs[j]) {
        cudaGraph_t g = nullptr;
        long long before = g_launches.load();
        cudaError_t e = cudaStreamBeginCapture(bh->s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        bstep(bh, j);
        e = cudaStreamEndCapture(bh->s, &g);
        if (e != cudaSuccess) return e;
        bh->graph_kernels[j] = g_launches.load() - before;
        g_launches.fetch_sub(bh->graph_kernels[j]);
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        bh->graphs[j] = ex;
    }
    g_launches.fetch_add(bh->graph_kernels[j]);
    return cudaGraphLaunch(bh->graphs[j], bh->s);
}

extern "C" void mgr_free_batched(mgr_batch bh) {
    if (!bh) return;
    cudaStreamSynchronize(bh->s);
    for (auto g : bh->graphs) if (g) cudaGraphExecDestroy(g);
    for (auto h : bh->hs) mgr_free(h);
    if (bh->hstat) cudaFreeHost(bh->hstat);
    bh->ar.free_all();
    if (bh->own_stream) cudaStreamDestroy(bh->s);
    delete bh;
}

extern "C" mgr_status mgr_setup_batched(int32_t nsys, const mgr_bsr *A, const mgr_labels *cf,
                                        const mgr_options *opt, void *stream, mgr_batch *out) {
    if (!out || nsys < 1 || !A || !cf) return bfail(nullptr, MGR_ERR_INVALID, "bad batched arguments");
    *out = nullptr;
    mgr_batch bh = new mgr_batch_ctx();
    bh->nsys = nsys;
    bh->s = (cudaStream_t)stream;
    if (!bh->s) {
        if (cudaStreamCreate(&bh->s) != cudaSuccess) { delete bh; return bfail(nullptr, MGR_ERR_CUDA, "stream"); }
        bh->own_stream = true;
    }
    mgr_options o;
    if (opt) o = *opt; else mgr_options_default(&o);
    bh->prec = o.precision;
    bh->nlev = cf[0].num_levels;
    bh->b = A[0].b;
    if (bh->nlev < 1) { mgr_free_batched(bh); return bfail(nullptr, MGR_ERR_UNSUPPORTED, "batched solves need at least one MGR level"); }
    for (int l = 0; l < bh->nlev; l++) {
        if (o.relax_sweeps[l] > 1) { mgr_free_batched(bh); return bfail(nullptr, MGR_ERR_UNSUPPORTED, "batched solves use one F-relaxation sweep"); }

    }
    for (int s = 0; s < nsys; s++) {
        if (A[s].b != bh->b || cf[s].num_levels != bh->nlev) {
            mgr_free_batched(bh);
            return bfail(nullptr, MGR_ERR_INVALID, "all systems of a batch need the same block size and MGR level count");
        }
        mgr_handle h = nullptr;
        g_no_tune = true;
        mgr_status st = mgr_setup(&A[s], &cf[s], &o, bh->s, &h);
        g_no_tune = false;
        if (st != MGR_OK) {
            std::string m = g_last_error;
            mgr_free_batched(bh);
            char buf[64];
            snprintf(buf, sizeof buf, "system %d: ", s);
            return bfail(nullptr, st, buf + m);
        }
        h->in_batch = true;
        bh->hs.push_back(h);
        bh->kmax = std::max(bh->kmax, h->H.namg - 1);
    }
    bh->m = bh->hs[0]->kr.m;
    Arena &ar = bh->ar;
    bh->active = ar.alloc<int>(nsys);
    bh->kk = ar.alloc<int>(nsys);
    bh->tol = ar.alloc<double>(nsys);
    bh->stat = ar.alloc<double>(8 * nsys);
    bh->kry = ar.alloc<BKry>(nsys);
    cudaMallocHost(&bh->hstat, sizeof(double) * 8 * nsys);
    if (!bh->active || !bh->kk || !bh->tol || !bh->stat || !bh->kry || !bh->hstat) {
        mgr_free_batched(bh);
        return bfail(nullptr, MGR_ERR_NOMEM, "batch workspace");
    }
    std::vector<BKry> hk(nsys);
    for (int s = 0; s < nsys; s++) {
        Krylov &K = bh->hs[s]->kr;
        hk[s] = BKry{K.h1, K.h2, K.nrm2, K.nrmB, K.H, K.cs, K.sn, K.g, K.hn, bh->stat + 8 * s,
                     K.beta, K.y, bh->tol + s, K.flag, bh->active + s, bh->kk + s};
    }
    cudaMemcpyAsync(bh->kry, hk.data(), sizeof(BKry) * nsys, cudaMemcpyHostToDevice, bh->s);
    std::vector<int> ones(nsys, 1);
    cudaMemcpyAsync(bh->active, ones.data(), sizeof(int) * nsys, cudaMemcpyHostToDevice, bh->s);
    int rc = bh->prec == MGR_PREC_FP32 ? build_tables<float>(bh) : build_tables<double>(bh);
    if (!rc) rc = bh->prec == MGR_PREC_FP32 ? finish_tables<float>(bh) : finish_tables<double>(bh);
    // the residual/update tables point at per-solve user vectors: filled per call
    bh->resid_user.kind = bh->b == 1 ? 0 : 1;
    bh->xupd.kind = 1;
    cudaStreamSynchronize(bh->s);
    if (rc || cudaGetLastError() != cudaSuccess) {
        mgr_free_batched(bh);
        return bfail(nullptr, rc == ST_NOMEM ? MGR_ERR_NOMEM : MGR_ERR_CUDA, "batched tables");
    }
    *out = bh;
    return MGR_OK;
}

extern "C" mgr_status mgr_batch_handle(mgr_batch bh, int32_t i, mgr_handle *out) {
    if (!bh || !out || i < 0 || i >= bh->nsys) return bfail(bh, MGR_ERR_INVALID, "no such system");
    *out = bh->hs[i];
    return MGR_OK;
}

extern "C" mgr_status mgr_solve_batched(mgr_batch bh, const double *const *bvec, double *const *xvec,
                                        double rtol, int32_t maxit, mgr_solve_info *info) {
    if (!bh || !bvec || !xvec) return bfail(bh, MGR_ERR_INVALID, "NULL argument");
    auto t0 = std::chrono::steady_clock::now();
    const int ns = bh->nsys, m = bh->m;
    cudaStream_t s = bh->s;
    // per-call tables over the user's vectors
    bh->resid_user.host.clear();
    bh->xupd.host.clear();
    for (int i = 0; i < ns; i++) {
        mgr_handle h = bh->hs[i];
        BJob r; r.n = h->n; r.rp = h->brp; r.ci = h->bci; r.v = h->bval; r.x = xvec[i]; r.r = bvec[i];
        r.o1 = h->kr.r; r.active = bh->active + i;
        bh->resid_user.host.push_back(r);
        BJob u; u.n = h->n; u.v = h->kr.Z; u.r = h->kr.y; u.o1 = xvec[i]; u.gz = bh->kk + i;
        bh->xupd.host.push_back(u);
    }
    // b == 1: a CSR chunk table (rows per warp from its density when the
    // outer product runs on SELL slices); b > 1: one item per scalar row
    bh->resid_user.R = bh->b == 1 && bh->outer.kind == 3 ? table_R0(bh, bh->resid_user) : bh->outer.R;
    if (upload_table(bh, bh->resid_user) || upload_table(bh, bh->xupd)) return bfail(bh, MGR_ERR_NOMEM, "tables");
    std::vector<int> act(ns, 1), done(ns, 0), iters(ns, 0), kk(ns, 0);
    std::vector<double> bn(ns, 0.0), relres(ns, 0.0);
    // |b| per system (the residual table with x = 0 is not needed: norms of b)
    {
        BTable bt; bt.kind = 2;
        for (int i = 0; i < ns; i++) {
            Krylov &K = bh->hs[i]->kr;
            BJob d; d.n = bh->hs[i]->n; d.v = bvec[i]; d.x = bvec[i]; d.partial = K.partial;
            d.ticket = K.ticket; d.flag = K.flag; d.nblk = K.nblk; d.o1 = K.beta;
            bt.host.push_back(d);
        }
        if (upload_table(bh, bt)) return bfail(bh, MGR_ERR_NOMEM, "tables");
        launch_bdots(1, bt.jobs, bt.prefix, bt.njobs, bt.total, 0, 0, 1, s);
        for (int i = 0; i < ns; i++)
            cudaMemcpyAsync(&bn[i], bh->hs[i]->kr.beta, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        bh->ar.release(bt.jobs); bh->ar.release(bt.prefix);
    }
    std::vector<double> tol(ns);
    for (int i = 0; i < ns; i++) {
        if (!std::isfinite(bn[i])) return bfail(bh, MGR_ERR_INVALID, "right-hand side is not finite");
        tol[i] = rtol * bn[i];
        if (bn[i] == 0.0) { act[i] = 0; done[i] = 1; cudaMemsetAsync(xvec[i], 0, sizeof(double) * bh->hs[i]->n, s); }
    }
    cudaMemcpyAsync(bh->tol, tol.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s);
    const bool graphs = bh->hs[0]->opt.use_graphs && !bh->hs[0]->prof.on;
    mgr_status st = MGR_OK;
    for (;;) {
        // true residuals of the systems still open
        cudaMemcpyAsync(bh->active, act.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s);
        {
            KScope ks(bh->hs[0], "batched_residual", -1, 0.0);
            BTable &t = bh->resid_user;
            if (bh->b == 1) launch_bchunk<double, double>(BOP_OUTER_CSR, t.jobs, t.prefix, t.njobs, t.total, t.R, 0, s);
            else launch_bbsr(bh->b, t.jobs, t.prefix, t.njobs, t.total, 0, s);
        }
        launch_bdots(1, bh->rnorm.jobs, bh->rnorm.prefix, bh->rnorm.njobs, bh->rnorm.total, 0, 0, 1, s);
        std::vector<double> beta(ns, 0.0);
        for (int i = 0; i < ns; i++)
            if (act[i]) cudaMemcpyAsync(&beta[i], bh->hs[i]->kr.beta, sizeof(double), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        if (cudaGetLastError() != cudaSuccess) return cuda_fail(nullptr, "batched residual");
        bool any = false;
        for (int i = 0; i < ns; i++) {
            if (!act[i]) continue;
            relres[i] = beta[i] / bn[i];
            if (!std::isfinite(beta[i])) { act[i] = 0; done[i] = 2; continue; }
            if (beta[i] <= tol[i]) { act[i] = 0; done[i] = 1; continue; }
            if (iters[i] >= maxit) { act[i] = 0; continue; }
            any = true;
        }
        if (!any) break;
        cudaMemcpyAsync(bh->active, act.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s);
        launch_bscale(bh->v0scale.jobs, bh->v0scale.prefix, bh->v0scale.njobs, bh->v0scale.total, 0, 1, s);
        k_binit_g<<<ns, 32, 0, s>>>(bh->kry, ns, m);
        std::vector<int> cyc(act);  // systems in this restart cycle
        std::fill(kk.begin(), kk.end(), 0);
        for (int j = 0; j < m; j++) {
            cudaError_t ge = brun_step(bh, j, graphs);
            cudaStreamSynchronize(s);
            if (ge != cudaSuccess || cudaGetLastError() != cudaSuccess) return cuda_fail(nullptr, "batched step");
            bool changed = false, open = false;
            for (int i = 0; i < ns; i++) {
                if (!act[i]) continue;
                iters[i]++;
                kk[i] = j + 1;
                const double *st8 = bh->hstat + 8 * i;
                if (!std::isfinite(st8[0])) { act[i] = 0; done[i] = 2; changed = true; continue; }
                if (st8[1] != 0.0 || st8[2] != 0.0 || iters[i] >= maxit) { act[i] = 0; changed = true; continue; }
                open = true;
            }
            if (changed) cudaMemcpyAsync(bh->active, act.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s);
            if (!open) break;
        }
        // x += Z y for every system of this cycle
        for (int i = 0; i < ns; i++) if (!cyc[i]) kk[i] = 0;
        cudaMemcpyAsync(bh->kk, kk.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s);
        k_bsolve_upper<<<(ns + 31) / 32, 32, 0, s>>>(bh->kry, ns, m);
        launch_bmulti_axpy(bh->xupd.jobs, bh->xupd.prefix, bh->xupd.njobs, bh->xupd.total, s);
        // every system of the cycle gets its true residual checked next
        for (int i = 0; i < ns; i++) if (cyc[i] && done[i] == 0) act[i] = 1;
    }
    cudaStreamSynchronize(s);
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    bool all = true, bad = false;
    for (int i = 0; i < ns; i++) {
        if (done[i] != 1) all = false;
        if (done[i] == 2) bad = true;
        if (info) {
            memset(&info[i], 0, sizeof(mgr_solve_info));
            info[i].iterations = iters[i];
            info[i].rel_residual = relres[i];
            info[i].setup_ms = bh->hs[i]->setup_ms;
            info[i].solve_ms = ms;
            info[i].mgr_levels = bh->hs[i]->nlev;
            info[i].amg_levels = bh->hs[i]->H.namg;
        }
    }
    if (bad) return bfail(bh, MGR_ERR_INVALID, "a residual became non-finite");
    if (!all) return bfail(bh, MGR_ERR_NOT_CONVERGED, "maximum iterations reached for some system");
    return st;
}
