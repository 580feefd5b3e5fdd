// C ABI of the MGR library (include/mgr_gb300.h): handle, setup
// orchestration, the V-cycle driver and flexible GMRES.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <string>
#include <vector>

#include "../../include/mgr_gb300.h"
#include "common.cuh"

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
    int8_t *dlevel = nullptr;
    int nlev = 0;
    MgrLevel lev[MGR_MAX_LEVELS];
    int namg = 0;
    AmgLevel amg[32];
    int nco = 0;
    double *coinv = nullptr, *coinvT = nullptr;
    int *errw = nullptr;
    Krylov kr;
    Prof prof;
    double setup_ms = 0.0;
    std::string err;
};

static thread_local std::string g_last_error;

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
    o->amg_max_coarse = 256;
    o->amg_pmax = 4;
    o->amg_num_functions = 1;
    o->precision = MGR_PREC_FP64;
    o->restart = 30;
    o->use_graphs = 1;
}

// ---------------------------------------------------------------- helpers
static int read_errw(mgr_handle h) {
    int e = 0;
    cudaMemcpyAsync(&e, h->errw, sizeof(int), cudaMemcpyDeviceToHost, h->s);
    cudaStreamSynchronize(h->s);
    cudaMemsetAsync(h->errw, 0, sizeof(int), h->s);
    return e;
}

static int to_f32(mgr_handle h, DCSR &M) {
    if (M.nnz == 0) { M.v32 = h->ar.alloc<float>(1); return M.v32 ? 0 : ST_NOMEM; }
    M.v32 = h->ar.alloc<float>(M.nnz);
    if (!M.v32) return ST_NOMEM;
    launch_cast_f32(M.v, M.v32, M.nnz, h->s);
    return 0;
}

static mgr_status setup_amg(mgr_handle h, DCSR A0) {
    Arena &ar = h->ar;
    cudaStream_t s = h->s;
    const mgr_options &o = h->opt;
    int maxl = o.amg_max_levels < 1 ? 1 : (o.amg_max_levels > 32 ? 32 : o.amg_max_levels);
    h->amg[0].A = A0;
    h->amg[0].func = ar.alloc<int>(A0.n + 1);
    if (!h->amg[0].func) return fail(h, MGR_ERR_NOMEM, "amg func");
    launch_iota_mod(h->amg[0].func, A0.n, o.amg_num_functions, s);
    int k = 0;
    for (;;) {
        AmgLevel &L = h->amg[k];
        int n = L.A.n;
        h->namg = k + 1;
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
        AmgLevel &C = h->amg[k + 1];
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
    AmgLevel &Lc = h->amg[h->namg - 1];
    h->nco = Lc.A.n;
    if (h->nco > 1024) return fail(h, MGR_ERR_UNSUPPORTED, "AMG coarsening stalled above 1024 rows");
    h->coinv = ar.alloc<double>((size_t)h->nco * h->nco + 1);
    h->coinvT = ar.alloc<double>((size_t)h->nco * h->nco + 1);
    if (!h->coinv || !h->coinvT) return fail(h, MGR_ERR_NOMEM, "coarsest inverse");
    if (h->nco > 0) {
        if (dense_inverse(Lc.A, h->coinv, h->errw, s, ar)) return fail(h, MGR_ERR_NOMEM, "coarsest");
        if (read_errw(h) & ERRW_SINGULAR) return fail(h, MGR_ERR_SINGULAR, "singular coarsest AMG grid");
        launch_transpose_dense(h->nco, h->coinv, h->coinvT, s);
    }
    // FP32 copies and work vectors
    for (int q = 0; q < h->namg; q++) {
        AmgLevel &L = h->amg[q];
        int n = L.A.n;
        if (to_f32(h, L.A) || to_f32(h, L.AT)) return fail(h, MGR_ERR_NOMEM, "fp32 copies");
        if (q < h->namg - 1 && (to_f32(h, L.P) || to_f32(h, L.R))) return fail(h, MGR_ERR_NOMEM, "fp32 copies");
        L.r = ar.alloc<double>(n + 1); L.x = ar.alloc<double>(n + 1);
        L.xw = ar.alloc<double>(n + 1); L.res = ar.alloc<double>(n + 1);
        L.r32 = ar.alloc<float>(n + 1); L.x32 = ar.alloc<float>(n + 1);
        L.xw32 = ar.alloc<float>(n + 1); L.res32 = ar.alloc<float>(n + 1);
        if (!L.r || !L.x || !L.xw || !L.res || !L.r32 || !L.x32 || !L.xw32 || !L.res32)
            return fail(h, MGR_ERR_NOMEM, "amg vectors");
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
    // level-0 scalar CSR
    DCSR A0;
    A0.n = A0.m = n;
    A0.nnz = (int)(nnzb * b * b);
    A0.rp = ar.alloc<int>(n + 1);
    A0.ci = ar.alloc<int>(A0.nnz);
    A0.v = ar.alloc<double>(A0.nnz);
    if (!A0.rp || !A0.ci || !A0.v) { mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "scalar copy"); }
    launch_bsr_to_csr(nb, b, h->brp, h->bci, h->bval, A0, s);
    if (transpose(A0, h->A0T, s, ar)) { mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "A^T"); }
    h->nlev = cf->num_levels;
    DCSR cur = A0;
    int *gdof = nullptr;
    for (int l = 0; l < h->nlev; l++) {
        MgrLevel &L = h->lev[l];
        L.A = cur; L.gdof = gdof; L.n = cur.n;
        L.relax = h->opt.relax_type[l];
        L.sweeps = h->opt.relax_sweeps[l] < 1 ? 1 : h->opt.relax_sweeps[l];
        L.omega = h->opt.relax_weight[l];
        if (L.relax < 0 || L.relax > 2) { mgr_free(h); return fail(nullptr, MGR_ERR_INVALID, "relax type"); }
        int nl = L.n;
        int *isF = ar.alloc<int>(nl + 1), *isC = ar.alloc<int>(nl + 1);
        int *fpos = ar.alloc<int>(nl + 1), *cpos = ar.alloc<int>(nl + 1);
        int *fmap = ar.alloc<int>(nl + 1), *cmap = ar.alloc<int>(nl + 1);
        L.fidx = ar.alloc<int>(nl + 1); L.cidx = ar.alloc<int>(nl + 1);
        if (!isF || !isC || !fpos || !cpos || !fmap || !cmap || !L.fidx || !L.cidx) {
            mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "level maps");
        }
        launch_level_flags(h->dlevel, gdof, nl, l, isF, isC, h->errw, s);
        int nF = 0, nC = 0;
        scan_exclusive(isF, fpos, nl, s, ar, &nF);
        scan_exclusive(isC, cpos, nl, s, ar, &nC);
        if (read_errw(h)) { mgr_free(h); return fail(nullptr, MGR_ERR_INVALID, "labels: a dof eliminated twice"); }
        if (nF == 0 || nC == 0) {
            char buf[128];
            snprintf(buf, sizeof buf, "MGR level %d has an empty %s set", l, nF == 0 ? "F" : "C");
            mgr_free(h); return fail(nullptr, MGR_ERR_INVALID, buf);
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
        if (rc || !L.gstart || !L.gsize || !L.dinv || !L.dinv32) { mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "level blocks"); }
        mgr_dinv(L.AFF, L.fidx, gdof, b, L.relax, L.gstart, L.gsize, L.dinv, h->errw, s);
        if (read_errw(h) & ERRW_SINGULAR) {
            char buf[128];
            snprintf(buf, sizeof buf, "singular D_FF (zero diagonal or singular block) at MGR level %d", l);
            mgr_free(h); return fail(nullptr, MGR_ERR_SINGULAR, buf);
        }
        launch_cast_f32(L.dinv, L.dinv32, (long long)nF * 4, s);
        if (mgr_build_w(L.AFC, L.gstart, L.gsize, L.dinv, L.W, s, ar)) { mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "W"); }
        DCSR next;
        if (spgemm(L.ACF, L.W, &ACC, next, s, ar)) { mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "coarse operator"); }
        ar.release(ACC.rp); ar.release(ACC.ci); ar.release(ACC.v);
        if (transpose(L.AFF, L.AFFT, s, ar) || transpose(L.ACF, L.ACFT, s, ar) || transpose(L.W, L.WT, s, ar)) {
            mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "level transposes");
        }
        if (to_f32(h, L.AFF) || to_f32(h, L.ACF) || to_f32(h, L.W) || to_f32(h, L.AFFT) ||
            to_f32(h, L.ACFT) || to_f32(h, L.WT)) { mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "fp32"); }
        L.fiota = ar.alloc<int>(nF + 1);
        L.zF = ar.alloc<double>(nF + 1); L.rF = ar.alloc<double>(nF + 1);
        L.vC = ar.alloc<double>(nC + 1); L.eC = ar.alloc<double>(nC + 1);
        L.zF32 = ar.alloc<float>(nF + 1); L.rF32 = ar.alloc<float>(nF + 1);
        L.vC32 = ar.alloc<float>(nC + 1); L.eC32 = ar.alloc<float>(nC + 1);
        int *g2 = ar.alloc<int>(nC + 1);
        if (!L.fiota || !L.zF || !L.rF || !L.vC || !L.eC || !L.zF32 || !L.rF32 || !L.vC32 || !L.eC32 || !g2) {
            mgr_free(h); return fail(nullptr, MGR_ERR_NOMEM, "level vectors");
        }
        launch_iota(L.fiota, nF, s);
        // original dof of each C point (the next level's rows)
        if (gdof) launch_gather_int(L.cidx, nC, gdof, g2, s);
        else cudaMemcpyAsync(g2, L.cidx, sizeof(int) * nC, cudaMemcpyDeviceToDevice, s);
        ar.release(isF); ar.release(isC); ar.release(fpos); ar.release(cpos); ar.release(fmap); ar.release(cmap);
        gdof = g2;
        cur = next;
    }
    mgr_status st = setup_amg(h, cur);
    if (st != MGR_OK) { std::string m = h->err; mgr_free(h); return fail(nullptr, st, m); }
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
    cudaStreamSynchronize(s);
    if (cudaGetLastError() != cudaSuccess) { mgr_free(h); return cuda_fail(nullptr, "setup"); }
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
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
    static const float *dinv(MgrLevel &L) { return L.dinv32; }
    static const float *dinv(AmgLevel &L) { return L.dinv32; }
    static float *r(AmgLevel &L) { return L.r32; }
    static float *x(AmgLevel &L) { return L.x32; }
    static float *xw(AmgLevel &L) { return L.xw32; }
    static float *res(AmgLevel &L) { return L.res32; }
};

// AMG V(1,1) on level k: r (TV) -> x (TV).  On entry L.xw already holds the
// pre-smoothed iterate D_k r (l1-Jacobi from zero), written by whoever
// produced r.  trans uses A_k^T and the transposed coarsest inverse (the
// exact transpose of the cycle).
template <class T, class TV>
static void amg_cycle(mgr_handle h, int k, const TV *r, TV *x, int trans) {
    cudaStream_t s = h->s;
    AmgLevel &L = h->amg[k];
    if (k == h->namg - 1) {
        KScope ks(h, "coarsest_dense_solve", k, (double)h->nco * h->nco * 8 + 2.0 * h->nco * sizeof(TV),
                  (double)h->nco * h->nco);
        launch_dense_matvec<TV>(h->nco, trans ? h->coinvT : h->coinv, r, x, s);
        return;
    }
    const DCSR &A = trans ? L.AT : L.A;
    const T *av = Sel<T>::v(A);
    const T *d = Sel<T>::dinv(L);
    T *xw = Sel<T>::xw(L), *res = Sel<T>::res(L);
    AmgLevel &C = h->amg[k + 1];
    const bool c_coarsest = (k + 1 == h->namg - 1);
    const double ts = sizeof(T), tv = sizeof(TV);
    const double f64 = sizeof(T) == 8 ? 1.0 : 0.0;  // FP64 FMAs only in the FP64 form
    double an = A.n, annz = A.nnz, nc = C.A.n;
    {
        KScope ks(h, "amg_residual", k, annz * (ts + 4) + (an + 1) * 4 + an * (2 * ts + tv), f64 * annz);
        launch_amg_residual<T, TV>(A, av, xw, r, res, s);
    }
    {
        KScope ks(h, "amg_restrict", k, (double)L.R.nnz * (ts + 4) + (nc + 1) * 4 + an * ts + nc * ts * (c_coarsest ? 1 : 3),
                  f64 * L.R.nnz);
        if (c_coarsest) launch_csr_spmv<T>(L.R, Sel<T>::v(L.R), res, Sel<T>::r(C), s);
        else launch_restrict_scaled<T>(L.R, Sel<T>::v(L.R), res, Sel<T>::r(C), Sel<T>::dinv(C), Sel<T>::xw(C), s);
    }
    amg_cycle<T, T>(h, k + 1, Sel<T>::r(C), Sel<T>::x(C), trans);
    {
        KScope ks(h, "amg_prolong", k, (double)L.P.nnz * (ts + 4) + (an + 1) * 4 + nc * ts + 2 * an * ts, f64 * L.P.nnz);
        launch_csr_spmv_add<T>(L.P, Sel<T>::v(L.P), Sel<T>::x(C), xw, s);
    }
    {
        KScope ks(h, "amg_post_smooth", k, annz * (ts + 4) + (an + 1) * 4 + an * (2 * ts + 2 * tv), f64 * (annz + an));
        launch_amg_post_smooth<T, TV>(A, av, d, r, xw, x, s);
    }
}

// x_0 = D_0 r for the AMG entry when r is not produced by a fused epilogue
template <class T, class TV>
static void amg_prepare(mgr_handle h, const TV *r) {
    if (h->namg < 2) return;
    AmgLevel &L = h->amg[0];
    KScope ks(h, "amg_scale", 0, (double)L.A.n * (2 * sizeof(T) + sizeof(TV)));
    launch_scale<T, TV>(L.A.n, Sel<T>::dinv(L), r, Sel<T>::xw(L), h->s);
}

// MGR level l forward cycle (Algorithm 1): v (TV) -> z (TV)
template <class T, class TV>
static void mgr_cycle(mgr_handle h, int l, const TV *v, TV *z) {
    cudaStream_t s = h->s;
    if (l == h->nlev) {
        if (l == 0) amg_prepare<T, TV>(h, v);
        amg_cycle<T, TV>(h, 0, v, z, 0);
        return;
    }
    MgrLevel &L = h->lev[l];
    T *zF = Sel<T>::zF(L), *rF = Sel<T>::rF(L), *vC = Sel<T>::vC(L), *eC = Sel<T>::eC(L);
    const T *dinv = Sel<T>::dinv(L);
    T om = (T)L.omega;
    const double ts = sizeof(T), tv = sizeof(TV);
    const double f64 = sizeof(T) == 8 ? 1.0 : 0.0;
    double nF = L.nF, nC = L.nC, gs = L.relax == 2 ? 4.0 : 1.0;
    {
        KScope ks(h, "mgr_frelax_first", l, nF * (gs * ts + 4 + tv + ts + (L.relax == 2 ? 8 : 0)));
        launch_frelax_first<T, TV>(L.nF, L.fidx, L.gstart, L.gsize, dinv, om, v, zF, s);
    }
    for (int sw = 1; sw < L.sweeps; sw++) {
        {
            KScope ks(h, "mgr_frelax_residual", l, (double)L.AFF.nnz * (ts + 4) + (nF + 1) * 4 + nF * (4 + tv + 2 * ts));
            launch_frelax_residual<T, TV>(L.AFF, Sel<T>::v(L.AFF), L.fidx, v, zF, rF, s);
        }
        KScope ks(h, "mgr_frelax_update", l, nF * (gs * ts + 3 * ts + 8));
        launch_frelax_update<T>(L.nF, L.gstart, L.gsize, dinv, om, rF, zF, 0, s);
    }
    {
        const bool fuse = (l + 1 == h->nlev) && h->namg > 1;
        KScope ks(h, "mgr_restrict", l, (double)L.ACF.nnz * (ts + 4) + (nC + 1) * 4 + nF * ts + nC * (4 + tv + ts + (fuse ? 2 * ts : 0)),
                  f64 * L.ACF.nnz);
        if (fuse) launch_mgr_restrict_scaled<T, TV>(L.ACF, Sel<T>::v(L.ACF), L.cidx, v, zF, vC,
                                                    Sel<T>::dinv(h->amg[0]), Sel<T>::xw(h->amg[0]), s);
        else launch_mgr_restrict<T, TV>(L.ACF, Sel<T>::v(L.ACF), L.cidx, v, zF, vC, s);
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
        amg_prepare<T, TV>(h, v);
        amg_cycle<T, TV>(h, 0, v, z, 1);
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
    // K^T y_F: sweeps of z += omega D^{-T} (y - A_FF^T z) from z = 0
    cudaMemsetAsync(zF, 0, sizeof(T) * L.nF, s);
    { KScope ks(h, "mgrT_frelax_update", l, nF * (gs * ts + 3 * ts + 8));
      launch_frelax_update<T>(L.nF, L.gstart, L.gsize, dinv, om, rF, zF, 1, s); }
    if (L.sweeps > 1) {
        // keep y_F in vC's tail is unsafe; y_F must survive: copy to eC-sized scratch is not
        // possible (sizes differ), so rebuild it from v each sweep.
        for (int sw = 1; sw < L.sweeps; sw++) {
            // rF <- y_F - A_FF^T z  with y_F = v_F - A_CF^T e_C
            { KScope ks(h, "mgrT_interp", l, (double)L.ACFT.nnz * (ts + 4) + (nF + 1) * 4 + nC * ts + nF * (4 + tv + ts));
              launch_csr_axpy_gather<T, TV>(L.ACFT, Sel<T>::v(L.ACFT), eC, L.fidx, v, (T)-1, rF, s); }
            { KScope ks(h, "mgrT_frelax_residual", l, (double)L.AFFT.nnz * (ts + 4) + (nF + 1) * 4 + nF * (4 + 3 * ts));
              launch_csr_axpy_gather<T, T>(L.AFFT, Sel<T>::v(L.AFFT), zF, L.fiota, rF, (T)-1, rF, s); }
            { KScope ks(h, "mgrT_frelax_update", l, nF * (gs * ts + 3 * ts + 8));
              launch_frelax_update<T>(L.nF, L.gstart, L.gsize, dinv, om, rF, zF, 1, s); }
        }
    }
    { KScope ks(h, "mgrT_scatter", l, (nF + nC) * (4 + ts + tv));
      launch_scatter2<T, TV>(L.nF, L.nC, L.fidx, L.cidx, zF, eC, z, s); }
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
    else launch_bsr_spmv(h->nb, h->b, h->brp, h->bci, h->bval, x, y, 1.0, 0.0, h->s, h->nnzb);
}

static void outer_residual(mgr_handle h, const double *x, const double *bvec, double *y, int trans) {
    KScope ks(h, trans ? "residual_AT" : "residual_A", -1, outer_bytes(h) + h->n * 8.0, (double)h->nnzb * h->b * h->b);
    if (trans) launch_csr_residual(h->A0T, x, bvec, y, h->s);
    else launch_bsr_residual(h->nb, h->b, h->brp, h->bci, h->bval, x, bvec, y, h->s, h->nnzb);
}

extern "C" mgr_status mgr_apply(mgr_handle h, const double *v, double *z) {
    if (!h || !v || !z) return fail(h, MGR_ERR_INVALID, "NULL argument");
    vcycle(h, v, z, 0);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_apply");
    return MGR_OK;
}

extern "C" mgr_status mgr_apply_transpose(mgr_handle h, const double *v, double *z) {
    if (!h || !v || !z) return fail(h, MGR_ERR_INVALID, "NULL argument");
    vcycle(h, v, z, 1);
    if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "mgr_apply_transpose");
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
    if (!(rtol >= 0.0)) return fail(h, MGR_ERR_INVALID, "rtol must be >= 0");
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
        cudaMemsetAsync(x, 0, sizeof(double) * n, s);
        cudaStreamSynchronize(s);
        relres = 0.0;
        st = MGR_OK;
    } else {
        double tol_abs = rtol * bn;
        cudaMemcpyAsync(K.tol, &tol_abs, sizeof(double), cudaMemcpyHostToDevice, s);
        for (;;) {
            outer_residual(h, x, b, K.r, trans);
            { KScope ks(h, "norm", -1, n * 8.0);
              launch_dot(K.r, K.r, (int)n, K.partial, K.beta, K.ticket, 1, K.nblk, s); }
            double beta = 0.0;
            cudaMemcpyAsync(&beta, K.beta, sizeof(double), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            if (cudaGetLastError() != cudaSuccess) return cuda_fail(h, "solve residual");
            relres = beta / bn;
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
                int conv = K.hstat[1] != 0.0, brk = K.hstat[2] != 0.0;
                if (!isfinite(est)) { st = MGR_ERR_INVALID; break; }
                if (K.hstat[4] != 0.0) reorth++;
                if (conv || brk) break;
            }
            if (st == MGR_ERR_INVALID) { h->err = "preconditioned residual is not finite"; break; }
            { KScope ks(h, "givens", -1, 0.0);
              launch_solve_upper(k, m, K.H, K.g, K.y, s); }
            { KScope ks(h, "update_x", -1, (k + 2.0) * n * 8, (double)k * n);
              launch_multi_axpy(K.Z, n, k, K.y, x, (int)n, s); }
        }
    }
    cudaStreamSynchronize(s);
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iterations = it;
        info->rel_residual = relres;
        info->setup_ms = h->setup_ms;
        info->solve_ms = ms;
        info->mgr_levels = h->nlev;
        info->amg_levels = h->namg;
        int q = 0;
        double tot = 0, base = 0;
        for (int l = 0; l < h->nlev && q < 40; l++, q++) { info->level_rows[q] = h->lev[l].n; info->level_nnz[q] = h->lev[l].A.nnz; }
        for (int k = 0; k < h->namg && q < 40; k++, q++) {
            info->level_rows[q] = h->amg[k].A.n; info->level_nnz[q] = h->amg[k].A.nnz;
            tot += h->amg[k].A.nnz;
            if (k == 0) base = h->amg[k].A.nnz;
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
static const DCSR *pick(mgr_handle h, int amg, int level, int which) {
    if (!amg) {
        if (level < 0 || level > h->nlev) return nullptr;
        if (level == h->nlev) return which == 0 ? &h->amg[0].A : nullptr;
        MgrLevel &L = h->lev[level];
        switch (which) {
            case 0: return &L.A;
            case 1: return &L.AFF;
            case 2: return &L.AFC;
            case 3: return &L.ACF;
            case 4: return &L.W;
        }
        return nullptr;
    }
    if (level < 0 || level >= h->namg) return nullptr;
    if (which == 0) return &h->amg[level].A;
    if (which == 1) return h->amg[level].P.rp ? &h->amg[level].P : nullptr;
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
    if (!h || !cf) return fail(h, MGR_ERR_INVALID, "NULL argument");
    if (level < 0 || level >= h->namg - 1 || !h->amg[level].cf) return fail(h, MGR_ERR_INVALID, "no C/F split on that level");
    cudaStreamSynchronize(h->s);
    cudaMemcpy(cf, h->amg[level].cf, sizeof(int) * h->amg[level].A.n, cudaMemcpyDeviceToHost);
    return MGR_OK;
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

extern "C" mgr_status mgr_get_info(mgr_handle h, int32_t *out) {
    if (!h || !out) return fail(h, MGR_ERR_INVALID, "NULL argument");
    out[0] = h->nlev; out[1] = h->namg; out[2] = h->n;
    return MGR_OK;
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
