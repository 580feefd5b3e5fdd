// Krylov kernels of FGMRES (FP64): the Arnoldi projection and update, dots,
// scalings, the solution update, the Givens bookkeeping, and small helpers.
#include <cuda_runtime.h>
#include <stdlib.h>

#include "common.cuh"
#include "reduce.cuh"
#include "spmv.cuh"

namespace mgr {

int multidot_blocks(int n) {
    long long b = ((long long)n + RED_THREADS * RED_EPT - 1) / (RED_THREADS * RED_EPT);
    if (b > NUM_SMS * 2) b = NUM_SMS * 2;
    return (int)(b < 1 ? 1 : b);
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

// y = x * s  or  y = x * (1/s)  (s a device scalar).  The factor is formed
// once per block: an FP64 division in every thread costs more FP64 issue
// than the whole pass over n.
__global__ void k_vec_scale(const double *x, double *y, const double *sc, int invert, int n) {
    __shared__ double fs;
    pdl_wait();
    pdl_launch_dependents();
    if (threadIdx.x == 0) fs = invert ? 1.0 / *sc : *sc;
    __syncthreads();
    const double f = fs;
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


}  // namespace mgr
