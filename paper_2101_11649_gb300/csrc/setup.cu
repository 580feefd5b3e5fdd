// Setup-phase kernels of the MGR hierarchy and its AMG coarse solver.
//
// Compiled with --fmad=false: every product and sum is rounded separately,
// and each loop below accumulates in the order stated in its comment, so
// that the hierarchy is reproducible bit for bit (a reading: the paper
// fixes no summation order).  Work is spread one thread per row; setup is
// not on the timed path.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace mgr {

#define GRID(n, t) (unsigned)(((long long)(n) + (t)-1) / (t) > 0 ? ((long long)(n) + (t)-1) / (t) : 1)

// ------------------------------------------------------------------ arena
void *Arena::get(size_t nbytes) {
    nbytes = (nbytes + 255) & ~(size_t)255;
    if (nbytes == 0) nbytes = 256;
    // a pooled block at most 1/8 (plus 64 KiB) larger than the request
    auto it = pool.lower_bound(nbytes);
    if (it != pool.end() && it->first <= nbytes + nbytes / 8 + (64u << 10)) {
        void *p = it->second;
        blocks.push_back({p, it->first});
        pool.erase(it);
        return p;
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess && !pool.empty()) {
        cudaGetLastError();
        trim();
        e = cudaMalloc(&p, nbytes);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        status = ST_NOMEM;
        return nullptr;
    }
    blocks.push_back({p, nbytes});
    bytes += nbytes;
    return p;
}

void Arena::release(void *p) {
    if (!p) return;
    for (size_t i = 0; i < blocks.size(); i++)
        if (blocks[i].first == p) {
            pool.insert({blocks[i].second, p});
            blocks[i] = blocks.back();
            blocks.pop_back();
            return;
        }
}

void Arena::recycle() {
    for (auto &b : blocks) pool.insert({b.second, b.first});
    blocks.clear();
}

void Arena::trim() {
    for (auto &q : pool) {
        cudaFree(q.second);
        bytes -= q.first;
    }
    pool.clear();
}

void Arena::free_all() {
    trim();
    for (auto &b : blocks) cudaFree(b.first);
    blocks.clear();
    bytes = 0;
}

// ------------------------------------------------------------------ scan
template <class T>
__global__ void k_block_sums(const int *in, int n, T *sums, int per_block) {
    __shared__ T sh[32];
    long long base = (long long)blockIdx.x * per_block;
    T s = 0;
    for (int t = threadIdx.x; t < per_block; t += blockDim.x) {
        long long i = base + t;
        if (i < n) s += (T)in[i];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffff, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        T v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : (T)0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffff, v, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = v;
    }
}

// single block: exclusive scan of sums in place, total to sums[nb]
template <class T>
__global__ void k_scan_sums(T *sums, int nb) {
    __shared__ T carry;
    __shared__ T warp_tot[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x;
        T v = i < nb ? sums[i] : (T)0;
        T x = v;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffff, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            T t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : (T)0;
            for (int o = 1; o < 32; o <<= 1) {
                T y = __shfl_up_sync(0xffffffff, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        T incl = x + (w > 0 ? warp_tot[w - 1] : (T)0) + carry;
        if (i < nb) sums[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

template <class T>
__global__ void k_scan_blocks(const int *in, int n, const T *sums, T *out, int per_block) {
    __shared__ T warp_tot[32];
    __shared__ T carry;
    long long base = (long long)blockIdx.x * per_block;
    if (threadIdx.x == 0) carry = sums[blockIdx.x];
    __syncthreads();
    for (int off = 0; off < per_block; off += blockDim.x) {
        long long i = base + off + threadIdx.x;
        T v = i < n ? (T)in[i] : (T)0;
        T x = v;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffff, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            T t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : (T)0;
            for (int o = 1; o < 32; o <<= 1) {
                T y = __shfl_up_sync(0xffffffff, t, o);
                if (lane >= o) t += y;
            }
            warp_tot[lane] = t;
        }
        __syncthreads();
        T incl = x + (w > 0 ? warp_tot[w - 1] : (T)0) + carry;
        if (i < n) out[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = incl;
        __syncthreads();
    }
}

template <class T>
__global__ void k_set_total(T *out, int n, const T *sums, int nb) { out[n] = sums[nb]; }

template <class T>
static int scan_impl(const int *in, T *out, int n, cudaStream_t s, Arena &ar, T *total) {
    const int per = 4096, thr = 512;
    int nb = (n + per - 1) / per;
    if (nb < 1) nb = 1;
    T *sums = ar.alloc<T>(nb + 1);
    if (!sums) return ST_NOMEM;
    k_block_sums<T><<<nb, thr, 0, s>>>(in, n, sums, per);
    k_scan_sums<T><<<1, 1024, 0, s>>>(sums, nb);
    k_scan_blocks<T><<<nb, thr, 0, s>>>(in, n, sums, out, per);
    k_set_total<T><<<1, 1, 0, s>>>(out, n, sums, nb);
    if (total) {
        cudaMemcpyAsync(total, out + n, sizeof(T), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
    }
    ar.release(sums);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// out has n+1 entries; out[n] = total
int scan_exclusive(const int *in, int *out, int n, cudaStream_t s, Arena &ar, int *total) {
    return scan_impl<int>(in, out, n, s, ar, total);
}
int scan_exclusive_ll(const int *in, long long *out, int n, cudaStream_t s, Arena &ar,
                      long long *total) {
    return scan_impl<long long>(in, out, n, s, ar, total);
}

// ------------------------------------------------------------- BSR -> CSR
// Scalar row I*b+r: blocks of row I in ascending J, entries (r, 0..b-1).
__global__ void k_bsr_to_csr(int nb, int b, const int *rp, const int *ci, const double *val,
                             int *crp, int *cci, double *cv) {
    long long nrows = (long long)nb * b;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nrows;
         t += (long long)gridDim.x * blockDim.x) {
        int I = (int)(t / b), r = (int)(t % b);
        int p0 = rp[I], p1 = rp[I + 1];
        long long base = (long long)p0 * b * b + (long long)r * (p1 - p0) * b;
        crp[t] = (int)base;
        for (int p = p0; p < p1; p++)
            for (int c = 0; c < b; c++) {
                long long q = base + (long long)(p - p0) * b + c;
                cci[q] = ci[p] * b + c;
                cv[q] = val[((long long)p * b + r) * b + c];
            }
        if (t == 0) crp[nrows] = (int)((long long)rp[nb] * b * b);
    }
}

void launch_bsr_to_csr(int nb, int b, const int *rp, const int *ci, const double *val, DCSR &A,
                       cudaStream_t s) {
    long long n = (long long)nb * b;
    k_bsr_to_csr<<<GRID(n, 256), 256, 0, s>>>(nb, b, rp, ci, val, A.rp, A.ci, A.v);
}

// --------------------------------------------------------------- level split
__global__ void k_level_flags(const int8_t *lvl, const int *gdof, int n, int level, int *isF,
                              int *isC, int *err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int g = gdof ? gdof[i] : i;
    int lv = lvl[g];
    isF[i] = lv == level;
    isC[i] = lv > level;
    if (lv < level) atomicOr(err, ERRW_INVALID);
}

void launch_level_flags(const int8_t *dof_level_g, const int *gdof, int n, int level, int *isF,
                        int *isC, int *err, cudaStream_t s) {
    k_level_flags<<<GRID(n, 256), 256, 0, s>>>(dof_level_g, gdof, n, level, isF, isC, err);
}

__global__ void k_index_maps(const int *isF, const int *isC, const int *fpos, const int *cpos,
                             int n, int *fidx, int *cidx, int *fmap, int *cmap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (isF[i]) { fidx[fpos[i]] = i; fmap[i] = fpos[i]; } else fmap[i] = -1;
    if (isC[i]) { cidx[cpos[i]] = i; cmap[i] = cpos[i]; } else cmap[i] = -1;
}

void launch_index_maps(const int *isF, const int *isC, const int *fpos_ex, const int *cpos_ex,
                       int n, int *fidx, int *cidx, int *fmap, int *cmap, cudaStream_t s) {
    k_index_maps<<<GRID(n, 256), 256, 0, s>>>(isF, isC, fpos_ex, cpos_ex, n, fidx, cidx, fmap, cmap);
}

// ------------------------------------------------------------ submatrix
__global__ void k_sub_count(const int *rp, const int *ci, const int *ridx, int nr, const int *cmap,
                            int *cnt) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    int i = ridx[r], c = 0;
    for (int p = rp[i]; p < rp[i + 1]; p++) c += cmap[ci[p]] >= 0;
    cnt[r] = c;
}

__global__ void k_sub_fill(const int *rp, const int *ci, const double *v, const int *ridx, int nr,
                           const int *cmap, const int *orp, int *oci, double *ov) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    int i = ridx[r], q = orp[r];
    for (int p = rp[i]; p < rp[i + 1]; p++) {
        int c = cmap[ci[p]];
        if (c >= 0) { oci[q] = c; ov[q] = v[p]; q++; }
    }
}

int extract_submatrix(const DCSR &A, const int *ridx, int nr, const int *cmap, int ncols, DCSR &out,
                      cudaStream_t s, Arena &ar) {
    out.n = nr; out.m = ncols;
    out.rp = ar.alloc<int>(nr + 1);
    int *cnt = ar.alloc<int>(nr + 1);
    if (!out.rp || !cnt) return ST_NOMEM;
    k_sub_count<<<GRID(nr, 256), 256, 0, s>>>(A.rp, A.ci, ridx, nr, cmap, cnt);
    int tot = 0;
    int rc = scan_exclusive(cnt, out.rp, nr, s, ar, &tot);
    ar.release(cnt);
    if (rc) return rc;
    out.nnz = tot;
    out.ci = ar.alloc<int>(tot + 1);
    out.v = ar.alloc<double>(tot + 1);
    if (!out.ci || !out.v) return ST_NOMEM;
    k_sub_fill<<<GRID(nr, 256), 256, 0, s>>>(A.rp, A.ci, A.v, ridx, nr, cmap, out.rp, out.ci, out.v);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// ------------------------------------------------------------ D_FF^{-1}
__device__ double csr_get(const int *rp, const int *ci, const double *v, int i, int j) {
    for (int p = rp[i]; p < rp[i + 1]; p++)
        if (ci[p] == j) return v[p];
    return 0.0;
}

// Gauss-Jordan with partial pivoting (first row of largest |pivot|),
// singular when |pivot| <= 1e-14 ||B||_inf.  Same operation order as the
// CPU reading.
__device__ int block_inverse(int k, const double *B, double *inv) {
    double m[16], x[16];
    double nrm = 0.0;
    for (int r = 0; r < k; r++) {
        double s = 0.0;
        for (int c = 0; c < k; c++) s = s + fabs(B[r * k + c]);
        if (s > nrm) nrm = s;
    }
    for (int t = 0; t < k * k; t++) { m[t] = B[t]; x[t] = 0.0; }
    for (int r = 0; r < k; r++) x[r * k + r] = 1.0;
    for (int c = 0; c < k; c++) {
        int p = c;
        for (int r = c + 1; r < k; r++)
            if (fabs(m[r * k + c]) > fabs(m[p * k + c])) p = r;
        if (!(fabs(m[p * k + c]) > 1e-14 * nrm)) return 1;
        if (p != c)
            for (int t = 0; t < k; t++) {
                double s = m[c * k + t]; m[c * k + t] = m[p * k + t]; m[p * k + t] = s;
                s = x[c * k + t]; x[c * k + t] = x[p * k + t]; x[p * k + t] = s;
            }
        double piv = m[c * k + c];
        for (int t = 0; t < k; t++) { m[c * k + t] = m[c * k + t] / piv; x[c * k + t] = x[c * k + t] / piv; }
        for (int r = 0; r < k; r++) {
            if (r == c) continue;
            double f = m[r * k + c];
            for (int t = 0; t < k; t++) {
                m[r * k + t] = m[r * k + t] - f * m[c * k + t];
                x[r * k + t] = x[r * k + t] - f * x[c * k + t];
            }
        }
    }
    for (int t = 0; t < k * k; t++) inv[t] = x[t];
    return 0;
}

__global__ void k_mgr_dinv(int nF, const int *rp, const int *ci, const double *v, const int *fidx,
                           const int *gdof, int b, int relax, int *gstart, int *gsize,
                           double *dinv, int *errw) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nF) return;
    if (relax != 2) {
        double aii = csr_get(rp, ci, v, f, f);
        double d = aii;
        if (relax == 1) {
            double s = 0.0;
            for (int p = rp[f]; p < rp[f + 1]; p++)
                if (ci[p] != f) s = s + fabs(v[p]);
            d = aii < 0.0 ? aii - s : aii + s;
        }
        gstart[f] = f; gsize[f] = 1;
        if (d == 0.0) {
            atomicOr(errw, ERRW_SINGULAR);
            atomicMin(errw + 1, f);  // the first singular F point
            dinv[(long long)f * 4] = 0.0;
            return;
        }
        dinv[(long long)f * 4] = 1.0 / d;
        dinv[(long long)f * 4 + 1] = dinv[(long long)f * 4 + 2] = dinv[(long long)f * 4 + 3] = 0.0;
        return;
    }
    auto blk = [&](int q) { int g = gdof ? gdof[fidx[q]] : fidx[q]; return g / b; };
    int my = blk(f);
    int g0 = f;
    while (g0 > 0 && f - g0 < 3 && blk(g0 - 1) == my) g0--;
    int k = 0;
    while (g0 + k < nF && k < 4 && blk(g0 + k) == my) k++;
    double B[16], inv[16];
    for (int r = 0; r < k; r++)
        for (int c = 0; c < k; c++) B[r * k + c] = csr_get(rp, ci, v, g0 + r, g0 + c);
    gstart[f] = g0; gsize[f] = k;
    int rr = f - g0;
    if (block_inverse(k, B, inv)) {
        atomicOr(errw, ERRW_SINGULAR);
        atomicMin(errw + 1, f);
        for (int c = 0; c < 4; c++) dinv[(long long)f * 4 + c] = 0.0;
        return;
    }
    for (int c = 0; c < 4; c++) dinv[(long long)f * 4 + c] = c < k ? inv[rr * k + c] : 0.0;
}

int mgr_dinv(const DCSR &AFF, const int *fidx, const int *gdof, int b, int relax, int *gstart,
             int *gsize, double *dinv, int *errw, cudaStream_t s) {
    k_mgr_dinv<<<GRID(AFF.n, 128), 128, 0, s>>>(AFF.n, AFF.rp, AFF.ci, AFF.v, fidx, gdof, b, relax,
                                                 gstart, gsize, dinv, errw);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// --------------------------------------------------------------------- W
// Row f of W = -D^{-1} A_FC: merge of the A_FC rows of f's block (<= 4
// sorted lists); at each column, acc = sum over block rows q ascending of
// dinv[f][q] * a_qj (from +0.0), then W = -acc.
template <bool FILL>
__global__ void k_build_w(int nF, const int *rp, const int *ci, const double *v, const int *gstart,
                          const int *gsize, const double *dinv, int *cnt, const int *wrp, int *wci,
                          double *wv) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nF) return;
    int g0 = gstart[f], k = gsize[f];
    int head[4], end[4];
    for (int q = 0; q < k; q++) { head[q] = rp[g0 + q]; end[q] = rp[g0 + q + 1]; }
    int c = 0;
    int out = FILL ? wrp[f] : 0;
    for (;;) {
        int j = 0x7fffffff;
        for (int q = 0; q < k; q++)
            if (head[q] < end[q] && ci[head[q]] < j) j = ci[head[q]];
        if (j == 0x7fffffff) break;
        double acc = 0.0;
        for (int q = 0; q < k; q++)
            if (head[q] < end[q] && ci[head[q]] == j) {
                if (FILL) acc = acc + dinv[(long long)f * 4 + q] * v[head[q]];
                head[q]++;
            }
        if (FILL) { wci[out] = j; wv[out] = -acc; out++; }
        c++;
    }
    if (!FILL) cnt[f] = c;
}

int mgr_build_w(const DCSR &AFC, const int *gstart, const int *gsize, const double *dinv, DCSR &W,
                cudaStream_t s, Arena &ar) {
    int nF = AFC.n;
    W.n = nF; W.m = AFC.m;
    W.rp = ar.alloc<int>(nF + 1);
    int *cnt = ar.alloc<int>(nF + 1);
    if (!W.rp || !cnt) return ST_NOMEM;
    k_build_w<false><<<GRID(nF, 128), 128, 0, s>>>(nF, AFC.rp, AFC.ci, AFC.v, gstart, gsize, dinv,
                                                   cnt, nullptr, nullptr, nullptr);
    int tot = 0;
    int rc = scan_exclusive(cnt, W.rp, nF, s, ar, &tot);
    ar.release(cnt);
    if (rc) return rc;
    W.nnz = tot;
    W.ci = ar.alloc<int>(tot + 1);
    W.v = ar.alloc<double>(tot + 1);
    if (!W.ci || !W.v) return ST_NOMEM;
    k_build_w<true><<<GRID(nF, 128), 128, 0, s>>>(nF, AFC.rp, AFC.ci, AFC.v, gstart, gsize, dinv,
                                                  nullptr, W.rp, W.ci, W.v);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// ---------------------------------------------------------------- SpGEMM
// Row i of C = A*B (+E): for (i,k) in A ascending k, for (k,j) in B
// ascending j: acc[j] = acc[j] + a_ik*b_kj (acc = +0.0 on first touch);
// then acc[j] = acc[j] + e_ij.  One thread per row, private open-addressing
// table in global scratch; the output row is then sorted by column.
__global__ void k_spgemm_bound(int n, const int *arp, const int *aci, const int *brp,
                               const int *erp, int *bound) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    long long s = 0;
    for (int p = arp[i]; p < arp[i + 1]; p++) { int k = aci[p]; s += brp[k + 1] - brp[k]; }
    if (erp) s += erp[i + 1] - erp[i];
    // hash capacity: power of two >= 2*bound (>= 8)
    long long cap = 8;
    while (cap < 2 * s) cap <<= 1;
    bound[i] = (int)(cap > 0x40000000LL ? 0x40000000LL : cap);
}

__device__ __forceinline__ unsigned hash_col(int j) { return (unsigned)j * 2654435761u; }

// One warp per row of C = A B (+ E).  The entries p of A's row are taken in
// order; for each, the lanes insert the distinct columns of B's row k = a_p
// into the row's hash table at once (slots claimed with atomicCAS), and the
// warp synchronises before the next p, so every entry of C receives its
// contributions in ascending p order and E's entry last, as the row-by-row
// definition sums them.  NUMERIC = false counts the distinct columns; the
// numeric pass gathers the table and sorts the row by column.
__device__ __forceinline__ void spgemm_insert(int *key, double *val, unsigned cap, int j, double prod,
                                              bool numeric, int &claimed, int *errw) {
    unsigned h = hash_col(j) & (cap - 1);
    for (unsigned probe = 0; probe < cap; probe++) {
        int kk = ((volatile int *)key)[h];
        if (kk < 0) {
            kk = atomicCAS(key + h, -1, j);
            if (kk < 0) {
                if (numeric) { val[h] = 0.0; val[h] = val[h] + prod; }
                claimed++;
                return;
            }
        }
        if (kk == j) {
            if (numeric) val[h] = val[h] + prod;
            return;
        }
        h = (h + 1) & (cap - 1);
    }
    atomicOr(errw, ERRW_OVERFLOW);  // table full: cannot happen when cap >= 2 * distinct
}

// The slot of column j in the row's table, claimed when absent (fresh).
// -1 when the table is full (cannot happen when cap >= 2 * distinct).
__device__ __forceinline__ int spgemm_slot(int *key, unsigned cap, int j, bool &fresh, int *errw) {
    unsigned h = hash_col(j) & (cap - 1);
    for (unsigned probe = 0; probe < cap; probe++) {
        int kk = ((volatile int *)key)[h];
        if (kk < 0) {
            kk = atomicCAS(key + h, -1, j);
            if (kk < 0) {
                fresh = true;
                return (int)h;
            }
        }
        if (kk == j) return (int)h;
        h = (h + 1) & (cap - 1);
    }
    atomicOr(errw, ERRW_OVERFLOW);
    return -1;
}

template <bool NUMERIC>
__global__ void k_spgemm_row(int r0, int r1, const int *arp, const int *aci, const double *av,
                             const int *brp, const int *bci, const double *bv, const int *erp,
                             const int *eci, const double *ev, const long long *capoff,
                             long long base, int *hkey, double *hval, int *cnt, const int *crp,
                             int *cci, double *cv, int *errw) {
    const unsigned FULL = 0xffffffffu;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= r1 - r0) return;  // whole warps
    const int i = r0 + (int)wid;
    const long long off = capoff[i] - base;
    const unsigned cap = (unsigned)(capoff[i + 1] - capoff[i]);
    int *key = hkey + off;
    double *val = hval + off;
    for (unsigned t = lane; t < cap; t += 32) key[t] = -1;
    __syncwarp();
    int claimed = 0;
    // The products a_ip b_pj in (p, j) order, 32 at a time: a chunk may span
    // several short rows of B.  Lanes of a chunk with the same column form a
    // group (__match_any_sync); its lowest lane adds the group's products in
    // lane order, which is ascending p, so every entry still receives its
    // contributions in the order of the row-by-row definition.
    __shared__ int own_s[8][32], bef_s[8][32];
    __shared__ double prod_s[8][32];
    const int wib = threadIdx.x >> 5;
    int p = arp[i], qoff = 0;  // next product: entry qoff of B's row a_p
    const int pe = arp[i + 1];
    while (p < pe) {
        const int pl = p + lane;
        int len = 0;
        if (pl < pe) {
            const int kk = aci[pl];
            len = brp[kk + 1] - brp[kk] - (lane == 0 ? qoff : 0);
        }
        int cum = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, cum, o);
            if (lane >= o) cum += y;
        }
        const int before = cum - len;
        const int total = __shfl_sync(FULL, cum, 31);
        const int nprod = total < 32 ? total : 32;
        bef_s[wib][lane] = before;
        for (int t = before; t < cum && t < 32; t++) own_s[wib][t] = lane;
        __syncwarp();
        int j = -1;
        if (lane < nprod) {
            const int l = own_s[wib][lane];
            const int pp = p + l;
            const int kk = aci[pp];
            const int q = brp[kk] + (l == 0 ? qoff : 0) + (lane - bef_s[wib][l]);
            j = bci[q];
            prod_s[wib][lane] = NUMERIC ? av[pp] * bv[q] : 0.0;
        }
        const unsigned act = __ballot_sync(FULL, lane < nprod);
        __syncwarp();
        if (lane < nprod) {
            const unsigned grp = __match_any_sync(act, j);
            if ((grp & ((1u << lane) - 1u)) == 0u) {  // the group's lowest lane
                bool fresh = false;
                const int h = spgemm_slot(key, cap, j, fresh, errw);
                if (h >= 0) {
                    if (fresh) claimed++;
                    if (NUMERIC) {
                        double acc = fresh ? 0.0 : val[h];
                        for (unsigned rest = grp; rest; rest &= rest - 1u) acc = acc + prod_s[wib][__ffs(rest) - 1];
                        val[h] = acc;
                    }
                }
            }
        }
        __syncwarp();
        if (total <= 32) {
            p += 32;
            qoff = 0;
        } else {
            const int ls = __ffs(__ballot_sync(FULL, cum > 32)) - 1;  // first row not used up
            const int bls = __shfl_sync(FULL, before, ls);
            qoff = (ls == 0 ? qoff : 0) + (32 - bls);
            p += ls;
        }
    }
    if (erp) {
        for (int q = erp[i] + lane; q < erp[i + 1]; q += 32)
            spgemm_insert(key, val, cap, eci[q], NUMERIC ? ev[q] : 0.0, NUMERIC, claimed, errw);
        __syncwarp();
    }
    if (!NUMERIC) {
        for (int o = 16; o > 0; o >>= 1) claimed += __shfl_xor_sync(FULL, claimed, o);
        if (lane == 0) cnt[i] = claimed;
        return;
    }
    // gather the table into the row (unsorted), then sort by column
    const int o = crp[i];
    int len = 0;
    const unsigned below = (1u << lane) - 1u;
    for (unsigned t0 = 0; t0 < cap; t0 += 32) {
        const unsigned t = t0 + lane;
        const bool has = t < cap && key[t] >= 0;
        const unsigned m = __ballot_sync(FULL, has);
        if (has) {
            cci[o + len + __popc(m & below)] = key[t];
            cv[o + len + __popc(m & below)] = val[t];
        }
        len += __popc(m);
    }
    __syncwarp();
    if (len <= 2048) {
        // rank sort (columns are distinct): entry e goes to the number of smaller columns,
        // through the table's storage, then back
        for (int e = lane; e < len; e += 32) {
            const int ce = cci[o + e];
            int r = 0;
            for (int f = 0; f < len; f++) r += cci[o + f] < ce;
            key[r] = ce;
            val[r] = cv[o + e];
        }
        __syncwarp();
        for (int e = lane; e < len; e += 32) {
            cci[o + e] = key[e];
            cv[o + e] = val[e];
        }
    } else if (lane == 0) {
        // shell sort (Ciura gaps) for long rows
        const int gaps[8] = {701, 301, 132, 57, 23, 10, 4, 1};
        for (int gi = 0; gi < 8; gi++) {
            const int g = gaps[gi];
            for (int a2 = g; a2 < len; a2++) {
                const int kc = cci[o + a2];
                const double kv = cv[o + a2];
                int b2 = a2;
                while (b2 >= g && cci[o + b2 - g] > kc) {
                    cci[o + b2] = cci[o + b2 - g];
                    cv[o + b2] = cv[o + b2 - g];
                    b2 -= g;
                }
                cci[o + b2] = kc;
                cv[o + b2] = kv;
            }
        }
    }
}

int spgemm(const DCSR &A, const DCSR &B, const DCSR *E, DCSR &C, cudaStream_t s, Arena &ar) {
    int n = A.n;
    C.n = n; C.m = B.m;
    int *capv = ar.alloc<int>(n + 1);
    long long *capoff = ar.alloc<long long>(n + 1);
    int *cnt = ar.alloc<int>(n + 1);
    C.rp = ar.alloc<int>(n + 1);
    if (!capv || !capoff || !cnt || !C.rp) return ST_NOMEM;
    k_spgemm_bound<<<GRID(n, 256), 256, 0, s>>>(n, A.rp, A.ci, B.rp, E ? E->rp : nullptr, capv);
    long long totcap = 0;
    int rc = scan_exclusive_ll(capv, capoff, n, s, ar, &totcap);
    if (rc) return rc;
    std::vector<long long> hoff(n + 1);
    cudaMemcpyAsync(hoff.data(), capoff, sizeof(long long) * (n + 1), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    const long long budget = 1LL << 26;  // hash slots per chunk
    long long maxchunk = 0;
    std::vector<int> cuts{0};
    while (cuts.back() < n) {
        int r0 = cuts.back(), r1 = r0 + 1;
        while (r1 < n && hoff[r1 + 1] - hoff[r0] <= budget) r1++;
        maxchunk = std::max(maxchunk, hoff[r1] - hoff[r0]);
        cuts.push_back(r1);
    }
    int *errw = ar.alloc<int>(1);
    if (!errw) return ST_NOMEM;
    cudaMemsetAsync(errw, 0, sizeof(int), s);
    int *hkey = ar.alloc<int>(maxchunk + 1);
    double *hval = ar.alloc<double>(maxchunk + 1);
    if (!hkey || !hval) return ST_NOMEM;
    const int *erp = E ? E->rp : nullptr, *eci = E ? E->ci : nullptr;
    const double *ev = E ? E->v : nullptr;
    for (size_t c = 0; c + 1 < cuts.size(); c++) {
        int r0 = cuts[c], r1 = cuts[c + 1];
        k_spgemm_row<false><<<GRID((long long)(r1 - r0) * 32, 256), 256, 0, s>>>(
            r0, r1, A.rp, A.ci, A.v, B.rp, B.ci, B.v, erp, eci, ev, capoff, hoff[r0], hkey, hval,
            cnt, nullptr, nullptr, nullptr, errw);
    }
    int tot = 0;
    rc = scan_exclusive(cnt, C.rp, n, s, ar, &tot);
    if (rc) return rc;
    C.nnz = tot;
    C.ci = ar.alloc<int>(tot + 1);
    C.v = ar.alloc<double>(tot + 1);
    if (!C.ci || !C.v) return ST_NOMEM;
    for (size_t c = 0; c + 1 < cuts.size(); c++) {
        int r0 = cuts[c], r1 = cuts[c + 1];
        k_spgemm_row<true><<<GRID((long long)(r1 - r0) * 32, 256), 256, 0, s>>>(
            r0, r1, A.rp, A.ci, A.v, B.rp, B.ci, B.v, erp, eci, ev, capoff, hoff[r0], hkey, hval,
            cnt, C.rp, C.ci, C.v, errw);
    }
    int herr = 0;
    cudaMemcpyAsync(&herr, errw, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    ar.release(hkey); ar.release(hval); ar.release(capv); ar.release(capoff); ar.release(cnt);
    ar.release(errw);
    if (herr) return ST_NOMEM;
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// -------------------------------------------------------------- transpose
__global__ void k_col_count(int nnz, const int *ci, int *cnt) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz;
         p += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[p]], 1);
}

// one warp per source row (the order inside a row of the transpose is
// fixed by k_row_sort afterwards)
__global__ void k_tr_fill(int n, const int *rp, const int *ci, const double *v, const int *trp,
                          int *cursor, int *tci, double *tv) {
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    for (int p = rp[i] + lane; p < rp[i + 1]; p += 32) {
        const int j = ci[p];
        const int q = trp[j] + atomicAdd(&cursor[j], 1);
        tci[q] = (int)i;
        if (v) tv[q] = v[p];
    }
}

// sort each row by column (source row index; the keys of a row are
// distinct).  One warp per row: rows of up to 128 entries by rank (each
// lane holds up to 4 entries, counts the smaller keys of the row, and all
// writes wait for all reads); longer rows by one lane's shell sort.
__global__ void k_row_sort(int n, const int *rp, int *ci, double *v) {
    const unsigned FULL = 0xffffffffu;
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int o = rp[i], len = rp[i + 1] - o;
    if (len <= 128) {
        int key[4], rank[4];
        double val[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int e = lane + 32 * u;
            key[u] = e < len ? ci[o + e] : 0;
            val[u] = (e < len && v) ? v[o + e] : 0.0;
            rank[u] = 0;
        }
        for (int f = 0; f < len; f++) {
            const int kf = ci[o + f];
#pragma unroll
            for (int u = 0; u < 4; u++) rank[u] += kf < key[u];
        }
        __syncwarp(FULL);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int e = lane + 32 * u;
            if (e < len) {
                ci[o + rank[u]] = key[u];
                if (v) v[o + rank[u]] = val[u];
            }
        }
        return;
    }
    if (lane != 0) return;
    const int gaps[8] = {701, 301, 132, 57, 23, 10, 4, 1};
    for (int gi = 0; gi < 8; gi++) {
        int g = gaps[gi];
        for (int a = g; a < len; a++) {
            int kc = ci[o + a];
            double kv = v ? v[o + a] : 0.0;
            int b = a;
            while (b >= g && ci[o + b - g] > kc) {
                ci[o + b] = ci[o + b - g];
                if (v) v[o + b] = v[o + b - g];
                b -= g;
            }
            ci[o + b] = kc;
            if (v) v[o + b] = kv;
        }
    }
}

int transpose(const DCSR &A, DCSR &T, cudaStream_t s, Arena &ar) {
    T.n = A.m; T.m = A.n; T.nnz = A.nnz;
    T.rp = ar.alloc<int>(A.m + 1);
    int *cnt = ar.alloc<int>(A.m + 1);
    T.ci = ar.alloc<int>(A.nnz + 1);
    T.v = A.v ? ar.alloc<double>(A.nnz + 1) : nullptr;
    if (!T.rp || !cnt || !T.ci || (A.v && !T.v)) return ST_NOMEM;
    cudaMemsetAsync(cnt, 0, sizeof(int) * (A.m + 1), s);
    k_col_count<<<GRID(A.nnz, 256) > 4096 ? 4096 : GRID(A.nnz, 256), 256, 0, s>>>(A.nnz, A.ci, cnt);
    int rc = scan_exclusive(cnt, T.rp, A.m, s, ar, nullptr);
    if (rc) return rc;
    cudaMemsetAsync(cnt, 0, sizeof(int) * (A.m + 1), s);
    k_tr_fill<<<GRID((long long)A.n * 32, 256), 256, 0, s>>>(A.n, A.rp, A.ci, A.v, T.rp, cnt, T.ci, T.v);
    k_row_sort<<<GRID((long long)A.m * 32, 256), 256, 0, s>>>(A.m, T.rp, T.ci, T.v);
    cudaStreamSynchronize(s);
    ar.release(cnt);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// --------------------------------------------------------------- strength
// s_i = -1 if a_ii < 0 else +1; m_i = max over off-diagonal same-function j
// of -s_i a_ij (from 0); j strong iff m_i > 0 and -s_i a_ij >= theta m_i.
// One warp per row.  s_i = sign(a_ii); m_i = max over same-function j != i
// of -s_i a_ij; j is strong when m_i > 0 and -s_i a_ij >= theta m_i.  The
// maximum and the comparisons do not depend on the order of the entries.
__global__ void k_strength(int n, const int *rp, const int *ci, const double *v, const int *func,
                           double theta, uint8_t *sflag, int *cnt) {
    const unsigned FULL = 0xffffffffu;
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int a = rp[i], e = rp[i + 1];
    double aii = 0.0;
    for (int p = a + lane; p < e; p += 32)
        if (ci[p] == i) aii = v[p];
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_xor_sync(FULL, aii, o);
        if (y != 0.0) aii = y;  // the one diagonal entry (or zero)
    }
    const bool neg = aii < 0.0;
    const int fi = func[i];
    double m = 0.0;
    for (int p = a + lane; p < e; p += 32) {
        const int j = ci[p];
        if (j == i || func[j] != fi) continue;
        const double val = neg ? v[p] : -v[p];
        if (val > m) m = val;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(FULL, m, o));
    const double thr = theta * m;
    int c = 0;
    for (int p0 = a; p0 < e; p0 += 32) {
        const int p = p0 + lane;
        bool st = false;
        if (p < e) {
            const int j = ci[p];
            if (m > 0.0 && j != i && func[j] == fi) {
                const double val = neg ? v[p] : -v[p];
                st = val >= thr;
            }
            sflag[p] = st;
        }
        c += __popc(__ballot_sync(FULL, st));
    }
    if (lane == 0) cnt[i] = c;
}

// one warp per row: strong entries in row order
__global__ void k_strength_fill(int n, const int *rp, const int *ci, const uint8_t *sflag,
                                const int *srp, int *sci) {
    const unsigned FULL = 0xffffffffu;
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    int q = srp[i];
    const int e = rp[i + 1];
    for (int p0 = rp[i]; p0 < e; p0 += 32) {
        const int p = p0 + lane;
        const bool st = p < e && sflag[p];
        const unsigned b = __ballot_sync(FULL, st);
        if (st) sci[q + __popc(b & ((1u << lane) - 1u))] = ci[p];
        q += __popc(b);
    }
}

int amg_strength(const DCSR &A, const int *func, double theta, uint8_t *sflag, DCSR &S,
                 cudaStream_t s, Arena &ar) {
    int n = A.n;
    S.n = S.m = n;
    S.rp = ar.alloc<int>(n + 1);
    int *cnt = ar.alloc<int>(n + 1);
    if (!S.rp || !cnt) return ST_NOMEM;
    k_strength<<<GRID((long long)n * 32, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, func, theta, sflag, cnt);
    int tot = 0;
    int rc = scan_exclusive(cnt, S.rp, n, s, ar, &tot);
    ar.release(cnt);
    if (rc) return rc;
    S.nnz = tot;
    S.ci = ar.alloc<int>(tot + 1);
    S.v = nullptr;
    if (!S.ci) return ST_NOMEM;
    k_strength_fill<<<GRID((long long)n * 32, 256), 256, 0, s>>>(n, A.rp, A.ci, sflag, S.rp, S.ci);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// ------------------------------------------------------------------- PMIS
// Weight u(i, level): the SplitMix64 output function (Steele, Lea & Flood
// 2014) of the state i + 2^32 level, top 53 bits times 2^-53.
__device__ double pmis_u01(unsigned i, unsigned level) {
    unsigned long long z = (unsigned long long)i + ((unsigned long long)level << 32);
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void k_pmis_init(int n, const int *strp, int level, double *w, int *cf, int *und) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = strp[i + 1] - strp[i];
    w[i] = (double)c + pmis_u01((unsigned)i, (unsigned)level);
    cf[i] = c == 0 ? -1 : 0;
    if (c) atomicAdd(und, 1);
}

__global__ void k_pmis_select(int n, const int *srp, const int *sci, const int *strp,
                              const int *stci, const double *w, const int *cf, int *sel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int best = 0;
    if (cf[i] == 0) {
        best = 1;
        double wi = w[i];
        for (int p = srp[i]; p < srp[i + 1] && best; p++) {
            int j = sci[p];
            if (cf[j] == 0 && (w[j] > wi || (w[j] == wi && j > i))) best = 0;
        }
        for (int p = strp[i]; p < strp[i + 1] && best; p++) {
            int j = stci[p];
            if (cf[j] == 0 && (w[j] > wi || (w[j] == wi && j > i))) best = 0;
        }
    }
    sel[i] = best;
}

__global__ void k_pmis_mark_c(int n, const int *sel, int *cf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && sel[i]) cf[i] = 1;
}

__global__ void k_pmis_mark_f(int n, const int *srp, const int *sci, int *cf, int *und) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cf[i] != 0) return;
    for (int p = srp[i]; p < srp[i + 1]; p++)
        if (cf[sci[p]] == 1) { cf[i] = -1; return; }
    atomicAdd(und, 1);
}

int amg_pmis(const DCSR &S, const DCSR &ST, int level, int *cf, cudaStream_t s, Arena &ar) {
    int n = S.n;
    double *w = ar.alloc<double>(n + 1);
    int *sel = ar.alloc<int>(n + 1);
    int *und = ar.alloc<int>(1);
    if (!w || !sel || !und) return ST_NOMEM;
    cudaMemsetAsync(und, 0, sizeof(int), s);
    k_pmis_init<<<GRID(n, 256), 256, 0, s>>>(n, ST.rp, level, w, cf, und);
    int hund = 0;
    cudaMemcpyAsync(&hund, und, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int rounds = 0;
    while (hund > 0 && rounds < 10000) {
        k_pmis_select<<<GRID(n, 256), 256, 0, s>>>(n, S.rp, S.ci, ST.rp, ST.ci, w, cf, sel);
        k_pmis_mark_c<<<GRID(n, 256), 256, 0, s>>>(n, sel, cf);
        cudaMemsetAsync(und, 0, sizeof(int), s);
        k_pmis_mark_f<<<GRID(n, 256), 256, 0, s>>>(n, S.rp, S.ci, cf, und);
        cudaMemcpyAsync(&hund, und, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        rounds++;
    }
    ar.release(w); ar.release(sel); ar.release(und);
    if (hund > 0) return ST_TIMEOUT;
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// -------------------------------------------------------- extended+i
__device__ __forceinline__ double abar(double akk, double akl) {
    if (akk >= 0.0) return akl < 0.0 ? akl : 0.0;
    return akl > 0.0 ? akl : 0.0;
}

__device__ __forceinline__ bool in_sorted(const int *a, int len, int j) {
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int x = a[mid];
        if (x == j) return true;
        if (x < j) lo = mid + 1; else hi = mid - 1;
    }
    return false;
}

// bound on |Chat_i| candidates: sum over strong j of (C ? 1 : |S_j|)
__global__ void k_extpi_bound(int n, const int *rp, const int *ci, const uint8_t *sflag,
                              const int *srp, const int *cf, int *bound) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int b = 0;
    if (cf[i] != 1)
        for (int p = rp[i]; p < rp[i + 1]; p++)
            if (sflag[p]) { int j = ci[p]; b += cf[j] == 1 ? 1 : srp[j + 1] - srp[j]; }
    bound[i] = b + 1;
}

// Pass 1: Chat_i (sorted, unique) and the untruncated weights into scratch;
// final row length into len[i].  One warp per row.  Lanes gather candidates,
// compute terms and update the num slots (within one neighbour row k every
// entry names a different column, so every slot gets at most one term per k);
// every scalar the definition accumulates in order (the diagonal, each den)
// is summed in that order by all lanes alike, from shuffled terms, so the
// result equals the row-by-row definition bit for bit.
__device__ __forceinline__ int find_sorted(const int *a, int len, int j) {
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int x = a[mid];
        if (x == j) return mid;
        if (x < j) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

// acc += the terms t of the lanes in mask, in ascending lane order (all lanes)
__device__ __forceinline__ double ordered_add(double acc, unsigned mask, double t) {
    for (unsigned m = mask; m; m &= m - 1) acc = acc + __shfl_sync(0xffffffffu, t, __ffs(m) - 1);
    return acc;
}

__global__ void k_extpi_weights(int n, const int *rp, const int *ci, const double *v,
                                const uint8_t *sflag, const int *cf, const int *func,
                                const long long *boff, int *cand, double *wts, int *chat_len,
                                int *len, int pmax) {
    const unsigned FULL = 0xffffffffu;
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= n) return;  // whole warps
    const int i = (int)wid;
    if (cf[i] == 1) {
        if (lane == 0) { len[i] = 1; chat_len[i] = 0; }
        return;
    }
    int *L = cand + boff[i];
    double *num = wts + boff[i];
    const int r0 = rp[i], r1 = rp[i + 1];
    const unsigned below = (1u << lane) - 1u;
    // candidates: strong C neighbours, and strong C neighbours of strong F neighbours
    int cnt = 0;
    for (int p0 = r0; p0 < r1; p0 += 32) {
        const int p = p0 + lane;
        bool take = false;
        int j = 0;
        if (p < r1 && sflag[p]) { j = ci[p]; take = cf[j] == 1; }
        const unsigned m = __ballot_sync(FULL, take);
        if (take) L[cnt + __popc(m & below)] = j;
        cnt += __popc(m);
    }
    for (int p = r0; p < r1; p++) {
        if (!sflag[p]) continue;
        const int j = ci[p];
        if (cf[j] == 1) continue;
        const int q1 = rp[j + 1];
        for (int q0 = rp[j]; q0 < q1; q0 += 32) {
            const int q = q0 + lane;
            bool take = false;
            int c = 0;
            if (q < q1 && sflag[q]) { c = ci[q]; take = cf[c] == 1; }
            const unsigned m = __ballot_sync(FULL, take);
            if (take) L[cnt + __popc(m & below)] = c;
            cnt += __popc(m);
        }
    }
    __syncwarp();
    // sort + unique (one lane)
    if (lane == 0) {
        const int gaps[8] = {701, 301, 132, 57, 23, 10, 4, 1};
        for (int gi = 0; gi < 8; gi++) {
            const int g = gaps[gi];
            for (int a = g; a < cnt; a++) {
                int kc = L[a], b = a;
                while (b >= g && L[b - g] > kc) { L[b] = L[b - g]; b -= g; }
                L[b] = kc;
            }
        }
        int u = 0;
        for (int a = 0; a < cnt; a++)
            if (u == 0 || L[a] != L[u - 1]) L[u++] = L[a];
        cnt = u;
        chat_len[i] = cnt;
    }
    cnt = __shfl_sync(FULL, cnt, 0);
    __syncwarp();
    if (cnt == 0) {
        if (lane == 0) len[i] = 0;
        return;
    }
    for (int t = lane; t < cnt; t += 32) num[t] = 0.0;
    double diag = 0.0;
    for (int p0 = r0; p0 < r1; p0 += 32) {
        const int p = p0 + lane;
        const bool d = p < r1 && ci[p] == i;
        const unsigned m = __ballot_sync(FULL, d);
        if (m) diag = __shfl_sync(FULL, d ? v[p] : 0.0, 31 - __clz(m));
    }
    const int fi = func[i];
    __syncwarp();
    // phase 1
    for (int p0 = r0; p0 < r1; p0 += 32) {
        const int p = p0 + lane;
        bool dt = false;
        double t = 0.0;
        if (p < r1) {
            const int j = ci[p];
            if (j != i && func[j] == fi) {
                const int at = find_sorted(L, cnt, j);
                if (at >= 0) num[at] = num[at] + v[p];
                else if (!sflag[p]) { dt = true; t = v[p]; }
            }
        }
        diag = ordered_add(diag, __ballot_sync(FULL, dt), t);
    }
    __syncwarp();
    // phase 2: strong F neighbours k in row order
    for (int p = r0; p < r1; p++) {
        const int k = ci[p];
        if (k == i || !sflag[p] || cf[k] == 1) continue;
        const double aik = v[p];
        const int k0 = rp[k], k1 = rp[k + 1];
        double akk = 0.0;
        for (int q0 = k0; q0 < k1; q0 += 32) {
            const int q = q0 + lane;
            const bool d = q < k1 && ci[q] == k;
            const unsigned m = __ballot_sync(FULL, d);
            if (m) akk = __shfl_sync(FULL, d ? v[q] : 0.0, 31 - __clz(m));
        }
        const int fk = func[k];
        double den = 0.0;
        for (int q0 = k0; q0 < k1; q0 += 32) {
            const int q = q0 + lane;
            bool sel = false;
            double t = 0.0;
            if (q < k1) {
                const int l = ci[q];
                if (l != k && func[l] == fk && (l == i || find_sorted(L, cnt, l) >= 0)) {
                    sel = true;
                    t = abar(akk, v[q]);
                }
            }
            den = ordered_add(den, __ballot_sync(FULL, sel), t);
        }
        if (den == 0.0) { diag = diag + aik; continue; }
        const double f = aik / den;
        for (int q0 = k0; q0 < k1; q0 += 32) {
            const int q = q0 + lane;
            bool dt = false;
            double t = 0.0;
            if (q < k1) {
                const int l = ci[q];
                if (l != k && func[l] == fk) {
                    const int at = find_sorted(L, cnt, l);
                    if (at >= 0) num[at] = num[at] + f * abar(akk, v[q]);
                    else if (l == i) { dt = true; t = f * abar(akk, v[q]); }
                }
            }
            diag = ordered_add(diag, __ballot_sync(FULL, dt), t);
        }
        __syncwarp();
    }
    if (diag == 0.0) {
        if (lane == 0) len[i] = 0;
        return;
    }
    for (int t = lane; t < cnt; t += 32) num[t] = -(num[t] / diag);
    if (lane == 0) len[i] = (pmax > 0 && cnt > pmax) ? pmax : cnt;
}

// Pass 2: truncation (pmax largest |w|, ties to the lower column; rescale by
// sum(all)/sum(kept) when sum(kept) != 0) and coarse renumbering.
__global__ void k_extpi_fill(int n, const int *cf, const int *cnum, const long long *boff,
                             const int *cand, const double *wts, const int *chat_len, const int *prp,
                             int *pci, double *pv, int pmax) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = prp[i], len = prp[i + 1] - o;
    if (cf[i] == 1) { pci[o] = cnum[i]; pv[o] = 1.0; return; }
    if (len == 0) return;
    const int *L = cand + boff[i];
    const double *w = wts + boff[i];
    int cnt = chat_len[i];
    if (!(pmax > 0 && cnt > pmax)) {
        for (int t = 0; t < cnt; t++) { pci[o + t] = cnum[L[t]]; pv[o + t] = w[t]; }
        return;
    }
    int ord[64];
    int K = pmax < 64 ? pmax : 64;
    // the K largest |w| (ties to the lower position), picked one at a time
    for (int s2 = 0; s2 < K; s2++) {
        int best = -1;
        for (int t = 0; t < cnt; t++) {
            bool used = false;
            for (int u = 0; u < s2; u++) if (ord[u] == t) { used = true; break; }
            if (used) continue;
            if (best < 0) { best = t; continue; }
            double x = fabs(w[t]), y = fabs(w[best]);
            if (x > y || (x == y && t < best)) best = t;
        }
        ord[s2] = best;
    }
    for (int a = 1; a < K; a++) {
        int kc = ord[a], b = a;
        while (b > 0 && ord[b - 1] > kc) { ord[b] = ord[b - 1]; b--; }
        ord[b] = kc;
    }
    double sall = 0.0, skept = 0.0;
    for (int t = 0; t < cnt; t++) sall = sall + w[t];
    for (int s2 = 0; s2 < K; s2++) skept = skept + w[ord[s2]];
    double scale = skept != 0.0 ? sall / skept : 1.0;
    for (int s2 = 0; s2 < K; s2++) {
        pci[o + s2] = cnum[L[ord[s2]]];
        pv[o + s2] = skept != 0.0 ? w[ord[s2]] * scale : w[ord[s2]];
    }
}

__global__ void k_count_flags(int n, const int *rp, const uint8_t *flag, int *cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int p = rp[i]; p < rp[i + 1]; p++) c += flag[p];
    cnt[i] = c;
}

__global__ void k_is_c(int n, const int *cf, int *isc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) isc[i] = cf[i] == 1;
}

int amg_extpi(const DCSR &A, const uint8_t *sflag, const int *cf, const int *func, int pmax,
              DCSR &P, int *nc, cudaStream_t s, Arena &ar) {
    int n = A.n;
    if (pmax > 64) pmax = 64;
    int *isc = ar.alloc<int>(n + 1);
    int *cnum = ar.alloc<int>(n + 1);
    int *bound = ar.alloc<int>(n + 1);
    long long *boff = ar.alloc<long long>(n + 1);
    int *chat = ar.alloc<int>(n + 1);
    int *len = ar.alloc<int>(n + 1);
    if (!isc || !cnum || !bound || !boff || !chat || !len) return ST_NOMEM;
    k_is_c<<<GRID(n, 256), 256, 0, s>>>(n, cf, isc);
    int rc = scan_exclusive(isc, cnum, n, s, ar, nc);
    if (rc) return rc;
    // strength row pointers from sflag (S rows are A rows filtered)
    int *scnt = ar.alloc<int>(n + 1), *srp = ar.alloc<int>(n + 1);
    if (!scnt || !srp) return ST_NOMEM;
    k_count_flags<<<GRID(n, 256), 256, 0, s>>>(n, A.rp, sflag, scnt);
    rc = scan_exclusive(scnt, srp, n, s, ar, nullptr);
    if (rc) return rc;
    k_extpi_bound<<<GRID(n, 128), 128, 0, s>>>(n, A.rp, A.ci, sflag, srp, cf, bound);
    long long totb = 0;
    rc = scan_exclusive_ll(bound, boff, n, s, ar, &totb);
    if (rc) return rc;
    int *cand = ar.alloc<int>(totb + 1);
    double *wts = ar.alloc<double>(totb + 1);
    if (!cand || !wts) return ST_NOMEM;
    k_extpi_weights<<<GRID((long long)n * 32, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, sflag, cf, func, boff,
                                                                 cand, wts, chat, len, pmax);
    P.n = n; P.m = *nc;
    P.rp = ar.alloc<int>(n + 1);
    if (!P.rp) return ST_NOMEM;
    int tot = 0;
    rc = scan_exclusive(len, P.rp, n, s, ar, &tot);
    if (rc) return rc;
    P.nnz = tot;
    P.ci = ar.alloc<int>(tot + 1);
    P.v = ar.alloc<double>(tot + 1);
    if (!P.ci || !P.v) return ST_NOMEM;
    k_extpi_fill<<<GRID(n, 128), 128, 0, s>>>(n, cf, cnum, boff, cand, wts, chat, P.rp, P.ci, P.v,
                                              pmax);
    cudaStreamSynchronize(s);
    ar.release(cand); ar.release(wts); ar.release(isc); ar.release(cnum); ar.release(bound);
    ar.release(boff); ar.release(chat); ar.release(len); ar.release(scnt); ar.release(srp);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// ------------------------------------------------------------- l1 inverse
// d_i = a_ii + sign(a_ii) sum_{j != i} |a_ij| (ascending), 1/d_i.
__global__ void k_l1_inverse(int n, const int *rp, const int *ci, const double *v, double *dinv,
                             float *dinv32, int *errw) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double aii = 0.0, s = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; p++) {
        if (ci[p] == i) { aii = v[p]; continue; }
        s = s + fabs(v[p]);
    }
    double d = aii < 0.0 ? aii - s : aii + s;
    if (d == 0.0) { atomicOr(errw, ERRW_SINGULAR); dinv[i] = 0.0; if (dinv32) dinv32[i] = 0.f; return; }
    dinv[i] = 1.0 / d;
    if (dinv32) dinv32[i] = (float)dinv[i];
}

int l1_inverse(const DCSR &A, double *dinv, float *dinv32, int *errw, cudaStream_t s) {
    k_l1_inverse<<<GRID(A.n, 256), 256, 0, s>>>(A.n, A.rp, A.ci, A.v, dinv, dinv32, errw);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

__global__ void k_coarse_func(int n, const int *cf, const int *func, const int *prp, const int *pci,
                              int *cfunc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && cf[i] == 1) cfunc[pci[prp[i]]] = func[i];
}

void launch_coarse_func(const int *cf, const int *func, const DCSR &P, int *cfunc, int n,
                        cudaStream_t s) {
    k_coarse_func<<<GRID(n, 256), 256, 0, s>>>(n, cf, func, P.rp, P.ci, cfunc);
}

__global__ void k_iota_mod(int *f, int n, int nf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = nf > 1 ? i % nf : 0;
}

void launch_iota_mod(int *func, int n, int nf, cudaStream_t s) {
    k_iota_mod<<<GRID(n, 256), 256, 0, s>>>(func, n, nf);
}

// ------------------------------------------------------- coarsest inverse
// Gauss-Jordan with partial pivoting on [A | I].
__global__ void k_dense_fill(int n, const int *rp, const int *ci, const double *v, double *M) {
    int i = blockIdx.x;
    if (i >= n) return;
    for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) M[(long long)i * 2 * n + c] = (c - n == i) ? 1.0 : 0.0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int p = rp[i]; p < rp[i + 1]; p++) M[(long long)i * 2 * n + ci[p]] = v[p];
}

// Gauss-Jordan inverse with partial pivoting (the largest |entry| of the
// column, ties to the lower row), one launch per pivot column over at most
// one CTA per SM.  Step c reads the augmented matrix [A | I] from Min and
// writes Mout (the two alternate, so no CTA reads a row another CTA is
// writing): every CTA takes the pivot p from the per-CTA candidates of the
// previous step, stages the pivot row scaled by 1/a_pc in shared memory,
// and updates its share of the entries; row c takes the scaled pivot row,
// row p the eliminated old row c, and column c becomes e_c.  While it
// writes column c + 1 it also records its best pivot candidate there, so a
// step reads 16 bytes per CTA instead of the whole column.  The operations
// per entry are a division for the pivot row and a separately rounded
// multiply and subtract elsewhere.
static constexpr int GJ_THREADS = 512;

struct GJCand {
    double v;  // |entry|, -1 when the CTA saw no candidate
    int r;
    int pad;
};

__device__ __forceinline__ bool gj_better(double b, int ib, double a, int ia) {
    return b > a || (b == a && ib < ia);
}

// CTA-wide best candidate -> cand[blockIdx.x]
__device__ void gj_block_best(double best, int bi, GJCand *cand) {
    __shared__ double rv[GJ_THREADS / 32];
    __shared__ int ri[GJ_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        const double b = __shfl_down_sync(0xffffffffu, best, o);
        const int ib = __shfl_down_sync(0xffffffffu, bi, o);
        if (gj_better(b, ib, best, bi)) { best = b; bi = ib; }
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { rv[w] = best; ri[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = rv[0];
        int ib = ri[0];
        for (int q = 1; q < GJ_THREADS / 32; q++)
            if (gj_better(rv[q], ri[q], b, ib)) { b = rv[q]; ib = ri[q]; }
        cand[blockIdx.x].v = b;
        cand[blockIdx.x].r = ib;
    }
}

// candidates of column 0 (rows 0..n-1), in the layout the steps use
__global__ void __launch_bounds__(GJ_THREADS) k_gj_first(int n, const double *__restrict__ M,
                                                         GJCand *cand) {
    const long long ld = 2LL * n;
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int r = blockIdx.x * GJ_THREADS + threadIdx.x; r < n; r += gridDim.x * GJ_THREADS) {
        const double x = fabs(M[r * ld]);
        if (gj_better(x, r, best, bi)) { best = x; bi = r; }
    }
    gj_block_best(best, bi, cand);
}

__global__ void __launch_bounds__(GJ_THREADS) k_gj_step(int n, int c, const double *__restrict__ Min,
                                                        double *__restrict__ Mout,
                                                        const GJCand *__restrict__ cin, GJCand *cout,
                                                        int ncand, int *errw) {
    extern __shared__ double prow[];  // [2n] scaled pivot row, then [nr] row factors
    __shared__ int piv;
    pdl_wait();
    pdl_launch_dependents();
    const int tid = threadIdx.x;
    const long long ld = 2LL * n;
    if (tid < 32) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int q = tid; q < ncand; q += 32)
            if (gj_better(cin[q].v, cin[q].r, best, bi)) { best = cin[q].v; bi = cin[q].r; }
        for (int o = 16; o > 0; o >>= 1) {
            const double b = __shfl_down_sync(0xffffffffu, best, o);
            const int ib = __shfl_down_sync(0xffffffffu, bi, o);
            if (gj_better(b, ib, best, bi)) { best = b; bi = ib; }
        }
        if (tid == 0) piv = (bi >= c && bi < n) ? bi : c;
    }
    __syncthreads();
    const int p = piv;
    const double pv = Min[p * ld + c];
    if (pv == 0.0) {
        if (blockIdx.x == 0 && tid == 0) atomicOr(errw, ERRW_SINGULAR);
        return;
    }
    // rows r_k = blockIdx.x + k gridDim.x (k < nr) to this CTA, columns to threads;
    // after the swap row p holds the old row c
    const int nr = (n - 1 - (int)blockIdx.x) / (int)gridDim.x + 1;
    double *fk = prow + 2 * n;
    for (int t = tid; t < 2 * n; t += GJ_THREADS) prow[t] = Min[p * ld + t] / pv;
    for (int k = tid; k < nr; k += GJ_THREADS) {
        const int r = blockIdx.x + k * gridDim.x;
        fk[k] = Min[(long long)(r == p ? c : r) * ld + c];
    }
    __syncthreads();
    const int cn = c + 1;  // the next pivot column
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int t = tid; t < 2 * n; t += GJ_THREADS) {
        const double pt = prow[t];
#pragma unroll 4
        for (int k = 0; k < nr; k++) {
            const int r = blockIdx.x + k * gridDim.x;
            double out;
            if (r == c) out = pt;
            else if (t == c) out = 0.0;
            else out = Min[(long long)(r == p ? c : r) * ld + t] - fk[k] * pt;
            Mout[r * ld + t] = out;
            if (t == cn && r >= cn) {
                const double x = fabs(out);
                if (gj_better(x, r, best, bi)) { best = x; bi = r; }
            }
        }
    }
    if (cn < n) gj_block_best(best, bi, cout);
}

__global__ void k_gj_extract(int n, const double *M, double *inv) {
    const long long ld = 2LL * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), t = (int)(e % n);
        inv[e] = M[r * ld + n + t];
    }
}

// Blocked Gauss-Jordan (the same partial pivoting: the largest |entry| of
// the column among the rows not yet pivots, ties to the lower position), for
// n <= GJB_MAXN.  Panel k0..k0+nb-1 (nb <= 16):
//  * k_gjb_panel: one cluster of GJB_CL CTAs, one thread per row (CTA c owns
//    the rows that sit at positions c*R .. c*R+R-1 when the panel starts).
//    Each pivot step picks the pivot (each CTA reduces its rows' keys, |v|'s
//    IEEE bits compared as integers, and sends its best row to every CTA of
//    the cluster through distributed shared memory; one cluster barrier per
//    step) and eliminates the panel columns of every other row (LU-style: the
//    pivot rows of the panel are not reduced against each other here).  Out:
//    each row's multipliers f (F), the panel's pivot block as L\U with the
//    pivots' reciprocals (LG), the new row order (perm: position -> row of
//    the input) and the original row index of each position (orig).
//  * k_gjb_update: the rest of the step on the other columns.  With B the
//    panel columns of the pivot rows (B = L U), the Gauss-Jordan result is
//    new pivot rows = B^-1 (old pivot rows) = U^-1 W and every other row
//    old - f W, where W = L^-1 (old pivot rows).
// Right-half column bookkeeping: the right half of [A | I] keeps, for each
// position s < k0, the column of the inverse that belongs to the row placed
// at s (orig[s]); a column whose row has not been a pivot yet is still a unit
// vector and is not stored.  So each panel updates n columns (the left
// columns right of the panel and the right-half slots 0..k0+nb-1), not 2n-k0,
// and the slots of the panel's own pivots start as unit vectors (o = e_i).
// The inverse is read out at the end as inv[r][orig[s]] = Q[r][n+s].
static constexpr int GJB_NB = 16;
static constexpr int GJB_MAXN = 1024;
static constexpr int GJB_CL = 8;                   // CTAs per cluster (portable size)
static constexpr int GJB_MAXT = GJB_MAXN / GJB_CL;  // threads per CTA
static constexpr int GJB_STRIP = 8;                // most columns per update block
static constexpr int GJB_SMS = 152;                // update blocks (one per SM)
void launch_iota(int *a, int n, cudaStream_t s);

// 1/v by Newton's iteration for the reciprocal (r <- r + r (1 - m r), twice)
// on the mantissa m in [1, 2), from a single-precision seed with about 2^-22
// relative error, so two steps reach double precision; the exponent is put
// back with integer arithmetic.  A pivot step waits on this chain, and FP64
// latency is long here, so 4 dependent FMAs replace the longer division
// sequence.  Zero, subnormal and very large |v| take the division.
__device__ __forceinline__ double gj_recip(double v) {
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0 || ex > 2044) return 1.0 / v;
    const double m = __longlong_as_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const float mf = __int_as_float(0x3f800000 | (int)((b >> 29) & 0x7fffff));
    float rf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(mf));
    const int fb = __float_as_int(rf);
    double r = __longlong_as_double(((long long)(((fb >> 23) & 0xff) - 127 + 1023) << 52) |
                                    ((long long)(fb & 0x7fffff) << 29));
    double e = fma(-m, r, 1.0);
    r = fma(r, e, r);
    e = fma(-m, r, 1.0);
    r = fma(r, e, r);
    const long long rb = __double_as_longlong(r);
    const long long re = ((rb >> 52) & 0x7ff) - (ex - 1023);
    return __longlong_as_double((b & (long long)0x8000000000000000ULL) | (re << 52) | (rb & 0x000fffffffffffffLL));
}

// a CTA's candidate for one pivot step, as 64-bit words: the row's panel
// entries (its multipliers left of the step), the key (|v|'s bits), position
// | row << 32, the value and its reciprocal
enum { GJW_KEY = GJB_NB, GJW_POS, GJW_V, GJW_DINV, GJW_N };
struct GJRec {
    unsigned long long wd[GJW_N];
};

// warp argmax of the key (hi, lo), lowest position among equal keys; every
// lane gets the result and the winning lane's index
__device__ __forceinline__ int gjb_warp_best(unsigned &hi, unsigned &lo, unsigned &pos) {
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    const unsigned mp = __reduce_min_sync(0xffffffffu, (hi == mh && lo == ml) ? pos : 0xffffffffu);
    const unsigned bal = __ballot_sync(0xffffffffu, hi == mh && lo == ml && pos == mp);
    hi = mh;
    lo = ml;
    pos = mp;
    return __ffs(bal) - 1;
}

__device__ __forceinline__ unsigned gjb_cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// all threads of the cluster; release/acquire orders the records sent before it
__device__ __forceinline__ void gjb_cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void gjb_store_remote(const void *local, unsigned rank, unsigned long long v) {
    const unsigned l = (unsigned)__cvta_generic_to_shared(local);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(l), "r"(rank));
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(r), "l"(v) : "memory");
}

// P[i][tid] -= f e[i] for i = JJ+1 .. nb-1 (the pivot row's entries loaded
// first, so the loads and FMAs pipeline); returns the new entry JJ+1
template <int JJ>
__device__ __forceinline__ double gjb_elim(double f, const unsigned long long *e, double *P, int T, int tid, int nb) {
    double ev[GJB_NB], pv[GJB_NB];
#pragma unroll
    for (int i = JJ + 1; i < GJB_NB; i++) {
        ev[i] = __longlong_as_double((long long)e[i]);
        pv[i] = P[i * T + tid];
    }
    double r = 0.0;
#pragma unroll
    for (int i = JJ + 1; i < GJB_NB; i++)
        if (i < nb) {
            const double x = fma(-f, ev[i], pv[i]);
            P[i * T + tid] = x;
            if (i == JJ + 1) r = x;
        }
    return r;
}

__global__ void __launch_bounds__(GJB_MAXT) k_gjb_panel(int n, int k0, int nb, const double *__restrict__ Q,
                                                       long long ld, double *__restrict__ F, int *__restrict__ perm,
                                                       int *__restrict__ orig, double *__restrict__ LG, int *errw) {
    extern __shared__ double gjb_sm[];
    const int T = blockDim.x;
    double *P = gjb_sm;                              // [GJB_NB][T] this CTA's rows, panel columns
    GJRec *rec = (GJRec *)(P + (size_t)GJB_NB * T);  // [2][GJB_CL] candidates (by step parity)
    double *LU = (double *)(rec + 2 * GJB_CL);       // [GJB_NB][GJB_NB]
    double *dv = LU + GJB_NB * GJB_NB;               // [GJB_NB] pivot reciprocals
    unsigned *wk = (unsigned *)(dv + GJB_NB);        // [4][32] warp keys: hi, lo, pos, thread
    const unsigned cta = gjb_cluster_rank();
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = T >> 5;
    const int R = (n + GJB_CL - 1) / GJB_CL;
    const int g = (int)cta * R + tid;
    const bool valid = tid < R && g < n;
    int mypos = g, done = 0, og = 0;
    double cur = 0.0;  // this row's entry in the current pivot column
    if (valid) {
        for (int l = 0; l < GJB_NB; l++) P[l * T + tid] = l < nb ? Q[(long long)g * ld + k0 + l] : 0.0;
        cur = P[tid];
        og = orig[g];
    }
    for (int jj = 0; jj < nb; jj++) {
        const int j = k0 + jj, par = jj & 1;
        // this CTA's best candidate (rows at positions >= j not yet pivots)
        unsigned hi = 0u, lo = 0u, pos = 0xffffffffu;
        if (valid && !done && mypos >= j) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(cur) & 0x7fffffffffffffffULL;
            hi = (unsigned)(b >> 32);
            lo = (unsigned)b;
            pos = (unsigned)mypos;
        }
        const int wl = gjb_warp_best(hi, lo, pos);
        if (lane == 0) {
            wk[w] = hi;
            wk[32 + w] = lo;
            wk[64 + w] = pos;
            wk[96 + w] = (unsigned)(w * 32 + wl);
        }
        __syncthreads();
        if (w == 0) {
            hi = lane < nw ? wk[lane] : 0u;
            lo = lane < nw ? wk[32 + lane] : 0u;
            pos = lane < nw ? wk[64 + lane] : 0xffffffffu;
            const int bl = gjb_warp_best(hi, lo, pos);
            const int t = (int)__shfl_sync(0xffffffffu, lane < nw ? wk[96 + lane] : 0u, bl);
            const bool have = pos != 0xffffffffu;
            const double vv = have ? P[jj * T + t] : 0.0;
            const double di = (have && (hi | lo)) ? gj_recip(vv) : 0.0;
            unsigned long long word = 0ull;
            if (lane < GJB_NB) word = (have && lane < nb) ? (unsigned long long)__double_as_longlong(P[lane * T + t]) : 0ull;
            else if (lane == GJW_KEY) word = ((unsigned long long)hi << 32) | lo;
            else if (lane == GJW_POS)
                word = (unsigned long long)pos | ((unsigned long long)(unsigned)(have ? (int)cta * R + t : 0) << 32);
            else if (lane == GJW_V) word = (unsigned long long)__double_as_longlong(vv);
            else if (lane == GJW_DINV) word = (unsigned long long)__double_as_longlong(di);
            // one word per lane to every CTA's slot for this CTA (records of
            // step jj+2 reuse the slot only after the barrier of step jj+1,
            // which every CTA reaches after reading this step's records)
            if (lane < GJW_N) {
                const GJRec *mine = rec + par * GJB_CL + cta;
#pragma unroll
                for (int c = 0; c < GJB_CL; c++) gjb_store_remote(&mine->wd[lane], (unsigned)c, word);
            }
        }
        gjb_cluster_sync();
        // the cluster's pivot: the best CTA record (each warp on its own; every
        // thread of the cluster reaches the same decision)
        const GJRec *rs = rec + par * GJB_CL;
        unsigned bh = 0u, bo = 0u, bp = 0xffffffffu;
        if (lane < GJB_CL) {
            const unsigned long long k = rs[lane].wd[GJW_KEY];
            bh = (unsigned)(k >> 32);
            bo = (unsigned)k;
            bp = (unsigned)rs[lane].wd[GJW_POS];
        }
        const int cb = gjb_warp_best(bh, bo, bp);
        // a zero, infinite or NaN pivot (or no candidate row) ends the panel
        if (bp == 0xffffffffu || (bh | bo) == 0u || bh >= 0x7ff00000u) {
            if (cta == 0 && tid == 0) atomicOr(errw, ERRW_SINGULAR);
            return;
        }
        const GJRec &pr = rs[cb];
        const int prow = (int)(pr.wd[GJW_POS] >> 32);
        const double dinv = __longlong_as_double((long long)pr.wd[GJW_DINV]);
        if (tid < GJB_NB) LU[jj * GJB_NB + tid] = __longlong_as_double((long long)pr.wd[tid]);
        if (tid == GJB_NB) dv[jj] = dinv;
        // the pivot moves to position j, the row at j to the pivot's position
        if (mypos == j) mypos = (int)bp;
        else if (g == prow) mypos = j;
        if (g == prow) done = 1;
        if (valid && !done) {
            const double f = cur * dinv;
            P[jj * T + tid] = f;
            switch (jj) {
#define GJB_E(J) \
    case J: cur = gjb_elim<J>(f, pr.wd, P, T, tid, nb); break;
                GJB_E(0) GJB_E(1) GJB_E(2) GJB_E(3) GJB_E(4) GJB_E(5) GJB_E(6) GJB_E(7)
                GJB_E(8) GJB_E(9) GJB_E(10) GJB_E(11) GJB_E(12) GJB_E(13) GJB_E(14) GJB_E(15)
#undef GJB_E
                default: break;
            }
        }
    }
    __syncthreads();
    if (valid) {
        for (int l = 0; l < GJB_NB; l++) F[(long long)g * GJB_NB + l] = l < nb ? P[l * T + tid] : 0.0;
        perm[mypos] = g;
        orig[mypos] = og;  // every CTA read orig before the first barrier
    }
    if (cta == 0)
        for (int e = tid; e < GJB_NB * GJB_NB + GJB_NB; e += T)
            LG[e] = e < GJB_NB * GJB_NB ? LU[e] : dv[e - GJB_NB * GJB_NB];
}

// Block b takes a strip of NC active columns (left columns k0+nb..n-1, then
// right-half slots 0..k0+nb-1) and every row.  Per column, one half-warp:
// the pivot rows' old entries o (a unit vector for a slot of this panel's
// pivots), W = L^-1 o, the new pivot rows U^-1 W.  Then each other row:
// old - f . W, the strip's columns as independent FMA chains.
template <int NC>
__device__ __forceinline__ void gjb_rows(int n, int k0, int nb, int tid, const double *__restrict__ Qin,
                                        double *__restrict__ Qout, long long ld, const double *__restrict__ F,
                                        const int *__restrict__ perm, const int *colv, const double (*W)[GJB_NB]) {
    for (int pos = tid; pos < n; pos += 256) {
        if (pos >= k0 && pos < k0 + nb) continue;
        const int src = perm[pos];
        const double *fr = F + (long long)src * GJB_NB;
        double acc[NC];
#pragma unroll
        for (int q = 0; q < NC; q++) {
            const int col = colv[q];
            acc[q] = (col >= n && col - n >= k0) ? 0.0 : Qin[(long long)src * ld + col];
        }
#pragma unroll 4
        for (int l = 0; l < nb; l++) {
            const double fl = fr[l];
#pragma unroll
            for (int q = 0; q < NC; q++) acc[q] = fma(-fl, W[q][l], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < NC; q++) Qout[(long long)pos * ld + colv[q]] = acc[q];
    }
}

__global__ void __launch_bounds__(256) k_gjb_update(int n, int k0, int nb, const double *__restrict__ Qin,
                                                   double *__restrict__ Qout, long long ld,
                                                   const double *__restrict__ F, const int *__restrict__ perm,
                                                   const double *__restrict__ LG) {
    __shared__ double Ls[GJB_NB * GJB_NB + GJB_NB];
    __shared__ double W[GJB_STRIP][GJB_NB];
    __shared__ int pivr[GJB_NB], colv[GJB_STRIP];
    const int c0 = (int)(((long long)blockIdx.x * n) / gridDim.x);
    const int c1 = (int)(((long long)(blockIdx.x + 1) * n) / gridDim.x);
    const int nc = c1 - c0;
    const int tid = threadIdx.x, nl = n - k0 - nb;
    for (int e = tid; e < GJB_NB * GJB_NB + GJB_NB; e += 256) Ls[e] = LG[e];
    if (tid < GJB_NB) pivr[tid] = tid < nb ? perm[k0 + tid] : 0;
    if (tid < GJB_STRIP) {
        int col = 0;
        if (tid < nc) {
            const int cc = c0 + tid;
            col = cc < nl ? k0 + nb + cc : n + (cc - nl);
        }
        colv[tid] = col;
    }
    __syncthreads();
    const double *dvs = Ls + GJB_NB * GJB_NB;
    const int q = tid >> 4, i = tid & 15;
    const bool act = q < nc;
    const int col = act ? colv[q] : 0;
    const int slot = col - n - k0;  // >= 0: a slot of this panel's pivots
    double o = 0.0;
    if (act && i < nb) o = (col >= n && slot >= 0) ? (i == slot ? 1.0 : 0.0) : Qin[(long long)pivr[i] * ld + col];
    // every lane runs the same shuffles; lanes outside the strip carry zeros
    for (int l = 0; l < nb; l++) {
        const double wl = __shfl_sync(0xffffffffu, o, l, 16);
        if (i > l && i < nb) o = fma(-Ls[i * GJB_NB + l], wl, o);
    }
    if (act) W[q][i] = o;
    for (int l = nb - 1; l >= 0; l--) {
        if (i == l) o *= dvs[l];
        const double zl = __shfl_sync(0xffffffffu, o, l, 16);
        if (i < l) o = fma(-Ls[i * GJB_NB + l], zl, o);
    }
    if (act && i < nb) Qout[(long long)(k0 + i) * ld + col] = o;
    __syncthreads();
    switch (nc) {
#define GJB_R(C) \
    case C: gjb_rows<C>(n, k0, nb, tid, Qin, Qout, ld, F, perm, colv, W); break;
        GJB_R(1) GJB_R(2) GJB_R(3) GJB_R(4) GJB_R(5) GJB_R(6) GJB_R(7) GJB_R(8)
#undef GJB_R
        default: break;
    }
}

__global__ void k_gjb_extract(int n, const double *__restrict__ Q, const int *__restrict__ orig, double *inv) {
    const long long ld = 2LL * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / n), s = (int)(e % n);
        inv[(long long)r * n + orig[s]] = Q[r * ld + n + s];
    }
}

static int dense_inverse_blocked(int n, double *M, double *M2, double *inv, int *errw, cudaStream_t s,
                                 Arena &ar) {
    double *F = ar.alloc<double>((size_t)n * GJB_NB);
    double *LG = ar.alloc<double>(GJB_NB * GJB_NB + GJB_NB);
    int *perm = ar.alloc<int>(n);
    int *orig = ar.alloc<int>(n);
    if (!F || !LG || !perm || !orig) return ST_NOMEM;
    // perm and orig always hold row indexes inside the matrix, also after a
    // panel that meets a zero pivot and stops before writing them
    launch_iota(perm, n, s);
    launch_iota(orig, n, s);
    cudaMemsetAsync(F, 0, sizeof(double) * n * GJB_NB, s);
    cudaMemsetAsync(LG, 0, sizeof(double) * (GJB_NB * GJB_NB + GJB_NB), s);
    const int R = (n + GJB_CL - 1) / GJB_CL;
    const int T = ((R + 31) / 32) * 32;
    const size_t sh = (size_t)GJB_NB * T * sizeof(double) + 2 * GJB_CL * sizeof(GJRec) +
                      (GJB_NB * GJB_NB + GJB_NB) * sizeof(double) + 128 * sizeof(unsigned);
    if (cudaFuncSetAttribute(k_gjb_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh) != cudaSuccess)
        return ST_CUDA;
    const long long ld = 2LL * n;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(GJB_CL);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = sh;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = GJB_CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // update blocks: n columns in strips of at most GJB_STRIP (n <= 1024 over
    // min(n, GJB_SMS) blocks gives at most 7)
    const int ub = n < GJB_SMS ? n : GJB_SMS;
    double *a = M, *b = M2;
    for (int k0 = 0; k0 < n; k0 += GJB_NB) {
        const int nb = n - k0 < GJB_NB ? n - k0 : GJB_NB;
        if (cudaLaunchKernelEx(&cfg, k_gjb_panel, n, k0, nb, (const double *)a, ld, F, perm, orig, LG, errw) !=
            cudaSuccess)
            return ST_CUDA;
        k_gjb_update<<<ub, 256, 0, s>>>(n, k0, nb, a, b, ld, F, perm, LG);
        double *t = a;
        a = b;
        b = t;
    }
    k_gjb_extract<<<GRID((long long)n * n, 256) > 8192 ? 8192 : GRID((long long)n * n, 256), 256, 0, s>>>(n, a, orig,
                                                                                                        inv);
    cudaStreamSynchronize(s);
    ar.release(F);
    ar.release(LG);
    ar.release(perm);
    ar.release(orig);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

int dense_inverse(const DCSR &A, double *inv, int *errw, cudaStream_t s, Arena &ar) {
    const int n = A.n;
    if (n <= 0) return ST_OK;
    if (n <= GJB_MAXN) {
        double *M = ar.alloc<double>((size_t)n * 2 * n + 1);
        double *M2 = ar.alloc<double>((size_t)n * 2 * n + 1);
        if (!M || !M2) return ST_NOMEM;
        k_dense_fill<<<n, 256, 0, s>>>(n, A.rp, A.ci, A.v, M);
        const int rc = dense_inverse_blocked(n, M, M2, inv, errw, s, ar);
        ar.release(M);
        ar.release(M2);
        return rc;
    }
    double *M = ar.alloc<double>((size_t)n * 2 * n + 1);
    double *M2 = ar.alloc<double>((size_t)n * 2 * n + 1);
    const long long tot = 2LL * n * n;
    long long blocks = (tot + GJ_THREADS * 16 - 1) / (GJ_THREADS * 16);
    if (blocks > n) blocks = n;
    if (blocks > 152) blocks = 152;
    if (blocks < 1) blocks = 1;
    GJCand *cand = ar.alloc<GJCand>(2 * blocks);
    if (!M || !M2 || !cand) return ST_NOMEM;
    k_dense_fill<<<n, 256, 0, s>>>(n, A.rp, A.ci, A.v, M);
    k_gj_first<<<(unsigned)blocks, GJ_THREADS, 0, s>>>(n, M, cand);
    const size_t sh = (size_t)(2 * n + (n + blocks - 1) / blocks) * sizeof(double);
    if (sh > 48 * 1024 &&
        cudaFuncSetAttribute(k_gj_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh) != cudaSuccess)
        return ST_CUDA;
    double *a = M, *b = M2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(GJ_THREADS);
    cfg.dynamicSmemBytes = sh;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_on() ? 1 : 0;  // the next step's launch overlaps this one's tail
    for (int c = 0; c < n; c++) {
        GJCand *ci = cand + (c & 1) * blocks, *co = cand + ((c + 1) & 1) * blocks;
        cudaLaunchKernelEx(&cfg, k_gj_step, n, c, (const double *)a, b, (const GJCand *)ci, co, (int)blocks, errw);
        double *t = a;
        a = b;
        b = t;
    }
    k_gj_extract<<<GRID((long long)n * n, 256) > 8192 ? 8192 : GRID((long long)n * n, 256), 256, 0, s>>>(n, a, inv);
    cudaStreamSynchronize(s);
    ar.release(M);
    ar.release(M2);
    ar.release(cand);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

__global__ void k_cast_f32(const double *in, float *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

void launch_cast_f32(const double *in, float *out, long long n, cudaStream_t s) {
    unsigned g = GRID(n, 256);
    k_cast_f32<<<g > 8192 ? 8192 : g, 256, 0, s>>>(in, out, n);
}

// Positions of the scalar transpose's entries in the BSR value array: the
// scalar CSR of a BSR whose values are their own indices, transposed; so
// that new values reach A^T by one gather.
__global__ void k_iota_f64(double *v, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        v[i] = (double)i;
}

__global__ void k_f64_to_i32(const double *in, int *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (int)in[i];
}

int transpose_sources(int nb, int b, const int *brp, const int *bci, long long nnzb, int *src,
                      cudaStream_t s) {
    Arena tmp;
    const long long nv = nnzb * b * b;
    double *idx = tmp.alloc<double>(nv + 1);
    DCSR A;
    A.n = A.m = nb * b;
    A.nnz = (int)nv;
    A.rp = tmp.alloc<int>(A.n + 1);
    A.ci = tmp.alloc<int>(nv + 1);
    A.v = tmp.alloc<double>(nv + 1);
    if (!idx || !A.rp || !A.ci || !A.v) { tmp.free_all(); return ST_NOMEM; }
    unsigned g = GRID(nv, 256);
    k_iota_f64<<<g > 8192 ? 8192 : g, 256, 0, s>>>(idx, nv);
    launch_bsr_to_csr(nb, b, brp, bci, idx, A, s);
    DCSR T;
    if (transpose(A, T, s, tmp)) { tmp.free_all(); return ST_NOMEM; }
    k_f64_to_i32<<<g > 8192 ? 8192 : g, 256, 0, s>>>(T.v, src, nv);
    cudaStreamSynchronize(s);
    tmp.free_all();
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

__global__ void k_gather_f64(const int *src, const double *in, double *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = in[src[i]];
}

void launch_gather_f64(const int *src, const double *in, double *out, long long n, cudaStream_t s) {
    if (n <= 0) return;
    unsigned g = GRID(n, 256);
    k_gather_f64<<<g > 8192 ? 8192 : g, 256, 0, s>>>(src, in, out, n);
}

// flag |= 1 when a and b differ in any bit of their n values
__global__ void k_bits_differ(const unsigned long long *a, const unsigned long long *b, long long n,
                              int *flag) {
    int d = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        d |= a[i] != b[i];
    if (__syncthreads_or(d) && threadIdx.x == 0) atomicOr(flag, 1);
}

int same_bits(const double *a, const double *b, long long n, cudaStream_t s, Arena &ar) {
    int *flag = ar.alloc<int>(1);
    if (!flag) return -1;
    int h = 1;
    cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (n > 0) {
        unsigned g = GRID(n, 256);
        k_bits_differ<<<g > 8192 ? 8192 : g, 256, 0, s>>>((const unsigned long long *)a,
                                                         (const unsigned long long *)b, n, flag);
    }
    cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    ar.release(flag);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return h ? 0 : 1;
}

}  // namespace mgr

namespace mgr {

// ----------------------------------------------------------- SELL-C-sigma
// Rows are sorted by decreasing length (ties: ascending row) inside windows
// of SELL_WIN rows, then cut into slices of C = 32/G rows with G lanes per
// row.  Step t of a slice holds 32 consecutive entries: position r*G + g
// carries entry t*G + g of the slice's row r.
static const int SELL_WIN = 1024;

__global__ void k_sell_sort(int n, const int *rp, int *perm) {
    __shared__ unsigned long long key[SELL_WIN];
    const int w0 = blockIdx.x * SELL_WIN;
    for (int t = threadIdx.x; t < SELL_WIN; t += blockDim.x) {
        int row = w0 + t;
        if (row < n) {
            unsigned len = (unsigned)(rp[row + 1] - rp[row]);
            key[t] = ((unsigned long long)(0x7fffffffu - len) << 32) | (unsigned)row;
        } else {
            key[t] = ~0ULL;
        }
    }
    __syncthreads();
    // bitonic sort, ascending
    for (int k = 2; k <= SELL_WIN; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < SELL_WIN; t += blockDim.x) {
                int q = t ^ j;
                if (q > t) {
                    bool up = (t & k) == 0;
                    unsigned long long a = key[t], b = key[q];
                    if ((a > b) == up) { key[t] = b; key[q] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < SELL_WIN; t += blockDim.x) {
        unsigned long long k2 = key[t];
        perm[w0 + t] = k2 == ~0ULL ? -1 : (int)(k2 & 0xffffffffu);
    }
}

// longest row (the first row of each sorted window)
__global__ void k_sell_maxlen(int nwin, const int *rp, const int *perm, int *out) {
    int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwin) return;
    int row = perm[(long long)w * SELL_WIN];
    if (row >= 0) atomicMax(out, rp[row + 1] - rp[row]);
}

// slice width in steps (the longest row of the slice comes first); w32 =
// stored entries of the slice
__global__ void k_sell_width(int nsl, int G, const int *rp, const int *perm, int *slen, int *w32) {
    int s2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (s2 >= nsl) return;
    int row = perm[(long long)s2 * (32 / G)];
    int len = row >= 0 ? rp[row + 1] - rp[row] : 0;
    int w = (len + G - 1) / G;
    slen[s2] = w;
    w32[s2] = w * 32;
}

__global__ void k_sell_fill(int nsl, int G, const int *rp, const int *ci, const double *v, const float *v32,
                            const int *perm, const long long *sptr, const int *slen, int *sci,
                            double *sv, float *sv32) {
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= (long long)nsl * 32) return;
    int s2 = (int)(p >> 5), lane = (int)(p & 31);
    int r = lane / G, g = lane % G;
    int row = perm[(long long)s2 * (32 / G) + r];
    int len = row >= 0 ? rp[row + 1] - rp[row] : 0;
    int base = row >= 0 ? rp[row] : 0;
    int padc = len > 0 ? ci[base + len - 1] : 0;
    long long o = sptr[s2] + lane;
    for (int t = 0; t < slen[s2]; t++, o += 32) {
        int k = t * G + g;
        if (k < len) {
            sci[o] = ci[base + k];
            if (sv) sv[o] = v[base + k];
            if (sv32) sv32[o] = v32[base + k];
        } else {
            sci[o] = padc;
            if (sv) sv[o] = 0.0;
            if (sv32) sv32[o] = 0.0f;
        }
    }
}

// Lanes per row (rules fitted to timings of the solve-phase kernels on
// GB300 over the AMG levels of a 1M-unknown system, and of the 2M-unknown
// compositional system whose pressure block has a few well-coupled rows
// seven times longer than the rest).  A lane's chain should hold <= 24
// entries on average and, while lanes keep >= 4 entries, <= 128 in the
// longest row; a matrix with fewer than 64 warps per SM spreads rows
// over more lanes while chains keep >= 16 entries; and a matrix too small
// to give every SM 8 warps is bound by the dependent load-then-gather
// rounds of its longest row, which are cut to <= 8 entries.
static int sell_lanes(double avg, int maxlen, long long n) {
    int G = 1;
    while (G < 32) {
        const double steps = avg / G, longest = (double)maxlen / G;
        const long long warps = n * G / 32;
        const bool more = steps > 24.0 || (steps >= 4.0 && longest > 128.0) ||
                          (warps < 152LL * 64 && steps >= 16.0) || (warps < 152LL * 8 && longest > 8.0);
        if (!more) break;
        G *= 2;
    }
    return G;
}

int build_sell(DCSR &M, cudaStream_t s, Arena &ar, const SellTune *tn) {
    if (M.n <= 0) return ST_OK;
    M.sched = 0;
    const int nwin = (M.n + SELL_WIN - 1) / SELL_WIN;
    M.perm = ar.alloc<int>((size_t)nwin * SELL_WIN);
    int *dmax = ar.alloc<int>(1);
    if (!M.perm || !dmax) return ST_NOMEM;
    k_sell_sort<<<nwin, 512, 0, s>>>(M.n, M.rp, M.perm);
    cudaMemsetAsync(dmax, 0, sizeof(int), s);
    k_sell_maxlen<<<(nwin + 255) / 256, 256, 0, s>>>(nwin, M.rp, M.perm, dmax);
    int maxlen = 0;
    if (cudaMemcpyAsync(&maxlen, dmax, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return ST_CUDA;
    ar.release(dmax);
    const int G = sell_lanes((double)M.nnz / M.n, maxlen, M.n);
    const int nsl = nwin * (SELL_WIN / (32 / G));
    M.sg = G;
    M.nsl = nsl;
    M.slen = ar.alloc<int>(nsl + 1);
    M.sptr = ar.alloc<long long>(nsl + 1);
    int *w32 = ar.alloc<int>(nsl + 1);
    if (!M.slen || !M.sptr || !w32) return ST_NOMEM;
    k_sell_width<<<(nsl + 255) / 256, 256, 0, s>>>(nsl, G, M.rp, M.perm, M.slen, w32);
    long long tot = 0;
    int rc = scan_exclusive_ll(w32, M.sptr, nsl, s, ar, &tot);
    ar.release(w32);
    if (rc) return rc;
    M.sell_stored = tot;
    M.sci = ar.alloc<int>(tot + 1);
    M.sv = M.v ? ar.alloc<double>(tot + 1) : nullptr;
    M.sv32 = M.v32 ? ar.alloc<float>(tot + 1) : nullptr;
    if (!M.sci || (M.v && !M.sv) || (M.v32 && !M.sv32)) return ST_NOMEM;
    refresh_sell(M, s);
    if (cudaGetLastError() != cudaSuccess) return ST_CUDA;
    return tn ? sell_tune(M, *tn, s, ar) : ST_OK;
}

void refresh_sell(DCSR &M, cudaStream_t s) {
    if (!M.sptr) return;
    long long np = (long long)M.nsl * 32;
    k_sell_fill<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(M.nsl, M.sg, M.rp, M.ci, M.v, M.v32, M.perm,
                                                          M.sptr, M.slen, M.sci, M.sv, M.sv32);
}

}  // namespace mgr
