// Structure checks of a built hierarchy (mgr_check_hierarchy): every index
// array the solve-phase kernels read through is checked against the size of
// the array it indexes.  The kernels address memory only through these
// arrays and through loop bounds derived from the matrix sizes, so a clean
// check means that no solve-phase gather, scatter or row walk leaves its
// array.  Each check adds its violations to a device counter; nothing is
// written outside the counter.
#include <cuda_runtime.h>

#include "common.cuh"

namespace mgr {

#define CGRID(n) (unsigned)((((long long)(n) + 255) / 256) > 8192 ? 8192 : ((((long long)(n) + 255) / 256) < 1 ? 1 : (((long long)(n) + 255) / 256)))

// CSR: rp[0] = 0, rp non-decreasing, rp[n] = nnz; 0 <= ci < m, ascending in a row
__global__ void k_chk_csr(int n, int m, int nnz, const int *rp, const int *ci,
                          unsigned long long *bad) {
    unsigned long long b = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int a = rp[i], e = rp[i + 1];
        if (i == 0 && a != 0) b++;
        if (i == n - 1 && e != nnz) b++;
        if (a > e || a < 0 || e > nnz) { b++; continue; }
        for (int p = a; p < e; p++) {
            const int j = ci[p];
            if (j < 0 || j >= m) b++;
            if (p > a && j <= ci[p - 1]) b++;
        }
    }
    if (b) atomicAdd(bad, b);
}

// SELL-C-sigma: sptr[s+1] - sptr[s] = 32 slen[s] and sptr[nsl] = stored;
// every slice row is -1 or a row < n, seen once; a slice is at least as wide
// as its rows need (ceil(len / G) steps)
__global__ void k_chk_sell_slices(int n, int nsl, int G, const int *rp, const long long *sptr,
                                  const int *slen, const int *perm, long long stored, int *seen,
                                  unsigned long long *bad) {
    const int C = 32 / G;
    unsigned long long b = 0;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nsl;
         s += (long long)gridDim.x * blockDim.x) {
        if (s == 0 && sptr[0] != 0) b++;
        if (s == nsl - 1 && sptr[nsl] != stored) b++;
        const int L = slen[s];
        if (L < 0 || sptr[s + 1] - sptr[s] != 32LL * L) b++;
        for (int r = 0; r < C; r++) {
            const int row = perm[s * C + r];
            if (row < -1 || row >= n) { b++; continue; }
            if (row < 0) continue;
            atomicAdd(seen + row, 1);
            const int len = rp[row + 1] - rp[row];
            if ((long long)L * G < len) b++;
        }
    }
    if (b) atomicAdd(bad, b);
}

__global__ void k_chk_once(int n, const int *seen, unsigned long long *bad) {
    unsigned long long b = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b += seen[i] != 1;
    if (b) atomicAdd(bad, b);
}

__global__ void k_chk_range(const int *a, long long len, int lo, int hi, int increasing,
                            unsigned long long *bad) {
    unsigned long long b = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = a[i];
        if (x < lo || x >= hi) b++;
        if (increasing && i > 0 && x <= a[i - 1]) b++;
    }
    if (b) atomicAdd(bad, b);
}

__global__ void k_chk_mark(const int *a, long long len, int hi, int *seen) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x)
        if (a[i] >= 0 && a[i] < hi) atomicAdd(seen + a[i], 1);
}

__global__ void k_chk_add(unsigned long long *bad, unsigned long long v) { atomicAdd(bad, v); }

// D_FF blocks: 1 <= gsize <= 4, gstart <= f < gstart + gsize <= nF
__global__ void k_chk_groups(int nF, const int *gstart, const int *gsize, unsigned long long *bad) {
    unsigned long long b = 0;
    for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < nF;
         f += (long long)gridDim.x * blockDim.x) {
        const int g = gstart[f], k = gsize[f];
        if (k < 1 || k > 4 || g < 0 || g > f || f >= g + k || g + k > nF) b++;
    }
    if (b) atomicAdd(bad, b);
}

int check_add(unsigned long long *bad, unsigned long long v, cudaStream_t s) {
    if (v) k_chk_add<<<1, 1, 0, s>>>(bad, v);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

int check_iota(const int *a, int n, unsigned long long *bad, cudaStream_t s) {
    if (n > 0) k_chk_range<<<CGRID(n), 256, 0, s>>>(a, n, 0, n, 1, bad);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

int check_csr(const DCSR &M, unsigned long long *bad, cudaStream_t s, Arena &ar) {
    if (M.n <= 0) return ST_OK;
    k_chk_csr<<<CGRID(M.n), 256, 0, s>>>(M.n, M.m, M.nnz, M.rp, M.ci, bad);
    if (!M.sptr) return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
    int *seen = ar.alloc<int>(M.n + 1);
    if (!seen) return ST_NOMEM;
    cudaMemsetAsync(seen, 0, sizeof(int) * M.n, s);
    k_chk_sell_slices<<<CGRID(M.nsl), 256, 0, s>>>(M.n, M.nsl, M.sg, M.rp, M.sptr, M.slen, M.perm,
                                                  M.sell_stored, seen, bad);
    k_chk_once<<<CGRID(M.n), 256, 0, s>>>(M.n, seen, bad);
    k_chk_range<<<CGRID(M.sell_stored), 256, 0, s>>>(M.sci, M.sell_stored, 0, M.m > 0 ? M.m : 1, 0, bad);
    cudaStreamSynchronize(s);
    ar.release(seen);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

int check_split(int n, const int *fidx, int nF, const int *cidx, int nC, const int *gstart,
                const int *gsize, unsigned long long *bad, cudaStream_t s, Arena &ar) {
    if (nF + nC != n) {
        k_chk_add<<<1, 1, 0, s>>>(bad, 1ull);
        return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
    }
    int *seen = ar.alloc<int>(n + 1);
    if (!seen) return ST_NOMEM;
    cudaMemsetAsync(seen, 0, sizeof(int) * n, s);
    k_chk_range<<<CGRID(nF), 256, 0, s>>>(fidx, nF, 0, n, 1, bad);
    k_chk_range<<<CGRID(nC), 256, 0, s>>>(cidx, nC, 0, n, 1, bad);
    k_chk_mark<<<CGRID(nF), 256, 0, s>>>(fidx, nF, n, seen);
    k_chk_mark<<<CGRID(nC), 256, 0, s>>>(cidx, nC, n, seen);
    k_chk_once<<<CGRID(n), 256, 0, s>>>(n, seen, bad);
    k_chk_groups<<<CGRID(nF), 256, 0, s>>>(nF, gstart, gsize, bad);
    cudaStreamSynchronize(s);
    ar.release(seen);
    return cudaGetLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

}  // namespace mgr
