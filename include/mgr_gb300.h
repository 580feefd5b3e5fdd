/*
 * mgr_gb300.h -- C ABI of the GB300 (sm_103a) multigrid-reduction solver.
 *
 * The library solves the block linear systems A x = b of Eq. 1 (arXiv
 * 2101.11649, Sec. 1) with flexible GMRES(m), right-preconditioned by one
 * multilevel MGR V-cycle (Algorithm 1, Sec. 3) whose final coarse block is
 * solved by one algebraic-multigrid V(1,1) cycle (Sec. 5.1).  Every step of
 * setup and solve runs in CUDA kernels on one GPU.
 *
 * Conventions shared by all entry points:
 *   - Pointers named "device" are CUDA device (or managed) addresses on the
 *     handle's device; "host" pointers are ordinary host memory.
 *   - Vectors are FP64, length n = nb * b, in the caller's dof order.
 *   - All work is enqueued on the handle's stream; entry points that return
 *     scalars (solve statistics) synchronise that stream before returning.
 *   - No entry point throws or aborts.  Each returns an mgr_status; the
 *     message of the last failure is available from mgr_last_error().
 *   - The caller keeps ownership of everything it passes in.  The handle
 *     owns its copies of the matrix and the whole hierarchy until mgr_free.
 */
#ifndef MGR_GB300_H
#define MGR_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MGR_OK = 0,
    MGR_ERR_INVALID = 1,       /* malformed input (sizes, pattern, labels, NaN) */
    MGR_ERR_NOMEM = 2,         /* device allocation failed */
    MGR_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    MGR_ERR_SINGULAR = 4,      /* a zero pivot in D_FF, a block inverse or the coarsest solve */
    MGR_ERR_NOT_CONVERGED = 5, /* maxit reached; x holds the last iterate */
    MGR_ERR_TIMEOUT = 6,       /* a bounded device wait ran out */
    MGR_ERR_UNSUPPORTED = 7    /* valid request outside what the library supports */
} mgr_status;

typedef struct mgr_ctx *mgr_handle;

/*
 * Square block-CSR matrix (the block system of Eq. 1).  b in 1..4; block
 * row I holds blocks row_ptr[I]..row_ptr[I+1]-1 with strictly ascending
 * col_idx; each block is b*b FP64 values, row-major; every block row must
 * contain its diagonal block.  on_device != 0 means the three arrays are
 * device pointers, else host pointers.  They are copied by mgr_setup.
 */
typedef struct {
    int32_t nb, b;
    int64_t nnzb;
    const int32_t *row_ptr, *col_idx;
    const double *val;
    int32_t on_device;
} mgr_bsr;

/*
 * MGR C/F labels (the physics-based reduction order of Sec. 3-4).
 * dof_level[i] (host, int8, length n) is the level at which scalar dof i is
 * an F-point (0..num_levels-1); num_levels means that dof survives to the
 * final coarse block solved by AMG.  Level l's F set is {dof_level == l}
 * and its C set is {dof_level > l}, both in ascending dof order; the coarse
 * numbering follows ascending dof order.
 */
typedef struct {
    int32_t num_levels;
    const int8_t *dof_level;
} mgr_labels;

enum { MGR_RELAX_JACOBI = 0, MGR_RELAX_L1_JACOBI = 1, MGR_RELAX_BLOCK_JACOBI = 2, MGR_RELAX_AMG = 3 };
enum { MGR_RESTRICT_INJECTION = 0, MGR_RESTRICT_JACOBI = 1 };
enum { MGR_PREC_FP64 = 0, MGR_PREC_FP32 = 1 };
#define MGR_MAX_LEVELS 8

/*
 * Options.  Per MGR level l: F-relaxation type (D_FF of Eq. 4 is the same
 * matrix: its diagonal, its l1-row-scaled diagonal, or its per-block-row
 * F-by-F blocks), number of sweeps (from z = 0) and weight omega.
 * MGR_RELAX_AMG (MGR_U of Sec. 4.3): each sweep applies one AMG V(1,1)
 * cycle on A_FF, from an AMG hierarchy of A_FF built at setup with the AMG
 * parameters below and relax_functions[l] functions of the unknown approach
 * (function of an F dof = its F index mod relax_functions[l]); the
 * interpolation uses D_FF = diag(A_FF).  A sweep computes
 * z_F += omega * B (v_F - A_FF z_F) with B the V-cycle.  Batched solves take
 * it with one sweep.
 * restrict_type[l]: MGR_RESTRICT_INJECTION (R~ = [0, I], the default) or
 * MGR_RESTRICT_JACOBI (R~ = [-A_CF D^{-1}, I] of Eq. 5, the transpose of
 * P~ for symmetric A): the coarse operator becomes the triple product
 * R~ A P~ and the cycle restricts v_C - A_CF z_F + Z (v_F - A_FF z_F),
 * Z = -A_CF D^{-1}.  It needs a diagonal D (not block-Jacobi:
 * MGR_ERR_UNSUPPORTED); batched solves take it too.
 * spin_limit: polls before a grid-barrier wait of the fused AMG tail gives
 * up (0: the default, about half a second); a test knob that makes the wait
 * run out on purpose, so that the MGR_ERR_TIMEOUT path can be exercised
 * without a GPU fault.
 * AMG: strength threshold theta, level and coarse-size limits, max
 * interpolation entries per row (0 = no truncation), number of functions
 * of the unknown approach (function of a coarse-block dof = its index mod
 * num_functions).  precision selects FP64 or FP32 storage and arithmetic of
 * the whole V-cycle (FGMRES, residuals and the coarsest dense solve stay
 * FP64).  restart = FGMRES m.  use_graphs != 0 replays the per-iteration
 * kernel sequence from captured CUDA graphs.  amg_tail_nnz: the AMG levels
 * from the first level k >= 1 whose operator has at most this many nonzeros
 * down to the coarsest run as one cooperative launch over the GPU, the steps
 * separated by grid-wide barriers (same arithmetic, bitwise the same result
 * as one launch per step); 0 (the default) runs every step as its own
 * launch.  Devices without cooperative launches ignore it.  A barrier wait
 * that runs out (it should not) makes mgr_solve, mgr_apply and
 * mgr_apply_transpose return MGR_ERR_TIMEOUT; with the tail on, the two
 * apply calls synchronise the stream to read its error word, and a solve
 * stops at the first step whose tail gave up, leaving x as it was at the
 * last restart.
 */
typedef struct {
    int32_t relax_type[MGR_MAX_LEVELS];
    int32_t relax_sweeps[MGR_MAX_LEVELS];
    double relax_weight[MGR_MAX_LEVELS];
    double amg_theta;
    int32_t amg_max_levels, amg_max_coarse, amg_pmax, amg_num_functions;
    int32_t precision;
    int32_t restart;
    int32_t use_graphs;
    int32_t amg_tail_nnz;
    int32_t relax_functions[MGR_MAX_LEVELS];
    int32_t restrict_type[MGR_MAX_LEVELS];
    int32_t spin_limit;
} mgr_options;

/* Solve report.  level_rows/level_nnz list the MGR levels, then the AMG levels. */
typedef struct {
    int32_t iterations;        /* preconditioner applications */
    double rel_residual;       /* true ||b - A x|| / ||b|| at exit */
    double setup_ms, solve_ms;
    int32_t mgr_levels, amg_levels;
    int64_t level_rows[40], level_nnz[40];
    double operator_complexity;
    int32_t reorth_steps;      /* Arnoldi steps that needed the second Gram-Schmidt pass */
} mgr_solve_info;

/* Defaults: Jacobi, 1 sweep, omega 1 on every level; theta 0.25, 25 AMG
 * levels, coarsest <= 1024 rows, P_max 4, 1 function; FP64; m = 30; graphs on;
 * no fused AMG tail; 1 function in every F-relaxation AMG hierarchy;
 * injection restriction on every level; the default barrier wait limit. */
void mgr_options_default(mgr_options *opt);

/*
 * Build the MGR hierarchy (Sec. 3): per level, the F/C split, D_FF^{-1},
 * W = -D_FF^{-1} A_FC and the coarse operator A_{l+1} = A_CC + A_CF W (the
 * product R~ A P~ of Eq. 4 operators); then the AMG hierarchy of the final
 * block (strength, PMIS, extended+i, Galerkin P^T A P, dense inverse of the
 * coarsest grid).  stream: a cudaStream_t for all of the handle's work; NULL
 * makes the handle create its own blocking stream, which the legacy default
 * stream orders against implicitly.
 * Errors: INVALID (pattern/labels/sizes, an empty F or C set), SINGULAR
 * (a zero diagonal or singular block in D_FF), NOMEM, CUDA.
 */
mgr_status mgr_setup(const mgr_bsr *A, const mgr_labels *cf, const mgr_options *opt,
                     void *stream, mgr_handle *out);

/* z = M^{-1} v: one MGR V-cycle (Algorithm 1 without global relaxation).
 * device v, z.  TIMEOUT when a fused AMG tail (amg_tail_nnz) gave up. */
mgr_status mgr_apply(mgr_handle h, const double *v, double *z);

/* z = M^{-T} v: the exact transpose of mgr_apply's operator. device v, z. */
mgr_status mgr_apply_transpose(mgr_handle h, const double *v, double *z);

/* y = A x with the handle's copy of A (device x, y). */
mgr_status mgr_spmv(mgr_handle h, const double *x, double *y);

/*
 * Right-preconditioned flexible GMRES(m) (Sec. 5.1) on A x = b from the x
 * given (device b, x).  Stops when the true residual ||b - A x||_2 <=
 * rtol ||b||_2 (NOT_CONVERGED after maxit preconditioner applications, with
 * x the last iterate).  info may be NULL.
 */
mgr_status mgr_solve(mgr_handle h, const double *b, double *x, double rtol, int32_t maxit,
                     mgr_solve_info *info);

/* The same on A^T lambda = g with the transposed cycle (adjoint solve). */
mgr_status mgr_solve_transpose(mgr_handle h, const double *g, double *lam, double rtol,
                               int32_t maxit, mgr_solve_info *info);

/* Replace the stored values of A (same pattern; val as in mgr_bsr, host or
 * device) in the operator that mgr_spmv, mgr_solve and mgr_solve_transpose
 * apply, keeping the MGR/AMG hierarchy built by mgr_setup as the
 * preconditioner: the reuse of a hierarchy across Newton steps (Sec. 5.3).
 * Synchronises the stream.  INVALID on a non-finite value (the handle is
 * left unchanged). */
mgr_status mgr_update_values(mgr_handle h, const double *val, int32_t on_device);

/* Replace the values of A (same pattern, as mgr_update_values) and rebuild
 * the hierarchy numerically from them: every MGR level (D_FF, W, Z, coarse
 * operators) and the final coarse block's AMG hierarchy, while every AMG
 * F-relaxation hierarchy built before is kept as it is (the setup reuse of
 * Sec. 4.3: the mechanics block of MGR_U is fixed across Newton steps, so its
 * AMG hierarchy is reused; when A_FF did change, the kept hierarchy is the
 * one built from the old A_FF, and the level's own residuals use the new
 * A_FF).  Labels and options are those of mgr_setup.  Synchronises the
 * stream.  INVALID on a non-finite value; UNSUPPORTED for a handle of a
 * batch; on any other failure the handle reports INVALID from then on. */
mgr_status mgr_refresh(mgr_handle h, const double *val, int32_t on_device);

/* dA_val[p*b*b + r*b + c] = -lam[I*b + r] * x[J*b + c] for block p = (I, J):
 * the gradient of a scalar loss with respect to the stored values of A when
 * lam solves A^T lam = dL/dx.  device pointers. */
mgr_status mgr_grad_values(mgr_handle h, const double *lam, const double *x, double *dA_val);

/*
 * Standalone block-CSR product y = alpha A x + beta y on device arrays
 * (b in 1..4) without a handle.  stream as in mgr_setup.
 */
mgr_status mgr_bsr_spmv(int32_t nb, int32_t b, const int32_t *row_ptr, const int32_t *col_idx,
                        const double *val, const double *x, double *y, double alpha, double beta,
                        void *stream);

/*
 * Residual r = bvec - A x and its norm without any allocation (the paper has
 * no counterpart; this serves callers that cannot call cudaMalloc: plug-ins
 * whose host application owns all device memory through its own pool and
 * forbids allocations behind its back, and real-time loops that must never
 * enter the allocator, whose calls can block or fail at any moment).  A is
 * a block-CSR matrix on the device (as mgr_bsr_spmv);
 * x, bvec, r (length n = nb*b) and norm_out (one double, = ||r||_2) are
 * caller-owned device memory.  The reduction's only scratch is a file-scope
 * static device array of MGR_NOALLOC_MAX_BLOCKS partial sums plus a ticket
 * (32 KiB per GPU, held until the process exits); one partial covers 4096
 * entries, so n may be at most 16,777,216 (MGR_ERR_UNSUPPORTED beyond).
 * The first call on a device looks up the array's device address (make it
 * before any stream capture).  Calls share the array: calls that overlap on
 * the GPU race.  Enqueued on stream; returns without synchronising.
 */
#define MGR_NOALLOC_MAX_BLOCKS 4096
mgr_status mgr_residual_norm_noalloc(int32_t nb, int32_t b, const int32_t *row_ptr,
                                     const int32_t *col_idx, const double *val, const double *x,
                                     const double *bvec, double *r, double *norm_out, void *stream);

/* --------------------------------------------------------------- batched
 * Many systems of uneven sizes (different time steps or models) solved
 * together.  Each system keeps its own hierarchy, and every kernel class of
 * the V-cycle, the outer product and the Arnoldi reductions runs as one
 * launch over all systems (a job table of per-system operands; per-system
 * convergence flags drop finished systems).  The sparse products run over
 * the members' SELL-C-sigma copies or the chunk engine, whichever the
 * autotuner timed faster at setup for that kernel class and level.  An AMG
 * F-relaxation level (MGR_U) runs its members' F hierarchies as one
 * level-synchronous V-cycle; the restriction of Eq. 5 adds its two products.
 * All systems need the same block size, MGR level count and options, at
 * least one MGR level, and one F-relaxation sweep (MGR_ERR_UNSUPPORTED
 * otherwise).
 */
typedef struct mgr_batch_ctx *mgr_batch;

/* A[nsys], cf[nsys] as for mgr_setup; stream as for mgr_setup. */
mgr_status mgr_setup_batched(int32_t nsys, const mgr_bsr *A, const mgr_labels *cf,
                             const mgr_options *opt, void *stream, mgr_batch *out);

/* FGMRES(m) for every system: b[i], x[i] device vectors (x[i] in: x0, out: x);
 * info[nsys] may be NULL.  NOT_CONVERGED if any system hit maxit. */
mgr_status mgr_solve_batched(mgr_batch h, const double *const *b, double *const *x, double rtol,
                             int32_t maxit, mgr_solve_info *info);

/* The single-system handle of system i (owned by the batch): for
 * mgr_solve_transpose, mgr_grad_values and inspection. */
mgr_status mgr_batch_handle(mgr_batch h, int32_t i, mgr_handle *out);

void mgr_free_batched(mgr_batch h);

/* Release the handle and everything it owns.  NULL is a no-op. */
void mgr_free(mgr_handle h);

/* Message of the last failure on h (thread-local last failure when h is NULL). */
const char *mgr_last_error(mgr_handle h);

/* -------------------------------------------------- hierarchy inspection
 * For parity tests and tooling.  which: 0 = the level matrix; for MGR
 * levels 1 = A_FF, 2 = A_FC, 3 = A_CF, 4 = W, 5 = Z (restriction of Eq. 5
 * only); for AMG levels 1 = P.
 * amg = 0 selects MGR level `level` (level == mgr levels is the final coarse
 * block), amg = 1 AMG level `level` of the final coarse block's hierarchy,
 * amg = 2 + l AMG level `level` of MGR level l's AMG F-relaxation.  dims (host int32[3]) receives rows,
 * cols, nnz; when rp/ci/v (host) are non-NULL they receive the CSR arrays
 * (rp: rows+1, ci and v: nnz).  INVALID if the matrix does not exist.
 */
mgr_status mgr_get_matrix(mgr_handle h, int32_t amg, int32_t level, int32_t which, int32_t *dims,
                          int32_t *rp, int32_t *ci, double *v);

/* AMG level C/F marks (host int32[rows]: +1 C, -1 F) of the final coarse
 * block's hierarchy. */
mgr_status mgr_get_cf(mgr_handle h, int32_t level, int32_t *cf);

/* The same for hierarchy amg: 1 = the final coarse block's, 2 + l = the AMG
 * F-relaxation hierarchy of MGR level l.  INVALID if there is none or the
 * level has no C/F split (the coarsest). */
mgr_status mgr_get_amg_cf(mgr_handle h, int32_t amg, int32_t level, int32_t *cf);

/* AMG levels of hierarchy amg (numbered as above); 0 if it does not exist. */
int32_t mgr_get_amg_levels(mgr_handle h, int32_t amg);

/* MGR level D_FF^{-1}: per F point 4 slots (its row of the block inverse)
 * and its block size (host double[nF*4], int32[nF]). */
mgr_status mgr_get_dinv(mgr_handle h, int32_t level, double *dinv, int32_t *gsize);

/* Level counts: out[0] = MGR levels, out[1] = AMG levels, out[2] = n. */
mgr_status mgr_get_info(mgr_handle h, int32_t *out);

/* Structure check of the built hierarchy, in place of a memory checker:
 * every index array the solve phase reads through (CSR row offsets and
 * columns, SELL-C-sigma slice offsets, widths, row maps and columns, the
 * C/F index maps, D_FF block descriptors) is checked on the device against
 * the size of the array it indexes, and consecutive operators against each
 * other's shapes.  *violations (host) receives the number of violations
 * (0 for a sound hierarchy).  Synchronises the stream. */
mgr_status mgr_check_hierarchy(mgr_handle h, int64_t *violations);

/* Relative residuals of the handle's last solve: out[0] = ||b - A x0|| / ||b||,
 * out[i] = the Arnoldi estimate |g_{i}| / ||b|| after preconditioner
 * application i (restarts included), as the oracle's history.  Copies at
 * most cap values to out (host; may be NULL) and returns the count
 * (iterations + 1). */
int32_t mgr_solve_history(mgr_handle h, double *out, int32_t cap);

/* ------------------------------------------------------- instrumentation
 * Kernel launches this library has made (all handles, solve-phase kernels,
 * counted on the host when enqueued).  */
int64_t mgr_launch_count(void);

/* Enable (on != 0) or disable per-kernel-class timing on h and reset the
 * table.  While on, every solve-phase launch is bracketed by a CUDA event
 * pair on the handle's stream, tagged with the kernel class (and level) and
 * the algorithmic bytes one launch moves (each operand read or written once).  */
mgr_status mgr_profile(mgr_handle h, int32_t on);

/* Number of kernel classes recorded so far (synchronises the stream). */
int32_t mgr_profile_entries(mgr_handle h);

/* Entry i: name (host buffer of name_cap bytes), summed device time, number
 * of launches, and per launch (averaged over launches) the algorithmic bytes
 * and FP64 fused multiply-adds.  */
mgr_status mgr_profile_entry(mgr_handle h, int32_t i, char *name, int32_t name_cap,
                             double *total_ms, int64_t *launches, double *bytes_per_launch,
                             double *fp64_fma_per_launch);

/* Measured FP64 fused-multiply-add rate of the current device (FMA per
 * second, best of reps timed launches after one warm-up, on stream): every
 * thread of a full-occupancy grid runs independent FMA chains in registers.
 * Instrumentation, not part of the method: the roofline denominator of the
 * FP64 products, which issue one FMA per stored entry.  Synchronises. */
mgr_status mgr_measure_fp64_fma(void *stream, int32_t reps, double *fma_per_s);

#ifdef __cplusplus
}
#endif

#endif /* MGR_GB300_H */
