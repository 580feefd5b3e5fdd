"""ctypes wrapper of the C oracle (``mgr_oracle.c``).  TEST INFRASTRUCTURE ONLY.

Only tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  It never touches the CUDA library and the CUDA library never calls
it.  Building it is plain ``gcc -O2 -ffp-contract=off -fopenmp`` (no fused
multiply-add, no fast-math), so setup arithmetic follows the C source's
stated operation order exactly; the solve phase's independent loops run on
all cores of the process's affinity set (``set_threads`` changes that),
with results that do not depend on the thread count.  Without OpenMP the
same source builds single-threaded.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "mgr_oracle.c")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libmgr_oracle.so")

OK, INVALID, NOMEM, SINGULAR, NOT_CONVERGED = 0, 1, 2, 4, 5
RELAX = {"jacobi": 0, "l1_jacobi": 1, "block_jacobi": 2, "amg": 3}
RESTRICT = {"injection": 0, "jacobi": 1}


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/lib`` (idempotent)."""
    os.makedirs(LIBDIR, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
        r = subprocess.run(base + ["-fopenmp", SRC, "-lm", "-o", tmp], capture_output=True)
        if r.returncode != 0:  # a toolchain without OpenMP: the same source, one thread
            subprocess.check_call(base + [SRC, "-lm", "-o", tmp])
        os.replace(tmp, LIB)
    return LIB


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel solve loops (n <= 0: keep); returns
    the count in effect."""
    return int(lib().or_set_threads(int(n)))


def affinity_cores() -> int:
    """Cores of this process's affinity set (the oracle's default thread count)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        vp, ip, dp = C.c_void_p, C.c_int, C.c_double
        L.or_setup.restype = vp
        L.or_setup.argtypes = [ip, ip, vp, vp, vp, vp, ip, vp, vp, vp, vp, vp, dp, ip, ip, ip, ip, vp, vp]
        L.or_free.argtypes = [vp]
        L.or_apply.argtypes = [vp, vp, vp]
        L.or_apply_transpose.argtypes = [vp, vp, vp]
        L.or_solve.argtypes = [vp, vp, vp, dp, ip, ip, ip, ip, vp, vp, vp]
        L.or_spmv_bsr.argtypes = [ip, ip, vp, vp, vp, vp, vp]
        L.or_dense_solve.argtypes = [ip, vp, vp, vp]
        L.or_set_threads.argtypes = [ip]
        L.or_set_threads.restype = ip
        L.or_pmis_u01.restype = dp
        L.or_pmis_u01.argtypes = [C.c_uint, C.c_uint]
        for nm in ("or_n", "or_mgr_nlevels", "or_amg_nlevels", "or_amg_coarse_n"):
            getattr(L, nm).argtypes = [vp]
        L.or_mat_dims.argtypes = [vp, ip, ip, ip, vp]
        L.or_mat_copy.argtypes = [vp, ip, ip, ip, vp, vp, vp]
        L.or_mgr_dinv.argtypes = [vp, ip, vp, vp]
        L.or_amg_cf.argtypes = [vp, ip, ip, vp]
        L.or_amg_dinv.argtypes = [vp, ip, ip, vp]
        L.or_amg_nlevels_of.argtypes = [vp, ip]
        L.or_amg_split_interp.argtypes = [ip, vp, vp, vp, vp, dp, ip, ip, vp, vp, vp, vp, ip, vp]
        L.or_amg_strength.argtypes = [ip, vp, vp, vp, vp, dp, vp, vp, ip]
        # all cores of the affinity set (OpenMP's default may count others)
        L.or_set_threads(affinity_cores())
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def spmv_bsr(nb, b, row_ptr, col_idx, val, x):
    """y = A x for a BSR matrix, by its definition."""
    rp, ci, v, xx = _i32(row_ptr), _i32(col_idx), _f64(val), _f64(x)
    y = np.zeros(nb * b)
    lib().or_spmv_bsr(nb, b, _p(rp), _p(ci), _p(v), _p(xx), _p(y))
    return y


def dense_solve(A, rhs):
    A = _f64(A); rhs = _f64(rhs)
    n = A.shape[0]
    x = np.zeros(n)
    rc = lib().or_dense_solve(n, _p(A), _p(rhs), _p(x))
    if rc:
        raise RuntimeError(f"dense_solve status {rc}")
    return x


def pmis_u01(i, level):
    return lib().or_pmis_u01(int(i), int(level))


@dataclass
class Options:
    """MGR/AMG options (readings of the paper's unspecified parameters)."""
    relax: list = field(default_factory=lambda: ["jacobi"])
    sweeps: list = field(default_factory=list)
    weights: list = field(default_factory=list)
    theta: float = 0.25
    max_levels: int = 25
    max_coarse: int = 1024
    pmax: int = 4
    num_functions: int = 1
    relax_functions: list = field(default_factory=list)
    # per-level restriction: "injection" (R = [0, I]) or "jacobi" (R = [-A_CF D^-1, I], Eq. 5)
    restrict: list = field(default_factory=list)
    restart: int = 30


class Oracle:
    """An MGR hierarchy built by the oracle for one :class:`BlockSystem`."""

    def __init__(self, sysm, opts: Options | None = None, reuse: "Oracle | None" = None):
        """reuse: an oracle built before on the same pattern and labels whose
        AMG F-relaxation hierarchies are taken over (the setup reuse of
        Sec. 4.3); it is closed afterwards."""
        if opts is None:
            opts = Options(relax=list(sysm.relax), num_functions=sysm.num_functions,
                           relax_functions=list(getattr(sysm, "relax_functions", ())))
        L = lib()
        nl = sysm.num_levels
        self.opts = opts
        self.sysm = sysm
        self._keep = [_i32(sysm.row_ptr), _i32(sysm.col_idx), _f64(sysm.val),
                      np.ascontiguousarray(sysm.dof_level, dtype=np.int8)]
        rt = np.array([RELAX[r] for r in (opts.relax + ["jacobi"] * nl)[:nl]] + [0], np.int32)
        sw = np.array(((opts.sweeps or []) + [1] * nl)[:nl] + [1], np.int32)
        wt = np.array(((opts.weights or []) + [1.0] * nl)[:nl] + [1.0], np.float64)
        fn = np.array(((opts.relax_functions or []) + [1] * nl)[:nl] + [1], np.int32)
        rs = np.array([RESTRICT[r] if isinstance(r, str) else int(r)
                       for r in ((opts.restrict or []) + ["injection"] * nl)[:nl]] + [0], np.int32)
        self._keep += [rt, sw, wt, fn, rs]
        st = np.zeros(1, np.int32)
        rp, ci, v, lv = self._keep[:4]
        self.h = L.or_setup(sysm.nb, sysm.b, _p(rp), _p(ci), _p(v), _p(lv), nl, _p(rt), _p(sw),
                            _p(wt), _p(fn), _p(rs), opts.theta, opts.max_levels, opts.max_coarse, opts.pmax,
                            opts.num_functions, reuse.h if reuse is not None else None, _p(st))
        if reuse is not None:
            reuse.close()
        self.status = int(st[0])
        if not self.h:
            raise RuntimeError(f"oracle setup failed with status {self.status}")
        self.n = L.or_n(self.h)

    def close(self):
        if getattr(self, "h", None):
            lib().or_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, v):
        v = _f64(v); z = np.zeros(self.n)
        lib().or_apply(self.h, _p(v), _p(z))
        return z

    def apply_transpose(self, v):
        v = _f64(v); z = np.zeros(self.n)
        lib().or_apply_transpose(self.h, _p(v), _p(z))
        return z

    def solve(self, rhs, x0=None, rtol=1e-8, maxit=300, restart=None, precond=True, trans=False):
        rhs = _f64(rhs)
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        it = np.zeros(1, np.int32); rr = np.zeros(1); hist = np.zeros(maxit + 1)
        m = restart or self.opts.restart
        rc = lib().or_solve(self.h, _p(rhs), _p(x), rtol, maxit, m, int(precond), int(trans),
                            _p(it), _p(rr), _p(hist))
        return dict(x=x, iters=int(it[0]), relres=float(rr[0]), hist=hist[:int(it[0]) + 1],
                    status=int(rc))

    # ---- inspection
    @property
    def mgr_nlevels(self):
        return lib().or_mgr_nlevels(self.h)

    @property
    def amg_nlevels(self):
        return lib().or_amg_nlevels(self.h)

    def _mat(self, amg, lvl, which):
        d = np.zeros(3, np.int32)
        if lib().or_mat_dims(self.h, amg, lvl, which, _p(d)):
            return None
        n, m, nnz = map(int, d)
        rp = np.zeros(n + 1, np.int32); ci = np.zeros(max(nnz, 1), np.int32)
        v = np.zeros(max(nnz, 1))
        lib().or_mat_copy(self.h, amg, lvl, which, _p(rp), _p(ci), _p(v))
        return rp, ci[:nnz], v[:nnz], (n, m)

    MGR_WHICH = {"A": 0, "AFF": 1, "AFC": 2, "ACF": 3, "W": 4, "Z": 5}

    def mgr_matrix(self, lvl, which="A"):
        """CSR (rp, ci, v, shape) of MGR level ``lvl``; lvl == num_levels is
        the final coarse block handed to AMG."""
        return self._mat(0, lvl, self.MGR_WHICH[which])

    def amg_matrix(self, k, which="A", frelax_level=None):
        """AMG level k of the final coarse block, or of MGR level
        ``frelax_level``'s AMG F-relaxation."""
        amg = 1 if frelax_level is None else 2 + frelax_level
        return self._mat(amg, k, {"A": 0, "P": 1}[which])

    def amg_cf(self, k, frelax_level=None):
        amg = 1 if frelax_level is None else 2 + frelax_level
        n = self.amg_matrix(k, "A", frelax_level)[3][0]
        cf = np.zeros(n, np.int32)
        if lib().or_amg_cf(self.h, amg, k, _p(cf)):
            return None
        return cf

    def amg_dinv(self, k, frelax_level=None):
        """1/d_i of the l1-Jacobi smoother of AMG level k (not the coarsest)."""
        amg = 1 if frelax_level is None else 2 + frelax_level
        n = self.amg_matrix(k, "A", frelax_level)[3][0]
        d = np.zeros(n)
        if lib().or_amg_dinv(self.h, amg, k, _p(d)):
            return None
        return d

    def frelax_amg_nlevels(self, lvl):
        """AMG levels of MGR level ``lvl``'s F-relaxation (0: not AMG)."""
        return lib().or_amg_nlevels_of(self.h, 2 + lvl)

    def mgr_dinv(self, lvl):
        rp = self.mgr_matrix(lvl, "AFF")[0]
        nF = rp.size - 1
        d = np.zeros(nF * 4); g = np.zeros(nF, np.int32)
        lib().or_mgr_dinv(self.h, lvl, _p(d), _p(g))
        return d.reshape(nF, 4), g


def amg_split_interp(rp, ci, v, func=None, theta=0.25, level=0, pmax=4):
    """Strength + PMIS + extended+i on one CSR matrix: returns (cf, P-CSR, nc)."""
    rp, ci, v = _i32(rp), _i32(ci), _f64(v)
    n = rp.size - 1
    func = np.zeros(n, np.int32) if func is None else _i32(func)
    cf = np.zeros(n, np.int32)
    cap = n * max(pmax, 1) + 1 if pmax > 0 else int(rp[-1]) * 64 + n + 1
    prp = np.zeros(n + 1, np.int32); pci = np.zeros(cap, np.int32); pv = np.zeros(cap)
    nc = np.zeros(1, np.int32)
    rc = lib().or_amg_split_interp(n, _p(rp), _p(ci), _p(v), _p(func), theta, level, pmax,
                                   _p(cf), _p(prp), _p(pci), _p(pv), cap, _p(nc))
    if rc:
        raise RuntimeError(f"amg_split_interp status {rc}")
    nnz = int(prp[-1])
    return cf, (prp, pci[:nnz], pv[:nnz], (n, int(nc[0])))


def amg_strength(rp, ci, v, func=None, theta=0.25):
    rp, ci, v = _i32(rp), _i32(ci), _f64(v)
    n = rp.size - 1
    func = np.zeros(n, np.int32) if func is None else _i32(func)
    srp = np.zeros(n + 1, np.int32); sci = np.zeros(max(int(rp[-1]), 1), np.int32)
    rc = lib().or_amg_strength(n, _p(rp), _p(ci), _p(v), _p(func), theta, _p(srp), _p(sci),
                               sci.size)
    if rc:
        raise RuntimeError(f"amg_strength status {rc}")
    return srp, sci[:int(srp[-1])]
