"""ctypes binding of libmgr_gb300.so (include/mgr_gb300.h).

Argument marshalling only: every step of setup and solve runs in the CUDA
library.  Vectors are torch CUDA float64 tensors on the handle's device;
the handle's stream is torch's current stream at construction.  If the
library cannot be loaded this module raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

MGR_OK, MGR_ERR_INVALID, MGR_ERR_NOMEM, MGR_ERR_CUDA, MGR_ERR_SINGULAR = 0, 1, 2, 3, 4
MGR_ERR_NOT_CONVERGED, MGR_ERR_TIMEOUT, MGR_ERR_UNSUPPORTED = 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "NOMEM", 3: "CUDA", 4: "SINGULAR", 5: "NOT_CONVERGED",
                6: "TIMEOUT", 7: "UNSUPPORTED"}
RELAX = {"jacobi": 0, "l1_jacobi": 1, "block_jacobi": 2, "amg": 3}
RESTRICT = {"injection": 0, "jacobi": 1}
MAX_LEVELS = 8


class MGRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mgr_bsr(C.Structure):
    _fields_ = [("nb", C.c_int32), ("b", C.c_int32), ("nnzb", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p),
                ("on_device", C.c_int32)]


class mgr_labels(C.Structure):
    _fields_ = [("num_levels", C.c_int32), ("dof_level", C.c_void_p)]


class mgr_options(C.Structure):
    _fields_ = [("relax_type", C.c_int32 * MAX_LEVELS), ("relax_sweeps", C.c_int32 * MAX_LEVELS),
                ("relax_weight", C.c_double * MAX_LEVELS), ("amg_theta", C.c_double),
                ("amg_max_levels", C.c_int32), ("amg_max_coarse", C.c_int32),
                ("amg_pmax", C.c_int32), ("amg_num_functions", C.c_int32),
                ("precision", C.c_int32), ("restart", C.c_int32), ("use_graphs", C.c_int32),
                ("amg_tail_nnz", C.c_int32), ("relax_functions", C.c_int32 * MAX_LEVELS),
                ("restrict_type", C.c_int32 * MAX_LEVELS), ("spin_limit", C.c_int32)]


class mgr_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("rel_residual", C.c_double),
                ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("mgr_levels", C.c_int32), ("amg_levels", C.c_int32),
                ("level_rows", C.c_int64 * 40), ("level_nnz", C.c_int64 * 40),
                ("operator_complexity", C.c_double), ("reorth_steps", C.c_int32)]

    def as_dict(self):
        nl = self.mgr_levels + self.amg_levels
        return dict(iterations=self.iterations, rel_residual=self.rel_residual,
                    setup_ms=self.setup_ms, solve_ms=self.solve_ms, mgr_levels=self.mgr_levels,
                    amg_levels=self.amg_levels, level_rows=list(self.level_rows[:nl]),
                    level_nnz=list(self.level_nnz[:nl]),
                    operator_complexity=self.operator_complexity,
                    reorth_steps=self.reorth_steps)


_lib = None


def lib(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree first when stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA library not built: {_build.LIB}")
    L = C.CDLL(_build.LIB)
    vp, i32, dp = C.c_void_p, C.c_int32, C.c_double
    L.mgr_options_default.argtypes = [C.POINTER(mgr_options)]
    L.mgr_options_default.restype = None
    L.mgr_setup.argtypes = [C.POINTER(mgr_bsr), C.POINTER(mgr_labels), C.POINTER(mgr_options), vp,
                            C.POINTER(vp)]
    for nm in ("mgr_apply", "mgr_apply_transpose", "mgr_spmv"):
        getattr(L, nm).argtypes = [vp, vp, vp]
    L.mgr_solve.argtypes = [vp, vp, vp, dp, i32, C.POINTER(mgr_solve_info)]
    L.mgr_solve_transpose.argtypes = [vp, vp, vp, dp, i32, C.POINTER(mgr_solve_info)]
    L.mgr_grad_values.argtypes = [vp, vp, vp, vp]
    L.mgr_update_values.argtypes = [vp, vp, i32]
    L.mgr_refresh.argtypes = [vp, vp, i32]
    L.mgr_bsr_spmv.argtypes = [i32, i32, vp, vp, vp, vp, vp, dp, dp, vp]
    L.mgr_free.argtypes = [vp]
    L.mgr_free.restype = None
    L.mgr_last_error.argtypes = [vp]
    L.mgr_last_error.restype = C.c_char_p
    L.mgr_get_matrix.argtypes = [vp, i32, i32, i32, vp, vp, vp, vp]
    L.mgr_get_cf.argtypes = [vp, i32, vp]
    L.mgr_get_amg_cf.argtypes = [vp, i32, i32, vp]
    L.mgr_get_amg_levels.argtypes = [vp, i32]
    L.mgr_get_amg_levels.restype = i32
    L.mgr_get_dinv.argtypes = [vp, i32, vp, vp]
    L.mgr_get_info.argtypes = [vp, vp]
    L.mgr_check_hierarchy.argtypes = [vp, C.POINTER(C.c_int64)]
    L.mgr_solve_history.argtypes = [vp, vp, i32]
    L.mgr_solve_history.restype = i32
    L.mgr_residual_norm_noalloc.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.mgr_measure_fp64_fma.argtypes = [vp, i32, C.POINTER(C.c_double)]
    L.mgr_launch_count.argtypes = []
    L.mgr_launch_count.restype = C.c_int64
    L.mgr_profile.argtypes = [vp, i32]
    L.mgr_profile_entries.argtypes = [vp]
    L.mgr_profile_entries.restype = i32
    L.mgr_profile_entry.argtypes = [vp, i32, C.c_char_p, i32, C.POINTER(C.c_double),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]
    _lib = L
    return L


def _check(st, h=None):
    if st != MGR_OK:
        msg = lib().mgr_last_error(h).decode(errors="replace")
        raise MGRError(st, msg)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _value_key(val):
    """Identity of a values tensor for MGRSolver.holds_values: its storage
    address, shape, dtype and in-place version counter (None for arrays that
    are not torch tensors, which the solver copies and cannot track)."""
    import torch
    if not isinstance(val, torch.Tensor):
        return None
    return (val.data_ptr(), tuple(val.shape), val.dtype, val._version)


def options(relax=("jacobi",), sweeps=(), weights=(), theta=0.25, max_levels=25, max_coarse=1024,
            pmax=4, num_functions=1, precision="fp64", restart=30, use_graphs=True,
            tail_nnz=None, relax_functions=(), restrict=(), spin_limit=None) -> mgr_options:
    o = mgr_options()
    lib().mgr_options_default(C.byref(o))
    for l, r in enumerate(relax):
        o.relax_type[l] = RELAX[r] if isinstance(r, str) else int(r)
    for l, s in enumerate(sweeps):
        o.relax_sweeps[l] = int(s)
    for l, w in enumerate(weights):
        o.relax_weight[l] = float(w)
    o.amg_theta = theta
    o.amg_max_levels = max_levels
    o.amg_max_coarse = max_coarse
    o.amg_pmax = pmax
    o.amg_num_functions = num_functions
    o.precision = {"fp64": 0, "fp32": 1}[precision] if isinstance(precision, str) else int(precision)
    o.restart = restart
    o.use_graphs = int(bool(use_graphs))
    if tail_nnz is not None:
        o.amg_tail_nnz = int(tail_nnz)
    for l, f in enumerate(relax_functions):
        o.relax_functions[l] = int(f)
    for l, r in enumerate(restrict):
        o.restrict_type[l] = RESTRICT[r] if isinstance(r, str) else int(r)
    if spin_limit is not None:
        o.spin_limit = int(spin_limit)
    return o


class MGRSolver:
    """MGR-preconditioned FGMRES for one block system (one GPU)."""

    def __init__(self, row_ptr, col_idx, val, b, dof_level, num_levels, opts=None, device=None,
                 stream=None):
        import torch
        L = lib()
        self.device = torch.device(device or "cuda")
        self.b = int(b)
        on_dev = isinstance(val, torch.Tensor) and val.is_cuda
        if on_dev:
            rp = row_ptr.to(self.device, torch.int32).contiguous()
            ci = col_idx.to(self.device, torch.int32).contiguous()
            vv = val.to(self.device, torch.float64).contiguous()
            keep = (rp, ci, vv)
            ptrs = (rp.data_ptr(), ci.data_ptr(), vv.data_ptr())
            nb = rp.numel() - 1
            nnzb = ci.numel()
        else:
            rp = np.ascontiguousarray(row_ptr, np.int32)
            ci = np.ascontiguousarray(col_idx, np.int32)
            vv = np.ascontiguousarray(val, np.float64)
            keep = (rp, ci, vv)
            ptrs = (rp.ctypes.data, ci.ctypes.data, vv.ctypes.data)
            nb = rp.size - 1
            nnzb = ci.size
        lv = np.ascontiguousarray(dof_level, np.int8)
        A = mgr_bsr(nb, self.b, nnzb, ptrs[0], ptrs[1], ptrs[2], int(on_dev))
        labels = mgr_labels(int(num_levels), lv.ctypes.data)
        self.opts = opts if opts is not None else options()
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            self._stream = stream if stream is not None else torch.cuda.current_stream()
            st = L.mgr_setup(C.byref(A), C.byref(labels), C.byref(self.opts),
                             C.c_void_p(self._stream.cuda_stream), C.byref(h))
        if st != MGR_OK:
            raise MGRError(st, L.mgr_last_error(None).decode(errors="replace"))
        del keep
        self.h = h
        self.n = nb * self.b
        self.nb = nb
        self.nnzb = nnzb
        self._held = _value_key(val)

    @classmethod
    def from_system(cls, sysm, precision="fp64", **kw):
        kw.setdefault("relax_functions", tuple(getattr(sysm, "relax_functions", ())))
        o = options(relax=tuple(sysm.relax), num_functions=sysm.num_functions, precision=precision,
                    **kw)
        return cls(sysm.row_ptr, sysm.col_idx, sysm.val, sysm.b, sysm.dof_level, sysm.num_levels,
                   o)

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().mgr_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _vec(self, t):
        import torch
        assert isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
        assert t.numel() == self.n and t.is_contiguous()
        return _ptr(t)

    def apply(self, v, z=None, transpose=False):
        import torch
        z = torch.empty_like(v) if z is None else z
        f = lib().mgr_apply_transpose if transpose else lib().mgr_apply
        _check(f(self.h, self._vec(v), self._vec(z)), self.h)
        return z

    def spmv(self, x, y=None):
        import torch
        y = torch.empty_like(x) if y is None else y
        _check(lib().mgr_spmv(self.h, self._vec(x), self._vec(y)), self.h)
        return y

    def solve(self, rhs, x=None, rtol=1e-8, maxit=500, transpose=False, check=True):
        import torch
        x = torch.zeros_like(rhs) if x is None else x
        info = mgr_solve_info()
        f = lib().mgr_solve_transpose if transpose else lib().mgr_solve
        st = f(self.h, self._vec(rhs), self._vec(x), float(rtol), int(maxit), C.byref(info))
        if check and st not in (MGR_OK, MGR_ERR_NOT_CONVERGED):
            _check(st, self.h)
        d = info.as_dict()
        d["status"] = int(st)
        return x, d

    def holds_values(self, val):
        """True when `val` is the tensor the solver last took its values from
        (setup, refresh or update_values) and has not been modified since."""
        return self._held is not None and _value_key(val) == self._held

    def update_values(self, val):
        """New values of A (same pattern) for the outer operator; the
        hierarchy from setup stays the preconditioner."""
        import torch
        if isinstance(val, torch.Tensor) and val.is_cuda:
            v = val.to(torch.float64).contiguous()
            _check(lib().mgr_update_values(self.h, _ptr(v), 1), self.h)
        else:
            v = np.ascontiguousarray(val, np.float64)
            _check(lib().mgr_update_values(self.h, v.ctypes.data, 0), self.h)
        self._held = _value_key(val)

    def refresh(self, val):
        """New values of A (same pattern): the MGR levels and the final AMG
        hierarchy are rebuilt from them, AMG F-relaxation hierarchies are
        kept (setup reuse)."""
        import torch
        self._held = None
        if isinstance(val, torch.Tensor) and val.is_cuda:
            v = val.to(torch.float64).contiguous()
            _check(lib().mgr_refresh(self.h, _ptr(v), 1), self.h)
        else:
            v = np.ascontiguousarray(val, np.float64)
            _check(lib().mgr_refresh(self.h, v.ctypes.data, 0), self.h)
        self._held = _value_key(val)

    def grad_values(self, lam, x):
        import torch
        dA = torch.empty(self.nnzb * self.b * self.b, dtype=torch.float64, device=lam.device)
        _check(lib().mgr_grad_values(self.h, self._vec(lam), self._vec(x), _ptr(dA)), self.h)
        return dA.view(self.nnzb, self.b, self.b)

    # ---------------------------------------------------- instrumentation
    def profile(self, on=True):
        """Start (and reset) or stop per-kernel-class event timing."""
        _check(lib().mgr_profile(self.h, int(bool(on))), self.h)

    def profile_table(self):
        """[{name, ms, launches, bytes_per_launch, fp64_fma_per_launch}] since profile(True)."""
        L = lib()
        out = []
        for i in range(L.mgr_profile_entries(self.h)):
            buf = C.create_string_buffer(96)
            ms, cnt, by, fm = C.c_double(), C.c_int64(), C.c_double(), C.c_double()
            _check(L.mgr_profile_entry(self.h, i, buf, 96, C.byref(ms), C.byref(cnt),
                                       C.byref(by), C.byref(fm)), self.h)
            out.append(dict(name=buf.value.decode(), ms=ms.value, launches=cnt.value,
                            bytes_per_launch=by.value, fp64_fma_per_launch=fm.value))
        return out

    # -------------------------------------------------------- inspection
    def info(self):
        out = np.zeros(3, np.int32)
        _check(lib().mgr_get_info(self.h, out.ctypes.data), self.h)
        return dict(mgr_levels=int(out[0]), amg_levels=int(out[1]), n=int(out[2]))

    def matrix(self, amg, level, which=0):
        d = np.zeros(3, np.int32)
        st = lib().mgr_get_matrix(self.h, int(amg), int(level), int(which), d.ctypes.data, None,
                                  None, None)
        if st != MGR_OK:
            return None
        n, m, nnz = map(int, d)
        rp = np.zeros(n + 1, np.int32)
        ci = np.zeros(max(nnz, 1), np.int32)
        v = np.zeros(max(nnz, 1))
        _check(lib().mgr_get_matrix(self.h, int(amg), int(level), int(which), d.ctypes.data,
                                    rp.ctypes.data, ci.ctypes.data, v.ctypes.data), self.h)
        return rp, ci[:nnz], v[:nnz], (n, m)

    def amg_cf(self, level, frelax_level=None):
        """C/F marks of AMG level ``level`` of the final coarse block's
        hierarchy, or of MGR level ``frelax_level``'s AMG F-relaxation."""
        amg = 1 if frelax_level is None else 2 + int(frelax_level)
        n = self.matrix(amg, level)[3][0]
        cf = np.zeros(n, np.int32)
        st = lib().mgr_get_amg_cf(self.h, amg, int(level), cf.ctypes.data)
        return cf if st == MGR_OK else None

    def history(self):
        """Relative residuals of the last solve: the initial true residual,
        then the Arnoldi estimate after every preconditioner application."""
        n = lib().mgr_solve_history(self.h, None, 0)
        out = np.zeros(max(n, 1))
        lib().mgr_solve_history(self.h, out.ctypes.data, n)
        return out[:n]

    def check(self):
        """Number of index-range and shape violations in the built hierarchy
        (0 for a sound one)."""
        v = C.c_int64(-1)
        _check(lib().mgr_check_hierarchy(self.h, C.byref(v)), self.h)
        return int(v.value)

    def frelax_amg_levels(self, level):
        """AMG levels of MGR level ``level``'s F-relaxation (0: not AMG)."""
        return int(lib().mgr_get_amg_levels(self.h, 2 + int(level)))

    def mgr_dinv(self, level):
        rp = self.matrix(0, level, 1)[0]
        nF = rp.size - 1
        d = np.zeros(nF * 4)
        g = np.zeros(nF, np.int32)
        _check(lib().mgr_get_dinv(self.h, int(level), d.ctypes.data, g.ctypes.data), self.h)
        return d.reshape(nF, 4), g


def bsr_spmv(row_ptr, col_idx, val, b, x, y=None, alpha=1.0, beta=0.0, stream=None):
    """y = alpha A x + beta y for device BSR arrays (no handle)."""
    import torch
    y = torch.zeros_like(x) if y is None else y
    nb = row_ptr.numel() - 1
    _check(lib().mgr_bsr_spmv(nb, int(b), _ptr(row_ptr), _ptr(col_idx), _ptr(val), _ptr(x), _ptr(y),
                              float(alpha), float(beta), _stream_ptr(stream)))
    return y


def measure_fp64_fma(reps=10, stream=None) -> float:
    """Measured FP64 FMA rate of the current device (FMA/s, best of reps)."""
    out = C.c_double()
    _check(lib().mgr_measure_fp64_fma(_stream_ptr(stream), int(reps), C.byref(out)))
    return out.value


def launch_count() -> int:
    """Kernel launches made by the library so far (all handles)."""
    return int(lib().mgr_launch_count())


def residual_norm_noalloc(row_ptr, col_idx, val, b, x, bvec, r=None, norm=None, stream=None):
    """r = bvec - A x and ||r||_2 (device tensors) through the allocation-free
    entry point: its reduction scratch is a static device array, so the call
    itself never allocates (torch allocates r and norm here when they are not
    passed in)."""
    import torch
    r = torch.empty_like(x) if r is None else r
    norm = torch.empty(1, dtype=torch.float64, device=x.device) if norm is None else norm
    nb = row_ptr.numel() - 1
    st = lib().mgr_residual_norm_noalloc(nb, int(b), _ptr(row_ptr), _ptr(col_idx), _ptr(val),
                                         _ptr(x), _ptr(bvec), _ptr(r), _ptr(norm),
                                         _stream_ptr(stream))
    if st != MGR_OK:
        raise MGRError(st, "mgr_residual_norm_noalloc")
    return r, norm


class _BorrowedSolver(MGRSolver):
    """A system handle owned by a batch (not freed by this object)."""

    def __init__(self, h, n, nb, b, nnzb, device):
        self.h = h
        self.n, self.nb, self.b, self.nnzb = n, nb, b, nnzb
        self.device = device
        self._held = None

    def close(self):
        self.h = C.c_void_p()


class MGRBatch:
    """Many systems solved together: one launch per kernel class for all."""

    def __init__(self, systems, precision="fp64", device=None, **kw):
        import torch
        L = lib()
        L.mgr_setup_batched.argtypes = [C.c_int32, C.POINTER(mgr_bsr), C.POINTER(mgr_labels),
                                        C.POINTER(mgr_options), C.c_void_p, C.POINTER(C.c_void_p)]
        L.mgr_solve_batched.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int32,
                                        C.POINTER(mgr_solve_info)]
        L.mgr_batch_handle.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p)]
        L.mgr_free_batched.argtypes = [C.c_void_p]
        L.mgr_free_batched.restype = None
        self.device = torch.device(device or "cuda")
        ns = len(systems)
        s0 = systems[0]
        kw.setdefault("relax_functions", tuple(getattr(s0, "relax_functions", ())))
        self.opts = options(relax=tuple(s0.relax), num_functions=s0.num_functions,
                            precision=precision, **kw)
        keep = []
        As = (mgr_bsr * ns)()
        Ls = (mgr_labels * ns)()
        for i, s in enumerate(systems):
            rp = np.ascontiguousarray(s.row_ptr, np.int32)
            ci = np.ascontiguousarray(s.col_idx, np.int32)
            vv = np.ascontiguousarray(s.val, np.float64)
            lv = np.ascontiguousarray(s.dof_level, np.int8)
            keep += [rp, ci, vv, lv]
            As[i] = mgr_bsr(rp.size - 1, s.b, ci.size, rp.ctypes.data, ci.ctypes.data,
                            vv.ctypes.data, 0)
            Ls[i] = mgr_labels(s.num_levels, lv.ctypes.data)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = L.mgr_setup_batched(ns, As, Ls, C.byref(self.opts),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(h))
        if st != MGR_OK:
            raise MGRError(st, L.mgr_last_error(None).decode(errors="replace"))
        self.h = h
        self.nsys = ns
        self.sizes = [s.n for s in systems]
        self._meta = [(s.n, s.nb, s.b, s.nnzb) for s in systems]

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().mgr_free_batched(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def system(self, i):
        """The borrowed single-system solver of member i (transpose solves,
        gradients, inspection); valid while the batch lives."""
        hh = C.c_void_p()
        _check(lib().mgr_batch_handle(self.h, int(i), C.byref(hh)))
        n, nb, b, nnzb = self._meta[i]
        return _BorrowedSolver(hh, n, nb, b, nnzb, self.device)

    def solve(self, rhs, xs=None, rtol=1e-8, maxit=500, check=True):
        import torch
        xs = [torch.zeros_like(r) for r in rhs] if xs is None else xs
        for r, x, n in zip(rhs, xs, self.sizes):
            assert r.is_cuda and r.dtype == torch.float64 and r.numel() == n and r.is_contiguous()
            assert x.is_cuda and x.dtype == torch.float64 and x.numel() == n and x.is_contiguous()
        bp = (C.c_void_p * self.nsys)(*[r.data_ptr() for r in rhs])
        xp = (C.c_void_p * self.nsys)(*[x.data_ptr() for x in xs])
        infos = (mgr_solve_info * self.nsys)()
        st = lib().mgr_solve_batched(self.h, bp, xp, float(rtol), int(maxit), infos)
        if check and st not in (MGR_OK, MGR_ERR_NOT_CONVERGED):
            _check(st)
        out = []
        for i in range(self.nsys):
            d = infos[i].as_dict()
            d["status"] = int(st)
            out.append(d)
        return xs, out
