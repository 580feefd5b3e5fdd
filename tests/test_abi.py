"""The C-ABI library loads and exports every entry point the header declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

from paper_2101_11649_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(mgr_\w+)\s*\(", txt, flags=re.M))
    return names


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("mgr_setup", "mgr_apply", "mgr_solve", "mgr_free", "mgr_apply_transpose",
                 "mgr_solve_transpose", "mgr_grad_values", "mgr_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_options_default_and_null_handling():
    lib = ctypes.CDLL(_build.build())
    from paper_2101_11649_gb300 import mgr as M
    o = M.mgr_options()
    lib.mgr_options_default(ctypes.byref(o))
    assert o.amg_theta == 0.25 and o.amg_max_coarse == 1024 and o.amg_pmax == 4 and o.restart == 30
    assert list(o.relax_sweeps)[:2] == [1, 1] and o.relax_weight[0] == 1.0
    # the fields after the AMG block: a layout mismatch between the ctypes
    # mirror and the C struct would show here
    assert o.amg_num_functions == 1 and o.precision == 0 and o.use_graphs == 1
    assert o.amg_tail_nnz == 0 and o.spin_limit == 0
    assert list(o.relax_functions) == [1] * M.MAX_LEVELS
    assert list(o.restrict_type) == [0] * M.MAX_LEVELS
    assert ctypes.sizeof(o) == 8 * 4 + 8 * 4 + 8 * 8 + 8 + 4 * 4 + 4 * 4 + 8 * 4 + 8 * 4 + 4 + 4
    lib.mgr_free(None)  # no-op
    lib.mgr_setup.restype = ctypes.c_int
    # NULL out pointer -> INVALID, no CUDA call made
    assert lib.mgr_setup(None, None, None, None, None) == 1
    lib.mgr_last_error.restype = ctypes.c_char_p
    assert b"NULL" in lib.mgr_last_error(None)


def test_python_options_mapping():
    """Names and per-level lists of the Python options() reach the C struct."""
    from paper_2101_11649_gb300 import mgr as M
    o = M.options(relax=("amg", "l1_jacobi", "block_jacobi"), sweeps=(2,), weights=(0.8,),
                  relax_functions=(3,), restrict=("jacobi", "injection"), spin_limit=7,
                  max_coarse=32, precision="fp32", tail_nnz=1000)
    assert list(o.relax_type)[:3] == [M.RELAX["amg"], M.RELAX["l1_jacobi"], M.RELAX["block_jacobi"]]
    assert o.relax_sweeps[0] == 2 and o.relax_sweeps[1] == 1 and o.relax_weight[0] == 0.8
    assert o.relax_functions[0] == 3 and o.relax_functions[1] == 1
    assert list(o.restrict_type)[:2] == [1, 0] and o.spin_limit == 7
    assert o.amg_max_coarse == 32 and o.precision == 1 and o.amg_tail_nnz == 1000
