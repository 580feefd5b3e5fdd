"""CUDA path vs the CPU oracle, through the C ABI (marked gpu).

Setup is compared bit for bit (both sides follow the same stated operation
order without fused multiply-add); the solve phase within the tolerances of
the FP64 arithmetic: SpMV per entry relative to sum_j |a_ij x_j| (1e-13);
V-cycle outputs entry by entry, per MGR level's F set and per final coarse
block, within 1e-11 of the set's largest entry (1e-4 for the FP32 cycle);
FGMRES iterations +-1; solutions converged to 1e-12 within 1e-8 in the
2-norm and per set.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_11649_gb300.synth import (make_compositional, make_mimetic, make_poromech,
                                          make_two_phase)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2101_11649_gb300 import mgr as M  # noqa: E402
from parity_checks import cycle_close  # noqa: E402

DEV = torch.device("cuda:0")

SMALL = {
    "two_phase": lambda: make_two_phase(8, 7, 5),
    "mimetic": lambda: make_mimetic(7, 6, 5),
    # TPFA with the face multipliers as F-points (MGR_Pi, Sec. 4.1)
    "mimetic_tpfa_mgr_pi": lambda: make_mimetic(7, 6, 5, scheme="tpfa", strategy="mgr_pi"),
    "compositional": lambda: make_compositional(16, 12, 4),
    # the 4-level order of Sec. 4.2: Jacobi, Jacobi, AMG F-relaxation of the
    # reservoir pressure, wells solved directly on the coarsest grid
    "compositional_4level": lambda: make_compositional(16, 12, 4, strategy="mgr4"),
    "poromech": lambda: make_poromech(8, 4),
    # MGR_U (Sec. 4.3): displacement first, one AMG V-cycle as F-relaxation
    "poromech_mgr_u": lambda: make_poromech(8, 4, strategy="mgr_u"),
    # an AMG F-relaxation of a nonsymmetric (upwinded) A_FF, so that the
    # transposed V-cycle differs from the forward one
    "two_phase_amg_relax": lambda: dataclasses.replace(make_two_phase(8, 7, 5), relax=["amg"],
                                                       relax_functions=[1]),
}


def t(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device=DEV)


def solver(sysm, precision="fp64", **kw):
    return M.MGRSolver.from_system(sysm, precision=precision, **kw)


# the small systems stop coarsening at 32 rows (both sides), so their AMG
# hierarchies keep several levels under the default coarsest size of 1024
SMALL_COARSE = 32


def oracle_of(sysm, **kw):
    return O.Oracle(sysm, O.Options(relax=list(sysm.relax), num_functions=sysm.num_functions,
                                    relax_functions=list(sysm.relax_functions), **kw))


# ------------------------------------------------------------------ SpMV
@pytest.mark.parametrize("b", [1, 2, 3, 4])
@pytest.mark.parametrize("nb", [1, 7, 33, 1000])
def test_bsr_spmv_parity(b, nb):
    rng = np.random.default_rng(100 * b + nb)
    from paper_2101_11649_gb300.synth.bsr import assemble_bsr
    rows, cols = [], []
    for i in range(nb):
        if i % 5 == 3:
            continue  # empty block rows
        js = np.unique(rng.integers(0, nb, 1 + rng.integers(0, 9)))
        rows += [i] * len(js); cols += list(js)
    rp, ci, val = assemble_bsr(nb, b, np.array(rows, np.int64), np.array(cols, np.int64),
                               rng.standard_normal((len(rows), b, b)))
    x = rng.standard_normal(nb * b)
    y0 = rng.standard_normal(nb * b)
    ref = O.spmv_bsr(nb, b, rp, ci, val, x)
    absref = O.spmv_bsr(nb, b, rp, ci, np.abs(val), np.abs(x)) + 1e-300
    trp = torch.as_tensor(rp, device=DEV); tci = torch.as_tensor(ci, device=DEV)
    tv = t(val.ravel())
    y = M.bsr_spmv(trp, tci, tv, b, t(x))
    torch.cuda.synchronize()
    err = np.abs(y.cpu().numpy() - ref) / absref
    assert err.max() <= 1e-13
    # alpha, beta form
    y2 = M.bsr_spmv(trp, tci, tv, b, t(x), y=t(y0), alpha=-2.0, beta=0.5)
    ref2 = -2.0 * ref + 0.5 * y0
    assert (np.abs(y2.cpu().numpy() - ref2) / (2 * absref + 0.5 * np.abs(y0))).max() <= 1e-13


# ------------------------------------------- SELL-C-sigma over row shapes
def _banded_m_matrix(n, K, keep, seed):
    """Scalar symmetric M-matrix (AMG only, no MGR level): the pair (i, i+d),
    d = 1..K, is kept with probability ``keep`` (ragged rows of up to 2K+1
    entries); off-diagonals -U(0.1, 1), diagonal = sum of the row's
    off-diagonal magnitudes + U(0.1, 1)."""
    from paper_2101_11649_gb300.synth.bsr import BlockSystem, assemble_bsr
    rng = np.random.default_rng(seed)
    ii = [np.flatnonzero(rng.random(n - d) < keep) for d in range(1, K + 1)]
    jj = np.concatenate([i + d for d, i in zip(range(1, K + 1), ii)])
    ii = np.concatenate(ii)
    w = rng.uniform(0.1, 1.0, ii.size)
    diag = np.bincount(ii, w, n) + np.bincount(jj, w, n) + rng.uniform(0.1, 1.0, n)
    rows = np.concatenate([ii, jj, np.arange(n)])
    cols = np.concatenate([jj, ii, np.arange(n)])
    rp, ci, val = assemble_bsr(n, 1, rows, cols, np.concatenate([-w, -w, diag]))
    return BlockSystem(f"band{n}x{K}", 1, rp, ci, val, np.zeros(n, np.int8), 0,
                       rng.standard_normal(n))


# (rows, half band, kept fraction): average row lengths 7 .. 200 at row
# counts 3k .. 300k, so the layout's lanes per row range over 1 .. 32; none
# of the row counts is a multiple of 32
BANDS = [(300007, 3, 1.0), (120001, 20, 0.95), (60007, 40, 0.95), (40009, 75, 1.0),
         (10007, 60, 1.0), (3001, 100, 1.0), (50021, 30, 0.3)]


@pytest.mark.parametrize("n,K,keep", BANDS)
def test_sell_products_over_row_shapes(n, K, keep):
    s = _banded_m_matrix(n, K, keep, seed=n)
    g = solver(s)
    x = np.random.default_rng(7).standard_normal(n)
    y = g.spmv(t(x)).cpu().numpy()
    ref = O.spmv_bsr(n, 1, s.row_ptr, s.col_idx, s.val, x)
    absref = O.spmv_bsr(n, 1, s.row_ptr, s.col_idx, np.abs(s.val), np.abs(x)) + 1e-300
    assert (np.abs(y - ref) / absref).max() <= 1e-13
    if n <= 10007:
        # every coarse level's product, both precisions, through the V-cycle
        o = O.Oracle(s)
        zo = o.apply(x)
        zg = g.apply(t(x)).cpu().numpy()
        cycle_close(s, zg, zo, 1e-11, "fp64")
        z32 = solver(s, precision="fp32").apply(t(x)).cpu().numpy()
        cycle_close(s, z32, zo, 1e-4, "fp32")


# ------------------------------------------------------- fused AMG tail
TAIL_SYSTEMS = {
    "mimetic24": lambda: make_mimetic(24, 24, 24),
    "two_phase32x32x16": lambda: make_two_phase(32, 32, 16),
}


@pytest.mark.parametrize("name", list(TAIL_SYSTEMS))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fused_tail_is_bitwise_the_per_level_cycle(name, precision):
    """The coarse AMG levels as one cluster launch give the same bits as one
    launch per step (same row sums and epilogues), forward and transposed."""
    s = TAIL_SYSTEMS[name]()
    fused = solver(s, precision=precision, tail_nnz=400000)
    plain = solver(s, precision=precision, tail_nnz=0)
    assert fused.info()["amg_levels"] >= 3
    v = t(np.random.default_rng(11).standard_normal(s.n))
    fused.profile(True)
    for trans in (False, True):
        a = fused.apply(v, transpose=trans)
        b = plain.apply(v, transpose=trans)
        torch.cuda.synchronize()
        assert torch.equal(a, b), (trans, float((a - b).abs().max()))
    names = [r["name"] for r in fused.profile_table()]
    fused.profile(False)
    assert any(n.startswith("amg_tail") for n in names), names
    assert not any(n.startswith("amg_tail") for n in [r["name"] for r in plain.profile_table()])
    xf, inf_f = fused.solve(t(s.rhs), rtol=1e-8)
    xp, inf_p = plain.solve(t(s.rhs), rtol=1e-8)
    assert inf_f["iterations"] == inf_p["iterations"] and torch.equal(xf, xp)


def test_programmatic_launch_changes_no_bits(tmp_path):
    """Kernels may be scheduled while their predecessor drains (programmatic
    dependent launch) but wait for its results: the same solves in a fresh
    process with MGR_PDL=0 (plain stream order) give the same bits."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import numpy as np, torch\n"
        "from paper_2101_11649_gb300 import mgr as M\n"
        "from paper_2101_11649_gb300.synth import make_mimetic\n"
        "s = make_mimetic(24, 24, 24)\n"
        "b = torch.as_tensor(s.rhs, device='cuda')\n"
        "for p in ('fp64', 'fp32'):\n"
        "    x, info = M.MGRSolver.from_system(s, precision=p).solve(b, rtol=1e-10)\n"
        f"    np.save(r'{tmp_path}' + '/x_' + p + '.npy', x.cpu().numpy())\n")
    env = dict(os.environ, MGR_PDL="0")
    subprocess.run([sys.executable, "-c", code], env=env, check=True, cwd=root, timeout=600)
    s = make_mimetic(24, 24, 24)
    for p in ("fp64", "fp32"):
        x, _ = solver(s, precision=p).solve(t(s.rhs), rtol=1e-10)
        x0 = np.load(tmp_path / f"x_{p}.npy")
        assert np.array_equal(x0.view(np.int64), x.cpu().numpy().view(np.int64)), p


def test_slice_order_changes_no_bits(tmp_path):
    """Setup times each SELL product in two slice orders (grid-stride and
    contiguous per block), FP64 products also with the pipelined chain, and
    keeps the fastest form; which warp sums a row, and when its loads are
    issued, must not change a bit.  Solves in fresh processes with every
    product forced into each form (MGR_SELL_ORDER), both precisions, forward
    and transposed, give the same bits."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import numpy as np, torch, sys\n"
        "from paper_2101_11649_gb300 import mgr as M\n"
        "from paper_2101_11649_gb300.synth import make_compositional, make_mimetic\n"
        "for name, s in (('mim', make_mimetic(24, 24, 24)), ('comp', make_compositional(32, 24, 8))):\n"
        "    b = torch.as_tensor(s.rhs, device='cuda')\n"
        "    for p in ('fp64', 'fp32'):\n"
        "        g = M.MGRSolver.from_system(s, precision=p)\n"
        "        for tr in (False, True):\n"
        "            x, info = g.solve(b, rtol=1e-10, transpose=tr)\n"
        "            np.save(sys.argv[1] + f'/{name}_{p}_{tr}.npy', x.cpu().numpy())\n")
    outs = {}
    forms = ("grid", "contig", "grid_pipe", "contig_pipe")
    for order in forms:
        d = tmp_path / order
        d.mkdir()
        env = dict(os.environ, MGR_SELL_ORDER=order)
        subprocess.run([sys.executable, "-c", code, str(d)], env=env, check=True, cwd=root, timeout=900)
        outs[order] = d
    for f in sorted(os.listdir(outs["grid"])):
        a = np.load(outs["grid"] / f)
        for order in forms[1:]:
            b = np.load(outs[order] / f)
            assert np.array_equal(a.view(np.int64), b.view(np.int64)), (f, order)


# ------------------------------------------------------ setup, bit-exact
def _same_csr(a, b, what):
    assert a is not None and b is not None, what
    assert a[3] == b[3], (what, a[3], b[3])
    assert np.array_equal(a[0], b[0]), what + " row_ptr"
    assert np.array_equal(a[1], b[1]), what + " col_idx"
    assert np.array_equal(a[2].view(np.int64), b[2].view(np.int64)), \
        (what + " values", np.max(np.abs(a[2] - b[2])))


@pytest.mark.parametrize("name", list(SMALL))
def test_hierarchy_bit_exact(name):
    s = SMALL[name]()
    g = solver(s, max_coarse=SMALL_COARSE)
    o = oracle_of(s, max_coarse=SMALL_COARSE)
    info = g.info()
    assert info["mgr_levels"] == o.mgr_nlevels
    assert info["amg_levels"] == o.amg_nlevels
    for l in range(s.num_levels + 1):
        _same_csr(g.matrix(0, l, 0), o.mgr_matrix(l, "A"), f"MGR A_{l}")
    for l in range(s.num_levels):
        for w, nm in ((1, "AFF"), (2, "AFC"), (3, "ACF"), (4, "W")):
            _same_csr(g.matrix(0, l, w), o.mgr_matrix(l, nm), f"MGR {nm}_{l}")
        gd, gg = g.mgr_dinv(l)
        od, og = o.mgr_dinv(l)
        assert np.array_equal(gg, og)
        assert np.array_equal(gd.view(np.int64), od.view(np.int64)), f"D^-1 level {l}"
    for k in range(o.amg_nlevels):
        _same_csr(g.matrix(1, k, 0), o.amg_matrix(k, "A"), f"AMG A_{k}")
        if k < o.amg_nlevels - 1:
            _same_csr(g.matrix(1, k, 1), o.amg_matrix(k, "P"), f"AMG P_{k}")
            assert np.array_equal(g.amg_cf(k), o.amg_cf(k)), f"C/F split level {k}"
    _same_frelax_hierarchies(g, o, s)


def _same_frelax_hierarchies(g, o, s):
    """The AMG hierarchies of AMG F-relaxations (MGR_U), level by level."""
    for l in range(s.num_levels):
        nl = o.frelax_amg_nlevels(l)
        assert g.frelax_amg_levels(l) == nl, (l, g.frelax_amg_levels(l), nl)
        for k in range(nl):
            _same_csr(g.matrix(2 + l, k, 0), o.amg_matrix(k, "A", frelax_level=l), f"F-AMG[{l}] A_{k}")
            if k < nl - 1:
                _same_csr(g.matrix(2 + l, k, 1), o.amg_matrix(k, "P", frelax_level=l),
                          f"F-AMG[{l}] P_{k}")
                assert np.array_equal(g.amg_cf(k, frelax_level=l), o.amg_cf(k, frelax_level=l))


@pytest.mark.parametrize("name", list(SMALL))
@pytest.mark.parametrize("restrict", ["injection", "jacobi"])
def test_hierarchy_index_structure(name, restrict):
    """Every index array of the built hierarchy lies inside the array it
    indexes, and consecutive operators have matching shapes (the device-side
    check that stands in for a memory checker)."""
    s = SMALL[name]()
    if restrict == "jacobi" and "block_jacobi" in s.relax:
        pytest.skip("the restriction of Eq. 5 takes a diagonal D")
    for prec in ("fp64", "fp32"):
        g = solver(s, precision=prec, max_coarse=SMALL_COARSE, restrict=[restrict] * s.num_levels)
        assert g.check() == 0


# -------------------------------------------------------- V-cycle, solve
@pytest.mark.parametrize("name", list(SMALL))
def test_vcycle_parity(name):
    s = SMALL[name]()
    g = solver(s, max_coarse=SMALL_COARSE)
    o = oracle_of(s, max_coarse=SMALL_COARSE)
    rng = np.random.default_rng(5)
    for trans in (False, True):
        v = rng.standard_normal(s.n)
        zg = g.apply(t(v), transpose=trans).cpu().numpy()
        zo = o.apply_transpose(v) if trans else o.apply(v)
        cycle_close(s, zg, zo, 1e-11, f"trans={trans}")


# Coarsest AMG grids that stay large under the default coarsest size (1024):
# the GPU inverts them in panels of 16 columns (a ragged last panel for 924,
# 969 and 759 rows; 1024 is the largest size that takes the blocked form),
# the oracle factors them (LU, partial pivoting).
LARGE_COARSEST = {
    "two_phase_924": lambda: make_two_phase(12, 11, 7),
    "mimetic_969": lambda: make_mimetic(10, 10, 10),
    "compositional_1024": lambda: make_compositional(16, 16, 4),
    "poromech_759": lambda: make_poromech(10, 5),
}


@pytest.mark.parametrize("name", list(LARGE_COARSEST))
def test_vcycle_parity_large_coarsest_grid(name):
    s = LARGE_COARSEST[name]()
    g = solver(s)
    o = oracle_of(s)
    assert g.info()["amg_levels"] == o.amg_nlevels
    k = o.amg_nlevels - 1
    _same_csr(g.matrix(1, k, 0), o.amg_matrix(k, "A"), f"AMG A_{k}")
    rp, ci, v, (nc, _) = o.amg_matrix(k)
    assert 700 <= nc <= 1024
    dense = np.zeros((nc, nc))
    for i in range(nc):
        dense[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    # an explicit inverse and an LU solve, both backward stable with partial
    # pivoting, agree to a small multiple of eps * cond(A_c) on the coarse
    # correction
    tol = max(1e-11, 64 * np.finfo(np.float64).eps * np.linalg.cond(dense))
    rng = np.random.default_rng(11)
    for trans in (False, True):
        v0 = rng.standard_normal(s.n)
        zg = g.apply(t(v0), transpose=trans).cpu().numpy()
        zo = o.apply_transpose(v0) if trans else o.apply(v0)
        cycle_close(s, zg, zo, tol, f"trans={trans}")


@pytest.mark.parametrize("name", ["poromech_mgr_u", "two_phase_amg_relax"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("sweeps,omega", [(2, 0.8), (3, 1.0)])
def test_amg_frelax_sweeps_and_weight(name, precision, sweeps, omega):
    """Repeated and weighted AMG F-relaxation sweeps, forward and transposed
    cycle.  FP32 hierarchies against the FP64 oracle within 1e-4."""
    s = SMALL[name]()
    g = solver(s, precision=precision, max_coarse=SMALL_COARSE, sweeps=[sweeps], weights=[omega])
    o = oracle_of(s, max_coarse=SMALL_COARSE, sweeps=[sweeps], weights=[omega])
    tol = 1e-11 if precision == "fp64" else 1e-4
    rng = np.random.default_rng(9)
    for trans in (False, True):
        v = rng.standard_normal(s.n)
        zg = g.apply(t(v), transpose=trans).cpu().numpy()
        zo = o.apply_transpose(v) if trans else o.apply(v)
        cycle_close(s, zg, zo, tol, f"trans={trans}")


@pytest.mark.parametrize("name", ["poromech_mgr_u", "two_phase_amg_relax", "compositional_4level"])
@pytest.mark.parametrize("restrict", ["injection", "jacobi"])
def test_amg_frelax_single_level_hierarchy(name, restrict):
    """AMG F-relaxations whose A_FF is small enough to be the coarsest grid
    (one dense level, no SELL copy shared with the hierarchy): cycle parity
    forward and transposed, and solve parity."""
    s = SMALL[name]()
    rs = [restrict] * s.num_levels
    g = solver(s, max_coarse=4096, restrict=rs)
    o = oracle_of(s, max_coarse=4096, restrict=rs)
    for l in range(s.num_levels):
        if s.relax[l] == "amg":
            assert g.frelax_amg_levels(l) == o.frelax_amg_nlevels(l) == 1
    rng = np.random.default_rng(31)
    for trans in (False, True):
        v = rng.standard_normal(s.n)
        zg = g.apply(t(v), transpose=trans).cpu().numpy()
        zo = o.apply_transpose(v) if trans else o.apply(v)
        cycle_close(s, zg, zo, 1e-11, f"trans={trans}")
    ro = o.solve(s.rhs, rtol=1e-10, maxit=300)
    _, ig = g.solve(t(s.rhs), rtol=1e-10, maxit=300)
    assert ig["status"] == 0 and abs(ig["iterations"] - ro["iters"]) <= 1


def test_mgr_u_fewer_iterations_than_mgr_p_on_gpu():
    """The MGR_U strategy (AMG F-relaxation of the displacement) converges in
    fewer FGMRES iterations than MGR_P on the same fracture system."""
    its = {}
    for strat in ("mgr_p", "mgr_u"):
        s = make_poromech(16, 8, strategy=strat)
        _, info = solver(s).solve(t(s.rhs), rtol=1e-8)
        assert info["status"] == 0
        its[strat] = info["iterations"]
    assert its["mgr_u"] < its["mgr_p"], its


# the restriction of Eq. 5 (R = [-A_CF D^-1, I]) on every level
RESTRICT_CASES = ["two_phase", "mimetic", "poromech", "poromech_mgr_u", "compositional_4level"]


@pytest.mark.parametrize("name", RESTRICT_CASES)
def test_jacobi_restriction_hierarchy_bit_exact(name):
    s = SMALL[name]()
    rs = ["jacobi"] * s.num_levels
    g = solver(s, max_coarse=SMALL_COARSE, restrict=rs)
    o = oracle_of(s, max_coarse=SMALL_COARSE, restrict=rs)
    assert g.info()["amg_levels"] == o.amg_nlevels
    for l in range(s.num_levels + 1):
        _same_csr(g.matrix(0, l, 0), o.mgr_matrix(l, "A"), f"MGR A_{l}")
    for l in range(s.num_levels):
        _same_csr(g.matrix(0, l, 5), o.mgr_matrix(l, "Z"), f"MGR Z_{l}")
    for k in range(o.amg_nlevels):
        _same_csr(g.matrix(1, k, 0), o.amg_matrix(k, "A"), f"AMG A_{k}")
    _same_frelax_hierarchies(g, o, s)


@pytest.mark.parametrize("name", RESTRICT_CASES)
@pytest.mark.parametrize("sweeps,omega", [(1, 1.0), (2, 0.8)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_jacobi_restriction_vcycle_parity(name, sweeps, omega, precision):
    s = SMALL[name]()
    nl = s.num_levels
    kw = dict(max_coarse=SMALL_COARSE, restrict=["jacobi"] * nl, sweeps=[sweeps] * nl,
              weights=[omega] * nl)
    g = solver(s, precision=precision, **kw)
    o = oracle_of(s, **kw)
    tol = 1e-11 if precision == "fp64" else 1e-4
    rng = np.random.default_rng(21)
    for trans in (False, True):
        v = rng.standard_normal(s.n)
        zg = g.apply(t(v), transpose=trans).cpu().numpy()
        zo = o.apply_transpose(v) if trans else o.apply(v)
        cycle_close(s, zg, zo, tol, f"trans={trans}")


@pytest.mark.parametrize("name", RESTRICT_CASES)
def test_jacobi_restriction_solve_parity(name):
    s = SMALL[name]()
    rs = ["jacobi"] * s.num_levels
    g = solver(s, max_coarse=SMALL_COARSE, restrict=rs)
    o = oracle_of(s, max_coarse=SMALL_COARSE, restrict=rs)
    ro = o.solve(s.rhs, rtol=1e-8, maxit=500)
    xg, ig = g.solve(t(s.rhs), rtol=1e-8, maxit=500)
    assert ig["status"] == 0 and ro["status"] == 0
    assert abs(ig["iterations"] - ro["iters"]) <= 1, (ig["iterations"], ro["iters"])
    xl, il = g.solve(t(s.rhs), rtol=1e-8, maxit=500, transpose=True)
    rl = o.solve(s.rhs, rtol=1e-8, maxit=500, trans=True)
    assert il["status"] == 0 and abs(il["iterations"] - rl["iters"]) <= 1


def test_jacobi_restriction_rejected_with_block_jacobi():
    s = SMALL["compositional"]()
    with pytest.raises(M.MGRError) as e:
        solver(s, restrict=["jacobi", "injection"])
    assert e.value.status == M.MGR_ERR_UNSUPPORTED
    with pytest.raises(M.MGRError) as e:
        M.MGRBatch([s, s], restrict=["jacobi", "injection"])
    assert e.value.status == M.MGR_ERR_UNSUPPORTED


@pytest.mark.parametrize("name", list(SMALL))
def test_solve_parity(name):
    s = SMALL[name]()
    g = solver(s, max_coarse=SMALL_COARSE)
    o = oracle_of(s, max_coarse=SMALL_COARSE)
    ro = o.solve(s.rhs, rtol=1e-8)
    xg, ig = g.solve(t(s.rhs), rtol=1e-8)
    assert ig["status"] == 0 and ro["status"] == 0
    assert abs(ig["iterations"] - ro["iters"]) <= 1, (ig["iterations"], ro["iters"])
    assert ig["rel_residual"] <= 1e-8
    # solutions when both are converged tightly
    ro = o.solve(s.rhs, rtol=1e-12, maxit=1000)
    xg, ig = g.solve(t(s.rhs), rtol=1e-12, maxit=1000)
    xo = ro["x"]
    assert np.linalg.norm(xg.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)
    cycle_close(s, xg.cpu().numpy(), xo, 1e-8, "solution")


@pytest.mark.parametrize("name", list(SMALL))
def test_fp32_preconditioner_reaches_fp64_tolerance(name):
    s = SMALL[name]()
    g = solver(s, precision="fp32", max_coarse=SMALL_COARSE)
    o = oracle_of(s, max_coarse=SMALL_COARSE)
    xg, ig = g.solve(t(s.rhs), rtol=1e-8)
    assert ig["status"] == 0 and ig["rel_residual"] <= 1e-8
    ro = o.solve(s.rhs, rtol=1e-8)
    assert ig["iterations"] <= ro["iters"] + 3
    # error against the FP64 oracle solution (both at 1e-8 residual)
    xo = ro["x"]
    rel = np.linalg.norm(xg.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert rel <= 1e-5, rel
    cycle_close(s, xg.cpu().numpy(), xo, 1e-5, "fp32 solution")


def test_transpose_solve_and_gradient():
    s = make_two_phase(6, 5, 4)
    g = solver(s, max_coarse=SMALL_COARSE)
    o = oracle_of(s, max_coarse=SMALL_COARSE)
    gvec = np.random.default_rng(9).standard_normal(s.n)
    lam, info = g.solve(t(gvec), rtol=1e-12, transpose=True)
    ro = o.solve(gvec, rtol=1e-12, trans=True)
    assert info["status"] == 0
    assert np.linalg.norm(lam.cpu().numpy() - ro["x"]) <= 1e-8 * np.linalg.norm(ro["x"])
    x, _ = g.solve(t(s.rhs), rtol=1e-12)
    dA = g.grad_values(lam, x).cpu().numpy()
    lam_n, x_n = lam.cpu().numpy(), x.cpu().numpy()
    b = s.b
    for p in range(0, s.nnzb, 7):
        I = np.searchsorted(s.row_ptr, p, side="right") - 1
        J = s.col_idx[p]
        ref = -np.outer(lam_n[I * b:(I + 1) * b], x_n[J * b:(J + 1) * b])
        assert np.array_equal(dA[p], ref)


# ------------------------------------------------------------ edge cases
def test_invalid_inputs_are_rejected():
    s = make_two_phase(3, 3, 2)
    # unsorted columns
    ci = s.col_idx.copy(); ci[[0, 1]] = ci[[1, 0]]
    with pytest.raises(M.MGRError) as e:
        M.MGRSolver(s.row_ptr, ci, s.val, s.b, s.dof_level, s.num_levels)
    assert e.value.status == M.MGR_ERR_INVALID
    # NaN value
    v = s.val.copy(); v[3, 0, 1] = np.nan
    with pytest.raises(M.MGRError) as e:
        M.MGRSolver(s.row_ptr, s.col_idx, v, s.b, s.dof_level, s.num_levels)
    assert e.value.status == M.MGR_ERR_INVALID
    # empty C set
    with pytest.raises(M.MGRError) as e:
        M.MGRSolver(s.row_ptr, s.col_idx, s.val, s.b, np.zeros(s.n, np.int8), 1)
    assert e.value.status == M.MGR_ERR_INVALID
    # label out of range
    with pytest.raises(M.MGRError) as e:
        M.MGRSolver(s.row_ptr, s.col_idx, s.val, s.b, np.full(s.n, 3, np.int8), 1)
    assert e.value.status == M.MGR_ERR_INVALID


def test_singular_f_block_reports_singular():
    s = make_two_phase(3, 3, 2)
    v = s.val.copy()
    # zero the saturation diagonal of block row 4 (an F point under Jacobi)
    diag = [p for p in range(s.row_ptr[4], s.row_ptr[5]) if s.col_idx[p] == 4][0]
    v[diag, 1, 1] = 0.0
    with pytest.raises(M.MGRError) as e:
        M.MGRSolver(s.row_ptr, s.col_idx, v, s.b, s.dof_level, s.num_levels,
                    M.options(relax=("jacobi",)))
    assert e.value.status == M.MGR_ERR_SINGULAR
    assert "dof 9" in str(e.value), str(e.value)   # block row 4, second unknown


def test_tail_barrier_timeout_is_reported_and_the_context_survives():
    """A grid-barrier wait of the fused AMG tail that runs out (forced with a
    spin limit of one poll) ends the kernel, and the solve reports
    MGR_ERR_TIMEOUT; the next solve on a handle with the default limit
    converges normally."""
    s = TAIL_SYSTEMS["mimetic24"]()
    g = solver(s, tail_nnz=400000, spin_limit=1)
    x = torch.zeros(s.n, dtype=torch.float64, device=DEV)
    _, info = g.solve(t(s.rhs), x, rtol=1e-8, maxit=3, check=False)
    assert info["status"] == M.MGR_ERR_TIMEOUT, info
    # the solve stops at the first step whose tail gave up, and the broken
    # preconditioner output never reaches x
    assert info["iterations"] == 1 and float(x.abs().max()) == 0.0
    # a single cycle reports the timeout too, in both orientations
    v = t(np.random.default_rng(3).standard_normal(s.n))
    for trans in (False, True):
        with pytest.raises(M.MGRError) as e:
            g.apply(v, transpose=trans)
        assert e.value.status == M.MGR_ERR_TIMEOUT
    ok = solver(s, tail_nnz=400000)
    _, info2 = ok.solve(t(s.rhs), rtol=1e-8)
    assert info2["status"] == 0 and info2["rel_residual"] <= 1e-8


@pytest.mark.parametrize("name", ["two_phase", "poromech_mgr_u"])
def test_solve_history_matches_oracle(name):
    """The residual history of a solve (initial true residual, then the
    Arnoldi estimate per iteration) against the oracle's."""
    s = SMALL[name]()
    g = solver(s, max_coarse=SMALL_COARSE)
    o = oracle_of(s, max_coarse=SMALL_COARSE)
    _, ig = g.solve(t(s.rhs), rtol=1e-10, maxit=300)
    ro = o.solve(s.rhs, rtol=1e-10, maxit=300)
    hg, ho = g.history(), ro["hist"]
    assert hg.size == ig["iterations"] + 1 and ho.size == ro["iters"] + 1
    assert hg[0] == pytest.approx(1.0) and ho[0] == pytest.approx(1.0)
    k = min(hg.size, ho.size)
    assert np.all(np.abs(hg[:k] - ho[:k]) <= 1e-6 * ho[:k] + 1e-14), np.max(np.abs(hg[:k] - ho[:k]) / ho[:k])
    assert np.all(np.diff(hg[1:]) <= 1e-12)   # GMRES residual estimates never increase within a cycle


def test_maxit_and_zero_rhs():
    s = make_two_phase(6, 6, 3)
    g = solver(s)
    x, info = g.solve(t(s.rhs), rtol=1e-12, maxit=2)
    assert info["status"] == M.MGR_ERR_NOT_CONVERGED and info["iterations"] == 2
    x, info = g.solve(torch.zeros(s.n, dtype=torch.float64, device=DEV), rtol=1e-8)
    assert info["status"] == 0 and info["iterations"] == 0 and float(x.abs().max()) == 0.0


def test_single_block_system():
    from paper_2101_11649_gb300.synth.bsr import BlockSystem
    val = np.array([[[4.0, 1.0], [2.0, 3.0]]])
    s = BlockSystem("one", 2, np.array([0, 1], np.int32), np.array([0], np.int32), val,
                    np.array([1, 0], np.int8), 1, np.array([1.0, 2.0]), relax=["jacobi"])
    g = solver(s)
    x, info = g.solve(t(s.rhs), rtol=1e-12)
    assert info["status"] == 0
    assert np.allclose(x.cpu().numpy(), np.linalg.solve(val[0], s.rhs), rtol=1e-12)


def test_repeat_solves_bitwise_identical():
    s = SMALL["mimetic"]()
    g = solver(s)
    x1, i1 = g.solve(t(s.rhs), rtol=1e-10)
    x2, i2 = g.solve(t(s.rhs), rtol=1e-10)
    assert i1["iterations"] == i2["iterations"]
    assert torch.equal(x1, x2)


# ------------------------------------------------ full-size configurations
FULL = ["mimetic_64", "mimetic_64_tpfa_mgr_pi", "compositional_128x128x32", "compositional_128x128x32_4level", "poromech_64",
        "poromech_64_mgr_u"]


@pytest.mark.slow
@pytest.mark.parametrize("name", FULL)
def test_full_size(name):
    """The large configurations at their full sizes (mimetic 64^3: 1,060,864
    unknowns; compositional 128x128x32 with wells: 2,097,216; poromechanics
    64^3 with a fracture plane: 826,179): bit-exact hierarchy on every MGR and
    AMG level, the outer SpMV entry by entry, one V-cycle, iteration parity
    and the true residual of both precisions."""
    from paper_2101_11649_gb300.synth import CONFIGS
    s = CONFIGS[name]()
    g = solver(s)
    o = O.Oracle(s)
    assert g.info()["mgr_levels"] == o.mgr_nlevels and g.info()["amg_levels"] == o.amg_nlevels
    assert g.check() == 0
    for l in range(s.num_levels + 1):
        _same_csr(g.matrix(0, l, 0), o.mgr_matrix(l, "A"), f"MGR A_{l}")
    for k in range(o.amg_nlevels):
        _same_csr(g.matrix(1, k, 0), o.amg_matrix(k, "A"), f"AMG A_{k}")
    for l in range(s.num_levels):
        assert g.frelax_amg_levels(l) == o.frelax_amg_nlevels(l)
        for k in range(o.frelax_amg_nlevels(l)):
            _same_csr(g.matrix(2 + l, k, 0), o.amg_matrix(k, "A", frelax_level=l), f"F-AMG[{l}] A_{k}")
    rng = np.random.default_rng(1)
    x = rng.standard_normal(s.n)
    y = g.spmv(t(x)).cpu().numpy()
    ref = O.spmv_bsr(s.nb, s.b, s.row_ptr, s.col_idx, s.val, x)
    absref = O.spmv_bsr(s.nb, s.b, s.row_ptr, s.col_idx, np.abs(s.val), np.abs(x)) + 1e-300
    assert (np.abs(y - ref) / absref).max() <= 1e-13
    v = rng.standard_normal(s.n)
    zg = g.apply(t(v)).cpu().numpy()
    zo = o.apply(v)
    cycle_close(s, zg, zo, 1e-11, "fp64")
    # the FP32 cycle entry by entry against the FP64 oracle
    z32 = solver(s, precision="fp32").apply(t(v)).cpu().numpy()
    cycle_close(s, z32, zo, 1e-4, "fp32")
    ro = o.solve(s.rhs, rtol=1e-8)
    bn = np.linalg.norm(s.rhs)
    for prec in ("fp64", "fp32"):
        gp = g if prec == "fp64" else solver(s, precision=prec)
        xg, info = gp.solve(t(s.rhs), rtol=1e-8)
        assert info["status"] == 0 and info["rel_residual"] <= 1e-8
        r = s.rhs - O.spmv_bsr(s.nb, s.b, s.row_ptr, s.col_idx, s.val, xg.cpu().numpy())
        assert np.linalg.norm(r) <= 1.01e-8 * bn
        if prec == "fp64":
            assert abs(info["iterations"] - ro["iters"]) <= 1, (info["iterations"], ro["iters"])
