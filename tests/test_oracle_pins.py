"""Pins of the CPU oracle to what the paper and the mathematics fix.

Each test checks the oracle against an independent fact (a dense definition,
a closed form, a published test vector, an invariant), never against a
retyped copy of its own formula.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_11649_gb300.synth import (make_compositional, make_mimetic, make_poromech,
                                          make_two_phase)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_of(sysm):
    """Dense matrix of a BlockSystem from its blocks (numpy only)."""
    n, b = sysm.n, sysm.b
    A = np.zeros((n, n))
    for I in range(sysm.nb):
        for p in range(sysm.row_ptr[I], sysm.row_ptr[I + 1]):
            J = sysm.col_idx[p]
            A[I * b:(I + 1) * b, J * b:(J + 1) * b] += sysm.val[p]
    return A


def csr_dense(m):
    rp, ci, v, (n, mm) = m
    A = np.zeros((n, mm))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] += v[rp[i]:rp[i + 1]]
    return A


def random_bsr(nb, b, density, rng, empty_rows=()):
    rows, cols = [], []
    for i in range(nb):
        if i in empty_rows:
            continue
        js = np.flatnonzero(rng.random(nb) < density)
        rows += [i] * len(js); cols += list(js)
    from paper_2101_11649_gb300.synth.bsr import assemble_bsr
    blocks = rng.standard_normal((len(rows), b, b))
    return assemble_bsr(nb, b, np.array(rows, np.int64), np.array(cols, np.int64), blocks)


# ---------------------------------------------------------------- SpMV
@pytest.mark.parametrize("b", [1, 2, 3, 4])
def test_spmv_matches_dense(b):
    rng = np.random.default_rng(b)
    nb = 37
    rp, ci, val = random_bsr(nb, b, 0.15, rng, empty_rows=(0, 5, 36))
    x = rng.standard_normal(nb * b)
    y = O.spmv_bsr(nb, b, rp, ci, val, x)
    A = np.zeros((nb * b, nb * b))
    for I in range(nb):
        for p in range(rp[I], rp[I + 1]):
            A[I * b:(I + 1) * b, ci[p] * b:(ci[p] + 1) * b] = val[p]
    ref = A @ x
    scale = np.abs(A) @ np.abs(x) + 1e-300
    assert np.max(np.abs(y - ref) / scale) < 1e-14
    sp = pytest.importorskip("scipy.sparse")
    Bs = sp.bsr_matrix((val, ci, rp), shape=A.shape)
    assert np.max(np.abs(y - Bs @ x) / scale) < 1e-14


def test_dense_lu_matches_numpy():
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 50, 200):
        A = rng.standard_normal((n, n)) + n * 0.1 * np.eye(n)
        bb = rng.standard_normal(n)
        x = O.dense_solve(A, bb)
        ref = np.linalg.solve(A, bb)
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref) * max(1, np.linalg.cond(A) / 1e3)


# --------------------------------------------------- reduced operator (Eq. 2, 4)
def test_reduced_operator_is_schur_complement_diagonal_F():
    """A_FF diagonal (MGR_P on the mimetic system, Eq. 9): the coarse
    operator A_CC - A_CF D^{-1} A_FC is the exact Schur complement of Eq. 2."""
    s = make_mimetic(5, 4, 3)
    o = O.Oracle(s)
    A = dense_of(s)
    F = np.flatnonzero(s.dof_level == 0); Cc = np.flatnonzero(s.dof_level == 1)
    AFF = A[np.ix_(F, F)]
    assert np.count_nonzero(AFF - np.diag(np.diag(AFF))) == 0
    S = A[np.ix_(Cc, Cc)] - A[np.ix_(Cc, F)] @ np.linalg.solve(AFF, A[np.ix_(F, Cc)])
    got = csr_dense(o.mgr_matrix(1, "A"))
    assert np.max(np.abs(got - S)) <= 1e-13 * np.max(np.abs(S))
    # W = -D^{-1} A_FC, the Jacobi interpolation block of Eq. 4
    W = csr_dense(o.mgr_matrix(0, "W"))
    assert np.max(np.abs(W + np.diag(1 / np.diag(AFF)) @ A[np.ix_(F, Cc)])) < 1e-13 * np.abs(W).max()


def test_reduced_operator_block_jacobi_wells_exact():
    """Level 1 of the compositional system eliminates the wells with exact
    2x2 block inverses; wells do not couple, so A_FF is block-diagonal and
    the reduced operator is the exact Schur complement, including the
    zero-diagonal pressure-controlled wells (Sec. 4.2)."""
    s = make_compositional(8, 8, 3, nwell_side=2)
    o = O.Oracle(s)
    A1 = csr_dense(o.mgr_matrix(1, "A"))
    lvl1 = s.dof_level[s.dof_level >= 1]
    F = np.flatnonzero(lvl1 == 1); Cc = np.flatnonzero(lvl1 == 2)
    AFF = A1[np.ix_(F, F)]
    assert (np.abs(np.diag(AFF)) == 0).any(), "expected zero diagonals from BHP wells"
    S = A1[np.ix_(Cc, Cc)] - A1[np.ix_(Cc, F)] @ np.linalg.solve(AFF, A1[np.ix_(F, Cc)])
    got = csr_dense(o.mgr_matrix(2, "A"))
    assert np.max(np.abs(got - S)) <= 1e-12 * np.max(np.abs(S))


def test_block_jacobi_inverse_blocks():
    s = make_compositional(4, 4, 2, nwell_side=2)
    o = O.Oracle(s)
    d, g = o.mgr_dinv(0)
    AFF = csr_dense(o.mgr_matrix(0, "AFF"))
    f = 0
    while f < g.size:
        k = g[f]
        inv = np.linalg.inv(AFF[f:f + k, f:f + k])
        assert np.allclose(d[f:f + k, :k], inv, rtol=1e-12, atol=1e-14 * np.abs(inv).max())
        f += k


# ------------------------------------------------ MGR as a direct solver
def test_two_level_mgr_is_direct_solver():
    """Exact F solve (diagonal A_FF, one Jacobi sweep) + exact coarse solve
    (dense LU) make the V-cycle equal A^{-1} (LDU of Eq. 2), so FGMRES
    converges in one iteration."""
    s = make_mimetic(4, 4, 4)
    assert (s.dof_level == 1).sum() <= 256
    o = O.Oracle(s)
    assert o.amg_nlevels == 1
    A = dense_of(s)
    v = np.random.default_rng(0).standard_normal(s.n)
    z = o.apply(v)
    ref = np.linalg.solve(A, v)
    assert np.linalg.norm(z - ref) <= 1e-10 * np.linalg.norm(ref)
    r = o.solve(s.rhs, rtol=1e-12)
    assert r["status"] == 0 and r["iters"] == 1 and r["relres"] <= 1e-12


def test_extra_sweeps_on_diagonal_F_level_change_nothing():
    """A diagonal F block is solved exactly by one Jacobi sweep (Sec. 4.2,
    the rho_2 level); further sweeps leave z unchanged."""
    s = make_mimetic(4, 3, 3)
    v = np.random.default_rng(1).standard_normal(s.n)
    z1 = O.Oracle(s, O.Options(relax=["jacobi"], sweeps=[1])).apply(v)
    z3 = O.Oracle(s, O.Options(relax=["jacobi"], sweeps=[3])).apply(v)
    assert np.max(np.abs(z1 - z3)) <= 1e-13 * np.max(np.abs(z1))


# ----------------------------------------------------------- FGMRES
def _ls_residual(A, r0, basis):
    Q, _ = np.linalg.qr(basis)
    y, *_ = np.linalg.lstsq(A @ Q, r0, rcond=None)
    return np.linalg.norm(r0 - A @ Q @ y)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_fgmres_minimises_residual_over_krylov_space(k):
    """Unpreconditioned: x_k minimises ||b - A x|| over x0 + K_k(A, r0)."""
    rng = np.random.default_rng(k)
    s = make_two_phase(4, 3, 2)
    A = dense_of(s)
    o = O.Oracle(s)
    b = rng.standard_normal(s.n)
    r = o.solve(b, rtol=1e-30, maxit=k, precond=False)
    basis = np.stack([np.linalg.matrix_power(A, t) @ b for t in range(k)], 1)
    best = _ls_residual(A, b, basis)
    got = np.linalg.norm(b - A @ r["x"])
    assert abs(got - best) <= 1e-9 * np.linalg.norm(b)


def test_right_preconditioned_fgmres_minimises_over_preconditioned_space():
    """With the fixed MGR preconditioner M, x_k minimises the residual over
    span{M^{-1} r0, M^{-1}(A M^{-1}) r0, ...} (right preconditioning)."""
    s = make_two_phase(6, 5, 2)
    A = dense_of(s)
    o = O.Oracle(s)
    Minv = np.stack([o.apply(e) for e in np.eye(s.n)], 1)
    b = s.rhs
    k = 4
    r = o.solve(b, rtol=1e-30, maxit=k)
    AM = A @ Minv
    basis = np.stack([Minv @ np.linalg.matrix_power(AM, t) @ b for t in range(k)], 1)
    best = _ls_residual(A, b, basis)
    assert abs(np.linalg.norm(b - A @ r["x"]) - best) <= 1e-9 * np.linalg.norm(b)


def test_fgmres_restart_converges_true_residual():
    s = make_two_phase(8, 8, 4)
    o = O.Oracle(s)
    r = o.solve(s.rhs, rtol=1e-10, restart=3, maxit=200)
    A = dense_of(s)
    assert r["status"] == 0
    assert np.linalg.norm(s.rhs - A @ r["x"]) <= 1e-10 * np.linalg.norm(s.rhs)


# ---------------------------------------------------------------- AMG
def poisson(nx, ny=1, nz=1, periodic=False):
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    dims = [(nx, 2), (ny, 1), (nz, 0)]
    for size, ax in dims:
        if size == 1:
            continue
        a = idx; b = np.roll(idx, -1, axis=ax)
        if not periodic:
            sl = [slice(None)] * 3; sl[ax] = slice(0, size - 1)
            a = a[tuple(sl)]; b = b[tuple(sl)]
        a = a.ravel(); b = b.ravel()
        rows += [a, b, a, b]; cols += [b, a, a, b]
        vals += [-np.ones(a.size), -np.ones(a.size), np.ones(a.size), np.ones(a.size)]
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    if not periodic:  # Dirichlet: add the missing neighbours to the diagonal
        deg = 2 * sum(1 for s_, _ in dims if s_ > 1)
        cnt = np.bincount(rows[rows != cols], minlength=n)
        rows = np.concatenate([rows, np.arange(n)]); cols = np.concatenate([cols, np.arange(n)])
        vals = np.concatenate([vals, (deg - cnt).astype(float)])
    from paper_2101_11649_gb300.synth.bsr import assemble_bsr
    rp, ci, v = assemble_bsr(n, 1, rows, cols, vals)
    return rp, ci, v.ravel()


def test_splitmix64_published_vectors():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    outs = [int(h, 16) for h in g["outputs_seed0"]]
    gamma = int(g["golden_gamma"], 16)
    # output 1: state gamma  <- i = 0, level = 0
    assert O.pmis_u01(0, 0) == (outs[0] >> 11) * 2.0 ** -53
    # output 2: state 2*gamma = gamma + gamma -> i + 2^32 level = gamma
    assert O.pmis_u01(gamma & 0xFFFFFFFF, gamma >> 32) == (outs[1] >> 11) * 2.0 ** -53


def test_strength_hand_example():
    # row 0: a00 = 4, a01 = -1, a02 = -0.2 (0.2 < 0.25 * 1: weak), a03 = +3 (positive: weak)
    rp = np.array([0, 4, 5, 6, 7]); ci = np.array([0, 1, 2, 3, 1, 2, 3])
    v = np.array([4.0, -1.0, -0.2, 3.0, 1.0, 1.0, 1.0])
    srp, sci = O.amg_strength(rp, ci, v)
    assert list(sci[srp[0]:srp[1]]) == [1]
    # negative diagonal flips the sign test
    v2 = v.copy(); v2[0] = -4.0
    srp, sci = O.amg_strength(rp, ci, v2)
    assert list(sci[srp[0]:srp[1]]) == [3]


def _strength_sets(rp, ci, v):
    srp, sci = O.amg_strength(rp, ci, v)
    n = rp.size - 1
    S = [set(sci[srp[i]:srp[i + 1]]) for i in range(n)]
    ST = [set() for _ in range(n)]
    for i in range(n):
        for j in S[i]:
            ST[j].add(i)
    return S, ST


@pytest.mark.parametrize("shape", [(30, 1, 1), (12, 11, 1), (7, 6, 5)])
def test_pmis_independent_and_covering(shape):
    rp, ci, v = poisson(*shape)
    cf, P = O.amg_split_interp(rp, ci, v)
    S, ST = _strength_sets(rp, ci, v)
    C = set(np.flatnonzero(cf == 1))
    for i in C:  # independence in the symmetrised strength graph
        assert not (S[i] | ST[i]) & C
    for i in np.flatnonzero(cf == -1):  # every F point either influences nobody or depends on a C point
        assert len(ST[i]) == 0 or (S[i] & C)
    assert set(np.unique(cf)) <= {-1, 1}


def _random_2d_coupling(nx, ny, seed):
    """Symmetric 2D 5-point M-matrix with couplings U(0.05, 1): some
    connections fall below theta * max and are weak; rows sum to U(0.05, 0.5)."""
    rng = np.random.default_rng(seed)
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    pairs = [(idx[:, :-1].ravel(), idx[:, 1:].ravel()), (idx[:-1, :].ravel(), idx[1:, :].ravel())]
    a = np.concatenate([p[0] for p in pairs]); b = np.concatenate([p[1] for p in pairs])
    w = rng.uniform(0.05, 1.0, a.size)
    diag = np.bincount(a, w, n) + np.bincount(b, w, n) + rng.uniform(0.05, 0.5, n)
    rows = np.concatenate([a, b, np.arange(n)]); cols = np.concatenate([b, a, np.arange(n)])
    from paper_2101_11649_gb300.synth.bsr import assemble_bsr
    rp, ci, v = assemble_bsr(n, 1, rows, cols, np.concatenate([-w, -w, diag]))
    return rp, ci, v.ravel()


@pytest.mark.parametrize("case", ["poisson2d", "random2d", "poisson3d"])
def test_pmis_first_round_from_the_published_measure(case):
    """PMIS (De Sterck, Yang & Heys 2006) with measure w_i = |S^T_i| + u_i,
    u_i the published SplitMix64 draw: a point that influences nobody is F;
    every other point whose measure beats those of all its strong neighbours
    that influence somebody (S_i u S^T_i; ties to the larger index) is
    selected in the first round, so it is C, and every point that strongly
    depends on such a point is F.  Catches a measure built from |S_i|, a
    reversed comparison, or another random stream."""
    rp, ci, v = {"poisson2d": lambda: poisson(13, 11), "random2d": lambda: _random_2d_coupling(17, 13, 3),
                 "poisson3d": lambda: poisson(7, 6, 5)}[case]()
    cf, _ = O.amg_split_interp(rp, ci, v)
    S, ST = _strength_sets(rp, ci, v)
    n = rp.size - 1
    w = np.array([len(ST[i]) + O.pmis_u01(i, 0) for i in range(n)])
    first = []
    for i in range(n):
        if not ST[i]:
            assert cf[i] == -1, i
            continue
        rivals = [j for j in (S[i] | ST[i]) if ST[j]]
        if all(w[j] < w[i] or (w[j] == w[i] and j < i) for j in rivals):
            first.append(i)
    assert first
    for i in first:
        assert cf[i] == 1, i
    for i in range(n):
        if S[i] & set(first):
            assert cf[i] == -1, i


def _upwind_2d(nx, ny, seed):
    """Nonsymmetric 2D M-matrix (diffusion plus first-order upwinding of a
    random velocity): S and S^T differ."""
    rng = np.random.default_rng(seed)
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    rows, cols, vals = [], [], []
    for a, b in ((idx[:, :-1].ravel(), idx[:, 1:].ravel()), (idx[:-1, :].ravel(), idx[1:, :].ravel())):
        d = rng.uniform(0.2, 1.0, a.size)
        u = rng.uniform(-3.0, 3.0, a.size)
        rows += [a, b]; cols += [b, a]
        vals += [-(d + np.maximum(-u, 0)), -(d + np.maximum(u, 0))]
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    diag = -np.bincount(rows, vals, n) + rng.uniform(0.05, 0.5, n)
    from paper_2101_11649_gb300.synth.bsr import assemble_bsr
    rp, ci, v = assemble_bsr(n, 1, np.concatenate([rows, np.arange(n)]),
                             np.concatenate([cols, np.arange(n)]), np.concatenate([vals, diag]))
    return rp, ci, v.ravel()


@pytest.mark.parametrize("case", ["poisson2d", "random2d", "upwind2d", "poisson3d"])
def test_pmis_equals_the_sequential_pass_in_measure_order(case):
    """With fixed measures w_i = |S^T_i| + u_i, PMIS's parallel rounds give
    the split of one sequential pass over the points in decreasing measure
    (ties: larger index first): a point that influences nobody is F; any
    other point is F when a point of its S_i already made C, else C.  (A
    point becomes F only through a C point of its S_i that beat it, and is
    selected only once every neighbour above it is decided.)"""
    rp, ci, v = {"poisson2d": lambda: poisson(13, 11), "random2d": lambda: _random_2d_coupling(17, 13, 3),
                 "upwind2d": lambda: _upwind_2d(18, 14, 5), "poisson3d": lambda: poisson(7, 6, 5)}[case]()
    cf, _ = O.amg_split_interp(rp, ci, v)
    S, ST = _strength_sets(rp, ci, v)
    n = rp.size - 1
    w = [len(ST[i]) + O.pmis_u01(i, 0) for i in range(n)]
    status = np.zeros(n, np.int32)
    for i in sorted(range(n), key=lambda i: (w[i], i), reverse=True):
        if not ST[i] or any(status[j] == 1 for j in S[i]):
            status[i] = -1
        else:
            status[i] = 1
    assert np.array_equal(cf, status)


def test_extpi_reduces_to_direct_interpolation_without_strong_f_neighbours():
    """Where every strong neighbour of an F point is a C point, extended+i
    (De Sterck, Falgout, Nolting & Yang 2008) is classical direct
    interpolation with the weak connections lumped into the diagonal:
    w_ij = -a_ij / (a_ii + sum over weak k of a_ik), j in C_i^s."""
    for seed in (3, 4):
        rp, ci, v = _random_2d_coupling(19, 15, seed)
        cf, P = O.amg_split_interp(rp, ci, v, pmax=0)
        S, _ = _strength_sets(rp, ci, v)
        A = np.zeros((rp.size - 1,) * 2)
        for i in range(rp.size - 1):
            A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
        Pd = csr_dense(P)
        cols = np.flatnonzero(cf == 1)          # P's columns: C points in ascending order
        checked = 0
        for i in np.flatnonzero(cf == -1):
            if any(cf[j] == -1 for j in S[i]) or not S[i]:
                continue
            weak = [k for k in np.flatnonzero(A[i]) if k != i and k not in S[i]]
            d = A[i, i] + sum(A[i, k] for k in weak)
            ref = np.zeros(cols.size)
            for j in S[i]:
                ref[np.searchsorted(cols, j)] = -A[i, j] / d
            assert np.allclose(Pd[i], ref, rtol=1e-14, atol=0), i
            checked += 1
        assert checked > 20


def test_extpi_truncation_keeps_the_largest_and_the_row_sum():
    """P_max truncation (BoomerAMG's rule, as the oracle states it): with the
    split unchanged, each row of the truncated interpolation keeps the pmax
    weights of largest magnitude of the untruncated row (ties: lower column),
    rescaled by (sum of all weights) / (sum of kept weights)."""
    for rp, ci, v in (_random_2d_coupling(19, 15, 7), _upwind_2d(18, 14, 9), poisson(9, 8, 6)):
        cf0, P0 = O.amg_split_interp(rp, ci, v, pmax=0)
        cf4, P4 = O.amg_split_interp(rp, ci, v, pmax=4)
        assert np.array_equal(cf0, cf4)
        D0, D4 = csr_dense(P0), csr_dense(P4)
        wide = 0
        for i in range(D0.shape[0]):
            nz = np.flatnonzero(D0[i])
            if nz.size <= 4:
                assert np.array_equal(D0[i], D4[i]), i
                continue
            wide += 1
            order = sorted(nz, key=lambda j: (-abs(D0[i, j]), j))[:4]
            ref = np.zeros_like(D0[i])
            ref[order] = D0[i, order] * (D0[i, nz].sum() / D0[i, order].sum())
            assert np.allclose(D4[i], ref, rtol=1e-13, atol=0), i
        assert wide > 0


def test_extpi_reproduces_constants_zero_row_sum():
    """Extended+i interpolates constants exactly when rows sum to zero (De
    Sterck et al. 2008), with truncation rescaled to keep row sums."""
    for shape in ((9, 8, 1), (6, 5, 4)):
        rp, ci, v = poisson(*shape, periodic=True)
        for pmax in (0, 4):
            cf, P = O.amg_split_interp(rp, ci, v, pmax=pmax)
            Pd = csr_dense(P)
            rows = np.flatnonzero(np.diff(P[0]) > 0)
            assert np.max(np.abs(Pd[rows].sum(1) - 1.0)) < 1e-13
            # C rows are identity rows
            for i in np.flatnonzero(cf == 1):
                nz = np.flatnonzero(Pd[i]); assert nz.size == 1 and Pd[i, nz[0]] == 1.0


def test_extpi_linear_in_1d():
    """1D Laplacian: each F point interpolates linearly between its nearest C
    points on both sides (weights 1/2, or 2/3 and 1/3 across an F-F pair)."""
    g = json.load(open(os.path.join(GOLDEN, "extpi_1d_laplacian.json")))
    rp, ci, v = poisson(40)
    cf, P = O.amg_split_interp(rp, ci, v, pmax=0)
    Pd = csr_dense(P)
    cpts = np.flatnonzero(cf == 1)
    x = np.arange(40.0)
    for i in np.flatnonzero(cf == -1):
        if i < cpts[0] or i > cpts[-1]:
            continue
        assert abs(Pd[i] @ x[cpts] - x[i]) < 1e-13
        left, right = cpts[cpts < i][-1], cpts[cpts > i][0]
        if right - left == 2:
            assert np.allclose(Pd[i][Pd[i] != 0], g["weight"])


def test_galerkin_product_matches_dense():
    s = make_two_phase(8, 6, 3)
    o = O.Oracle(s)
    for k in range(o.amg_nlevels - 1):
        A = csr_dense(o.amg_matrix(k, "A")); P = csr_dense(o.amg_matrix(k, "P"))
        Ac = csr_dense(o.amg_matrix(k + 1, "A"))
        ref = P.T @ A @ P
        assert np.max(np.abs(Ac - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_amg_vcycle_convergence_factor_poisson():
    """Sanity (not exact): AMG V(1,1) with l1-Jacobi on the 7-point Poisson
    problem contracts the residual by < 0.3 per cycle inside GMRES terms."""
    from paper_2101_11649_gb300.synth.bsr import BlockSystem
    rp, ci, v = poisson(14, 13, 12)
    n = rp.size - 1
    s = BlockSystem("poisson", 1, rp, ci, v.reshape(-1, 1, 1), np.zeros(n, np.int8), 0,
                    np.random.default_rng(0).standard_normal(n))
    o = O.Oracle(s, O.Options(relax=[]))
    r = o.solve(s.rhs, rtol=1e-8, maxit=100)
    assert r["status"] == 0
    rate = (r["relres"]) ** (1.0 / r["iters"])
    assert rate < 0.3, rate



def _amg_only(rp, ci, v, rhs=None):
    """A scalar system whose every dof belongs to the final coarse block, so
    the oracle's preconditioner is the AMG V(1,1) cycle alone."""
    from paper_2101_11649_gb300.synth.bsr import BlockSystem
    n = rp.size - 1
    rhs = np.zeros(n) if rhs is None else rhs
    return BlockSystem("amg", 1, rp, ci, v.reshape(-1, 1, 1), np.zeros(n, np.int8), 0, rhs)


def test_amg_l1_smoother_hand_example():
    """The l1-Jacobi smoother of an AMG level (Sec. 5.1 names an l1
    smoother): d_i = a_ii + sign(a_ii) sum_{j != i} |a_ij| over the whole row,
    sign(0) = +1.  Expected 1/d_i worked out by hand: row 1 has a negative
    diagonal, row 2 sums to zero, row 5 couples across the whole grid."""
    from paper_2101_11649_gb300.synth.bsr import assemble_bsr
    A = np.array([[4.0, -1.0, 0.0, 0.0, 0.0, -2.0],
                  [-1.0, -3.0, 0.5, 0.0, 0.0, 0.0],
                  [0.0, -1.0, 2.0, -1.0, 0.0, 0.0],
                  [0.0, 0.0, -1.0, 3.0, -0.5, 0.0],
                  [0.0, 0.0, 0.0, -2.0, 5.0, -1.0],
                  [-0.25, 0.0, 0.0, 0.0, -1.0, 2.0]])
    # d = 4+3, -3-1.5, 2+2, 3+1.5, 5+3, 2+1.25
    expected = np.array([1 / 7, -2 / 9, 1 / 4, 2 / 9, 1 / 8, 4 / 13])
    r, c = np.nonzero(A)
    rp, ci, v = assemble_bsr(6, 1, r, c, A[r, c])
    o = O.Oracle(_amg_only(rp, ci, v.ravel()), O.Options(relax=[], max_coarse=1))
    assert o.amg_nlevels >= 2  # level 0 is smoothed, not the coarsest grid
    np.testing.assert_allclose(o.amg_dinv(0), expected, rtol=1e-15, atol=0)


def _row_l1_inverse(A):
    """1/d_i of the l1 smoother by the reading, from a dense matrix."""
    dg = np.diag(A).copy()
    off = np.abs(A).sum(axis=1) - np.abs(dg)
    return 1.0 / np.where(dg < 0, dg - off, dg + off)


def _vcycle_dense(A, Ps):
    """Dense operator B of the AMG V(1,1) cycle x = B r from x = 0 on A with
    the interpolation matrices Ps (one per level, coarsest solved exactly):
    x1 = D r; x2 = x1 + P B_c P^T (r - A x1); x = x2 + D (r - A x2), with
    B_c the cycle on the Galerkin operator P^T A P and D the l1 inverse
    diagonal of A.  Built from the definitions only."""
    if not Ps:
        return np.linalg.inv(A)
    P = Ps[0]
    D = np.diag(_row_l1_inverse(A))
    Bc = _vcycle_dense(P.T @ A @ P, Ps[1:])
    I = np.eye(A.shape[0])
    X2 = D + P @ Bc @ P.T @ (I - A @ D)
    return X2 + D @ (I - A @ X2)


def _convection_diffusion(nx, ny, seed):
    """2D 5-point diffusion plus an upwinded convection term (nonsymmetric)
    with every third row's sign flipped (negative diagonals)."""
    from paper_2101_11649_gb300.synth.bsr import assemble_bsr
    rp, ci, v = poisson(nx, ny)
    n = rp.size - 1
    rng = np.random.default_rng(seed)
    A = np.zeros((n, n))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    for i in range(n):  # upwind convection to the left neighbour
        if i % nx:
            w = 0.6 * rng.random()
            A[i, i - 1] -= w
            A[i, i] += w
    A[::3] *= -1.0
    r, c = np.nonzero(A)
    rp, ci, v = assemble_bsr(n, 1, r, c, A[r, c])
    return rp, ci, v.ravel(), A


@pytest.mark.parametrize("max_coarse,nfunc", [(150, 1), (40, 1), (40, 2)])
def test_amg_vcycle_equals_dense_multigrid_operator(max_coarse, nfunc):
    """The oracle's AMG V(1,1) cycle, forward and transposed, equals the
    dense composition of its definition (l1 pre-smoothing from zero,
    restriction by P^T, Galerkin coarse operators, exact coarsest solve,
    prolongation, l1 post-smoothing) built in the test from the oracle's
    interpolation matrices alone: two levels (max_coarse 150) and three or
    more (40), with the unknown approach's two functions, on a nonsymmetric
    matrix with negative diagonals."""
    rp, ci, v, A = _convection_diffusion(16, 12, 3)
    o = O.Oracle(_amg_only(rp, ci, v), O.Options(relax=[], max_coarse=max_coarse,
                                                 num_functions=nfunc))
    nl = o.amg_nlevels
    assert nl >= (2 if max_coarse == 150 else 3)
    Ps = [csr_dense(o.amg_matrix(k, "P")) for k in range(nl - 1)]
    # the smoother of every level is the reading's l1 row scaling of its
    # Galerkin operator (all functions counted)
    Ak = A
    for k in range(nl - 1):
        np.testing.assert_allclose(o.amg_dinv(k), _row_l1_inverse(Ak), rtol=1e-13)
        Ak = Ps[k].T @ Ak @ Ps[k]
    B = _vcycle_dense(A, Ps)
    rng = np.random.default_rng(11)
    for _ in range(2):
        r = rng.standard_normal(A.shape[0])
        z = o.apply(r)
        zt = o.apply_transpose(r)
        ref, reft = B @ r, B.T @ r
        assert np.max(np.abs(z - ref)) <= 1e-12 * np.max(np.abs(ref))
        assert np.max(np.abs(zt - reft)) <= 1e-12 * np.max(np.abs(reft))

# ------------------------------------------------- transposed cycle (adjoint)
@pytest.mark.parametrize("make,opts", [
    (lambda: make_two_phase(6, 5, 3), None),
    (lambda: make_two_phase(6, 5, 3), O.Options(relax=["l1_jacobi"], sweeps=[3], weights=[0.8])),
    (lambda: make_compositional(8, 8, 2, nwell_side=2), None),
    (lambda: make_compositional(8, 8, 2, nwell_side=2),
     O.Options(relax=["block_jacobi", "block_jacobi"], sweeps=[2, 1])),
    (lambda: make_poromech(6, 4), None),
    (lambda: make_poromech(6, 4, strategy="mgr_u"),
     O.Options(relax=["amg"], relax_functions=[3], max_coarse=32)),
    # a nonsymmetric A_FF (upwinded saturation block): the transposed
    # V-cycle differs from the forward one
    (lambda: make_two_phase(8, 6, 3), O.Options(relax=["amg"], max_coarse=16)),
    # the restriction of Eq. 5 (R = [-A_CF D^-1, I]) on a nonsymmetric system,
    # with repeated weighted sweeps, and on every level of the 4-level order
    (lambda: make_two_phase(8, 6, 3),
     O.Options(relax=["jacobi"], sweeps=[2], weights=[0.8], restrict=["jacobi"], max_coarse=16)),
    (lambda: make_compositional(16, 12, 4, nwell_side=2, strategy="mgr4"),
     O.Options(relax=["jacobi", "jacobi", "amg"], restrict=["jacobi"] * 3, max_coarse=32)),
    (lambda: make_poromech(6, 4, strategy="mgr_u"),
     O.Options(relax=["amg"], relax_functions=[3], sweeps=[2], weights=[0.8], max_coarse=32)),
])
def test_transpose_cycle_is_adjoint(make, opts):
    s = make()
    o = O.Oracle(s, opts) if opts else O.Oracle(s)
    rng = np.random.default_rng(7)
    u = rng.standard_normal(s.n); v = rng.standard_normal(s.n)
    lhs = u @ o.apply(v)
    rhs = o.apply_transpose(u) @ v
    assert abs(lhs - rhs) <= 1e-11 * (np.abs(u) @ np.abs(o.apply(v)) + 1e-300)


def test_transpose_solve_and_gradient_match_dense():
    """A^T lambda = g solved with the transposed cycle; dL/dA_ij = -lambda_i x_j."""
    s = make_two_phase(5, 4, 2)
    A = dense_of(s)
    o = O.Oracle(s)
    g = np.random.default_rng(2).standard_normal(s.n)
    r = o.solve(g, rtol=1e-13, trans=True)
    lam = np.linalg.solve(A.T, g)
    assert r["status"] == 0
    assert np.linalg.norm(r["x"] - lam) <= 1e-10 * np.linalg.norm(lam)


# ------------------------------------------------- configs, qualitative
def test_iteration_counts_mesh_independent_two_phase():
    """Mesh-independent iteration counts (Sec. 5.2, 5.4): a qualitative pin."""
    its = [O.Oracle(s).solve(s.rhs, rtol=1e-8)["iters"]
           for s in (make_two_phase(8, 8, 4), make_two_phase(16, 16, 8), make_two_phase(24, 24, 12))]
    assert max(its) - min(its) <= 4, its


def test_compositional_and_poromech_small_converge():
    for s in (make_compositional(16, 16, 4), make_poromech(8, 4)):
        r = O.Oracle(s).solve(s.rhs, rtol=1e-8)
        assert r["status"] == 0 and r["relres"] <= 1e-8


# ------------------------------------- AMG F-relaxation (MGR_U, Sec. 4.3)
def _mgr_cycle_dense(A, F, Cc, K):
    """Algorithm 1 with F-relaxation operator K, W = -diag(A_FF)^-1 A_FC
    (Jacobi interpolation, D_uu = diag(A_uu)) and an exact coarse solve, as
    one dense matrix M^-1 = [K 0; 0 0] + [W; I] S^-1 [-A_CF K, I]."""
    AFF, AFC = A[np.ix_(F, F)], A[np.ix_(F, Cc)]
    ACF, ACC = A[np.ix_(Cc, F)], A[np.ix_(Cc, Cc)]
    W = -AFC / np.diag(AFF)[:, None]
    S = ACC + ACF @ W
    nF, nC = F.size, Cc.size
    Mf = np.zeros((A.shape[0], A.shape[0]))
    blk = np.zeros((nF + nC, nF + nC))
    blk[:nF, :nF] = K
    Pc = np.vstack([W, np.eye(nC)])
    Rc = np.hstack([-ACF @ K, np.eye(nC)])
    blk += Pc @ np.linalg.solve(S, Rc)
    order = np.concatenate([F, Cc])
    Mf[np.ix_(order, order)] = blk
    return Mf


@pytest.mark.parametrize("sweeps,omega", [(1, 1.0), (2, 0.8), (3, 0.6)])
def test_amg_frelax_exact_grids_match_dense_cycle(sweeps, omega):
    """MGR_U with both AMG hierarchies a single dense level (max_coarse above
    both block sizes): one V-cycle on A_uu is an exact solve, so s weighted
    sweeps from zero give K = (1 - (1 - omega)^s) A_uu^-1, and the MGR cycle
    and its transpose equal the dense operator of Algorithm 1 with that K."""
    s = make_poromech(6, 4, strategy="mgr_u")
    o = O.Oracle(s, O.Options(relax=["amg"], relax_functions=[3], sweeps=[sweeps],
                              weights=[omega], max_coarse=4096))
    assert o.frelax_amg_nlevels(0) == 1 and o.amg_nlevels == 1
    A = dense_of(s)
    F = np.flatnonzero(s.dof_level == 0); Cc = np.flatnonzero(s.dof_level == 1)
    K = (1 - (1 - omega) ** sweeps) * np.linalg.inv(A[np.ix_(F, F)])
    Mi = _mgr_cycle_dense(A, F, Cc, K)
    rng = np.random.default_rng(11)
    v = rng.standard_normal(s.n)
    ref = Mi @ v
    assert np.linalg.norm(o.apply(v) - ref) <= 1e-10 * np.linalg.norm(ref)
    reft = Mi.T @ v
    assert np.linalg.norm(o.apply_transpose(v) - reft) <= 1e-10 * np.linalg.norm(reft)


def test_amg_frelax_on_diagonal_F_block_is_direct():
    """An AMG F-relaxation of a diagonal A_FF (MGR_P on the mimetic system)
    finds no strong couplings, keeps one level and solves A_FF exactly; with
    an exact coarse solve the cycle is A^-1 and FGMRES takes one iteration."""
    s = make_mimetic(4, 4, 4)
    o = O.Oracle(s, O.Options(relax=["amg"], relax_functions=[1]))
    assert o.frelax_amg_nlevels(0) == 1 and o.amg_nlevels == 1
    A = dense_of(s)
    v = np.random.default_rng(3).standard_normal(s.n)
    ref = np.linalg.solve(A, v)
    assert np.linalg.norm(o.apply(v) - ref) <= 1e-10 * np.linalg.norm(ref)
    r = o.solve(s.rhs, rtol=1e-12)
    assert r["status"] == 0 and r["iters"] == 1


def test_amg_frelax_hierarchy_is_galerkin_on_A_uu():
    """The F-relaxation hierarchy starts from A_FF itself (not A or the
    coarse block) and every coarser operator is P^T A P, densely; the
    unknown approach keeps P from mixing displacement components."""
    s = make_poromech(6, 4, strategy="mgr_u")
    o = O.Oracle(s, O.Options(relax=["amg"], relax_functions=[3], max_coarse=32))
    nl = o.frelax_amg_nlevels(0)
    assert nl >= 3
    A0 = csr_dense(o.amg_matrix(0, "A", frelax_level=0))
    assert np.array_equal(A0, csr_dense(o.mgr_matrix(0, "AFF")))
    func = np.arange(A0.shape[0]) % 3
    for k in range(nl - 1):
        Ak = csr_dense(o.amg_matrix(k, "A", frelax_level=0))
        P = csr_dense(o.amg_matrix(k, "P", frelax_level=0))
        Ac = csr_dense(o.amg_matrix(k + 1, "A", frelax_level=0))
        ref = P.T @ Ak @ P
        assert np.max(np.abs(Ac - ref)) <= 1e-12 * np.max(np.abs(ref))
        cf = o.amg_cf(k, frelax_level=0)
        assert set(np.unique(cf)) <= {-1, 1}
        # each coarse column takes the function of the C point it comes from
        cfunc = func[cf == 1]
        rows, cols = np.nonzero(P)
        assert np.all(func[rows] == cfunc[cols])
        func = cfunc


def test_mgr_u_fewer_iterations_than_mgr_p():
    """Sec. 4.3 / Table 7: eliminating the displacement first (MGR_U, AMG
    F-relaxation) needs fewer FGMRES iterations than eliminating the
    fracture pressure first (MGR_P) on the same system."""
    its = {}
    for strat in ("mgr_p", "mgr_u"):
        s = make_poromech(16, 8, strategy=strat)
        r = O.Oracle(s).solve(s.rhs, rtol=1e-8, maxit=500)
        assert r["status"] == 0
        its[strat] = r["iters"]
    assert its["mgr_u"] < its["mgr_p"], its


# --------------------------- 4-level compositional order (Sec. 4.2, mgr4)
def test_compositional_4level_first_reduction_is_exact():
    """The volume-constraint rows, aligned with a density, are diagonal in
    every unknown: level 0's A_FF is diagonal, so the first reduction is the
    exact Schur complement and one Jacobi sweep is an exact F solve."""
    s = make_compositional(8, 6, 3, nwell_side=2, strategy="mgr4")
    o = O.Oracle(s)
    A = dense_of(s)
    F = np.flatnonzero(s.dof_level == 0); Cc = np.flatnonzero(s.dof_level > 0)
    AFF = A[np.ix_(F, F)]
    assert np.count_nonzero(AFF - np.diag(np.diag(AFF))) == 0
    S = A[np.ix_(Cc, Cc)] - A[np.ix_(Cc, F)] @ np.linalg.solve(AFF, A[np.ix_(F, Cc)])
    got = csr_dense(o.mgr_matrix(1, "A"))
    assert np.max(np.abs(got - S)) <= 1e-13 * np.max(np.abs(S))


def test_compositional_4level_keeps_wells_to_a_direct_coarsest_solve():
    """Wells survive to the final coarse block (2 dofs per well), which is
    solved directly (one dense level) although its BHP-control rows have zero
    diagonals; those rows pass every reduction unchanged.  The reservoir
    pressure level is relaxed by an AMG V-cycle."""
    s = make_compositional(16, 12, 4, nwell_side=2, strategy="mgr4")
    o = O.Oracle(s, O.Options(relax=list(s.relax), relax_functions=list(s.relax_functions),
                              max_coarse=32))
    nw = s.meta["n_wells"]
    Af = csr_dense(o.mgr_matrix(3, "A"))
    assert Af.shape == (2 * nw, 2 * nw) and o.amg_nlevels == 1
    assert o.frelax_amg_nlevels(2) >= 2
    for w in range(0, nw, 2):          # BHP control: row q = p_w
        row = np.zeros(2 * nw); row[2 * w] = 1.0
        assert np.array_equal(Af[2 * w + 1], row)
    r = o.solve(s.rhs, rtol=1e-10, maxit=300)
    assert r["status"] == 0 and r["relres"] <= 1e-10


def test_compositional_4level_is_a_row_permutation_of_the_3level_system():
    a3 = make_compositional(6, 5, 3, nwell_side=2)
    a4 = make_compositional(6, 5, 3, nwell_side=2, strategy="mgr4")
    D3, D4 = dense_of(a3), dense_of(a4)
    nc = 6 * 5 * 3
    perm = np.arange(a3.n)
    perm[:4 * nc].reshape(nc, 4)[:, [0, 1]] = perm[:4 * nc].reshape(nc, 4)[:, [1, 0]]
    assert np.array_equal(D4, D3[perm])
    assert np.array_equal(a4.rhs, a3.rhs[perm])


# ------------------------------------- MGR_Pi on the TPFA scheme (Sec. 4.1)
def test_mgr_pi_tpfa_coarse_operator_is_the_harmonic_tpfa_stencil():
    """TPFA makes Abar_pipi diagonal, so with faces as F-points one Jacobi
    sweep and the Jacobi interpolation are exact, and the coarse operator is
    the exact Schur complement of Eq. 8.  Eliminating the face multipliers
    reproduces the cell-centred TPFA scheme: neighbours couple through the
    harmonic combination T1 T2 / (T1 + T2) of their half-transmissibilities
    (read from the matrix: Abar_ppi = -T), boundary faces carry no flux."""
    s = make_mimetic(5, 4, 3, scheme="tpfa", strategy="mgr_pi")
    o = O.Oracle(s)
    A = dense_of(s)
    nc = s.meta["n_cells"]
    cells, faces = np.arange(nc), np.arange(nc, s.n)
    assert np.array_equal(np.flatnonzero(s.dof_level == 1), cells)
    Aff = A[np.ix_(faces, faces)]
    assert np.count_nonzero(Aff - np.diag(np.diag(Aff))) == 0
    T = -A[np.ix_(cells, faces)]                     # half-transmissibilities, [cell, face]
    S = np.diag(np.diag(A)[:nc])
    for f in range(faces.size):
        on = np.flatnonzero(T[:, f])
        tot = T[on, f].sum()
        assert np.isclose(tot, Aff[f, f], rtol=1e-14)
        if on.size == 2:
            c1, c2 = on
            h = T[c1, f] * T[c2, f] / tot
            S[c1, c2] -= h; S[c2, c1] -= h
            S[c1, c1] -= T[c1, f] ** 2 / tot; S[c2, c2] -= T[c2, f] ** 2 / tot
        else:                                        # boundary face: no flux
            S[on[0], on[0]] -= T[on[0], f]
    got = csr_dense(o.mgr_matrix(1, "A"))
    assert np.max(np.abs(got - S)) <= 1e-12 * np.max(np.abs(S))
    assert max(np.count_nonzero(np.abs(S[i]) > 1e-12 * np.abs(S).max()) for i in range(nc)) <= 7


def test_mgr_pi_tpfa_two_level_is_direct():
    """With the coarse grid solved exactly, MGR_Pi on TPFA is a direct solver."""
    s = make_mimetic(6, 5, 4, scheme="tpfa", strategy="mgr_pi")
    o = O.Oracle(s)
    assert o.amg_nlevels == 1
    v = np.random.default_rng(8).standard_normal(s.n)
    ref = np.linalg.solve(dense_of(s), v)
    assert np.linalg.norm(o.apply(v) - ref) <= 1e-10 * np.linalg.norm(ref)
    assert o.solve(s.rhs, rtol=1e-12)["iters"] == 1


# ------------------------------------------ the SPD restriction of Eq. 5
def _two_level_blocks(A, lvl):
    F = np.flatnonzero(lvl == 0); Cc = np.flatnonzero(lvl > 0)
    return F, Cc, A[np.ix_(F, F)], A[np.ix_(F, Cc)], A[np.ix_(Cc, F)], A[np.ix_(Cc, Cc)]


@pytest.mark.parametrize("make,relax", [
    (lambda: make_two_phase(6, 5, 3), "jacobi"),
    (lambda: make_poromech(6, 4), "l1_jacobi"),
])
def test_jacobi_restriction_coarse_operator_is_petrov_galerkin(make, relax):
    """With R~ = [-A_CF D^-1, I] and P~ = [-D^-1 A_FC; I] (Eq. 5) the coarse
    operator is the triple product R~ A P~, densely."""
    s = make()
    o = O.Oracle(s, O.Options(relax=[relax], restrict=["jacobi"], num_functions=s.num_functions))
    A = dense_of(s)
    F, Cc, AFF, AFC, ACF, ACC = _two_level_blocks(A, s.dof_level)
    d = np.diag(AFF).copy()
    if relax == "l1_jacobi":
        off = np.abs(AFF).sum(1) - np.abs(d)
        d = np.where(d < 0, d - off, d + off)
    R = np.hstack([-ACF / d[None, :], np.eye(Cc.size)])
    P = np.vstack([-AFC / d[:, None], np.eye(Cc.size)])
    Ap = np.block([[AFF, AFC], [ACF, ACC]])
    S = R @ Ap @ P
    got = csr_dense(o.mgr_matrix(1, "A"))
    assert np.max(np.abs(got - S)) <= 1e-12 * np.max(np.abs(S))
    Z = csr_dense(o.mgr_matrix(0, "Z"))
    assert np.max(np.abs(Z - R[:, :F.size])) <= 1e-15 * np.abs(Z).max()


def test_jacobi_restriction_keeps_spd_coarse_grids():
    """Sec. 3: for an SPD matrix, R~ = P~^T (Eq. 5) makes each coarse
    operator the Galerkin product P~^T A P~, again SPD, and the coarse-grid
    correction I - P~ S^-1 P~^T A an A-orthogonal projection (it never
    increases the energy norm of the error)."""
    from paper_2101_11649_gb300.synth.bsr import BlockSystem
    rp, ci, v = poisson(12, 10)
    n = 120
    k = np.arange(n)
    lvl = np.where(k % 3 == 0, 1, 0).astype(np.int8)      # coupled F points
    lvl[(lvl == 1) & (k % 2 == 0)] = 2
    sysm = BlockSystem(name="poisson2d", b=1, row_ptr=rp, col_idx=ci, val=v.reshape(-1, 1, 1),
                       dof_level=lvl, num_levels=2, rhs=np.ones(n), relax=["jacobi", "jacobi"])
    o = O.Oracle(sysm, O.Options(relax=["jacobi", "jacobi"], restrict=["jacobi"] * 2, max_coarse=4))
    Al = csr_dense(o.mgr_matrix(0, "A"))
    rng = np.random.default_rng(13)
    for lv in (0, 1):
        assert np.count_nonzero(csr_dense(o.mgr_matrix(lv, "AFF")) - np.diag(np.diag(
            csr_dense(o.mgr_matrix(lv, "AFF"))))) > 0
        S = csr_dense(o.mgr_matrix(lv + 1, "A"))
        assert np.max(np.abs(S - S.T)) <= 1e-14 * np.max(np.abs(S))
        assert np.linalg.eigvalsh(S).min() > 0
        # P~ in the level's own ordering: identity on C rows, W on F rows
        sub = lvl[lvl >= lv] if lv == 0 else lvl[lvl >= 1]
        F = np.flatnonzero(sub == lv); Cc = np.flatnonzero(sub > lv)
        P = np.zeros((sub.size, Cc.size))
        P[F] = csr_dense(o.mgr_matrix(lv, "W")); P[Cc, np.arange(Cc.size)] = 1.0
        assert np.max(np.abs(P.T @ Al @ P - S)) <= 1e-13 * np.max(np.abs(S))
        for _ in range(5):
            e = rng.standard_normal(sub.size)
            e2 = e - P @ np.linalg.solve(S, P.T @ (Al @ e))
            assert e2 @ Al @ e2 <= e @ Al @ e * (1 + 1e-12)
        Al = S


@pytest.mark.parametrize("sweeps,omega", [(1, 1.0), (2, 0.7)])
def test_jacobi_restriction_cycle_matches_dense_algorithm_1(sweeps, omega):
    """Algorithm 1 with R~ of Eq. 5, s weighted Jacobi sweeps from zero and an
    exact coarse solve: M^-1 = K_e + P~ S^-1 R~ (I - A K_e), K_e = [K 0; 0 0],
    K = (I - (I - omega D^-1 A_FF)^s) A_FF^-1; and its transpose."""
    s = make_two_phase(6, 5, 3)
    o = O.Oracle(s, O.Options(relax=["jacobi"], sweeps=[sweeps], weights=[omega],
                              restrict=["jacobi"], max_coarse=4096))
    assert o.amg_nlevels == 1
    A = dense_of(s)
    F, Cc, AFF, AFC, ACF, ACC = _two_level_blocks(A, s.dof_level)
    d = np.diag(AFF)
    E = np.eye(F.size) - omega * AFF / d[:, None]
    K = (np.eye(F.size) - np.linalg.matrix_power(E, sweeps)) @ np.linalg.inv(AFF)
    R = np.hstack([-ACF / d[None, :], np.eye(Cc.size)])
    P = np.vstack([-AFC / d[:, None], np.eye(Cc.size)])
    Ap = np.block([[AFF, AFC], [ACF, ACC]])
    Ke = np.zeros_like(Ap); Ke[:F.size, :F.size] = K
    Mp = Ke + P @ np.linalg.solve(R @ Ap @ P, R @ (np.eye(s.n) - Ap @ Ke))
    order = np.concatenate([F, Cc])
    Mi = np.zeros_like(Mp); Mi[np.ix_(order, order)] = Mp
    v = np.random.default_rng(12).standard_normal(s.n)
    for got, ref in ((o.apply(v), Mi @ v), (o.apply_transpose(v), Mi.T @ v)):
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


# ------------------------------------------ setup reuse (Sec. 4.3, Sec. 5)
def _perturbed(sysm, seed, touch_uu):
    """The same pattern with new values: pressure rows and couplings scaled
    by U[0.9, 1.1] per block; the displacement block A_uu too if touch_uu."""
    import dataclasses
    rng = np.random.default_rng(seed)
    NN = (sysm.meta["ne"] + 1) ** 3
    rows = np.repeat(np.arange(sysm.nb), np.diff(sysm.row_ptr))
    cols = sysm.col_idx
    sel = (rows >= NN) | (cols >= NN) | touch_uu
    val = sysm.val.copy()
    val[sel] *= rng.uniform(0.9, 1.1, int(sel.sum()))[:, None, None]
    if sysm.n_pad:   # the padding dofs (F-points, identity rows) stay as they are
        last = np.flatnonzero((rows == sysm.nb - 1) & (cols == sysm.nb - 1))[0]
        for t in range(sysm.b - sysm.n_pad, sysm.b):
            val[last, t, t] = sysm.val[last, t, t]
    return dataclasses.replace(sysm, val=val)


def _mgr_u_opts():
    return O.Options(relax=["amg"], relax_functions=[3], max_coarse=32)


def test_reuse_with_unchanged_A_uu_equals_a_fresh_setup():
    """MGR_U keeps the displacement AMG hierarchy across Newton steps; when
    A_uu did not change, the refreshed preconditioner is the one a fresh
    setup builds (same coarse operators and final AMG, same cycle bits)."""
    s1 = make_poromech(6, 4, strategy="mgr_u")
    s2 = _perturbed(s1, 1, touch_uu=False)
    o1 = O.Oracle(s1, _mgr_u_opts())
    o2 = O.Oracle(s2, _mgr_u_opts(), reuse=o1)
    f2 = O.Oracle(s2, _mgr_u_opts())
    for lv in (0, 1):
        assert np.array_equal(o2.mgr_matrix(lv, "A")[2], f2.mgr_matrix(lv, "A")[2])
    assert o2.amg_nlevels == f2.amg_nlevels and o2.frelax_amg_nlevels(0) == f2.frelax_amg_nlevels(0)
    v = np.random.default_rng(2).standard_normal(s1.n)
    assert np.array_equal(o2.apply(v), f2.apply(v))
    assert np.array_equal(o2.apply_transpose(v), f2.apply_transpose(v))


def test_reuse_with_changed_A_uu_keeps_the_old_F_hierarchy():
    """When A_uu changed, the F-relaxation still uses the hierarchy built from
    the old A_uu while W, the coarse block and its AMG hierarchy follow the
    new values; the stale preconditioner still converges."""
    s1 = make_poromech(6, 4, strategy="mgr_u")
    s2 = _perturbed(s1, 3, touch_uu=True)
    o1 = O.Oracle(s1, _mgr_u_opts())
    old_A0 = o1.amg_matrix(0, "A", frelax_level=0)
    old_A1 = o1.amg_matrix(1, "A", frelax_level=0)
    o2 = O.Oracle(s2, _mgr_u_opts(), reuse=o1)
    f2 = O.Oracle(s2, _mgr_u_opts())
    kept0 = o2.amg_matrix(0, "A", frelax_level=0)
    assert np.array_equal(kept0[2], old_A0[2])
    assert np.array_equal(o2.amg_matrix(1, "A", frelax_level=0)[2], old_A1[2])
    assert not np.array_equal(kept0[2], o2.mgr_matrix(0, "AFF")[2])
    assert np.array_equal(o2.mgr_matrix(0, "AFF")[2], f2.mgr_matrix(0, "AFF")[2])
    assert np.array_equal(o2.mgr_matrix(1, "A")[2], f2.mgr_matrix(1, "A")[2])
    for k in range(f2.amg_nlevels):
        assert np.array_equal(o2.amg_matrix(k, "A")[2], f2.amg_matrix(k, "A")[2])
    r = o2.solve(s2.rhs, rtol=1e-8, maxit=300)
    assert r["status"] == 0 and r["relres"] <= 1e-8


def test_paper_strategies_converge_mesh_independently():
    """Qualitative pin (Sec. 5.2-5.4, Tables 4 and 7): the iteration counts of
    MGR_U, the 4-level compositional order and MGR_Pi on TPFA stay bounded
    as the grids grow."""
    cases = {
        "mgr_u": [make_poromech(8, 4, strategy="mgr_u"), make_poromech(16, 8, strategy="mgr_u"),
                  make_poromech(24, 12, strategy="mgr_u")],
        "mgr4": [make_compositional(16, 16, 4, strategy="mgr4"),
                 make_compositional(32, 32, 8, strategy="mgr4"),
                 make_compositional(48, 48, 12, strategy="mgr4")],
        "mgr_pi": [make_mimetic(12, 12, 12, scheme="tpfa", strategy="mgr_pi"),
                   make_mimetic(20, 20, 20, scheme="tpfa", strategy="mgr_pi"),
                   make_mimetic(28, 28, 28, scheme="tpfa", strategy="mgr_pi")],
    }
    for name, systems in cases.items():
        its = []
        for sysm in systems:
            r = O.Oracle(sysm).solve(sysm.rhs, rtol=1e-8, maxit=300)
            assert r["status"] == 0, name
            its.append(r["iters"])
        assert max(its) - min(its) <= 8 and max(its) <= 40, (name, its)


def test_oracle_refuses_eq5_restriction_with_block_jacobi():
    """The restriction of Eq. 5 is stated for D_FF = diag(A_FF): a block-Jacobi
    level with it is refused."""
    s = make_compositional(6, 5, 2, nwell_side=2)
    with pytest.raises(RuntimeError):
        O.Oracle(s, O.Options(relax=["block_jacobi", "block_jacobi"], restrict=["jacobi"]))
