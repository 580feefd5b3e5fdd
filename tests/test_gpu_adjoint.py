"""Adjoint form: gradients of L = w . x, x = A^{-1} b, through the autograd
Function (transposed MGR cycle on the GPU), checked against the dense
gradient, the CPU oracle's gradient and central finite differences."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_11649_gb300.synth import make_batch, make_poromech, make_two_phase

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2101_11649_gb300 import mgr as M  # noqa: E402
from paper_2101_11649_gb300.autograd import mgr_solve_fn  # noqa: E402

DEV = torch.device("cuda:0")


def dense_of(s):
    A = np.zeros((s.n, s.n))
    b = s.b
    for I in range(s.nb):
        for p in range(s.row_ptr[I], s.row_ptr[I + 1]):
            J = s.col_idx[p]
            A[I * b:(I + 1) * b, J * b:(J + 1) * b] = s.val[p]
    return A


def grads_from(s, lam, x):
    """dL/dA on the stored pattern: -lam_i x_j per block entry."""
    b = s.b
    rows = np.repeat(np.arange(s.nb), np.diff(s.row_ptr))
    L = lam.reshape(s.nb, b)[rows]          # [nnzb, b]
    X = x.reshape(-1, b)[s.col_idx]         # [nnzb, b]
    return -L[:, :, None] * X[:, None, :]


def ad_gradients(s, w, rtol=1e-12):
    solver = M.MGRSolver.from_system(s)
    vals = torch.as_tensor(s.val, device=DEV).requires_grad_(True)
    rhs = torch.as_tensor(s.rhs, device=DEV).requires_grad_(True)
    x = mgr_solve_fn(vals, rhs, solver, rtol, 2000)
    loss = (torch.as_tensor(w, device=DEV) * x).sum()
    loss.backward()
    return x.detach().cpu().numpy(), vals.grad.cpu().numpy(), rhs.grad.cpu().numpy()


def test_autograd_matches_dense_gradient():
    s = make_two_phase(6, 5, 4)
    w = np.random.default_rng(3).standard_normal(s.n)
    A = dense_of(s)
    x_ref = O.dense_solve(A, s.rhs)
    lam_ref = O.dense_solve(A.T.copy(), w)
    x, dA, db = ad_gradients(s, w)
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert np.linalg.norm(db - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    g_ref = grads_from(s, lam_ref, x_ref)
    assert np.max(np.abs(dA - g_ref)) <= 1e-9 * np.max(np.abs(g_ref))


@pytest.mark.parametrize("restrict", ["injection", "jacobi"])
def test_autograd_mgr_u_matches_dense_gradient(restrict):
    """The adjoint through an AMG F-relaxation (MGR_U) and, optionally, the
    restriction of Eq. 5: gradients against dense LU."""
    s = make_poromech(6, 4, strategy="mgr_u")
    w = np.random.default_rng(17).standard_normal(s.n)
    A = dense_of(s)
    x_ref = O.dense_solve(A, s.rhs)
    lam_ref = O.dense_solve(A.T.copy(), w)
    solver = M.MGRSolver.from_system(s, restrict=[restrict], max_coarse=32)
    vals = torch.as_tensor(s.val, device=DEV).requires_grad_(True)
    rhs = torch.as_tensor(s.rhs, device=DEV).requires_grad_(True)
    x = mgr_solve_fn(vals, rhs, solver, 1e-12, 2000)
    (torch.as_tensor(w, device=DEV) * x).sum().backward()
    assert np.linalg.norm(x.detach().cpu().numpy() - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    db = rhs.grad.cpu().numpy()
    assert np.linalg.norm(db - lam_ref) <= 1e-9 * np.linalg.norm(lam_ref)
    g_ref = grads_from(s, lam_ref, x_ref)
    assert np.max(np.abs(vals.grad.cpu().numpy() - g_ref)) <= 1e-8 * np.max(np.abs(g_ref))


@pytest.fixture(scope="module")
def member16():
    systems, weights = make_batch(nsys=1)
    s, w = systems[0], weights[0]
    assert s.meta["grid"] == (16, 16, 16)
    return s, w


def test_autograd_matches_oracle_gradient_16cubed(member16):
    s, w = member16
    o = O.Oracle(s)
    rx = o.solve(s.rhs, rtol=1e-13, maxit=2000)
    rl = o.solve(w, rtol=1e-13, maxit=2000, trans=True)
    g_or = grads_from(s, rl["x"], rx["x"])
    x, dA, db = ad_gradients(s, w, rtol=1e-13)
    assert np.linalg.norm(db - rl["x"]) <= 1e-8 * np.linalg.norm(rl["x"])
    assert np.max(np.abs(dA - g_or)) <= 1e-8 * np.max(np.abs(g_or))


def test_autograd_matches_central_differences_16cubed(member16):
    """Central differences, h_k = 1e-6 |A_k| (relative), on 64 seeded random
    stored entries; relative error <= 1e-5 with the denominator
    max(|g_ad|, 1e-8 max|g_ad|).  Each perturbed system A +- h e_k is solved
    by FGMRES warm-started at x with the hierarchy of A kept as the
    preconditioner (mgr_update_values) and a fixed 40 iterations, so the
    O(h) change of x is resolved to many digits and the two solves of a pair
    share their rounding history."""
    s, w = member16
    x, dA, _ = ad_gradients(s, w, rtol=1e-13)
    gmax = np.max(np.abs(dA))
    rng = np.random.default_rng(64)
    flat = s.val.reshape(-1)
    nz = np.flatnonzero(flat != 0.0)
    picks = rng.choice(nz, 64, replace=False)
    rhs = torch.as_tensor(s.rhs, device=DEV)
    wt = torch.as_tensor(w, device=DEV)
    xt = torch.as_tensor(x, device=DEV)
    sv = M.MGRSolver.from_system(s)

    # scalar coordinates of every stored value, for extended-precision residuals
    b = s.b
    blk_rows = np.repeat(np.arange(s.nb), np.diff(s.row_ptr))
    rr = (blk_rows[:, None, None] * b + np.arange(b)[None, :, None]) + 0 * np.arange(b)[None, None, :]
    cc = (s.col_idx[:, None, None] * b + np.arange(b)[None, None, :]) + 0 * np.arange(b)[None, :, None]
    rr, cc = rr.reshape(-1), cc.reshape(-1)
    order = np.argsort(rr, kind="stable")
    cc_o = cc[order]
    starts = np.flatnonzero(np.r_[True, np.diff(rr[order]) != 0])
    assert starts.size == s.n
    LD = np.longdouble
    b_ld = s.rhs.astype(LD)

    def solution_with(vals):
        """x = (A')^{-1} b by iterative refinement: residuals in extended
        precision on the host, corrections by the GPU FP64 solver (hierarchy
        of A kept as the preconditioner)."""
        sv.update_values(vals)
        v_ld = vals.astype(LD)[order]
        x_ld = x.astype(LD)
        for _ in range(3):
            r_ld = b_ld - np.add.reduceat(v_ld * x_ld[cc_o], starts)
            d, info = sv.solve(torch.as_tensor(r_ld.astype(np.float64), device=DEV), rtol=1e-10,
                               maxit=200)
            x_ld = x_ld + d.cpu().numpy().astype(LD)
        return x_ld

    w_ld = w.astype(LD)
    worst = 0.0
    for k in picks:
        h = 1e-6 * abs(flat[k])
        vp = flat.copy(); vp[k] += h
        vm = flat.copy(); vm[k] -= h
        # L(A+h) - L(A-h) = w . (x+ - x-), differenced entry-wise in extended
        # precision so the O(h) change survives
        fd = float(np.sum(w_ld * (solution_with(vp) - solution_with(vm))) / (2 * LD(h)))
        ad = dA.reshape(-1)[k]
        err = abs(fd - ad) / max(abs(ad), 1e-8 * gmax)
        worst = max(worst, err)
    assert worst <= 1e-5, worst


def test_autograd_follows_the_values_it_is_given():
    """Values that differ from the ones the solver was built from (a later
    Newton step) reach the outer operator before the forward solve, so x and
    the gradients belong to them; a wrong shape is refused."""
    s = make_two_phase(6, 5, 4)
    solver = M.MGRSolver.from_system(s)
    rng = np.random.default_rng(11)
    val2 = s.val * rng.uniform(0.9, 1.1, s.val.shape[0])[:, None, None]
    s2 = dataclasses.replace(s, val=val2)
    w = rng.standard_normal(s.n)
    A2 = dense_of(s2)
    x_ref = O.dense_solve(A2, s.rhs)
    lam_ref = O.dense_solve(A2.T.copy(), w)
    vals = torch.as_tensor(val2, device=DEV).requires_grad_(True)
    rhs = torch.as_tensor(s.rhs, device=DEV).requires_grad_(True)
    x = mgr_solve_fn(vals, rhs, solver, 1e-12, 2000)
    (torch.as_tensor(w, device=DEV) * x).sum().backward()
    assert np.linalg.norm(x.detach().cpu().numpy() - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    g_ref = grads_from(s2, lam_ref, x_ref)
    assert np.max(np.abs(vals.grad.cpu().numpy() - g_ref)) <= 1e-9 * np.max(np.abs(g_ref))
    assert solver.holds_values(vals)
    with pytest.raises(ValueError):
        mgr_solve_fn(vals[:-1], rhs, solver, 1e-12, 2000)
