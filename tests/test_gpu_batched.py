"""Batched form: many uneven systems solved with one launch per kernel class.

Each member keeps its own hierarchy, so a batched solve must agree with the
single-system path (iterations +-1, solutions 1e-8 when both are converged
to 1e-12) and with the CPU oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_11649_gb300.synth import make_batch, make_poromech, make_two_phase

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2101_11649_gb300 import mgr as M  # noqa: E402

DEV = torch.device("cuda:0")
GRIDS = [(16, 16, 16), (12, 9, 7), (20, 11, 5), (8, 8, 8), (24, 10, 6), (5, 4, 3)]


@pytest.fixture(scope="module")
def small_batch():
    systems, weights = make_batch(grids=GRIDS)
    return systems, weights


def t(x):
    return torch.as_tensor(np.ascontiguousarray(x), device=DEV)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_matches_single_system_path(small_batch, precision):
    systems, _ = small_batch
    batch = M.MGRBatch(systems, precision=precision)
    rhs = [t(s.rhs) for s in systems]
    xs, infos = batch.solve(rhs, rtol=1e-8)
    for s, x, inf in zip(systems, xs, infos):
        single = M.MGRSolver.from_system(s, precision=precision)
        xs1, i1 = single.solve(t(s.rhs), rtol=1e-8)
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-8
        assert abs(inf["iterations"] - i1["iterations"]) <= 1, (inf["iterations"], i1["iterations"])
    xs, infos = batch.solve(rhs, rtol=1e-12, maxit=1000)
    for s, x in zip(systems, xs):
        single = M.MGRSolver.from_system(s, precision=precision)
        x1, _ = single.solve(t(s.rhs), rtol=1e-12, maxit=1000)
        rel = float(torch.linalg.norm(x - x1) / torch.linalg.norm(x1))
        assert rel <= 1e-8, rel


def test_batched_matches_oracle(small_batch):
    systems, _ = small_batch
    batch = M.MGRBatch(systems)
    xs, infos = batch.solve([t(s.rhs) for s in systems], rtol=1e-12, maxit=1000)
    for i in (0, 2, 5):
        ro = O.Oracle(systems[i]).solve(systems[i].rhs, rtol=1e-12, maxit=1000)
        x = xs[i].cpu().numpy()
        assert np.linalg.norm(x - ro["x"]) <= 1e-8 * np.linalg.norm(ro["x"])
    # iteration parity at 1e-8
    xs, infos = batch.solve([t(s.rhs) for s in systems], rtol=1e-8)
    for i in range(len(systems)):
        ro = O.Oracle(systems[i]).solve(systems[i].rhs, rtol=1e-8)
        assert abs(infos[i]["iterations"] - ro["iters"]) <= 1


def test_batched_member_handles_and_gradients(small_batch):
    systems, weights = small_batch
    batch = M.MGRBatch(systems)
    xs, infos = batch.solve([t(s.rhs) for s in systems], rtol=1e-12, maxit=1000)
    i = 1
    sv = batch.system(i)
    assert all(batch.system(k).check() == 0 for k in range(len(systems)))
    lam, info = sv.solve(t(weights[i]), rtol=1e-12, transpose=True)
    ro = O.Oracle(systems[i]).solve(weights[i], rtol=1e-12, trans=True)
    assert info["status"] == 0
    assert np.linalg.norm(lam.cpu().numpy() - ro["x"]) <= 1e-8 * np.linalg.norm(ro["x"])
    dA = sv.grad_values(lam, xs[i]).cpu().numpy()
    assert dA.shape == systems[i].val.shape and np.isfinite(dA).all()


def test_batched_zero_rhs_member_and_repeat(small_batch):
    systems, _ = small_batch
    batch = M.MGRBatch(systems)
    rhs = [t(s.rhs) for s in systems]
    rhs[3] = torch.zeros_like(rhs[3])
    xs, infos = batch.solve(rhs, rtol=1e-10)
    assert infos[3]["iterations"] == 0 and float(xs[3].abs().max()) == 0.0
    xs2, infos2 = batch.solve(rhs, rtol=1e-10)
    for a, b in zip(xs, xs2):
        assert torch.equal(a, b)


@pytest.mark.slow
def test_batched_48_uneven_systems():
    """The 48-member batch (grids 16^3 .. 96x96x48, 4.74M cells, 9.5M unknowns)."""
    systems, _ = make_batch(48)
    batch = M.MGRBatch(systems, precision="fp32")
    xs, infos = batch.solve([t(s.rhs) for s in systems], rtol=1e-8)
    assert all(inf["status"] == 0 and inf["rel_residual"] <= 1e-8 for inf in infos)
    for i in (0, 17, 47):
        ro = O.Oracle(systems[i]).solve(systems[i].rhs, rtol=1e-8)
        assert abs(infos[i]["iterations"] - ro["iters"]) <= 1, (i, infos[i]["iterations"], ro["iters"])


# the paper's strategies in a batch: MGR_U (one AMG V-cycle as F-relaxation,
# Sec. 4.3), with and without a weight, and the restriction of Eq. 5
STRATEGIES = {
    "mgr_u": (lambda: [make_poromech(n, f, seed=k, strategy="mgr_u")
                       for k, (n, f) in enumerate(((6, 4), (8, 4), (10, 6)))],
              dict(max_coarse=32)),
    "mgr_u_weighted_eq5": (lambda: [make_poromech(n, f, seed=k, strategy="mgr_u")
                                    for k, (n, f) in enumerate(((6, 4), (8, 6)))],
                           dict(max_coarse=32, weights=[0.9], restrict=["jacobi"])),
    "eq5": (lambda: [make_two_phase(*g) for g in GRIDS[:4]],
            dict(max_coarse=32, restrict=["jacobi"])),
}


@pytest.mark.parametrize("name", list(STRATEGIES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batched_paper_strategies_match_single_system_path(name, precision):
    """Each member of a batch with an AMG F-relaxation or the restriction of
    Eq. 5 converges like its own single-system handle (iterations +-1, the
    same true residual bound) and, in FP64, like the oracle (+-1)."""
    make, kw = STRATEGIES[name]
    systems = make()
    batch = M.MGRBatch(systems, precision=precision, **kw)
    xs, infos = batch.solve([t(s.rhs) for s in systems], rtol=1e-8, maxit=500)
    for s, x, inf in zip(systems, xs, infos):
        single = M.MGRSolver.from_system(s, precision=precision, **kw)
        _, i1 = single.solve(t(s.rhs), rtol=1e-8, maxit=500)
        assert inf["status"] == 0 and inf["rel_residual"] <= 1e-8, inf
        assert abs(inf["iterations"] - i1["iterations"]) <= 1, (inf["iterations"], i1["iterations"])
        if precision == "fp64":
            okw = dict(kw)
            ro = O.Oracle(s, O.Options(relax=list(s.relax), num_functions=s.num_functions,
                                       relax_functions=list(s.relax_functions),
                                       max_coarse=okw.get("max_coarse", 1024),
                                       weights=okw.get("weights", []),
                                       restrict=okw.get("restrict", []))).solve(s.rhs, rtol=1e-8)
            assert abs(inf["iterations"] - ro["iters"]) <= 1, (inf["iterations"], ro["iters"])
    # converged tightly, the batched solution is the single-system one
    xs, _ = batch.solve([t(s.rhs) for s in systems], rtol=1e-12, maxit=1000)
    for s, x in zip(systems, xs):
        single = M.MGRSolver.from_system(s, precision=precision, **kw)
        x1, _ = single.solve(t(s.rhs), rtol=1e-12, maxit=1000)
        assert float(torch.linalg.norm(x - x1) / torch.linalg.norm(x1)) <= 1e-8
