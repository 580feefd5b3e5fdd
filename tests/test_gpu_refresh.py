"""Setup reuse through mgr_refresh (Sec. 4.3): new values on the same pattern
rebuild the MGR levels and the final AMG hierarchy while AMG F-relaxation
hierarchies are kept.  Checked against the oracle's reuse, bit for bit on
the hierarchy and within the FP64 tolerances on the cycle and the solve."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2101_11649_gb300.synth import make_poromech, make_two_phase
from parity_checks import cycle_close
from test_gpu_parity import _same_csr, _same_frelax_hierarchies, oracle_of, solver, t
from test_oracle_pins import _perturbed

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2101_11649_gb300 import mgr as M  # noqa: E402

COARSE = 32


def _pair(touch_uu, seed=5, ne=8, nf=4):
    s1 = make_poromech(ne, nf, strategy="mgr_u")
    return s1, _perturbed(s1, seed, touch_uu)


@pytest.mark.parametrize("touch_uu", [False, True])
@pytest.mark.parametrize("restrict", ["injection", "jacobi"])
def test_refresh_matches_oracle_reuse(touch_uu, restrict):
    s1, s2 = _pair(touch_uu)
    g = solver(s1, max_coarse=COARSE, restrict=[restrict])
    g.refresh(s2.val)
    assert g.check() == 0
    o1 = oracle_of(s1, max_coarse=COARSE, restrict=[restrict])
    o2 = O.Oracle(s2, O.Options(relax=list(s2.relax), relax_functions=list(s2.relax_functions),
                                num_functions=s2.num_functions, max_coarse=COARSE,
                                restrict=[restrict]), reuse=o1)
    assert g.info()["amg_levels"] == o2.amg_nlevels
    for l in range(s2.num_levels + 1):
        _same_csr(g.matrix(0, l, 0), o2.mgr_matrix(l, "A"), f"MGR A_{l}")
    for w, nm in ((1, "AFF"), (4, "W")):
        _same_csr(g.matrix(0, 0, w), o2.mgr_matrix(0, nm), nm)
    for k in range(o2.amg_nlevels):
        _same_csr(g.matrix(1, k, 0), o2.amg_matrix(k, "A"), f"AMG A_{k}")
    _same_frelax_hierarchies(g, o2, s2)
    rng = np.random.default_rng(6)
    for trans in (False, True):
        v = rng.standard_normal(s2.n)
        zg = g.apply(t(v), transpose=trans).cpu().numpy()
        zo = o2.apply_transpose(v) if trans else o2.apply(v)
        cycle_close(s2, zg, zo, 1e-11, f"trans={trans}")
    ro = o2.solve(s2.rhs, rtol=1e-8, maxit=500)
    xg, ig = g.solve(t(s2.rhs), rtol=1e-8, maxit=500)
    assert ig["status"] == 0 and abs(ig["iterations"] - ro["iters"]) <= 1


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_refresh_with_fixed_A_uu_is_a_fresh_setup(precision):
    """With A_uu unchanged the refreshed handle applies bit for bit the
    preconditioner of a fresh setup on the new values."""
    s1, s2 = _pair(False, seed=7)
    g = solver(s1, precision=precision, max_coarse=COARSE)
    g.refresh(s2.val)
    f = solver(s2, precision=precision, max_coarse=COARSE)
    v = t(np.random.default_rng(8).standard_normal(s2.n))
    for trans in (False, True):
        a = g.apply(v, transpose=trans).cpu().numpy()
        b = f.apply(v, transpose=trans).cpu().numpy()
        assert np.array_equal(a.view(np.int64), b.view(np.int64)), trans


def test_refresh_without_amg_relaxation_rebuilds_everything():
    """On a hierarchy without AMG F-relaxations a refresh is a fresh setup."""
    import dataclasses
    s1 = make_two_phase(8, 7, 5)
    rng = np.random.default_rng(9)
    s2 = dataclasses.replace(s1, val=s1.val * rng.uniform(0.95, 1.05, s1.val.shape[0])[:, None, None])
    g = solver(s1, max_coarse=COARSE)
    g.refresh(s2.val)
    f = solver(s2, max_coarse=COARSE)
    for l in range(s2.num_levels + 1):
        _same_csr(g.matrix(0, l, 0), f.matrix(0, l, 0), f"MGR A_{l}")
    x1, i1 = g.solve(t(s2.rhs), rtol=1e-10)
    x2, i2 = f.solve(t(s2.rhs), rtol=1e-10)
    assert i1["iterations"] == i2["iterations"]
    assert np.array_equal(x1.cpu().numpy().view(np.int64), x2.cpu().numpy().view(np.int64))


def test_refresh_memory_is_bounded():
    """Each refresh frees the hierarchy it replaces."""
    s1 = make_poromech(24, 12, strategy="mgr_u")
    vals = [_perturbed(s1, 10 + k, touch_uu=False).val for k in range(5)]
    g = solver(s1)
    g.refresh(vals[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for v in vals[1:]:
        g.refresh(v)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free0 - free1) <= 32 << 20, (free0 - free1) / 2**20
    _, info = g.solve(t(s1.rhs), rtol=1e-8)
    assert info["status"] == 0


def test_refresh_rejects_batch_members_and_bad_values():
    s = make_two_phase(6, 5, 3)
    bt = M.MGRBatch([s, s])
    with pytest.raises(M.MGRError) as e:
        bt.system(0).refresh(s.val)
    assert e.value.status == M.MGR_ERR_UNSUPPORTED
    bt.close()
    g = solver(s)
    bad = s.val.copy()
    bad[0, 0, 0] = np.nan
    with pytest.raises(M.MGRError) as e:
        g.refresh(bad)
    assert e.value.status == M.MGR_ERR_INVALID
