"""The allocation-free residual entry point (collected last on purpose).

mgr_residual_norm_noalloc serves callers that cannot call cudaMalloc (a
plug-in whose host application owns all device memory, a real-time loop that
must never enter the allocator): its reduction scratch is a static device
array.
Checked through the C ABI against the entry points that do allocate: the
residual against b - mgr_spmv(x), the norm against the true residual that
mgr_solve reports, on two calls in a row (the static scratch is reused).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2101_11649_gb300 import mgr as M  # noqa: E402
from paper_2101_11649_gb300.synth import make_mimetic, make_two_phase  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.mark.parametrize("make", [lambda: make_mimetic(9, 8, 7), lambda: make_two_phase(12, 10, 6)])
def test_noalloc_residual_matches_allocating_entry_points(make):
    s = make()
    g = M.MGRSolver.from_system(s)
    rp = torch.as_tensor(s.row_ptr, device=DEV)
    ci = torch.as_tensor(s.col_idx, device=DEV)
    val = torch.as_tensor(s.val.ravel(), device=DEV)
    bvec = torch.as_tensor(s.rhs, device=DEV)
    x, info = g.solve(bvec, rtol=1e-6)
    assert info["status"] == 0
    ax = g.spmv(x)
    r_ref = (bvec - ax).cpu().numpy()
    scale = (np.abs(s.rhs) + M.bsr_spmv(rp, ci, val.abs(), s.b, x.abs()).cpu().numpy()) + 1e-300
    norm_ref = info["rel_residual"] * float(torch.linalg.norm(bvec))
    prev = None
    for _ in range(2):
        r, norm = M.residual_norm_noalloc(rp, ci, val, s.b, x, bvec)
        torch.cuda.synchronize()
        rn = r.cpu().numpy()
        assert np.max(np.abs(rn - r_ref) / scale) <= 1e-13
        nv = float(norm.item())
        # the two paths may sum b - A x in different orders; the norms then
        # differ by at most |r_a - r_b| <= 1e-13 |scale| (triangle inequality)
        assert abs(nv - norm_ref) <= 1e-13 * np.linalg.norm(scale) + 1e-12 * norm_ref
        assert abs(nv - np.linalg.norm(rn)) <= 1e-13 * nv
        if prev is not None:
            assert torch.equal(r, prev[0]) and float(prev[1].item()) == nv
        prev = (r.clone(), norm.clone())


def test_noalloc_rejects_sizes_beyond_static_scratch():
    # 4096 partial sums of 4096 entries each: n = 16,777,217 needs one more.
    # Rejected on the host before any device access (the pointers are never read).
    lib = M.lib()
    nb = 16_777_217
    dummy = torch.zeros(8, dtype=torch.float64, device=DEV)
    idx = torch.zeros(8, dtype=torch.int32, device=DEV)
    st = lib.mgr_residual_norm_noalloc(nb, 1, M._ptr(idx), M._ptr(idx), M._ptr(dummy),
                                       M._ptr(dummy), M._ptr(dummy), M._ptr(dummy),
                                       M._ptr(dummy), M._stream_ptr())
    assert st == M.MGR_ERR_UNSUPPORTED
