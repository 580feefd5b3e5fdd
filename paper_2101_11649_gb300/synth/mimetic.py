"""Statically condensed hybrid mimetic (MFD) single-phase Jacobian (Sec. 4.1).

Recipe:
  * nx*ny*nz hexahedra on a unit-spaced lattice whose interior nodes are
    moved by U[-distort, distort] per coordinate (boundary nodes fixed), so
    cells are non-orthogonal and each 6x6 inner-product block is dense, as
    in the paper's consistent approach on distorted cells (App. A).
  * Per cell K = kappa_c diag(1, 1, 0.1), ln kappa_c ~ N(0, 2^2).
  * Parametric mimetic inner product, stability parameter 2 (App. A):
      M_c = X K^{-1} X^T / |c| + t (I - Q Q^T),
      t = 2 tr(X K^{-1} X^T) / (6 |c|),
    X = face-centroid offsets from the cell centroid, N = outward vector
    areas, Q = orthonormal basis of range(N).  Consistency M_c N K = X holds
    when X^T N = |c| I.
  * Saddle point of Eq. 6 with A_ww = blockdiag(M_c), A_wp = -D,
    A_wpi = C (= -1 one-sided-face-to-face incidence), incompressible
    A_pw = D^T, A_pp = 1e-3 mean(kappa) I; statically condensed as in Eq. 7:
      Abar_pp = A_pp + D^T M^{-1} D            (diagonal)
      Abar_ppi = D^T M^{-1} C,  Abar_pip = C^T M^{-1} D,
      Abar_pipi = C^T M^{-1} C.
  * scheme="tpfa" (the TPFA approach of Sec. 4.1): every block of A_ww is
    diagonal, M_c = diag(1 / T_cf) with the half-transmissibilities
    T_cf = (N_f . K N_f) / (X_f . N_f), so Abar_pipi is diagonal too.
  * Unknown order: cell pressures, then x-, y-, z-face multipliers.
  * Labels, strategy "mgr_p" (default): cells -> level 0 (F, Jacobi;
    Abar_pp diagonal, inverted exactly), faces -> level 1 (C, AMG).  This
    is MGR_P, Eq. 9.  Strategy "mgr_pi" (for TPFA): faces -> level 0 (F,
    Jacobi on the diagonal Abar_pipi: exact relaxation and ideal
    interpolation), cells -> level 1 (C, AMG on the exact Schur complement
    of Eq. 8, the cell-centred TPFA operator).
  * rhs ~ N(0,1).
"""
from __future__ import annotations

import numpy as np

from .bsr import BlockSystem, scalar_coo_to_bsr1, streams


def _face_ids(nx, ny, nz):
    """Global face numbers of the 6 faces of every cell (x-, x+, y-, y+, z-, z+)."""
    nfx = (nx + 1) * ny * nz
    nfy = nx * (ny + 1) * nz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    fx = lambda ii: ii + (nx + 1) * (j + ny * k)
    fy = lambda jj: nfx + i + nx * (jj + (ny + 1) * k)
    fz = lambda kk: nfx + nfy + i + nx * (j + ny * kk)
    return np.stack([fx(i), fx(i + 1), fy(j), fy(j + 1), fz(k), fz(k + 1)], 1), \
        nfx + nfy + nx * ny * (nz + 1)


def _geometry(nx, ny, nz, distort, rng):
    gx, gy, gz = np.meshgrid(np.arange(nx + 1.0), np.arange(ny + 1.0), np.arange(nz + 1.0),
                             indexing="ij")
    nodes = np.stack([gx, gy, gz], -1)  # [nx+1, ny+1, nz+1, 3]
    d = rng.uniform(-distort, distort, nodes.shape)
    interior = np.zeros(nodes.shape[:3], dtype=bool)
    interior[1:-1, 1:-1, 1:-1] = True
    nodes = nodes + d * interior[..., None]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    P = lambda a, b_, c: nodes[i + a, j + b_, k + c]  # [nc, 3]

    def quad(a, b_, c_, d_):
        # vector area of a (possibly warped) quad a-b-c-d = half the diagonal cross product
        area = 0.5 * np.cross(c_ - a, d_ - b_)
        cent = 0.25 * (a + b_ + c_ + d_)
        return area, cent

    faces = []
    # x-faces at i (normal +x): (0,0,0)-(0,1,0)-(0,1,1)-(0,0,1)
    for off in (0, 1):
        faces.append(quad(P(off, 0, 0), P(off, 1, 0), P(off, 1, 1), P(off, 0, 1)))
    for off in (0, 1):
        faces.append(quad(P(0, off, 0), P(0, off, 1), P(1, off, 1), P(1, off, 0)))
    for off in (0, 1):
        faces.append(quad(P(0, 0, off), P(1, 0, off), P(1, 1, off), P(0, 1, off)))
    area = np.stack([f[0] for f in faces], 1)  # [nc, 6, 3] oriented +axis
    cent = np.stack([f[1] for f in faces], 1)
    sign = np.array([-1.0, 1.0, -1.0, 1.0, -1.0, 1.0])
    N = area * sign[None, :, None]  # outward
    corners = np.stack([P(a, b_, c) for a in (0, 1) for b_ in (0, 1) for c in (0, 1)], 1)
    xc = corners.mean(1)
    vol = (cent * N).sum(-1).sum(-1) / 3.0
    X = cent - xc[:, None, :]
    return N, X, vol


def make_mimetic(nx=64, ny=64, nz=64, seed=0, distort=0.1, name="mimetic", scheme="consistent",
                 strategy="mgr_p") -> BlockSystem:
    if scheme not in ("consistent", "tpfa") or strategy not in ("mgr_p", "mgr_pi"):
        raise ValueError(f"unknown mimetic scheme/strategy {scheme!r}/{strategy!r}")
    nc = nx * ny * nz
    rs = streams(seed, ["perm", "geom", "rhs"])
    kappa = np.exp(2.0 * rs["perm"].standard_normal(nc))
    N, X, vol = _geometry(nx, ny, nz, distort, rs["geom"])
    kinv = 1.0 / (kappa[:, None] * np.array([1.0, 1.0, 0.1])[None, :])  # diag K^{-1}
    XKX = np.einsum("cfa,ca,cga->cfg", X, kinv, X)
    t = 2.0 * np.trace(XKX, axis1=1, axis2=2) / (6.0 * vol)
    Q, _ = np.linalg.qr(N)  # [nc, 6, 3]
    stab = np.eye(6)[None] - np.einsum("cfa,cga->cfg", Q, Q)
    M = XKX / vol[:, None, None] + t[:, None, None] * stab
    Minv = np.linalg.inv(M)
    Minv = 0.5 * (Minv + np.transpose(Minv, (0, 2, 1)))
    if scheme == "tpfa":
        # half-transmissibility of each one-sided face: (N.K N) / (X.N)
        NKN = np.einsum("cfa,ca,cfa->cf", N, 1.0 / kinv, N)
        Thalf = NKN / np.einsum("cfa,cfa->cf", X, N)
        Minv = np.zeros((nc, 6, 6))
        Minv[:, np.arange(6), np.arange(6)] = Thalf
    fid, nf = _face_ids(nx, ny, nz)
    app = 1e-3 * kappa.mean()

    rowsum = Minv.sum(2)  # M^{-1} 1, [nc, 6]
    cells = np.arange(nc)
    # C = -incidence, D = +incidence
    r_pp, c_pp, v_pp = cells, cells, app + Minv.sum((1, 2))
    r_pf = np.repeat(cells, 6); c_pf = nc + fid.ravel(); v_pf = -rowsum.ravel()
    r_fp = nc + fid.ravel(); c_fp = np.repeat(cells, 6); v_fp = -rowsum.ravel()
    r_ff = nc + np.repeat(fid, 6, axis=1).ravel()
    c_ff = nc + np.tile(fid, (1, 6)).ravel()
    v_ff = Minv.reshape(nc, 36).ravel()
    rows = np.concatenate([r_pp, r_pf, r_fp, r_ff])
    cols = np.concatenate([c_pp, c_pf, c_fp, c_ff])
    vals = np.concatenate([v_pp, v_pf, v_fp, v_ff])
    n = nc + nf
    rp, ci, val = scalar_coo_to_bsr1(n, rows, cols, vals)
    if strategy == "mgr_p":
        lvl = np.concatenate([np.zeros(nc, np.int8), np.ones(nf, np.int8)])
    else:
        lvl = np.concatenate([np.ones(nc, np.int8), np.zeros(nf, np.int8)])
    rhs = rs["rhs"].standard_normal(n)
    return BlockSystem(name=name, b=1, row_ptr=rp, col_idx=ci, val=val, dof_level=lvl,
                       num_levels=1, rhs=rhs, relax=["jacobi"], num_functions=1,
                       meta=dict(grid=(nx, ny, nz), n_cells=nc, n_faces=nf, seed=seed,
                                 distort=distort, scheme=scheme, strategy=strategy))
