"""Two-phase immiscible TPFA Jacobian (2x2 BSR), the small two-level case.

Recipe (synthetic stand-in; the paper's own compositional and single-phase
models are Sec. 4.1-4.2 and App. A-B):
  * nx*ny*nz unit cells, porosity 0.2, ln K ~ N(0,1) i.i.d. per cell,
    harmonic face transmissibility T_ij = 2 K_i K_j / (K_i + K_j).
  * Water saturation S ~ U[0.2, 0.8]; Corey kr_w = S^2, kr_n = (1-S)^2;
    viscosities mu_w = 1, mu_n = 5 (non-wetting / wetting ratio 5).
  * Reference pressure p = x + 0.1 N(0,1) decides single-point upwinding.
  * Unknowns per cell (p, S); rows (total = water + non-wetting, water).
    Accumulation phi V / dt on the saturation derivatives (cancelling in the
    total row) and a compressibility term c_t phi V / dt (c_t = 1e-2) on the
    total-row pressure diagonal.
  * dt is the largest value for which every saturation row of the S-S block
    satisfies a_ii >= 2 sum_{j != i} |a_ij|.
  * Labels: S -> level 0 (F, l1-Jacobi), p -> level 1 (C, AMG).
  * rhs ~ N(0,1).
"""
from __future__ import annotations

import numpy as np

from .bsr import BlockSystem, assemble_bsr, streams


def _neighbor_pairs(nx, ny, nz):
    """All ordered pairs (i, j) of face-adjacent cells."""
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    pairs = []
    for a, b in ((idx[:, :, :-1], idx[:, :, 1:]), (idx[:, :-1, :], idx[:, 1:, :]),
                 (idx[:-1, :, :], idx[1:, :, :])):
        a = a.ravel(); b = b.ravel()
        pairs.append(np.stack([a, b], 1))
        pairs.append(np.stack([b, a], 1))
    p = np.concatenate(pairs, 0)
    return p[:, 0], p[:, 1]


def make_two_phase(nx=16, ny=16, nz=8, seed=0, name="two_phase") -> BlockSystem:
    nc = nx * ny * nz
    rs = streams(seed, ["perm", "sat", "pres", "rhs"])
    K = np.exp(rs["perm"].standard_normal(nc))
    S = rs["sat"].uniform(0.2, 0.8, nc)
    xc = np.tile(np.arange(nx, dtype=np.float64), ny * nz)
    p = xc + 0.1 * rs["pres"].standard_normal(nc)
    phi, V, mu_w, mu_n, c_t = 0.2, 1.0, 1.0, 5.0, 1e-2

    i, j = _neighbor_pairs(nx, ny, nz)
    T = 2.0 * K[i] * K[j] / (K[i] + K[j])
    dp = p[i] - p[j]
    up = np.where(dp > 0, i, j)
    Su = S[up]
    lw, ln_ = Su ** 2 / mu_w, (1.0 - Su) ** 2 / mu_n
    dlw, dln = 2.0 * Su / mu_w, -2.0 * (1.0 - Su) / mu_n
    up_is_i = up == i

    # flux derivatives of row i: d/dp_i, d/dp_j, d/dS_up  (water, non-wetting)
    w_dpi, n_dpi = T * lw, T * ln_
    w_dS, n_dS = T * dp * dlw, T * dp * dln

    # saturation block flux parts, for the dt rule
    sflux_diag = np.bincount(i, weights=np.where(up_is_i, w_dS, 0.0), minlength=nc)
    soff = np.bincount(i, weights=np.where(up_is_i, 0.0, np.abs(w_dS)), minlength=nc)
    need = (2.0 * soff - sflux_diag).max()
    dt = phi * V / need if need > 0 else 1.0
    acc = phi * V / dt

    b = 2
    # diagonal blocks: rows (t, w), cols (p, S)
    dblk = np.zeros((nc, b, b))
    dblk[:, 0, 0] = c_t * acc
    dblk[:, 1, 1] = acc
    dblk[:, 0, 0] += np.bincount(i, weights=w_dpi + n_dpi, minlength=nc)
    dblk[:, 1, 0] += np.bincount(i, weights=w_dpi, minlength=nc)
    dblk[:, 0, 1] += np.bincount(i, weights=np.where(up_is_i, w_dS + n_dS, 0.0), minlength=nc)
    dblk[:, 1, 1] += sflux_diag
    # off-diagonal blocks (i, j)
    oblk = np.zeros((i.size, b, b))
    oblk[:, 0, 0] = -(w_dpi + n_dpi)
    oblk[:, 1, 0] = -w_dpi
    oblk[:, 0, 1] = np.where(up_is_i, 0.0, w_dS + n_dS)
    oblk[:, 1, 1] = np.where(up_is_i, 0.0, w_dS)

    rows = np.concatenate([np.arange(nc), i])
    cols = np.concatenate([np.arange(nc), j])
    rp, ci, val = assemble_bsr(nc, b, rows, cols, np.concatenate([dblk, oblk], 0))
    lvl = np.tile(np.array([1, 0], dtype=np.int8), nc)
    rhs = rs["rhs"].standard_normal(nc * b)
    sysm = BlockSystem(name=name, b=b, row_ptr=rp, col_idx=ci, val=val, dof_level=lvl,
                       num_levels=1, rhs=rhs, relax=["l1_jacobi"], num_functions=1,
                       meta=dict(grid=(nx, ny, nz), dt=dt, seed=seed))
    return sysm
