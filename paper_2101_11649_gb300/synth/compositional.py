"""Compositional flow with wells (4x4 BSR), shaped like Sec. 4.2 / Eq. 12.

Recipe (a synthetic stand-in; the paper's EOS-based model is App. B):
  * nx*ny*nz unit cells, ln K ~ N(0, 1.5^2), harmonic transmissibility.
  * Unknowns per cell (p, m1, m2, m3).  Rows: a cell-local volume
    constraint aligned with p (like the paper's rho_2 constraint rows,
    which are diagonal in every unknown), then one mass balance per
    component aligned with m_c.
  * Component mobility lambda_c = m_c / sum(m) (total mobility 1),
    m ~ U[0.1, 1]; single-point upwinding on p = x + 0.1 N(0,1).
  * Mass-balance rows: accumulation a (e_c + r_c) on the mass columns,
    r_c ~ U[-0.1, 0.1]^3 (a random inter-component coupling), plus the
    derivatives of the upwinded fluxes T lambda_c (p_i - p_j) with respect
    to p and the upstream masses.
  * Volume row: a (sum_c m_c / rho_c - c_v p) with rho = (1, 0.8, 0.6),
    c_v = 1e-3.  The accumulation scale a = phi V / dt is twice the largest
    off-diagonal flux mass of any cell's mass rows, so that every mass block
    row is diagonally dominant (the dt rule of the two-phase case).
  * 16 vertical wells on a 4x4 lattice of columns, each perforating every
    layer.  Well unknowns (p_w, q), padded to a 4x4 block row with two
    identity pads.  p_w row: sum_k WI_k (p_w - p_k) - q; q row: p_w (bottom-
    hole-pressure control, even wells: zero diagonal, Sec. 4.2) or q (rate
    control, odd wells).  Perforation sources WI_k lambda_c (p_k - p_w) enter
    the cell mass balances; WI_k = K_k.
  * Labels, strategy "mgr3" (default): cell masses and pads -> level 0
    (F, 3x3 / 2x2 block-Jacobi), well dofs -> level 1 (F, exact 2x2), cell
    pressure -> level 2 (C, AMG).
  * Strategy "mgr4" (the 4-level order of Sec. 4.2, wells kept to the
    coarsest grid): the first two rows of every cell block are swapped, so
    that the volume constraint row is aligned with m1 (a density whose row
    is diagonal in every unknown, like the paper's rho_2) and the first mass
    balance with p.  Levels: m1 and pads -> 0 (Jacobi, exact), m2, m3 -> 1
    (Jacobi), cell pressure -> 2 (F-relaxation by one AMG V-cycle on the
    reduced pressure block, the CPR-like pressure system), well dofs -> 3
    (the final coarse block, 2 dofs per well: one dense direct solve, its
    BHP-controlled rows with zero diagonals included).
  * rhs ~ N(0,1) on real dofs, 0 on pads.
"""
from __future__ import annotations

import numpy as np

from .bsr import BlockSystem, assemble_bsr, streams
from .two_phase import _neighbor_pairs


def make_compositional(nx=128, ny=128, nz=32, nwell_side=4, seed=0,
                       name="compositional", strategy="mgr3") -> BlockSystem:
    if strategy not in ("mgr3", "mgr4"):
        raise ValueError(f"unknown compositional strategy {strategy!r}")
    nc = nx * ny * nz
    rs = streams(seed, ["perm", "mass", "pres", "coup", "rhs"])
    K = np.exp(1.5 * rs["perm"].standard_normal(nc))
    m = rs["mass"].uniform(0.1, 1.0, (nc, 3))
    xc = np.tile(np.arange(nx, dtype=np.float64), ny * nz)
    p = xc + 0.1 * rs["pres"].standard_normal(nc)
    rho = np.array([1.0, 0.8, 0.6])
    c_v = 1e-3
    msum = m.sum(1)
    lam = m / msum[:, None]                       # [nc, 3]
    # d lambda_c / d m_k = (delta_ck * S - m_c) / S^2
    dlam = (np.eye(3)[None] * msum[:, None, None] - m[:, :, None]) / (msum ** 2)[:, None, None]

    i, j = _neighbor_pairs(nx, ny, nz)
    T = 2.0 * K[i] * K[j] / (K[i] + K[j])
    dp = p[i] - p[j]
    up = np.where(dp > 0, i, j)
    up_is_i = up == i
    fl_p = T[:, None] * lam[up]                   # [npair, 3] d/dp_i
    fl_m = (T * dp)[:, None, None] * dlam[up]     # [npair, 3(c), 3(k)] d/dm_up

    offmass = np.bincount(i, weights=np.where(up_is_i, 0.0, np.abs(fl_m).sum((1, 2))), minlength=nc)
    acc = 2.0 * float(offmass.max()) if np.any(offmass > 0) else 1.0

    b = 4
    coup = rs["coup"].uniform(-0.1, 0.1, (nc, 3, 3))
    dblk = np.zeros((nc, b, b))
    dblk[:, 0, 0] = -acc * c_v
    dblk[:, 0, 1:] = acc / rho[None, :]
    dblk[:, 1:, 1:] = acc * (np.eye(3)[None] + coup)
    for c in range(3):
        dblk[:, 1 + c, 0] += np.bincount(i, weights=fl_p[:, c], minlength=nc)
        for k in range(3):
            dblk[:, 1 + c, 1 + k] += np.bincount(i, weights=np.where(up_is_i, fl_m[:, c, k], 0.0),
                                                 minlength=nc)
    oblk = np.zeros((i.size, b, b))
    oblk[:, 1:, 0] = -fl_p
    oblk[:, 1:, 1:] = np.where(up_is_i[:, None, None], 0.0, fl_m)

    # wells
    wx = (np.arange(nwell_side) * nx) // nwell_side + nx // (2 * nwell_side)
    wy = (np.arange(nwell_side) * ny) // nwell_side + ny // (2 * nwell_side)
    wells = [(x, y) for y in wy for x in wx]
    nw = len(wells)
    rows, cols, blks = [np.arange(nc), i], [np.arange(nc), j], [dblk, oblk]
    wdiag = np.zeros((nw, b, b))
    for w, (x, y) in enumerate(wells):
        perf = x + nx * (y + ny * np.arange(nz))
        WI = K[perf]
        wr = nc + w
        wdiag[w, 0, 0] = WI.sum()
        wdiag[w, 0, 1] = -1.0
        if w % 2 == 0:
            wdiag[w, 1, 0] = 1.0       # bottom-hole pressure control: zero diagonal
        else:
            wdiag[w, 1, 1] = 1.0       # rate control
        wdiag[w, 2, 2] = wdiag[w, 3, 3] = 1.0
        # well row -> cells
        wb = np.zeros((nz, b, b)); wb[:, 0, 0] = -WI
        rows.append(np.full(nz, wr)); cols.append(perf); blks.append(wb)
        # cells -> well (p_w column), and cell diagonal source derivative
        cb = np.zeros((nz, b, b)); cb[:, 1:, 0] = -(WI[:, None] * lam[perf])
        rows.append(perf); cols.append(np.full(nz, wr)); blks.append(cb)
        db = np.zeros((nz, b, b)); db[:, 1:, 0] = WI[:, None] * lam[perf]
        rows.append(perf); cols.append(perf); blks.append(db)
    rows.append(nc + np.arange(nw)); cols.append(nc + np.arange(nw)); blks.append(wdiag)
    nb = nc + nw
    rp, ci, val = assemble_bsr(nb, b, np.concatenate(rows), np.concatenate(cols),
                               np.concatenate(blks, 0))
    rhs = rs["rhs"].standard_normal(nb * b)
    rhs[nc * b:].reshape(nw, b)[:, 2:] = 0.0
    meta = dict(grid=(nx, ny, nz), n_wells=nw, acc=acc, seed=seed, strategy=strategy)
    if strategy == "mgr4":
        cell_rows = np.repeat(np.arange(nb) < nc, np.diff(rp))
        val[cell_rows] = val[cell_rows][:, [1, 0, 2, 3], :]
        rhs[:nc * b].reshape(nc, b)[:, [0, 1]] = rhs[:nc * b].reshape(nc, b)[:, [1, 0]]
        lvl = np.concatenate([np.tile(np.array([2, 0, 1, 1], np.int8), nc),
                              np.tile(np.array([3, 3, 0, 0], np.int8), nw)])
        return BlockSystem(name=name, b=b, row_ptr=rp, col_idx=ci, val=val, dof_level=lvl,
                           num_levels=3, rhs=rhs, relax=["jacobi", "jacobi", "amg"],
                           num_functions=1, relax_functions=[1, 1, 1], n_pad=2 * nw, meta=meta)
    lvl = np.concatenate([np.tile(np.array([2, 0, 0, 0], np.int8), nc),
                          np.tile(np.array([1, 1, 0, 0], np.int8), nw)])
    return BlockSystem(name=name, b=b, row_ptr=rp, col_idx=ci, val=val, dof_level=lvl,
                       num_levels=2, rhs=rhs, relax=["block_jacobi", "block_jacobi"],
                       num_functions=1, n_pad=2 * nw, meta=meta)
