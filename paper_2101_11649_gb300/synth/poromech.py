"""Poromechanics with a planar hydraulic fracture (3x3 BSR), Sec. 4.3 / Eq. 13.

Recipe (a synthetic stand-in for the paper's GEOSX fracture model, App. C):
  * ne^3 trilinear hexahedra of side h = 4 m, (ne+1)^3 nodes, 3 displacement
    dofs per node in nodal order (ux, uy, uz).  Young's modulus
    E = 10 GPa exp(N(0, 0.5^2)) per element, Poisson ratio 0.25.  Element
    stiffness E h K0 with K0 the unit-cube Q1 stiffness (2x2x2 Gauss).
    Dirichlet u = 0 on every outer node: identity rows, and their couplings
    removed from the interior rows.
  * Fracture: nf x nf elements on the node plane y = ne/2, starting at
    element ne/8 in x and z.  Apertures w ~ U[1e-4, 1e-3] m; cubic-law
    transmissibility w^3 / (12 eta), eta = 0.01 Pa s, harmonic between
    neighbours; storage w A / (K_f dt), K_f = 2 GPa, dt = 1 s.
  * Coupling: A_up(node_y, e) = -A_e / 4 on the 4 corner nodes' y dofs,
    A_pu(e, node_y) = A_e / (4 dt).
  * A symmetric per-field diagonal scaling (one factor for u, one for p)
    brings both block diagonals to O(1); both sides see the scaled matrix.
  * Fracture pressures are packed three per 3x3 block row after the nodes.
  * Labels, strategy "mgr_p" (default): p -> level 0 (F, l1-Jacobi),
    u -> level 1 (C, AMG with the unknown approach, 3 functions).  This is
    MGR_P of Sec. 4.3.
  * Strategy "mgr_u" (MGR_U of Sec. 4.3): u -> level 0 (F), relaxed by one
    AMG V-cycle on A_uu with the unknown approach (3 functions), and
    D_uu = diag(A_uu) in the interpolation; p -> level 1, the final coarse
    block S = A_pp - A_pu D_uu^-1 A_up, one AMG V-cycle (1 function).  The
    padding dofs keep label 0.
  * rhs ~ N(0,1).
"""
from __future__ import annotations

import numpy as np

from .bsr import BlockSystem, assemble_bsr, streams


def q1_unit_stiffness(nu=0.25):
    """24x24 stiffness of the unit cube, E = 1, local node q = a + 2b + 4c."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[np.arange(3, 6), np.arange(3, 6)] = mu
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    K = np.zeros((24, 24))
    loc = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    for x in g:
        for y in g:
            for z in g:
                dN = np.zeros((8, 3))
                for q, (a, b, c) in enumerate(loc):
                    fx = x if a else 1 - x
                    fy = y if b else 1 - y
                    fz = z if c else 1 - z
                    sx, sy, sz = (1 if a else -1), (1 if b else -1), (1 if c else -1)
                    dN[q] = (sx * fy * fz, fx * sy * fz, fx * fy * sz)
                B = np.zeros((6, 24))
                for q in range(8):
                    B[0, 3 * q] = dN[q, 0]
                    B[1, 3 * q + 1] = dN[q, 1]
                    B[2, 3 * q + 2] = dN[q, 2]
                    B[3, 3 * q] = dN[q, 1]; B[3, 3 * q + 1] = dN[q, 0]
                    B[4, 3 * q + 1] = dN[q, 2]; B[4, 3 * q + 2] = dN[q, 1]
                    B[5, 3 * q] = dN[q, 2]; B[5, 3 * q + 2] = dN[q, 0]
                K += 0.125 * B.T @ D @ B
    return K


def make_poromech(ne=64, nf=48, seed=0, name="poromech", strategy="mgr_p") -> BlockSystem:
    nn1 = ne + 1
    NN = nn1 ** 3
    h, nu, eta, Kf, dt = 4.0, 0.25, 0.01, 2e9, 1.0
    rs = streams(seed, ["young", "aper", "rhs"])
    E = 1e10 * np.exp(0.5 * rs["young"].standard_normal(ne ** 3)).reshape(ne, ne, ne)  # [k,j,i]
    K0 = q1_unit_stiffness(nu)
    Epad = np.zeros((ne + 2, ne + 2, ne + 2))
    Epad[1:-1, 1:-1, 1:-1] = E * h
    kk, jj, ii = np.meshgrid(np.arange(nn1), np.arange(nn1), np.arange(nn1), indexing="ij")
    bnd = (ii == 0) | (ii == ne) | (jj == 0) | (jj == ne) | (kk == 0) | (kk == ne)
    bnd = bnd.ravel()
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    blocks = np.zeros((27, NN, 3, 3))
    for o, (dx, dy, dz) in enumerate(offs):
        acc = np.zeros((nn1, nn1, nn1, 3, 3))
        for c in (0, 1):
            for b_ in (0, 1):
                for a in (0, 1):
                    a2, b2, c2 = a + dx, b_ + dy, c + dz
                    if not (0 <= a2 <= 1 and 0 <= b2 <= 1 and 0 <= c2 <= 1):
                        continue
                    q1, q2 = a + 2 * b_ + 4 * c, a2 + 2 * b2 + 4 * c2
                    # element (i-a, j-b, k-c) in padded coordinates (+1)
                    Ee = Epad[1 - c:1 - c + nn1, 1 - b_:1 - b_ + nn1, 1 - a:1 - a + nn1]
                    acc += Ee[..., None, None] * K0[3 * q1:3 * q1 + 3, 3 * q2:3 * q2 + 3]
        blocks[o] = acc.reshape(NN, 3, 3)
    node = np.arange(NN)
    ni, nj, nk = ii.ravel(), jj.ravel(), kk.ravel()
    rows, cols, vals = [], [], []
    for o, (dx, dy, dz) in enumerate(offs):
        ti, tj, tk = ni + dx, nj + dy, nk + dz
        ok = (ti >= 0) & (ti <= ne) & (tj >= 0) & (tj <= ne) & (tk >= 0) & (tk <= ne)
        tgt = ti + nn1 * (tj + nn1 * tk)
        ok &= ~bnd
        ok[ok] &= ~bnd[tgt[ok]]
        rows.append(node[ok]); cols.append(tgt[ok]); vals.append(blocks[o][ok])
    rows.append(node[bnd]); cols.append(node[bnd])
    vals.append(np.broadcast_to(np.eye(3), (int(bnd.sum()), 3, 3)))
    # fracture
    nfe = nf * nf
    f0 = ne // 8
    jplane = ne // 2
    w = rs["aper"].uniform(1e-4, 1e-3, nfe)
    Ae = h * h
    tf = w ** 3 / (12 * eta)
    fidx = np.arange(nfe).reshape(nf, nf)  # [fz, fx]
    pp_r, pp_c, pp_v = [np.arange(nfe)], [np.arange(nfe)], [w * Ae / (Kf * dt)]
    for a_, b_ in ((fidx[:, :-1], fidx[:, 1:]), (fidx[:-1, :], fidx[1:, :])):
        a_ = a_.ravel(); b_ = b_.ravel()
        T = 2 * tf[a_] * tf[b_] / (tf[a_] + tf[b_])
        for x_, y_ in ((a_, b_), (b_, a_)):
            pp_r += [x_, x_]; pp_c += [x_, y_]; pp_v += [T, -T]
    pp_r = np.concatenate(pp_r); pp_c = np.concatenate(pp_c); pp_v = np.concatenate(pp_v)
    fx, fz = np.arange(nfe) % nf, np.arange(nfe) // nf
    corners = []
    for a, c in ((0, 0), (1, 0), (0, 1), (1, 1)):
        corners.append((f0 + fx + a) + nn1 * (jplane + nn1 * (f0 + fz + c)))
    corners = np.stack(corners, 1)  # [nfe, 4]
    # per-field symmetric scaling
    diag_u = blocks[13][~bnd][:, [0, 1, 2], [0, 1, 2]]
    su = 1.0 / np.sqrt(np.median(diag_u))
    dpp = np.bincount(pp_r, weights=np.where(pp_r == pp_c, pp_v, 0.0), minlength=nfe)
    sp = 1.0 / np.sqrt(np.median(dpp))
    # scale the u-u values (identity rows stay identity)
    for t in range(len(vals) - 1):
        vals[t] = vals[t] * su * su
    # coupling blocks, pressure packed 3 per block row at NN + f // 3
    prow = NN + np.arange(nfe) // 3
    pcomp = np.arange(nfe) % 3
    up_rows, up_cols, up_vals = [], [], []
    pu_rows, pu_cols, pu_vals = [], [], []
    for q in range(4):
        blk = np.zeros((nfe, 3, 3))
        blk[np.arange(nfe), 1, pcomp] = -Ae / 4 * su * sp
        up_rows.append(corners[:, q]); up_cols.append(prow); up_vals.append(blk)
        blk2 = np.zeros((nfe, 3, 3))
        blk2[np.arange(nfe), pcomp, 1] = Ae / (4 * dt) * su * sp
        pu_rows.append(prow); pu_cols.append(corners[:, q]); pu_vals.append(blk2)
    ppb = np.zeros((pp_r.size, 3, 3))
    ppb[np.arange(pp_r.size), pp_r % 3, pp_c % 3] = pp_v * sp * sp
    nbp = (nfe + 2) // 3
    rows += up_rows + pu_rows + [NN + pp_r // 3]
    cols += up_cols + pu_cols + [NN + pp_c // 3]
    vals += up_vals + pu_vals + [ppb]
    nb = NN + nbp
    # the padded tail of the last pressure block row (if nfe % 3) gets identity
    npad = nbp * 3 - nfe
    if npad:
        pb = np.zeros((1, 3, 3))
        for t in range(3 - npad, 3):
            pb[0, t, t] = 1.0
        rows.append(np.array([nb - 1])); cols.append(np.array([nb - 1])); vals.append(pb)
    rp, ci, val = assemble_bsr(nb, 3, np.concatenate(rows), np.concatenate(cols),
                               np.concatenate(vals, 0))
    rhs = rs["rhs"].standard_normal(nb * 3)
    if npad:
        rhs[-npad:] = 0.0
    meta = dict(ne=ne, nf=nf, seed=seed, su=su, sp=sp, strategy=strategy)
    if strategy == "mgr_u":
        lvl = np.concatenate([np.zeros(NN * 3, np.int8), np.ones(nbp * 3, np.int8)])
        if npad:
            lvl[-npad:] = 0
        return BlockSystem(name=name, b=3, row_ptr=rp, col_idx=ci, val=val, dof_level=lvl,
                           num_levels=1, rhs=rhs, relax=["amg"], num_functions=1,
                           relax_functions=[3], n_pad=npad, meta=meta)
    if strategy != "mgr_p":
        raise ValueError(f"unknown poromechanics strategy {strategy!r}")
    lvl = np.concatenate([np.ones(NN * 3, np.int8), np.zeros(nbp * 3, np.int8)])
    return BlockSystem(name=name, b=3, row_ptr=rp, col_idx=ci, val=val, dof_level=lvl,
                       num_levels=1, rhs=rhs, relax=["l1_jacobi"], num_functions=3,
                       n_pad=npad, meta=meta)
