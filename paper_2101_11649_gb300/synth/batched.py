"""A batch of two-phase Jacobians of uneven sizes (many time steps / models).

Recipe: member i is the two-phase TPFA system with seed 1000 + i and grid
nx, ny ~ U{16..96}, nz ~ U{16..48} drawn from one PCG64 stream (seed 0);
member 0 is forced to 16^3.  The loss weights w_i ~ N(0,1) per unknown
come from a second stream.
"""
from __future__ import annotations

import numpy as np

from .bsr import streams
from .two_phase import make_two_phase


def batch_grids(nsys=48, seed=0, lo=16, hi_xy=96, hi_z=48):
    rs = streams(seed, ["grid"])["grid"]
    g = []
    for i in range(nsys):
        nx, ny = (int(v) for v in rs.integers(lo, hi_xy + 1, 2))
        nz = int(rs.integers(lo, hi_z + 1))
        g.append((16, 16, 16) if i == 0 else (nx, ny, nz))
    return g


def make_batch(nsys=48, seed=0, grids=None):
    grids = grids or batch_grids(nsys, seed)
    systems = [make_two_phase(*grids[i], seed=1000 + i, name=f"two_phase_{i}")
               for i in range(len(grids))]
    ws = streams(seed, ["grid", "loss"])["loss"]
    weights = [ws.standard_normal(s.n) for s in systems]
    return systems, weights
