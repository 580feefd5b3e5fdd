"""Container and COO->BSR assembly for the seeded synthetic Jacobians.

This module only stores and assembles input matrices.  It contains none of
the solver's arithmetic (no products, reductions or eliminations of the
multigrid-reduction method); both the CUDA path and the CPU oracle consume
its output.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class BlockSystem:
    """A square block-CSR (BSR) system ``A x = b`` with per-dof MGR labels.

    Layout (block linear system of Sec. 1, Eq. 1):
      * ``row_ptr``  int32[nb+1]   block-row offsets
      * ``col_idx``  int32[nnzb]   block columns, strictly ascending per row
      * ``val``      float64[nnzb, b, b] row-major dense blocks
      * ``dof_level`` int8[nb*b]   level at which each scalar dof is an
        F-point (0..num_levels-1), or ``num_levels`` if it survives to the
        final coarse block that AMG solves
      * ``rhs``      float64[nb*b]
    """

    name: str
    b: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    val: np.ndarray
    dof_level: np.ndarray
    num_levels: int
    rhs: np.ndarray
    # per-level relaxation type names ("jacobi", "l1_jacobi", "block_jacobi",
    # "amg": one AMG V-cycle on A_FF)
    relax: list = field(default_factory=list)
    # AMG "unknown approach" function count on the final coarse block
    num_functions: int = 1
    # per-level function count of an "amg" F-relaxation's hierarchy
    relax_functions: list = field(default_factory=list)
    # dofs that are identity padding (excluded from algorithmic byte counts)
    n_pad: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def nb(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def n(self) -> int:
        return self.nb * self.b

    @property
    def nnzb(self) -> int:
        return int(self.col_idx.shape[0])

    def check(self) -> None:
        """Structural validation (sorted unique columns, diagonal present)."""
        rp, ci = self.row_ptr, self.col_idx
        assert rp.dtype == np.int32 and ci.dtype == np.int32
        assert self.val.dtype == np.float64 and self.val.shape == (ci.size, self.b, self.b)
        assert rp[0] == 0 and rp[-1] == ci.size
        rows = np.repeat(np.arange(self.nb, dtype=np.int64), np.diff(rp))
        if ci.size:
            same = rows[1:] == rows[:-1]
            assert np.all(ci[1:][same] > ci[:-1][same]), "columns not strictly ascending"
        diag = np.zeros(self.nb, dtype=bool)
        diag[rows[ci == rows]] = True
        assert diag.all(), "missing diagonal block"
        assert self.dof_level.shape == (self.n,) and self.dof_level.dtype == np.int8
        assert self.dof_level.min() >= 0 and self.dof_level.max() <= self.num_levels
        assert self.rhs.shape == (self.n,)
        assert np.isfinite(self.val).all() and np.isfinite(self.rhs).all()


def assemble_bsr(nb: int, b: int, rows: np.ndarray, cols: np.ndarray,
                 blocks: np.ndarray):
    """Sum duplicate (row, col) blocks and return sorted BSR arrays."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    blocks = np.asarray(blocks, dtype=np.float64).reshape(-1, b, b)
    key = rows * nb + cols
    order = np.argsort(key, kind="stable")
    key = key[order]
    blocks = blocks[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(blocks, start, axis=0) if key.size else blocks[:0]
    urow = (uniq // nb).astype(np.int64)
    ucol = (uniq % nb).astype(np.int32)
    counts = np.bincount(urow, minlength=nb)
    row_ptr = np.zeros(nb + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr.astype(np.int32), ucol, np.ascontiguousarray(summed)


def scalar_coo_to_bsr1(n: int, rows, cols, vals):
    """Scalar COO (duplicates summed) as a 1x1-block BSR."""
    return assemble_bsr(n, 1, rows, cols, np.asarray(vals).reshape(-1, 1, 1))


def streams(seed: int, names):
    """Independent PCG64 generators, one per named field, from one seed."""
    ss = np.random.SeedSequence(seed)
    kids = ss.spawn(len(names))
    return {nm: np.random.Generator(np.random.PCG64(k)) for nm, k in zip(names, kids)}
