"""Entry-wise comparison of a GPU V-cycle output with the oracle's, shared by
the GPU tests (plain numpy, no GPU)."""
import numpy as np


def cycle_close(sysm, zg, zo, tol, what=""):
    """z = M^{-1} v from the GPU against the oracle's, entry by entry and set
    by set: on every MGR level's F set (dof_level == l) and on the final
    coarse block, the largest entry difference stays within tol times the
    largest oracle entry of that same set.  An error confined to a small set
    (the well dofs of a compositional system, a tiny level) fails here even
    when a 2-norm over all entries would hide it.  Returns the worst ratio."""
    lv = np.asarray(sysm.dof_level)
    worst = 0.0
    for l in range(int(sysm.num_levels) + 1):
        S = lv == l
        if not S.any():
            continue
        m = float(np.max(np.abs(zo[S])))
        d = float(np.max(np.abs(zg[S] - zo[S])))
        assert d <= tol * m, f"{what} set {l} ({int(S.sum())} dofs): max|dz| = {d:.3e} > {tol:g} * {m:.3e}"
        worst = max(worst, d / m if m > 0 else 0.0)
    return worst
