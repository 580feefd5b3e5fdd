"""Seeded synthetic Jacobians shaped like the paper's three applications.

Inputs only: every generator returns a :class:`BlockSystem` and holds none of
the multigrid-reduction arithmetic.  Both the CUDA path and the CPU oracle
read these systems.
"""
from .bsr import BlockSystem, assemble_bsr
from .two_phase import make_two_phase
from .mimetic import make_mimetic
from .compositional import make_compositional
from .poromech import make_poromech
from .batched import make_batch, batch_grids

# The named workloads at full size (small variants for fast tests); the
# mimetic (consistent MGR_P, TPFA MGR_Pi), compositional (3- and 4-level)
# and fracture (MGR_P, MGR_U) systems come with two variants each.
CONFIGS = {
    "two_phase_16x16x8": lambda: make_two_phase(16, 16, 8),
    "mimetic_64": lambda: make_mimetic(64, 64, 64),
    "mimetic_64_tpfa_mgr_pi": lambda: make_mimetic(64, 64, 64, name="mimetic_tpfa",
                                                   scheme="tpfa", strategy="mgr_pi"),
    "compositional_128x128x32": lambda: make_compositional(128, 128, 32),
    "compositional_128x128x32_4level": lambda: make_compositional(
        128, 128, 32, name="compositional_4level", strategy="mgr4"),
    "poromech_64": lambda: make_poromech(64, 48),
    "poromech_64_mgr_u": lambda: make_poromech(64, 48, name="poromech_mgr_u", strategy="mgr_u"),
}

__all__ = ["BlockSystem", "assemble_bsr", "make_two_phase", "make_mimetic",
           "make_compositional", "make_poromech", "make_batch", "batch_grids", "CONFIGS"]
