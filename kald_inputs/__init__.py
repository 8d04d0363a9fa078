"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Geometry, seeded masses and analytic pair-potential force constants only: no
step of the phonon / linewidth / conductivity computation lives here.
"""

from .system import System
from .lattice import (fcc_primitive, fcc_conventional, l11_binary, reciprocal,
                      mesh_fractions, mesh_qpoints)
from .lj import lj_system, lj_radial, pair_tensors, LJ_EPSILON, LJ_SIGMA, LJ_CUTOFF
from .configs import (Workload, WORKLOADS, c1, c2, c3, c4, c5, small_fcc_prim,
                      small_binary, random_fc3_system, supercell_of, A_FCC,
                      fcc_supercell_system)
from .rng import SplitMix64, shuffled_labels

__all__ = [
    "System", "fcc_primitive", "fcc_conventional", "l11_binary", "reciprocal",
    "mesh_fractions", "mesh_qpoints", "lj_system", "lj_radial", "pair_tensors",
    "LJ_EPSILON", "LJ_SIGMA", "LJ_CUTOFF", "Workload", "WORKLOADS", "c1", "c2",
    "c3", "c4", "c5", "small_fcc_prim", "small_binary", "random_fc3_system",
    "supercell_of", "A_FCC", "fcc_supercell_system", "SplitMix64", "shuffled_labels",
]
