"""The five workloads (C1..C5) and the small systems used by the tests.

C1  fcc LJ, 1-atom primitive cell, 6x6x6 mesh, T = 50 K, sigma = 0.1 THz.
C2  2x2x2 conventional fcc (32 atoms, 96 branches), masses 28.09/72.63 amu at
    50/50 (seed 2), 8x8x8 mesh, T = 300 K, sigma = 0.05 THz.
C3  6x6x6 conventional (864 atoms, 2592 modes), 50/50 masses (seed 3),
    Gamma-only, T = 300 K, sigma = 0.05 THz.
C4  24 Gamma-only supercells: 8 each of 3^3, 4^3, 5^3 conventional cells, seeds
    1000+i, heavy fraction x_i ~ U[0.1, 0.5] drawn from seed 999, T = 300 K,
    sigma = 0.05 THz.
C5  two-atom L1_1 binary on fcc, masses 28.09/72.63, 24x24x24 mesh, T = 300 K,
    sigma = 0.05 THz.
All use LJ eps = 0.0104 eV, sigma_LJ = 3.4 A, cutoff 2.5 sigma_LJ, a = 5.26 A and
a 3-sigma truncation of the Gaussian energy delta.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .lattice import fcc_conventional, fcc_primitive, l11_binary
from .lj import lj_system
from .rng import SplitMix64, shuffled_labels
from .system import System

A_FCC = 5.26
M_AR = 39.95
M_LIGHT = 28.09
M_HEAVY = 72.63


@dataclass
class Workload:
    name: str
    systems: list            # list[System]
    mesh: tuple              # (1,1,1) means Gamma-only
    T: float                 # K
    sigma_thz: float
    n_sigma: float = 3.0
    precision: str = "fp64"  # "fp64" | "fp32"
    description: str = ""

    @property
    def n_q(self) -> int:
        return int(np.prod(self.mesh))

    def unique_triplets(self) -> int:
        """Momentum-conserving projections: one per (q s, q' s', q'' s'') with
        q'' fixed by q and q' (Nk^2 nb^3 per system)."""
        return int(sum(self.n_q ** 2 * s.n_branches ** 3 for s in self.systems))


def binary_masses(n_atoms: int, n_heavy: int, seed: int) -> np.ndarray:
    lab = shuffled_labels(n_atoms, n_heavy, seed)
    return np.where(np.array(lab) == 1, M_HEAVY, M_LIGHT).astype(float)


def fcc_supercell_system(ncell, seed, heavy_fraction=0.5, name="") -> System:
    lat, pos = fcc_conventional(A_FCC, ncell)
    n = pos.shape[0]
    n_heavy = int(np.floor(n * heavy_fraction)) if heavy_fraction == 0.5 else int(round(heavy_fraction * n))
    m = binary_masses(n, n_heavy, seed)
    return lj_system(lat, pos, m, name=name or f"fcc{ncell}conv_seed{seed}")


def c1() -> Workload:
    lat, pos = fcc_primitive(A_FCC)
    s = lj_system(lat, pos, [M_AR], name="fcc_prim_Ar")
    return Workload("C1", [s], (6, 6, 6), 50.0, 0.1, 3.0, "fp64",
                    "fcc LJ 1-atom cell, 6^3 mesh, T=50 K, sigma=0.1 THz")


def c2() -> Workload:
    s = fcc_supercell_system(2, seed=2, name="fcc2conv_32at")
    return Workload("C2", [s], (8, 8, 8), 300.0, 0.05, 3.0, "fp32",
                    "32-atom cubic cell (96 branches), 8^3 mesh, T=300 K, sigma=0.05 THz")


def c3() -> Workload:
    s = fcc_supercell_system(6, seed=3, name="fcc6conv_864at")
    return Workload("C3", [s], (1, 1, 1), 300.0, 0.05, 3.0, "fp32",
                    "864-atom Gamma-only disordered supercell, T=300 K, sigma=0.05 THz")


def c4_fractions() -> list[float]:
    g = SplitMix64(999)
    return [0.1 + 0.4 * g.uniform() for _ in range(24)]


def c4() -> Workload:
    xs = c4_fractions()
    systems = []
    for i in range(24):
        ncell = (3, 4, 5)[i // 8]
        systems.append(fcc_supercell_system(ncell, seed=1000 + i, heavy_fraction=xs[i],
                                            name=f"c4_{i}_fcc{ncell}conv"))
    return Workload("C4", systems, (1, 1, 1), 300.0, 0.05, 3.0, "fp32",
                    "24 Gamma-only supercells of 108/256/500 atoms")


def c5(mesh=(24, 24, 24)) -> Workload:
    lat, pos = l11_binary(A_FCC)
    s = lj_system(lat, pos, [M_LIGHT, M_HEAVY], name="L11_binary")
    return Workload("C5", [s], tuple(mesh), 300.0, 0.05, 3.0, "fp32",
                    "2-atom L1_1 binary, 24^3 mesh, T=300 K, sigma=0.05 THz")


WORKLOADS = {"C1": c1, "C2": c2, "C3": c3, "C4": c4, "C5": c5}


# ---- small systems for tests -------------------------------------------------

def small_fcc_prim(mesh=(3, 3, 3), T=300.0, sigma=0.2) -> Workload:
    lat, pos = fcc_primitive(A_FCC)
    s = lj_system(lat, pos, [M_AR], name="fcc_prim_Ar")
    return Workload("small_prim", [s], tuple(mesh), T, sigma, 3.0, "fp64")


def small_binary(mesh=(3, 3, 3), T=300.0, sigma=0.2) -> Workload:
    lat, pos = l11_binary(A_FCC)
    s = lj_system(lat, pos, [M_LIGHT, M_HEAVY], name="L11_binary")
    return Workload("small_binary", [s], tuple(mesh), T, sigma, 3.0, "fp64")


def random_fc3_system(base: System, n_extra: int, seed: int, scale: float = 0.05) -> System:
    """A copy of `base` whose fc3 gets `n_extra` random blocks with both
    replica vectors non-zero and different (sparsity a pair potential never
    produces), drawn from splitmix64(seed).  Used only to exercise the general
    phase-sum path; it is not symmetrised."""
    g = SplitMix64(seed)
    reps = base.replicas()
    reps = reps[np.any(reps != 0, axis=1)]
    n = base.n_atoms
    idx, val = [], []
    for _ in range(n_extra):
        i = g.below(n)
        j = g.below(n)
        k = g.below(n)
        rj = reps[g.below(len(reps))]
        rk = reps[g.below(len(reps))]
        while np.all(rk == rj):
            rk = reps[g.below(len(reps))]
        idx.append([i, j, *rj, k, *rk])
        val.append([scale * g.normal() for _ in range(27)])
    fc3_idx = np.concatenate([base.fc3_idx, np.array(idx, dtype=np.int32)], axis=0)
    fc3 = np.concatenate([base.fc3, np.array(val).reshape(-1, 3, 3, 3)], axis=0)
    return System(base.masses.copy(), base.positions.copy(), base.lattice.copy(),
                  base.fc2_idx.copy(), base.fc2.copy(), fc3_idx, fc3,
                  name=base.name + f"_rand{n_extra}", meta=dict(base.meta))


def supercell_of(lattice, positions, masses, ncell, name="") -> System:
    """LJ system of the ncell x ncell x ncell repetition of a cell (atoms
    ordered cell-major: atom index = cell_index * n_basis + basis)."""
    lattice = np.asarray(lattice, float)
    positions = np.asarray(positions, float)
    nb = positions.shape[0]
    pos, ms = [], []
    cells = []
    for c0 in range(ncell):
        for c1 in range(ncell):
            for c2 in range(ncell):
                cells.append((c0, c1, c2))
    for c in cells:
        off = np.array(c, float) @ lattice
        for b in range(nb):
            pos.append(positions[b] + off)
            ms.append(masses[b])
    sl = ncell * lattice
    s = lj_system(sl, np.array(pos), np.array(ms), name=name or f"super{ncell}")
    s.meta["cells"] = np.array(cells)
    s.meta["n_basis"] = nb
    return s
