"""Container for one crystal unit cell (or one Gamma-only supercell) in the
sparse atom-block force-constant form that the library boundary takes.

Layout (numpy, C-contiguous):
  masses    [n]               amu
  positions [n, 3]            Cartesian, Angstrom (atoms of the home cell)
  lattice   [3, 3]            rows are the cell vectors A1, A2, A3 (Angstrom)
  fc2_idx   [n_fc2, 5]        int32: i, j, R0, R1, R2 (atom j sits in cell R,
                              R in units of the cell vectors; i in cell 0)
  fc2       [n_fc2, 3, 3]     eV/A^2: d2E / du_{i0,a} du_{jR,b}
  fc3_idx   [n_fc3, 9]        int32: i, j, Rj(3), k, Rk(3)
  fc3       [n_fc3, 3, 3, 3]  eV/A^3: d3E / du_{i0,a} du_{jRj,b} du_{kRk,c}

The first atom of every block is always in the home cell (the home-cell-first storage of the paper's appendix,
"Code details").  A Gamma-only supercell is the same structure with mesh 1x1x1:
the cell vectors are the supercell vectors, and R keeps the image each pair is
seen through, so true interatomic distances stay available.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class System:
    masses: np.ndarray
    positions: np.ndarray
    lattice: np.ndarray
    fc2_idx: np.ndarray
    fc2: np.ndarray
    fc3_idx: np.ndarray
    fc3: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.masses.shape[0])

    @property
    def n_branches(self) -> int:
        return 3 * self.n_atoms

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))

    def replicas(self) -> np.ndarray:
        """Distinct cell vectors (integer triples) used by any block."""
        r = [self.fc2_idx[:, 2:5], self.fc3_idx[:, 2:5], self.fc3_idx[:, 6:9]]
        return np.unique(np.concatenate(r, axis=0), axis=0)

    def validate(self) -> None:
        n = self.n_atoms
        assert self.positions.shape == (n, 3)
        assert self.lattice.shape == (3, 3)
        assert self.fc2_idx.shape[1] == 5 and self.fc2.shape[1:] == (3, 3)
        assert self.fc3_idx.shape[1] == 9 and self.fc3.shape[1:] == (3, 3, 3)
        assert self.fc2_idx.shape[0] == self.fc2.shape[0]
        assert self.fc3_idx.shape[0] == self.fc3.shape[0]
        for a in (self.fc2_idx[:, 0], self.fc2_idx[:, 1], self.fc3_idx[:, 0],
                  self.fc3_idx[:, 1], self.fc3_idx[:, 5]):
            assert a.min() >= 0 and a.max() < n
        assert np.all(self.masses > 0)

    def contiguous(self) -> "System":
        """Copy with every array C-contiguous in the dtypes the boundary takes."""
        return System(
            masses=np.ascontiguousarray(self.masses, dtype=np.float64),
            positions=np.ascontiguousarray(self.positions, dtype=np.float64),
            lattice=np.ascontiguousarray(self.lattice, dtype=np.float64),
            fc2_idx=np.ascontiguousarray(self.fc2_idx, dtype=np.int32),
            fc2=np.ascontiguousarray(self.fc2, dtype=np.float64),
            fc3_idx=np.ascontiguousarray(self.fc3_idx, dtype=np.int32),
            fc3=np.ascontiguousarray(self.fc3, dtype=np.float64),
            name=self.name, meta=dict(self.meta))
