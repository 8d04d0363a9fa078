"""Lattices, supercells and Gamma-centred q-meshes for the synthetic systems.

Everything here is geometry (cell vectors, atom positions, integer mesh
indices); none of it is part of the anharmonic method itself.
"""

from __future__ import annotations

import numpy as np


def fcc_primitive(a: float):
    """One-atom primitive fcc cell (rows = cell vectors), atom at the origin."""
    lat = 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    pos = np.zeros((1, 3))
    return lat, pos


def fcc_conventional(a: float, n: int | tuple[int, int, int]):
    """n1 x n2 x n3 conventional cubic fcc cells (4 atoms each) as one cubic
    cell; atoms ordered by cell (x fastest... z slowest) then basis site."""
    if isinstance(n, int):
        n = (n, n, n)
    basis = 0.5 * a * np.array([[0, 0, 0], [0, 1, 1], [1, 0, 1], [1, 1, 0]], dtype=float)
    pos = []
    for c2 in range(n[2]):
        for c1 in range(n[1]):
            for c0 in range(n[0]):
                off = a * np.array([c0, c1, c2], dtype=float)
                for b in basis:
                    pos.append(off + b)
    lat = a * np.diag(np.array(n, dtype=float))
    return lat, np.array(pos)


def l11_binary(a: float):
    """Two-atom rhombohedral cell of fcc sites coloured by alternating (111)
    planes (L1_1 / CuPt-type order).  Species A at the origin, B at (a/2)(1,1,0).
    Every site keeps the 12 fcc nearest neighbours."""
    lat = 0.5 * a * np.array([[1.0, -1.0, 0.0], [0.0, 1.0, -1.0], [1.0, 2.0, 1.0]])
    pos = 0.5 * a * np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 0.0]])
    return lat, pos


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_i with A_j . b_i = 2 pi delta_ij (Angstrom^-1)."""
    return 2.0 * np.pi * np.linalg.inv(lattice).T


def mesh_fractions(mesh) -> np.ndarray:
    """[Nq, 3] integer mesh coordinates k, index q = (k0*N1 + k1)*N2 + k2."""
    n0, n1, n2 = (int(m) for m in mesh)
    k = np.stack(np.meshgrid(np.arange(n0), np.arange(n1), np.arange(n2), indexing="ij"), axis=-1)
    return k.reshape(-1, 3)


def mesh_qpoints(lattice: np.ndarray, mesh) -> np.ndarray:
    """Cartesian q = sum_i k_i b_i / N_i for the Gamma-centred mesh (1/Angstrom)."""
    k = mesh_fractions(mesh).astype(float)
    frac = k / np.asarray(mesh, dtype=float)[None, :]
    return frac @ reciprocal(lattice)


def neighbour_cells(lattice: np.ndarray, rc: float) -> np.ndarray:
    """All integer cell vectors n that can hold an atom within rc of an atom in
    cell 0 (a safe superset: plane spacing bound plus one cell)."""
    vol = abs(np.linalg.det(lattice))
    nmax = []
    for k in range(3):
        l, m = [x for x in range(3) if x != k]
        spacing = vol / np.linalg.norm(np.cross(lattice[l], lattice[m]))
        nmax.append(int(np.ceil(rc / spacing)) + 1)
    r = [np.arange(-nm, nm + 1) for nm in nmax]
    g = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    return g
