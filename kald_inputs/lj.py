"""Analytic second- and third-order force constants of a truncated
Lennard-Jones pair potential, in the home-cell-first sparse block form.

This stands in for the external force calculators that produce the IFCs in
the paper (Eq. potential_expansion, Eq. second_and_third_ifc): the pair
potential V(r) = 4 eps [(s/r)^12 - (s/r)^6], r < rc, is differentiated by the
chain rule.  For a pair (a, b) with r = x_b - x_a, unit vector e = r/|r|:

  K_ab   = V'' e_a e_b + (V'/r)(d_ab - e_a e_b)                 (d2V/dr_a dr_b)
  T_abc  = (V''' - 3V''/r + 3V'/r^2) e_a e_b e_c
           + (V''/r - V'/r^2)(d_ab e_c + d_ac e_b + d_bc e_a)      (d3V/dr^3)

and each derivative taken with respect to the displacement of atom a (rather
than b) brings a factor -1.  No energy shift is needed: only derivatives enter.
"""

from __future__ import annotations

from collections import defaultdict

import numpy as np

from .lattice import neighbour_cells
from .system import System

LJ_EPSILON = 0.0104   # eV
LJ_SIGMA = 3.4        # Angstrom
LJ_CUTOFF = 2.5 * LJ_SIGMA


def lj_radial(r, eps=LJ_EPSILON, sig=LJ_SIGMA):
    """V, V', V'', V''' of the LJ pair potential at distance r."""
    sr6 = (sig / r) ** 6
    sr12 = sr6 * sr6
    v = 4 * eps * (sr12 - sr6)
    v1 = 4 * eps * (-12 * sr12 + 6 * sr6) / r
    v2 = 4 * eps * (156 * sr12 - 42 * sr6) / r ** 2
    v3 = 4 * eps * (-2184 * sr12 + 336 * sr6) / r ** 3
    return v, v1, v2, v3


def pair_tensors(rvec, eps=LJ_EPSILON, sig=LJ_SIGMA):
    """K [.., 3, 3] and T [.., 3, 3, 3] for separation vectors rvec [.., 3]."""
    r = np.linalg.norm(rvec, axis=-1)
    e = rvec / r[..., None]
    _, v1, v2, v3 = lj_radial(r, eps, sig)
    eye = np.eye(3)
    ee = e[..., :, None] * e[..., None, :]
    K = v2[..., None, None] * ee + (v1 / r)[..., None, None] * (eye - ee)
    a = (v3 - 3 * v2 / r + 3 * v1 / r ** 2)[..., None, None, None]
    b = (v2 / r - v1 / r ** 2)[..., None, None, None]
    eee = ee[..., :, :, None] * e[..., None, None, :]
    dterm = (eye[:, :, None] * e[..., None, None, :]
             + eye[:, None, :] * e[..., None, :, None]
             + eye[None, :, :] * e[..., :, None, None])
    T = a * eee + b * dterm
    return K, T


def neighbour_list(lattice, positions, rc):
    """(i, j, n, rvec) for every ordered pair with 0 < |x_j + n.A - x_i| < rc."""
    cells = neighbour_cells(lattice, rc)
    shifts = cells @ lattice
    out_i, out_j, out_n, out_r = [], [], [], []
    for i, xi in enumerate(positions):
        d = positions[None, :, :] + shifts[:, None, :] - xi[None, None, :]   # [C, n, 3]
        dist = np.linalg.norm(d, axis=-1)
        c_idx, j_idx = np.nonzero((dist < rc) & (dist > 1e-8))
        out_i.append(np.full(c_idx.shape, i))
        out_j.append(j_idx)
        out_n.append(cells[c_idx])
        out_r.append(d[c_idx, j_idx])
    return (np.concatenate(out_i), np.concatenate(out_j),
            np.concatenate(out_n).astype(np.int64), np.concatenate(out_r))


def lj_system(lattice, positions, masses, rc=LJ_CUTOFF, eps=LJ_EPSILON,
              sig=LJ_SIGMA, name="") -> System:
    """Build the System with analytic LJ fc2/fc3 blocks (home atom first).

    fc2: (i, jR) = -K(r) for each neighbour, (i, i0) = sum of K.
    fc3 per neighbour pair (i, jR): (i;i0;i0) += -T, (i;i0;jR) += T,
    (i;jR;i0) += T, (i;jR;jR) += -T.
    """
    lattice = np.asarray(lattice, dtype=float)
    positions = np.asarray(positions, dtype=float)
    n_at = positions.shape[0]
    pi, pj, pn, pr = neighbour_list(lattice, positions, rc)
    K, T = pair_tensors(pr, eps, sig)

    fc2 = defaultdict(lambda: np.zeros((3, 3)))
    fc3 = defaultdict(lambda: np.zeros((3, 3, 3)))
    zero = (0, 0, 0)
    for p in range(pi.shape[0]):
        i, j = int(pi[p]), int(pj[p])
        n = tuple(int(x) for x in pn[p])
        fc2[(i, j) + n] = fc2[(i, j) + n] - K[p]
        fc2[(i, i) + zero] = fc2[(i, i) + zero] + K[p]
        fc3[(i, i) + zero + (i,) + zero] = fc3[(i, i) + zero + (i,) + zero] - T[p]
        fc3[(i, i) + zero + (j,) + n] = fc3[(i, i) + zero + (j,) + n] + T[p]
        fc3[(i, j) + n + (i,) + zero] = fc3[(i, j) + n + (i,) + zero] + T[p]
        fc3[(i, j) + n + (j,) + n] = fc3[(i, j) + n + (j,) + n] - T[p]
    k2 = sorted(fc2.keys())
    k3 = sorted(fc3.keys())
    sysm = System(
        masses=np.asarray(masses, dtype=float).reshape(n_at),
        positions=positions,
        lattice=lattice,
        fc2_idx=np.array(k2, dtype=np.int32).reshape(-1, 5),
        fc2=np.array([fc2[k] for k in k2]).reshape(-1, 3, 3),
        fc3_idx=np.array(k3, dtype=np.int32).reshape(-1, 9),
        fc3=np.array([fc3[k] for k in k3]).reshape(-1, 3, 3, 3),
        name=name,
        meta={"potential": "LJ", "eps": eps, "sigma": sig, "rc": rc},
    )
    sysm.validate()
    return sysm
