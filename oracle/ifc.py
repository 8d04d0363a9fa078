"""Finite-difference force constants of a pair potential (oracle).

TEST INFRASTRUCTURE ONLY: the library never imports this module.

The paper obtains the second and third order IFCs (Eq. second_and_third_ifc)
by finite differences of forces: an atom is displaced by a small shift along a
Cartesian direction and the change of the forces is recorded (2 N force
evaluations for the second order, 4 N^2 for the third).  With the
home-cell-first storage (code-details appendix) only atoms of the home cell
need displacing for Phi2, and a home atom together with a second atom for
Phi3:

  Phi2_{i a, jR b}       = -[F_{jR b}(+h e_{i a}) - F_{jR b}(-h e_{i a})] / (2 h)
  Phi3_{i a, jRj b, kRk c} = -sum_{s, t = +-1} s t F_{kRk c}(s h e_{i a}, t h e_{jRj b}) / (4 h^2)

(two displacements of the same atom add up).  The forces are the pair forces
of the infinite crystal: F_x = sum over the neighbours m of x, within the
cutoff of the undisplaced structure, of V'(r) (x_m - x_x) / r.

Implemented for the truncated Lennard-Jones pair potential of kald_inputs;
pinned against its analytic derivatives (O(h^2) convergence) and the
acoustic sum rule.
"""

from __future__ import annotations

import numpy as np

from kald_inputs.lattice import neighbour_cells


def lj_dv(r, eps, sig):
    """V'(r) of V = 4 eps [(sig/r)^12 - (sig/r)^6]."""
    sr6 = (sig / r) ** 6
    return 4.0 * eps * (-12.0 * sr6 * sr6 + 6.0 * sr6) / r


def _neighbours(lattice, positions, rc):
    """Per basis atom k: (basis b, cell offset n, vector x_b + n A - x_k) of
    every neighbour within rc."""
    cells = neighbour_cells(lattice, rc)
    shifts = cells @ lattice
    out = []
    for k, xk in enumerate(positions):
        d = positions[None, :, :] + shifts[:, None, :] - xk[None, None, :]
        dist = np.linalg.norm(d, axis=-1)
        c_idx, b_idx = np.nonzero((dist < rc) & (dist > 1e-8))
        out.append((b_idx, cells[c_idx].astype(np.int64), d[c_idx, b_idx]))
    return out


def _force(nbr, k, Rk, disp, eps, sig):
    """Force on atom (k, Rk) with displacements disp = {(atom, cell tuple): vector}."""
    b_idx, n_off, dvec = nbr[k]
    dt = np.zeros(3)
    for (a, cell), v in disp.items():
        if a == k and cell == tuple(Rk):
            dt = dt + v
    d = dvec.copy()
    for (a, cell), v in disp.items():
        m = (b_idx == a) & np.all(n_off + np.asarray(Rk)[None, :] == np.asarray(cell)[None, :], axis=1)
        d[m] += v
    d -= dt[None, :]
    r = np.linalg.norm(d, axis=1)
    return np.sum((lj_dv(r, eps, sig) / r)[:, None] * d, axis=0)


def fd_force_constants(sys, h=1e-3, eps=None, sig=None, rc=None):
    """(fc2 [n_fc2, 3, 3], fc3 [n_fc3, 3, 3, 3]) by central finite differences
    for the blocks listed in sys.fc2_idx / sys.fc3_idx (the sparsity pattern;
    their values are not used).  Potential parameters default to sys.meta."""
    eps = sys.meta["eps"] if eps is None else eps
    sig = sys.meta["sigma"] if sig is None else sig
    rc = sys.meta["rc"] if rc is None else rc
    nbr = _neighbours(sys.lattice, sys.positions, rc)
    e = np.eye(3)
    fc2 = np.zeros((sys.fc2_idx.shape[0], 3, 3))
    for x, key in enumerate(sys.fc2_idx):
        i, j, R = int(key[0]), int(key[1]), tuple(int(v) for v in key[2:5])
        for a in range(3):
            fp = _force(nbr, j, R, {(i, (0, 0, 0)): h * e[a]}, eps, sig)
            fm = _force(nbr, j, R, {(i, (0, 0, 0)): -h * e[a]}, eps, sig)
            fc2[x, a, :] = -(fp - fm) / (2.0 * h)
    fc3 = np.zeros((sys.fc3_idx.shape[0], 3, 3, 3))
    for x, key in enumerate(sys.fc3_idx):
        i = int(key[0])
        j, Rj = int(key[1]), tuple(int(v) for v in key[2:5])
        k, Rk = int(key[5]), tuple(int(v) for v in key[6:9])
        for a in range(3):
            for b in range(3):
                acc = np.zeros(3)
                for s in (1.0, -1.0):
                    for t in (1.0, -1.0):
                        disp = {}
                        for atom, v in (((i, (0, 0, 0)), s * h * e[a]), ((j, Rj), t * h * e[b])):
                            disp[atom] = disp.get(atom, np.zeros(3)) + v
                        acc += s * t * _force(nbr, k, Rk, disp, eps, sig)
                fc3[x, a, b, :] = -acc / (4.0 * h * h)
    return fc2, fc3
