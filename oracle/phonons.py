"""Harmonic phonons of the oracle: dynamical matrix, eigenpairs, velocities.

Plain FP64 NumPy/SciPy, one q-point at a time.  TEST INFRASTRUCTURE ONLY:
the library never imports this module.

Conventions (paper, section "Lattice Dynamics"):
  D_{ia,jb}(q) = sum_R Phi2(i0, jR)_{ab} / sqrt(m_i m_j) * chi(q, R),
  chi(q, R) = exp(-i q.R)                         (Bloch sum, Eq. before
                                                   eigenvectors_crystal)
  D(q) eta_s = omega_s^2 eta_s                    (Eq. eigenvectors_crystal)
Eigenvectors are returned row-major: eig[q, s, dof] = eta_{dof}(q, s).
Frequencies nu = omega / 2 pi in THz, negative for imaginary modes.

Group velocity (Eq. velocity_crystal, printed garbled; reading): the
Hellmann-Feynman derivative of D with respect to q,
  dD/dq_a = sum_R (-i R_a) Phi2/sqrt(mm) exp(-i q.R),
  V^a_{ss'} = eta_s^dagger (dD/dq_a) eta_s' / (2 sqrt(omega_s omega_s')),
whose diagonal is v_s = d omega_s / dq.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg

from kald_inputs.lattice import mesh_qpoints
from .units import EV_A2_AMU, TWO_PI


def _mass_scaled_fc2(sys):
    m = sys.masses
    i = sys.fc2_idx[:, 0]
    j = sys.fc2_idx[:, 1]
    return sys.fc2 / np.sqrt(m[i] * m[j])[:, None, None]


def dynamical_matrix(sys, q_cart, with_derivative=False, atom_phase=False):
    """D(q) (nb x nb complex, eV/(A^2 amu)); optionally dD/dq_a [3, nb, nb]
    (eV/(A amu)).  atom_phase=True uses the phase exp(-i q.(R + x_j - x_i))
    (the gauge in which the interband velocity of QHGK folds exactly)."""
    n = sys.n_atoms
    nb = 3 * n
    blocks = _mass_scaled_fc2(sys)
    i = sys.fc2_idx[:, 0]
    j = sys.fc2_idx[:, 1]
    R = sys.fc2_idx[:, 2:5].astype(float) @ sys.lattice          # [B, 3] Cartesian
    if atom_phase:
        R = R + sys.positions[j] - sys.positions[i]
    ph = np.exp(-1j * (R @ q_cart))                              # [B]
    # scatter-add every block into its (i, j) 3x3 position
    rows = (3 * i[:, None, None] + np.arange(3)[None, :, None]) * nb
    cols = 3 * j[:, None, None] + np.arange(3)[None, None, :]
    flat = (rows + cols).reshape(-1)
    D = np.zeros(nb * nb, dtype=complex)
    np.add.at(D, flat, (blocks * ph[:, None, None]).reshape(-1))
    D = D.reshape(nb, nb)
    dD = None
    if with_derivative:
        dD = np.zeros((3, nb * nb), dtype=complex)
        for a in range(3):
            np.add.at(dD[a], flat, ((-1j * R[:, a] * ph)[:, None, None] * blocks).reshape(-1))
        dD = dD.reshape(3, nb, nb)
    D = 0.5 * (D + D.conj().T)
    if with_derivative:
        dD = 0.5 * (dD + np.conj(np.transpose(dD, (0, 2, 1))))
        return D, dD
    return D


def eigvals_to_thz(lam):
    """omega = sign(lam) sqrt(|lam| * EV_A2_AMU) rad/ps, nu = omega / 2 pi."""
    return np.sign(lam) * np.sqrt(np.abs(lam) * EV_A2_AMU) / TWO_PI


def phonons(sys, mesh):
    """nu [Nq, nb] THz and eig [Nq, nb(mode), nb(dof)] complex for the
    Gamma-centred mesh.  scipy.linalg.eigh returns ascending eigenvalues."""
    qs = mesh_qpoints(sys.lattice, mesh)
    nb = 3 * sys.n_atoms
    nu = np.zeros((qs.shape[0], nb))
    eig = np.zeros((qs.shape[0], nb, nb), dtype=complex)
    for k, q in enumerate(qs):
        D = dynamical_matrix(sys, q)
        if not np.any(D.imag):
            # a real D (q = 0, or a Gamma-only supercell): real eigenvectors
            lam, vec = scipy.linalg.eigh(D.real)
        else:
            lam, vec = scipy.linalg.eigh(D)
        nu[k] = eigvals_to_thz(lam)
        eig[k] = vec.T
    return nu, eig


def velocity_matrices(sys, q_cart, eig_q, nu_q, atom_phase=False):
    """V^a_{ss'} [3, nb, nb] in A/ps (generalised velocity at one q).  Rows of
    eig_q are the eigenvectors; modes with nu <= 0 get zero rows/columns."""
    _, dD = dynamical_matrix(sys, q_cart, with_derivative=True, atom_phase=atom_phase)
    omega = TWO_PI * nu_q
    good = omega > 0
    w = np.where(good, omega, 1.0)
    E = eig_q.T                                        # columns = modes
    V = np.stack([E.conj().T @ dD[a] @ E for a in range(3)])   # eta^dagger dD eta
    V = V * EV_A2_AMU / (2.0 * np.sqrt(np.outer(w, w)))[None]
    V[:, ~good, :] = 0.0
    V[:, :, ~good] = 0.0
    return V


def group_velocities(sys, mesh, nu, eig):
    """Diagonal v [Nq, nb, 3] (A/ps) = Re V^a_{ss}."""
    qs = mesh_qpoints(sys.lattice, mesh)
    out = np.zeros(nu.shape + (3,))
    for k, q in enumerate(qs):
        V = velocity_matrices(sys, q, eig[k], nu[k])
        out[k] = np.real(np.einsum("ass->sa", V))
    return out


def degenerate_sets(nu_q, tol):
    """Groups of mode indices whose frequencies chain within tol (THz)."""
    order = np.argsort(nu_q, kind="stable")
    sets, cur = [], [int(order[0])]
    for a, b in zip(order[:-1], order[1:]):
        if abs(nu_q[b] - nu_q[a]) < tol:
            cur.append(int(b))
        else:
            sets.append(cur)
            cur = [int(b)]
    sets.append(cur)
    return sets
