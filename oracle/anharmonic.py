"""Three-phonon linewidths of the oracle, written from the paper's equations.

Plain FP64 NumPy/SciPy.  TEST INFRASTRUCTURE ONLY: the library never imports
this module, and this module imports nothing from the library.

Definitions followed (paper, section "Boltzman Transport Equation"):
  populations      n = 1 / (exp(hbar omega / kB T) - 1)           Eq. bose_einstein
                   classical: n = kB T / (hbar omega)               Eq. classic_n
  projection       phi^+-(qs, q's', q''s'') = sum_{i, l'i', l''i''}
                     Phi3 / sqrt(m m' m'') eta_i(qs) eta^+-_i'(q's')
                     eta*_i''(q''s'') chi^+-(q', l') chi*(q'', l'')   Eq. projection_plus
                   eta^+ = eta, chi^+ = chi; eta^- = eta*, chi^- = chi*;
                   chi(q, l) = exp(-i q.R_l); q'' = q +- q' (mod G)  Eq. delta_deconstructed
  rates            Gamma^+- = (hbar pi / 8) g^+- |phi^+-|^2 / (omega omega' omega'')
                                                                      Eq. gamma_operators
  phase space      g^+ = (n' - n'') delta(omega + omega' - omega'')
                   g^- = (1 + n' + n'') delta(omega - omega' - omega'')  Eq. phase_space
  linewidth        gamma_mu = Gamma^0_mu = (1/N_k) sum_{mu' mu''}
                                (Gamma^+ + 1/2 Gamma^-)
  full scattering  Gamma~_{mu mu'} = delta Gamma^0_mu + Gamma^1_{mu mu'}, Gamma^1 from
  operator         the four rate terms of section "Boltzman Transport Equation"
                   (see scattering_matrix)
Readings where the paper is silent or inconsistent:
  * the 1/2 on Gamma^- (present in the linearised BTE, absent from the
    printed Gamma^0) and the 1/N_k (present in the BTE, absent from Gamma^0)
    are both included; the 1/N_k is pinned by the supercell folding test;
  * delta is a Gaussian in angular frequency with standard deviation
    2 pi sigma (sigma in THz), truncated at |d nu| < n_sigma sigma (strict),
    not renormalised; the Lorentzian (half width at half maximum 2 pi sigma)
    and the triangle (half base 2 pi sigma) of the code's options are
    truncated the same way (`delta` argument);
  * modes with nu < omega_min are excluded as mu, mu' and mu'' (their gamma is 0);
  * gamma is averaged over degenerate sets |d nu| < degen_tol at each q.
Units: gamma in ps^-1 (an angular-frequency rate), tau = 1 / (2 gamma) in ps.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse

from kald_inputs.lattice import mesh_fractions, mesh_qpoints
from .phonons import degenerate_sets
from .units import EV_A2_AMU, HBAR_EVPS, KB_EVK, TWO_PI


def bose(omega, T, classical=False):
    """n(omega) at temperature T (omega in rad/ps); 0 where omega <= 0."""
    omega = np.asarray(omega, dtype=float)
    out = np.zeros_like(omega)
    good = omega > 0
    x = HBAR_EVPS * omega[good] / (KB_EVK * T)
    if classical:
        out[good] = 1.0 / x
    else:
        out[good] = 1.0 / np.expm1(np.minimum(x, 700.0))   # n underflows to ~0 beyond
    return out


def gaussian_delta(d_omega, sigma_omega, n_sigma):
    """Gaussian delta in angular frequency (ps), zero for |d| >= n_sigma sigma."""
    d_omega = np.asarray(d_omega)
    g = np.exp(-0.5 * (d_omega / sigma_omega) ** 2) / (np.sqrt(2 * np.pi) * sigma_omega)
    return np.where(np.abs(d_omega) < n_sigma * sigma_omega, g, 0.0)


def lorentzian_delta(d_omega, sigma_omega, n_sigma):
    """Lorentzian delta (ps), half width at half maximum sigma:
    (sigma / pi) / (d^2 + sigma^2), zero for |d| >= n_sigma sigma."""
    d_omega = np.asarray(d_omega)
    g = (sigma_omega / np.pi) / (d_omega ** 2 + sigma_omega ** 2)
    return np.where(np.abs(d_omega) < n_sigma * sigma_omega, g, 0.0)


def triangular_delta(d_omega, sigma_omega, n_sigma):
    """Triangular delta (ps) of half base sigma: (1 - |d| / sigma) / sigma for
    |d| < sigma, and zero for |d| >= n_sigma sigma as for the other shapes."""
    d_omega = np.asarray(d_omega)
    g = np.maximum(0.0, 1.0 - np.abs(d_omega) / sigma_omega) / sigma_omega
    return np.where(np.abs(d_omega) < n_sigma * sigma_omega, g, 0.0)


DELTA_SHAPES = ("gaussian", "lorentzian", "triangular")


def energy_delta(d_omega, sigma_omega, n_sigma, shape="gaussian"):
    """The energy-conservation delta of Eq. phase_space in one of the three
    shapes the code-details options list (reading: sigma = 2 pi sigma_THz is
    the standard deviation, the half width at half maximum, or the half base)."""
    if shape == "gaussian":
        return gaussian_delta(d_omega, sigma_omega, n_sigma)
    if shape == "lorentzian":
        return lorentzian_delta(d_omega, sigma_omega, n_sigma)
    if shape == "triangular":
        return triangular_delta(d_omega, sigma_omega, n_sigma)
    raise ValueError(f"unknown delta shape {shape!r}")


def mesh_index(mesh, k):
    """Flat index of integer mesh coordinates (taken modulo the mesh)."""
    n0, n1, n2 = mesh
    k = np.asarray(k) % np.asarray(mesh)
    return (k[..., 0] * n1 + k[..., 1]) * n2 + k[..., 2]


def mass_scaled_eigvecs(sys, eig):
    """eps[q, s, dof] = eta[q, s, dof] / sqrt(m_atom(dof))."""
    m = np.repeat(sys.masses, 3)
    return eig / np.sqrt(m)[None, None, :]


def fc3_scatter_matrix(sys):
    """Sparse map from per-block phases to the dense nb^3 array:
    M[(a, b, c)] = sum_blocks Phi3[block, alpha, beta, gamma] * P[block]
    with a = 3 i + alpha, b = 3 j + beta, c = 3 k + gamma."""
    nb = 3 * sys.n_atoms
    nblk = sys.fc3.shape[0]
    i = sys.fc3_idx[:, 0]
    j = sys.fc3_idx[:, 1]
    k = sys.fc3_idx[:, 5]
    al = np.arange(3)
    a = 3 * i[:, None, None, None] + al[None, :, None, None]
    b = 3 * j[:, None, None, None] + al[None, None, :, None]
    c = 3 * k[:, None, None, None] + al[None, None, None, :]
    rows = ((a * nb + b) * nb + c).reshape(-1)
    cols = np.repeat(np.arange(nblk), 27)
    vals = sys.fc3.reshape(-1)
    return scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(nb ** 3, nblk))


def projections(sys, mesh, eps, q, qp_list, process, S=None):
    """phi^{+-}(s, s', s'') for the triplets (q, q', q'' = q +- q'), one array
    [len(qp_list), nb, nb, nb] (Eq. projection_plus).  eps = mass-scaled
    eigenvectors [Nq, nb, nb] (rows = modes)."""
    nb = 3 * sys.n_atoms
    if S is None:
        S = fc3_scatter_matrix(sys)
    kf = mesh_fractions(mesh)
    qcart = mesh_qpoints(sys.lattice, mesh)
    Rj = sys.fc3_idx[:, 2:5].astype(float) @ sys.lattice
    Rk = sys.fc3_idx[:, 6:9].astype(float) @ sys.lattice
    qp_list = np.asarray(qp_list, dtype=int)
    sign = 1 if process == "+" else -1
    qpp = mesh_index(mesh, kf[q][None, :] + sign * kf[qp_list])          # q'' = q +- q'
    # chi^+-(q', l'): exp(-i q'.R) for +, its conjugate for -
    chi_p = np.exp(-1j * sign * (Rj @ qcart[qp_list].T))                  # [B, X]
    # chi*(q'', l''); a reciprocal-lattice shift G leaves exp(-i G.R) = 1
    chi_pp = np.exp(+1j * (Rk @ qcart[qpp].T))                            # [B, X]
    M = (S @ (chi_p * chi_pp)).T.reshape(len(qp_list), nb, nb, nb)
    eps_p = eps[qp_list] if process == "+" else eps[qp_list].conj()
    return np.einsum("xabc,sa,xtb,xuc->xstu", M, eps[q], eps_p, eps[qpp].conj(),
                     optimize=True)


def linewidths(sys, mesh, nu, eig, T, sigma_thz, n_sigma=3.0, omega_min_thz=0.01,
               degen_tol_thz=1e-5, classical=False, q_list=None, average=True,
               return_parts=False, delta="gaussian"):
    """gamma [len(q_list), nb] in ps^-1 for the crystal on the mesh.

    Both processes are computed literally: for each q' the + triplet uses
    q'' = q + q' and the - triplet q'' = q - q'.
    """
    nq, nb = nu.shape
    if q_list is None:
        q_list = list(range(nq))
    omega = TWO_PI * nu
    valid = nu > omega_min_thz
    n = bose(np.where(valid, omega, 0.0), T, classical)
    eps = mass_scaled_eigvecs(sys, eig)
    S = fc3_scatter_matrix(sys)
    kf = mesh_fractions(mesh)
    sig_w = TWO_PI * sigma_thz
    inv_w = np.where(valid, 1.0 / np.where(valid, omega, 1.0), 0.0)
    # (hbar pi / 8) * conversion of phi^2 / omega^3 to ps^-2, per N_k
    pref = HBAR_EVPS * np.pi / 8.0 * EV_A2_AMU ** 3 / nq
    g_plus = np.zeros((len(q_list), nb))
    g_minus = np.zeros((len(q_list), nb))
    chunk = max(1, (1 << 22) // nb ** 3)
    for xi, q in enumerate(q_list):
        for c0 in range(0, nq, chunk):
            qps = np.arange(c0, min(nq, c0 + chunk))
            for proc, sign in (("+", 1), ("-", -1)):
                qpp = mesh_index(mesh, kf[q][None, :] + sign * kf[qps])
                phi = projections(sys, mesh, eps, q, qps, proc, S)
                w = omega[q][None, :, None, None]
                wp = omega[qps][:, None, :, None]
                wpp = omega[qpp][:, None, None, :]
                npr = n[qps][:, None, :, None]
                npp = n[qpp][:, None, None, :]
                if proc == "+":
                    g = (npr - npp) * energy_delta(w + wp - wpp, sig_w, n_sigma, delta)
                else:
                    g = 0.5 * (1.0 + npr + npp) * energy_delta(w - wp - wpp, sig_w, n_sigma, delta)
                mask = (valid[q][None, :, None, None] & valid[qps][:, None, :, None]
                        & valid[qpp][:, None, None, :])
                wt = (g * inv_w[q][None, :, None, None] * inv_w[qps][:, None, :, None]
                      * inv_w[qpp][:, None, None, :])
                contrib = np.sum(np.where(mask, wt * np.abs(phi) ** 2, 0.0), axis=(0, 2, 3))
                if proc == "+":
                    g_plus[xi] += pref * contrib
                else:
                    g_minus[xi] += pref * contrib
    gamma = g_plus + g_minus
    if average:
        for xi, q in enumerate(q_list):
            gamma[xi] = degenerate_average(nu[q], gamma[xi], degen_tol_thz)
    if return_parts:
        return gamma, g_plus, g_minus
    return gamma


def phase_space(mesh, nu, T, sigma_thz, n_sigma=3.0, omega_min_thz=0.01, classical=False,
                return_parts=False, delta="gaussian"):
    """Normalised phase space per mode g_mu = (1/N_k) sum_{mu' mu''} g_{mu mu' mu''}
    (Eq. phase_space and the definition after Eq. delta_deconstructed), [N_k, nb]
    in ps: the weights of Eq. phase_space over the momentum-conserving
    triplets (q'' = q +- q'), with the same readings as `linewidths` (1/2 on
    the - process, Gaussian delta, masked modes).  No matrix elements enter."""
    nq, nb = nu.shape
    omega = TWO_PI * nu
    valid = nu > omega_min_thz
    n = bose(np.where(valid, omega, 0.0), T, classical)
    kf = mesh_fractions(mesh)
    sig_w = TWO_PI * sigma_thz
    g_plus = np.zeros((nq, nb))
    g_minus = np.zeros((nq, nb))
    qps = np.arange(nq)
    for q in range(nq):
        for sign in (1, -1):
            qpp = mesh_index(mesh, kf[q][None, :] + sign * kf[qps])
            w = omega[q][None, :, None, None]
            wp = omega[qps][:, None, :, None]
            wpp = omega[qpp][:, None, None, :]
            npr = n[qps][:, None, :, None]
            npp = n[qpp][:, None, None, :]
            mask = (valid[q][None, :, None, None] & valid[qps][:, None, :, None]
                    & valid[qpp][:, None, None, :])
            if sign == 1:
                g = (npr - npp) * energy_delta(w + wp - wpp, sig_w, n_sigma, delta)
                g_plus[q] += np.sum(np.where(mask, g, 0.0), axis=(0, 2, 3)) / nq
            else:
                g = 0.5 * (1.0 + npr + npp) * energy_delta(w - wp - wpp, sig_w, n_sigma, delta)
                g_minus[q] += np.sum(np.where(mask, g, 0.0), axis=(0, 2, 3)) / nq
    if return_parts:
        return g_plus + g_minus, g_plus, g_minus
    return g_plus + g_minus


def scattering_matrix(sys, mesh, nu, eig, T, sigma_thz, n_sigma=3.0, omega_min_thz=0.01,
                      classical=False, delta="gaussian"):
    """The full linearised-BTE scattering operator of section "Boltzman
    Transport Equation": Gamma~_{mu mu'} = delta_{mu mu'} Gamma^0_mu + Gamma^1_{mu mu'}
    with (flat mode index mu = q nb + s)
      Gamma^0_mu      = sum_{mu' mu''} (Gamma^+_{mu mu' mu''} + Gamma^-_{mu mu' mu''})
      Gamma^1_{mu mu'} = (omega_mu' / omega_mu) sum_{mu''} (Gamma^+_{mu mu' mu''}
                         - Gamma^+_{mu mu'' mu'} - Gamma^-_{mu mu' mu''} - Gamma^-_{mu mu'' mu'}).
    Gamma^+- are the rates of Eq. gamma_operators with the same readings as
    `linewidths` (1/N_k, the 1/2 on Gamma^-, Gaussian delta, masked modes);
    no degenerate averaging, so Gamma^0 is the unaveraged linewidth.  For each
    rate Gamma^+-_{mu a b} of a triplet (mu; a = (q', s'); b = (q'', s'')), the
    sum over mu'' places (omega_a / omega_mu) Gamma^+-_{mu a b} at column a with
    the sign of the first (+) or third (-) term, and (omega_b / omega_mu)
    Gamma^+-_{mu a b} at column b with the sign of the second or fourth.
    Returns (gamma0 [N], G1 [N, N]), N = N_k nb, in ps^-1."""
    nq, nb = nu.shape
    N = nq * nb
    omega = TWO_PI * nu
    valid = nu > omega_min_thz
    n = bose(np.where(valid, omega, 0.0), T, classical)
    eps = mass_scaled_eigvecs(sys, eig)
    S = fc3_scatter_matrix(sys)
    kf = mesh_fractions(mesh)
    sig_w = TWO_PI * sigma_thz
    inv_w = np.where(valid, 1.0 / np.where(valid, omega, 1.0), 0.0)
    pref = HBAR_EVPS * np.pi / 8.0 * EV_A2_AMU ** 3 / nq
    gamma0 = np.zeros(N)
    G1 = np.zeros((N, N))
    qps = np.arange(nq)
    for q in range(nq):
        rows = slice(q * nb, (q + 1) * nb)
        for proc, sign in (("+", 1), ("-", -1)):
            qpp = mesh_index(mesh, kf[q][None, :] + sign * kf[qps])
            phi = projections(sys, mesh, eps, q, qps, proc, S)            # [q', s, s', s'']
            w = omega[q][None, :, None, None]
            wp = omega[qps][:, None, :, None]
            wpp = omega[qpp][:, None, None, :]
            npr = n[qps][:, None, :, None]
            npp = n[qpp][:, None, None, :]
            if proc == "+":
                g = (npr - npp) * energy_delta(w + wp - wpp, sig_w, n_sigma, delta)
            else:
                g = 0.5 * (1.0 + npr + npp) * energy_delta(w - wp - wpp, sig_w, n_sigma, delta)
            mask = (valid[q][None, :, None, None] & valid[qps][:, None, :, None]
                    & valid[qpp][:, None, None, :])
            rate = pref * np.where(mask, g * inv_w[q][None, :, None, None] * inv_w[qps][:, None, :, None]
                                   * inv_w[qpp][:, None, None, :] * np.abs(phi) ** 2, 0.0)
            gamma0[rows] += rate.sum(axis=(0, 2, 3))
            # column a = (q', s'): + first term, - third term
            to_a = rate.sum(axis=3)                                       # [q', s, s']
            # column b = (q'', s''): - second term (+ process), - fourth term (- process)
            to_b = rate.sum(axis=2)                                       # [q', s, s'']
            sa = 1.0 if proc == "+" else -1.0
            for x in range(nq):
                ca = slice(qps[x] * nb, (qps[x] + 1) * nb)
                cb = slice(qpp[x] * nb, (qpp[x] + 1) * nb)
                G1[rows, ca] += sa * to_a[x] * omega[qps[x]][None, :] * inv_w[q][:, None]
                G1[rows, cb] -= to_b[x] * omega[qpp[x]][None, :] * inv_w[q][:, None]
    return gamma0, G1


def degenerate_average(nu_q, gamma_q, tol):
    """Average gamma over each degenerate set of one q-point."""
    out = np.array(gamma_q, dtype=float)
    for s in degenerate_sets(nu_q, tol):
        out[s] = np.mean(gamma_q[s])
    return out


def fc3_mode_matrix(sys, eps_mode):
    """Y(b, c) = sum_{blocks} sum_alpha Phi3[block] eps_mode(3 i + alpha), all
    phases 1: the first-index contraction at the Gamma point (nb x nb)."""
    nb = 3 * sys.n_atoms
    i = sys.fc3_idx[:, 0]
    j = sys.fc3_idx[:, 1]
    k = sys.fc3_idx[:, 5]
    e = eps_mode.reshape(-1, 3)[i]                                  # [B, 3]
    w = np.einsum("kabc,ka->kbc", sys.fc3, e)                       # [B, 3, 3]
    al = np.arange(3)
    b = 3 * j[:, None, None] + al[None, :, None]
    c = 3 * k[:, None, None] + al[None, None, :]
    Y = np.zeros(nb * nb, dtype=w.dtype)
    np.add.at(Y, (b * nb + c).reshape(-1), w.reshape(-1))
    return Y.reshape(nb, nb)


def linewidths_gamma_only(sys, nu, eig, T, sigma_thz, n_sigma=3.0, omega_min_thz=0.01,
                          degen_tol_thz=1e-5, classical=False, modes=None, average=True,
                          delta="gaussian"):
    """gamma [len(modes)] (ps^-1) of a Gamma-only supercell with real
    eigenvectors eig [1, nb, nb].  At q = q' = q'' = 0 all phases are 1 and
    phi^+ = phi^- (eta real), so phi(mu, mu', mu'') = eps_mu'^T Y_mu eps_mu''
    with Y_mu the first-index contraction; both weights of Eq. phase_space
    apply to the same projection.  N_k = 1."""
    nb = nu.shape[1]
    if modes is None:
        modes = list(range(nb))
    nu0 = nu[0]
    omega = TWO_PI * nu0
    valid = nu0 > omega_min_thz
    n = bose(np.where(valid, omega, 0.0), T, classical)
    eps = mass_scaled_eigvecs(sys, eig)[0].real
    sig_w = TWO_PI * sigma_thz
    inv_w = np.where(valid, 1.0 / np.where(valid, omega, 1.0), 0.0)
    pref = HBAR_EVPS * np.pi / 8.0 * EV_A2_AMU ** 3
    wp = omega[:, None]
    wpp = omega[None, :]
    npr, npp = n[:, None], n[None, :]
    pair_ok = valid[:, None] & valid[None, :]
    gamma = np.zeros(len(modes))
    for x, mu in enumerate(modes):
        if not valid[mu]:
            continue
        Y = fc3_mode_matrix(sys, eps[mu])
        phi = eps @ Y @ eps.T
        w = omega[mu]
        g = ((npr - npp) * energy_delta(w + wp - wpp, sig_w, n_sigma, delta)
             + 0.5 * (1.0 + npr + npp) * energy_delta(w - wp - wpp, sig_w, n_sigma, delta))
        wt = g * inv_w[mu] * inv_w[:, None] * inv_w[None, :]
        gamma[x] = pref * np.sum(np.where(pair_ok, wt * phi ** 2, 0.0))
    if average and len(modes) == nb:
        gamma = degenerate_average(nu0, gamma, degen_tol_thz)
    return gamma
