"""Thermal conductivity of the oracle: BTE-RTA for crystals and QHGK.

Plain FP64 NumPy.  TEST INFRASTRUCTURE ONLY: the library never imports this
module.

BTE-RTA (paper Eq. RTA, Eq. heat_capacity):
  kappa_ab = 1/(N_k V) sum_mu c_mu v_mu,a v_mu,b tau_mu,  tau = 1/(2 gamma),
  c_mu = hbar omega dn/dT = kB x^2 e^x / (e^x - 1)^2,  x = hbar omega / kB T
  (classical limit c = kB, section "Classical limit").
  Reading for degenerate modes (paper silent): inside each degenerate set D
  at one q, v_a v_b is replaced by the basis-invariant trace
  sum_{s,s' in D} Re(V^a_{ss'} conj(V^b_{ss'})), which equals v_a v_b
  outside degeneracies.

QHGK (paper Eq. conductivity_amorphous, twod_heat_capacity,
generalized_velocity, lorentzian_amorphous):
  kappa_ab = 1/V sum_{mu mu'} c_{mu mu'} Re(v^a_{mu mu'} conj(v^b_{mu mu'})) tau_{mu mu'}
  c_{mu mu'} = (hbar omega omega' / T) (n' - n) / (omega - omega')   [reading:
      the printed order of n - n' gives -c_mu in the limit omega' -> omega;
      the limit c_mu is used for |d nu| < degen_tol]
  tau_{mu mu'} = (gamma + gamma') / ((omega - omega')^2 + (gamma + gamma')^2)
  v^a_{mu mu'} = i (E^T A_a E)_{mu mu'} / (2 sqrt(omega omega'))   [reading of
      the garbled print: A_a(i, j) = sum_L (x_i - x_j - L)_a D(i, jL), the
      real antisymmetric position-weighted dynamical matrix with true image
      distances; i A_a is Hermitian]
Full BTE (paper Eq. inversemeanfreepath, full_conductivity,
mfp_from_scattering_inv, self-consistent, conductivity_from_lambda):
  kappa_ab = 1/(N_k V) sum_mu c_mu v_mu,a lambda_mu,b with lambda solving
  2 (Gamma^0 + Gamma^1) lambda = v [reading: the printed v = Gamma~ lambda with
  the factor 2 of tau = 1/(2 Gamma^0), so that Gamma^1 = 0 gives Eq. RTA],
  by direct solution or by the series / self-consistent recursion.
Units: kappa in W/(m K); V in A^3; v in A/ps; tau in ps; c in J/K.
"""

from __future__ import annotations

import numpy as np

from kald_inputs.lattice import mesh_qpoints
from .anharmonic import bose
from .phonons import degenerate_sets, velocity_matrices
from .units import EV_A2_AMU, HBAR_EVPS, KB_EVK, KB_JK, TWO_PI

#: (J/K) (A/ps)^2 ps / A^3  ->  W / (m K)
KAPPA_SI = 1e4 * 1e-12 / 1e-30


def heat_capacity(omega, T, classical=False):
    """c_mu in J/K for omega in rad/ps (0 where omega <= 0)."""
    omega = np.asarray(omega, dtype=float)
    out = np.zeros_like(omega)
    good = omega > 0
    if classical:
        out[good] = KB_JK
        return out
    x = HBAR_EVPS * omega[good] / (KB_EVK * T)
    ex = np.exp(-x)
    out[good] = KB_JK * x * x * ex / (1.0 - ex) ** 2
    return out


def kappa_rta(sys, mesh, nu, eig, gamma, T, omega_min_thz=0.01, degen_tol_thz=1e-5,
              classical=False):
    """3x3 kappa (W/(m K)) from Eq. RTA with the degenerate trace form."""
    qs = mesh_qpoints(sys.lattice, mesh)
    nq = qs.shape[0]
    kappa = np.zeros((3, 3))
    for k in range(nq):
        V = velocity_matrices(sys, qs[k], eig[k], nu[k])
        omega = TWO_PI * nu[k]
        valid = nu[k] > omega_min_thz
        c = heat_capacity(np.where(valid, omega, 0.0), T, classical)
        for D in degenerate_sets(nu[k], degen_tol_thz):
            D = [s for s in D if valid[s] and gamma[k, s] > 0]
            if not D:
                continue
            sub = V[:, D][:, :, D]                                   # [3, d, d]
            vv = np.real(np.einsum("ast,bst->ab", sub, sub.conj()))  # trace form
            # c and tau are equal inside a set (gamma already averaged)
            ct = np.mean(c[D] / (2.0 * gamma[k, D]))
            kappa += ct * vv
    return kappa * KAPPA_SI / (nq * sys.volume)


def position_weighted_dynmat(sys):
    """A_a [3, nb, nb] (eV/(A amu)): A_a(i,j) = sum_L (x_i - x_j - L)_a
    Phi2(i, jL) / sqrt(m_i m_j), with L the image each block is seen through."""
    nb = 3 * sys.n_atoms
    m = sys.masses
    i = sys.fc2_idx[:, 0]
    j = sys.fc2_idx[:, 1]
    L = sys.fc2_idx[:, 2:5].astype(float) @ sys.lattice
    d = sys.positions[i] - sys.positions[j] - L                        # [B, 3]
    blk = sys.fc2 / np.sqrt(m[i] * m[j])[:, None, None]
    rows = (3 * i[:, None, None] + np.arange(3)[None, :, None]) * nb
    cols = 3 * j[:, None, None] + np.arange(3)[None, None, :]
    flat = (rows + cols).reshape(-1)
    A = np.zeros((3, nb * nb))
    for a in range(3):
        np.add.at(A[a], flat, (d[:, a, None, None] * blk).reshape(-1))
    A = A.reshape(3, nb, nb)
    return A


def generalized_velocity(sys, nu, eig, omega_min_thz=0.01):
    """W_a [3, nb, nb] (A/ps), the imaginary part of v^a_{mu mu'}:
    v^a = i W_a with W_a = (E^T A_a E) / (2 sqrt(omega omega'))
    (Eq. generalized_velocity, reading above).  Masked modes give zero rows."""
    E = eig[0].real.T                                   # columns = modes
    omega = TWO_PI * nu[0]
    valid = nu[0] > omega_min_thz
    w = np.where(valid, omega, 1.0)
    A = position_weighted_dynmat(sys)
    W = np.stack([E.T @ A[a] @ E for a in range(3)]) * EV_A2_AMU
    W = W / (2.0 * np.sqrt(np.outer(w, w)))[None]
    W[:, ~valid, :] = 0.0
    W[:, :, ~valid] = 0.0
    return W


def generalized_heat_capacity(omega, T, degen_tol_omega, classical=False):
    """c_{mu mu'} [nb, nb] (J/K) for valid omega (rad/ps) (reading above)."""
    n = bose(omega, T, classical)
    c = heat_capacity(omega, T, classical)
    w1, w2 = omega[:, None], omega[None, :]
    dw = w1 - w2
    close = np.abs(dw) < degen_tol_omega
    safe = np.where(close, 1.0, dw)
    hbar_J = HBAR_EVPS * 1.602176634e-19 * 1e-12       # J s
    # (hbar omega omega' / T) (n' - n)/(omega - omega'); omega in rad/ps -> 1e12
    cc = hbar_J * (w1 * 1e12) * (w2 * 1e12) / T * (n[None, :] - n[:, None]) / (safe * 1e12)
    cmid = 0.5 * (c[:, None] + c[None, :])
    return np.where(close, cmid, cc)


def lorentzian_tau(omega, gamma, bandwidth_w=None, threshold_w=None):
    """tau_{mu mu'} [nb, nb] in ps (Eq. lorentzian_amorphous).

    Options of the QHGK engine (code-details appendix), readings:
      bandwidth_w  a fixed width (rad/ps) in place of gamma + gamma' for every
                   pair -- the Allen-Feldman model the appendix names;
      threshold_w  tau = 0 for pairs with |omega - omega'| > threshold (the
                   printed '<' would discard the near-degenerate pairs that
                   carry the diffusive transport, so it is read reversed)."""
    gs = gamma[:, None] + gamma[None, :]
    if bandwidth_w is not None:
        gs = np.full_like(gs, float(bandwidth_w))
    dw = omega[:, None] - omega[None, :]
    den = dw * dw + gs * gs
    tau = np.where(den > 0, gs / np.where(den > 0, den, 1.0), 0.0)
    if threshold_w is not None:
        tau = np.where(np.abs(dw) > threshold_w, 0.0, tau)
    return tau


def kappa_qhgk(sys, nu, eig, gamma, T, omega_min_thz=0.01, degen_tol_thz=1e-5,
               classical=False, W=None, bandwidth_thz=None, threshold_thz=None):
    """3x3 kappa (W/(m K)) of a Gamma-only system (Eq. conductivity_amorphous).
    With bandwidth_thz the linewidths are not used (every mode with
    nu > omega_min takes part) and gamma + gamma' becomes 2 pi bandwidth;
    threshold_thz drops the pairs with |d nu| > threshold (lorentzian_tau)."""
    omega = TWO_PI * nu[0]
    if bandwidth_thz is None:
        valid = (nu[0] > omega_min_thz) & (gamma > 0)
    else:
        valid = nu[0] > omega_min_thz
    if W is None:
        W = generalized_velocity(sys, nu, eig, omega_min_thz)
    cc = generalized_heat_capacity(np.where(valid, omega, 1.0), T, TWO_PI * degen_tol_thz, classical)
    tau = lorentzian_tau(omega, np.where(valid, gamma, 0.0),
                         None if bandwidth_thz is None else TWO_PI * bandwidth_thz,
                         None if threshold_thz is None else TWO_PI * threshold_thz)
    pair = valid[:, None] & valid[None, :]
    wgt = np.where(pair, cc * tau, 0.0)
    kappa = np.einsum("mn,amn,bmn->ab", wgt, W, W)
    return kappa * KAPPA_SI / sys.volume


def interpolate_gamma(nu_src, gamma_src, nu_dst, omega_min_thz=0.01, degen_tol_thz=1e-5):
    """Linewidths of a large system from those of a smaller one, as a function
    of frequency (the QHGK section's interpolation of lifetimes with
    third-order splines, read as a cubic spline of gamma(nu)):
      * source modes with nu <= omega_min or gamma <= 0 are left out, and
        frequencies closer than degen_tol are merged (their gamma averaged) so
        that the abscissae increase strictly;
      * the spline is scipy's CubicSpline with not-a-knot ends;
      * destination modes with nu <= omega_min get 0; outside the source
        range gamma is held at the nearest end value (no extrapolation, so it
        cannot turn negative).
    Returns gamma_dst (same shape as nu_dst)."""
    from scipy.interpolate import CubicSpline
    nu_src = np.asarray(nu_src, float).reshape(-1)
    g_src = np.asarray(gamma_src, float).reshape(-1)
    keep = (nu_src > omega_min_thz) & (g_src > 0)
    x = nu_src[keep]
    y = g_src[keep]
    o = np.argsort(x, kind="stable")
    x, y = x[o], y[o]
    xs, ys = [], []
    i = 0
    while i < len(x):
        j = i + 1
        while j < len(x) and x[j] - x[j - 1] < degen_tol_thz:
            j += 1
        xs.append(np.mean(x[i:j]))
        ys.append(np.mean(y[i:j]))
        i = j
    xs, ys = np.array(xs), np.array(ys)
    nu_dst = np.asarray(nu_dst, float)
    out = np.zeros_like(nu_dst)
    live = nu_dst > omega_min_thz
    xq = np.clip(nu_dst[live], xs[0], xs[-1])
    out[live] = CubicSpline(xs, ys, bc_type="not-a-knot")(xq)
    return out


def diffusivity(sys, nu, eig, gamma, omega_min_thz=0.01, W=None, bandwidth_thz=None, threshold_thz=None):
    """Mode diffusivity D_mu [nb] (A^2/ps) of a Gamma-only system, Eq.
    diffusivity_per_mode read as D_mu = (1/3) sum_a sum_mu' |v^a_{mu mu'}|^2 tau_{mu mu'}
    (the Allen-Feldman diffusivity averaged over the three directions; the
    printed 1/(N_k V) prefactor would not give a diffusivity and is dropped).
    With classical populations c_{mu mu'} = kB, so that tr(kappa_QHGK) / 3 =
    kB / V sum_mu D_mu."""
    omega = TWO_PI * nu[0]
    if bandwidth_thz is None:
        valid = (nu[0] > omega_min_thz) & (gamma > 0)
    else:
        valid = nu[0] > omega_min_thz
    if W is None:
        W = generalized_velocity(sys, nu, eig, omega_min_thz)
    tau = lorentzian_tau(omega, np.where(valid, gamma, 0.0),
                         None if bandwidth_thz is None else TWO_PI * bandwidth_thz,
                         None if threshold_thz is None else TWO_PI * threshold_thz)
    pair = valid[:, None] & valid[None, :]
    D = np.einsum("amn,mn->m", W * W, np.where(pair, tau, 0.0)) / 3.0
    return np.where(valid, D, 0.0)


def kappa_qhgk_mesh(sys, mesh, nu, eig, gamma, T, omega_min_thz=0.01, degen_tol_thz=1e-5,
                    classical=False, degenerate_pairs_only=False):
    """q-resolved QHGK on a mesh (same-q interband pairs), with velocities in
    the atom-position phase gauge; equals kappa_qhgk of the folded supercell.
    degenerate_pairs_only keeps the pairs with |d nu| < degen_tol (the part
    that reduces to BTE-RTA)."""
    qs = mesh_qpoints(sys.lattice, mesh)
    nq = qs.shape[0]
    kappa = np.zeros((3, 3))
    for k in range(nq):
        valid = (nu[k] > omega_min_thz) & (gamma[k] > 0)
        # eigenvectors in the atom-phase gauge: eta~ = P eta, P = diag(exp(i q.x))
        ph = np.exp(1j * (np.repeat(sys.positions, 3, axis=0) @ qs[k]))
        eig_t = eig[k] * ph[None, :]
        V = velocity_matrices(sys, qs[k], eig_t, nu[k], atom_phase=True)
        omega = TWO_PI * nu[k]
        cc = generalized_heat_capacity(np.where(valid, omega, 1.0), T, TWO_PI * degen_tol_thz, classical)
        tau = lorentzian_tau(omega, np.where(valid, gamma[k], 0.0))
        pair = valid[:, None] & valid[None, :]
        if degenerate_pairs_only:
            pair &= np.abs(nu[k][:, None] - nu[k][None, :]) < degen_tol_thz
        wgt = np.where(pair, cc * tau, 0.0)
        kappa += np.real(np.einsum("mn,amn,bmn->ab", wgt, V, V.conj()))
    return kappa * KAPPA_SI / (nq * sys.volume)


# ---------------------------------------------------------------- full BTE
def group_velocities(sys, mesh, nu, eig):
    """Diagonal group velocities v[N, 3] (A/ps), v_mu,a = Re V^a_{mu mu} in the
    basis of `eig` (flat mode index mu = q nb + s)."""
    qs = mesh_qpoints(sys.lattice, mesh)
    nq, nb = nu.shape
    v = np.zeros((nq * nb, 3))
    for k in range(nq):
        V = velocity_matrices(sys, qs[k], eig[k], nu[k])
        v[k * nb:(k + 1) * nb] = np.real(np.einsum("ass->sa", V))
    return v


def _bte_kappa(sys, nq, c, v, lam):
    """Eq. conductivity_from_lambda: kappa_ab = 1/(N_k V) sum_mu c_mu v_mu,a lambda_mu,b."""
    return np.einsum("m,ma,mb->ab", c, v, lam) * KAPPA_SI / (nq * sys.volume)


def kappa_bte_direct(sys, mesh, nu, eig, gamma0, G1, T, omega_min_thz=0.01, classical=False):
    """kappa (W/(m K)) from the inverted scattering operator, Eq.
    inversemeanfreepath and full_conductivity: lambda_b = (2 Gamma~)^-1 v_b on
    the valid modes.  Reading: the printed v = Gamma~ lambda is taken with the
    factor 2 of tau = 1/(2 Gamma^0), so that Gamma^1 = 0 gives Eq. RTA.  The
    velocities are the diagonal ones of `group_velocities`; inside a degenerate
    set the result depends on the eigenvector basis, as the rates do."""
    nq = nu.shape[0]
    flat = nu.reshape(-1)
    valid = (flat > omega_min_thz) & (gamma0 > 0)
    c = heat_capacity(np.where(valid, TWO_PI * flat, 0.0), T, classical)
    v = group_velocities(sys, mesh, nu, eig)
    idx = np.flatnonzero(valid)
    A = 2.0 * (np.diag(gamma0[idx]) + G1[np.ix_(idx, idx)])
    lam = np.zeros_like(v)
    lam[idx] = np.linalg.solve(A, v[idx])
    return _bte_kappa(sys, nq, c, v, lam)


def kappa_bte_self_consistent(sys, mesh, nu, eig, gamma0, G1, T, omega_min_thz=0.01,
                              classical=False, tol=1e-12, max_iter=500):
    """kappa from the series of Eq. mfp_from_scattering_inv summed term by term
    with the recursion of Eq. self-consistent (same reading of the factor 2):
      lambda^0 = v / (2 Gamma^0),  lambda^{n+1} = -(1/Gamma^0) Gamma^1 lambda^n,
      lambda = sum_n lambda^n.
    Returns (kappa, n_terms, converged); the series converges only when the
    spectral radius of Gamma^1 / Gamma^0 is below 1."""
    nq = nu.shape[0]
    flat = nu.reshape(-1)
    valid = (flat > omega_min_thz) & (gamma0 > 0)
    c = heat_capacity(np.where(valid, TWO_PI * flat, 0.0), T, classical)
    v = group_velocities(sys, mesh, nu, eig)
    idx = np.flatnonzero(valid)
    g0 = gamma0[idx]
    B = G1[np.ix_(idx, idx)] / g0[:, None]
    term = v[idx] / (2.0 * g0[:, None])
    total = term.copy()
    converged = False
    n_terms = 1
    for _ in range(max_iter):
        term = -(B @ term)
        total += term
        n_terms += 1
        if np.abs(term).max() <= tol * np.abs(total).max():
            converged = True
            break
    lam = np.zeros_like(v)
    lam[idx] = total
    return _bte_kappa(sys, nq, c, v, lam), n_terms, converged
