"""Pins of the oracle's energy delta and of its absolute unit constants.

The other oracle pins (detailed balance, T -> 0, s^2 scaling, folding, the
BTE pins) are all invariant under a constant rescaling of the delta and of
the unit constants, so they cannot see a width taken in the wrong unit or a
wrong conversion factor.  These tests fix both against things outside the
oracle:

* the Gaussian delta against scipy.stats.norm (a library density) and its
  truncated integral erf(n_sigma / sqrt 2);
* the width in THz through the callers: with frequencies chosen so that
  exactly one triplet falls inside the window, the phase space equals
  (n' - n'') times the normal density in angular frequency with standard
  deviation 2 pi sigma, with n from Planck's h and k_B in SI; the linewidth
  of that triplet scales with sigma exactly as that density does;
* the whole linewidth of a small supercell, and kappa_RTA and kappa_QHGK of
  small cells, recomputed from scratch in SI units (J, kg, m, s) with
  scipy.constants, against the oracle's eV / amu / Angstrom / ps chain.

scipy.constants follows CODATA 2022 and the oracle CODATA 2018; the two differ
by about 1e-9 relative (the atomic mass unit), so the SI pins use 1e-7.  Each
pin fails by orders of magnitude on the plausible slips: sigma read in rad/ps
(a factor 2 pi in the width), a delta normalised in THz instead of rad/ps, a
missing 1e-12, a wrong eV/amu/Angstrom conversion.
"""

import numpy as np
import pytest
import scipy.constants as sc
from scipy.special import erf
from scipy.stats import norm

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import conductivity as co
from oracle import phonons as ph

TWO_PI = 2.0 * np.pi
# SI conversions taken from scipy.constants (not from oracle.units)
EV = sc.e                                   # J
AMU = sc.physical_constants["atomic mass constant"][0]      # kg
ANG = sc.angstrom                           # m
THZ = 1e12                                  # Hz


# ---------------------------------------------------------------- the delta itself
@pytest.mark.parametrize("sigma_w,n_sigma", [(0.1 * TWO_PI, 3.0), (0.05 * TWO_PI, 3.0), (0.7, 2.0)])
def test_gaussian_delta_is_the_truncated_normal_density(sigma_w, n_sigma):
    d = np.linspace(-n_sigma * sigma_w * 1.2, n_sigma * sigma_w * 1.2, 240001)
    g = an.gaussian_delta(d, sigma_w, n_sigma)
    inside = np.abs(d) < n_sigma * sigma_w
    np.testing.assert_allclose(g[inside], norm.pdf(d[inside], scale=sigma_w), rtol=1e-13)
    assert np.all(g[~inside] == 0.0)
    # strict cut: zero exactly at the edge
    assert an.gaussian_delta(np.array([n_sigma * sigma_w]), sigma_w, n_sigma)[0] == 0.0
    # the truncated integral over angular frequency (midpoint rule on the window)
    cut = n_sigma * sigma_w
    h = 2.0 * cut / 200000
    mid = -cut + (np.arange(200000) + 0.5) * h
    integral = np.sum(an.gaussian_delta(mid, sigma_w, n_sigma)) * h
    assert abs(integral - erf(n_sigma / np.sqrt(2.0))) < 1e-9
    # one standard deviation away: exp(-1/2) / (sqrt(2 pi) sigma)
    v = an.gaussian_delta(np.array([sigma_w]), sigma_w, n_sigma)[0]
    assert abs(v - np.exp(-0.5) / (np.sqrt(TWO_PI) * sigma_w)) < 1e-14 * v


# ---------------------------------------------------------------- width in THz through the callers
def _bose_si(nu_thz, T, classical=False):
    """Planck occupation from h nu / kB T with h and kB in SI."""
    x = sc.h * np.asarray(nu_thz) * THZ / (sc.k * T)
    return 1.0 / x if classical else 1.0 / np.expm1(x)


def _one_triplet_nu(d_thz, nb):
    """Frequencies (THz) at a single q-point where mode 0 has exactly one
    triplet inside a window of half-width < 0.6 THz (for |d| < 0.1): the +
    process 0 + 1 -> 2 with nu0 + nu1 - nu2 = d; every other combination of
    mode 0 is at least 0.7 THz from energy conservation."""
    base = [1.0, 2.7, 3.7, 7.7, 13.1, 29.0, 47.3, 71.9, 101.7, 150.3, 211.9, 307.1]
    nu = np.array(base[:nb], dtype=float)
    nu[2] -= d_thz
    return nu


def _check_single_triplet(nu, cut_thz):
    n = len(nu)
    hits = []
    for a in range(n):
        for b in range(n):
            if abs(nu[0] + nu[a] - nu[b]) < cut_thz:
                hits.append(("+", a, b))
            if abs(nu[0] - nu[a] - nu[b]) < cut_thz:
                hits.append(("-", a, b))
    assert hits == [("+", 1, 2)], hits


def phase_space_pin_error(sigma_thz, d_thz, T=300.0, classical=False):
    """Relative deviation of the oracle's phase space of mode 0 from
    (n1 - n2) * N(2 pi d; 0, 2 pi sigma) for the single-triplet spectrum."""
    nu = _one_triplet_nu(d_thz, 3)[None, :]
    _check_single_triplet(nu[0], 3.0 * sigma_thz)
    g = an.phase_space((1, 1, 1), nu, T, sigma_thz, 3.0, classical=classical)[0, 0]
    n = _bose_si(nu[0], T, classical)
    want = (n[1] - n[2]) * norm.pdf(TWO_PI * d_thz, scale=TWO_PI * sigma_thz)
    return abs(g - want) / abs(want)


@pytest.mark.parametrize("classical", [False, True])
@pytest.mark.parametrize("sigma_thz,d_frac", [(0.1, 0.0), (0.1, 1.0), (0.05, 1.0), (0.05, 2.5)])
def test_phase_space_delta_width_is_sigma_in_thz(sigma_thz, d_frac, classical):
    assert phase_space_pin_error(sigma_thz, d_frac * sigma_thz, classical=classical) < 1e-9


def test_phase_space_pin_catches_a_width_in_rad_per_ps(monkeypatch):
    """Plant the slip in the oracle (on the CPU): a delta whose width is sigma
    taken as rad/ps instead of THz.  The pin must fail by a wide margin."""
    good = an.gaussian_delta
    monkeypatch.setattr(an, "gaussian_delta", lambda d, s, n: good(d, s / TWO_PI, n))
    assert phase_space_pin_error(0.1, 0.1) > 0.5
    # and a delta normalised as a density in THz instead of rad/ps
    monkeypatch.setattr(an, "gaussian_delta", lambda d, s, n: TWO_PI * good(d, s, n))
    assert phase_space_pin_error(0.1, 0.1) > 0.5


def _gamma_only_cell():
    base = ki.fcc_supercell_system(1, seed=7)          # 4 atoms, 12 modes, cubic
    return ki.random_fc3_system(base, 30, seed=5, scale=0.05)


@pytest.mark.parametrize("d_frac", [0.0, 0.7, 1.9])
def test_linewidth_scales_with_sigma_as_the_density(d_frac):
    """Same single-triplet spectrum inside the linewidth: phi, n and 1/omega
    are unchanged between two widths, so gamma(sigma1)/gamma(sigma2) must be
    N(2 pi d; 2 pi sigma1) / N(2 pi d; 2 pi sigma2) exactly (d in THz)."""
    s = _gamma_only_cell()
    _, eig = ph.phonons(s, (1, 1, 1))
    s1, s2 = 0.06, 0.1
    d = d_frac * s1
    nu = _one_triplet_nu(d, 12)[None, :]
    _check_single_triplet(nu[0], 3.0 * s2)
    g1 = an.linewidths_gamma_only(s, nu, eig, 300.0, s1, modes=[0], average=False)[0]
    g2 = an.linewidths_gamma_only(s, nu, eig, 300.0, s2, modes=[0], average=False)[0]
    want = norm.pdf(TWO_PI * d, scale=TWO_PI * s1) / norm.pdf(TWO_PI * d, scale=TWO_PI * s2)
    assert g1 > 0 and g2 > 0
    assert abs(g1 / g2 - want) < 1e-12 * want
    # the crystal route at mesh 1x1x1 applies the same delta
    c1 = an.linewidths(s, (1, 1, 1), nu, eig, 300.0, s1, average=False)[0, 0]
    assert abs(c1 - g1) < 1e-12 * g1


# ---------------------------------------------------------------- SI recomputations
def _dense_fc3_si(sys):
    """Phi3 over the supercell dofs in J/m^3 (Gamma-only: images folded)."""
    nb = 3 * sys.n_atoms
    F = np.zeros((nb, nb, nb))
    for key, blk in zip(sys.fc3_idx, sys.fc3):
        i, j, k = key[0], key[1], key[5]
        F[3 * i:3 * i + 3, 3 * j:3 * j + 3, 3 * k:3 * k + 3] += blk
    return F * EV / ANG ** 3


def _dense_fc2_si(sys, q_si=None, deriv=False):
    """D(q) in s^-2 (and optionally dD/dq_a in m/s^2), blocks summed with
    exp(-i q.R), R in metres, q in 1/m."""
    nb = 3 * sys.n_atoms
    m = sys.masses * AMU
    D = np.zeros((nb, nb), complex)
    dD = np.zeros((3, nb, nb), complex)
    q = np.zeros(3) if q_si is None else q_si
    for key, blk in zip(sys.fc2_idx, sys.fc2):
        i, j = key[0], key[1]
        R = (key[2:5].astype(float) @ sys.lattice) * ANG
        b = blk * EV / ANG ** 2 / np.sqrt(m[i] * m[j])
        ph_ = np.exp(-1j * q @ R)
        D[3 * i:3 * i + 3, 3 * j:3 * j + 3] += b * ph_
        if deriv:
            for a in range(3):
                dD[a, 3 * i:3 * i + 3, 3 * j:3 * j + 3] += -1j * R[a] * b * ph_
    return (D, dD) if deriv else D


def test_gamma_only_linewidth_recomputed_in_si():
    """Every linewidth of a 12-mode supercell at 300 K (both processes, all
    triplets inside the 3-sigma window) from SI quantities:
    Gamma = (hbar pi / 8) |phi|^2 / (w w' w'') [(n'-n'') d(w+w'-w'') + 1/2 (1+n'+n'') d(w-w'-w'')],
    phi in J m^-3 kg^-3/2, w in rad/s, the Gaussian in seconds."""
    s = _gamma_only_cell()
    nu, eig = ph.phonons(s, (1, 1, 1))
    T, sig = 300.0, 0.3
    g_or = an.linewidths_gamma_only(s, nu, eig, T, sig, average=False)
    nb = nu.shape[1]
    m = np.repeat(s.masses * AMU, 3)
    E = eig[0].real / np.sqrt(m)[None, :]                     # rows = modes, kg^-1/2
    F = _dense_fc3_si(s)
    phi = np.einsum("abc,sa,tb,uc->stu", F, E, E, E)
    w = TWO_PI * nu[0] * THZ                                  # rad/s
    valid = nu[0] > 0.01
    n = np.where(valid, _bose_si(np.where(valid, nu[0], 1.0), T), 0.0)
    sw = TWO_PI * sig * THZ
    cut = 3.0 * sw
    for mu in range(nb):
        if not valid[mu]:
            assert g_or[mu] == 0.0
            continue
        tot = 0.0
        for a in range(nb):
            for b in range(nb):
                if not (valid[a] and valid[b]):
                    continue
                dp, dm = w[mu] + w[a] - w[b], w[mu] - w[a] - w[b]
                gp = (n[a] - n[b]) * norm.pdf(dp, scale=sw) if abs(dp) < cut else 0.0
                gm = 0.5 * (1 + n[a] + n[b]) * norm.pdf(dm, scale=sw) if abs(dm) < cut else 0.0
                tot += phi[mu, a, b] ** 2 / (w[mu] * w[a] * w[b]) * (gp + gm)
        gamma_si = sc.hbar * np.pi / 8.0 * tot                # 1/s
        assert abs(gamma_si * 1e-12 - g_or[mu]) <= 1e-7 * abs(g_or[mu]) + 1e-30, mu


def test_kappa_rta_recomputed_in_si():
    """kappa_ab = 1/(N_k V) sum c tau (trace form of the velocity matrices)
    with c = kB x^2 e^x/(e^x-1)^2, V in m^3, v in m/s, tau = 1/(2 gamma) in s."""
    w = ki.small_binary(mesh=(3, 3, 3), sigma=0.2)      # (2x2x2 has v = 0 at every q)
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    gam = 0.05 + 0.01 * np.round(nu, 3)                     # ps^-1, equal inside degenerate sets
    kap_or = co.kappa_rta(s, w.mesh, nu, eig, gam, w.T)
    qs = ki.mesh_qpoints(s.lattice, w.mesh) / ANG             # 1/m
    V = abs(np.linalg.det(s.lattice)) * ANG ** 3
    kap = np.zeros((3, 3))
    for k in range(len(qs)):
        _, dD = _dense_fc2_si(s, qs[k], deriv=True)
        Ek = eig[k].T                                        # columns = modes
        wk = TWO_PI * nu[k] * THZ
        for D_set in ph.degenerate_sets(nu[k], 1e-5):
            D_set = [x for x in D_set if nu[k][x] > 0.01]
            if not D_set:
                continue
            sub = np.stack([Ek[:, D_set].conj().T @ dD[a] @ Ek[:, D_set] for a in range(3)])
            sub = sub / (2.0 * np.sqrt(np.outer(wk[D_set], wk[D_set])))[None]     # m/s
            x = sc.hbar * wk[D_set] / (sc.k * w.T)
            c = sc.k * x * x * np.exp(x) / np.expm1(x) ** 2
            tau = 1.0 / (2.0 * gam[k][D_set] * 1e12)
            vv = np.real(np.einsum("ast,bst->ab", sub, sub.conj()))
            kap += np.mean(c * tau) * vv
    kap /= len(qs) * V
    assert np.abs(kap).max() > 0.1
    np.testing.assert_allclose(kap_or, kap, rtol=1e-7, atol=1e-7 * np.abs(kap).max())


def test_kappa_qhgk_recomputed_in_si():
    """kappa_ab = 1/V sum c_mm' tau_mm' W^a W^b with A_a in m/s^2,
    W = E^T A E / (2 sqrt(w w')) in m/s, c_mm' = hbar w w'/T (n'-n)/(w-w') in J/K
    and tau_mm' = (g+g')/((w-w')^2 + (g+g')^2) in s."""
    lat, pos = ki.l11_binary(ki.A_FCC)
    s = ki.supercell_of(lat, pos, [28.09, 72.63], 2)          # 16 atoms, 48 modes
    nu, eig = ph.phonons(s, (1, 1, 1))
    T = 300.0
    nb = nu.shape[1]
    gam = 0.02 + 0.004 * np.arange(nb) / nb                   # ps^-1
    kap_or = co.kappa_qhgk(s, nu, eig, gam, T, degen_tol_thz=1e-5)
    m = s.masses * AMU
    A = np.zeros((3, nb, nb))
    for key, blk in zip(s.fc2_idx, s.fc2):
        i, j = key[0], key[1]
        L = key[2:5].astype(float) @ s.lattice
        d = (s.positions[i] - s.positions[j] - L) * ANG
        b = blk * EV / ANG ** 2 / np.sqrt(m[i] * m[j])
        for a in range(3):
            A[a, 3 * i:3 * i + 3, 3 * j:3 * j + 3] += d[a] * b
    E = eig[0].real.T
    valid = nu[0] > 0.01
    wv = TWO_PI * nu[0] * THZ
    ws = np.where(valid, wv, 1.0)
    W = np.stack([E.T @ A[a] @ E for a in range(3)]) / (2.0 * np.sqrt(np.outer(ws, ws)))[None]
    n = np.where(valid, _bose_si(np.where(valid, nu[0], 1.0), T), 0.0)
    x = sc.hbar * ws / (sc.k * T)
    c = np.where(valid, sc.k * x * x * np.exp(x) / np.expm1(x) ** 2, 0.0)
    g = gam * 1e12
    kap = np.zeros((3, 3))
    for mu in range(nb):
        for nu_ in range(nb):
            if not (valid[mu] and valid[nu_]):
                continue
            dw = wv[mu] - wv[nu_]
            if abs(nu[0][mu] - nu[0][nu_]) < 1e-5:
                cc = 0.5 * (c[mu] + c[nu_])
            else:
                cc = sc.hbar * wv[mu] * wv[nu_] / T * (n[nu_] - n[mu]) / dw
            gs = g[mu] + g[nu_]
            tau = gs / (dw * dw + gs * gs)
            kap += cc * tau * np.outer(W[:, mu, nu_], W[:, mu, nu_])
    kap /= abs(np.linalg.det(s.lattice)) * ANG ** 3
    assert np.abs(kap).max() > 0
    np.testing.assert_allclose(kap_or, kap, rtol=1e-7, atol=1e-7 * np.abs(kap).max())


# ---------------------------------------------------------------- the other delta shapes
@pytest.mark.parametrize("sigma_w,n_sigma", [(0.1 * TWO_PI, 3.0), (0.7, 2.0)])
def test_lorentzian_delta_is_the_truncated_cauchy_density(sigma_w, n_sigma):
    from scipy.stats import cauchy
    cut = n_sigma * sigma_w
    d = np.linspace(-1.2 * cut, 1.2 * cut, 100001)
    g = an.lorentzian_delta(d, sigma_w, n_sigma)
    inside = np.abs(d) < cut
    np.testing.assert_allclose(g[inside], cauchy.pdf(d[inside], scale=sigma_w), rtol=1e-13)
    assert np.all(g[~inside] == 0.0)
    h = 2.0 * cut / 200000
    mid = -cut + (np.arange(200000) + 0.5) * h
    integral = np.sum(an.lorentzian_delta(mid, sigma_w, n_sigma)) * h
    assert abs(integral - 2.0 / np.pi * np.arctan(n_sigma)) < 1e-9
    # half maximum at one half width
    assert abs(an.lorentzian_delta(np.array([sigma_w]), sigma_w, n_sigma)[0] * 2.0
               - an.lorentzian_delta(np.array([0.0]), sigma_w, n_sigma)[0]) < 1e-14 / sigma_w


@pytest.mark.parametrize("sigma_w", [0.1 * TWO_PI, 0.7])
def test_triangular_delta_is_the_symmetric_triangle_density(sigma_w):
    from scipy.stats import triang
    d = np.linspace(-2.0 * sigma_w, 2.0 * sigma_w, 100001)
    g = an.triangular_delta(d, sigma_w, 3.0)
    np.testing.assert_allclose(g, triang.pdf(d, 0.5, loc=-sigma_w, scale=2.0 * sigma_w), rtol=1e-12,
                               atol=1e-14 / sigma_w)
    h = 2.0 * sigma_w / 200000
    mid = -sigma_w + (np.arange(200000) + 0.5) * h
    assert abs(np.sum(an.triangular_delta(mid, sigma_w, 3.0)) * h - 1.0) < 1e-9


@pytest.mark.parametrize("shape", ["lorentzian", "triangular"])
@pytest.mark.parametrize("d_frac", [0.0, 0.4, 0.9])
def test_phase_space_uses_the_chosen_shape_in_thz(shape, d_frac):
    """Single-triplet spectrum: the phase space of mode 0 equals (n1 - n2)
    times the library density of the chosen shape at 2 pi d, width 2 pi sigma."""
    from scipy.stats import cauchy, triang
    sigma = 0.1
    d = d_frac * sigma
    nu = _one_triplet_nu(d, 3)[None, :]
    _check_single_triplet(nu[0], 3.0 * sigma)
    g = an.phase_space((1, 1, 1), nu, 300.0, sigma, 3.0, delta=shape)[0, 0]
    n = _bose_si(nu[0], 300.0)
    sw = TWO_PI * sigma
    dens = cauchy.pdf(TWO_PI * d, scale=sw) if shape == "lorentzian" else \
        triang.pdf(TWO_PI * d, 0.5, loc=-sw, scale=2 * sw)
    assert abs(g - (n[1] - n[2]) * dens) <= 1e-9 * abs((n[1] - n[2]) * dens)


@pytest.mark.parametrize("shape", ["lorentzian", "triangular"])
def test_linewidth_shape_ratio_matches_the_densities(shape):
    """With one triplet in the window, gamma with a given shape over gamma with
    the Gaussian is the ratio of the two densities at the mismatch."""
    from scipy.stats import cauchy, triang
    s = _gamma_only_cell()
    _, eig = ph.phonons(s, (1, 1, 1))
    sigma, d = 0.1, 0.03
    nu = _one_triplet_nu(d, 12)[None, :]
    _check_single_triplet(nu[0], 3.0 * sigma)
    g_s = an.linewidths_gamma_only(s, nu, eig, 300.0, sigma, modes=[0], average=False, delta=shape)[0]
    g_g = an.linewidths_gamma_only(s, nu, eig, 300.0, sigma, modes=[0], average=False)[0]
    sw = TWO_PI * sigma
    dens = cauchy.pdf(TWO_PI * d, scale=sw) if shape == "lorentzian" else \
        triang.pdf(TWO_PI * d, 0.5, loc=-sw, scale=2 * sw)
    want = dens / norm.pdf(TWO_PI * d, scale=sw)
    assert abs(g_s / g_g - want) < 1e-12 * want
    c = an.linewidths(s, (1, 1, 1), nu, eig, 300.0, sigma, average=False, delta=shape)[0, 0]
    assert abs(c - g_s) < 1e-12 * g_s
