"""Pins of the oracle's conductivity part.

* c_mu = hbar omega dn/dT against a numerical temperature derivative, its
  classical and high-T limits (kB);
* c_{mu mu'} -> c_mu as omega' -> omega and c_{mu mu'} = kB classically;
* tau_{mu mu} = 1/(2 gamma_mu);
* kappa_RTA symmetric, isotropic for the cubic crystal, scales as 1/s^2
  with Phi3 -> s Phi3;
* QHGK restricted to degenerate same-q pairs equals kappa_RTA;
* folding: Gamma-only QHGK on an N^3 supercell equals q-resolved QHGK on the
  N^3 mesh; the generalised velocity is antisymmetric and real.
"""

import numpy as np
import pytest

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import conductivity as co
from oracle import phonons as ph
from oracle.units import KB_JK, TWO_PI


def test_heat_capacity_is_hbar_omega_dn_dT():
    omega = np.array([0.3, 2.0, 10.0, 25.0])     # rad/ps
    T = 120.0
    h = 1e-3
    dn = (an.bose(omega, T + h) - an.bose(omega, T - h)) / (2 * h)
    hbar_J = 1.054571817e-34
    np.testing.assert_allclose(co.heat_capacity(omega, T), hbar_J * omega * 1e12 * dn, rtol=1e-7)
    np.testing.assert_allclose(co.heat_capacity(omega, 1e7), KB_JK, rtol=1e-6)
    np.testing.assert_allclose(co.heat_capacity(omega, T, classical=True), KB_JK)


def test_generalized_heat_capacity_limits():
    omega = np.array([3.0, 3.0 * (1 + 1e-7), 9.0])
    T = 300.0
    cc = co.generalized_heat_capacity(omega, T, degen_tol_omega=1e-12)
    c = co.heat_capacity(omega, T)
    np.testing.assert_allclose(cc[0, 1], c[0], rtol=1e-6)
    np.testing.assert_allclose(np.diag(co.generalized_heat_capacity(omega, T, 1e-9)), c)
    # the near-degenerate pair loses ~1e-9 to cancellation in (n'-n)/(w-w')
    np.testing.assert_allclose(co.generalized_heat_capacity(omega, T, 1e-12, classical=True), KB_JK,
                               rtol=1e-8)
    assert np.all(cc > 0)


def test_lorentzian_diagonal_is_rta_lifetime():
    omega = np.array([1.0, 2.0, 2.5])
    gamma = np.array([0.1, 0.02, 0.3])
    np.testing.assert_allclose(np.diag(co.lorentzian_tau(omega, gamma)), 1.0 / (2 * gamma))


@pytest.fixture(scope="module")
def prim4():
    w = ki.small_fcc_prim(mesh=(4, 4, 4), T=50.0, sigma=0.1)
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    g = an.linewidths(s, w.mesh, nu, eig, w.T, w.sigma_thz)
    return w, s, nu, eig, g


def test_kappa_rta_symmetric_isotropic_and_scaling(prim4):
    w, s, nu, eig, g = prim4
    k = co.kappa_rta(s, w.mesh, nu, eig, g, w.T)
    np.testing.assert_allclose(k, k.T, atol=1e-14 * np.abs(k).max())
    np.testing.assert_allclose(k, k[0, 0] * np.eye(3), atol=1e-12 * k[0, 0])
    assert k[0, 0] > 0
    k2 = co.kappa_rta(s, w.mesh, nu, eig, 4.0 * g, w.T)   # gamma -> s^2 gamma, s = 2
    np.testing.assert_allclose(k2, k / 4.0, rtol=1e-12, atol=1e-16)


def test_qhgk_degenerate_pairs_reduce_to_rta(prim4):
    w, s, nu, eig, g = prim4
    k_rta = co.kappa_rta(s, w.mesh, nu, eig, g, w.T)
    k_deg = co.kappa_qhgk_mesh(s, w.mesh, nu, eig, g, w.T, degenerate_pairs_only=True)
    np.testing.assert_allclose(k_deg, k_rta, rtol=1e-10, atol=1e-14)
    k_all = co.kappa_qhgk_mesh(s, w.mesh, nu, eig, g, w.T)
    # the interband (coherence) term is non-negative on the diagonal
    assert np.all(np.diag(k_all) >= np.diag(k_rta) * (1 - 1e-12))


@pytest.mark.parametrize("kind,N", [("prim", 3), ("binary", 2)])
def test_qhgk_supercell_folding_equals_q_resolved(kind, N):
    if kind == "prim":
        lat, pos = ki.fcc_primitive(ki.A_FCC)
        masses = [39.95]
    else:
        lat, pos = ki.l11_binary(ki.A_FCC)
        masses = [28.09, 72.63]
    cell = ki.lj_system(lat, pos, masses)
    sup = ki.supercell_of(lat, pos, masses, N)
    T, sig = 300.0, 0.15
    mesh = (N, N, N)
    nu_m, eig_m = ph.phonons(cell, mesh)
    g_m = an.linewidths(cell, mesh, nu_m, eig_m, T, sig)
    nu_s, eig_s = ph.phonons(sup, (1, 1, 1))
    g_s = an.linewidths_gamma_only(sup, nu_s, eig_s, T, sig)
    W = co.generalized_velocity(sup, nu_s, eig_s)
    np.testing.assert_allclose(W, -np.transpose(W, (0, 2, 1)), atol=1e-12 * np.abs(W).max())
    k_s = co.kappa_qhgk(sup, nu_s, eig_s, g_s, T, W=W)
    k_m = co.kappa_qhgk_mesh(cell, mesh, nu_m, eig_m, g_m, T)
    np.testing.assert_allclose(k_s, k_m, rtol=1e-8, atol=1e-12 * np.abs(k_m).max())
    np.testing.assert_allclose(k_s, k_s.T, atol=1e-12 * np.abs(k_s).max())
