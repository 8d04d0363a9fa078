"""Pins of the oracle's phase space g_mu and mode diffusivity D_mu.

* phase space, exact energy conservation (frequencies on a grid, sigma much
  smaller than the step): every triplet a + b -> c enters sum_mu n(1+n) g_mu
  through a and b in the + part and through c in the - part with equal
  weight n_a n_b (n_c (1 + n_a + n_b) = n_a n_b when w_c = w_a + w_b), so the
  + part is twice the - part once the - part carries its 1/2; T -> 0 removes
  the + part;
* diffusivity: with classical populations the generalised heat capacity is
  kB for every pair, so tr(kappa_QHGK) / 3 = kB / V sum_mu D_mu -- this fixes
  the 1/3 and the absence of a volume factor in D_mu against the pinned
  kappa_QHGK (the two share the velocities and the Lorentzian lifetimes).
"""

import numpy as np

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import conductivity as co
from oracle import phonons as ph
from oracle.units import KB_JK, TWO_PI


def test_phase_space_detailed_balance_and_zero_temperature():
    w = ki.small_binary(mesh=(3, 3, 3))
    s = w.systems[0]
    nu, _ = ph.phonons(s, w.mesh)
    d = 0.05
    nu_q = np.round(nu / d) * d
    T = 150.0
    g, gp, gm = an.phase_space(w.mesh, nu_q, T, sigma_thz=0.004, return_parts=True)
    valid = nu_q > 0.01
    n = an.bose(np.where(valid, TWO_PI * nu_q, 0.0), T)
    plus = np.sum(n * (1 + n) * gp)
    minus = np.sum(n * (1 + n) * gm)
    assert plus > 0 and minus > 0
    np.testing.assert_allclose(plus, 2.0 * minus, rtol=1e-12)
    np.testing.assert_allclose(g, gp + gm)
    _, gp0, gm0 = an.phase_space(w.mesh, nu, 0.05, sigma_thz=0.2, return_parts=True)
    assert np.abs(gp0).max() < 1e-12 * np.abs(gm0).max() and gm0.max() > 0


def test_classical_diffusivity_sums_to_qhgk_trace():
    s = ki.fcc_supercell_system((2, 2, 3), seed=17, heavy_fraction=0.3)
    nu, eig = ph.phonons(s, (1, 1, 1))
    g = an.linewidths_gamma_only(s, nu, eig, 300.0, 0.05, classical=True)
    kappa = co.kappa_qhgk(s, nu, eig, g, 300.0, classical=True)
    D = co.diffusivity(s, nu, eig, g)
    assert np.all(D >= 0) and D.max() > 0
    np.testing.assert_allclose(np.trace(kappa) / 3.0, co.KAPPA_SI * KB_JK / s.volume * D.sum(), rtol=1e-12)
