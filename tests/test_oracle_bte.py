"""Pins of the oracle's full linearised BTE (scattering operator and solvers).

* the diagonal Gamma^0 of the operator equals the (pinned) unaveraged
  linewidths, computed by a different loop;
* exact energy conservation (frequencies on a grid, sigma much smaller than
  the grid step): a uniform lambda, i.e. psi_mu proportional to omega_mu (a
  shift of temperature), is annihilated by Gamma~ -- every triplet contributes
  (omega +- omega' - omega'') / omega = 0 -- which fixes the signs and weights
  of the four Gamma^1 terms against Gamma^0;
* detailed balance under the same condition: n_mu (n_mu + 1) omega_mu
  Gamma~_{mu mu'} / omega_mu' is symmetric and positive semidefinite (the
  linearised collision operator in the psi variables);
* Gamma^1 = 0 reproduces the RTA conductivity of the separate kappa_rta
  (on a cell without degenerate modes, where the trace form is v v);
* the self-consistent series equals the direct inversion, and a divergent
  series is reported as such.
"""

import numpy as np
import pytest

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import conductivity as co
from oracle import phonons as ph
from oracle.units import TWO_PI


def _grid_operator():
    """small binary cell, 3^3 mesh, frequencies rounded to a 0.05 THz grid and
    sigma = 0.004 THz: only exactly energy-conserving triplets survive."""
    w = ki.small_binary(mesh=(3, 3, 3))
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    d = 0.05
    nu_q = np.round(nu / d) * d
    T = 150.0
    g0, G1 = an.scattering_matrix(s, w.mesh, nu_q, eig, T, sigma_thz=0.004, n_sigma=3.0)
    valid = nu_q.reshape(-1) > 0.01
    return nu_q, T, g0, G1, valid


@pytest.fixture(scope="module")
def four_mass_cell():
    """The conventional fcc cell with four different masses (point group D2h,
    abelian: no symmetry-forced degeneracies), 3^3 mesh, 300 K."""
    lat, pos = ki.fcc_conventional(ki.configs.A_FCC, 1)
    s = ki.lj_system(lat, pos, [28.09, 40.0, 55.0, 72.63])
    mesh = (3, 3, 3)
    nu, eig = ph.phonons(s, mesh)
    g0, G1 = an.scattering_matrix(s, mesh, nu, eig, 300.0, 0.2)
    return s, mesh, nu, eig, g0, G1


def test_diagonal_equals_unaveraged_linewidths():
    w = ki.small_binary(mesh=(3, 3, 3))
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    g0, G1 = an.scattering_matrix(s, w.mesh, nu, eig, 300.0, 0.2)
    g = an.linewidths(s, w.mesh, nu, eig, 300.0, 0.2, average=False)
    np.testing.assert_allclose(g0, g.reshape(-1), rtol=1e-12, atol=1e-14 * g.max())
    assert np.abs(G1).max() > 0.1 * g0.max()       # the off-diagonal part is not small


def test_uniform_lambda_is_annihilated_under_exact_energy_conservation():
    nu_q, T, g0, G1, valid = _grid_operator()
    Gt = np.diag(g0) + G1
    rows = np.abs(Gt).sum(axis=1)
    assert np.all(rows[valid] > 0)
    np.testing.assert_array_less(np.abs(Gt.sum(axis=1))[valid], 1e-12 * rows[valid])


def test_detailed_balance_symmetric_positive_semidefinite():
    nu_q, T, g0, G1, valid = _grid_operator()
    om = TWO_PI * nu_q.reshape(-1)
    n = an.bose(np.where(valid, om, 0.0), T)
    Gt = (np.diag(g0) + G1)[np.ix_(valid, valid)]
    w = om[valid]
    C = (n[valid] * (n[valid] + 1.0) * w)[:, None] * Gt / w[None, :]
    scale = np.abs(C).max()
    np.testing.assert_allclose(C, C.T, rtol=0, atol=1e-12 * scale)
    ev = np.linalg.eigvalsh(0.5 * (C + C.T))
    assert ev.min() > -1e-12 * ev.max()


def test_no_off_diagonal_part_reduces_to_rta(four_mass_cell):
    s, mesh, nu, eig, g0, G1 = four_mass_cell
    for k in range(nu.shape[0]):
        for D in ph.degenerate_sets(nu[k], 1e-5):
            assert len(D) == 1 or nu[k][D[0]] <= 0.01        # only the masked acoustic zeros
    k_bte = co.kappa_bte_direct(s, mesh, nu, eig, g0, np.zeros_like(G1), 300.0)
    k_rta = co.kappa_rta(s, mesh, nu, eig, g0.reshape(nu.shape), 300.0)
    np.testing.assert_allclose(k_bte, k_rta, rtol=1e-12, atol=1e-14 * np.abs(k_rta).max())


def test_self_consistent_series_equals_direct_inversion(four_mass_cell):
    s, mesh, nu, eig, g0, G1 = four_mass_cell
    k_dir = co.kappa_bte_direct(s, mesh, nu, eig, g0, G1, 300.0)
    k_sc, n_terms, ok = co.kappa_bte_self_consistent(s, mesh, nu, eig, g0, G1, 300.0)
    assert ok and n_terms > 3
    np.testing.assert_allclose(k_sc, k_dir, rtol=1e-10, atol=1e-12 * np.abs(k_dir).max())
    k_rta = co.kappa_rta(s, mesh, nu, eig, g0.reshape(nu.shape), 300.0)
    assert not np.allclose(k_dir, k_rta, rtol=1e-3)          # the off-diagonal part matters here
    # an off-diagonal part ten times larger makes the series diverge
    _, _, ok_big = co.kappa_bte_self_consistent(s, mesh, nu, eig, g0, 10.0 * G1, 300.0, max_iter=60)
    assert not ok_big
