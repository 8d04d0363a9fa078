"""Pins of the oracle's projection and linewidths.

* brute force: the projection equals the explicit real-space triple sum over
  an N x N x N supercell with Bloch displacement patterns (divided by N^3),
  and vanishes when q'' != q + q' -- for LJ and for a random Phi3 with both
  replica vectors non-zero;
* time reversal: phi^-(q; q'; q-q') = phi^+(q; -q'; q-q') up to gauge;
* gamma(q) = gamma(-q); gamma scales as s^2 with Phi3 -> s Phi3;
* T -> 0 removes the + process;
* detailed balance under exact energy conservation pins the factor 1/2 on
  Gamma^- relative to Gamma^+ and the Bose factor combinations;
* folding: a Gamma-only N^3 supercell gives the same linewidths as the N^3
  mesh (pins the 1/N_k normalisation and the phase conventions);
* the crystal route at mesh 1x1x1 and the Gamma-only route agree.
"""

import numpy as np
import pytest

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import phonons as ph
from oracle.units import TWO_PI


def _supercell_fc3(sys, N):
    """Dense Phi3 over the N^3-cell supercell dofs (l, i, a), images folded."""
    n = sys.n_atoms
    cells = ki.mesh_fractions((N, N, N))
    cidx = {tuple(c): x for x, c in enumerate(cells)}
    nd = 3 * n * len(cells)
    F = np.zeros((nd, nd, nd))
    for key, blk in zip(sys.fc3_idx, sys.fc3):
        i, j, rj, k, rk = key[0], key[1], key[2:5], key[5], key[6:9]
        for l, c in enumerate(cells):
            lj = cidx[tuple((c + rj) % N)]
            lk = cidx[tuple((c + rk) % N)]
            a = 3 * (l * n + i)
            b = 3 * (lj * n + j)
            cc = 3 * (lk * n + k)
            F[a:a + 3, b:b + 3, cc:cc + 3] += blk
    return F, cells


def _bloch(sys, eps_q, q_cart, cells):
    """u_{(l,i,a)}(q, s) = eps_{ia}(q, s) exp(-i q.R_l) for every mode s."""
    R = cells.astype(float) @ sys.lattice
    ph_l = np.exp(-1j * (R @ q_cart))                               # [L]
    return (ph_l[None, :, None] * eps_q[:, None, :]).reshape(eps_q.shape[0], -1)


@pytest.mark.parametrize("kind", ["prim", "binary", "binary_random"])
def test_projection_matches_real_space_triple_sum(kind):
    N = 3 if kind == "prim" else 2
    w = ki.small_fcc_prim() if kind == "prim" else ki.small_binary()
    s = w.systems[0]
    if kind == "binary_random":
        s = ki.random_fc3_system(s, 40, seed=7)
    mesh = (N, N, N)
    nu, eig = ph.phonons(s, mesh)
    eps = an.mass_scaled_eigvecs(s, eig)
    F, cells = _supercell_fc3(s, N)
    qs = ki.mesh_qpoints(s.lattice, mesh)
    kf = ki.mesh_fractions(mesh)
    L = len(cells)
    scale = np.abs(an.projections(s, mesh, eps, 1, list(range(len(qs))), "+")).max()
    for q, qp in ((1, 2), (3, 5), (0, 4), (7, 7), (2, 6)):
        qpp = int(an.mesh_index(mesh, kf[q] + kf[qp]))
        phi = an.projections(s, mesh, eps, q, [qp], "+")[0]
        u = _bloch(s, eps[q], qs[q], cells)
        up = _bloch(s, eps[qp], qs[qp], cells)
        upp = _bloch(s, eps[qpp], qs[qpp], cells)
        brute = np.einsum("abc,sa,tb,uc->stu", F, u, up, upp.conj()) / L
        np.testing.assert_allclose(phi, brute, atol=1e-11 * scale)
        # a q'' that breaks momentum conservation gives zero
        bad = (qpp + 1) % len(qs)
        ub = _bloch(s, eps[bad], qs[bad], cells)
        zero = np.einsum("abc,sa,tb,uc->stu", F, u, up, ub.conj()) / L
        assert np.abs(zero).max() < 1e-11 * scale


def _collapse(x, sets_list):
    """Sum |phi|^2 over degenerate sets along each of the three axes."""
    for ax, sets in enumerate(sets_list):
        x = np.stack([np.take(x, s, axis=ax).sum(axis=ax) for s in sets], axis=ax)
    return x


def test_time_reversal_of_the_minus_process():
    w = ki.small_binary(mesh=(3, 3, 3))
    s = w.systems[0]
    mesh = w.mesh
    nu, eig = ph.phonons(s, mesh)
    eps = an.mass_scaled_eigvecs(s, eig)
    kf = ki.mesh_fractions(mesh)
    for q, qp in ((1, 4), (5, 11), (2, 2)):
        mqp = int(an.mesh_index(mesh, -kf[qp]))
        qpp = int(an.mesh_index(mesh, kf[q] - kf[qp]))
        a = np.abs(an.projections(s, mesh, eps, q, [qp], "-")[0]) ** 2
        b = np.abs(an.projections(s, mesh, eps, q, [mqp], "+")[0]) ** 2
        sets = [ph.degenerate_sets(nu[x], 1e-6) for x in (q, qp, qpp)]
        np.testing.assert_allclose(_collapse(a, sets), _collapse(b, sets),
                                   rtol=1e-9, atol=1e-12 * a.max())


def test_gamma_even_in_q_and_scaling():
    w = ki.small_binary(mesh=(3, 3, 3))
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    kf = ki.mesh_fractions(w.mesh)
    qs = [1, 5, 13]
    mq = [int(an.mesh_index(w.mesh, -kf[q])) for q in qs]
    g = an.linewidths(s, w.mesh, nu, eig, w.T, w.sigma_thz, q_list=qs + mq)
    np.testing.assert_allclose(g[:3], g[3:], rtol=1e-10)
    s2 = ki.System(s.masses, s.positions, s.lattice, s.fc2_idx, s.fc2, s.fc3_idx,
                   1.7 * s.fc3)
    g2 = an.linewidths(s2, w.mesh, nu, eig, w.T, w.sigma_thz, q_list=qs)
    np.testing.assert_allclose(g2, 1.7 ** 2 * g[:3], rtol=1e-12)
    assert np.all(g[:3] > 0)


def test_zero_temperature_removes_plus_process():
    w = ki.small_binary(mesh=(3, 3, 3))
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    _, gp, gm = an.linewidths(s, w.mesh, nu, eig, 0.05, w.sigma_thz, q_list=[4, 9],
                              average=False, return_parts=True)
    assert np.all(gm[:, -1] > 0)
    assert np.abs(gp).max() < 1e-12 * np.abs(gm).max()


def test_detailed_balance_pins_half_on_minus_process():
    """With frequencies on a grid of step d and sigma << d only exactly
    energy-conserving triplets survive; then every triplet a + b -> c
    contributes the same amount to sum_mu n(1+n) gamma_mu through each of its
    three members (n_c(1+n_a+n_b) = n_a n_b when w_c = w_a + w_b), so the +
    part of that sum is exactly twice the - part.  Without the 1/2 on
    Gamma^- the two parts would be equal."""
    w = ki.small_binary(mesh=(3, 3, 3))
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    d = 0.05
    nu_q = np.round(nu / d) * d
    T = 150.0
    _, gp, gm = an.linewidths(s, w.mesh, nu_q, eig, T, sigma_thz=0.004, n_sigma=3.0,
                              average=False, return_parts=True)
    valid = nu_q > 0.01
    n = an.bose(np.where(valid, TWO_PI * nu_q, 0.0), T)
    wgt = n * (1 + n)
    plus = np.sum(wgt * gp)
    minus = np.sum(wgt * gm)
    assert plus > 0 and minus > 0
    np.testing.assert_allclose(plus, 2.0 * minus, rtol=1e-9)


def _match_by_frequency(nu_a, g_a, nu_b, g_b, tol=1e-6):
    """Sort both spectra, check they coincide, and compare gamma averaged over
    clusters of equal frequency (gauge-free comparison)."""
    ia, ib = np.argsort(nu_a), np.argsort(nu_b)
    na, nb_ = nu_a[ia], nu_b[ib]
    np.testing.assert_allclose(na, nb_, atol=1e-6)   # Gamma acoustic zeros are ~1e-8 noise
    ga, gb = g_a[ia], g_b[ib]
    start = 0
    out_a, out_b = [], []
    for x in range(1, len(na) + 1):
        if x == len(na) or na[x] - na[x - 1] > tol:
            out_a.append(ga[start:x].mean())
            out_b.append(gb[start:x].mean())
            start = x
    return np.array(out_a), np.array(out_b)


@pytest.mark.parametrize("kind,N", [("prim", 3), ("binary", 2)])
def test_supercell_folding_equals_mesh(kind, N):
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
    assert np.abs(eig_s.imag).max() == 0.0
    g_s = an.linewidths_gamma_only(sup, nu_s, eig_s, T, sig)
    a, b = _match_by_frequency(nu_m.reshape(-1), g_m.reshape(-1), nu_s[0], g_s)
    np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-12)
    # the crystal route evaluated at mesh 1x1x1 agrees with the Gamma-only route
    g_c = an.linewidths(sup, (1, 1, 1), nu_s, eig_s, T, sig)[0]
    np.testing.assert_allclose(g_c, g_s, rtol=1e-9, atol=1e-12)
