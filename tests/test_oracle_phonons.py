"""Pins of the oracle's harmonic part: closed-form Born-von Karman spectrum of
the monatomic fcc crystal, zero acoustic frequencies at Gamma, eigenpair
residuals, and Hellmann-Feynman velocities against finite differences."""

import numpy as np
import pytest
import scipy.linalg

import kald_inputs as ki
from kald_inputs.lj import neighbour_list, pair_tensors
from oracle import phonons as ph
from oracle.units import EV_A2_AMU, TWO_PI


def _bvk_nu(q, lat, pos, m):
    """Monatomic closed form D(q) = (1/m) sum_R (1 - cos q.R) K(R)."""
    _, _, _, r = neighbour_list(lat, pos, ki.LJ_CUTOFF)
    K, _ = pair_tensors(r)
    D = np.einsum("r,rab->ab", 1.0 - np.cos(r @ q), K) / m
    lam = np.linalg.eigvalsh(D)
    return np.sqrt(np.abs(lam) * EV_A2_AMU) / TWO_PI * np.sign(lam)


def test_bvk_closed_form_monatomic_fcc():
    w = ki.c1()
    s = w.systems[0]
    nu, _ = ph.phonons(s, w.mesh)
    qs = ki.mesh_qpoints(s.lattice, w.mesh)
    lat, pos = ki.fcc_primitive(ki.A_FCC)
    for k in range(0, len(qs), 7):
        # compare nu^2 (sqrt amplifies the rounding of the zero modes at Gamma)
        ref = _bvk_nu(qs[k], lat, pos, 39.95)
        np.testing.assert_allclose(np.sign(nu[k]) * nu[k] ** 2, np.sign(ref) * ref ** 2,
                                   atol=1e-12 * np.max(ref ** 2) + 1e-14)


@pytest.mark.parametrize("wl", ["C1", "C5"])
def test_acoustic_zero_at_gamma_and_positive_elsewhere(wl):
    w = ki.WORKLOADS[wl](**({"mesh": (4, 4, 4)} if wl == "C5" else {}))
    s = w.systems[0]
    mesh = w.mesh if wl == "C1" else (4, 4, 4)
    nu, eig = ph.phonons(s, mesh)
    assert np.all(np.abs(nu[0, :3]) < 1e-5)
    assert np.all(nu[1:] > 0.05)
    # residual and orthonormality of the eigenpairs
    qs = ki.mesh_qpoints(s.lattice, mesh)
    for k in (1, 5, len(qs) - 1):
        D = ph.dynamical_matrix(s, qs[k])
        E = eig[k].T
        lam = np.sign(nu[k]) * (TWO_PI * nu[k]) ** 2 / EV_A2_AMU
        np.testing.assert_allclose(D @ E, E * lam[None, :], atol=1e-12 * np.abs(D).max())
        np.testing.assert_allclose(E.conj().T @ E, np.eye(E.shape[0]), atol=1e-12)


def test_velocity_matches_finite_difference():
    s = ki.c5(mesh=(2, 2, 2)).systems[0]
    q = np.array([0.11, -0.07, 0.05])
    h = 1e-5
    D = ph.dynamical_matrix(s, q)
    lam, vec = scipy.linalg.eigh(D)
    nu = ph.eigvals_to_thz(lam)
    assert np.min(np.diff(nu)) > 1e-3          # non-degenerate point
    V = ph.velocity_matrices(s, q, vec.T, nu)
    v_hf = np.real(np.einsum("ass->sa", V))
    v_fd = np.zeros_like(v_hf)
    for a in range(3):
        dq = np.zeros(3); dq[a] = h
        lp = ph.eigvals_to_thz(np.linalg.eigvalsh(ph.dynamical_matrix(s, q + dq)))
        lm = ph.eigvals_to_thz(np.linalg.eigvalsh(ph.dynamical_matrix(s, q - dq)))
        v_fd[:, a] = TWO_PI * (lp - lm) / (2 * h)          # d omega / dq in A/ps
    np.testing.assert_allclose(v_hf, v_fd, rtol=1e-6, atol=1e-6 * np.abs(v_fd).max())


def test_sound_velocity_isotropy_small_q():
    """Near Gamma, the longitudinal sound speed along [100] equals
    sqrt(C11 / rho) from the same force constants; here we only pin that the
    Hellmann-Feynman |v| of each acoustic branch tends to omega/|q|."""
    s = ki.c1().systems[0]
    qdir = np.array([1.0, 0.0, 0.0])
    for qq in (1e-3, 2e-3):
        q = qq * qdir
        lam, vec = scipy.linalg.eigh(ph.dynamical_matrix(s, q))
        nu = ph.eigvals_to_thz(lam)
        V = ph.velocity_matrices(s, q, vec.T, nu)
        # degenerate transverse pair: use the trace over the pair
        vl = np.real(V[0, 2, 2])
        np.testing.assert_allclose(vl, TWO_PI * nu[2] / qq, rtol=1e-5)
