"""The exact symmetries the GPU linewidth paths use to project fewer momentum
triples, checked on the CPU with the oracle's own projections (no GPU).

Time reversal: Phi3 is real, so the projection of (-q, -q', -q'') is the
conjugate of that of (q, q', q'') and w(-q) = w(q); the averaged linewidths
of -q equal those of q.

Permutations: for Phi3 symmetric under permutations of its three indices the
squared projection of a momentum triple (q1, q2, q3), q1 + q2 + q3 = 0 modulo
G, is the same for every order of the triple.  Summing Eq. gamma_operators
over the orbit of one ordered triple under the six permutations and
inversion, each member position p of the triple receives

    (|orbit| / 12) F_p |phi|^2 / (w1 w2 w3)   for q_p and for -q_p,

    F1 = (n2 - n3)(D3 - D2) + (1 + n2 + n3) D1
    F2 = (n1 - n3)(D3 - D1) + (1 + n1 + n3) D2
    F3 = (n1 - n2)(D2 - D1) + (1 + n1 + n2) D3

with D1 = delta(w2 + w3 - w1), D2 = delta(w1 + w3 - w2), D3 = delta(w1 + w2 -
w3): one projection per orbit then gives every linewidth of the mesh.  The
test builds gamma that way from the oracle's projections and compares it with
the oracle's literal sum over all (q, q') and both processes."""

import itertools

import numpy as np
import pytest

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import phonons as ph


def _orbit_gamma(w, delta="gaussian", slip=None):
    s = w.systems[0]
    mesh = w.mesh
    nu, eig = ph.phonons(s, mesh)
    nq, nb = nu.shape
    kf = an.mesh_fractions(mesh)

    def idx(k):
        return int(an.mesh_index(mesh, np.asarray(k)))
    neg = [idx(-kf[q]) for q in range(nq)]
    omega = an.TWO_PI * nu
    valid = nu > 0.01
    n = an.bose(np.where(valid, omega, 0.0), w.T, False)
    inv_w = np.where(valid, 1.0 / np.where(valid, omega, 1.0), 0.0)
    eps = an.mass_scaled_eigvecs(s, eig)
    S = an.fc3_scatter_matrix(s)
    sig_w = an.TWO_PI * w.sigma_thz
    acc = np.zeros((nq, nb))
    n_proj = 0
    for q1 in range(nq):
        for q2 in range(nq):
            q3 = neg[idx(kf[q1] + kf[q2])]
            t = (q1, q2, q3)
            orbit = set()
            for p in itertools.permutations(t):
                orbit.add(p)
                orbit.add(tuple(neg[x] for x in p))
            if t != min(orbit):
                continue
            n_proj += 1
            # phi^+(q1 s1, q2 s2, q1 + q2 s3): position 3 is -(q1 + q2) = q3
            v2 = np.abs(an.projections(s, mesh, eps, q1, [q2], "+", S)[0]) ** 2

            def on(v, pos):
                shape = [1, 1, 1]
                shape[pos] = nb
                return v.reshape(shape)
            w1, w2, w3 = (on(omega[q], i) for i, q in enumerate(t))
            n1, n2, n3 = (on(n[q], i) for i, q in enumerate(t))
            mask = on(valid[q1], 0) & on(valid[q2], 1) & on(valid[q3], 2)
            base = np.where(mask, v2 * on(inv_w[q1], 0) * on(inv_w[q2], 1) * on(inv_w[q3], 2), 0.0)

            def d(x):
                return an.energy_delta(x, sig_w, w.n_sigma, delta)
            D1, D2, D3 = d(w2 + w3 - w1), d(w1 + w3 - w2), d(w1 + w2 - w3)
            F = ((n2 - n3) * (D3 - D2) + (1 + n2 + n3) * D1,
                 (n1 - n3) * (D3 - D1) + (1 + n1 + n3) * D2,
                 (n1 - n2) * (D2 - D1) + (1 + n1 + n2) * D3)
            axes = ((1, 2), (0, 2), (0, 1))
            for pos in range(3):
                weight = 1.0 / 12.0 if slip == "orbit_weight" else len(orbit) / 12.0
                Fp = F[0] if slip == "position" else F[pos]
                c = weight * np.sum(base * Fp, axis=axes[pos])
                acc[t[pos]] += c
                acc[neg[t[pos]]] += c
    pref = an.HBAR_EVPS * np.pi / 8.0 * an.EV_A2_AMU ** 3 / nq
    gam = np.array([an.degenerate_average(nu[q], pref * acc[q], 1e-5) for q in range(nq)])
    ref = an.linewidths(s, mesh, nu, eig, w.T, w.sigma_thz, w.n_sigma, delta=delta)
    return gam, ref, n_proj


@pytest.mark.parametrize("mesh,delta,n_orbits", [((3, 3, 3), "gaussian", 79), ((4, 2, 1), "lorentzian", 11),
                                                 ((4, 4, 1), "triangular", 31)])
def test_one_projection_per_orbit_gives_the_oracle_linewidths(mesh, delta, n_orbits):
    w = ki.small_binary(mesh=mesh, sigma=0.1)
    gam, ref, n_proj = _orbit_gamma(w, delta)
    assert n_proj == n_orbits
    floor = 1e-6 * ref.max()
    assert np.max(np.abs(gam - ref) / np.maximum(np.abs(ref), floor)) < 1e-12


def test_time_reversal_gives_equal_linewidths_at_q_and_minus_q():
    w = ki.small_binary(mesh=(4, 3, 2), sigma=0.1)
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    g = an.linewidths(s, w.mesh, nu, eig, w.T, w.sigma_thz, w.n_sigma)
    kf = an.mesh_fractions(w.mesh)
    for q in range(len(kf)):
        qn = int(an.mesh_index(w.mesh, -kf[q]))
        np.testing.assert_allclose(g[q], g[qn], rtol=1e-11, atol=1e-14 * g.max())


@pytest.mark.parametrize("slip", ["orbit_weight", "position"])
def test_a_plausible_slip_in_the_orbit_sums_is_caught(slip):
    """Counting every orbit once (weight 1/12 instead of |orbit| / 12), or
    giving every position the weights of position 1, moves gamma far beyond
    the 1e-12 bar of the test above."""
    w = ki.small_binary(mesh=(3, 3, 1), sigma=0.1)
    gam, ref, _ = _orbit_gamma(w, slip=slip)
    assert np.max(np.abs(gam - ref) / np.maximum(np.abs(ref), 1e-6 * ref.max())) > 1e-3


@pytest.mark.parametrize("mesh", [(2, 2, 2), (3, 3, 1), (4, 2, 1), (3, 4, 5)])
def test_orbit_count_of_the_bench_matches_a_brute_force_enumeration(mesh):
    """bench.orbit_pairs (the projections the tensor path makes on a whole
    mesh) equals the number of orbits of ordered momentum triples under the
    six permutations and inversion, enumerated here one triple at a time."""
    import bench
    kf = an.mesh_fractions(mesh)
    nq = len(kf)

    def idx(k):
        return int(an.mesh_index(mesh, np.asarray(k)))
    neg = [idx(-kf[q]) for q in range(nq)]
    seen, n = set(), 0
    for q1 in range(nq):
        for q2 in range(nq):
            t = (q1, q2, neg[idx(kf[q1] + kf[q2])])
            if t in seen:
                continue
            n += 1
            for p in itertools.permutations(t):
                seen.add(p)
                seen.add(tuple(neg[x] for x in p))
    assert bench.orbit_pairs(mesh) == n
    assert len(seen) == nq * nq
