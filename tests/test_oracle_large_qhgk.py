"""Pins of the oracle's large-system QHGK options (code-details appendix and
the QHGK section): the Allen-Feldman bandwidth, the energy threshold on the
Lorentzian tau, and the interpolation of gamma(nu) by third-order splines.

* bandwidth b: identical to QHGK with every linewidth equal to pi b (so that
  gamma + gamma' = 2 pi b), and, with classical populations, the Allen-Feldman
  relation tr(kappa)/3 = kB/V sum_mu D_mu with the diffusivities of the same
  bandwidth;
* threshold: kappa_xx grows monotonically with the threshold (every pair adds
  c tau W^2 >= 0 with classical populations) and equals the unthresholded
  kappa once the threshold exceeds the width of the spectrum;
* spline: reproduces a cubic gamma(nu) exactly (not-a-knot ends), passes
  through the data, holds the end values outside the data range, averages
  merged (degenerate) frequencies, and masks low modes.
"""

import numpy as np
import pytest

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import conductivity as co
from oracle import phonons as ph

KB = 1.380649e-23


@pytest.fixture(scope="module")
def cell():
    lat, pos = ki.l11_binary(ki.A_FCC)
    s = ki.supercell_of(lat, pos, [28.09, 72.63], 2)          # 16 atoms, 48 modes
    nu, eig = ph.phonons(s, (1, 1, 1))
    g = an.linewidths_gamma_only(s, nu, eig, 300.0, 0.1)
    return s, nu, eig, g


def test_bandwidth_equals_uniform_linewidths(cell):
    s, nu, eig, g = cell
    b = 0.3
    k_bw = co.kappa_qhgk(s, nu, eig, g, 300.0, bandwidth_thz=b)
    k_uni = co.kappa_qhgk(s, nu, eig, np.full_like(g, np.pi * b), 300.0)
    np.testing.assert_allclose(k_bw, k_uni, rtol=1e-13, atol=1e-15 * np.abs(k_uni).max())
    assert np.abs(k_bw - co.kappa_qhgk(s, nu, eig, g, 300.0)).max() > 1e-3 * np.abs(k_bw).max()


def test_bandwidth_allen_feldman_relation(cell):
    s, nu, eig, g = cell
    b = 0.25
    k = co.kappa_qhgk(s, nu, eig, g, 300.0, classical=True, bandwidth_thz=b)
    D = co.diffusivity(s, nu, eig, g, bandwidth_thz=b)
    lhs = np.trace(k) / 3.0
    rhs = KB / s.volume * np.sum(D) * co.KAPPA_SI
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_threshold_is_monotone_and_saturates(cell):
    s, nu, eig, g = cell
    full = co.kappa_qhgk(s, nu, eig, g, 300.0, classical=True)
    prev = -1.0
    for t in (1e-9, 0.01, 0.05, 0.2, 1.0, 3.0):
        kxx = co.kappa_qhgk(s, nu, eig, g, 300.0, classical=True, threshold_thz=t)[0, 0]
        assert kxx >= prev - 1e-15 * abs(full[0, 0])
        prev = kxx
    width = nu.max() - nu[nu > 0.01].min()
    big = co.kappa_qhgk(s, nu, eig, g, 300.0, classical=True, threshold_thz=width * 1.01)
    np.testing.assert_array_equal(big, full)
    assert co.kappa_qhgk(s, nu, eig, g, 300.0, classical=True, threshold_thz=0.01)[0, 0] < full[0, 0]


def test_spline_reproduces_a_cubic_and_the_data():
    g = ki.SplitMix64(5)
    x = np.sort(np.array([0.2 + 9.0 * g.uniform() for _ in range(40)]))
    cubic = lambda v: 0.05 + 0.01 * v - 0.002 * v ** 2 + 0.0003 * v ** 3
    y = cubic(x)
    xq = np.linspace(x[0], x[-1], 301)
    np.testing.assert_allclose(co.interpolate_gamma(x, y, xq), cubic(xq), rtol=1e-11)
    np.testing.assert_allclose(co.interpolate_gamma(x, y, x), y, rtol=1e-13)
    # outside the data: held at the end values; low modes masked
    out = co.interpolate_gamma(x, y, np.array([0.005, 0.1, 20.0]))
    assert out[0] == 0.0 and out[1] == pytest.approx(y[0], rel=1e-14) and out[2] == pytest.approx(y[-1], rel=1e-14)


def test_spline_merges_degenerate_frequencies():
    x = np.array([1.0, 2.0, 2.0 + 1e-7, 3.0, 4.0, 5.0])
    y = np.array([0.1, 0.2, 0.4, 0.3, 0.35, 0.5])
    ref = co.interpolate_gamma(np.array([1.0, 2.0 + 5e-8, 3.0, 4.0, 5.0]), np.array([0.1, 0.3, 0.3, 0.35, 0.5]),
                               np.array([2.5]))
    assert co.interpolate_gamma(x, y, np.array([2.5]))[0] == pytest.approx(ref[0], rel=1e-12)
