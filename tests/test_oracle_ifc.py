"""Pins of the oracle's finite-difference force constants (oracle/ifc.py):
against the analytic chain-rule derivatives of the same Lennard-Jones pair
potential (kald_inputs), with the O(h^2) convergence of central differences,
and the acoustic sum rule of the forces (Newton's third law)."""

import numpy as np
import pytest

import kald_inputs as ki
from oracle import ifc


@pytest.fixture(scope="module")
def binary():
    return ki.small_binary(mesh=(2, 2, 2)).systems[0]


def test_fd_matches_analytic_with_second_order_convergence(binary):
    s = binary
    errs2, errs3 = [], []
    for h in (4e-3, 2e-3):
        f2, f3 = ifc.fd_force_constants(s, h=h)
        errs2.append(np.abs(f2 - s.fc2).max() / np.abs(s.fc2).max())
        errs3.append(np.abs(f3 - s.fc3).max() / np.abs(s.fc3).max())
    assert errs2[1] < 1e-5 and errs3[1] < 1e-4
    # halving h divides the error by about four
    assert 3.0 < errs2[0] / errs2[1] < 5.0
    assert 3.0 < errs3[0] / errs3[1] < 5.0


def test_fd_acoustic_sum_rule(binary):
    s = binary
    f2, f3 = ifc.fd_force_constants(s, h=1e-3)
    for i in range(s.n_atoms):
        tot = f2[s.fc2_idx[:, 0] == i].sum(axis=0)
        assert np.abs(tot).max() < 1e-10 * np.abs(f2).max()
    # Phi3 summed over its last atom (every image) vanishes for each (i, jRj)
    keys = {}
    for x, key in enumerate(s.fc3_idx):
        keys.setdefault(tuple(key[:5]), []).append(x)
    worst = max(np.abs(f3[v].sum(axis=0)).max() for v in keys.values())
    assert worst < 1e-8 * np.abs(f3).max()
