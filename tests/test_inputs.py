"""Pins of the synthetic inputs: the RNG against its published outputs, the
analytic LJ force constants against finite differences of the pair energy,
the acoustic sum rules and the permutation symmetry of Phi3."""

import numpy as np
import pytest

import kald_inputs as ki
from kald_inputs.lj import lj_radial, neighbour_list


def test_splitmix64_reference_values():
    # Published output stream of splitmix64 seeded with 1234567 (the test
    # vector in Vigna's reference C implementation).
    g = ki.SplitMix64(1234567)
    got = [g.next_u64() for _ in range(5)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_shuffled_labels_exact_count_and_seeded():
    a = ki.shuffled_labels(32, 16, 2)
    b = ki.shuffled_labels(32, 16, 2)
    c = ki.shuffled_labels(32, 16, 3)
    assert sum(a) == 16 and a == b and a != c


def test_lj_radial_derivatives_finite_difference():
    r = np.linspace(3.3, 8.4, 11)
    h = 1e-4
    v, v1, v2, v3 = lj_radial(r)
    vp, v1p, v2p, _ = lj_radial(r + h)
    vm, v1m, v2m, _ = lj_radial(r - h)
    for exact, num in ((v1, (vp - vm) / (2 * h)), (v2, (v1p - v1m) / (2 * h)),
                       (v3, (v2p - v2m) / (2 * h))):
        np.testing.assert_allclose(exact, num, rtol=1e-6, atol=1e-7 * np.abs(exact).max())


def _home_force(pos, home, rc=ki.LJ_CUTOFF):
    """Force on atom `home` of a finite cluster, from V' only (no K or T)."""
    d = pos - pos[home][None, :]                        # x_b - x_home
    r = np.linalg.norm(d, axis=-1)
    r[home] = np.inf
    _, v1, _, _ = lj_radial(np.where(np.isfinite(r), r, 1.0))
    v1 = np.where(r < rc, v1, 0.0)
    # F_home = -dE/dx_home = sum_b V'(r) (x_b - x_home)/r
    return np.sum((v1 / np.where(np.isfinite(r), r, 1.0))[:, None] * d, axis=0)


@pytest.mark.parametrize("builder", ["prim", "binary"])
def test_lj_fc2_fc3_match_finite_differences_of_forces(builder):
    if builder == "prim":
        lat, pos = ki.fcc_primitive(ki.A_FCC)
    else:
        lat, pos = ki.l11_binary(ki.A_FCC)
    sysm = ki.lj_system(lat, pos, np.ones(len(pos)))
    # finite cluster: every atom within 1.2 rc of the home atom
    cells = np.stack(np.meshgrid(*[np.arange(-5, 6)] * 3, indexing="ij"), -1).reshape(-1, 3)
    allpos, lab = [], []
    for c in cells:
        for a in range(len(pos)):
            x = c @ lat + pos[a]
            if np.linalg.norm(x - pos[0]) < 1.2 * ki.LJ_CUTOFF:
                allpos.append(x)
                lab.append((a, tuple(c)))
    allpos = np.array(allpos)
    index = {l: n for n, l in enumerate(lab)}
    home = index[(0, (0, 0, 0))]
    fc2 = {tuple(k): v for k, v in zip(sysm.fc2_idx.tolist(), sysm.fc2)}
    fc3 = {tuple(k): v for k, v in zip(sysm.fc3_idx.tolist(), sysm.fc3)}
    h = 2e-4
    rng = np.random.default_rng(0)
    # Phi2(i0, jR)_{ab} = -dF_{i0,a}/du_{jR,b}
    for (i, j, *R), blk in list(fc2.items())[:12]:
        if i != 0:
            continue
        t = index[(j, tuple(R))]
        num = np.zeros((3, 3))
        for b in range(3):
            dp = allpos.copy(); dp[t, b] += h
            dm = allpos.copy(); dm[t, b] -= h
            num[:, b] = -(_home_force(dp, home) - _home_force(dm, home)) / (2 * h)
        np.testing.assert_allclose(blk, num, atol=2e-7 * max(1.0, np.abs(blk).max()))
    # Phi3(i0, jRj, kRk)_{abc} = -d2F_{i0,a}/du_{jRj,b} du_{kRk,c}
    keys = list(fc3.keys())
    for n in rng.choice(len(keys), 10, replace=False):
        i, j, r0, r1, r2, k, s0, s1, s2 = keys[n]
        if i != 0:
            continue
        tj, tk = index[(j, (r0, r1, r2))], index[(k, (s0, s1, s2))]
        blk = fc3[keys[n]]
        num = np.zeros((3, 3, 3))
        for b in range(3):
            for c in range(3):
                acc = 0.0
                for sb, sc in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
                    dp = allpos.copy()
                    dp[tj, b] += sb * h
                    dp[tk, c] += sc * h
                    acc = acc + sb * sc * _home_force(dp, home)
                num[:, b, c] = -acc / (4 * h * h)
        np.testing.assert_allclose(blk, num, atol=2e-5 * max(1.0, np.abs(blk).max()))


@pytest.mark.parametrize("wl", ["C1", "C2", "C5"])
def test_acoustic_sum_rules(wl):
    s = ki.WORKLOADS[wl]().systems[0]
    n = s.n_atoms
    acc2 = np.zeros((n, 3, 3))
    np.add.at(acc2, s.fc2_idx[:, 0], s.fc2)
    assert np.abs(acc2).max() < 1e-12 * np.abs(s.fc2).max()
    # sum over the last atom (k, Rk) of Phi3 vanishes for each (i, jRj)
    acc3 = {}
    for key, blk in zip(s.fc3_idx.tolist(), s.fc3):
        kk = tuple(key[:5])
        acc3[kk] = acc3.get(kk, 0.0) + blk
    worst = max(np.abs(v).max() for v in acc3.values())
    assert worst < 1e-12 * np.abs(s.fc3).max()


def test_fc3_permutation_symmetry():
    s = ki.c2().systems[0]
    n = s.n_atoms
    table = {tuple(k): v for k, v in zip(s.fc3_idx.tolist(), s.fc3)}
    # Phi3(i0, jRj, kRk)_{abc} == Phi3(j0, i(-Rj), k(Rk-Rj))_{bac}
    #                         == Phi3(i0, kRk, jRj)_{acb}
    for (i, j, a0, a1, a2, k, b0, b1, b2), blk in list(table.items())[::37]:
        Rj = np.array([a0, a1, a2]); Rk = np.array([b0, b1, b2])
        other = table[(j, i, *(-Rj), k, *(Rk - Rj))]
        np.testing.assert_allclose(blk, np.transpose(other, (1, 0, 2)), atol=1e-13)
        swap = table[(i, k, *Rk, j, *Rj)]
        np.testing.assert_allclose(blk, np.transpose(swap, (0, 2, 1)), atol=1e-13)
    assert n == 32


def test_neighbour_counts_fcc():
    lat, pos = ki.fcc_primitive(ki.A_FCC)
    i, j, nvec, r = neighbour_list(lat, pos, ki.LJ_CUTOFF)
    d = np.sort(np.round(np.linalg.norm(r, axis=1), 2))
    # fcc shells up to 8.5 A: 12 + 6 + 24 + 12 + 24 = 78 neighbours
    assert len(d) == 78
    assert np.allclose(np.unique(d), [3.72, 5.26, 6.44, 7.44, 8.32], atol=0.01)
