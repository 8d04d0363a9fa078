"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Stage-isolated where the eigensolver gauge would get in the way: the GPU
linewidth and conductivity calls are fed the oracle's frequencies and
eigenvectors, so gamma and kappa are compared element by element.  End-to-end
checks compare only gauge-invariant results.

Tolerances: FP64 path 1e-10 relative (the arithmetic is the same up to the
order of the sums); FP32 path 1e-5 relative on gamma and 1e-4 on kappa.
"""

import numpy as np
import pytest

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import conductivity as co
from oracle import phonons as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def k():
    from paper_2009_01967_gb300 import build
    build.build()
    import paper_2009_01967_gb300 as kk
    ctx = kk.Context(0)
    yield kk, ctx
    ctx.close()


def _opts(kk, w, precision="fp64", **kw):
    return kk.Options(temperature_K=w.T, sigma_thz=w.sigma_thz, n_sigma=w.n_sigma,
                      precision=precision, **kw)


def _rel(a, b, floor):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor))


# ---------------------------------------------------------------- phonons
@pytest.mark.parametrize("case", ["C1", "binary3", "C2"])
def test_phonons_match_oracle(k, case):
    kk, ctx = k
    if case == "C1":
        w = ki.c1()
    elif case == "binary3":
        w = ki.small_binary(mesh=(3, 3, 3))
    else:
        w = ki.c2()
    s = w.systems[0]
    nu, eig, vel = kk.kald_phonons(ctx, s, w.mesh)
    nu_o, eig_o = ph.phonons(s, w.mesh)
    # squared frequencies to 1e-12 of the largest (sqrt amplifies zeros at Gamma)
    sq = lambda x: np.sign(x) * x * x
    np.testing.assert_allclose(sq(nu), sq(nu_o), atol=1e-12 * np.max(nu_o) ** 2)
    assert np.all(np.diff(nu, axis=1) >= -1e-12)             # ascending
    qs = ki.mesh_qpoints(s.lattice, w.mesh)
    scale = np.abs(ph.dynamical_matrix(s, qs[len(qs) // 2])).max()   # D(Gamma) ~ 0 for C1
    for q in range(0, len(qs), max(1, len(qs) // 9)):
        D = ph.dynamical_matrix(s, qs[q])
        E = eig[q].T
        np.testing.assert_allclose(E.conj().T @ E, np.eye(E.shape[0]), atol=1e-12)
        res = D @ E - E * (np.diag(E.conj().T @ D @ E).real)[None, :]
        assert np.abs(res).max() < 1e-11 * scale
    # velocities of non-degenerate modes (degenerate ones depend on the basis)
    v_o = ph.group_velocities(s, w.mesh, nu_o, eig_o)
    for q in range(len(qs)):
        gaps = np.diff(nu_o[q])
        nd = np.ones(nu_o.shape[1], bool)
        nd[:-1] &= gaps > 1e-6
        nd[1:] &= gaps > 1e-6
        nd &= nu_o[q] > 0.01
        np.testing.assert_allclose(vel[q][nd], v_o[q][nd], rtol=1e-8, atol=1e-9)


# ---------------------------------------------------------------- linewidths
def _lw_case(case):
    if case == "C1":
        return ki.c1()
    if case == "binary3":
        return ki.small_binary(mesh=(3, 3, 3), sigma=0.1)
    if case == "binary_random":
        w = ki.small_binary(mesh=(3, 3, 3), sigma=0.1)
        w.systems = [ki.random_fc3_system(w.systems[0], 60, seed=11)]
        return w
    if case == "gamma_only_32":
        s = ki.fcc_supercell_system(2, seed=5)
        return ki.Workload("g32", [s], (1, 1, 1), 300.0, 0.1, 3.0)
    if case == "C5_mesh6":
        return ki.c5(mesh=(6, 6, 6))
    if case == "binary_mesh234":
        # uneven mesh: the phase roots have order lcm(2, 3, 4) = 12
        return ki.small_binary(mesh=(2, 3, 4), sigma=0.1)
    raise KeyError(case)


def _cell_case(case):
    """Crystal cells of 4 and 32 atoms: fcc4_mesh3 (12 branches, the FP32
    CUDA-core kernel in the split mode), fcc32_mesh2 / fcc32_mesh211 (96
    branches, the tensor-core path), fcc32_random (96 branches with random
    third-order blocks whose two lattice vectors are both non-zero)."""
    if case == "fcc4_mesh3":
        return ki.Workload("fcc4", [ki.fcc_supercell_system(1, seed=7)], (3, 3, 3), 300.0, 0.1, 3.0)
    if case == "fcc32_mesh2":
        return ki.Workload("fcc32", [ki.fcc_supercell_system(2, seed=2)], (2, 2, 2), 300.0, 0.1, 3.0)
    if case == "fcc32_mesh211":
        return ki.Workload("fcc32", [ki.fcc_supercell_system(2, seed=2)], (2, 1, 1), 300.0, 0.1, 3.0)
    if case == "fcc32_mesh311":
        # (1/3, 0, 0) carries group velocities (on a 2 x 1 x 1 mesh they vanish by symmetry)
        return ki.Workload("fcc32", [ki.fcc_supercell_system(2, seed=2)], (3, 1, 1), 300.0, 0.1, 3.0)
    if case == "fcc32_random":
        base = ki.fcc_supercell_system(2, seed=2)
        return ki.Workload("fcc32r", [ki.random_fc3_system(base, 400, seed=13)], (2, 1, 1), 300.0, 0.1, 3.0)
    raise KeyError(case)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["C1", "binary3", "binary_random", "gamma_only_32", "C5_mesh6",
                                  "binary_mesh234"])
def test_linewidths_match_oracle(k, case, precision):
    kk, ctx = k
    w = _lw_case(case)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, precision))
    g = g.reshape(g_o.shape)
    assert tot == w.n_q ** 2 * s.n_branches ** 3
    floor = 1e-6 * g_o.max()
    if precision == "fp64":
        assert _rel(g, g_o, floor) < 1e-10
    else:
        assert _rel(g, g_o, floor) < 1e-5
    assert np.all(g[nu_o <= 0.01] == 0.0)
    # delta-allowed count: (s, s', s'') with both modes valid and |d nu| < n sigma sigma
    if precision == "fp64":
        nq, nb = nu_o.shape
        kf = ki.mesh_fractions(w.mesh)
        valid = nu_o > 0.01
        cnt = 0
        cut = w.n_sigma * w.sigma_thz * 2 * np.pi
        om = 2 * np.pi * nu_o
        for q in range(nq):
            qpp = an.mesh_index(w.mesh, kf[q][None, :] + kf)
            a = om[q][:, None, None]
            b = om[:, None, :, None]
            c = om[qpp][:, None, None, :]
            ok = valid[q][:, None, None] & valid[:, None, :, None] & valid[qpp][:, None, None, :]
            hit = (np.abs(a + b - c) < cut) | (np.abs(a - b - c) < cut)
            cnt += int(np.sum(ok & hit))
        assert allowed == cnt


def test_linewidths_c2_sampled_q(k):
    """Full-size 32-atom / 8^3 workload in the launch configuration the
    benchmark times (FP32), checked at sampled q-points against the oracle."""
    kk, ctx = k
    w = ki.c2()
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "fp32"))
    g = g.reshape(nu_o.shape)
    qs = [1, 137]
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma, q_list=qs)
    assert _rel(g[qs], g_o, 1e-6 * g_o.max()) < 1e-5
    assert tot == 512 ** 2 * 96 ** 3 and 0 < allowed < tot


@pytest.mark.parametrize("case", ["binary3", "binary_random", "C5_mesh6", "fcc4_mesh3", "fcc32_mesh2",
                                  "fcc32_random"])
def test_crystal_bf16split_tensor_cores(k, case):
    """Crystal linewidths in the BF16-split mode: the contractions on tcgen05
    (BF16 pieces, FP32 accumulation) for cells of 65 to 96 branches, the FP32
    CUDA-core kernel for 3 to 64 branches, the FP32 register kernel for one-
    and two-atom cells.  The delta windows are decided in FP32 as in the FP32
    CUDA-core path, so the allowed counts agree (exactly, or within the
    rounding of the window edges where one projection per orbit of momentum
    triples counts every member's windows); gamma within 1e-5 of the FP64
    oracle."""
    kk, ctx = k
    if case.startswith("fcc"):
        w = _cell_case(case)
    else:
        w = _lw_case(case)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "bf16split"))
    _, (_, allowed32) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "fp32"))
    g = g.reshape(g_o.shape)
    assert tot == w.n_q ** 2 * s.n_branches ** 3
    assert abs(allowed - allowed32) <= 1e-5 * allowed32
    assert np.all(g[nu_o <= 0.01] == 0.0)
    err = _rel(g, g_o, 1e-6 * g_o.max())
    print(f"{case}: bf16 split gamma max rel err {err:.3e}")
    assert err < 1e-5


@pytest.mark.parametrize("case", ["fcc32_random", "fcc32_mesh2"])
def test_crystal_bf16split_phase_sum_kernels(k, case, monkeypatch):
    """The phase sum Y_s(b, c) of the tensor-core crystal path computed either
    way -- as a tcgen05 GEMM over the phase-folded fc3 blocks (the default)
    or on CUDA cores (KALD_TCX_Y=0) -- gives gamma within 1e-5 of the FP64
    oracle and the same delta-allowed count."""
    kk, ctx = k
    w = _cell_case(case)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    out = {}
    for yk in ("1", "0"):
        monkeypatch.setenv("KALD_TCX_Y", yk)
        g, (tot, allowed) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "bf16split"))
        out[yk] = (g.reshape(g_o.shape), allowed)
    monkeypatch.delenv("KALD_TCX_Y")
    assert out["1"][1] == out["0"][1]
    for yk, (g, _) in out.items():
        err = _rel(g, g_o, 1e-6 * g_o.max())
        print(f"{case} phase sum on {'tensor' if yk == '1' else 'CUDA'} cores: gamma max rel err {err:.3e}")
        assert err < 1e-5


def test_crystal_bf16split_c2_sampled_q(k):
    """The 32-atom / 8^3 workload on tensor cores in the benchmark's launch
    configuration, checked at sampled q-points against the oracle."""
    kk, ctx = k
    w = ki.c2()
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "bf16split"))
    g = g.reshape(nu_o.shape)
    qs = [1, 137]
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma, q_list=qs)
    err = _rel(g[qs], g_o, 1e-6 * g_o.max())
    print(f"C2 bf16 split gamma max rel err {err:.3e}")
    # error against frequency at the acoustic edge (q = 1 is the mesh point next to Gamma)
    order = np.argsort(nu_o[1])
    low = [m for m in order if nu_o[1][m] > 0.01][:8]
    for m in low:
        print(f"  q=1 mode {m}: nu {nu_o[1][m]:.4f} THz, rel err {abs(g[1][m] - g_o[0][m]) / g_o[0][m]:.2e}")
    assert err < 1e-5
    assert tot == 512 ** 2 * 96 ** 3 and 0 < allowed < tot


# ---------------------------------------------------------------- kappa
def test_kappa_rta_matches_oracle(k):
    kk, ctx = k
    w = ki.c1()
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    kap = kk.kald_kappa_rta(ctx, s, w.mesh, nu_o, eig_o, g_o, _opts(kk, w))
    kap_o = co.kappa_rta(s, w.mesh, nu_o, eig_o, g_o, w.T)
    np.testing.assert_allclose(kap, kap_o, rtol=1e-10, atol=1e-12 * np.abs(kap_o).max())


def test_kappa_rta_binary_anisotropic(k):
    kk, ctx = k
    w = ki.small_binary(mesh=(4, 4, 4), sigma=0.1)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    kap = kk.kald_kappa_rta(ctx, s, w.mesh, nu_o, eig_o, g_o, _opts(kk, w))
    kap_o = co.kappa_rta(s, w.mesh, nu_o, eig_o, g_o, w.T)
    np.testing.assert_allclose(kap, kap_o, rtol=1e-10, atol=1e-12 * np.abs(kap_o).max())


@pytest.mark.parametrize("kind", ["fcc32", "binary16"])
def test_kappa_qhgk_matches_oracle(k, kind):
    """(The 4-atom cubic cell is not used: every atom is an inversion centre
    of its images there, so the generalised velocity vanishes identically.)"""
    kk, ctx = k
    if kind == "fcc32":
        s = ki.fcc_supercell_system(2, seed=5)
    else:
        lat, pos = ki.l11_binary(ki.A_FCC)
        s = ki.supercell_of(lat, pos, [28.09, 72.63], 2)
    T, sig = 300.0, 0.1
    nu_o, eig_o = ph.phonons(s, (1, 1, 1))
    g_o = an.linewidths_gamma_only(s, nu_o, eig_o, T, sig)
    w = ki.Workload("q", [s], (1, 1, 1), T, sig, 3.0)
    kap, vgen = kk.kald_kappa_qhgk(ctx, [s], nu_o, eig_o, g_o, _opts(kk, w), want_vgen=True)
    W_o = co.generalized_velocity(s, nu_o, eig_o)
    kap_o = co.kappa_qhgk(s, nu_o, eig_o, g_o, T, W=W_o)
    np.testing.assert_allclose(vgen, W_o, rtol=1e-10, atol=1e-11 * np.abs(W_o).max())
    np.testing.assert_allclose(kap[0], kap_o, rtol=1e-10, atol=1e-12 * np.abs(kap_o).max())


# ---------------------------------------------------------------- end to end
def test_end_to_end_c1_gauge_free(k):
    kk, ctx = k
    w = ki.c1()
    s = w.systems[0]
    nu, eig, _ = kk.kald_phonons(ctx, s, w.mesh)
    g, _ = kk.kald_linewidths(ctx, s, w.mesh, nu, eig, _opts(kk, w))
    kap = kk.kald_kappa_rta(ctx, s, w.mesh, nu, eig, g, _opts(kk, w))
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    kap_o = co.kappa_rta(s, w.mesh, nu_o, eig_o, g_o, w.T)
    err_g = _rel(g.reshape(g_o.shape), g_o, 1e-6 * g_o.max())
    err_k = np.max(np.abs(kap - kap_o)) / np.max(np.abs(kap_o))
    print(f"C1 end to end (GPU phonons): gamma rel err {err_g:.2e}, kappa rel err {err_k:.2e}")
    assert err_g < 1e-10
    assert err_k < 1e-10


def test_device_pointers_in_and_out(k):
    torch = pytest.importorskip("torch")
    kk, ctx = k
    w = ki.small_binary(mesh=(3, 3, 3), sigma=0.1)
    s = w.systems[0]
    nq, nb = w.n_q, s.n_branches
    nu = torch.zeros((nq, nb), dtype=torch.float64, device="cuda")
    eig = torch.zeros((nq, nb, nb), dtype=torch.complex128, device="cuda")
    kk.kald_phonons(ctx, s, w.mesh, nu_thz=nu, eigvec=eig, want_vel=False)
    g = torch.zeros(nq * nb, dtype=torch.float64, device="cuda")
    kk.kald_linewidths(ctx, s, w.mesh, nu, eig, _opts(kk, w), gamma=g)
    kap = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    kk.kald_kappa_rta(ctx, s, w.mesh, nu, eig, g, _opts(kk, w), kappa=kap)
    nu_h, eig_h, _ = kk.kald_phonons(ctx, s, w.mesh, want_vel=False)
    g_h, _ = kk.kald_linewidths(ctx, s, w.mesh, nu_h, eig_h, _opts(kk, w))
    kap_h = kk.kald_kappa_rta(ctx, s, w.mesh, nu_h, eig_h, g_h, _opts(kk, w))
    np.testing.assert_allclose(kap.cpu().numpy(), kap_h, rtol=1e-12)


# ---------------------------------------------------------------- errors
def test_invalid_inputs_are_rejected(k):
    kk, ctx = k
    w = ki.small_binary(mesh=(2, 2, 2))
    s = w.systems[0]
    bad = ki.System(np.array([28.09, -1.0]), s.positions, s.lattice, s.fc2_idx, s.fc2,
                    s.fc3_idx, s.fc3)
    with pytest.raises(kk.KaldError) as e:
        kk.kald_phonons(ctx, bad, w.mesh)
    assert e.value.status == 1
    with pytest.raises(kk.KaldError) as e:
        kk.kald_phonons(ctx, s, (0, 2, 2))
    assert e.value.status == 1
    nu, eig, _ = kk.kald_phonons(ctx, s, w.mesh)
    o = _opts(kk, w)
    o.n_sigma = 0.0
    with pytest.raises(kk.KaldError) as e:
        kk.kald_linewidths(ctx, s, w.mesh, nu, eig, o)
    assert e.value.status == 1
    big = ki.fcc_supercell_system(3, seed=1)        # 108 atoms: nb = 324 > 96
    with pytest.raises(kk.KaldError) as e:
        kk.kald_phonons(ctx, big, (2, 1, 1))         # large cells only at Gamma
    assert e.value.status == 6


# ---------------------------------------------------------------- large Gamma-only cells
@pytest.fixture(scope="module")
def big324():
    """108-atom (324-mode) disordered supercell, the smallest of the batched
    Gamma-only workload (heavy fraction 0.3, seed 1000)."""
    s = ki.fcc_supercell_system(3, seed=1000, heavy_fraction=0.3)
    nu_o, eig_o = ph.phonons(s, (1, 1, 1))
    g_o = an.linewidths_gamma_only(s, nu_o, eig_o, 300.0, 0.05)
    return s, nu_o, eig_o, g_o


def test_large_gamma_phonons_match_oracle(k, big324):
    kk, ctx = k
    s, nu_o, eig_o, _ = big324
    nu, eig, _ = kk.kald_phonons(ctx, s, (1, 1, 1), want_vel=False)
    sq = lambda x: np.sign(x) * x * x
    np.testing.assert_allclose(sq(nu), sq(nu_o), atol=1e-11 * np.max(nu_o) ** 2)
    assert np.abs(eig.imag).max() == 0.0
    E = eig[0].real.T
    np.testing.assert_allclose(E.T @ E, np.eye(E.shape[0]), atol=1e-11)
    D = ph.dynamical_matrix(s, np.zeros(3)).real
    res = D @ E - E * np.diag(E.T @ D @ E)[None, :]
    assert np.abs(res).max() < 1e-11 * np.abs(D).max()


@pytest.mark.parametrize("ncell", [4, 5])
def test_large_gamma_phonons_768_and_1500_modes(k, ncell):
    """The 256- and 500-atom supercells of the batched Gamma-only workload
    (768 and 1500 modes: several CTAs per tridiagonalisation step, several
    eigenvectors per back-transformation CTA).  Eigenvalues against LAPACK on
    the oracle's dynamical matrix; the smallest relative gap between
    non-acoustic eigenvalues is about 3e-5, so inverse-iteration vectors are
    orthogonal to about eps / gap ~ 1e-11."""
    kk, ctx = k
    s = ki.fcc_supercell_system(ncell, seed=1000 + ncell, heavy_fraction=0.3)
    nu_o, _ = ph.phonons(s, (1, 1, 1))
    nu, eig, _ = kk.kald_phonons(ctx, s, (1, 1, 1), want_vel=False)
    sq = lambda x: np.sign(x) * x * x
    np.testing.assert_allclose(sq(nu), sq(nu_o), atol=1e-11 * np.max(nu_o) ** 2)
    assert np.abs(eig.imag).max() == 0.0
    E = eig[0].real.T
    orth = np.abs(E.T @ E - np.eye(E.shape[0])).max()
    D = ph.dynamical_matrix(s, np.zeros(3)).real
    res = np.abs(D @ E - E * np.diag(E.T @ D @ E)[None, :]).max() / np.abs(D).max()
    print(f"{E.shape[0]} modes: |E^T E - 1| {orth:.2e}, residual {res:.2e}")
    assert orth < 1e-10
    assert res < 1e-11


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_large_gamma_linewidths_match_oracle(k, big324, precision, tol):
    kk, ctx = k
    s, nu_o, eig_o, g_o = big324
    w = ki.Workload("g324", [s], (1, 1, 1), 300.0, 0.05, 3.0)
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, (1, 1, 1), nu_o, eig_o, _opts(kk, w, precision))
    assert tot == 324 ** 3 and 0 < allowed < tot
    assert _rel(g, g_o, 1e-6 * g_o.max()) < tol


def test_large_gamma_end_to_end_qhgk(k, big324):
    kk, ctx = k
    s, nu_o, eig_o, g_o = big324
    w = ki.Workload("g324", [s], (1, 1, 1), 300.0, 0.05, 3.0)
    nu, eig, _ = kk.kald_phonons(ctx, s, (1, 1, 1), want_vel=False)
    g, _ = kk.kald_linewidths(ctx, s, (1, 1, 1), nu, eig, _opts(kk, w))
    kap, _ = kk.kald_kappa_qhgk(ctx, [s], nu, eig, g, _opts(kk, w))
    kap_o = co.kappa_qhgk(s, nu_o, eig_o, g_o, 300.0)
    assert _rel(g, g_o, 1e-6 * g_o.max()) < 1e-8        # gauge-free after degenerate averaging
    np.testing.assert_allclose(kap[0], kap_o, rtol=1e-8, atol=1e-10 * np.abs(kap_o).max())


@pytest.mark.parametrize("kind", ["lj", "random_fc3"])
def test_large_gamma_bf16split_tensor_cores(k, big324, kind):
    """tcgen05 BF16 hi+lo path (three MMAs per product, FP32 accumulation in
    tensor memory), gamma within 1e-5 of the FP64 oracle.  The LJ system has a permutation-symmetric Phi3, so only
    the upper triangle of phi is computed; the random extra blocks break that
    symmetry and the full delta band is computed."""
    kk, ctx = k
    s, nu_o, eig_o, g_o = big324
    if kind == "random_fc3":
        s = ki.random_fc3_system(s, 400, seed=21, scale=0.02)
        g_o = an.linewidths_gamma_only(s, nu_o, eig_o, 300.0, 0.05)
    w = ki.Workload("g324", [s], (1, 1, 1), 300.0, 0.05, 3.0)
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, (1, 1, 1), nu_o, eig_o, _opts(kk, w, "bf16split"))
    g64, (_, allowed64) = kk.kald_linewidths(ctx, s, (1, 1, 1), nu_o, eig_o, _opts(kk, w, "fp64"))
    assert allowed == allowed64
    err = _rel(g, g_o, 1e-6 * g_o.max())
    print(f"bf16 split gamma max rel err {err:.3e}")
    assert err < 1e-5


def test_gamma_only_144_modes_partial_tiles_and_batch(k):
    """A 2x2x3 conventional supercell (48 atoms, 144 modes): two 128-row tiles
    per side with 112 padded columns, and a last batch of 16 modes after four
    full batches of the tensor-core path.  Eigenpairs, gamma (FP64, BF16 split)
    and the QHGK kappa against the oracle."""
    kk, ctx = k
    s = ki.fcc_supercell_system((2, 2, 3), seed=17, heavy_fraction=0.3)
    assert s.n_branches == 144
    nu_o, eig_o = ph.phonons(s, (1, 1, 1))
    g_o = an.linewidths_gamma_only(s, nu_o, eig_o, 300.0, 0.05)
    w = ki.Workload("g144", [s], (1, 1, 1), 300.0, 0.05, 3.0)
    nu, eig, _ = kk.kald_phonons(ctx, s, (1, 1, 1), want_vel=False)
    sq = lambda x: np.sign(x) * x * x
    np.testing.assert_allclose(sq(nu), sq(nu_o), atol=1e-11 * np.max(nu_o) ** 2)
    g64, (tot, allowed) = kk.kald_linewidths(ctx, s, (1, 1, 1), nu_o, eig_o, _opts(kk, w, "fp64"))
    assert tot == 144 ** 3 and 0 < allowed < tot
    assert _rel(np.ravel(g64), np.ravel(g_o), 1e-6 * g_o.max()) < 1e-10
    gbf, (_, allowed_bf) = kk.kald_linewidths(ctx, s, (1, 1, 1), nu_o, eig_o, _opts(kk, w, "bf16split"))
    assert allowed_bf == allowed
    err = _rel(np.ravel(gbf), np.ravel(g_o), 1e-6 * g_o.max())
    print(f"144 modes: bf16 split gamma max rel err {err:.3e}")
    assert err < 1e-5
    kap, _ = kk.kald_kappa_qhgk(ctx, [s], nu_o, eig_o, np.ravel(g64), _opts(kk, w))
    kap_o = co.kappa_qhgk(s, nu_o, eig_o, g_o, 300.0)
    np.testing.assert_allclose(kap[0], kap_o, rtol=1e-8, atol=1e-10 * np.abs(kap_o).max())


@pytest.mark.parametrize("precision", ["fp64", "bf16split"])
def test_batched_gamma_only_systems_match_single_calls(k, big324, precision):
    """n_sys > 1, the batched Gamma-only mode of the 24-supercell workload: two
    108-atom cells (different seeds and heavy fractions) in one call give,
    bit for bit, the gamma and triplet counts of one call per system; the
    first system is the oracle-checked cell of the tests above."""
    kk, ctx = k
    s1, nu1, eig1, g_o = big324
    s2 = ki.fcc_supercell_system(3, seed=1001, heavy_fraction=0.45)
    nu2, eig2 = ph.phonons(s2, (1, 1, 1))
    w = ki.Workload("g324x2", [s1, s2], (1, 1, 1), 300.0, 0.05, 3.0)
    opt = _opts(kk, w, precision)
    nu = np.ascontiguousarray(np.concatenate([nu1.ravel(), nu2.ravel()]))
    eig = np.ascontiguousarray(np.concatenate([eig1.ravel(), eig2.ravel()]))
    g, (tot, allowed) = kk.kald_linewidths(ctx, [s1, s2], (1, 1, 1), nu, eig, opt)
    ga, (ta, aa) = kk.kald_linewidths(ctx, s1, (1, 1, 1), nu1, eig1, opt)
    gb, (tb, ab) = kk.kald_linewidths(ctx, s2, (1, 1, 1), nu2, eig2, opt)
    np.testing.assert_array_equal(g[:324], np.ravel(ga))
    np.testing.assert_array_equal(g[324:], np.ravel(gb))
    assert tot == ta + tb == 2 * 324 ** 3 and allowed == aa + ab
    assert _rel(np.ravel(ga), np.ravel(g_o), 1e-6 * g_o.max()) < (1e-10 if precision == "fp64" else 1e-5)


def test_c3_bf16split_sampled_modes(k):
    """The 864-atom Gamma-only workload (2592 modes) on tensor cores, at full
    size in the benchmark's launch configuration, checked at sampled modes that
    are not degenerate (so the oracle's unaveraged gamma applies)."""
    kk, ctx = k
    w = ki.c3()
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "bf16split"))
    g = g.reshape(nu_o.shape)[0]
    nu0 = nu_o[0]
    modes = []
    for m in (5, 700, 1300, 1900, 2500):
        gap = min(abs(nu0[m] - nu0[m - 1]), abs(nu0[m + 1] - nu0[m]))
        if gap > 1e-4:
            modes.append(m)
    assert len(modes) >= 3
    g_o = an.linewidths_gamma_only(s, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma, modes=modes, average=False)
    g64, _ = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "fp64"))
    g64 = g64.reshape(nu_o.shape)[0]
    for m, go in zip(modes, g_o):
        print(f"mode {m}: nu {nu0[m]:.5f} THz, oracle {go:.9e}, bf16 {g[m]:.9e}, fp64 {g64[m]:.9e}")
    err = np.max(np.abs(g[modes] - g_o) / np.abs(g_o))
    print(f"C3 bf16 split gamma max rel err {err:.3e} at modes {modes}")
    assert err < 1e-5
    assert tot == 2592 ** 3 and 0 < allowed < tot
    # kappa_QHGK at full size: the GPU's S8/S9 against the oracle's on the same
    # (FP64 GPU) linewidths, and the split path's kappa against the FP64 one
    kap64, _ = kk.kald_kappa_qhgk(ctx, [s], nu_o, eig_o, g64, _opts(kk, w, "fp64"))
    kap_o = co.kappa_qhgk(s, nu_o, eig_o, g64, w.T)
    np.testing.assert_allclose(kap64[0], kap_o, rtol=1e-10, atol=1e-12 * np.abs(kap_o).max())
    kapbf, _ = kk.kald_kappa_qhgk(ctx, [s], nu_o, eig_o, np.ascontiguousarray(g), _opts(kk, w, "bf16split"))
    errk = np.max(np.abs(kapbf[0] - kap64[0])) / np.max(np.abs(kap64[0]))
    print(f"C3 kappa_QHGK split vs fp64 rel err {errk:.3e}")
    assert errk < 1e-4


def test_c5_full_mesh_sampled_q(k):
    """The 2-atom / 24^3 workload (13824 q-points) in the benchmark's launch
    configuration (the FP32 register kernel behind the BF16-split request),
    checked at sampled q-points against the oracle."""
    kk, ctx = k
    w = ki.c5()
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "bf16split"))
    g = g.reshape(nu_o.shape)
    qs = [1, 5000]
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma, q_list=qs)
    err = _rel(g[qs], g_o, 1e-6 * g_o.max())
    print(f"C5 gamma max rel err {err:.3e}")
    assert err < 1e-5
    assert tot == 13824 ** 2 * 6 ** 3 and 0 < allowed < tot


@pytest.mark.parametrize("cell", ["binary", "fcc4", "fcc32"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16split"])
def test_no_third_order_blocks_gives_zero_gamma(k, cell, precision):
    """Degenerate input: without Phi3 blocks every projection vanishes, so
    gamma is exactly zero in every path (register kernel for the 2-atom cell,
    CUDA cores for the 4-atom cell, tensor cores or CUDA cores for the 32-atom
    cell), while the delta-allowed count, which depends on the frequencies
    only, is unchanged."""
    kk, ctx = k
    if cell == "binary":
        w = ki.small_binary(mesh=(3, 3, 3), sigma=0.1)
        base = w.systems[0]
    else:
        w = _cell_case("fcc4_mesh3" if cell == "fcc4" else "fcc32_mesh211")
        base = w.systems[0]
    empty = ki.System(base.masses.copy(), base.positions.copy(), base.lattice.copy(),
                      base.fc2_idx.copy(), base.fc2.copy(), np.zeros((0, 9), dtype=np.int32),
                      np.zeros((0, 3, 3, 3)), name=base.name + "_no_fc3")
    nu_o, eig_o = ph.phonons(base, w.mesh)
    g0, (tot0, al0) = kk.kald_linewidths(ctx, empty, w.mesh, nu_o, eig_o, _opts(kk, w, precision))
    _, (tot1, al1) = kk.kald_linewidths(ctx, base, w.mesh, nu_o, eig_o, _opts(kk, w, precision))
    assert np.all(g0 == 0.0)
    assert tot0 == tot1 and al0 == al1 > 0


@pytest.mark.parametrize("case", ["C2_mesh4", "C5_mesh8"])
def test_kappa_split_path_against_fp64_gpu_path(k, case):
    """kappa time-to-solution path: the BF16-split linewidths give kappa_RTA
    within 1e-4 (relative to the largest component) of the plain FP64 GPU
    path on the same GB300; both timings are printed."""
    import time
    kk, ctx = k
    if case == "C2_mesh4":
        w = ki.c2()
        w.mesh = (4, 4, 4)
    else:
        w = ki.c5(mesh=(8, 8, 8))
    s = w.systems[0]
    nu, eig = kk.kald_phonons(ctx, s, w.mesh)[:2]
    kap = {}
    for prec in ("fp64", "bf16split"):
        t0 = time.perf_counter()
        g, _ = kk.kald_linewidths(ctx, s, w.mesh, nu, eig, _opts(kk, w, prec))
        kap[prec] = kk.kald_kappa_rta(ctx, s, w.mesh, nu, eig, g, _opts(kk, w, prec))
        print(f"{case} {prec}: linewidths + kappa {time.perf_counter() - t0:.3f} s, "
              f"kappa_xx {kap[prec][0][0]:.6e}")
    a, b = np.asarray(kap["bf16split"]), np.asarray(kap["fp64"])
    err = np.max(np.abs(a - b)) / np.max(np.abs(b))
    print(f"{case}: kappa split vs fp64 rel err {err:.3e}")
    assert err < 1e-4


# ---------------------------------------------------------------- classical statistics
@pytest.mark.parametrize("case,precision", [("binary3", "fp64"), ("fcc4_mesh3", "bf16split"),
                                            ("fcc32_mesh311", "bf16split"), ("gamma_only_32", "fp64")])
def test_classical_statistics_match_oracle(k, case, precision):
    """classical = 1 (Eq. classic_n: n = kB T / hbar omega, c = kB) through the
    linewidths and kappa_RTA / kappa_QHGK, against the oracle run with the same
    statistics."""
    kk, ctx = k
    w = _cell_case(case) if case.startswith("fcc") else _lw_case(case)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    opt = _opts(kk, w, precision, classical=True)
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma, classical=True)
    g_q = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    assert np.max(np.abs(g_o - g_q)) > 1e-3 * g_q.max()      # the statistics matter here
    g, _ = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, opt)
    g = g.reshape(g_o.shape)
    err = _rel(g, g_o, 1e-6 * g_o.max())
    print(f"{case} classical {precision}: gamma rel err {err:.2e}")
    assert err < (1e-10 if precision == "fp64" else 1e-5)
    if w.n_q == 1:
        kap, _ = kk.kald_kappa_qhgk(ctx, [s], nu_o, eig_o, np.ravel(g_o), opt)
        kap_o = co.kappa_qhgk(s, nu_o, eig_o, np.ravel(g_o), w.T, classical=True)
        kap = kap[0]
    else:
        kap = kk.kald_kappa_rta(ctx, s, w.mesh, nu_o, eig_o, np.ravel(g_o), opt)
        kap_o = co.kappa_rta(s, w.mesh, nu_o, eig_o, g_o, w.T, classical=True)
    np.testing.assert_allclose(kap, kap_o, rtol=1e-10, atol=1e-12 * np.abs(kap_o).max())


# ---------------------------------------------------------------- the batched Gamma-only workload
@pytest.fixture(scope="module")
def c4w():
    """The 24 supercells of the batched Gamma-only workload (8 each of 108,
    256 and 500 atoms) with the oracle's phonons."""
    w = ki.c4()
    ph_all = [ph.phonons(s, (1, 1, 1)) for s in w.systems]
    return w, ph_all


def _sample_modes(nu0, picks, gap=1e-4):
    out = []
    for m in picks:
        if nu0[m] > 0.05 and min(abs(nu0[m] - nu0[m - 1]), abs(nu0[m + 1] - nu0[m])) > gap:
            out.append(m)
    return out


@pytest.mark.parametrize("which", [8, 16])
def test_c4_768_and_1500_mode_linewidths_sampled(k, c4w, which):
    """The 256- and 500-atom supercells of the batched workload (768 and 1500
    modes; the tensor-core path runs several modes per launch with 6 and 12
    tiles per side): gamma in FP64 and BF16 split against the oracle at
    sampled non-degenerate modes."""
    kk, ctx = k
    w, ph_all = c4w
    s = w.systems[which]
    nu_o, eig_o = ph_all[which]
    nb = s.n_branches
    modes = _sample_modes(nu_o[0], [7, nb // 5, nb // 2, (4 * nb) // 5, nb - 3])
    assert len(modes) >= 3
    g_o = an.linewidths_gamma_only(s, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma, modes=modes,
                                   average=False)
    for prec, tol in (("fp64", 1e-10), ("bf16split", 1e-5)):
        g, (tot, allowed) = kk.kald_linewidths(ctx, s, (1, 1, 1), nu_o, eig_o, _opts(kk, w, prec))
        g = np.ravel(g)
        err = np.max(np.abs(g[modes] - g_o) / np.abs(g_o))
        print(f"{nb} modes {prec}: gamma max rel err {err:.3e} at modes {modes}")
        assert err < tol
        assert tot == nb ** 3 and 0 < allowed < tot


def test_c4_full_batch_one_call_sampled(k, c4w):
    """All 24 supercells in one kald_linewidths call (BF16 split, the
    benchmark's configuration), checked at sampled modes of one system of each
    size against the oracle."""
    kk, ctx = k
    w, ph_all = c4w
    nu = np.ascontiguousarray(np.concatenate([p[0].ravel() for p in ph_all]))
    eig = np.ascontiguousarray(np.concatenate([p[1].ravel() for p in ph_all]))
    g, (tot, allowed) = kk.kald_linewidths(ctx, w.systems, (1, 1, 1), nu, eig, _opts(kk, w, "bf16split"))
    nbs = [s.n_branches for s in w.systems]
    assert tot == sum(b ** 3 for b in nbs) and 0 < allowed < tot
    offs = np.cumsum([0] + nbs)
    for x in (3, 11, 19):
        s = w.systems[x]
        nu_o, eig_o = ph_all[x]
        modes = _sample_modes(nu_o[0], [9, nbs[x] // 3, (2 * nbs[x]) // 3])
        g_o = an.linewidths_gamma_only(s, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma, modes=modes,
                                       average=False)
        gx = g[offs[x]:offs[x + 1]]
        err = np.max(np.abs(gx[modes] - g_o) / np.abs(g_o))
        print(f"system {x} ({nbs[x]} modes): gamma max rel err {err:.3e} at modes {modes}")
        assert err < 1e-5


def test_qhgk_kappa_split_path_against_oracle(k, big324):
    """kappa_QHGK from the BF16-split linewidths within 1e-4 of the oracle's
    kappa_QHGK from the oracle's FP64 linewidths (108-atom supercell)."""
    kk, ctx = k
    s, nu_o, eig_o, g_o = big324
    w = ki.Workload("g324", [s], (1, 1, 1), 300.0, 0.05, 3.0)
    g, _ = kk.kald_linewidths(ctx, s, (1, 1, 1), nu_o, eig_o, _opts(kk, w, "bf16split"))
    kap, _ = kk.kald_kappa_qhgk(ctx, [s], nu_o, eig_o, np.ravel(g), _opts(kk, w, "bf16split"))
    kap_o = co.kappa_qhgk(s, nu_o, eig_o, np.ravel(g_o), 300.0)
    err = np.max(np.abs(kap[0] - kap_o)) / np.max(np.abs(kap_o))
    print(f"324 modes: kappa_QHGK split vs oracle rel err {err:.3e}")
    assert err < 1e-4


def test_c2_kappa_split_vs_fp64_gpu_full_mesh(k):
    """The metric's second half on the full 32-atom / 8^3 workload: kappa_RTA
    from the BF16-split linewidths within 1e-4 of kappa_RTA from the plain
    FP64 GPU linewidths (same GPU phonons); both times printed."""
    import time
    kk, ctx = k
    w = ki.c2()
    s = w.systems[0]
    nu, eig = kk.kald_phonons(ctx, s, w.mesh, want_vel=False)[:2]
    kap, secs = {}, {}
    for prec in ("bf16split", "fp64"):
        t0 = time.perf_counter()
        g, _ = kk.kald_linewidths(ctx, s, w.mesh, nu, eig, _opts(kk, w, prec))
        kap[prec] = kk.kald_kappa_rta(ctx, s, w.mesh, nu, eig, g, _opts(kk, w, prec))
        secs[prec] = time.perf_counter() - t0
    a, b = np.asarray(kap["bf16split"]), np.asarray(kap["fp64"])
    err = np.max(np.abs(a - b)) / np.max(np.abs(b))
    print(f"C2 8^3: linewidths + kappa fp64 {secs['fp64']:.2f} s, split {secs['bf16split']:.2f} s, "
          f"kappa rel err {err:.3e}, kappa_xx {b[0][0]:.6e}")
    assert err < 1e-4


# ---------------------------------------------------------------- q ranges (the multi-GPU unit of work)
@pytest.mark.parametrize("case,precision", [("binary3", "fp32"), ("binary3", "fp64"),
                                            ("fcc4_mesh3", "fp64"), ("fcc4_mesh3", "bf16split"),
                                            ("fcc32_mesh2", "bf16split")])
def test_qrange_calls_concatenate_to_the_full_call(k, case, precision):
    """kald_linewidths_qrange over a partition of the mesh into uneven
    contiguous ranges, run back to back on the one GPU, gives the full call's
    gamma and triplet counts bit for bit (register, CUDA-core and tensor-core
    crystal paths; the full call with time reversal as its only symmetry, as
    the range calls)."""
    kk, ctx = k
    if case == "fcc4_mesh3":
        w = ki.Workload("fcc4", [ki.fcc_supercell_system(1, seed=7)], (3, 3, 3), 300.0, 0.1, 3.0)
    elif case == "fcc32_mesh2":
        w = ki.Workload("fcc32", [ki.fcc_supercell_system(2, seed=2)], (2, 2, 2), 300.0, 0.1, 3.0)
    else:
        w = _lw_case(case)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    opt = _opts(kk, w, precision, symmetry="inversion")   # the symmetry range calls use
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, opt)
    nq = w.n_q
    cuts = sorted({0, nq, max(1, nq // 5), max(1, (2 * nq) // 3)})
    parts, t_sum, a_sum = [], 0, 0
    for a, b in zip(cuts[:-1], cuts[1:]):
        gp, (t, al) = kk.kald_linewidths_qrange(ctx, s, w.mesh, nu_o, eig_o, opt, a, b)
        parts.append(gp)
        t_sum += t
        a_sum += al
    np.testing.assert_array_equal(np.concatenate(parts), np.ravel(g))
    assert t_sum == tot and a_sum == allowed
    with pytest.raises(kk.KaldError) as e:
        kk.kald_linewidths_qrange(ctx, s, w.mesh, nu_o, eig_o, opt, 2, 2)
    assert e.value.status == 1


# ---------------------------------------------------------------- time reversal: one projection per {q, -q}
def _tr_case(case):
    if case == "fcc4_mesh3":
        return ki.Workload("fcc4", [ki.fcc_supercell_system(1, seed=7)], (3, 3, 3), 300.0, 0.1, 3.0)
    if case == "fcc32_mesh331":
        return ki.Workload("fcc32", [ki.fcc_supercell_system(2, seed=2)], (3, 3, 1), 300.0, 0.1, 3.0)
    return _lw_case(case)


@pytest.mark.parametrize("case,precision,tol", [("binary3", "fp64", 1e-12), ("binary_random", "fp64", 1e-12),
                                                ("binary3", "fp32", 2e-6), ("fcc4_mesh3", "fp64", 1e-12),
                                                ("fcc4_mesh3", "fp32", 2e-6), ("fcc32_mesh331", "bf16split", 1e-5)])
def test_inversion_reuse_matches_projecting_every_q(k, case, precision, tol):
    """By default kald_linewidths projects one q-point of each pair {q, -q}
    and gives -q the averaged linewidths of q (Phi3 real: phi(-q, -q', -q'') is
    the conjugate of phi(q, q', q''), w(-q) = w(q)).  Projecting every q-point
    (symmetry "none") gives the same gamma: to rounding in FP64 (also for a random,
    non-symmetric Phi3), within the path's own error in FP32 and the BF16
    split; both agree with the oracle, and the delta-allowed counts agree."""
    kk, ctx = k
    w = _tr_case(case)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_r, (tot_r, al_r) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, precision))
    g_a, (tot_a, al_a) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, precision, symmetry="none"))
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    floor = 1e-6 * g_o.max()
    assert tot_r == tot_a
    assert abs(al_r - al_a) <= 1e-6 * al_a
    assert _rel(g_r.reshape(g_o.shape), g_a.reshape(g_o.shape), floor) < tol
    bar = 1e-10 if precision == "fp64" else 1e-5
    assert _rel(g_r.reshape(g_o.shape), g_o, floor) < bar
    assert _rel(g_a.reshape(g_o.shape), g_o, floor) < bar
    # gamma(-q) = gamma(q) on the reusing call (the same sums; each q-point
    # divides by its own w, equal to that of -q up to the phonons' rounding)
    nq = w.n_q
    m = w.mesh
    gr = g_r.reshape(nq, -1)
    for q in range(nq):
        k0, k1, k2 = q // (m[1] * m[2]), (q // m[2]) % m[1], q % m[2]
        qn = (((m[0] - k0) % m[0]) * m[1] + (m[1] - k1) % m[1]) * m[2] + (m[2] - k2) % m[2]
        np.testing.assert_allclose(gr[q], gr[qn], rtol=1e-12, atol=0.0)


@pytest.mark.parametrize("mesh", [(3, 3, 1), (2, 2, 2), (4, 2, 1), (3, 1, 1)])
def test_orbit_projections_match_every_pair(k, mesh):
    """The BF16-split tensor path with Phi3 symmetric under permutations (a
    pair potential) projects one momentum triple per orbit under permutations
    and inversion and feeds all three members' linewidths (the orbit sums are
    formed in a fixed order); gamma agrees with time reversal only, with every
    pair projected, and with the FP64 oracle (1e-5), and the delta-allowed
    counts agree within the rounding of window edges.  Meshes with
    self-inverse points (2q = 0), repeated members (q1 = q2) and orbits of
    every size."""
    kk, ctx = k
    w = ki.Workload("fcc32", [ki.fcc_supercell_system(2, seed=2)], mesh, 300.0, 0.1, 3.0)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    floor = 1e-6 * g_o.max()
    out = {}
    for sym in ("all", "inversion", "none"):
        g, (tot, al) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "bf16split", symmetry=sym))
        out[sym] = (g.reshape(g_o.shape), tot, al)
        err = _rel(out[sym][0], g_o, floor)
        print(f"{mesh} {sym}: gamma max rel err {err:.3e}, allowed {al}")
        assert err < 1e-5
        assert tot == w.n_q ** 2 * s.n_branches ** 3
    assert abs(out["all"][2] - out["none"][2]) <= 1e-5 * out["none"][2]
    assert _rel(out["all"][0], out["none"][0], floor) < 1e-5
    assert np.all(out["all"][0][nu_o <= 0.01] == 0.0)


def test_orbit_projections_need_a_symmetric_phi3(k):
    """With Phi3 not symmetric under permutations (random extra blocks), the
    default symmetry setting falls back to time reversal: the result equals
    the symmetry="inversion" call bit for bit and the oracle within 1e-5."""
    kk, ctx = k
    w = _cell_case("fcc32_random")
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_a, c_a = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "bf16split"))
    g_i, c_i = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, "bf16split", symmetry="inversion"))
    np.testing.assert_array_equal(g_a, g_i)
    assert c_a == c_i
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    assert _rel(g_a.reshape(g_o.shape), g_o, 1e-6 * g_o.max()) < 1e-5


@pytest.mark.parametrize("case,precision", [("binary3", "fp64"), ("binary3", "fp32"), ("fcc4_mesh3", "fp64"),
                                            ("fcc32_mesh331", "bf16split")])
def test_qlist_rows_equal_the_full_call(k, case, precision):
    """kald_linewidths_qlist on a shuffled list with repeats, lone members of
    pairs {q, -q} and whole pairs returns, row by row, the gamma of the full
    call with time reversal as its only symmetry bit for bit; the triplet counts add up over a partition of the mesh into
    lists; an entry outside the mesh is refused."""
    kk, ctx = k
    w = _tr_case(case)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    opt = _opts(kk, w, precision, symmetry="inversion")   # the symmetry list calls use
    g, (tot, allowed) = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, opt)
    nq = w.n_q
    g = g.reshape(nq, -1)
    rng = np.random.default_rng(5)
    ql = list(rng.permutation(nq)[: max(1, nq // 2)]) + [0, nq - 1, nq - 1]
    gl, (t, _) = kk.kald_linewidths_qlist(ctx, s, w.mesh, nu_o, eig_o, opt, ql)
    np.testing.assert_array_equal(gl.reshape(len(ql), -1), g[ql])
    assert t == len(ql) * nq * g.shape[1] ** 3
    perm = rng.permutation(nq)
    parts = [perm[: nq // 3], perm[nq // 3:]]
    t_sum = a_sum = 0
    for part in parts:
        gp, (tp, ap) = kk.kald_linewidths_qlist(ctx, s, w.mesh, nu_o, eig_o, opt, part)
        np.testing.assert_array_equal(gp.reshape(len(part), -1), g[part])
        t_sum += tp
        a_sum += ap
    assert t_sum == tot and a_sum == allowed
    with pytest.raises(kk.KaldError) as e:
        kk.kald_linewidths_qlist(ctx, s, w.mesh, nu_o, eig_o, opt, [0, nq])
    assert e.value.status == 1


# ---------------------------------------------------------------- batched Gamma-only calls
def test_phonons_batch_equals_one_call_per_system(k, c4w):
    """kald_phonons_batch over supercells of 108, 256 and 500 atoms (and a
    32-atom cell that takes the per-q solver) gives, bit for bit, the
    eigenpairs of one kald_phonons call per system."""
    kk, ctx = k
    w, _ = c4w
    systems = [w.systems[0], w.systems[9], ki.fcc_supercell_system(2, seed=5), w.systems[17], w.systems[1]]
    nu_b, eig_b = kk.kald_phonons_batch(ctx, systems)
    o_m, o_e = 0, 0
    for s in systems:
        nb = s.n_branches
        nu1, eig1, _ = kk.kald_phonons(ctx, s, (1, 1, 1), want_vel=False)
        np.testing.assert_array_equal(nu_b[o_m:o_m + nb], np.ravel(nu1))
        np.testing.assert_array_equal(eig_b[o_e:o_e + nb * nb], np.ravel(eig1))
        o_m += nb
        o_e += nb * nb


@pytest.mark.parametrize("precision", ["fp64", "bf16split"])
def test_batched_mixed_sizes_match_single_calls(k, c4w, precision):
    """One kald_linewidths and one kald_kappa_qhgk call over supercells of 324,
    768 and 1500 modes (the sizes of the batched workload, dealt over
    concurrent streams) equal one call per system bit for bit."""
    kk, ctx = k
    w, ph_all = c4w
    pick = [2, 10, 18] if precision == "bf16split" else [2, 10]
    systems = [w.systems[x] for x in pick]
    opt = _opts(kk, w, precision)
    nu = np.ascontiguousarray(np.concatenate([ph_all[x][0].ravel() for x in pick]))
    eig = np.ascontiguousarray(np.concatenate([ph_all[x][1].ravel() for x in pick]))
    g, (tot, allowed) = kk.kald_linewidths(ctx, systems, (1, 1, 1), nu, eig, opt)
    kap, _ = kk.kald_kappa_qhgk(ctx, systems, nu, eig, g, opt)
    o, t_sum, a_sum = 0, 0, 0
    for j, x in enumerate(pick):
        nb = w.systems[x].n_branches
        g1, (t1, a1) = kk.kald_linewidths(ctx, w.systems[x], (1, 1, 1), ph_all[x][0], ph_all[x][1], opt)
        np.testing.assert_array_equal(g[o:o + nb], np.ravel(g1))
        k1, _ = kk.kald_kappa_qhgk(ctx, [w.systems[x]], ph_all[x][0], ph_all[x][1], np.ravel(g1), opt)
        np.testing.assert_array_equal(kap[j], k1[0])
        t_sum += t1
        a_sum += a1
        o += nb
    assert tot == t_sum and allowed == a_sum


# ---------------------------------------------------------------- delta shapes
@pytest.mark.parametrize("shape", ["lorentzian", "triangular"])
@pytest.mark.parametrize("case,precision", [("binary3", "fp64"), ("binary3", "fp32"), ("fcc4_mesh3", "fp64"),
                                            ("fcc4_mesh3", "bf16split"), ("fcc32_mesh211", "bf16split"),
                                            ("g144", "fp64"), ("g144", "bf16split")])
def test_delta_shapes_match_oracle(k, case, precision, shape):
    """The Lorentzian and triangular energy deltas (delta_shape option) in
    every epilogue -- register, CUDA-core, crystal and Gamma-only tensor-core
    -- against the oracle with the same shape."""
    kk, ctx = k
    if case.startswith("fcc"):
        w = _cell_case(case)
    elif case == "g144":
        s = ki.fcc_supercell_system((2, 2, 3), seed=17, heavy_fraction=0.3)
        w = ki.Workload("g144", [s], (1, 1, 1), 300.0, 0.05, 3.0)
    else:
        w = _lw_case(case)
    s = w.systems[0]
    nu_o, eig_o = ph.phonons(s, w.mesh)
    if w.n_q == 1:
        g_o = an.linewidths_gamma_only(s, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma, delta=shape)
    else:
        g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma, delta=shape)
    g, _ = kk.kald_linewidths(ctx, s, w.mesh, nu_o, eig_o, _opts(kk, w, precision, delta=shape))
    err = _rel(np.ravel(g), np.ravel(g_o), 1e-6 * np.max(g_o))
    print(f"{case} {precision} {shape}: gamma rel err {err:.2e}")
    assert err < (1e-10 if precision == "fp64" else 1e-5)


# ---------------------------------------------------------------- phase space and diffusivity
@pytest.mark.parametrize("case,precision,shape", [("binary3", "fp64", "gaussian"), ("binary3", "fp32", "gaussian"),
                                                  ("fcc4_mesh4", "fp64", "gaussian"),
                                                  ("fcc4_mesh4", "fp32", "lorentzian"),
                                                  ("binary3", "fp64", "triangular")])
def test_phase_space_matches_oracle(k, case, precision, shape):
    """kald_phase_space (the weights of the linewidths without matrix elements)
    against the oracle's phase space; the oracle forms the - process with
    q'' = q - q', the GPU with q'' = q + q' and w(-q') = w(q'), equal up to the
    rounding of the two frequencies."""
    kk, ctx = k
    if case == "fcc4_mesh4":
        w = ki.Workload("fcc4", [ki.fcc_supercell_system(1, seed=7)], (4, 4, 4), 300.0, 0.1, 3.0)
    else:
        w = _lw_case(case)
    s = w.systems[0]
    nu_o, _ = ph.phonons(s, w.mesh)
    g_o = an.phase_space(w.mesh, nu_o, w.T, w.sigma_thz, w.n_sigma, delta=shape)
    g = kk.kald_phase_space(ctx, s, w.mesh, nu_o, _opts(kk, w, precision, delta=shape))
    err = _rel(g.reshape(g_o.shape), g_o, 1e-6 * g_o.max())
    print(f"{case} {precision} {shape}: phase space rel err {err:.2e}")
    assert err < (1e-9 if precision == "fp64" else 1e-5)
    assert np.all(g.reshape(g_o.shape)[nu_o <= 0.01] == 0.0)


def test_diffusivity_matches_oracle_and_the_classical_trace_identity(k, big324):
    """kald_diffusivity against the oracle (108-atom supercell), and the
    identity tr(kappa_QHGK)/3 = kB/V sum_mu D_mu of the GPU's own classical
    kappa_QHGK and diffusivities."""
    kk, ctx = k
    s, nu_o, eig_o, g_o = big324
    w = ki.Workload("g324", [s], (1, 1, 1), 300.0, 0.05, 3.0)
    g = np.ravel(g_o)
    D = kk.kald_diffusivity(ctx, [s], nu_o, eig_o, g, _opts(kk, w))
    D_o = co.diffusivity(s, nu_o, eig_o, g)
    np.testing.assert_allclose(D, D_o, rtol=1e-10, atol=1e-12 * np.abs(D_o).max())
    kap, _ = kk.kald_kappa_qhgk(ctx, [s], nu_o, eig_o, g, _opts(kk, w, classical=True))
    kb = 1.380649e-23
    lhs = np.trace(kap[0]) / 3.0
    rhs = kb / s.volume * np.sum(D) * co.KAPPA_SI
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


# ---------------------------------------------------------------- large-system QHGK options
@pytest.mark.parametrize("bandwidth,threshold", [(0.2, 0.0), (0.0, 0.5), (0.3, 1.0)])
def test_qhgk_bandwidth_and_threshold_match_oracle(k, big324, bandwidth, threshold):
    """The Allen-Feldman bandwidth and the threshold on tau (QHGK options) in
    kald_kappa_qhgk and kald_diffusivity against the oracle."""
    kk, ctx = k
    s, nu_o, eig_o, g_o = big324
    w = ki.Workload("g324", [s], (1, 1, 1), 300.0, 0.05, 3.0)
    g = np.ravel(g_o)
    opt = _opts(kk, w, qhgk_bandwidth_thz=bandwidth, qhgk_threshold_thz=threshold)
    kw = dict(bandwidth_thz=bandwidth or None, threshold_thz=threshold or None)
    kap, _ = kk.kald_kappa_qhgk(ctx, [s], nu_o, eig_o, g, opt)
    kap_o = co.kappa_qhgk(s, nu_o, eig_o, g, 300.0, **kw)
    np.testing.assert_allclose(kap[0], kap_o, rtol=1e-10, atol=1e-12 * np.abs(kap_o).max())
    D = kk.kald_diffusivity(ctx, [s], nu_o, eig_o, g, opt)
    D_o = co.diffusivity(s, nu_o, eig_o, g, **kw)
    np.testing.assert_allclose(D, D_o, rtol=1e-10, atol=1e-12 * np.abs(D_o).max())


def test_interpolate_gamma_matches_oracle(k, big324, c4w):
    """gamma(nu) of the 108-atom cell spline-interpolated onto the frequencies
    of a 500-atom cell, against the oracle's scipy spline; and a cubic gamma(nu)
    reproduced exactly."""
    kk, ctx = k
    s, nu_o, eig_o, g_o = big324
    w, ph_all = c4w
    nu_dst = np.ascontiguousarray(ph_all[16][0].ravel())
    opt = _opts(kk, ki.Workload("g", [s], (1, 1, 1), 300.0, 0.05, 3.0))
    g_dst = kk.kald_interpolate_gamma(ctx, np.ascontiguousarray(nu_o.ravel()), np.ascontiguousarray(np.ravel(g_o)),
                                      nu_dst, opt)
    ref = co.interpolate_gamma(nu_o.ravel(), np.ravel(g_o), nu_dst)
    np.testing.assert_allclose(g_dst, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    x = np.linspace(0.3, 9.0, 57)
    cubic = lambda v: 0.05 + 0.01 * v - 0.002 * v ** 2 + 0.0003 * v ** 3
    xq = np.linspace(0.3, 9.0, 201)
    np.testing.assert_allclose(kk.kald_interpolate_gamma(ctx, x, cubic(x), xq, opt), cubic(xq), rtol=1e-11)


# ---------------------------------------------------------------- finite-difference force constants
def test_fd_force_constants_match_oracle_and_feed_the_path(k):
    """kald_fd_force_constants (Lennard-Jones, h = 1e-3 A) against the oracle's
    finite differences, and the linewidths of the finite-difference system
    against those of the analytic one (O(h^2) apart)."""
    from oracle import ifc
    kk, ctx = k
    w = ki.small_binary(mesh=(3, 3, 3), sigma=0.1)
    s = w.systems[0]
    h = 1e-3
    f2, f3 = kk.kald_fd_force_constants(ctx, s, ki.LJ_EPSILON, ki.LJ_SIGMA, ki.LJ_CUTOFF, h)
    o2, o3 = ifc.fd_force_constants(s, h=h)
    e2 = np.abs(f2 - o2).max() / np.abs(o2).max()
    e3 = np.abs(f3 - o3).max() / np.abs(o3).max()
    a2 = np.abs(f2 - s.fc2).max() / np.abs(s.fc2).max()
    a3 = np.abs(f3 - s.fc3).max() / np.abs(s.fc3).max()
    print(f"FD vs oracle FD: fc2 {e2:.1e}, fc3 {e3:.1e}; FD vs analytic: fc2 {a2:.1e}, fc3 {a3:.1e}")
    assert e2 < 1e-9 and e3 < 1e-8
    assert a2 < 1e-5 and a3 < 1e-4
    fd = ki.System(s.masses.copy(), s.positions.copy(), s.lattice.copy(), s.fc2_idx.copy(), f2,
                   s.fc3_idx.copy(), f3, name="binary_fd")
    nu, eig, _ = kk.kald_phonons(ctx, fd, w.mesh)
    g, _ = kk.kald_linewidths(ctx, fd, w.mesh, nu, eig, _opts(kk, w))
    nu_a, eig_a, _ = kk.kald_phonons(ctx, s, w.mesh)
    g_a, _ = kk.kald_linewidths(ctx, s, w.mesh, nu_a, eig_a, _opts(kk, w))
    err = _rel(np.ravel(g), np.ravel(g_a), 1e-6 * np.max(g_a))
    print(f"linewidths from FD force constants vs analytic: {err:.1e}")
    assert err < 1e-3
