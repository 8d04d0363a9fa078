"""Failure detection without a GPU fault.

* Every wait inside the tensor-core pipelines is bounded.  A test shortens
  the pipeline waits to one poll (kald_set_wait_limit), so that they run out
  while the copies and MMAs they wait for are still in flight: the call must
  return KALD_E_TIMEOUT (the kernels wind down: issued copies and committed
  MMAs finish, tensor memory is freed), and the same context must then give
  correct linewidths with the default limit.
* A capped workspace (kald_set_workspace_limit) makes a call that needs more
  return KALD_E_NOMEM without allocating, and the context works again once
  the cap is lifted.
Nothing here faults, traps or hangs the GPU: the waits end by their own limit.
"""

import numpy as np
import pytest

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import phonons as ph

pytestmark = pytest.mark.gpu

KALD_E_NOMEM, KALD_E_TIMEOUT = 2, 5


@pytest.fixture(scope="module")
def k():
    from paper_2009_01967_gb300 import build
    build.build()
    import paper_2009_01967_gb300 as kk
    ctx = kk.Context(0)
    yield kk, ctx
    ctx.close()


def _rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-6 * np.abs(b).max()))


@pytest.mark.parametrize("case", ["crystal_fcc32_mesh2", "gamma_only_144"])
def test_pipeline_wait_timeout_is_reported_and_the_context_recovers(k, case):
    kk, ctx = k
    if case == "crystal_fcc32_mesh2":
        s = ki.fcc_supercell_system(2, seed=2)                 # 96 branches: tcgen05 crystal path
        mesh = (2, 2, 2)
    else:
        s = ki.fcc_supercell_system((2, 2, 3), seed=17, heavy_fraction=0.3)   # 144 modes: Gamma-only tcgen05
        mesh = (1, 1, 1)
    nu, eig = ph.phonons(s, mesh)
    opt = kk.Options(temperature_K=300.0, sigma_thz=0.1, n_sigma=3.0, precision="bf16split")
    ctx.set_wait_limit(1)
    try:
        with pytest.raises(kk.KaldError) as e:
            kk.kald_linewidths(ctx, s, mesh, nu, eig, opt)
        assert e.value.status == KALD_E_TIMEOUT
        print(f"{case}: {e.value}")
    finally:
        ctx.set_wait_limit(0)
    g, _ = kk.kald_linewidths(ctx, s, mesh, nu, eig, opt)
    if mesh == (1, 1, 1):
        g_o = an.linewidths_gamma_only(s, nu, eig, 300.0, 0.1, 3.0)
    else:
        g_o = an.linewidths(s, mesh, nu, eig, 300.0, 0.1, 3.0)
    assert _rel(np.ravel(g), np.ravel(g_o)) < 1e-5


def test_workspace_cap_gives_nomem_and_the_context_recovers(k):
    kk, ctx = k
    w = ki.small_binary(mesh=(4, 4, 4), sigma=0.1)
    s = w.systems[0]
    opt = kk.Options(temperature_K=w.T, sigma_thz=w.sigma_thz, n_sigma=w.n_sigma)
    ctx.set_workspace_limit(4096)
    try:
        for call in ("phonons", "linewidths"):
            with pytest.raises(kk.KaldError) as e:
                if call == "phonons":
                    kk.kald_phonons(ctx, s, w.mesh)
                else:
                    nu0, eig0 = ph.phonons(s, w.mesh)
                    kk.kald_linewidths(ctx, s, w.mesh, nu0, eig0, opt)
            assert e.value.status == KALD_E_NOMEM
            assert "limit" in str(e.value)
    finally:
        ctx.set_workspace_limit(0)
    nu, eig, _ = kk.kald_phonons(ctx, s, w.mesh)
    g, _ = kk.kald_linewidths(ctx, s, w.mesh, nu, eig, opt)
    nu_o, eig_o = ph.phonons(s, w.mesh)
    g_o = an.linewidths(s, w.mesh, nu_o, eig_o, w.T, w.sigma_thz, w.n_sigma)
    assert _rel(g.reshape(g_o.shape), g_o) < 1e-9
