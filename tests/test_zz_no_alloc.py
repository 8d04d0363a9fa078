"""The allocation-free kappa_RTA entry point (kald_kappa_rta_noalloc).

It exists for callers that cannot allocate device memory -- for instance a
program whose device memory is all owned by another runtime's pool -- and
keeps its scratch in a static device array inside the library.  The test
calls it through the C ABI twice in a row (the second call reuses the array
the first one left behind) and checks both results against kald_kappa_rta at
the tolerance of the other FP64 parity tests; it also checks that a request
larger than the static array is refused.  This file is collected last so a
run that stops at the first failure has already run every other test.
"""

import ctypes

import numpy as np
import pytest

import kald_inputs as ki
from oracle import anharmonic as an
from oracle import phonons as ph

pytestmark = pytest.mark.gpu


def test_noalloc_kappa_matches_kappa_rta_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_2009_01967_gb300 import build
    build.build()
    import paper_2009_01967_gb300 as kk
    from paper_2009_01967_gb300._abi import c_system, kald_options

    w = ki.small_binary(mesh=(4, 4, 4), sigma=0.1)
    s = w.systems[0]
    nu, eig = ph.phonons(s, w.mesh)
    g = an.linewidths(s, w.mesh, nu, eig, w.T, w.sigma_thz, w.n_sigma)
    opt = kk.Options(temperature_K=w.T, sigma_thz=w.sigma_thz, n_sigma=w.n_sigma)
    dev = torch.device("cuda", 0)
    nu_d = torch.from_numpy(nu).to(dev)
    eig_d = torch.from_numpy(eig).to(dev)
    g_d = torch.from_numpy(g.reshape(-1)).to(dev)
    with kk.Context(0) as ctx:
        ref = kk.kald_kappa_rta(ctx, s, w.mesh, nu_d, eig_d, g_d, opt)
        ref = ref.cpu().numpy() if hasattr(ref, "cpu") else ref
        lib = kk.load_library()
        cs, keep = c_system(s)
        mesh = (ctypes.c_int32 * 3)(*w.mesh)
        copt = opt.c()
        for call in range(2):
            out = torch.full((3, 3), float("nan"), dtype=torch.float64, device=dev)
            st = lib.kald_kappa_rta_noalloc(None, None, ctypes.byref(cs), mesh, nu_d.data_ptr(),
                                            eig_d.data_ptr(), g_d.data_ptr(), ctypes.byref(copt),
                                            out.data_ptr())
            assert st == 0, f"call {call}: status {st}"
            np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-10,
                                       atol=1e-12 * np.abs(ref).max())
        # a mesh whose per-q scratch exceeds the static array is refused
        big = (40, 40, 40)
        nq, nb = 40 ** 3, s.n_branches
        nu_b = torch.zeros((nq, nb), dtype=torch.float64, device=dev)
        eig_b = torch.zeros((nq, nb, nb), dtype=torch.complex128, device=dev)
        g_b = torch.zeros(nq * nb, dtype=torch.float64, device=dev)
        out = torch.zeros(9, dtype=torch.float64, device=dev)
        st = lib.kald_kappa_rta_noalloc(ctx.handle, None, ctypes.byref(cs), (ctypes.c_int32 * 3)(*big),
                                        nu_b.data_ptr(), eig_b.data_ptr(), g_b.data_ptr(),
                                        ctypes.byref(copt), out.data_ptr())
        assert st == 1
        assert "static array" in lib.kald_last_error(ctx.handle).decode()
        del keep
