"""ctypes binding of libkald.so (include/kald.h).  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.  There is
no fallback: without the built library (or without a GPU) the calls raise.

Bulk arrays may be numpy arrays (host) or torch tensors on the context's CUDA
device; the library detects the pointer kind.  Shapes and dtypes follow
include/kald.h: float64 for real arrays, complex128 for eigenvectors.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkald.so")

KALD_OK = 0
STATUS = {0: "KALD_OK", 1: "KALD_E_INVALID", 2: "KALD_E_NOMEM", 3: "KALD_E_CUDA",
          4: "KALD_E_NOCONV", 5: "KALD_E_TIMEOUT", 6: "KALD_E_UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "bf16split": 2}
DELTA_SHAPE = {"gaussian": 0, "lorentzian": 1, "triangular": 2}
SYMMETRY = {"all": 0, "inversion": 1, "none": 2}

EXPORTS = ["kald_ctx_create", "kald_ctx_destroy", "kald_last_error", "kald_set_stream",
           "kald_phonons", "kald_linewidths", "kald_kappa_rta", "kald_kappa_qhgk",
           "kald_kappa_rta_noalloc", "kald_kernel_launches", "kald_set_wait_limit",
           "kald_set_workspace_limit", "kald_profile_enable", "kald_profile_read",
           "kald_linewidths_qrange", "kald_linewidths_qlist", "kald_phonons_batch", "kald_phase_space", "kald_diffusivity",
           "kald_scattering_matrix", "kald_kappa_bte", "kald_interpolate_gamma", "kald_fd_force_constants"]
PROF_KERNELS = {"tcx_gather": 0, "tcx_gemm1": 1, "tcx_gemm2": 2, "tc_gemm1": 3, "tc_gemm2": 4,
                "small_nb": 5, "lw_main": 6}


class KaldError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class kald_system(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("masses", C.c_void_p), ("positions", C.c_void_p),
                ("lattice", C.c_double * 9), ("n_fc2", C.c_int32), ("fc2_idx", C.c_void_p),
                ("fc2", C.c_void_p), ("n_fc3", C.c_int32), ("fc3_idx", C.c_void_p),
                ("fc3", C.c_void_p)]


class kald_pair_potential(C.Structure):
    _fields_ = [("kind", C.c_int32), ("epsilon", C.c_double), ("sigma", C.c_double), ("cutoff", C.c_double)]


class kald_options(C.Structure):
    _fields_ = [("temperature_K", C.c_double), ("sigma_thz", C.c_double), ("n_sigma", C.c_double),
                ("omega_min_thz", C.c_double), ("degen_tol_thz", C.c_double),
                ("classical", C.c_int32), ("precision", C.c_int32), ("delta_shape", C.c_int32),
                ("qhgk_bandwidth_thz", C.c_double), ("qhgk_threshold_thz", C.c_double),
                ("symmetry", C.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libkald.so once; raise if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libkald.so not built at {path}; run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, i32, st = C.c_void_p, C.c_int32, C.c_int
    lib.kald_ctx_create.argtypes = [C.POINTER(vp), C.c_int]
    lib.kald_ctx_create.restype = st
    lib.kald_ctx_destroy.argtypes = [vp]
    lib.kald_ctx_destroy.restype = None
    lib.kald_last_error.argtypes = [vp]
    lib.kald_last_error.restype = C.c_char_p
    lib.kald_set_stream.argtypes = [vp, vp]
    lib.kald_set_stream.restype = st
    lib.kald_phonons.argtypes = [vp, C.POINTER(kald_system), C.POINTER(i32), vp, vp, vp]
    lib.kald_phonons.restype = st
    lib.kald_scattering_matrix.argtypes = [vp, C.POINTER(kald_system), C.POINTER(i32), vp, vp,
                                           C.POINTER(kald_options), vp, vp]
    lib.kald_scattering_matrix.restype = st
    lib.kald_kappa_bte.argtypes = [vp, C.POINTER(kald_system), C.POINTER(i32), vp, vp, C.POINTER(kald_options),
                                   i32, C.c_double, i32, vp, C.POINTER(i32)]
    lib.kald_kappa_bte.restype = st
    lib.kald_fd_force_constants.argtypes = [vp, C.POINTER(kald_system), C.POINTER(kald_pair_potential), C.c_double,
                                            vp, vp]
    lib.kald_fd_force_constants.restype = st
    lib.kald_interpolate_gamma.argtypes = [vp, i32, vp, vp, i32, vp, C.POINTER(kald_options), vp]
    lib.kald_interpolate_gamma.restype = st
    lib.kald_phase_space.argtypes = [vp, C.POINTER(kald_system), C.POINTER(i32), vp, C.POINTER(kald_options), vp]
    lib.kald_phase_space.restype = st
    lib.kald_diffusivity.argtypes = [vp, i32, C.POINTER(kald_system), vp, vp, vp, C.POINTER(kald_options), vp]
    lib.kald_diffusivity.restype = st
    lib.kald_phonons_batch.argtypes = [vp, i32, C.POINTER(kald_system), vp, vp]
    lib.kald_phonons_batch.restype = st
    lib.kald_linewidths.argtypes = [vp, i32, C.POINTER(kald_system), C.POINTER(i32), vp, vp,
                                    C.POINTER(kald_options), vp, C.POINTER(C.c_uint64)]
    lib.kald_linewidths.restype = st
    lib.kald_linewidths_qrange.argtypes = [vp, C.POINTER(kald_system), C.POINTER(i32), vp, vp,
                                           C.POINTER(kald_options), i32, i32, vp, C.POINTER(C.c_uint64)]
    lib.kald_linewidths_qrange.restype = st
    lib.kald_linewidths_qlist.argtypes = [vp, C.POINTER(kald_system), C.POINTER(i32), vp, vp,
                                          C.POINTER(kald_options), i32, vp, vp, C.POINTER(C.c_uint64)]
    lib.kald_linewidths_qlist.restype = st
    lib.kald_kappa_rta.argtypes = [vp, C.POINTER(kald_system), C.POINTER(i32), vp, vp, vp,
                                   C.POINTER(kald_options), vp]
    lib.kald_kappa_rta.restype = st
    lib.kald_kappa_qhgk.argtypes = [vp, i32, C.POINTER(kald_system), vp, vp, vp,
                                    C.POINTER(kald_options), vp, vp]
    lib.kald_kappa_qhgk.restype = st
    lib.kald_kappa_rta_noalloc.argtypes = [vp, vp, C.POINTER(kald_system), C.POINTER(i32), vp, vp, vp,
                                           C.POINTER(kald_options), vp]
    lib.kald_kappa_rta_noalloc.restype = st
    lib.kald_set_wait_limit.argtypes = [vp, C.c_uint32]
    lib.kald_set_wait_limit.restype = st
    lib.kald_set_workspace_limit.argtypes = [vp, C.c_uint64]
    lib.kald_set_workspace_limit.restype = st
    lib.kald_profile_enable.argtypes = [vp, C.c_int]
    lib.kald_profile_enable.restype = st
    lib.kald_profile_read.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_uint64)]
    lib.kald_profile_read.restype = st
    lib.kald_kernel_launches.argtypes = []
    lib.kald_kernel_launches.restype = C.c_uint64
    _lib = lib
    return lib


def kald_kernel_launches() -> int:
    """Kernel launches the library has made in this process (diagnostic)."""
    return int(load_library().kald_kernel_launches())


@dataclass
class Options:
    temperature_K: float
    sigma_thz: float
    n_sigma: float = 3.0
    omega_min_thz: float = 0.01
    degen_tol_thz: float = 1e-5
    classical: bool = False
    precision: str = "fp64"
    delta: str = "gaussian"
    qhgk_bandwidth_thz: float = 0.0
    qhgk_threshold_thz: float = 0.0
    symmetry: str = "all"          # "all", "inversion" (time reversal only) or "none"

    def c(self) -> kald_options:
        return kald_options(self.temperature_K, self.sigma_thz, self.n_sigma, self.omega_min_thz,
                            self.degen_tol_thz, int(bool(self.classical)), PRECISION[self.precision],
                            DELTA_SHAPE[self.delta], float(self.qhgk_bandwidth_thz),
                            float(self.qhgk_threshold_thz), SYMMETRY[self.symmetry])


class Context:
    """A library context on one CUDA device (own stream and workspace)."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        self.handle = C.c_void_p()
        s = self.lib.kald_ctx_create(C.byref(self.handle), int(device))
        if s != KALD_OK:
            raise KaldError(s, f"kald_ctx_create(device={device}) failed")
        self.device = device

    def check(self, status: int):
        if status != KALD_OK:
            raise KaldError(status, self.lib.kald_last_error(self.handle).decode())

    def set_stream(self, stream_ptr: int | None):
        self.check(self.lib.kald_set_stream(self.handle, C.c_void_p(stream_ptr or 0)))

    def set_wait_limit(self, polls: int):
        """Polls of the tensor-core pipeline waits (0: the default)."""
        self.check(self.lib.kald_set_wait_limit(self.handle, int(polls)))

    def set_workspace_limit(self, n_bytes: int):
        """Cap the device workspace (0: no cap); larger requests give KALD_E_NOMEM."""
        self.check(self.lib.kald_set_workspace_limit(self.handle, int(n_bytes)))

    def profile(self, on: bool):
        """Switch per-launch CUDA-event timing of the hot kernels (clears the totals)."""
        self.check(self.lib.kald_profile_enable(self.handle, int(bool(on))))

    def profile_read(self) -> dict:
        """{kernel: (total ms, launches)} since profiling was switched on."""
        out = {}
        for name, kid in PROF_KERNELS.items():
            ms, n = C.c_double(), C.c_uint64()
            self.check(self.lib.kald_profile_read(self.handle, kid, C.byref(ms), C.byref(n)))
            out[name] = (ms.value, int(n.value))
        return out

    def close(self):
        if self.handle:
            self.lib.kald_ctx_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---- marshalling helpers ------------------------------------------------------

def _ptr(a, dtype, n_elem, name):
    """Address of a contiguous float64/complex128 numpy array or torch tensor."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{name}: need a C-contiguous {np.dtype(dtype).name} array")
        if a.size != n_elem:
            raise ValueError(f"{name}: {a.size} elements, expected {n_elem}")
        return a.ctypes.data
    # torch tensor (duck-typed so torch stays optional)
    if hasattr(a, "data_ptr") and hasattr(a, "is_contiguous"):
        want = {np.float64: "torch.float64", np.complex128: "torch.complex128"}[dtype]
        if str(a.dtype) != want or not a.is_contiguous():
            raise TypeError(f"{name}: need a contiguous {want} tensor")
        if a.numel() != n_elem:
            raise ValueError(f"{name}: {a.numel()} elements, expected {n_elem}")
        return a.data_ptr()
    raise TypeError(f"{name}: numpy array or torch tensor expected")


def c_system(s) -> tuple[kald_system, list]:
    """kald_system for an object with the fields of kald_inputs.System; the
    second value keeps the host arrays alive for the call."""
    keep = [np.ascontiguousarray(s.masses, dtype=np.float64),
            np.ascontiguousarray(s.positions, dtype=np.float64),
            np.ascontiguousarray(s.fc2_idx, dtype=np.int32),
            np.ascontiguousarray(s.fc2, dtype=np.float64),
            np.ascontiguousarray(s.fc3_idx, dtype=np.int32),
            np.ascontiguousarray(s.fc3, dtype=np.float64)]
    lat = (C.c_double * 9)(*np.asarray(s.lattice, dtype=np.float64).reshape(-1))
    cs = kald_system(int(keep[0].shape[0]), keep[0].ctypes.data, keep[1].ctypes.data, lat,
                     int(keep[3].shape[0]), keep[2].ctypes.data, keep[3].ctypes.data,
                     int(keep[5].shape[0]), keep[4].ctypes.data, keep[5].ctypes.data)
    return cs, keep


def _mesh(mesh):
    m = (C.c_int32 * 3)(*[int(x) for x in mesh])
    return m, int(np.prod([int(x) for x in mesh]))


# ---- entry points (same names as the C ABI) -----------------------------------

def kald_phonons(ctx: Context, system, mesh, nu_thz=None, eigvec=None, vel=None, want_vel=True):
    """Phonons on the mesh; returns (nu_thz [Nq, nb], eigvec [Nq, nb, nb], vel [Nq, nb, 3] or None).
    Outputs default to new host numpy arrays."""
    cs, keep = c_system(system)
    m, nq = _mesh(mesh)
    nb = 3 * cs.n_atoms
    if nu_thz is None:
        nu_thz = np.zeros((nq, nb))
    if eigvec is None:
        eigvec = np.zeros((nq, nb, nb), dtype=np.complex128)
    if vel is None and want_vel:
        vel = np.zeros((nq, nb, 3))
    ctx.check(ctx.lib.kald_phonons(ctx.handle, C.byref(cs), m,
                                   _ptr(nu_thz, np.float64, nq * nb, "nu_thz"),
                                   _ptr(eigvec, np.complex128, nq * nb * nb, "eigvec"),
                                   _ptr(vel, np.float64, nq * nb * 3, "vel")))
    del keep
    return nu_thz, eigvec, vel


def _systems(systems):
    if not isinstance(systems, (list, tuple)):
        systems = [systems]
    arr = (kald_system * len(systems))()
    keep = []
    for x, s in enumerate(systems):
        cs, k = c_system(s)
        arr[x] = cs
        keep.append(k)
    return arr, keep, [3 * int(np.asarray(s.masses).shape[0]) for s in systems]


def kald_phonons_batch(ctx: Context, systems, nu_thz=None, eigvec=None):
    """Gamma-only phonons of several supercells in one launch sequence; returns
    (nu_thz [sum nb], eigvec [sum nb^2]) concatenated per system (host numpy
    arrays by default)."""
    arr, keep, nbs = _systems(systems)
    n_modes = sum(nbs)
    n_eig = sum(nb * nb for nb in nbs)
    if nu_thz is None:
        nu_thz = np.zeros(n_modes)
    if eigvec is None:
        eigvec = np.zeros(n_eig, dtype=np.complex128)
    ctx.check(ctx.lib.kald_phonons_batch(ctx.handle, len(nbs), arr,
                                         _ptr(nu_thz, np.float64, n_modes, "nu_thz"),
                                         _ptr(eigvec, np.complex128, n_eig, "eigvec")))
    del keep
    return nu_thz, eigvec


def kald_linewidths(ctx: Context, systems, mesh, nu_thz, eigvec, options: Options, gamma=None):
    """Linewidths gamma (ps^-1); returns (gamma, (n_triplets, n_allowed))."""
    arr, keep, nbs = _systems(systems)
    m, nq = _mesh(mesh)
    n_modes = sum(nq * nb for nb in nbs)
    n_eig = sum(nq * nb * nb for nb in nbs)
    if gamma is None:
        gamma = np.zeros(n_modes) if isinstance(nu_thz, np.ndarray) else None
        if gamma is None:
            import torch
            gamma = torch.zeros(n_modes, dtype=torch.float64, device=nu_thz.device)
    trip = (C.c_uint64 * 2)()
    opt = options.c()
    ctx.check(ctx.lib.kald_linewidths(ctx.handle, len(nbs), arr, m,
                                      _ptr(nu_thz, np.float64, n_modes, "nu_thz"),
                                      _ptr(eigvec, np.complex128, n_eig, "eigvec"),
                                      C.byref(opt), _ptr(gamma, np.float64, n_modes, "gamma"), trip))
    del keep
    return gamma, (int(trip[0]), int(trip[1]))


def kald_linewidths_qrange(ctx: Context, system, mesh, nu_thz, eigvec, options: Options, q_begin: int,
                           q_end: int, gamma=None):
    """Linewidths of the q-points [q_begin, q_end) of one crystal (full-mesh nu
    and eigvec in); returns (gamma [(q_end - q_begin) * nb], (n_triplets, n_allowed))."""
    cs, keep = c_system(system)
    m, nq = _mesh(mesh)
    nb = 3 * cs.n_atoms
    n_out = (int(q_end) - int(q_begin)) * nb
    if gamma is None:
        if isinstance(nu_thz, np.ndarray):
            gamma = np.zeros(max(n_out, 0))
        else:
            import torch
            gamma = torch.zeros(max(n_out, 0), dtype=torch.float64, device=nu_thz.device)
    trip = (C.c_uint64 * 2)()
    opt = options.c()
    ctx.check(ctx.lib.kald_linewidths_qrange(ctx.handle, C.byref(cs), m,
                                             _ptr(nu_thz, np.float64, nq * nb, "nu_thz"),
                                             _ptr(eigvec, np.complex128, nq * nb * nb, "eigvec"),
                                             C.byref(opt), int(q_begin), int(q_end),
                                             _ptr(gamma, np.float64, max(n_out, 0), "gamma"), trip))
    del keep
    return gamma, (int(trip[0]), int(trip[1]))


def kald_linewidths_qlist(ctx: Context, system, mesh, nu_thz, eigvec, options: Options, q_list, gamma=None):
    """Linewidths of the listed q-points of one crystal (full-mesh nu and
    eigvec in); returns (gamma [len(q_list) * nb], row j = q_list[j],
    (n_triplets, n_allowed))."""
    cs, keep = c_system(system)
    m, nq = _mesh(mesh)
    nb = 3 * cs.n_atoms
    ql = np.ascontiguousarray(np.asarray(q_list, dtype=np.int32).ravel())
    n_out = ql.size * nb
    if gamma is None:
        if isinstance(nu_thz, np.ndarray):
            gamma = np.zeros(max(n_out, 0))
        else:
            import torch
            gamma = torch.zeros(max(n_out, 0), dtype=torch.float64, device=nu_thz.device)
    trip = (C.c_uint64 * 2)()
    opt = options.c()
    ctx.check(ctx.lib.kald_linewidths_qlist(ctx.handle, C.byref(cs), m,
                                            _ptr(nu_thz, np.float64, nq * nb, "nu_thz"),
                                            _ptr(eigvec, np.complex128, nq * nb * nb, "eigvec"),
                                            C.byref(opt), int(ql.size), ql.ctypes.data,
                                            _ptr(gamma, np.float64, max(n_out, 0), "gamma"), trip))
    del keep
    return gamma, (int(trip[0]), int(trip[1]))


def kald_scattering_matrix(ctx: Context, system, mesh, nu_thz, eigvec, options: Options):
    """(Gamma^0 [N], Gamma^1 [N, N]) of the linearised BTE, N = Nq nb (host arrays)."""
    cs, keep = c_system(system)
    m, nq = _mesh(mesh)
    nb = 3 * cs.n_atoms
    N = nq * nb
    g0 = np.zeros(N)
    G1 = np.zeros((N, N))
    opt = options.c()
    ctx.check(ctx.lib.kald_scattering_matrix(ctx.handle, C.byref(cs), m, _ptr(nu_thz, np.float64, N, "nu_thz"),
                                             _ptr(eigvec, np.complex128, N * nb, "eigvec"), C.byref(opt),
                                             _ptr(g0, np.float64, N, "gamma0"), _ptr(G1, np.float64, N * N, "G1")))
    del keep
    return g0, G1


BTE_METHOD = {"krylov": 0, "self_consistent": 1}


def kald_kappa_bte(ctx: Context, system, mesh, nu_thz, eigvec, options: Options, method: str = "krylov",
                   tol: float = 1e-10, max_iter: int = 500, kappa=None):
    """kappa [3, 3] (W/(m K)) from the full linearised BTE; returns (kappa, iterations).
    Raises KaldError (KALD_E_NOCONV) when the iteration does not converge."""
    cs, keep = c_system(system)
    m, nq = _mesh(mesh)
    nb = 3 * cs.n_atoms
    N = nq * nb
    if kappa is None:
        kappa = np.zeros((3, 3))
    it = C.c_int32()
    opt = options.c()
    status = ctx.lib.kald_kappa_bte(ctx.handle, C.byref(cs), m, _ptr(nu_thz, np.float64, N, "nu_thz"),
                                    _ptr(eigvec, np.complex128, N * nb, "eigvec"), C.byref(opt),
                                    BTE_METHOD[method], float(tol), int(max_iter), _ptr(kappa, np.float64, 9, "kappa"),
                                    C.byref(it))
    del keep
    ctx.check(status)
    return kappa, int(it.value)


def kald_fd_force_constants(ctx: Context, system, epsilon: float, sigma: float, cutoff: float, h: float = 1e-3):
    """(fc2 [n_fc2, 3, 3], fc3 [n_fc3, 3, 3, 3]) of a Lennard-Jones pair potential by
    finite differences on the GPU, for the blocks of `system` (its values unused)."""
    cs, keep = c_system(system)
    pot = kald_pair_potential(0, float(epsilon), float(sigma), float(cutoff))
    fc2 = np.zeros((cs.n_fc2, 3, 3))
    fc3 = np.zeros((cs.n_fc3, 3, 3, 3))
    ctx.check(ctx.lib.kald_fd_force_constants(ctx.handle, C.byref(cs), C.byref(pot), float(h),
                                              fc2.ctypes.data if cs.n_fc2 else None,
                                              fc3.ctypes.data if cs.n_fc3 else None))
    del keep
    return fc2, fc3


def kald_interpolate_gamma(ctx: Context, nu_src, gamma_src, nu_dst, options: Options, gamma_dst=None):
    """gamma at nu_dst from (nu_src, gamma_src) by a not-a-knot cubic spline of gamma(nu)."""
    n_src = int(np.asarray(nu_src).size) if isinstance(nu_src, np.ndarray) else int(nu_src.numel())
    n_dst = int(np.asarray(nu_dst).size) if isinstance(nu_dst, np.ndarray) else int(nu_dst.numel())
    if gamma_dst is None:
        gamma_dst = np.zeros(n_dst)
    opt = options.c()
    ctx.check(ctx.lib.kald_interpolate_gamma(ctx.handle, n_src, _ptr(nu_src, np.float64, n_src, "nu_src"),
                                             _ptr(gamma_src, np.float64, n_src, "gamma_src"), n_dst,
                                             _ptr(nu_dst, np.float64, n_dst, "nu_dst"), C.byref(opt),
                                             _ptr(gamma_dst, np.float64, n_dst, "gamma_dst")))
    return gamma_dst


def kald_phase_space(ctx: Context, system, mesh, nu_thz, options: Options, g=None):
    """Phase space per mode g [Nq * nb] (ps)."""
    cs, keep = c_system(system)
    m, nq = _mesh(mesh)
    nb = 3 * cs.n_atoms
    if g is None:
        g = np.zeros(nq * nb)
    opt = options.c()
    ctx.check(ctx.lib.kald_phase_space(ctx.handle, C.byref(cs), m, _ptr(nu_thz, np.float64, nq * nb, "nu_thz"),
                                       C.byref(opt), _ptr(g, np.float64, nq * nb, "g")))
    del keep
    return g


def kald_diffusivity(ctx: Context, systems, nu_thz, eigvec, gamma, options: Options, D=None):
    """Mode diffusivity D [sum nb] (A^2/ps) of Gamma-only systems."""
    arr, keep, nbs = _systems(systems)
    n_modes = sum(nbs)
    n_eig = sum(nb * nb for nb in nbs)
    if D is None:
        D = np.zeros(n_modes)
    opt = options.c()
    ctx.check(ctx.lib.kald_diffusivity(ctx.handle, len(nbs), arr, _ptr(nu_thz, np.float64, n_modes, "nu_thz"),
                                       _ptr(eigvec, np.complex128, n_eig, "eigvec"),
                                       _ptr(gamma, np.float64, n_modes, "gamma"), C.byref(opt),
                                       _ptr(D, np.float64, n_modes, "D")))
    del keep
    return D


def kald_kappa_rta(ctx: Context, system, mesh, nu_thz, eigvec, gamma, options: Options, kappa=None):
    """BTE-RTA kappa [3, 3] in W/(m K)."""
    cs, keep = c_system(system)
    m, nq = _mesh(mesh)
    nb = 3 * cs.n_atoms
    if kappa is None:
        kappa = np.zeros((3, 3))
    opt = options.c()
    ctx.check(ctx.lib.kald_kappa_rta(ctx.handle, C.byref(cs), m,
                                     _ptr(nu_thz, np.float64, nq * nb, "nu_thz"),
                                     _ptr(eigvec, np.complex128, nq * nb * nb, "eigvec"),
                                     _ptr(gamma, np.float64, nq * nb, "gamma"), C.byref(opt),
                                     _ptr(kappa, np.float64, 9, "kappa")))
    del keep
    return kappa


def kald_kappa_qhgk(ctx: Context, systems, nu_thz, eigvec, gamma, options: Options, kappa=None,
                    vgen=None, want_vgen=False):
    """QHGK kappa [n_sys, 3, 3] (W/(m K)) and, optionally, W_a [3, nb, nb] of system 0."""
    arr, keep, nbs = _systems(systems)
    n_modes = sum(nbs)
    n_eig = sum(nb * nb for nb in nbs)
    if kappa is None:
        kappa = np.zeros((len(nbs), 3, 3))
    if vgen is None and want_vgen:
        vgen = np.zeros((3, nbs[0], nbs[0]))
    opt = options.c()
    ctx.check(ctx.lib.kald_kappa_qhgk(ctx.handle, len(nbs), arr,
                                      _ptr(nu_thz, np.float64, n_modes, "nu_thz"),
                                      _ptr(eigvec, np.complex128, n_eig, "eigvec"),
                                      _ptr(gamma, np.float64, n_modes, "gamma"), C.byref(opt),
                                      _ptr(kappa, np.float64, 9 * len(nbs), "kappa"),
                                      _ptr(vgen, np.float64, 3 * nbs[0] * nbs[0], "vgen")))
    del keep
    return kappa, vgen


def kald_kappa_rta_noalloc(ctx: Context | None, system, mesh, nu_thz, eigvec, gamma, options: Options,
                           kappa, stream_ptr: int | None = None):
    """kald_kappa_rta without any device allocation (static scratch inside the
    library); every array argument must be a CUDA tensor on the device."""
    lib = ctx.lib if ctx is not None else load_library()
    cs, keep = c_system(system)
    m, nq = _mesh(mesh)
    nb = 3 * cs.n_atoms
    opt = options.c()
    status = lib.kald_kappa_rta_noalloc(ctx.handle if ctx is not None else None, stream_ptr, C.byref(cs), m,
                                        _ptr(nu_thz, np.float64, nq * nb, "nu_thz"),
                                        _ptr(eigvec, np.complex128, nq * nb * nb, "eigvec"),
                                        _ptr(gamma, np.float64, nq * nb, "gamma"), C.byref(opt),
                                        _ptr(kappa, np.float64, 9, "kappa"))
    del keep
    if status != KALD_OK:
        msg = lib.kald_last_error(ctx.handle).decode() if ctx is not None else ""
        raise KaldError(status, msg or "kald_kappa_rta_noalloc failed")
    return kappa
