"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/kald.h declares.  No compute call is made here (no GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "kald.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kald_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_01967_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_hot_path_calls():
    names = _declared()
    for n in ("kald_phonons", "kald_linewidths", "kald_kappa_rta", "kald_kappa_qhgk"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_2009_01967_gb300 as k
    for n in _declared():
        assert n in k.EXPORTS


def test_context_without_gpu_reports_cuda_error(lib):
    """With no usable device the library refuses (KALD_E_CUDA), never falls back."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    lib.kald_ctx_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    assert lib.kald_ctx_create(ctypes.byref(h), 0) == 3
    assert not h.value


def test_launch_counter_starts_at_zero_without_gpu(lib):
    """The diagnostic launch counter is readable without a device and counts
    nothing when no call ran."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    lib.kald_kernel_launches.restype = ctypes.c_uint64
    assert lib.kald_kernel_launches() == 0
