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


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structures of the binding have the size and field offsets
    of the C structures in include/kald.h (compiled here with the host C
    compiler), so an added or reordered field cannot silently shift the
    arguments the library reads."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    from paper_2009_01967_gb300 import _abi
    structs = {"kald_options": _abi.kald_options, "kald_system": _abi.kald_system,
               "kald_pair_potential": _abi.kald_pair_potential}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kald.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln.strip():
            parts = ln.split()
            got[tuple(parts[:-1])] = int(parts[-1])
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
