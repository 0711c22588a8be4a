"""The C-ABI library builds, loads and exports every symbol include/bcrown.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "bcrown.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bcrown_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2103_06624_gb300 import build_native
    if not os.path.exists(build_native.LIB):
        build_native.build()
    return build_native.LIB


def test_header_declares_the_boundary():
    syms = _declared_symbols()
    for name in ["bcrown_load_net", "bcrown_root_bounds", "bcrown_bound", "bcrown_bound_grad", "bcrown_optimize"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (bcrown_\w+)", out))
    assert set(_declared_symbols()) <= exported


def test_binding_declares_the_same_names(lib_path):
    from paper_2103_06624_gb300 import native
    assert sorted(native.EXPORTS) == _declared_symbols()
    lib = native.load(lib_path)
    assert lib.bcrown_last_error() is not None


def test_argument_errors_without_gpu(lib_path):
    """Host-side argument checks run before any CUDA call."""
    from paper_2103_06624_gb300 import native as N
    lib = N.load(lib_path)
    h = ctypes.c_void_p()
    assert lib.bcrown_load_net(None, 0, None, 0, ctypes.byref(h)) == N.ERR_ARG
    assert b"null" in lib.bcrown_last_error()
    assert lib.bcrown_bound(None, None, None, None, None, 0, None, None) == N.ERR_ARG
    assert lib.bcrown_status(None, None) == N.ERR_ARG
