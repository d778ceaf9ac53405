"""The C ABI library builds for sm_103a, loads on a CPU-only host and exports
every entry point include/esplit.h declares (no compute call is made)."""
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "esplit.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(esplit_[a-z_0-9]+)\s*\(", src)))


def _lib_path():
    from paper_2305_07181_gb300 import build
    if not os.path.exists(build.LIB):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc unavailable and library not built")
        build.build()
    return build.LIB


def test_header_declares_expected_calls():
    names = declared()
    for n in ["esplit_create", "esplit_upload_operator", "esplit_upload_mesh", "esplit_residual",
              "esplit_rrk_step", "esplit_residual_vjp", "esplit_entropy", "esplit_get_status"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import ctypes
    lib = ctypes.CDLL(_lib_path())
    for n in declared():
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    _lib_path()
    from paper_2305_07181_gb300 import capi
    assert sorted(capi.exported_names()) == declared()
    for n in declared():
        assert callable(getattr(capi, n))
    assert capi.esplit_version() >= 100
