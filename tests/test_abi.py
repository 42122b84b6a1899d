"""CPU checks of the C ABI: the library builds, loads without a GPU and
exports every function include/ef.h declares; the binding lists them all.
No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ef.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char \*|void)\s*\**\s*(ef_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("ef_compute", "ef_compute_ex", "ef_ctx_create", "ef_ctx_destroy", "ef_last_error"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2306_00606_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in ef.h but not exported"


def test_binding_covers_header():
    import paper_2306_00606_gb300 as ef
    assert sorted(ef.EXPORTED) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(ef, name))


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2306_00606_gb300 as ef
    with pytest.raises(ef.EfError):
        ef._lib, saved = None, ef._lib
        try:
            ef.load_library(str(tmp_path / "missing.so"))
        finally:
            ef._lib = saved


def test_no_cuda_means_error_not_fallback():
    import torch
    import paper_2306_00606_gb300 as ef
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(ef.EfError):
        ef.Context(0)
