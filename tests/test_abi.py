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


C_NAMES = {"async_": "async"}   # binding field names that are Python keywords in C
STRUCTS = ("ef_csr", "ef_options", "ef_outputs", "ef_stats", "ef_tuning", "ef_partials", "ef_sir_params",
           "ef_sir_outputs", "ef_train_options", "ef_train_stats", "ef_rank_stats")


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every struct the binding passes by pointer has the size and the field
    names and offsets of its declaration in ef.h: a C program compiled
    against the header prints them (gcc, no CUDA needed)."""
    import shutil
    import subprocess
    import paper_2306_00606_gb300 as ef
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ef.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in getattr(ef, name)._fields_:
            cfield = C_NAMES.get(field, field)
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {cfield}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, "-std=c11", "-I", include, str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name in STRUCTS:
        cls = getattr(ef, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, f"{name}.{field}"
