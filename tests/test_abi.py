"""The C ABI library loads and exports every symbol include/lsq.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lsq.h")
LIB = os.path.join(ROOT, "paper_1911_02675_gb300", "_build", "liblsq.so")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^LSQ_API[^(]*?\b(lsq_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util

    spec = importlib.util.spec_from_file_location("_b", os.path.join(ROOT, "paper_1911_02675_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared()
    for required in ("lsq_sketch", "lsq_factor", "lsq_solve", "lsq_create", "lsq_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lsq_\w+)$", out, flags=re.M))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    for n in declared():
        getattr(lib, n)  # resolvable through dlsym


def test_host_only_entry_points(lib):
    lib.lsq_status_str.restype = ctypes.c_char_p
    lib.lsq_version.restype = ctypes.c_char_p
    assert lib.lsq_status_str(0) == b"ok"
    assert b"maxit" in lib.lsq_status_str(4)
    assert b"sm_103a" in lib.lsq_version()
    # null arguments are rejected before any CUDA call
    assert lib.lsq_sketch(None, None, 0, 16, 0, None, None) == 1
    assert lib.lsq_factor(None, None, 16, 4, None, None) == 1
    assert lib.lsq_factor_ex(None, None, 16, 4, None, None, 1) == 1
    assert lib.lsq_destroy(None) == 0
    assert lib.lsq_set_deferred_checks(None, 1) == 1
    assert lib.lsq_sync(None) == 1
    assert lib.lsq_upload_sketch(None, None, 4, None, 0, 16, 0, None, None) == 1


def test_python_binding_exports_match_header():
    src = open(os.path.join(ROOT, "paper_1911_02675_gb300", "__init__.py")).read()
    m = re.search(r"EXPORTS = \(([^)]*)\)", src, flags=re.S)
    names = set(re.findall(r'"(lsq_\w+)"', m.group(1)))
    assert names == set(declared())
