"""The C ABI library builds for sm_103a, loads, and exports every function include/spq.h
declares (no GPU needed: nothing here launches work)."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", "spq.h"), os.path.join(ROOT, "include", "spq_bench.h")]


def declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(spq_[a-z_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1503_07192_gb300 import _lib, build_ext

    build_ext.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["spq_build", "spq_query", "spq_free", "spq_strerror", "spq_footprint_bytes"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1503_07192_gb300 import _lib

    names = declared_functions()
    so = _lib.LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (spq_[a-z_]+)$", out, flags=re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    # and the Python binding declares a signature for each of them
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)
    for n in names:
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr)


def test_built_for_sm_103a_only(lib):
    from paper_1503_07192_gb300 import _lib

    r = subprocess.run(["cuobjdump", "--list-elf", _lib.LIB_PATH], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    archs = set(re.findall(r"sm_(\d+a?)", r.stdout))
    assert archs == {"103a"}, archs


def test_host_only_calls(lib):
    from paper_1503_07192_gb300 import SPQ_EINVAL, spq_opts_default, spq_strerror

    assert spq_strerror(0) == "success"
    assert "invalid" in spq_strerror(SPQ_EINVAL)
    o = spq_opts_default()
    assert o.struct_size == ctypes.sizeof(o) and o.skip_inf_tiles == 1
    lib.spq_free(None)  # NULL-safe
    assert lib.spq_footprint_bytes(None) == 0


def test_binding_raises_without_library(tmp_path):
    from paper_1503_07192_gb300 import _lib

    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "missing.so"))
