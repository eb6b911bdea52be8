"""CPU checks of the C ABI library: it builds, loads, and exports every entry
point include/cvrpsd.h declares; no compute call is made here."""
import ctypes
import os
import re

import pytest

import paper_2511_18022_gb300 as cv
from paper_2511_18022_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cvrpsd.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(cvrpsd_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("cvrpsd_split_eval", "cvrpsd_gen_demand", "cvrpsd_create", "cvrpsd_destroy"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) <= set(_lib.EXPORTS)


def test_strerror_and_version(lib):
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.cvrpsd_strerror(code).decode()
    assert "sm_103a" in cv.cvrpsd_version()


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "nope.so"))


def test_product_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2511_18022_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", src), f


def test_null_context_is_rejected(lib):
    assert lib.cvrpsd_split_eval(None, None, 1, None, None, 2, 0, 1, 0, 1,
                                 None, None, None, None, None) == _lib.ERR_ARG
    assert lib.cvrpsd_destroy(None) == _lib.ERR_ARG
