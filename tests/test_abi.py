"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/dfjk.h declares; the Python binding names the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "dfjk.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dfjk_[A-Za-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2404_09452_gb300 import build_lib

    return ctypes.CDLL(build_lib.build())


def test_header_declares_expected_entry_points():
    syms = header_symbols()
    for s in ("dfjk_setup", "dfjk_build", "dfjk_destroy", "dfjk_status_string", "dfjk_last_error"):
        assert s in syms


def test_library_exports_every_header_symbol(lib):
    for s in header_symbols():
        assert hasattr(lib, s), s


def test_binding_lists_the_header_symbols():
    from paper_2404_09452_gb300 import dfjk

    assert sorted(dfjk.EXPORTS) == header_symbols()


def test_status_strings_without_gpu(lib):
    lib.dfjk_status_string.restype = ctypes.c_char_p
    assert lib.dfjk_status_string(0) == b"ok"
    assert b"positive definite" in lib.dfjk_status_string(3)


def test_null_arguments_are_rejected_without_gpu(lib):
    # argument validation happens before any CUDA call
    assert lib.dfjk_setup(None, None, 0, None, None, None, None) == 1
    assert lib.dfjk_build(None, 1, 1, None, None, None, None, None, None) == 1
    assert lib.dfjk_destroy(None) == 0
