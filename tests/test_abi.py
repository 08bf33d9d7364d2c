"""The C-ABI library loads and exports every entry point declared in include/chfsi.h
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "chfsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chfsi_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1903_10959_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1903_10959_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == _declared()


def test_loader_fails_loudly_without_library(tmp_path):
    from paper_1903_10959_gb300 import _lib
    with pytest.raises(RuntimeError):
        _lib.load(str(tmp_path / "missing.so"))


def test_error_strings_without_device(lib):
    lib.chfsi_last_error.restype = ctypes.c_char_p
    lib.chfsi_last_error.argtypes = [ctypes.c_void_p]
    assert lib.chfsi_last_error(None) == b"null context"
    lib.chfsi_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.chfsi_create(None, None, None) == 1          # CHFSI_ERR_ARG, no device touched
