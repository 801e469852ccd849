"""The C-ABI library loads and exports every function that include/lya.h
declares; host-only entry points answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "lya.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lya_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_00129_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_hot_path():
    fns = header_functions()
    for name in ["lya_xi", "lya_dmat", "lya_xi_backward", "lya_xi_batched", "lya_pairs_build",
                 "lya_project", "lya_create", "lya_destroy"]:
        assert name in fns


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declaration():
    from paper_2507_00129_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == header_functions()


def test_status_strings_without_gpu(lib):
    assert lib.lya_status_string(0) == b"LYA_OK"
    assert lib.lya_status_string(-2) == b"LYA_ERR_UNSORTED"
    assert lib.lya_status_string(-99) == b"LYA_ERR_UNKNOWN"
    assert lib.lya_kernel_launches() >= 0


def test_null_handle_is_rejected_on_host(lib):
    assert lib.lya_xi(None, None, None, 1, None, None, None, None) == -1
    assert lib.lya_destroy(None) == -1
    assert lib.lya_last_error(None, None, 0) == -1
    # the extension entry points check the handle before touching the device
    assert lib.lya_xcf(None, None, None, None, None, None, None, None, None) == -1
    assert lib.lya_xdmat(None, None, None, None, None, 1, 1.0, 0, None, None, None) == -1
    assert lib.lya_xi1d(None, None, 10, 50.0, None, None, None, None) == -1
    assert lib.lya_xi_bin_means(None, None, None, None, None, None, None, None, None) == -1
    assert lib.lya_xi3(None, None, None, None, None, None, None) == -1


def test_api_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2507_00129_gb300 import _lib
    monkeypatch.setattr(_lib, "_LIB", None)
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load(str(tmp_path / "missing.so"))
