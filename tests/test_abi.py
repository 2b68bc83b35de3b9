"""CPU checks of the boundary: libddf.so builds for sm_103a, loads without a GPU and exports
every entry point include/ddf.h declares; the binding's signature table covers them all."""

import ctypes

import pytest

from tests._helpers import ensure_built


def test_library_exports_every_declared_symbol():
    ensure_built()
    from paper_2306_16142_gb300 import _abi
    declared = _abi.declared_symbols()
    assert len(declared) >= 15
    lib = ctypes.CDLL(_abi.LIB_PATH)
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    assert set(declared) == set(_abi._SIG), set(declared) ^ set(_abi._SIG)


def test_version_and_error_strings_without_gpu():
    ensure_built()
    from paper_2306_16142_gb300 import _abi
    lib = _abi.load()
    assert b"sm_103a" in lib.ddf_version()
    # argument checking happens before any CUDA call
    rc = lib.ddf_query(None, None, None, 1, None, None, None, None, None)
    assert rc == _abi.DDF_ERR_INVALID_ARG
    assert b"NULL" in lib.ddf_last_error()
    arch = _abi.ddf_arch(3, 64, 4, 0)       # odd in_freqs
    h = ctypes.c_void_p()
    assert lib.ddf_create(ctypes.byref(arch), None, 0, ctypes.byref(h)) == _abi.DDF_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2306_16142_gb300 import _abi
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        _abi.load()
