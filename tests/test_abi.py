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


def test_checkpoint_load_rejects_bad_files_without_gpu(tmp_path):
    """ddf_load validates the file before touching the device: missing file, wrong magic, a
    header whose architecture is invalid or disagrees with its parameter count, a truncated body."""
    import struct
    ensure_built()
    from paper_2306_16142_gb300 import _abi
    lib = _abi.load()
    h = ctypes.c_void_p()
    assert lib.ddf_load(str(tmp_path / "missing.ckpt").encode(), ctypes.byref(h)) == _abi.DDF_ERR_IO
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(b"NOTACKPT" + bytes(56))
    assert lib.ddf_load(str(bad).encode(), ctypes.byref(h)) == _abi.DDF_ERR_IO

    def header(F, W, L, prec, n_params, step=0, has_adam=0):
        return b"DDFCKPT1" + struct.pack("<4iqqi5i", F, W, L, prec, n_params, step, has_adam, 0, 0, 0, 0, 0)
    assert len(header(0, 64, 4, 0, 0)) == 64
    n_params = 6 * 64 + 64 + 3 * (64 * 64 + 64) + 2 * 64 + 2      # (0, 64, 4): E = 6
    for hdr in (header(3, 64, 4, 0, n_params),          # odd frequency count
                header(0, 64, 4, 0, n_params + 1),      # parameter count disagrees
                header(0, 64, 4, 9, n_params)):         # unknown precision
        bad.write_bytes(hdr + bytes(4 * n_params))
        assert lib.ddf_load(str(bad).encode(), ctypes.byref(h)) == _abi.DDF_ERR_IO, hdr
    bad.write_bytes(header(0, 64, 4, 0, n_params) + bytes(4 * n_params - 4))   # one float short
    assert lib.ddf_load(str(bad).encode(), ctypes.byref(h)) == _abi.DDF_ERR_IO
    assert b"truncated" in lib.ddf_last_error()
