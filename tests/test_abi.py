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


def test_checkpoint_head_fields_are_validated_without_gpu(tmp_path):
    """The head kind, delta and weight-norm flag in the header's spare words are checked before any
    device call; a weight-normalised file missing its (v, g) section reads as truncated."""
    import struct
    ensure_built()
    from paper_2306_16142_gb300 import _abi
    lib = _abi.load()
    h = ctypes.c_void_p()
    n_params = 6 * 64 + 64 + 3 * (64 * 64 + 64) + 2 * 64 + 2      # (0, 64, 4): E = 6
    bad = tmp_path / "head.ckpt"

    def header(kind, delta, wn):
        return b"DDFCKPT1" + struct.pack("<4iqqiifi2i", 0, 64, 4, 0, n_params, 0, 0, kind, delta, wn, 0, 0)
    assert len(header(0, 0.0, 0)) == 64
    for hdr in (header(7, 0.5, 0),                  # unknown head kind
                header(1, 0.0, 0),                  # clamp head without a positive delta
                header(2, float("nan"), 0),         # squish head with a NaN delta
                header(0, 0.0, 2)):                 # weight_norm is 0 or 1
        bad.write_bytes(hdr + bytes(4 * n_params))
        assert lib.ddf_load(str(bad).encode(), ctypes.byref(h)) == _abi.DDF_ERR_IO, hdr
    bad.write_bytes(header(1, 0.5, 1) + bytes(4 * n_params))     # the (v, g) section is missing
    assert lib.ddf_load(str(bad).encode(), ctypes.byref(h)) == _abi.DDF_ERR_IO
    assert b"truncated" in lib.ddf_last_error()


def test_newer_entry_points_reject_bad_arguments_without_gpu():
    """Every entry point added with the samplers, heads, BVH, AOV, mesh renderer and UDF rejects a
    NULL handle or argument on the host, before any device call."""
    ensure_built()
    from paper_2306_16142_gb300 import _abi
    lib = _abi.load()
    E = _abi.DDF_ERR_INVALID_ARG
    head = _abi.ddf_head(_abi.DDF_HEAD_CLAMP, 0.5, 0)
    cam = _abi.ddf_camera()
    pov = _abi.ddf_pov(10, 5, 8, 2.5, 0.27)
    smp = _abi.ddf_sampler(1, 1, 1, 1e-4, 0)
    n = ctypes.c_int64()
    out4 = (ctypes.c_int64 * 4)()
    arch = _abi.ddf_arch()
    assert lib.ddf_set_head(None, ctypes.byref(head), None) == E
    assert lib.ddf_get_weight_norm(None, None, 0, None, 0, None) == E
    assert lib.ddf_get_arch(None, ctypes.byref(arch)) == E
    assert lib.ddf_udf(None, None, 1, None, 1, None, None, None) == E
    assert lib.ddf_render_aov(None, ctypes.byref(cam), None, None, None) == E
    assert lib.ddf_mesh_render_aov(None, ctypes.byref(cam), None, None, None, None) == E
    assert lib.ddf_mesh_render(None, ctypes.byref(cam), 1, 1, None, None) == E
    assert lib.ddf_mesh_set_accel(None, _abi.DDF_ACCEL_BVH) == E
    assert lib.ddf_mesh_bvh_stats(None, out4) == E
    assert lib.ddf_sample_pov(None, ctypes.byref(pov), None, None, None, None, None) == E
    assert lib.ddf_sample_surface(None, ctypes.byref(smp), None, None, None, None, None, 0, ctypes.byref(n), None) == E
    assert b"NULL" in lib.ddf_last_error()
