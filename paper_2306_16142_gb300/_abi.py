"""ctypes binding of include/ddf.h: one Python function per C entry point, same names,
plain integers for pointers / streams. Loading fails loudly if libddf.so is missing: there is
no fallback implementation."""

from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libddf.so")

DDF_OK = 0
DDF_ERR_INVALID_ARG = -1
DDF_ERR_CUDA = -2
DDF_ERR_OOM = -3
DDF_ERR_UNSUPPORTED = -4
DDF_ERR_TIMEOUT = -5
DDF_ERR_NUMERIC = -6
DDF_ERR_IO = -7
DDF_FP32, DDF_BF16, DDF_FP8 = 0, 1, 2
DDF_HEAD_TWO, DDF_HEAD_CLAMP, DDF_HEAD_SQUISH = 0, 1, 2
DDF_ACCEL_NONE, DDF_ACCEL_BVH = 0, 1

ERR_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "UNSUPPORTED", -5: "TIMEOUT",
             -6: "NUMERIC", -7: "IO"}


class DDFError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed: DDF_ERR_{ERR_NAMES.get(code, code)} ({code}): {msg}")
        self.code = code


class ddf_sampler(C.Structure):
    _fields_ = [("s_fc", C.c_int32), ("s_dr", C.c_int32), ("s_p", C.c_int32), ("eps", C.c_float),
                ("seed", C.c_uint64)]


class ddf_pov(C.Structure):
    _fields_ = [("n_az", C.c_int32), ("n_pol", C.c_int32), ("res", C.c_int32), ("dist", C.c_float),
                ("tan_half_fov", C.c_float)]


class ddf_arch(C.Structure):
    _fields_ = [("in_freqs", C.c_int), ("width", C.c_int), ("hidden_layers", C.c_int),
                ("precision", C.c_int)]


class ddf_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int), ("height", C.c_int),
                ("seed", C.c_uint64), ("albedo", C.c_float), ("env", C.c_float)]


class ddf_head(C.Structure):
    _fields_ = [("kind", C.c_int32), ("delta", C.c_float), ("weight_norm", C.c_int32)]


class ddf_adam(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


_P = C.c_void_p
_I64 = C.c_int64
_SIG = {
    "ddf_version": (C.c_char_p, []),
    "ddf_last_error": (C.c_char_p, []),
    "ddf_create": (C.c_int, [C.POINTER(ddf_arch), _P, C.c_size_t, C.POINTER(_P)]),
    "ddf_sphere_create": (C.c_int, [C.c_float, C.POINTER(_P)]),
    "ddf_destroy": (C.c_int, [_P]),
    "ddf_set_precision": (C.c_int, [_P, C.c_int]),
    "ddf_device_status": (C.c_int, [_P]),
    "ddf_fp8_scales": (C.c_int, [_P, _P, C.c_size_t]),
    "ddf_selftest_wait": (C.c_int, [C.c_int, C.c_int]),
    "ddf_measure_peaks": (C.c_int, [C.POINTER(C.c_double), C.c_int]),
    "ddf_num_params": (C.c_int, [_P, C.POINTER(_I64)]),
    "ddf_set_weights": (C.c_int, [_P, _P, C.c_size_t, _P]),
    "ddf_get_weights": (C.c_int, [_P, _P, C.c_size_t, _P]),
    "ddf_query": (C.c_int, [_P, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "ddf_query_noalloc": (C.c_int, [_P, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "ddf_group_create": (C.c_int, [C.c_int, _P, C.POINTER(_P)]),
    "ddf_group_destroy": (C.c_int, [_P]),
    "ddf_query_grouped": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "ddf_group_capture": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "ddf_group_replay": (C.c_int, [_P, _P]),
    "ddf_group_status": (C.c_int, [_P]),
    "ddf_group_autotune": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int, C.c_char_p, _P]),
    "ddf_group_config": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "ddf_render": (C.c_int, [_P, C.POINTER(ddf_camera), C.c_int, C.c_int, _P, _P]),
    "ddf_render_trace": (C.c_int, [_P, C.POINTER(ddf_camera), C.c_int, C.c_int, _P, _P, _I64, _P, _P, _P]),
    "ddf_render_set_wave": (C.c_int, [_P, _I64]),
    "ddf_render_stats": (C.c_int, [_P, C.POINTER(_I64), C.c_int]),
    "ddf_profile_enable": (C.c_int, [_P, C.c_int]),
    "ddf_profile_read": (C.c_int, [_P, C.POINTER(C.c_double)]),
    "ddf_mesh_create": (C.c_int, [_P, _I64, _P, _I64, C.POINTER(_P)]),
    "ddf_mesh_destroy": (C.c_int, [_P]),
    "ddf_label_rays": (C.c_int, [_P, _P, _P, _I64, _P, _P, _P, _P]),
    "ddf_sample_surface": (C.c_int, [_P, C.POINTER(ddf_sampler), _P, _P, _P, _P, _P, _I64, C.POINTER(_I64), _P]),
    "ddf_sample_pov": (C.c_int, [_P, C.POINTER(ddf_pov), _P, _P, _P, _P, _P]),
    "ddf_sample_random": (C.c_int, [_P, _I64, C.c_uint64, _P, _P, _P, _P, _P]),
    "ddf_set_head": (C.c_int, [_P, C.POINTER(ddf_head), _P]),
    "ddf_mesh_set_accel": (C.c_int, [_P, C.c_int]),
    "ddf_bvh_selfcheck": (C.c_int, [_P, _I64, _P, _I64, C.POINTER(_I64)]),
    "ddf_mesh_bvh_stats": (C.c_int, [_P, C.POINTER(_I64)]),
    "ddf_render_aov": (C.c_int, [_P, C.POINTER(ddf_camera), _P, _P, _P]),
    "ddf_udf": (C.c_int, [_P, _P, _I64, _P, C.c_int32, _P, _P, _P]),
    "ddf_mesh_render_aov": (C.c_int, [_P, C.POINTER(ddf_camera), _P, _P, _P, _P]),
    "ddf_mesh_render": (C.c_int, [_P, C.POINTER(ddf_camera), C.c_int, C.c_int, _P, _P]),
    "ddf_get_arch": (C.c_int, [_P, C.POINTER(ddf_arch)]),
    "ddf_get_weight_norm": (C.c_int, [_P, _P, C.c_size_t, _P, C.c_size_t, _P]),
    "ddf_label_stats": (C.c_int, [_P, C.POINTER(_I64)]),
    "ddf_backward": (C.c_int, [_P, _P, _P, _I64, _P, _P, _P, _P, _P]),
    "ddf_train_step": (C.c_int, [_P, _P, _P, _P, _P, _I64, C.POINTER(ddf_adam), _P, _P]),
    "ddf_set_workspace_limit": (C.c_int, [_P, C.c_size_t]),
    "ddf_forward_train": (C.c_int, [_P, _P, _P, _I64, _P, _P, _P]),
    "ddf_save": (C.c_int, [_P, C.c_char_p]),
    "ddf_load": (C.c_int, [C.c_char_p, C.POINTER(_P)]),
}

_lib = None


def declared_symbols():
    """Every function name declared in include/ddf.h (parsed from the header text)."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "ddf.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"DDF_API\s+[\w\s\*]+?\b(ddf_\w+)\s*\(", txt)))


def load():
    """Load libddf.so (building it is build.py's job). Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libddf.so not built at {LIB_PATH}: run paper_2306_16142_gb300/build.py "
                          "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH, mode=C.RTLD_GLOBAL)
    for name, (res, args) in _SIG.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def check(fn: str, rc: int):
    if rc != DDF_OK:
        raise DDFError(fn, rc, load().ddf_last_error().decode())
    return rc


def __getattr__(name):
    if name in _SIG:
        return getattr(load(), name)
    raise AttributeError(name)
