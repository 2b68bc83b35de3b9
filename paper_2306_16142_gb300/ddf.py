"""Torch-tensor conveniences over the C ABI (argument marshalling only: every step runs in
libddf.so's kernels). Tensors must be contiguous CUDA tensors of the stated dtypes; calls are
ordered on torch's current CUDA stream."""

from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi
from ._abi import check, ddf_adam, ddf_arch, ddf_camera, ddf_head, ddf_pov, ddf_sampler

PRECISIONS = {"fp32": _abi.DDF_FP32, "bf16": _abi.DDF_BF16, "fp8": _abi.DDF_FP8}
HEADS = {"two": _abi.DDF_HEAD_TWO, "clamp": _abi.DDF_HEAD_CLAMP, "squish": _abi.DDF_HEAD_SQUISH}


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _rays(o, w):
    if o.dtype != torch.float32 or w.dtype != torch.float32 or o.shape != w.shape or o.dim() != 2 \
            or o.shape[1] != 3:
        raise ValueError("origins / directions must be float32 (n, 3) tensors of equal shape")
    return o.shape[0]


class DDFNet:
    """A DDF network handle (or the closed-form sphere field, DDFNet.sphere(r))."""

    def __init__(self, in_freqs: int, width: int, hidden_layers: int, weights,
                 precision: str = "fp32"):
        lib = _abi.load()
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
        arch = ddf_arch(in_freqs, width, hidden_layers, PRECISIONS[precision])
        h = C.c_void_p()
        check("ddf_create", lib.ddf_create(C.byref(arch), w.ctypes.data_as(C.c_void_p), w.nbytes,
                                          C.byref(h)))
        self.h = h
        self.arch = (in_freqs, width, hidden_layers)
        self.precision = precision
        self.n_params = w.size

    @classmethod
    def sphere(cls, radius: float):
        obj = cls.__new__(cls)
        h = C.c_void_p()
        check("ddf_sphere_create", _abi.load().ddf_sphere_create(radius, C.byref(h)))
        obj.h = h
        obj.arch = None
        obj.precision = "fp32"
        obj.n_params = 0
        return obj

    @classmethod
    def load(cls, path: str):
        """A new handle from a checkpoint written by save() (weights, precision, Adam state)."""
        obj = cls.__new__(cls)
        h = C.c_void_p()
        check("ddf_load", _abi.load().ddf_load(str(path).encode(), C.byref(h)))
        obj.h = h
        n = C.c_int64()
        check("ddf_num_params", _abi.load().ddf_num_params(h, C.byref(n)))
        obj.n_params = n.value
        a = ddf_arch()
        check("ddf_get_arch", _abi.load().ddf_get_arch(h, C.byref(a)))
        obj.arch = (a.in_freqs, a.width, a.hidden_layers)
        obj.precision = {v: k for k, v in PRECISIONS.items()}[a.precision]
        return obj

    def save(self, path: str):
        check("ddf_save", _abi.load().ddf_save(self.h, str(path).encode()))

    def close(self):
        if getattr(self, "h", None):
            _abi.load().ddf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self):
        """Raise DDFError(TIMEOUT) if a bounded device wait of this handle gave up."""
        check("ddf_device_status", _abi.load().ddf_device_status(self.h))

    def fp8_scales(self):
        """The FP8 path's static activation scales, float32 numpy [L, width] (layer 0: 1/448)."""
        if self.arch is None:
            raise ValueError("architecture unknown for this handle")
        _, width, layers = self.arch
        out = np.empty((layers, width), np.float32)
        check("ddf_fp8_scales", _abi.load().ddf_fp8_scales(self.h, out.ctypes.data, out.nbytes))
        return out

    def set_precision(self, precision: str):
        check("ddf_set_precision", _abi.load().ddf_set_precision(self.h, PRECISIONS[precision]))
        self.precision = precision

    def set_head(self, kind: str = "two", delta: float = 0.0, weight_norm: bool = False):
        """Head and training variant (ddf_set_head): "two" (distance + hit logit), or the
        paper's single field value with the clamp loss of Eq. 7 ("clamp") or the squish loss of
        Eq. 5 ("squish"), hit <=> value < delta; weight_norm trains the hidden layers as g v / |v|."""
        h = ddf_head(HEADS[kind], delta, int(bool(weight_norm)))
        check("ddf_set_head", _abi.load().ddf_set_head(self.h, C.byref(h), _stream()))

    def weight_norm_state(self):
        """(v, g): v in the blob layout (v in the hidden-weight slots), g [L * width]."""
        if self.arch is None:
            raise ValueError("architecture unknown for this handle")
        _, width, layers = self.arch
        v = torch.empty(self.n_params, device="cuda")
        g = torch.empty(layers * width, device="cuda")
        check("ddf_get_weight_norm", _abi.load().ddf_get_weight_norm(self.h, _ptr(v), v.numel() * 4, _ptr(g),
                                                                     g.numel() * 4, _stream()))
        return v, g

    def query(self, o: torch.Tensor, w: torch.Tensor, normals: bool = False, out=None):
        n = _rays(o, w)
        dev = o.device
        if out is None:
            out = {"dist": torch.empty(n, device=dev), "hit": torch.empty(n, dtype=torch.uint8, device=dev),
                   "logit": torch.empty(n, device=dev),
                   "normal": torch.zeros(n, 3, device=dev) if normals else None}
        check("ddf_query", _abi.load().ddf_query(self.h, _ptr(o), _ptr(w), n, _ptr(out["dist"]),
                                                 _ptr(out["hit"]), _ptr(out["logit"]),
                                                 _ptr(out.get("normal")), _stream()))
        return out

    def render(self, cam, spp: int, bounces: int, image: torch.Tensor | None = None):
        c = camera_struct(cam)
        if image is None:
            image = torch.empty(cam.height, cam.width, device="cuda")
        check("ddf_render", _abi.load().ddf_render(self.h, C.byref(c), spp, bounces, _ptr(image),
                                                   _stream()))
        return image

    def render_trace(self, cam, spp: int, bounces: int, pids: torch.Tensor, image: torch.Tensor | None = None):
        """ddf_render plus a record of every bounce of the paths in pids (CUDA int64): returns
        (image, trace, radiance), trace (len(pids), bounces, 12) = o, w, dist, logit, normal,
        throughput of each bounce's query (NaN where the path did not get that far)."""
        c = camera_struct(cam)
        if image is None:
            image = torch.empty(cam.height, cam.width, device="cuda")
        if pids.dtype != torch.int64:
            raise ValueError("pids must be an int64 tensor")
        n = pids.numel()
        trace = torch.empty(max(n, 1), bounces, 12, device="cuda")
        rad = torch.empty(max(n, 1), device="cuda")
        check("ddf_render_trace", _abi.load().ddf_render_trace(self.h, C.byref(c), spp, bounces, _ptr(image),
                                                               _ptr(pids), n, _ptr(trace), _ptr(rad), _stream()))
        return image, trace[:n], rad[:n]

    def set_wave(self, max_paths: int):
        """Paths per render wave (ddf_render_set_wave; default 2^24)."""
        check("ddf_render_set_wave", _abi.load().ddf_render_set_wave(self.h, max_paths))

    def render_aov(self, cam):
        """Depth (H, W; distance from the eye, inf on a miss) and normal (H, W, 3) maps of one
        primary ray per pixel (ddf_render_aov)."""
        c = camera_struct(cam)
        depth = torch.empty(cam.height, cam.width, device="cuda")
        normal = torch.empty(cam.height, cam.width, 3, device="cuda")
        check("ddf_render_aov", _abi.load().ddf_render_aov(self.h, C.byref(c), _ptr(depth), _ptr(normal), _stream()))
        return depth, normal

    def udf(self, points: torch.Tensor, dirs: torch.Tensor, with_arg: bool = False):
        """Eq. 4 over a direction set (ddf_udf): the minimum distance over the directions whose ray
        hits, per point (inf if none); with_arg also returns the minimising direction index."""
        if points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 3 or dirs.dim() != 2 \
                or dirs.shape[1] != 3 or dirs.dtype != torch.float32:
            raise ValueError("points and dirs must be float32 (n, 3) tensors")
        n = points.shape[0]
        out = torch.empty(n, device=points.device)
        arg = torch.empty(n, dtype=torch.int32, device=points.device) if with_arg else None
        check("ddf_udf", _abi.load().ddf_udf(self.h, _ptr(points), n, _ptr(dirs), dirs.shape[0], _ptr(out), _ptr(arg),
                                             _stream()))
        return (out, arg) if with_arg else out

    def render_stats(self, bounces: int):
        arr = (C.c_int64 * bounces)()
        check("ddf_render_stats", _abi.load().ddf_render_stats(self.h, arr, bounces))
        return list(arr)

    def profile(self, enable: bool = True):
        check("ddf_profile_enable", _abi.load().ddf_profile_enable(self.h, int(enable)))

    def profile_read(self):
        arr = (C.c_double * 8)()
        check("ddf_profile_read", _abi.load().ddf_profile_read(self.h, arr))
        keys = ["query", "shade", "raygen", "accumulate"]
        return {k: {"ms": arr[2 * i], "launches": int(arr[2 * i + 1])} for i, k in enumerate(keys)}

    def set_weights(self, wt: torch.Tensor):
        check("ddf_set_weights", _abi.load().ddf_set_weights(self.h, _ptr(wt), wt.numel() * 4, _stream()))

    def get_weights(self) -> torch.Tensor:
        out = torch.empty(self.n_params, device="cuda")
        check("ddf_get_weights", _abi.load().ddf_get_weights(self.h, _ptr(out), out.numel() * 4, _stream()))
        return out

    def forward_train(self, o, w):
        """(dist, logit) of the training forward pass."""
        n = _rays(o, w)
        dist = torch.empty(n, device=o.device)
        logit = torch.empty(n, device=o.device)
        check("ddf_forward_train", _abi.load().ddf_forward_train(self.h, _ptr(o), _ptr(w), n, _ptr(dist),
                                                                 _ptr(logit), _stream()))
        return dist, logit

    def backward(self, o, w, gdist, glogit, need_input: bool = False):
        n = _rays(o, w)
        gw = torch.empty(self.n_params, device=o.device)
        gin = torch.empty(n, 6, device=o.device) if need_input else None
        check("ddf_backward", _abi.load().ddf_backward(self.h, _ptr(o), _ptr(w), n, _ptr(gdist),
                                                       _ptr(glogit), _ptr(gw), _ptr(gin), _stream()))
        return gw, gin

    def train_step(self, o, w, dist_gt, hit_gt, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, loss=None):
        n = _rays(o, w)
        if loss is None:
            loss = torch.empty((), device=o.device)
        opt = ddf_adam(lr, beta1, beta2, eps)
        check("ddf_train_step", _abi.load().ddf_train_step(self.h, _ptr(o), _ptr(w), _ptr(dist_gt),
                                                           _ptr(hit_gt), n, C.byref(opt), _ptr(loss),
                                                           _stream()))
        return loss

    def set_workspace_limit(self, nbytes: int):
        check("ddf_set_workspace_limit", _abi.load().ddf_set_workspace_limit(self.h, nbytes))


class DDFMesh:
    """A triangle mesh prepared for ray labelling."""

    ACCEL = {"none": _abi.DDF_ACCEL_NONE, "bvh": _abi.DDF_ACCEL_BVH}

    def __init__(self, verts, tris, accel: str = "bvh"):
        v = np.ascontiguousarray(np.asarray(verts, np.float32))
        t = np.ascontiguousarray(np.asarray(tris, np.int32))
        h = C.c_void_p()
        check("ddf_mesh_create", _abi.load().ddf_mesh_create(v.ctypes.data_as(C.c_void_p), v.shape[0],
                                                             t.ctypes.data_as(C.c_void_p), t.shape[0],
                                                             C.byref(h)))
        self.h = h
        self.nt = t.shape[0]
        self.set_accel(accel)

    def set_accel(self, accel: str):
        """Face search of every labelling call: "bvh" (hierarchy) or "none" (all faces); the labels
        are the same either way (ddf_mesh_set_accel)."""
        check("ddf_mesh_set_accel", _abi.load().ddf_mesh_set_accel(self.h, self.ACCEL[accel]))
        self.accel = accel

    def close(self):
        if getattr(self, "h", None):
            _abi.load().ddf_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def label(self, o, w, out=None):
        n = _rays(o, w)
        if out is None:
            out = {"dist": torch.empty(n, device=o.device), "hit": torch.empty(n, dtype=torch.uint8, device=o.device),
                   "tri": torch.empty(n, dtype=torch.int32, device=o.device)}
        check("ddf_label_rays", _abi.load().ddf_label_rays(self.h, _ptr(o), _ptr(w), n, _ptr(out["dist"]),
                                                           _ptr(out["hit"]), _ptr(out.get("tri")), _stream()))
        return out

    def stats(self):
        arr = (C.c_int64 * 2)()
        check("ddf_label_stats", _abi.load().ddf_label_stats(self.h, arr))
        return {"retests": arr[0], "finals": arr[1]}

    def bvh_stats(self):
        """Hierarchy size and depth, and the node visits and face tests of the last labelling call."""
        arr = (C.c_int64 * 4)()
        check("ddf_mesh_bvh_stats", _abi.load().ddf_mesh_bvh_stats(self.h, arr))
        return {"nodes": arr[0], "depth": arr[1], "visits": arr[2], "face_tests": arr[3]}

    def render(self, cam, spp: int, bounces: int, image: torch.Tensor | None = None):
        """The path tracer with the mesh in place of the field (ddf_mesh_render)."""
        c = camera_struct(cam)
        if image is None:
            image = torch.empty(cam.height, cam.width, device="cuda")
        check("ddf_mesh_render", _abi.load().ddf_mesh_render(self.h, C.byref(c), spp, bounces, _ptr(image),
                                                             _stream()))
        return image

    def render_aov(self, cam):
        """Depth, normal and hit-face maps of the camera's pixel rays cast against the mesh
        (ddf_mesh_render_aov)."""
        c = camera_struct(cam)
        depth = torch.empty(cam.height, cam.width, device="cuda")
        normal = torch.empty(cam.height, cam.width, 3, device="cuda")
        tri = torch.empty(cam.height, cam.width, dtype=torch.int32, device="cuda")
        check("ddf_mesh_render_aov", _abi.load().ddf_mesh_render_aov(self.h, C.byref(c), _ptr(depth), _ptr(normal),
                                                                     _ptr(tri), _stream()))
        return depth, normal, tri

    @staticmethod
    def sample_buffers(cap: int):
        """Output tensors for sample_surface holding up to cap samples."""
        dev = torch.device("cuda")
        n = max(cap, 1)
        return {"o": torch.empty(n, 3, device=dev), "w": torch.empty(n, 3, device=dev),
                "dist": torch.empty(n, device=dev), "hit": torch.empty(n, dtype=torch.uint8, device=dev),
                "key": torch.empty(n, dtype=torch.int64, device=dev)}

    def sample_surface(self, s_fc: int, s_dr: int, s_p: int, eps: float = 1e-4, seed: int = 0,
                       cap: int | None = None, out: dict | None = None):
        """The surface-marching training set of Sec. 5.2 (ddf_sample_surface): dict of CUDA
        tensors o (n, 3), w (n, 3), dist (n,), hit (n,) and key (n,), in key order, and the
        total count (which may exceed cap). out: buffers from sample_buffers to reuse; cap
        defaults to their size, else to the 4 s_p samples of every candidate."""
        if out is None:
            cap = self.nt * s_fc * s_dr * s_p * 4 if cap is None else cap
            out = self.sample_buffers(cap)
        else:
            room = out["key"].shape[0]
            cap = room if cap is None else min(cap, room)
        prm = ddf_sampler(s_fc, s_dr, s_p, eps, seed)
        n = C.c_int64()
        check("ddf_sample_surface", _abi.load().ddf_sample_surface(
            self.h, C.byref(prm), _ptr(out["o"]), _ptr(out["w"]), _ptr(out["dist"]), _ptr(out["hit"]),
            _ptr(out["key"]), cap, C.byref(n), _stream()))
        k = min(n.value, cap)
        res = {name: t[:k] for name, t in out.items()}
        res["count"] = n.value
        return res

    def sample_random(self, n: int, seed: int = 0):
        """The random training set of Sec. 6 (ddf_sample_random): dict of CUDA tensors o, w (n, 3),
        dist (n,), hit (n,)."""
        dev = torch.device("cuda")
        out = {"o": torch.empty(max(n, 1), 3, device=dev), "w": torch.empty(max(n, 1), 3, device=dev),
               "dist": torch.empty(max(n, 1), device=dev), "hit": torch.empty(max(n, 1), dtype=torch.uint8, device=dev)}
        check("ddf_sample_random", _abi.load().ddf_sample_random(
            self.h, n, seed, _ptr(out["o"]), _ptr(out["w"]), _ptr(out["dist"]), _ptr(out["hit"]), _stream()))
        return {k: t[:n] for k, t in out.items()}

    def sample_pov(self, n_az: int = 10, n_pol: int = 5, res: int = 64, dist: float = 2.5,
                   tan_half_fov: float = 0.2679491924311227, out: dict | None = None):
        """The point-of-view training set of Sec. 6 (ddf_sample_pov): dict of CUDA tensors o
        (N, 3), w (N, 3), dist (N,), hit (N,), N = n_az n_pol res^2, camera by camera, rows from
        the top. The default field of view is 30 degrees."""
        n = n_az * n_pol * res * res
        if out is None:
            dev = torch.device("cuda")
            out = {"o": torch.empty(max(n, 1), 3, device=dev), "w": torch.empty(max(n, 1), 3, device=dev),
                   "dist": torch.empty(max(n, 1), device=dev),
                   "hit": torch.empty(max(n, 1), dtype=torch.uint8, device=dev)}
        elif out["hit"].shape[0] < n:
            raise ValueError("output buffers hold fewer than n_az n_pol res^2 rows")
        prm = ddf_pov(n_az, n_pol, res, dist, tan_half_fov)
        check("ddf_sample_pov", _abi.load().ddf_sample_pov(
            self.h, C.byref(prm), _ptr(out["o"]), _ptr(out["w"]), _ptr(out["dist"]), _ptr(out["hit"]), _stream()))
        return {name: t[:n] for name, t in out.items()}


def measure_peaks():
    """Measured FP32 / FP32x2 / FP64 FMA and BF16 / FP8 tensor-core throughput of the current
    device in TFLOP/s, and its SM count (ddf_measure_peaks)."""
    arr = (C.c_double * 7)()
    check("ddf_measure_peaks", _abi.load().ddf_measure_peaks(arr, 7))
    return {"fp32_fma_tflops": arr[0], "fp32x2_fma_tflops": arr[1], "fp64_fma_tflops": arr[2],
            "bf16_mma_tflops": arr[3], "fp8_mma_tflops": arr[4], "sms": int(arr[5])}


def camera_struct(cam) -> ddf_camera:
    c = ddf_camera()
    for k in range(3):
        c.eye[k] = cam.eye[k]
        c.look_at[k] = cam.look_at[k]
        c.up[k] = cam.up[k]
    c.vfov_deg = cam.vfov_deg
    c.width = cam.width
    c.height = cam.height
    c.seed = cam.seed
    c.albedo = cam.albedo
    c.env = cam.env
    return c


class DDFGroup:
    """Several BF16 networks queried together (ddf_query_grouped): rows of object i are
    [offsets[i], offsets[i+1]) of the concatenated ray tensors; offsets is a CUDA int64 tensor."""

    def __init__(self, nets):
        self.nets = list(nets)
        arr = (C.c_void_p * len(self.nets))(*[n.h.value for n in self.nets])
        h = C.c_void_p()
        check("ddf_group_create", _abi.load().ddf_group_create(len(self.nets), arr, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _abi.load().ddf_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _out(n, dev):
        return {"dist": torch.empty(n, device=dev), "hit": torch.empty(n, dtype=torch.uint8, device=dev),
                "logit": torch.empty(n, device=dev)}

    def query(self, offsets, o, w, out=None):
        n = _rays(o, w)
        out = out or self._out(n, o.device)
        check("ddf_query_grouped", _abi.load().ddf_query_grouped(
            self.h, _ptr(offsets), _ptr(o), _ptr(w), _ptr(out["dist"]), _ptr(out["hit"]), _ptr(out["logit"]),
            _stream()))
        return out

    def capture(self, offsets, o, w, out):
        check("ddf_group_capture", _abi.load().ddf_group_capture(
            self.h, _ptr(offsets), _ptr(o), _ptr(w), _ptr(out["dist"]), _ptr(out["hit"]), _ptr(out["logit"]),
            _stream()))

    def replay(self):
        check("ddf_group_replay", _abi.load().ddf_group_replay(self.h, _stream()))

    def status(self):
        check("ddf_group_status", _abi.load().ddf_group_status(self.h))

    def autotune(self, offsets, o, w, out, reps=3, cache_path=None):
        check("ddf_group_autotune", _abi.load().ddf_group_autotune(
            self.h, _ptr(offsets), _ptr(o), _ptr(w), _ptr(out["dist"]), _ptr(out["hit"]), reps,
            cache_path.encode() if cache_path else None, _stream()))
        cfg = (C.c_int * 9)()
        check("ddf_group_config", _abi.load().ddf_group_config(self.h, cfg))
        return [(cfg[3 * c], cfg[3 * c + 1], cfg[3 * c + 2]) for c in range(3) if cfg[3 * c]]
