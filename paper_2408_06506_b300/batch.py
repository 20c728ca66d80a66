"""Binding of the batched tactile step (``include/tacsl_batch.h``): pads with their own
taxel layout, object and sensor model in one pair of launches, an autotuner over the
launch configuration, and CUDA-graph replay.

Argument marshalling only, like the rest of the package: numpy arrays describe the
batch on the host, torch CUDA tensors hold the device buffers, and every step runs in
``libtacsl.so``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _Camera, _Params, _SdfSet, _check, _dev, _ptr, _stream, load

MAX_MODEL = 64

_P, _I32, _I64 = C.c_void_p, C.c_int32, C.c_int64


class _SensorModel(C.Structure):
    _fields_ = [("H", _I32), ("W", _I32), ("pitch_x", C.c_float), ("pitch_y", C.c_float), ("coeffs", _P)]


class _SensorSet(C.Structure):
    _fields_ = [("models", C.POINTER(_SensorModel)), ("n_model", _I32)]


class _BatchDesc(C.Structure):
    _fields_ = [("n_pad", _I32), ("obj_id", _P), ("layout", _P), ("sensor", _P), ("n_layout", _I32),
                ("layout_first", _P), ("layout_count", _P), ("n_points", _I64)]


class _Plan(C.Structure):
    _fields_ = [("n_pad", _I32), ("n_image", _I32), ("n_taxel_out", _I64), ("n_pixel_out", _I64),
                ("workspace_bytes", _I64), ("img_block", _I32), ("n_stages", _I32), ("force_np", _I32),
                ("force_dynamic", _I32), ("n_model", _I32), ("max_w", _I32),
                ("model_h", _I32 * MAX_MODEL), ("model_w", _I32 * MAX_MODEL),
                ("model_img_begin", _I32 * (MAX_MODEL + 1)), ("off_sched", _I64), ("off_images", _I64),
                ("fingerprint", C.c_uint64)]


class _BatchIO(C.Structure):
    _fields_ = [(n, _P) for n in ("taxels", "pad_pose", "pad_twist", "depth", "f_n", "f_t", "wrench", "depth_map",
                                  "rgb")]


_bound = False


def _lib():
    global _bound
    lib = load()
    if not _bound:
        PP, PS, PD, PI = C.POINTER(_Plan), C.POINTER(_SensorSet), C.POINTER(_BatchDesc), C.POINTER(_BatchIO)
        PSdf, PPrm = C.POINTER(_SdfSet), C.POINTER(_Params)
        sig = {
            "tacsl_batch_plan_create": [PD, PS, PP, _P, _P],
            "tacsl_batch_pack": [PP, PD, _P],
            "tacsl_batch_upload": [PP, PD, _P, _P],
            "tacsl_batch_forces": [PP, _P, PSdf, PPrm, PI, _P],
            "tacsl_batch_shade": [PP, _P, PS, PI, _P],
            "tacsl_batch_step": [PP, _P, PSdf, PPrm, PS, PI, _P],
            "tacsl_batch_render": [PP, _P, PSdf, C.POINTER(_Camera), _P, _P, _P],
            "tacsl_batch_autotune": [PP, _P, PSdf, PPrm, PS, PI, _I32, C.POINTER(C.c_double), _P],
            "tacsl_batch_graph_create": [PP, _P, PSdf, PPrm, PS, PI, C.POINTER(_P)],
            "tacsl_graph_launch": [_P, _P],
            "tacsl_graph_destroy": [_P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.restype = C.c_int
            f.argtypes = args
        _bound = True
    return lib


def cameras_array(cameras):
    """A ctypes array of tacsl_camera from a list of tacsl.Camera (None for an empty list)."""
    if not cameras:
        return None
    arr = (_Camera * len(cameras))()
    for m, c in enumerate(cameras):
        arr[m] = c.c
    return arr


class SensorSet:
    """Sensor models of a batch: a list of (coeffs [6, 3, H, W] float32 CUDA tensor,
    pitch_x, pitch_y); H and W multiples of 4."""

    def __init__(self, models):
        self.tensors = []
        self.sizes = []
        self._arr = (_SensorModel * max(1, len(models)))()
        for m, (coeffs, px, py) in enumerate(models):
            _dev(coeffs, torch.float32, f"models[{m}].coeffs")
            six, three, H, W = coeffs.shape
            if (six, three) != (6, 3):
                raise ValueError("coeffs must be [6, 3, H, W]")
            self.tensors.append(coeffs)
            self.sizes.append((H, W))
            self._arr[m] = _SensorModel(H, W, float(px), float(py), coeffs.data_ptr())
        self.c = _SensorSet(C.cast(self._arr, C.POINTER(_SensorModel)), len(models))

    @classmethod
    def sizes_only(cls, sizes):
        """Geometry for planning on a host without a GPU (coefficient pointers unset)."""
        self = cls.__new__(cls)
        self.tensors, self.sizes = [], list(sizes)
        self._arr = (_SensorModel * max(1, len(sizes)))()
        for m, (H, W) in enumerate(sizes):
            self._arr[m] = _SensorModel(int(H), int(W), 1.0, 1.0, None)
        self.c = _SensorSet(C.cast(self._arr, C.POINTER(_SensorModel)), len(sizes))
        return self


class BatchPlan:
    """Plan + device workspace of one batch.

    obj_id, layout, sensor: per pad (int, sensor -1 for no image); layout_first,
    layout_count: per taxel layout (first point in the taxel pool, point count);
    n_points: points in the taxel pool (default: the end of the last layout).
    ``device=None`` plans on the host only (no workspace)."""

    def __init__(self, obj_id, layout, sensor, layout_first, layout_count, sensors: SensorSet | None,
                 device="cuda", stream=None, n_points=None):
        self._h = {
            "obj_id": np.ascontiguousarray(obj_id, np.int32),
            "layout": np.ascontiguousarray(layout, np.int32),
            "sensor": np.ascontiguousarray(sensor, np.int32),
            "layout_first": np.ascontiguousarray(layout_first, np.int64),
            "layout_count": np.ascontiguousarray(layout_count, np.int32),
        }
        h = self._h
        n_pad = h["obj_id"].shape[0]
        if h["layout"].shape[0] != n_pad or h["sensor"].shape[0] != n_pad:
            raise ValueError("obj_id, layout and sensor must have one entry per pad")
        if n_points is None:
            n_points = int((h["layout_first"] + h["layout_count"]).max(initial=0))
        self.desc = _BatchDesc(n_pad, h["obj_id"].ctypes.data, h["layout"].ctypes.data, h["sensor"].ctypes.data,
                               h["layout_count"].shape[0], h["layout_first"].ctypes.data,
                               h["layout_count"].ctypes.data, int(n_points))
        self.sensors = sensors
        self.plan = _Plan()
        self.taxel_offset = np.zeros(n_pad, np.int64)
        self.pixel_offset = np.zeros(n_pad, np.int64)
        _check(_lib().tacsl_batch_plan_create(C.byref(self.desc), C.byref(sensors.c) if sensors else None,
                                              C.byref(self.plan), self.taxel_offset.ctypes.data,
                                              self.pixel_offset.ctypes.data))
        self.workspace = None
        if device is not None:
            self.workspace = torch.empty(max(256, self.plan.workspace_bytes), dtype=torch.uint8, device=device)
            _check(_lib().tacsl_batch_upload(C.byref(self.plan), C.byref(self.desc), _ptr(self.workspace),
                                             _stream(stream)))

    @property
    def n_pad(self):
        return self.plan.n_pad

    @property
    def n_taxel_out(self):
        return self.plan.n_taxel_out

    @property
    def n_pixel_out(self):
        return self.plan.n_pixel_out

    def config(self) -> dict:
        p = self.plan
        return {"img_block": p.img_block, "n_stages": p.n_stages, "force_np": p.force_np,
                "force_dynamic": p.force_dynamic}

    def set_config(self, img_block=None, n_stages=None, force_np=None, force_dynamic=None):
        for k, v in (("img_block", img_block), ("n_stages", n_stages), ("force_np", force_np),
                     ("force_dynamic", force_dynamic)):
            if v is not None:
                setattr(self.plan, k, int(v))

    def pack(self) -> np.ndarray:
        """The workspace bytes, built on the host."""
        buf = np.zeros(self.plan.workspace_bytes, np.uint8)
        _check(_lib().tacsl_batch_pack(C.byref(self.plan), C.byref(self.desc), buf.ctypes.data))
        return buf

    def outputs(self, device="cuda", with_wrench=True, with_images=True) -> dict:
        nt, npx = self.plan.n_taxel_out, self.plan.n_pixel_out
        out = {
            "depth": torch.empty(nt, dtype=torch.float32, device=device),
            "f_n": torch.empty(nt, 3, dtype=torch.float32, device=device),
            "f_t": torch.empty(nt, 3, dtype=torch.float32, device=device),
            "wrench": torch.empty(self.n_pad, 6, dtype=torch.float32, device=device) if with_wrench else None,
        }
        if with_images:
            out["rgb"] = torch.empty(max(npx, 1), 3, dtype=torch.uint8, device=device)[:npx]
        return out

    def _io(self, taxels=None, pose=None, twist=None, out=None, depth_map=None):
        out = out or {}
        for t, n, dt in ((taxels, "taxels", torch.float32), (pose, "pad_pose", torch.float32),
                         (twist, "pad_twist", torch.float32), (depth_map, "depth_map", torch.float32)):
            if t is not None:
                _dev(t, dt, n)
        io = _BatchIO(_ptr(taxels), _ptr(pose), _ptr(twist), _ptr(out.get("depth")), _ptr(out.get("f_n")),
                      _ptr(out.get("f_t")), _ptr(out.get("wrench")), _ptr(depth_map), _ptr(out.get("rgb")))
        return io

    def forces(self, sdfs, params, taxels, pose, twist, out=None, stream=None) -> dict:
        out = out or self.outputs(pose.device, with_images=False)
        io = self._io(taxels, pose, twist, out)
        _check(_lib().tacsl_batch_forces(C.byref(self.plan), _ptr(self.workspace), C.byref(sdfs.c),
                                         C.byref(params.c), C.byref(io), _stream(stream)))
        return out

    def shade(self, depth_map, rgb=None, stream=None):
        if rgb is None:
            rgb = torch.empty(self.plan.n_pixel_out, 3, dtype=torch.uint8, device=depth_map.device)
        io = self._io(depth_map=depth_map, out={"rgb": rgb})
        _check(_lib().tacsl_batch_shade(C.byref(self.plan), _ptr(self.workspace), C.byref(self.sensors.c),
                                        C.byref(io), _stream(stream)))
        return rgb

    def render(self, sdfs, cameras, pose, depth_map=None, stream=None):
        """Packed depth maps [n_pixel_out] of every pad with an image, rendered from its pose
        (cameras: one tacsl.Camera per sensor model of the plan)."""
        _dev(pose, torch.float32, "pad_pose")
        if depth_map is None:
            depth_map = torch.empty(max(self.plan.n_pixel_out, 4), dtype=torch.float32, device=pose.device)
        cams = cameras_array(cameras)
        _check(_lib().tacsl_batch_render(C.byref(self.plan), _ptr(self.workspace), C.byref(sdfs.c), cams,
                                         _ptr(pose), _ptr(depth_map), _stream(stream)))
        return depth_map

    def step(self, sdfs, params, taxels, pose, twist, depth_map, out=None, stream=None) -> dict:
        out = out or self.outputs(pose.device)
        io = self._io(taxels, pose, twist, out, depth_map)
        _check(_lib().tacsl_batch_step(C.byref(self.plan), _ptr(self.workspace), C.byref(sdfs.c), C.byref(params.c),
                                       C.byref(self.sensors.c) if self.sensors else None, C.byref(io),
                                       _stream(stream)))
        return out

    def autotune(self, sdfs, params, taxels, pose, twist, depth_map, out=None, reps=3, stream=None) -> float:
        """Pick the fastest launch configuration on these buffers; returns its step time (ms)."""
        out = out or self.outputs(pose.device)
        io = self._io(taxels, pose, twist, out, depth_map)
        best = C.c_double(0.0)
        _check(_lib().tacsl_batch_autotune(C.byref(self.plan), _ptr(self.workspace), C.byref(sdfs.c),
                                           C.byref(params.c), C.byref(self.sensors.c) if self.sensors else None,
                                           C.byref(io), int(reps), C.byref(best), _stream(stream)))
        return best.value

    def graph(self, sdfs, params, taxels, pose, twist, depth_map, out) -> "BatchGraph":
        """One step captured as a CUDA graph over these buffers (replay with .launch())."""
        io = self._io(taxels, pose, twist, out, depth_map)
        h = _P()
        _check(_lib().tacsl_batch_graph_create(C.byref(self.plan), _ptr(self.workspace), C.byref(sdfs.c),
                                               C.byref(params.c), C.byref(self.sensors.c) if self.sensors else None,
                                               C.byref(io), C.byref(h)))
        return BatchGraph(h, keep=(self, sdfs, params, taxels, pose, twist, depth_map, out))


class BatchGraph:
    """An instantiated CUDA graph of one batch step; holds its buffers alive."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def launch(self, stream=None):
        _check(_lib().tacsl_graph_launch(self._h, _stream(stream)))

    def close(self):
        if self._h is not None and self._h.value:
            _lib().tacsl_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
