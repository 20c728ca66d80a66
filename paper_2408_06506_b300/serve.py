"""Binding of the continuous-batching server (``include/tacsl_serve.h``).

The server runs inside ``libtacsl.so`` (a C++ worker thread driving the batched
kernels); this module marshals requests: numpy / torch CPU arrays in, torch CPU
(optionally pinned) outputs back.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import TacslError, _Camera, _check, _SdfSet, load
from .batch import MAX_MODEL, SensorSet, _SensorSet, cameras_array   # noqa: F401

_P, _I32, _I64 = C.c_void_p, C.c_int32, C.c_int64
TACSL_ERR_TIMEOUT = 4


class _Config(C.Structure):
    _fields_ = [("hbm_budget_bytes", _I64), ("max_pads", _I32), ("n_streams", _I32), ("batch_timeout_ms", _I32)]


class _Request(C.Structure):
    _fields_ = [("n_pad", _I32)] + [(n, _P) for n in (
        "obj_id", "layout", "sensor", "pad_pose", "pad_twist", "k_n", "k_d", "k_t", "mu", "depth_map", "depth", "f_n",
        "f_t", "wrench", "rgb")]


class _PoseRequest(C.Structure):
    _fields_ = [("n_pad", _I32)] + [(n, _P) for n in (
        "obj_id", "layout", "sensor", "pad_pose", "pad_twist", "k_n", "k_d", "k_t", "mu", "wrench", "depth", "f_n",
        "f_t", "rgb", "depth_map")]


class _Stats(C.Structure):
    _fields_ = [(n, _I64) for n in ("submitted", "completed", "batches", "pads_served", "arena_bytes",
                                    "arena_peak_bytes", "arena_used_bytes")] + [("max_batch_requests", _I32),
                                                                                ("pending", _I32)]


_bound = False


def _lib():
    global _bound
    lib = load()
    if not _bound:
        sig = {
            "tacsl_server_create": [C.POINTER(_Config), C.POINTER(_SdfSet), C.POINTER(_SensorSet), _P, _I64, _I32, _P,
                                    _P, C.POINTER(_P)],
            "tacsl_server_submit": [_P, C.POINTER(_Request), C.POINTER(_I64)],
            "tacsl_server_set_cameras": [_P, C.POINTER(_Camera), _I32],
            "tacsl_server_submit_poses": [_P, C.POINTER(_PoseRequest), C.POINTER(_I64)],
            "tacsl_server_wait": [_P, _I64, _I32, C.POINTER(_I32), C.POINTER(C.c_double)],
            "tacsl_server_get_stats": [_P, C.POINTER(_Stats)],
            "tacsl_server_destroy": [_P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.restype = C.c_int
            f.argtypes = args
        _bound = True
    return lib


def _host(a, dtype):
    """A contiguous host array of dtype (torch CPU tensors and numpy arrays accepted as is)."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise TypeError("request arrays live in host memory")
        t = a.contiguous()
        if t.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {t.dtype}")
        return t, t.data_ptr()
    n = np.ascontiguousarray(a, dtype={torch.float32: np.float32, torch.int32: np.int32,
                                        torch.uint8: np.uint8}[dtype])
    return n, n.ctypes.data


class Server:
    """Continuous-batching server over resident SDFs, sensor models and taxel layouts.

    sdfs: SdfSet; sensors: SensorSet or None; taxels: CUDA tensor [n_points, 3] (the
    pool); layout_first / layout_count: host arrays per layout."""

    def __init__(self, sdfs, sensors, taxels, layout_first, layout_count, hbm_budget_bytes, max_pads=65536,
                 n_streams=2, batch_timeout_ms=10000):
        self._keep = (sdfs, sensors, taxels)
        self.layout_first = np.ascontiguousarray(layout_first, np.int64)
        self.layout_count = np.ascontiguousarray(layout_count, np.int32)
        self.sizes = list(sensors.sizes) if sensors is not None else []
        cfg = _Config(int(hbm_budget_bytes), int(max_pads), int(n_streams), int(batch_timeout_ms))
        h = _P()
        _check(_lib().tacsl_server_create(C.byref(cfg), C.byref(sdfs.c), C.byref(sensors.c) if sensors else None,
                                          C.c_void_p(taxels.data_ptr()), taxels.shape[0], len(self.layout_count),
                                          self.layout_first.ctypes.data, self.layout_count.ctypes.data, C.byref(h)))
        self._h = h
        self._live = {}
        self._late = []

    def sizes_of(self, layout, sensor):
        """(taxels, pixels) of a request's outputs."""
        layout, sensor = np.asarray(layout), np.asarray(sensor)
        nt = int(self.layout_count[layout].sum())
        npx = int(sum(self.sizes[s][0] * self.sizes[s][1] for s in sensor if s >= 0))
        return nt, npx

    def outputs_for(self, layout, sensor, pin=True):
        nt, npx = self.sizes_of(layout, sensor)
        mk = (lambda *s, dtype=torch.float32: torch.empty(*s, dtype=dtype).pin_memory()) if pin else \
            (lambda *s, dtype=torch.float32: torch.empty(*s, dtype=dtype))
        return {"depth": mk(nt), "f_n": mk(nt, 3), "f_t": mk(nt, 3), "wrench": mk(len(layout), 6),
                "rgb": mk(max(npx, 1), 3, dtype=torch.uint8)}

    def submit(self, obj_id, layout, sensor, pad_pose, pad_twist, k_n, k_d, k_t, mu, depth_map, out) -> int:
        """Queue one request; its host arrays are kept alive until its wait returns."""
        keep = []

        def h(a, dt):
            arr, ptr = _host(a, dt)
            keep.append(arr)
            return ptr

        n = len(obj_id)
        req = _Request(n, h(obj_id, torch.int32), h(layout, torch.int32), h(sensor, torch.int32),
                       h(pad_pose, torch.float32), h(pad_twist, torch.float32), h(k_n, torch.float32),
                       h(k_d, torch.float32), h(k_t, torch.float32), h(mu, torch.float32),
                       h(depth_map, torch.float32) if depth_map is not None else None,
                       h(out["depth"], torch.float32), h(out["f_n"], torch.float32), h(out["f_t"], torch.float32),
                       h(out["wrench"], torch.float32) if out.get("wrench") is not None else None,
                       h(out["rgb"], torch.uint8) if out.get("rgb") is not None else None)
        rid = C.c_int64()
        _check(_lib().tacsl_server_submit(self._h, C.byref(req), C.byref(rid)))
        self._live[rid.value] = keep
        return rid.value

    def set_cameras(self, cameras):
        """The tactile camera of each sensor model (tacsl.Camera list), for pose requests."""
        arr = cameras_array(cameras)
        _check(_lib().tacsl_server_set_cameras(self._h, arr, len(cameras)))

    def pose_outputs_for(self, layout, sensor, want=("wrench", "f_n", "f_t"), pin=True):
        """Host outputs of a pose request: only the names in `want` (wrench, depth, f_n,
        f_t, rgb, depth_map); the others are None and do not travel back."""
        nt, npx = self.sizes_of(layout, sensor)
        mk = (lambda *s, dtype=torch.float32: torch.empty(*s, dtype=dtype).pin_memory()) if pin else \
            (lambda *s, dtype=torch.float32: torch.empty(*s, dtype=dtype))
        shapes = {"wrench": ((len(layout), 6), torch.float32), "depth": ((nt,), torch.float32),
                  "f_n": ((nt, 3), torch.float32), "f_t": ((nt, 3), torch.float32),
                  "rgb": ((max(npx, 1), 3), torch.uint8), "depth_map": ((max(npx, 1),), torch.float32)}
        return {k: (mk(*sh, dtype=dt) if k in want else None) for k, (sh, dt) in shapes.items()}

    def submit_poses(self, obj_id, layout, sensor, pad_pose, pad_twist, k_n, k_d, k_t, mu, out) -> int:
        """Queue one pose request: the server renders the depth maps of the pads with an
        image from their poses; out's None entries are not returned."""
        keep = []

        def h(a, dt):
            if a is None:
                return None
            arr, ptr = _host(a, dt)
            keep.append(arr)
            return ptr

        req = _PoseRequest(len(obj_id), h(obj_id, torch.int32), h(layout, torch.int32), h(sensor, torch.int32),
                           h(pad_pose, torch.float32), h(pad_twist, torch.float32), h(k_n, torch.float32),
                           h(k_d, torch.float32), h(k_t, torch.float32), h(mu, torch.float32),
                           h(out.get("wrench"), torch.float32), h(out.get("depth"), torch.float32),
                           h(out.get("f_n"), torch.float32), h(out.get("f_t"), torch.float32),
                           h(out.get("rgb"), torch.uint8), h(out.get("depth_map"), torch.float32))
        rid = C.c_int64()
        _check(_lib().tacsl_server_submit_poses(self._h, C.byref(req), C.byref(rid)))
        self._live[rid.value] = keep
        return rid.value

    def wait(self, rid, timeout_ms=-1):
        """(status, latency_ms) once the request has finished; TacslError (code 4) if it
        has not finished within timeout_ms."""
        st, lat = C.c_int32(), C.c_double()
        _check(_lib().tacsl_server_wait(self._h, int(rid), int(timeout_ms), C.byref(st), C.byref(lat)))
        keep = self._live.pop(rid, None)
        if st.value == TACSL_ERR_TIMEOUT:
            self._late.append(keep)    # its batch may still use these host arrays until close()
        return st.value, lat.value

    def stats(self) -> dict:
        s = _Stats()
        _check(_lib().tacsl_server_get_stats(self._h, C.byref(s)))
        return {n: getattr(s, n) for n, _ in _Stats._fields_}

    def close(self):
        if self._h is not None and self._h.value:
            _lib().tacsl_server_destroy(self._h)
        self._h = None
        self._live.clear()
        self._late.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
