"""B300-native batched tactile step of TacSL (arXiv 2408.06506).

A thin Python binding over the C ABI of ``libtacsl.so`` (declared in
``include/tacsl.h``).  The functions here only marshal arguments: torch CUDA tensors
become device pointers, the current torch stream becomes the launch stream, and
output tensors are allocated when not given.  Every step of the computation runs in
the library's CUDA kernels; there is no CPU path.  If the library is missing this
module raises instead of falling back.

Entry points (same names as the C ABI, without the ``tacsl_`` prefix):
``sdf_query``, ``penalty_forces``, ``pad_wrench``, ``shade_image``, ``tactile_step``,
``tactile_step_host``, ``render_depth``, ``render_step``, ``check_errors``.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

__all__ = ["SdfSet", "ContactParams", "Shading", "Camera", "TacslError", "sdf_query", "penalty_forces",
           "pad_wrench", "shade_image", "tactile_step", "tactile_step_host", "render_depth", "render_step",
           "check_errors", "library_path", "load"]

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libtacsl.so")
_lib = None

TACSL_OK = 0
DEVERR_BAD_OBJ_ID = 0x1
DEVERR_BAD_SENSOR_ID = 0x2
DEVERR_TIMEOUT = 0x4
MAX_SDF = 64
MAX_SENSOR = 16
MAX_TAXELS = 65536


class TacslError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tacsl error {code}: {msg}")
        self.code = code


class _Sdf(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("origin", C.c_float * 3), ("voxel", C.c_float), ("data", C.c_void_p)]


class _SdfSet(C.Structure):
    _fields_ = [("sdfs", C.POINTER(_Sdf)), ("n_sdf", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("k_n", C.c_void_p), ("k_d", C.c_void_p), ("k_t", C.c_void_p), ("mu", C.c_void_p),
                ("count", C.c_int32)]


class _Camera(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("pitch_x", C.c_float), ("pitch_y", C.c_float),
                ("x0", C.c_float), ("y0", C.c_float), ("d0", C.c_float), ("z_max", C.c_float)]


class _Shading(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("pitch_x", C.c_float), ("pitch_y", C.c_float),
                ("coeffs", C.c_void_p), ("n_sensor", C.c_int32)]


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libtacsl.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                               "`python -m paper_2408_06506_b300.build` (nvcc, sm_103a)")
        lib = C.CDLL(_LIB_PATH)
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        lib.tacsl_last_error.restype = C.c_char_p
        lib.tacsl_last_error.argtypes = []
        lib.tacsl_abi_version.restype = I32
        lib.tacsl_check_errors.restype = C.c_int
        lib.tacsl_check_errors.argtypes = [P, C.POINTER(C.c_uint32), I32]
        lib.tacsl_sdf_query.restype = C.c_int
        lib.tacsl_sdf_query.argtypes = [C.POINTER(_SdfSet), I64, P, P, P, P, P]
        lib.tacsl_penalty_forces.restype = C.c_int
        lib.tacsl_penalty_forces.argtypes = [C.POINTER(_SdfSet), C.POINTER(_Params), I32, I32, I32, P, P, P, P,
                                             P, P, P, P, P]
        lib.tacsl_pad_wrench.restype = C.c_int
        lib.tacsl_pad_wrench.argtypes = [I64, I32, P, P, P, P, P]
        lib.tacsl_shade_image.restype = C.c_int
        lib.tacsl_shade_image.argtypes = [C.POINTER(_Shading), I64, P, P, P, P]
        lib.tacsl_shade_image_wait_limit.restype = C.c_int
        lib.tacsl_shade_image_wait_limit.argtypes = [C.POINTER(_Shading), I64, P, P, P, C.c_uint64, P]
        lib.tacsl_tactile_step.restype = C.c_int
        lib.tacsl_tactile_step.argtypes = [C.POINTER(_SdfSet), C.POINTER(_Params), I32, I32, I32, P, P, P, P,
                                           P, P, P, P, C.POINTER(_Shading), P, P, P, P]
        lib.tacsl_render_depth.restype = C.c_int
        lib.tacsl_render_depth.argtypes = [C.POINTER(_SdfSet), I32, I32, P, P, C.POINTER(_Camera), P, P]
        lib.tacsl_tactile_step_host_workspace.restype = I64
        lib.tacsl_tactile_step_host_workspace.argtypes = [I32, I32, I32, I32, I32]
        lib.tacsl_tactile_step_host.restype = C.c_int
        lib.tacsl_tactile_step_host.argtypes = [C.POINTER(_SdfSet), C.POINTER(_Params), I32, I32, I32, P, P, P, P,
                                                P, P, P, P, C.POINTER(_Shading), P, P, P, I32, P, I64, P]
        lib.tacsl_render_step.restype = C.c_int
        lib.tacsl_render_step.argtypes = [C.POINTER(_SdfSet), C.POINTER(_Params), I32, I32, I32, P, P, P, P,
                                          P, P, P, P, C.POINTER(_Shading), C.POINTER(_Camera), P, P, P, P]
        _lib = lib
    return _lib


def _check(rc: int):
    if rc != TACSL_OK:
        raise TacslError(rc, load().tacsl_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# The current stream's raw handle: torch's accessor returns it without building a Stream
# object (which costs ~0.1 ms per call); the public call is the fallback.
_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)
_cur_device = getattr(torch._C, "_cuda_getDevice", None)


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream.cuda_stream)
    if _raw_stream is not None and _cur_device is not None:
        return C.c_void_p(_raw_stream(_cur_device()))
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class SdfSet:
    """Device-resident SDF grids of one call (descriptors kept on the host).

    grids: list of (data [n2, n1, n0] float32 CUDA tensor, origin (3 floats), voxel).
    """

    def __init__(self, grids):
        self.tensors = []
        self._arr = (_Sdf * max(1, len(grids)))()
        for i, (data, origin, voxel) in enumerate(grids):
            _dev(data, torch.float32, f"sdf[{i}].data")
            self.tensors.append(data)
            n2, n1, n0 = data.shape
            self._arr[i].n[0], self._arr[i].n[1], self._arr[i].n[2] = n0, n1, n2
            for a in range(3):
                self._arr[i].origin[a] = float(origin[a])
            self._arr[i].voxel = float(voxel)
            self._arr[i].data = data.data_ptr()
        self.c = _SdfSet(C.cast(self._arr, C.POINTER(_Sdf)), len(grids))

    @classmethod
    def from_grids(cls, grids, device="cuda"):
        """From objects with .data (numpy f32 [n2][n1][n0]), .origin, .voxel."""
        return cls([(torch.as_tensor(g.data, device=device).contiguous(), [float(v) for v in g.origin],
                     float(g.voxel)) for g in grids])


class ContactParams:
    """k_n, k_d, k_t, mu as float32 CUDA tensors of length 1 or E."""

    def __init__(self, k_n, k_d, k_t, mu):
        ts = [_dev(t, torch.float32, n) for t, n in zip((k_n, k_d, k_t, mu), ("k_n", "k_d", "k_t", "mu"))]
        counts = {t.numel() for t in ts}
        if len(counts) != 1:
            raise ValueError("k_n, k_d, k_t and mu must have the same length")
        self.tensors = ts
        self.count = counts.pop()
        self.c = _Params(*[t.data_ptr() for t in ts], self.count)


class Shading:
    """Per-pixel quadratic shading model: coeffs [S, 6, 3, H, W] float32 CUDA tensor."""

    def __init__(self, coeffs: torch.Tensor, pitch_x: float, pitch_y: float):
        _dev(coeffs, torch.float32, "coeffs")
        S, six, three, H, W = coeffs.shape
        if (six, three) != (6, 3):
            raise ValueError("coeffs must be [S, 6, 3, H, W]")
        self.coeffs, self.H, self.W, self.S = coeffs, H, W, S
        self.c = _Shading(H, W, float(pitch_x), float(pitch_y), coeffs.data_ptr(), S)


def check_errors(clear: bool = True, stream=None) -> int:
    """Synchronise the stream and return the device error word (DEVERR_* bits)."""
    flags = C.c_uint32(0)
    _check(load().tacsl_check_errors(_stream(stream), C.byref(flags), 1 if clear else 0))
    return int(flags.value)


def sdf_query(sdfs: SdfSet, pts, obj_id, phi=None, grad=None, stream=None):
    """phi [n], grad [n, 3] of object-frame points pts [n, 3] in grids obj_id [n]."""
    _dev(pts, torch.float32, "pts")
    _dev(obj_id, torch.int32, "obj_id")
    n = pts.shape[0]
    phi = torch.empty(n, dtype=torch.float32, device=pts.device) if phi is None else phi
    grad = torch.empty(n, 3, dtype=torch.float32, device=pts.device) if grad is None else grad
    _check(load().tacsl_sdf_query(C.byref(sdfs.c), n, _ptr(pts), _ptr(obj_id), _ptr(phi), _ptr(grad),
                                  _stream(stream)))
    return phi, grad


def _force_outputs(E, P, T, device, depth, f_n, f_t, wrench, with_wrench):
    depth = torch.empty(E, P, T, dtype=torch.float32, device=device) if depth is None else depth
    f_n = torch.empty(E, P, T, 3, dtype=torch.float32, device=device) if f_n is None else f_n
    f_t = torch.empty(E, P, T, 3, dtype=torch.float32, device=device) if f_t is None else f_t
    if wrench is None and with_wrench:
        wrench = torch.empty(E, P, 6, dtype=torch.float32, device=device)
    return depth, f_n, f_t, wrench


def penalty_forces(sdfs: SdfSet, params: ContactParams, taxels, obj_id, pad_pose, pad_twist,
                   depth=None, f_n=None, f_t=None, wrench=None, with_wrench=True, stream=None):
    """Force field of E x P pads; returns (depth [E,P,T], f_n [E,P,T,3], f_t [E,P,T,3], wrench [E,P,6])."""
    _dev(taxels, torch.float32, "taxels")
    _dev(obj_id, torch.int32, "obj_id")
    _dev(pad_pose, torch.float32, "pad_pose")
    _dev(pad_twist, torch.float32, "pad_twist")
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    T = taxels.shape[0]
    depth, f_n, f_t, wrench = _force_outputs(E, P, T, pad_pose.device, depth, f_n, f_t, wrench, with_wrench)
    _check(load().tacsl_penalty_forces(C.byref(sdfs.c), C.byref(params.c), E, P, T, _ptr(taxels), _ptr(obj_id),
                                       _ptr(pad_pose), _ptr(pad_twist), _ptr(depth), _ptr(f_n), _ptr(f_t),
                                       _ptr(wrench), _stream(stream)))
    return depth, f_n, f_t, wrench


def pad_wrench(taxels, f_n, f_t, wrench=None, stream=None):
    """wrench [B, 6] from force fields f_n, f_t [B, T, 3] (any leading shape flattened to B)."""
    _dev(taxels, torch.float32, "taxels")
    _dev(f_n, torch.float32, "f_n")
    _dev(f_t, torch.float32, "f_t")
    T = taxels.shape[0]
    B = f_n.numel() // (3 * T) if T > 0 else f_n.shape[0]
    wrench = torch.empty(B, 6, dtype=torch.float32, device=f_n.device) if wrench is None else wrench
    _check(load().tacsl_pad_wrench(B, T, _ptr(taxels), _ptr(f_n), _ptr(f_t), _ptr(wrench), _stream(stream)))
    return wrench


def shade_image(shading: Shading, sensor_id, depth_map, rgb=None, stream=None):
    """uint8 RGB [B, H, W, 3] from depth maps [B, H, W] (leading dims flattened to B)."""
    _dev(sensor_id, torch.int32, "sensor_id")
    _dev(depth_map, torch.float32, "depth_map")
    B = depth_map.numel() // (shading.H * shading.W)
    rgb = torch.empty(B, shading.H, shading.W, 3, dtype=torch.uint8, device=depth_map.device) if rgb is None else rgb
    _check(load().tacsl_shade_image(C.byref(shading.c), B, _ptr(sensor_id), _ptr(depth_map), _ptr(rgb),
                                    _stream(stream)))
    return rgb


def tactile_step(sdfs: SdfSet, params: ContactParams, taxels, obj_id, pad_pose, pad_twist,
                 shading: Shading | None = None, sensor_id=None, depth_map=None,
                 depth=None, f_n=None, f_t=None, wrench=None, rgb=None, with_wrench=True, stream=None):
    """Force field of E x P pads and (if shading is given) their E*P tactile images, one call.

    Returns (depth, f_n, f_t, wrench, rgb)."""
    _dev(taxels, torch.float32, "taxels")
    _dev(obj_id, torch.int32, "obj_id")
    _dev(pad_pose, torch.float32, "pad_pose")
    _dev(pad_twist, torch.float32, "pad_twist")
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    T = taxels.shape[0]
    depth, f_n, f_t, wrench = _force_outputs(E, P, T, pad_pose.device, depth, f_n, f_t, wrench, with_wrench)
    if shading is not None:
        _dev(sensor_id, torch.int32, "sensor_id")
        _dev(depth_map, torch.float32, "depth_map")
        if rgb is None:
            rgb = torch.empty(E * P, shading.H, shading.W, 3, dtype=torch.uint8, device=pad_pose.device)
    _check(load().tacsl_tactile_step(C.byref(sdfs.c), C.byref(params.c), E, P, T, _ptr(taxels), _ptr(obj_id),
                                     _ptr(pad_pose), _ptr(pad_twist), _ptr(depth), _ptr(f_n), _ptr(f_t),
                                     _ptr(wrench), C.byref(shading.c) if shading is not None else None,
                                     _ptr(sensor_id) if shading is not None else None,
                                     _ptr(depth_map) if shading is not None else None,
                                     _ptr(rgb) if shading is not None else None, _stream(stream)))
    return depth, f_n, f_t, wrench, rgb


class Camera:
    """Orthographic column camera of the depth renderer (see tacsl_camera)."""

    def __init__(self, H, W, pitch_x, pitch_y, x0, y0, d0, z_max):
        self.H, self.W = int(H), int(W)
        self.c = _Camera(self.H, self.W, float(pitch_x), float(pitch_y), float(x0), float(y0), float(d0),
                         float(z_max))


def render_depth(sdfs: SdfSet, camera: Camera, obj_id, pad_pose, depth_map=None, stream=None):
    """Depth maps [E, P, H, W] of E x P pads."""
    _dev(obj_id, torch.int32, "obj_id")
    _dev(pad_pose, torch.float32, "pad_pose")
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    if depth_map is None:
        depth_map = torch.empty(E, P, camera.H, camera.W, dtype=torch.float32, device=pad_pose.device)
    _check(load().tacsl_render_depth(C.byref(sdfs.c), E, P, _ptr(obj_id), _ptr(pad_pose), C.byref(camera.c),
                                     _ptr(depth_map), _stream(stream)))
    return depth_map


def render_step(sdfs: SdfSet, params: ContactParams, taxels, obj_id, pad_pose, pad_twist, shading: Shading,
                camera: Camera, sensor_id, depth_map=None, depth=None, f_n=None, f_t=None, wrench=None, rgb=None,
                with_wrench=True, stream=None):
    """Depth maps rendered from the poses, their RGB images and the force field, one call.

    Returns (depth, f_n, f_t, wrench, depth_map, rgb)."""
    for t, n, dt in ((taxels, "taxels", torch.float32), (obj_id, "obj_id", torch.int32),
                     (pad_pose, "pad_pose", torch.float32), (pad_twist, "pad_twist", torch.float32),
                     (sensor_id, "sensor_id", torch.int32)):
        _dev(t, dt, n)
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    T = taxels.shape[0]
    depth, f_n, f_t, wrench = _force_outputs(E, P, T, pad_pose.device, depth, f_n, f_t, wrench, with_wrench)
    if depth_map is None:
        depth_map = torch.empty(E, P, camera.H, camera.W, dtype=torch.float32, device=pad_pose.device)
    if rgb is None:
        rgb = torch.empty(E * P, shading.H, shading.W, 3, dtype=torch.uint8, device=pad_pose.device)
    _check(load().tacsl_render_step(C.byref(sdfs.c), C.byref(params.c), E, P, T, _ptr(taxels), _ptr(obj_id),
                                    _ptr(pad_pose), _ptr(pad_twist), _ptr(depth), _ptr(f_n), _ptr(f_t), _ptr(wrench),
                                    C.byref(shading.c), C.byref(camera.c), _ptr(sensor_id), _ptr(depth_map),
                                    _ptr(rgb), _stream(stream)))
    return depth, f_n, f_t, wrench, depth_map, rgb


def _host_t(t, dtype, name):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return t


def tactile_step_host(sdfs: SdfSet, params: ContactParams, taxels, obj_id, pad_pose, pad_twist,
                      shading: Shading | None = None, sensor_id=None, depth_map=None, out=None, chunk_envs=128,
                      workspace=None, stream=None):
    """tactile_step with the per-step arrays in host memory (pinned for overlap): obj_id,
    pad_pose, pad_twist, sensor_id, depth_map in; (depth, f_n, f_t, wrench, rgb) host
    tensors out, written when the stream reaches the end of the call.  chunk_envs: envs
    per pipelined chunk (128 measured best for 2-pad envs with 320x240 images: smaller
    chunks shorten the pipeline's head and tail, where only one direction copies)."""
    _dev(taxels, torch.float32, "taxels")
    for t, n, dt in ((obj_id, "obj_id", torch.int32), (pad_pose, "pad_pose", torch.float32),
                     (pad_twist, "pad_twist", torch.float32)):
        _host_t(t, dt, n)
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    T = taxels.shape[0]
    H, W = (shading.H, shading.W) if shading is not None else (0, 0)
    if shading is not None:
        _host_t(sensor_id, torch.int32, "sensor_id")
        _host_t(depth_map, torch.float32, "depth_map")
    if out is None:
        pin = lambda *sh, dtype=torch.float32: torch.empty(*sh, dtype=dtype).pin_memory()   # noqa: E731
        out = {"depth": pin(E, P, T), "f_n": pin(E, P, T, 3), "f_t": pin(E, P, T, 3), "wrench": pin(E, P, 6),
               "rgb": pin(E * P, H, W, 3, dtype=torch.uint8) if shading is not None else None}
    ch = max(1, min(int(chunk_envs), E))
    need = load().tacsl_tactile_step_host_workspace(ch, P, T, H, W)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=taxels.device)
    _check(load().tacsl_tactile_step_host(
        C.byref(sdfs.c), C.byref(params.c), E, P, T, _ptr(taxels), _ptr(obj_id), _ptr(pad_pose), _ptr(pad_twist),
        _ptr(out["depth"]), _ptr(out["f_n"]), _ptr(out["f_t"]), _ptr(out.get("wrench")),
        C.byref(shading.c) if shading is not None else None, _ptr(sensor_id) if shading is not None else None,
        _ptr(depth_map) if shading is not None else None, _ptr(out.get("rgb")) if shading is not None else None,
        ch, _ptr(workspace), workspace.numel(), _stream(stream)))
    return out["depth"], out["f_n"], out["f_t"], out.get("wrench"), out.get("rgb")
