"""FP64 CPU oracle of the TacSL tactile step -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
and reference legs may import this package.  It shares no code with the CUDA
library; it reads the same float32 inputs and computes in double precision.

The arithmetic lives in ``tacsl_oracle.c`` (plain C, OpenMP over independent
pads/images); this module only builds it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tacsl_oracle.c")
_HDR = os.path.join(_HERE, "tacsl_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (IEEE double, no fast-math)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Sdf(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("origin", C.c_float * 3), ("voxel", C.c_float),
                ("data", C.c_void_p)]


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(C.CDLL(build()))
    return _lib


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    P = C.c_void_p
    lib.orc_trilinear.restype = C.c_double
    lib.orc_trilinear.argtypes = [P, P]
    lib.orc_sdf_eval.restype = C.c_int
    lib.orc_sdf_eval.argtypes = [P, P, P, P]
    lib.orc_sdf_query.restype = C.c_int64
    lib.orc_sdf_query.argtypes = [P, C.c_int32, C.c_int64, P, P, P, P, C.c_int32]
    lib.orc_penalty_forces.restype = C.c_int64
    lib.orc_penalty_forces.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P, P, P,
                                       P, P, P, P, C.c_int32, P, P, P, P, C.c_int32]
    lib.orc_pad_wrench.restype = None
    lib.orc_pad_wrench.argtypes = [C.c_int64, C.c_int32, P, P, P, P, C.c_int32]
    lib.orc_depth_normals.restype = None
    lib.orc_depth_normals.argtypes = [C.c_int32, C.c_int32, C.c_float, C.c_float, P, P]
    lib.orc_shade.restype = C.c_int64
    lib.orc_shade.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_float, C.c_int64,
                              P, P, P, P, C.c_int32]
    lib.orc_quantize.restype = C.c_uint8
    lib.orc_quantize.argtypes = [C.c_double]
    lib.orc_render_depth.restype = C.c_int64
    lib.orc_render_depth.argtypes = [P, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, C.c_int32]
    lib.orc_column_phi.restype = C.c_double
    lib.orc_column_phi.argtypes = [P, P, C.c_double, C.c_double, C.c_double]
    return lib


class use_source:
    """Context manager: build the oracle from alternative C source text and route every
    call in this module through it (used by the tests that plant mistakes on purpose)."""

    def __init__(self, c_source: str, workdir: str):
        self.src, self.dir = c_source, workdir

    def __enter__(self):
        global _lib
        src = os.path.join(self.dir, "variant.c")
        with open(src, "w") as f:
            f.write(self.src)
        so = os.path.join(self.dir, f"variant{os.getpid()}_{id(self)}.so")
        subprocess.check_call(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-I", _HERE,
                               "-o", so, src, "-lm"])
        self.saved = _lib
        _lib = _bind(C.CDLL(so))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _sdf_array(grids):
    """Descriptor array for a list of objects with .data (f32 [n2][n1][n0]), .origin, .voxel."""
    arr = (_Sdf * max(1, len(grids)))()
    keep = []
    for i, g in enumerate(grids):
        data = _f32(g.data)
        keep.append(data)
        arr[i].n[0], arr[i].n[1], arr[i].n[2] = data.shape[2], data.shape[1], data.shape[0]
        for a in range(3):
            arr[i].origin[a] = float(np.float32(g.origin[a]))
        arr[i].voxel = float(np.float32(g.voxel))
        arr[i].data = data.ctypes.data
    return arr, keep


def trilinear(grid, u) -> float:
    arr, keep = _sdf_array([grid])
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64))
    return _load().orc_trilinear(C.byref(arr[0]), _ptr(u))


def sdf_eval(grid, x):
    """(phi, grad[3], in_domain) at one object-frame point (float64)."""
    arr, keep = _sdf_array([grid])
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    phi = np.zeros(1)
    g = np.zeros(3)
    inside = _load().orc_sdf_eval(C.byref(arr[0]), _ptr(x), _ptr(phi), _ptr(g))
    return float(phi[0]), g, bool(inside)


def sdf_query(grids, pts, obj_id, nthreads=None):
    pts = _f32(pts).reshape(-1, 3)
    obj_id = _i32(obj_id).reshape(-1)
    n = pts.shape[0]
    phi = np.empty(n)
    grad = np.empty((n, 3))
    arr, keep = _sdf_array(grids)
    bad = _load().orc_sdf_query(arr, len(grids), n, _ptr(pts), _ptr(obj_id), _ptr(phi), _ptr(grad),
                                nthreads or default_threads())
    return phi, grad, int(bad)


def penalty_forces(grids, taxels, obj_id, pad_pose, pad_twist, k_n, k_d, k_t, mu,
                   with_wrench=True, nthreads=None):
    """Force field of E x P pads: returns dict depth [E,P,T], f_n/f_t [E,P,T,3], wrench [E,P,6]."""
    taxels = _f32(taxels).reshape(-1, 3)
    pad_pose = _f32(pad_pose)
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    T = taxels.shape[0]
    pad_twist = _f32(pad_twist).reshape(E, P, 6)
    obj_id = _i32(obj_id).reshape(E)
    prm = [_f32(np.atleast_1d(v)) for v in (k_n, k_d, k_t, mu)]
    npar = prm[0].shape[0]
    assert all(p.shape[0] == npar for p in prm) and npar in (1, E)
    depth = np.empty((E, P, T))
    fn = np.empty((E, P, T, 3))
    ft = np.empty((E, P, T, 3))
    wr = np.empty((E, P, 6)) if with_wrench else None
    arr, keep = _sdf_array(grids)
    bad = _load().orc_penalty_forces(arr, len(grids), E, P, T, _ptr(taxels), _ptr(obj_id),
                                     _ptr(pad_pose), _ptr(pad_twist), *[_ptr(p) for p in prm], npar,
                                     _ptr(depth), _ptr(fn), _ptr(ft), _ptr(wr),
                                     nthreads or default_threads())
    return {"depth": depth, "f_n": fn, "f_t": ft, "wrench": wr, "bad": int(bad)}


def pad_wrench(taxels, f_n, f_t, nthreads=None):
    taxels = _f32(taxels).reshape(-1, 3)
    T = taxels.shape[0]
    f_n = _f32(f_n).reshape(-1, T, 3)
    f_t = _f32(f_t).reshape(-1, T, 3)
    B = f_n.shape[0]
    out = np.empty((B, 6))
    _load().orc_pad_wrench(B, T, _ptr(taxels), _ptr(f_n), _ptr(f_t), _ptr(out),
                           nthreads or default_threads())
    return out


def depth_normals(depth, pitch_x, pitch_y):
    depth = _f32(depth)
    H, W = depth.shape
    out = np.empty((H, W, 3))
    _load().orc_depth_normals(H, W, float(np.float32(pitch_x)), float(np.float32(pitch_y)),
                              _ptr(depth), _ptr(out))
    return out


def shade(coeffs, pitch_x, pitch_y, sensor_id, depth, with_intensity=False, rgb_init=None,
          nthreads=None):
    """Depth maps [B,H,W] -> rgb uint8 [B,H,W,3] (and intensities [B,H,W,3] if asked)."""
    coeffs = _f32(coeffs)
    S, _, _, H, W = coeffs.shape
    depth = _f32(depth).reshape(-1, H, W)
    B = depth.shape[0]
    sensor_id = _i32(sensor_id).reshape(B)
    rgb = (np.zeros((B, H, W, 3), np.uint8) if rgb_init is None
           else np.ascontiguousarray(rgb_init, dtype=np.uint8).copy())
    inten = np.empty((B, H, W, 3)) if with_intensity else None
    bad = _load().orc_shade(_ptr(coeffs), S, H, W, float(np.float32(pitch_x)), float(np.float32(pitch_y)),
                            B, _ptr(sensor_id), _ptr(depth), _ptr(inten), _ptr(rgb),
                            nthreads or default_threads())
    return (rgb, inten, int(bad)) if with_intensity else (rgb, int(bad))


def quantize(v: float) -> int:
    return int(_load().orc_quantize(float(v)))


class _Camera(C.Structure):
    _fields_ = [("H", C.c_int32), ("W", C.c_int32), ("pitch_x", C.c_float), ("pitch_y", C.c_float),
                ("x0", C.c_float), ("y0", C.c_float), ("d0", C.c_float), ("z_max", C.c_float)]


def render_depth(grids, obj_id, pad_pose, H, W, pitch_x, pitch_y, x0, y0, d0, z_max, nthreads=None):
    """Depth maps [E, P, H, W] (float64) of the orthographic column camera."""
    pad_pose = _f32(pad_pose)
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    obj_id = _i32(obj_id).reshape(E)
    cam = _Camera(H, W, pitch_x, pitch_y, x0, y0, d0, z_max)
    out = np.empty((E, P, H, W))
    arr, keep = _sdf_array(grids)
    bad = _load().orc_render_depth(arr, len(grids), E, P, _ptr(obj_id), _ptr(pad_pose), C.byref(cam), _ptr(out),
                                   nthreads or default_threads())
    return out, int(bad)


def column_phi(grid, pose7, x, y, z) -> float:
    """The SDF value the column march sees at pad-frame point (x, y, z)."""
    arr, keep = _sdf_array([grid])
    pose7 = _f32(pose7).reshape(7)
    return float(_load().orc_column_phi(C.byref(arr[0]), _ptr(pose7), float(x), float(y), float(z)))
