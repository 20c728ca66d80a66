"""Shared helpers for the GPU parity tests: move a synthetic scene to the device, call
the library through its binding, and compare with the FP64 oracle at the stated
tolerances (depth abs 1e-6 m; forces and wrenches rel 1e-4 with near-zero floors;
uint8 RGB within 1 LSB, and only next to a rounding tie)."""
import numpy as np
import torch

import paper_2408_06506_b300 as tacsl

DEPTH_ATOL = 1e-6          # metres
FORCE_RTOL = 1e-4
FORCE_FLOOR = 1e-5         # times the largest taxel force of the same pad
# Absolute floor from float32 arithmetic: the GPU's phi carries ~1e-8 m of rounding
# (a few ulp of 3 cm positions, 2^-24 of the continuous index times the voxel), so a
# force k_n*phi carries k_n*1e-8 N; 2e-8 m gives a factor-2 margin.  The shear's
# stick branch k_t*|v_t| carries k_t * 1e-6 * |x'| with |x'| < 0.2 m/s -> 2e-7 m/s.
PHI_F32_ERR = 2e-8         # metres
VT_F32_ERR = 2e-7          # metres / second
WRENCH_RTOL = 1e-4         # times sum_i |term_i| (condition-number floor)
RGB_TIE_BAND = 2e-3        # a 1-LSB difference is allowed only this close to a .5 tie


def force_abs_floor(sc):
    """Per-env absolute force floor [E, 1, 1] from the float32 error of phi and v_t."""
    E = sc.E
    kn = np.broadcast_to(np.asarray(sc.k_n, np.float64), (E,))
    kt = np.broadcast_to(np.asarray(sc.k_t, np.float64), (E,))
    return (PHI_F32_ERR * kn + VT_F32_ERR * kt)[:, None, None]


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def scene_to_device(sc):
    d = {
        "sdfs": tacsl.SdfSet.from_grids(sc.grids),
        "params": tacsl.ContactParams(dev(sc.k_n), dev(sc.k_d), dev(sc.k_t), dev(sc.mu)),
        "taxels": dev(sc.taxels),
        "obj_id": dev(sc.obj_id),
        "pose": dev(sc.pad_pose),
        "twist": dev(sc.pad_twist),
    }
    if sc.coeffs is not None:
        d["shading"] = tacsl.Shading(dev(sc.coeffs), sc.pitch_x, sc.pitch_y)
        d["sensor_id"] = dev(sc.sensor_id)
        d["depth_map"] = dev(sc.depth_map)
    return d


def assert_forces_close(gpu_f, ref_f, what="force", abs_floor=0.0):
    """Per taxel: |df| <= 1e-4 |f_ref| + max(1e-5 max_j |f_ref,j| (same pad), abs_floor)."""
    g = np.asarray(gpu_f, np.float64)
    r = np.asarray(ref_f, np.float64)
    nan_r = np.isnan(r)
    assert np.array_equal(np.isnan(g), nan_r), f"{what}: NaN pattern differs"
    g = np.where(nan_r, 0.0, g)
    r = np.where(nan_r, 0.0, r)
    err = np.linalg.norm(g - r, axis=-1)
    mag = np.linalg.norm(r, axis=-1)
    pad_max = mag.max(axis=-1, keepdims=True)
    tol = FORCE_RTOL * mag + np.maximum(FORCE_FLOOR * pad_max, abs_floor) + 1e-12
    bad = err > tol
    assert not bad.any(), (f"{what}: {bad.sum()} taxels out of tolerance; worst excess "
                           f"{(err - tol).max():.3e} at {np.unravel_index(np.argmax(err - tol), err.shape)}")


def wrench_scale(taxels, f):
    """sum_i |term_i| per wrench component, from per-taxel forces f [..., T, 3] (float64)."""
    p = np.asarray(taxels, np.float64)
    f = np.asarray(f, np.float64)
    m = np.cross(np.broadcast_to(p, f.shape), f)
    return np.concatenate([np.abs(f).sum(-2), np.abs(m).sum(-2)], -1)


def assert_wrench_close(gpu_w, ref_w, scale, what="wrench", abs_floor=0.0):
    """|dW_k| <= 1e-4 sum_i |term_i,k| + abs_floor (abs_floor: the per-taxel floor times the
    number of taxels in contact on either side, times the lever arm for the moment rows)."""
    g = np.asarray(gpu_w, np.float64)
    r = np.asarray(ref_w, np.float64)
    nan_r = np.isnan(r)
    assert np.array_equal(np.isnan(g), nan_r), f"{what}: NaN pattern differs"
    d = np.abs(np.where(nan_r, 0, g) - np.where(nan_r, 0, r))
    tol = WRENCH_RTOL * np.where(nan_r, 0, scale) + abs_floor + 1e-9
    assert (d <= tol).all(), f"{what}: worst excess {(d - tol).max():.3e}"


def assert_rgb_close(gpu_rgb, ref_rgb, ref_intensity):
    """|d| <= 1 everywhere; any difference sits within RGB_TIE_BAND of a rounding tie."""
    g = np.asarray(gpu_rgb).astype(np.int16)
    r = np.asarray(ref_rgb).astype(np.int16)
    d = np.abs(g - r)
    assert d.max(initial=0) <= 1, f"rgb differs by {d.max()} LSB"
    if d.any():
        I = np.asarray(ref_intensity)[d > 0]
        frac = np.clip(I, 0, 255) - np.floor(np.clip(I, 0, 255))
        near_tie = np.abs(frac - 0.5) < RGB_TIE_BAND
        assert near_tie.all(), f"{(~near_tie).sum()} 1-LSB differences away from a rounding tie"
    return int(d.sum())
