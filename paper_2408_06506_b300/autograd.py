"""torch.autograd bindings of the tactile step's adjoint kernels (``include/tacsl_grad.h``).

``force_field``, ``shade_intensity``, ``shade_mse`` and ``render_depth`` behave like
differentiable torch functions:
their forward runs the library's forward kernels and their backward the hand-written
adjoint kernels, so a calibration loss over force fields, wrenches and images can be
minimised with any torch optimiser over pad poses, twists, contact parameters and
shading coefficients; with ``render_depth`` the images depend on the pad poses too.  Argument marshalling only; every step runs in ``libtacsl.so``.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import (Camera, ContactParams, SdfSet, Shading, _Camera, _check, _dev, _Params, _ptr, _SdfSet, _Shading,
               _stream, load, penalty_forces)
from . import render_depth as _render_forward

_bound = False


def _lib():
    global _bound
    lib = load()
    if not _bound:
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        lib.tacsl_penalty_forces_adjoint.restype = C.c_int
        lib.tacsl_penalty_forces_adjoint.argtypes = [C.POINTER(_SdfSet), C.POINTER(_Params), I32, I32, I32, P, P, P,
                                                     P, P, P, P, P, P, P, P, P]
        lib.tacsl_shade_intensity.restype = C.c_int
        lib.tacsl_shade_intensity.argtypes = [C.POINTER(_Shading), I64, P, P, P, P]
        lib.tacsl_shade_adjoint.restype = C.c_int
        lib.tacsl_shade_adjoint.argtypes = [C.POINTER(_Shading), I64, P, P, P, P, P, P]
        lib.tacsl_shade_mse.restype = C.c_int
        lib.tacsl_shade_mse.argtypes = [C.POINTER(_Shading), I64, P, P, P, P, P, P, P, P]
        lib.tacsl_shade_mse_slopes.restype = C.c_int
        lib.tacsl_shade_mse_slopes.argtypes = [C.POINTER(_Shading), I64, P, P, P, P, P, P, P]
        lib.tacsl_shade_adjoint_slopes.restype = C.c_int
        lib.tacsl_shade_adjoint_slopes.argtypes = [C.POINTER(_Shading), I64, P, P, P, P, P, P]
        lib.tacsl_shade_depth_from_slopes.restype = C.c_int
        lib.tacsl_shade_depth_from_slopes.argtypes = [C.POINTER(_Shading), I64, P, P, P, P, P]
        lib.tacsl_render_depth_adjoint.restype = C.c_int
        lib.tacsl_render_depth_adjoint.argtypes = [C.POINTER(_SdfSet), I32, I32, P, P, C.POINTER(_Camera), P, P, P, P]
        _bound = True
    return lib


def _c(t):
    return None if t is None else t.contiguous()


class _ForceField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pose, twist, k_n, k_d, k_t, mu, sdfs, taxels, obj_id):
        params = ContactParams(k_n.detach(), k_d.detach(), k_t.detach(), mu.detach())
        depth, f_n, f_t, wrench = penalty_forces(sdfs, params, taxels, obj_id, pose.detach(), twist.detach())
        ctx.save_for_backward(pose, twist, k_n, k_d, k_t, mu)
        ctx.sdfs, ctx.taxels, ctx.obj_id = sdfs, taxels, obj_id
        return depth, f_n, f_t, wrench

    @staticmethod
    def backward(ctx, g_depth, g_fn, g_ft, g_wrench):
        pose, twist, k_n, k_d, k_t, mu = ctx.saved_tensors
        need = ctx.needs_input_grad
        E, P = pose.shape[0], pose.shape[1]
        T = ctx.taxels.shape[0]
        dev = pose.device
        grad_pose = torch.empty(E, P, 7, dtype=torch.float32, device=dev) if need[0] else None
        grad_twist = torch.empty(E, P, 6, dtype=torch.float32, device=dev) if need[1] else None
        count = k_n.numel()
        grad_params = torch.empty(count, 4, dtype=torch.float32, device=dev) if any(need[2:6]) else None
        params = ContactParams(k_n.detach(), k_d.detach(), k_t.detach(), mu.detach())
        gs = [_c(g) for g in (g_depth, g_fn, g_ft, g_wrench)]
        _check(_lib().tacsl_penalty_forces_adjoint(
            C.byref(ctx.sdfs.c), C.byref(params.c), E, P, T, _ptr(ctx.taxels), _ptr(ctx.obj_id), _ptr(pose.detach()),
            _ptr(twist.detach()), *[_ptr(g) for g in gs], _ptr(grad_pose), _ptr(grad_twist), _ptr(grad_params),
            _stream(None)))
        gp = [None] * 4
        if grad_params is not None:
            gp = [grad_params[:, i].reshape(k_n.shape) if need[2 + i] else None for i in range(4)]
        return (grad_pose, grad_twist, *gp, None, None, None)


def force_field(sdfs: SdfSet, taxels, obj_id, pose, twist, k_n, k_d, k_t, mu):
    """Differentiable penalty force field of E x P pads (as ``penalty_forces``):
    returns (depth [E,P,T], f_n [E,P,T,3], f_t [E,P,T,3], wrench [E,P,6]); gradients flow
    to pose [E,P,7], twist [E,P,6] and k_n, k_d, k_t, mu (length 1 or E)."""
    for t, n in ((pose, "pose"), (twist, "twist"), (k_n, "k_n"), (k_d, "k_d"), (k_t, "k_t"), (mu, "mu")):
        _dev(t.detach(), torch.float32, n)
    return _ForceField.apply(pose, twist, k_n, k_d, k_t, mu, sdfs, taxels, obj_id)


class _ShadeIntensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coeffs, depth_map, sensor_id, pitch_x, pitch_y):
        S, _, _, H, W = coeffs.shape
        B = depth_map.numel() // (H * W)
        sh = Shading(coeffs.detach().contiguous(), pitch_x, pitch_y)
        out = torch.empty(B, H, W, 3, dtype=torch.float32, device=depth_map.device)
        _check(_lib().tacsl_shade_intensity(C.byref(sh.c), B, _ptr(sensor_id), _ptr(depth_map.detach()), _ptr(out),
                                            _stream(None)))
        ctx.save_for_backward(coeffs, depth_map, sensor_id)
        ctx.pitch = (pitch_x, pitch_y)
        return out

    @staticmethod
    def backward(ctx, g):
        coeffs, depth_map, sensor_id = ctx.saved_tensors
        need = ctx.needs_input_grad
        S, _, _, H, W = coeffs.shape
        B = depth_map.numel() // (H * W)
        sh = Shading(coeffs.detach().contiguous(), *ctx.pitch)
        gc = torch.empty_like(coeffs) if need[0] else None
        gd = None
        if need[1]:
            # the coefficient adjoint also writes the pixel slopes; the depth gradient is
            # their transposed difference stencil
            gd = torch.empty(depth_map.shape, dtype=torch.float32, device=depth_map.device)
            slopes = torch.empty(B, H, W, 2, dtype=torch.float32, device=depth_map.device)
            _check(_lib().tacsl_shade_adjoint_slopes(C.byref(sh.c), B, _ptr(sensor_id), _ptr(depth_map.detach()),
                                                     _ptr(g.contiguous()), _ptr(gc), _ptr(slopes), _stream(None)))
            _check(_lib().tacsl_shade_depth_from_slopes(C.byref(sh.c), B, _ptr(sensor_id), _ptr(slopes), None,
                                                        _ptr(gd), _stream(None)))
        elif gc is not None:
            _check(_lib().tacsl_shade_adjoint(C.byref(sh.c), B, _ptr(sensor_id), _ptr(depth_map.detach()),
                                              _ptr(g.contiguous()), _ptr(gc), None, _stream(None)))
        return gc, gd, None, None, None


def shade_intensity(coeffs, depth_map, sensor_id, pitch_x, pitch_y):
    """Differentiable clamped intensity [B, H, W, 3] of depth maps [B, H, W] under the
    per-pixel coefficients [S, 6, 3, H, W]; gradients flow to coeffs and depth_map."""
    _dev(coeffs.detach(), torch.float32, "coeffs")
    _dev(depth_map.detach(), torch.float32, "depth_map")
    _dev(sensor_id, torch.int32, "sensor_id")
    return _ShadeIntensity.apply(coeffs, depth_map, sensor_id, float(pitch_x), float(pitch_y))


class _ShadeMse(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coeffs, depth_map, sensor_id, target, pitch_x, pitch_y):
        S, _, _, H, W = coeffs.shape
        B = depth_map.numel() // (H * W)
        sh = Shading(coeffs.detach().contiguous(), pitch_x, pitch_y)
        loss_map = torch.empty(S, H, W, dtype=torch.float32, device=depth_map.device)
        # the coefficient gradient and the depth map's pixel slopes cost the loss pass
        # little: take them here (for a unit upstream gradient) and scale them in backward
        gc = torch.empty_like(coeffs) if ctx.needs_input_grad[0] else None
        slopes = None
        if ctx.needs_input_grad[1] and B > 0:
            slopes = torch.empty(B, H, W, 2, dtype=torch.float32, device=depth_map.device)
            _check(_lib().tacsl_shade_mse_slopes(C.byref(sh.c), B, _ptr(sensor_id), _ptr(depth_map.detach()),
                                                 _ptr(target), _ptr(loss_map), _ptr(gc), _ptr(slopes),
                                                 _stream(None)))
        else:
            _check(_lib().tacsl_shade_mse(C.byref(sh.c), B, _ptr(sensor_id), _ptr(depth_map.detach()),
                                          _ptr(target), None, _ptr(loss_map), _ptr(gc), None, _stream(None)))
        ctx.save_for_backward(coeffs, depth_map, sensor_id)
        ctx.gc, ctx.slopes = gc, slopes
        ctx.pitch = (pitch_x, pitch_y)
        return loss_map.sum()

    @staticmethod
    def backward(ctx, g):
        coeffs, depth_map, sensor_id = ctx.saved_tensors
        need = ctx.needs_input_grad
        S, _, _, H, W = coeffs.shape
        B = depth_map.numel() // (H * W)
        gc = ctx.gc * g if need[0] and ctx.gc is not None else None
        gd = None
        if need[1]:
            gd = torch.empty(depth_map.shape, dtype=torch.float32, device=depth_map.device)
            if ctx.slopes is not None:
                sh = Shading(coeffs.detach().contiguous(), *ctx.pitch)
                scale = g.reshape(1).to(torch.float32).contiguous()
                _check(_lib().tacsl_shade_depth_from_slopes(C.byref(sh.c), B, _ptr(sensor_id), _ptr(ctx.slopes),
                                                            _ptr(scale), _ptr(gd), _stream(None)))
            else:
                gd.zero_()      # no images
        ctx.gc = ctx.slopes = None
        return gc, gd, None, None, None, None


def shade_mse(coeffs, depth_map, sensor_id, pitch_x, pitch_y, target):
    """Differentiable squared error sum((clamp(I) - target)^2) over the B images [B, H, W]
    against target intensities [B, H, W, 3], without materialising I: one fused pass
    forward (which also takes the coefficient gradient when coeffs require grad, and the
    pixel slopes of the depth gradient when depth_map does) and, backward, the
    transposed difference stencil of the slopes; gradients flow to coeffs and depth_map."""
    _dev(coeffs.detach(), torch.float32, "coeffs")
    _dev(depth_map.detach(), torch.float32, "depth_map")
    _dev(sensor_id, torch.int32, "sensor_id")
    _dev(target, torch.float32, "target")
    return _ShadeMse.apply(coeffs, depth_map, sensor_id, target.contiguous(), float(pitch_x), float(pitch_y))


def render_depth_adjoint(sdfs: SdfSet, camera: Camera, obj_id, pad_pose, depth_map, g_depth, grad_pose=None,
                         stream=None):
    """dL/d pad_pose [E, P, 7] of L = sum(g_depth * depth_map), depth_map [E, P, H, W] the
    render of pad_pose (``tacsl_render_depth_adjoint``)."""
    _dev(obj_id, torch.int32, "obj_id")
    _dev(pad_pose, torch.float32, "pad_pose")
    _dev(depth_map, torch.float32, "depth_map")
    _dev(g_depth, torch.float32, "g_depth")
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    if grad_pose is None:
        grad_pose = torch.empty(E, P, 7, dtype=torch.float32, device=pad_pose.device)
    _check(_lib().tacsl_render_depth_adjoint(C.byref(sdfs.c), E, P, _ptr(obj_id), _ptr(pad_pose), C.byref(camera.c),
                                             _ptr(depth_map), _ptr(g_depth), _ptr(grad_pose), _stream(stream)))
    return grad_pose


class _RenderDepth(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pose, sdfs, camera, obj_id):
        depth = _render_forward(sdfs, camera, obj_id, pose.detach())
        ctx.save_for_backward(pose, depth)
        ctx.sdfs, ctx.camera, ctx.obj_id = sdfs, camera, obj_id
        return depth

    @staticmethod
    def backward(ctx, g):
        pose, depth = ctx.saved_tensors
        grad_pose = render_depth_adjoint(ctx.sdfs, ctx.camera, ctx.obj_id, pose.detach(), depth, g.contiguous())
        return grad_pose, None, None, None


def render_depth(sdfs: SdfSet, camera: Camera, obj_id, pose):
    """Differentiable depth maps [E, P, H, W] of the column camera (as the library's
    ``render_depth``); gradients flow to pose [E, P, 7]."""
    _dev(pose.detach(), torch.float32, "pose")
    return _RenderDepth.apply(pose, sdfs, camera, obj_id)
