"""GPU parity of the two-pass depth gradient of the image (Sec. III-B shading):
tacsl_shade_mse_slopes and tacsl_shade_adjoint_slopes write per-pixel slopes
(dL/dD_x, dL/dD_y) in the pass that evaluates the shading anyway, and
tacsl_shade_depth_from_slopes applies the transposed difference stencil.

Checked: the slopes against the FP64 oracle's (oracle.grad.shade_slopes); the depth
gradient against the oracle's and against the one-pass kernels of tacsl_shade_mse and
tacsl_shade_adjoint; the loss map and coefficient gradient of the slope-writing passes
bit for bit against those of tacsl_shade_mse / tacsl_shade_adjoint; scale; images with a
bad sensor id (zero gradient); the full calibration workload (2048 maps of 320x240)
against the one-pass kernel everywhere; argument errors."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import paper_2408_06506_b300 as tacsl
from oracle import grad as G
from paper_2408_06506_b300 import autograd as ta
from paper_2408_06506_b300 import synth

from gpu_common import dev

pytestmark = pytest.mark.gpu
CLAMP_MARGIN = 0.05     # the kernels decide the clamp in float32: no intensity this close to 0 or 255
P = tacsl._ptr
ERR_INVALID_ARG = 1     # TACSL_ERR_INVALID_ARG: nothing launched


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06506_b300 import build
    build.build()
    tacsl.load()
    tacsl.check_errors(clear=True)


def _case(seed, S, B, H, W, px=2e-4, py=3e-4, relief=2e-5):
    rng = np.random.default_rng(seed)
    co = synth.shading_coeffs(S, H, W, seed + 100)
    dm = (synth.D0 + relief * rng.normal(size=(B, H, W))).astype(np.float32)
    sid = (np.arange(B) % S).astype(np.int32)
    _, inten, _ = oracle.shade(co, px, py, sid, dm, with_intensity=True)
    assert (np.minimum(np.abs(inten), np.abs(inten - 255)) > CLAMP_MARGIN).all()
    tgt = np.clip(inten + rng.normal(0, 15, size=inten.shape), 0, 255).astype(np.float32)
    gI = rng.normal(size=(B, H, W, 3)).astype(np.float32)
    return co, dm, sid, tgt, gI, px, py


def _close(got, want, rel, floor=1e-12):
    err = np.abs(np.asarray(got, np.float64) - want).max()
    assert err <= rel * np.abs(want).max() + floor, err / max(np.abs(want).max(), 1e-300)


def _two_pass(sh, B, H, W, sid, dm, u, mse, scale=None, S=None):
    """(loss map, coefficient gradient, slopes, depth gradient) of the two-pass path."""
    lib = ta._lib()
    lm = torch.full((S, H, W), float("nan"), device="cuda") if mse else None
    gc = torch.full((S, 6, 3, H, W), float("nan"), device="cuda")
    sl = torch.full((B, H, W, 2), float("nan"), device="cuda")
    gd = torch.full((B, H, W), float("nan"), device="cuda")
    if mse:
        rc = lib.tacsl_shade_mse_slopes(C.byref(sh.c), B, P(sid), P(dm), P(u), P(lm), P(gc), P(sl), None)
    else:
        rc = lib.tacsl_shade_adjoint_slopes(C.byref(sh.c), B, P(sid), P(dm), P(u), P(gc), P(sl), None)
    assert rc == 0, tacsl.load().tacsl_last_error()
    sc = None if scale is None else torch.tensor([scale], dtype=torch.float32, device="cuda")
    rc = lib.tacsl_shade_depth_from_slopes(C.byref(sh.c), B, P(sid), P(sl), P(sc), P(gd), None)
    assert rc == 0, tacsl.load().tacsl_last_error()
    torch.cuda.synchronize()
    return lm, gc, sl, gd


def _one_pass(sh, B, H, W, sid, dm, u, mse, S):
    lib = ta._lib()
    lm = torch.empty(S, H, W, device="cuda") if mse else None
    gc = torch.empty(S, 6, 3, H, W, device="cuda")
    gd = torch.empty(B, H, W, device="cuda")
    if mse:
        rc = lib.tacsl_shade_mse(C.byref(sh.c), B, P(sid), P(dm), P(u), None, P(lm), P(gc), P(gd), None)
    else:
        rc = lib.tacsl_shade_adjoint(C.byref(sh.c), B, P(sid), P(dm), P(u), P(gc), P(gd), None)
    assert rc == 0, tacsl.load().tacsl_last_error()
    torch.cuda.synchronize()
    return lm, gc, gd


# the last two: several 512-pixel strips per image with a ragged last strip, and one
# image row longer than a strip
SHAPES = [(2, 6, 24, 32), (1, 3, 7, 12), (3, 10, 16, 12), (1, 2, 1, 8), (2, 5, 9, 36), (2, 4, 5, 4), (1, 3, 2, 4),
          (2, 5, 40, 20), (1, 2, 3, 7040)]


@pytest.mark.parametrize("mse", [True, False], ids=["mse", "adjoint"])
@pytest.mark.parametrize("S,B,H,W", SHAPES)
def test_slopes_and_depth_gradient_match_oracle(S, B, H, W, mse):
    co, dm, sid, tgt, gI, px, py = _case(60 + B + H, S, B, H, W)
    sh = tacsl.Shading(dev(co), px, py)
    d_sid, d_dm = dev(sid), dev(dm)
    u = dev(tgt) if mse else dev(gI)
    lm, gc, sl, gd = _two_pass(sh, B, H, W, d_sid, d_dm, u, mse, S=S)
    assert tacsl.check_errors() == 0
    if mse:
        ref_sl = G.shade_slopes(co, px, py, sid, dm, target=tgt)
        ref = G.shade_mse(co, px, py, sid, dm, tgt)
    else:
        ref_sl = G.shade_slopes(co, px, py, sid, dm, g_intensity=gI)
        ref = G.shade_gradients(co, px, py, sid, dm, gI)
    _close(sl.cpu().numpy(), ref_sl, 1e-3)
    _close(gd.cpu().numpy(), ref["depth"], 1e-3)
    # against the one-pass kernels: the same loss map and coefficient gradient bit for bit;
    # the depth gradient to rounding (the slopes are summed in the same slot order)
    lm1, gc1, gd1 = _one_pass(sh, B, H, W, d_sid, d_dm, u, mse, S)
    if mse:
        assert torch.equal(lm, lm1)
    assert torch.equal(gc, gc1)
    _close(gd.cpu().numpy(), gd1.cpu().numpy().astype(np.float64), 1e-5)


def test_scale_bad_sensors_and_empty():
    S, B, H, W = 2, 6, 12, 16
    co, dm, sid, tgt, gI, px, py = _case(71, S, B, H, W)
    sh = tacsl.Shading(dev(co), px, py)
    bad = sid.copy()
    bad[1], bad[4] = -1, S
    d_bad, d_dm, d_t = dev(bad), dev(dm), dev(tgt)
    _, _, sl, gd = _two_pass(sh, B, H, W, d_bad, d_dm, d_t, True, S=S)
    _, _, _, gd3 = _two_pass(sh, B, H, W, d_bad, d_dm, d_t, True, scale=-3.5, S=S)
    tacsl.check_errors(clear=True)
    gd, gd3 = gd.cpu().numpy(), gd3.cpu().numpy()
    assert not gd[1].any() and not gd[4].any()
    keep = [0, 2, 3, 5]
    ref = G.shade_mse(co, px, py, sid[keep], dm[keep], tgt[keep])
    _close(gd[keep], ref["depth"], 1e-3)
    _close(gd3, -3.5 * gd.astype(np.float64), 1e-6)
    # slopes of bad images are not written
    assert bool(torch.isnan(sl[1]).all()) and bool(torch.isnan(sl[4]).all())
    # no images: nothing to do; per-sensor outputs still written
    lib = ta._lib()
    lm0 = torch.full((S, H, W), float("nan"), device="cuda")
    assert lib.tacsl_shade_mse_slopes(C.byref(sh.c), 0, None, None, None, P(lm0), None, None, None) == 0
    assert lib.tacsl_shade_depth_from_slopes(C.byref(sh.c), 0, None, None, None, None, None) == 0
    torch.cuda.synchronize()
    assert not bool(lm0.any())


def test_argument_errors():
    S, B, H, W = 1, 2, 4, 8
    co, dm, sid, tgt, gI, px, py = _case(72, S, B, H, W)
    sh = tacsl.Shading(dev(co), px, py)
    lib = ta._lib()
    d_sid, d_dm, d_t = dev(sid), dev(dm), dev(tgt)
    sl = torch.empty(B * H * W * 2 + 4, device="cuda")
    gd = torch.empty(B * H * W + 2, device="cuda")
    # slopes must be 16-byte aligned and present
    assert lib.tacsl_shade_mse_slopes(C.byref(sh.c), B, P(d_sid), P(d_dm), P(d_t), None, None, P(sl[1:]),
                                      None) == ERR_INVALID_ARG
    assert lib.tacsl_shade_adjoint_slopes(C.byref(sh.c), B, P(d_sid), P(d_dm), P(d_t), None, None,
                                          None) == ERR_INVALID_ARG
    # grad_depth must be 8-byte aligned
    assert lib.tacsl_shade_depth_from_slopes(C.byref(sh.c), B, P(d_sid), P(sl), None, P(gd[1:]),
                                             None) == ERR_INVALID_ARG
    assert lib.tacsl_shade_depth_from_slopes(None, B, P(d_sid), P(sl), None, P(gd), None) == ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0


def test_autograd_paths_use_the_slopes():
    """shade_mse and shade_intensity through torch.autograd (both now two-pass for the
    depth) against the one-pass kernels' gradients for the same upstream values."""
    S, B, H, W = 2, 8, 24, 32
    co, dm, sid, tgt, gI, px, py = _case(73, S, B, H, W, relief=4e-5)
    d_sid = dev(sid)
    c1, d1 = dev(co).requires_grad_(True), dev(dm).requires_grad_(True)
    L = ta.shade_mse(c1, d1, d_sid, px, py, dev(tgt))
    (0.75 * L).backward()
    sh = tacsl.Shading(dev(co), px, py)
    lib = ta._lib()
    gc = torch.empty(S, 6, 3, H, W, device="cuda")
    gd = torch.empty(B, H, W, device="cuda")
    sc = torch.tensor([0.75], device="cuda")
    assert lib.tacsl_shade_mse(C.byref(sh.c), B, P(d_sid), P(dev(dm)), P(dev(tgt)), P(sc), None, P(gc), P(gd),
                               None) == 0
    torch.cuda.synchronize()
    _close(d1.grad.cpu().numpy(), gd.cpu().numpy().astype(np.float64), 1e-5)
    _close(c1.grad.cpu().numpy(), gc.cpu().numpy().astype(np.float64), 1e-6)
    c2, d2 = dev(co).requires_grad_(True), dev(dm).requires_grad_(True)
    I = ta.shade_intensity(c2, d2, d_sid, px, py)
    I.backward(dev(gI))
    _, gc1, gd1 = _one_pass(sh, B, H, W, d_sid, dev(dm), dev(gI), False, S)
    assert torch.equal(c2.grad, gc1)
    _close(d2.grad.cpu().numpy(), gd1.cpu().numpy().astype(np.float64), 1e-5)
    # depth only (coefficients without grad): the slopes pass still runs
    d3 = dev(dm).requires_grad_(True)
    ta.shade_intensity(dev(co), d3, d_sid, px, py).backward(dev(gI))
    assert torch.equal(d3.grad, d2.grad)
    assert tacsl.check_errors() == 0


def test_full_size_against_one_pass():
    """The calibration workload (2048 maps of 320x240 over 2 sensors, realistic contact
    maps, targets of noisy intensities): the two-pass depth gradient equals the one-pass
    kernel's at every pixel to rounding, and the loss map and coefficient gradient bit
    for bit (the one-pass kernel is checked against the oracle on sampled windows in
    test_gpu_shade_mse.py)."""
    sc = synth.scene_objects(seed=2, E=1024, P=2, depth_maps="cycled", n_distinct_maps=64)
    H, W, S = sc.H, sc.W, sc.coeffs.shape[0]
    B = sc.E * sc.P
    sh = tacsl.Shading(dev(sc.coeffs), sc.pitch_x, sc.pitch_y)
    d_sid, d_dm = dev(sc.sensor_id), dev(np.ascontiguousarray(sc.depth_map.reshape(B, H, W)))
    tgt = torch.empty(B, H, W, 3, device="cuda")
    lib = ta._lib()
    assert lib.tacsl_shade_intensity(C.byref(sh.c), B, P(d_sid), P(d_dm), P(tgt), None) == 0
    tgt.add_(torch.randn(tgt.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(3)) * 10)
    lm, gc, sl, gd = _two_pass(sh, B, H, W, d_sid, d_dm, tgt, True, S=S)
    del sl
    lm1, gc1, gd1 = _one_pass(sh, B, H, W, d_sid, d_dm, tgt, True, S)
    assert tacsl.check_errors() == 0
    assert torch.equal(lm, lm1) and torch.equal(gc, gc1)
    err = (gd - gd1).abs()
    scale = gd1.abs().amax(dim=(1, 2), keepdim=True)
    assert bool((err <= 1e-5 * scale + 1e-30).all()), float((err / scale.clamp_min(1e-30)).max())
    assert bool(torch.isfinite(gd).all())


def test_flat_and_relief_warps_match_oracle():
    """Maps that are a flat gel except for a bump on some images, so that in one launch
    some warps take the flat form (every pixel of their 64-pixel segment flat) and others
    the full one: intensity, coefficient adjoint, loss map, coefficient gradient, slopes and
    depth gradient against the oracle, and the flat images' slopes against their closed
    form."""
    S, B, H, W = 2, 6, 24, 128
    px, py = 2e-4, 3e-4
    rng = np.random.default_rng(80)
    co = synth.shading_coeffs(S, H, W, 181)
    dm = np.full((B, H, W), synth.D0, np.float32)
    yy, xx = np.mgrid[0:H, 0:W]
    for b in (1, 2, 4):          # a bump of 40 um on part of the image
        cy, cx = rng.uniform(6, H - 6), rng.uniform(20, W - 20)
        dm[b] -= (4e-5 * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / 30.0)).astype(np.float32)
    sid = (np.arange(B) % S).astype(np.int32)
    _, inten, _ = oracle.shade(co, px, py, sid, dm, with_intensity=True)
    assert (np.minimum(np.abs(inten), np.abs(inten - 255)) > CLAMP_MARGIN).all()
    tgt = np.clip(inten + rng.normal(0, 15, size=inten.shape), 0, 255).astype(np.float32)
    gI = rng.normal(size=(B, H, W, 3)).astype(np.float32)
    sh = tacsl.Shading(dev(co), px, py)
    d_sid, d_dm = dev(sid), dev(dm)
    lib = ta._lib()
    out = torch.empty(B, H, W, 3, device="cuda")
    assert lib.tacsl_shade_intensity(C.byref(sh.c), B, P(d_sid), P(d_dm), P(out), None) == 0
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - inten).max() <= 1e-3
    for mse in (True, False):
        u = dev(tgt) if mse else dev(gI)
        lm, gc, sl, gd = _two_pass(sh, B, H, W, d_sid, d_dm, u, mse, S=S)
        if mse:
            ref = G.shade_mse(co, px, py, sid, dm, tgt)
            ref_sl = G.shade_slopes(co, px, py, sid, dm, target=tgt)
            _close(lm.cpu().numpy(), ref["loss_map"], 1e-4)
        else:
            ref = G.shade_gradients(co, px, py, sid, dm, gI)
            ref_sl = G.shade_slopes(co, px, py, sid, dm, g_intensity=gI)
        _close(gc.cpu().numpy(), ref["coeffs"], 1e-3)
        _close(sl.cpu().numpy(), ref_sl, 1e-3)
        _close(gd.cpu().numpy(), ref["depth"], 1e-3)
        # a flat image's slopes: (sum_c g_c A_1c, sum_c g_c A_2c) at every pixel
        slh = sl.cpu().numpy().astype(np.float64)
        for b in (0, 3, 5):
            A = co[sid[b]].astype(np.float64)
            g = 2 * (inten[b] - tgt[b]) if mse else gI[b].astype(np.float64)
            for axis in (0, 1):
                want = (g * np.moveaxis(A[1 + axis], 0, -1)).sum(-1)
                assert np.abs(slh[b, :, :, axis] - want).max() <= 1e-4 * np.abs(want).max()
    assert tacsl.check_errors() == 0
