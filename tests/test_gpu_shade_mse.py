"""GPU parity of the fused image loss (tacsl_shade_mse: squared error of the clamped
intensities against target images, Sec. III-B shading, and its gradient w.r.t. the
per-pixel coefficients and the depth maps) against the FP64 gradient oracle, and against
the unfused path (tacsl_shade_intensity + a PyTorch loss + tacsl_shade_adjoint)."""
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
    return co, dm, sid, tgt, px, py


def _mse(co, dm, sid, tgt, px, py, scale=None, want=("loss", "coeffs", "depth")):
    S, _, _, H, W = co.shape
    B = dm.shape[0]
    sh = tacsl.Shading(dev(co), px, py)
    d_sid, d_dm, d_t = dev(sid), dev(dm), dev(tgt)
    lm = torch.full((S, H, W), float("nan"), device="cuda") if "loss" in want else None
    gc = torch.full((S, 6, 3, H, W), float("nan"), device="cuda") if "coeffs" in want else None
    gd = torch.full((B, H, W), float("nan"), device="cuda") if "depth" in want else None
    sc = None if scale is None else torch.tensor([scale], dtype=torch.float32, device="cuda")
    P = tacsl._ptr
    rc = ta._lib().tacsl_shade_mse(C.byref(sh.c), B, P(d_sid), P(d_dm), P(d_t), P(sc), P(lm), P(gc), P(gd), None)
    assert rc == 0, tacsl.load().tacsl_last_error()
    torch.cuda.synchronize()
    return [None if t is None else t.cpu().numpy().astype(np.float64) for t in (lm, gc, gd)]


def _close(got, want, rel):
    assert np.abs(got - want).max() <= rel * np.abs(want).max() + 1e-12, np.abs(got - want).max() / np.abs(want).max()


@pytest.mark.parametrize("S,B,H,W", [(2, 6, 24, 32), (1, 3, 7, 12), (3, 10, 16, 12), (1, 2, 1, 8), (2, 5, 9, 36)])
def test_shade_mse_matches_oracle(S, B, H, W):
    co, dm, sid, tgt, px, py = _case(3 + B, S, B, H, W)
    lm, gc, gd = _mse(co, dm, sid, tgt, px, py)
    ref = G.shade_mse(co, px, py, sid, dm, tgt)
    _close(lm, ref["loss_map"], 1e-4)
    _close(gc, ref["coeffs"], 1e-3)
    _close(gd, ref["depth"], 1e-3)
    assert tacsl.check_errors() == 0


def test_shade_mse_scale_and_partial_outputs():
    co, dm, sid, tgt, px, py = _case(8, 2, 6, 16, 20)
    lm, gc, gd = _mse(co, dm, sid, tgt, px, py)
    lm2, gc2, gd2 = _mse(co, dm, sid, tgt, px, py, scale=3.5)
    assert np.array_equal(lm, lm2)                      # the loss map carries no scale
    _close(gc2, 3.5 * gc, 1e-6)
    _close(gd2, 3.5 * gd, 1e-6)
    # each output alone equals the same output computed with the others
    lm3, _, _ = _mse(co, dm, sid, tgt, px, py, want=("loss",))
    _, gc3, _ = _mse(co, dm, sid, tgt, px, py, want=("coeffs",))
    _, _, gd3 = _mse(co, dm, sid, tgt, px, py, want=("depth",))
    assert np.array_equal(lm3, lm) and np.array_equal(gc3, gc) and np.array_equal(gd3, gd)
    # repeatable bit for bit
    lm4, gc4, gd4 = _mse(co, dm, sid, tgt, px, py)
    assert np.array_equal(lm4, lm) and np.array_equal(gc4, gc) and np.array_equal(gd4, gd)


def test_shade_mse_bad_sensor_and_empty():
    co, dm, sid, tgt, px, py = _case(9, 2, 4, 8, 12)
    bad = sid.copy()
    bad[2] = 7
    lm, gc, gd = _mse(co, dm, bad, tgt, px, py)
    keep = np.array([0, 1, 3])
    ref = G.shade_mse(co, px, py, sid[keep], dm[keep], tgt[keep])
    _close(lm, ref["loss_map"], 1e-4)
    _close(gc, ref["coeffs"], 1e-3)
    assert not gd[2].any()
    _close(gd[keep], ref["depth"], 1e-3)
    tacsl.check_errors(clear=True)
    # no images: the per-sensor sums are zero
    lm0, gc0, _ = _mse(co, dm[:0], sid[:0], tgt[:0], px, py, want=("loss", "coeffs"))
    assert not lm0.any() and not gc0.any()


def test_autograd_equals_unfused_path():
    """shade_mse through torch.autograd against shade_intensity + ((I - T)^2).sum()."""
    co, dm, sid, tgt, px, py = _case(10, 2, 8, 24, 32, relief=4e-5)
    c1 = dev(co).requires_grad_(True)
    d1 = dev(dm).requires_grad_(True)
    L1 = ta.shade_mse(c1, d1, dev(sid), px, py, dev(tgt))
    (2.0 * L1).backward()
    c2 = dev(co).requires_grad_(True)
    d2 = dev(dm).requires_grad_(True)
    I = ta.shade_intensity(c2, d2, dev(sid), px, py)
    L2 = ((I - dev(tgt)) ** 2).sum()
    (2.0 * L2).backward()
    torch.cuda.synchronize()
    assert abs(L1.item() - L2.item()) <= 1e-5 * L2.item()
    _close(c1.grad.cpu().numpy(), c2.grad.cpu().numpy(), 1e-5)
    _close(d1.grad.cpu().numpy(), d2.grad.cpu().numpy(), 1e-5)


def test_full_size_sampled_windows():
    """The calibration workload's images (2048 maps of 320x240 over 2 sensors, realistic
    contact maps): loss map, coefficient and depth gradients at sampled pixels against
    the oracle on windows cropped around them (a pixel at least 2 from a cut edge, or on
    the image's own edge, sees the same stencils as in the full image)."""
    sc = synth.scene_objects(seed=2, E=1024, P=2, depth_maps="cycled", n_distinct_maps=64)
    H, W, S = sc.H, sc.W, sc.coeffs.shape[0]
    B = sc.E * sc.P
    dm = np.ascontiguousarray(sc.depth_map.reshape(B, H, W))
    rng = np.random.default_rng(5)
    tgt_dev = torch.empty(B, H, W, 3, device="cuda")
    sh = tacsl.Shading(dev(sc.coeffs), sc.pitch_x, sc.pitch_y)
    d_sid, d_dm = dev(sc.sensor_id), dev(dm)
    ta._lib().tacsl_shade_intensity(C.byref(sh.c), B, tacsl._ptr(d_sid), tacsl._ptr(d_dm), tacsl._ptr(tgt_dev), None)
    tgt_dev.add_(torch.randn(tgt_dev.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(2)) * 10)
    lm = torch.empty(S, H, W, device="cuda")
    gc = torch.empty(S, 6, 3, H, W, device="cuda")
    gd = torch.empty(B, H, W, device="cuda")
    P = tacsl._ptr
    assert ta._lib().tacsl_shade_mse(C.byref(sh.c), B, P(d_sid), P(d_dm), P(tgt_dev), None, P(lm), P(gc), P(gd),
                                     None) == 0
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    lm, gc = lm.cpu().numpy(), gc.cpu().numpy()
    checked = 0
    for _ in range(6):
        y, x = int(rng.integers(H)), int(rng.integers(W))
        y0, y1 = max(0, y - 2), min(H, y + 3)
        x0, x1 = max(0, x - 2), min(W, x + 3)
        crop = (slice(y0, y1), slice(x0, x1))
        tb = tgt_dev[:, y0:y1, x0:x1].cpu().numpy()
        # intensities near the clamp are decided in float32 on the GPU: skip such windows
        _, inten, _ = oracle.shade(np.ascontiguousarray(sc.coeffs[:, :, :, y0:y1, x0:x1]), sc.pitch_x, sc.pitch_y,
                                   sc.sensor_id, np.ascontiguousarray(dm[:, y0:y1, x0:x1]), with_intensity=True)
        if (np.minimum(np.abs(inten), np.abs(inten - 255)) < CLAMP_MARGIN).any():
            continue
        ref = G.shade_mse(np.ascontiguousarray(sc.coeffs[:, :, :, y0:y1, x0:x1]), sc.pitch_x, sc.pitch_y,
                          sc.sensor_id, np.ascontiguousarray(dm[:, y0:y1, x0:x1]), tb)
        yy, xx = y - y0, x - x0
        for s in range(S):
            want = ref["loss_map"][s, yy, xx]
            assert abs(lm[s, y, x] - want) <= 1e-4 * abs(want) + 1e-3
            wc = ref["coeffs"][s, :, :, yy, xx]
            assert np.abs(gc[s, :, :, y, x] - wc).max() <= 1e-3 * np.abs(wc).max() + 1e-3
        gdb = gd[:, y, x].cpu().numpy()
        wd = ref["depth"][:, yy, xx]
        assert np.abs(gdb - wd).max() <= 1e-3 * np.abs(wd).max() + 1e-6
        checked += 1
    assert checked >= 3


def _at_word_offset(a):
    """A device copy of float32 array a starting one word past an 8-byte boundary."""
    flat = torch.empty(a.size + 1, dtype=torch.float32, device="cuda")
    v = flat[1:].view(a.shape)
    v.copy_(torch.as_tensor(np.ascontiguousarray(a)))
    assert v.data_ptr() % 8 == 4
    return v


@pytest.mark.parametrize("S,B,H,W", [(2, 6, 24, 32), (1, 3, 7, 12)])
def test_word_aligned_arrays_take_the_4_byte_paths(S, B, H, W):
    """The image kernels copy upstream values and store intensities 8 bytes at a time when
    the arrays allow it; at a 4-byte-aligned address they fall back to 4-byte accesses with
    the same results, bit for bit."""
    co, dm, sid, tgt, px, py = _case(40 + B, S, B, H, W)
    sh = tacsl.Shading(dev(co), px, py)
    lib, P = ta._lib(), tacsl._ptr
    d_sid, d_dm = dev(sid), dev(dm)

    def run(t, g):
        lm = torch.empty(S, H, W, device="cuda")
        gc = torch.empty(S, 6, 3, H, W, device="cuda")
        gd = torch.empty(B, H, W, device="cuda")
        gc2 = torch.empty_like(gc)
        gd2 = torch.empty_like(gd)
        assert lib.tacsl_shade_mse(C.byref(sh.c), B, P(d_sid), P(d_dm), P(t), None, P(lm), P(gc), P(gd), None) == 0
        assert lib.tacsl_shade_adjoint(C.byref(sh.c), B, P(d_sid), P(d_dm), P(g), P(gc2), P(gd2), None) == 0
        return [x.cpu().numpy() for x in (lm, gc, gd, gc2, gd2)]

    g = np.random.default_rng(41).normal(size=(B, H, W, 3)).astype(np.float32)
    aligned = run(dev(tgt), dev(g))
    shifted = run(_at_word_offset(tgt), _at_word_offset(g))
    for a, b in zip(aligned, shifted):
        assert np.array_equal(a, b)
    inten = torch.empty(B, H, W, 3, device="cuda")
    inten_w = _at_word_offset(np.zeros((B, H, W, 3), np.float32))
    for out in (inten, inten_w):
        assert lib.tacsl_shade_intensity(C.byref(sh.c), B, P(d_sid), P(d_dm), P(out), None) == 0
    assert torch.equal(inten, inten_w)
    _, ref, _ = oracle.shade(co, px, py, sid, dm, with_intensity=True)
    assert np.abs(inten.cpu().numpy() - ref).max() <= 1e-3
    assert tacsl.check_errors() == 0
