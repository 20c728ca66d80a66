"""GPU parity of the render adjoint (tacsl_render_depth_adjoint: the depth maps of the
column camera, Sec. III-B, differentiated w.r.t. the pad poses) against the FP64
gradient oracle, evaluated at the same hit points (the maps the library rendered), and
of the pose -> depth -> intensity chain through torch.autograd."""
import numpy as np
import pytest
import torch

import paper_2408_06506_b300 as tacsl
from oracle import grad as G
from paper_2408_06506_b300 import autograd as ta
from paper_2408_06506_b300 import synth

from gpu_common import dev

pytestmark = pytest.mark.gpu
GRAZING_BAND = 2e-3    # columns this close to the grazing threshold may be classed differently
TERM_RTOL = 1e-5       # times the sum of |terms| (float32 sums of float32 terms)
GRAD_RTOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06506_b300 import build
    build.build()
    tacsl.load()
    tacsl.check_errors(clear=True)


def _cam(H, W, pitch, z_max=3e-3):
    return dict(H=H, W=W, pitch_x=pitch, pitch_y=pitch, x0=-(W - 1) / 2 * pitch, y0=-(H - 1) / 2 * pitch,
                d0=synth.D0, z_max=z_max)


def _scene(seed, E, P=2, n=64):
    grids = synth.object_set(seed, n_obj=4, n=n)
    return synth.scene_objects(seed=seed, E=E, P=P, ny=4, nx=4, pitch=1e-3, grids=grids, depth_maps="none")


def _upstream(shape, seed):
    return np.random.default_rng(seed).normal(size=shape).astype(np.float32)


def _masked(g, ref):
    """g with the columns near the grazing threshold zeroed (both sides then agree)."""
    pz = np.abs(ref["phi_z"])
    near = np.isfinite(pz) & (np.abs(pz - G.GRAZING) < GRAZING_BAND)
    return np.where(near, 0.0, g).astype(np.float32)


def _term_bound(ref, g, cam):
    """Per pad [B, 7]: sum over differentiated columns of |g| sqrt(3) / |phi_z| (t part),
    times the largest |p| (q part): the scale of the float32 sums."""
    pz = np.abs(ref["phi_z"])
    live = np.isfinite(pz) & (pz >= G.GRAZING)
    s = np.where(live, np.abs(g) * np.sqrt(3) / np.where(live, pz, 1.0), 0.0).sum(axis=(-2, -1))
    r = np.hypot(abs(cam["x0"]) + cam["W"] * cam["pitch_x"], abs(cam["y0"]) + cam["H"] * cam["pitch_y"]) + cam["z_max"]
    return np.concatenate([np.repeat(s[..., None], 3, -1), np.repeat(s[..., None] * 2 * r, 4, -1)], -1)


def _check(got, want, bound):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    err = np.abs(got - want)
    tol = GRAD_RTOL * np.abs(want) + TERM_RTOL * bound + 1e-12
    assert (err <= tol).all(), (err / tol).max()


def _adjoint(sc, d_sdfs, cam, D, g):
    return ta.render_depth_adjoint(d_sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(sc.pad_pose), D, dev(g))


@pytest.mark.parametrize("E,H,W,pitch", [(3, 96, 128, 0.125e-3), (160, 64, 64, 0.3e-3), (400, 12, 16, 1e-3)])
def test_render_adjoint_matches_oracle(E, H, W, pitch):
    """Cluster launches (few pads: up to 8 CTAs per pad) and one-CTA-per-pad launches."""
    sc = _scene(seed=E, E=E)
    cam = _cam(H, W, pitch)
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    D = tacsl.render_depth(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(sc.pad_pose))
    Dn = D.cpu().numpy().astype(np.float64)
    g = _upstream(Dn.shape, 5)
    probe = G.render_gradients(sc.grids, sc.obj_id, sc.pad_pose, g_depth=g, depth=Dn, **cam)
    g = _masked(g, probe)
    ref = G.render_gradients(sc.grids, sc.obj_id, sc.pad_pose, g_depth=g, depth=Dn, **cam)
    live = np.isfinite(ref["phi_z"]) & (np.abs(ref["phi_z"]) >= G.GRAZING)
    assert live.sum() >= 50 * min(E, 8)
    got = _adjoint(sc, sdfs, cam, D, g)
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    _check(got.cpu().numpy(), ref["pose"], _term_bound(ref, g, cam))
    again = _adjoint(sc, sdfs, cam, D, g)
    assert torch.equal(got, again)          # fixed summation order


def test_render_adjoint_edge_cases():
    sc = _scene(seed=2, E=4)
    cam = _cam(16, 20, 0.5e-3)
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    D = tacsl.render_depth(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(sc.pad_pose))
    zero = ta.render_depth_adjoint(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(sc.pad_pose), D,
                                   torch.zeros_like(D))
    assert not zero.any()
    # a miss everywhere (the pad far from every object) gives exactly zero
    far = sc.pad_pose.copy()
    far[..., 2] += 1.0
    Dfar = tacsl.render_depth(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(far))
    assert (Dfar == np.float32(synth.D0)).all()
    gz = ta.render_depth_adjoint(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(far), Dfar, torch.ones_like(Dfar))
    assert not gz.any()
    # a bad object id: NaN for that env's pads, the others unchanged, the error bit set
    tacsl.check_errors(clear=True)
    ids = sc.obj_id.copy()
    ids[1] = 99
    g = dev(_upstream(D.shape, 1))
    good = ta.render_depth_adjoint(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(sc.pad_pose), D, g)
    badg = ta.render_depth_adjoint(sdfs, tacsl.Camera(**cam), dev(ids), dev(sc.pad_pose), D, g)
    torch.cuda.synchronize()
    assert torch.isnan(badg[1]).all() and not torch.isnan(badg[[0, 2, 3]]).any()
    assert torch.equal(badg[[0, 2, 3]], good[[0, 2, 3]])
    assert tacsl.check_errors(clear=True) != 0
    # an empty batch is a no-op
    empty = torch.zeros(0, 2, 7, device="cuda")
    ta.render_depth_adjoint(sdfs, tacsl.Camera(**cam), dev(sc.obj_id[:0]), empty, D[:0], g[:0], grad_pose=empty)


def test_pose_to_intensity_chain_through_autograd():
    """L = sum(w * I(render(pose))): the shade adjoint then the render adjoint, against
    the oracle's shading gradient chained into its render gradient."""
    sc = _scene(seed=31, E=6)
    H, W, pitch = 24, 32, 0.5e-3
    cam = _cam(H, W, pitch)
    co = synth.shading_coeffs(2, H, W, 5)
    sid = np.arange(sc.E * sc.P, dtype=np.int32) % 2
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    pose = dev(sc.pad_pose).requires_grad_(True)
    D = ta.render_depth(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), pose)
    I = ta.shade_intensity(dev(co), D.reshape(-1, H, W), dev(sid), pitch, pitch)
    w = _upstream(I.shape, 9)
    # the oracle's depth gradient at the library's depth maps, then its pose gradient
    Dn = D.detach().cpu().numpy().astype(np.float64)
    gD = G.shade_gradients(co, pitch, pitch, sid, Dn.reshape(-1, H, W).astype(np.float32), w)["depth"]
    gD = gD.reshape(Dn.shape)
    probe = G.render_gradients(sc.grids, sc.obj_id, sc.pad_pose, g_depth=gD, depth=Dn, **cam)
    pz = np.abs(probe["phi_z"])
    assert not (np.isfinite(pz) & (np.abs(pz - G.GRAZING) < GRAZING_BAND)).any(), "a column near the threshold"
    (I * dev(w)).sum().backward()
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    # the depth gradient of the shade adjoint carries float32 rounding of its own: a
    # relative 1e-4 of the sum of |terms|
    _check(pose.grad.cpu().numpy(), probe["pose"], 10 * _term_bound(probe, gD, cam))
    assert np.abs(probe["pose"]).max() > 0


def test_render_adjoint_full_workload_sampled():
    """The 8192 pads (4096 envs x 2) of the object scene with 320x240 maps over the 24 x
    19 mm pad, in one call; 16 sampled pads in contact against the oracle."""
    sc = synth.scene_objects(seed=2, E=4096, P=2, ny=20, nx=25, pitch=1e-3, grids=synth.object_set(2, n_obj=8, n=128),
                             depth_maps="none")
    H, W = 240, 320
    px, py = 24e-3 / W, 19e-3 / H
    cam = dict(H=H, W=W, pitch_x=px, pitch_y=py, x0=-px * W / 2 + 0.5 * px, y0=-py * H / 2 + 0.5 * py,
               d0=synth.D0, z_max=3e-3)
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    D = tacsl.render_depth(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(sc.pad_pose))
    g = torch.randn(D.shape, device="cuda", generator=torch.Generator("cuda").manual_seed(4))
    got = ta.render_depth_adjoint(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(sc.pad_pose), D, g).cpu().numpy()
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    n_hit = (D < np.float32(synth.D0)).reshape(sc.E * sc.P, -1).sum(1).cpu().numpy()
    rng = np.random.default_rng(6)
    picks = rng.choice(np.flatnonzero(n_hit > 500), 16, replace=False)
    checked = 0
    for b in picks:
        e, p = divmod(int(b), sc.P)
        gb = g[e:e + 1, p:p + 1].cpu().numpy()
        Db = D[e:e + 1, p:p + 1].cpu().numpy().astype(np.float64)
        probe = G.render_gradients(sc.grids, sc.obj_id[e:e + 1], sc.pad_pose[e:e + 1, p:p + 1], g_depth=gb, depth=Db,
                                   **cam)
        pz = np.abs(probe["phi_z"])
        if (np.isfinite(pz) & (np.abs(pz - G.GRAZING) < GRAZING_BAND)).any():
            continue        # the kernel saw this column's g: skip the pad rather than mask it
        _check(got[e, p], probe["pose"][0, 0], _term_bound(probe, gb, cam)[0, 0])
        checked += 1
    assert checked >= 8
