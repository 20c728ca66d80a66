"""GPU parity of depth-map rendering (the column march of the in-sensor camera,
Sec. III-B) against the FP64 oracle, and of the render-from-poses step."""
from types import SimpleNamespace

import numpy as np
import pytest
import torch

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import synth

from gpu_common import DEPTH_ATOL, dev, scene_to_device

pytestmark = pytest.mark.gpu
TANGENT_PHI = 2e-6     # a column this close to the surface may flip hit/miss or move the hit
MAX_TANGENT_FRAC = 5e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06506_b300 import build
    build.build()
    tacsl.load()
    tacsl.check_errors(clear=True)


def _camera(sc, z_max=3e-3):
    ext_x, ext_y = sc.pitch_x * sc.W, sc.pitch_y * sc.H
    return dict(H=sc.H, W=sc.W, pitch_x=sc.pitch_x, pitch_y=sc.pitch_y, x0=-ext_x / 2 + 0.5 * sc.pitch_x,
                y0=-ext_y / 2 + 0.5 * sc.pitch_y, d0=synth.D0, z_max=z_max)


def _gpu_phi_at(sdfs, sc, b, zs, ii, jj, cam):
    """phi the GPU sees at pad-frame column points (x_i, y_j, z) of pad b."""
    e = b // sc.P
    pose = sc.pad_pose.reshape(-1, 7)[b].astype(np.float64)
    R = synth.quat_to_matrix(pose[3:])
    p = np.stack([cam["x0"] + ii * cam["pitch_x"], cam["y0"] + jj * cam["pitch_y"], zs], -1) @ R.T + pose[:3]
    ids = np.full(len(zs), sc.obj_id[e], np.int32)
    phi, _ = tacsl.sdf_query(sdfs, dev(p.astype(np.float32)), dev(ids))
    return phi.cpu().numpy().astype(np.float64)


def _check_render(orc, sc, sdfs, D_gpu, cam):
    D_ref, bad = orc.render_depth(sc.grids, sc.obj_id, sc.pad_pose, cam["H"], cam["W"], cam["pitch_x"],
                                  cam["pitch_y"], cam["x0"], cam["y0"], cam["d0"], cam["z_max"])
    D_gpu = D_gpu.reshape(D_ref.shape).astype(np.float64)
    nan = np.isnan(D_ref)
    assert np.array_equal(np.isnan(D_gpu), nan)
    diff = np.abs(np.where(nan, 0, D_gpu - D_ref))
    off = diff > DEPTH_ATOL
    n_off = int(off.sum())
    assert n_off <= MAX_TANGENT_FRAC * D_ref.size, f"{n_off} pixels off"
    # every disagreement must be a near-tangent column: each side's hit point lies on the
    # surface as seen by the other side
    d0 = np.float64(np.float32(cam["d0"]))
    for idx in zip(*np.nonzero(off.reshape(-1, cam["H"], cam["W"]))):
        b, j, i = (int(v) for v in idx)
        e = b // sc.P
        grid = sc.grids[sc.obj_id[e]]
        pose = sc.pad_pose.reshape(-1, 7)[b]
        zg = -(d0 - D_gpu.reshape(-1, cam["H"], cam["W"])[b, j, i])
        zr = -(d0 - D_ref.reshape(-1, cam["H"], cam["W"])[b, j, i])
        x, y = cam["x0"] + i * cam["pitch_x"], cam["y0"] + j * cam["pitch_y"]
        if zg < 0:
            assert orc.column_phi(grid, pose, x, y, zg) <= TANGENT_PHI
        if zr < 0:
            assert _gpu_phi_at(sdfs, sc, b, np.array([zr]), np.array([i]), np.array([j]), cam)[0] <= TANGENT_PHI
    return n_off


def test_render_sphere_pads(orc):
    sc = synth.scene_sphere_pad(seed=11, E=16)
    d = scene_to_device(sc)
    cam = _camera(sc)
    D = tacsl.render_depth(d["sdfs"], tacsl.Camera(**cam), d["obj_id"], d["pose"])
    _check_render(orc, sc, d["sdfs"], D.cpu().numpy(), cam)
    assert tacsl.check_errors() == 0


@pytest.mark.parametrize("H,W", [(24, 32), (1, 64), (7, 4), (60, 80)])
def test_render_objects(orc, H, W):
    sc = synth.scene_objects(seed=12, E=24, P=2, n=48, H=H, W=W)
    d = scene_to_device(sc)
    cam = _camera(sc, z_max=2.5e-3)
    D = tacsl.render_depth(d["sdfs"], tacsl.Camera(**cam), d["obj_id"], d["pose"])
    _check_render(orc, sc, d["sdfs"], D.cpu().numpy(), cam)


def test_render_bad_obj_id(orc):
    sc = synth.scene_objects(seed=13, E=4, P=2, n=32, H=8, W=12)
    ids = sc.obj_id.copy()
    ids[2] = -7
    d = scene_to_device(sc)
    cam = _camera(sc)
    D = tacsl.render_depth(d["sdfs"], tacsl.Camera(**cam), dev(ids), d["pose"]).cpu().numpy()
    assert np.isnan(D[2]).all() and not np.isnan(D[1]).any()
    assert tacsl.check_errors() == tacsl.DEVERR_BAD_OBJ_ID


def test_render_step_equals_render_then_step(orc):
    sc = synth.scene_objects(seed=14, E=40, P=2, n=48, H=24, W=32)
    d = scene_to_device(sc)
    cam = tacsl.Camera(**_camera(sc))
    depth, fn, ft, wr, dmap, rgb = tacsl.render_step(d["sdfs"], d["params"], d["taxels"], d["obj_id"], d["pose"],
                                                     d["twist"], d["shading"], cam, d["sensor_id"])
    dmap2 = tacsl.render_depth(d["sdfs"], cam, d["obj_id"], d["pose"])
    o = tacsl.tactile_step(d["sdfs"], d["params"], d["taxels"], d["obj_id"], d["pose"], d["twist"], d["shading"],
                           d["sensor_id"], dmap2)
    assert torch.equal(dmap, dmap2)
    for a, b in zip((depth, fn, ft, wr, rgb), o):
        assert torch.equal(a, b.view_as(a))
    # and the rendered images shade like the oracle's shading of the same maps
    from gpu_common import assert_rgb_close
    ref_rgb, ref_I, _ = orc.shade(sc.coeffs, sc.pitch_x, sc.pitch_y, sc.sensor_id, dmap.cpu().numpy(),
                                  with_intensity=True)
    assert_rgb_close(rgb.cpu().numpy(), ref_rgb, ref_I)


def _half_space_grid(nrm, n=64, h=0.5e-3):
    nrm = np.asarray(nrm, np.float64) / np.linalg.norm(nrm)
    return synth.bake_field(lambda x, y, z: nrm[0] * x + nrm[1] * y + nrm[2] * z, (n, n, n), h,
                            [-(n - 1) * h / 2] * 3), nrm


def _render_one(grid, pose, cam):
    sdfs = tacsl.SdfSet.from_grids([grid])
    return tacsl.render_depth(sdfs, tacsl.Camera(**cam), dev(np.zeros(1, np.int32)),
                              dev(np.asarray(pose, np.float32).reshape(1, 1, 7))).cpu().numpy()[0, 0]


def test_render_tilted_half_space_closed_form():
    """A half-space tilted against the pad: the first point inside on each column is
    z = -(n . p0) / (n . R e_z), to the march's resolution voxel * 2^-16 plus float32
    rounding of the grid index (a few 1e-9 m)."""
    grid, nrm = _half_space_grid([0.3, -0.2, 1.0])
    q = synth.quat_multiply(synth.quat_multiply([0.0, 1.0, 0.0, 0.0], synth.quat_from_axis_angle([1.0, 0.5, 0.0], 0.1)),
                            synth.quat_from_axis_angle([0.0, 0.0, 1.0], 0.7))
    R = synth.quat_to_matrix(np.asarray(q) / np.linalg.norm(q))
    pose = np.concatenate([-1.5e-3 * nrm + R @ np.array([0.3e-3, -0.2e-3, 0.0]), q]).astype(np.float32)
    H, W, pitch = 8, 12, 0.5e-3
    cam = dict(H=H, W=W, pitch_x=pitch, pitch_y=pitch, x0=-(W - 1) / 2 * pitch, y0=-(H - 1) / 2 * pitch,
               d0=synth.D0, z_max=3e-3)
    D = _render_one(grid, pose, cam)
    Rf = synth.quat_to_matrix(pose[3:].astype(np.float64) / np.linalg.norm(pose[3:].astype(np.float64)))
    f32 = np.float32
    xs = float(f32(cam["x0"])) + np.arange(W) * float(f32(pitch))
    ys = float(f32(cam["y0"])) + np.arange(H) * float(f32(pitch))
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    p0 = np.stack([xx, yy, np.zeros_like(xx)], -1) @ Rf.T + pose[:3].astype(np.float64)
    zc = -(p0 @ nrm) / (nrm @ Rf[:, 2])
    assert zc.max() < -1e-4 and zc.min() > -3e-3 + 1e-4
    want = float(f32(synth.D0)) + zc
    assert np.abs(D - want).max() <= grid.voxel / 65536 + 2e-8


def test_render_clamp_and_miss_exact():
    """An object below the camera's range reads exactly d0 - z_max (float32), a pad with a
    gap exactly d0, on every column."""
    grid, nrm = _half_space_grid([0.0, 0.0, 1.0], n=48)
    H, W, pitch = 8, 12, 0.5e-3
    cam = dict(H=H, W=W, pitch_x=pitch, pitch_y=pitch, x0=-(W - 1) / 2 * pitch, y0=-(H - 1) / 2 * pitch,
               d0=synth.D0, z_max=3e-3)
    flip = [0.0, 1.0, 0.0, 0.0]          # pad +z along -n: the column rises into the half-space
    deep = _render_one(grid, np.concatenate([[0.0, 0.0, -5e-3], flip]), cam)
    assert (deep == np.float32(np.float32(synth.D0) - np.float32(3e-3))).all()
    gap = _render_one(grid, np.concatenate([[0.0, 0.0, 5e-4], flip]), cam)
    assert (gap == np.float32(synth.D0)).all()


def test_render_columns_leaving_the_grid(orc):
    """A sphere's grid (a 15.5 mm box) under a 48 x 38 mm camera: most columns never enter
    the grid's domain and many cross its boundary part-way; parity with the oracle."""
    sc = synth.scene_sphere_pad(seed=15, E=12)
    d = scene_to_device(sc)
    W, H = 64, 48
    cam = dict(H=H, W=W, pitch_x=48e-3 / W, pitch_y=38e-3 / H, x0=-24e-3 + 24e-3 / W, y0=-19e-3 + 19e-3 / H,
               d0=synth.D0, z_max=3e-3)
    g = sc.grids[0]
    span = (np.asarray(g.data.shape) - 2) * g.voxel
    assert span.max() < 0.5 * 38e-3              # the camera is much wider than the domain
    D = tacsl.render_depth(d["sdfs"], tacsl.Camera(**cam), d["obj_id"], d["pose"]).cpu().numpy()
    _check_render(orc, sc, d["sdfs"], D, cam)
    assert (D < np.float32(synth.D0)).any() and (D == np.float32(synth.D0)).mean() > 0.5


def test_render_full_workload_sampled(orc):
    """The 4096-env object scene (8192 maps of 320x240, the benchmark's launch): 12
    sampled pads against the oracle's march, pad by pad, under the same rules."""
    sc = synth.scene_objects(seed=2, E=4096, P=2, depth_maps="none")
    H, W = 240, 320
    px, py = 24e-3 / W, 19e-3 / H
    cam = dict(H=H, W=W, pitch_x=px, pitch_y=py, x0=-px * W / 2 + 0.5 * px, y0=-py * H / 2 + 0.5 * py,
               d0=synth.D0, z_max=3e-3)
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    D = tacsl.render_depth(sdfs, tacsl.Camera(**cam), dev(sc.obj_id), dev(sc.pad_pose))
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    hits = (D < np.float32(synth.D0)).reshape(sc.E * sc.P, -1).sum(1).cpu().numpy()
    rng = np.random.default_rng(8)
    picks = np.concatenate([rng.choice(np.flatnonzero(hits > 1000), 8, replace=False),
                            rng.choice(np.flatnonzero(hits == 0), 4, replace=False)])
    for b in picks:
        e, p = divmod(int(b), sc.P)
        one = SimpleNamespace(grids=sc.grids, P=1, obj_id=sc.obj_id[e:e + 1],
                              pad_pose=np.ascontiguousarray(sc.pad_pose[e:e + 1, p:p + 1]))
        _check_render(orc, one, sdfs, D[e:e + 1, p:p + 1].cpu().numpy(), cam)
