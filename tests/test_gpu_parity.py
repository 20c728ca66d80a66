"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on the same
seeded inputs.  Tolerances: depth abs 1e-6 m; forces rel 1e-4 with a 1e-5 x pad-max
floor; wrench rel 1e-4 of sum |terms|; RGB within 1 LSB and only at rounding ties."""
import numpy as np
import pytest
import torch

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import synth

from gpu_common import (DEPTH_ATOL, RGB_TIE_BAND, assert_forces_close, assert_rgb_close, assert_wrench_close, dev,
                        force_abs_floor, scene_to_device, wrench_scale)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06506_b300 import build
    build.build()
    tacsl.load()
    tacsl.check_errors(clear=True)


def _oracle_forces(orc, sc, obj_id=None):
    return orc.penalty_forces(sc.grids, sc.taxels, sc.obj_id if obj_id is None else obj_id, sc.pad_pose,
                              sc.pad_twist, sc.k_n, sc.k_d, sc.k_t, sc.mu)


def _check_forces(sc, ref, depth, fn, ft, wr):
    depth, fn, ft = depth.cpu().numpy(), fn.cpu().numpy(), ft.cpu().numpy()
    nan = np.isnan(ref["depth"])
    assert np.array_equal(np.isnan(depth), nan)
    assert np.abs(np.where(nan, 0, depth - ref["depth"])).max(initial=0) <= DEPTH_ATOL
    floor = force_abs_floor(sc)
    assert_forces_close(fn, ref["f_n"], "f_n", floor)
    assert_forces_close(ft, ref["f_t"], "f_t", floor)
    # out of contact: exactly zero on both sides
    out = (ref["depth"] == 0) & (depth == 0)
    assert not fn[out].any() and not ft[out].any()
    assert np.abs(depth[ref["depth"] == 0]).max(initial=0) <= DEPTH_ATOL
    if wr is not None:
        f = np.where(np.isnan(ref["f_n"]), 0, ref["f_n"] + ref["f_t"])
        arm = np.linalg.norm(sc.taxels, axis=-1).max()
        n_contact = ((np.nan_to_num(ref["depth"]) > 0) | (np.nan_to_num(depth) > 0)).sum(-1)   # [E, P]
        wfloor = (n_contact * floor[:, :, 0])[..., None] * np.array([1, 1, 1, arm, arm, arm])
        assert_wrench_close(wr.cpu().numpy(), ref["wrench"], wrench_scale(sc.taxels, f), abs_floor=wfloor)


# ---------------------------------------------------------------------------
# SDF query
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 255, 100003])
def test_sdf_query_parity(orc, n):
    grids = synth.object_set(seed=21, n_obj=4, n=48) + [synth.bake(synth.Shape("sphere", (5e-3,)), 64, 0.25e-3)]
    g = np.random.default_rng(n)
    ids = g.integers(0, len(grids), size=n).astype(np.int32)
    ext = np.array([(gr.data.shape[2] - 1) * gr.voxel / 2 for gr in grids])[ids]
    pts = (g.uniform(-1.1, 1.1, size=(n, 3)) * ext[:, None]).astype(np.float32)
    phi_r, grad_r, bad = orc.sdf_query(grids, pts, ids)
    assert bad == 0
    sdfs = tacsl.SdfSet.from_grids(grids)
    phi, grad = tacsl.sdf_query(sdfs, dev(pts), dev(ids))
    phi, grad = phi.cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64)
    # exclude points within 1e-4 voxel of the domain boundary (either side may round across it)
    u = np.stack([(pts[:, a].astype(np.float64) - np.array([gr.origin[a] for gr in grids])[ids])
                  / np.array([gr.voxel for gr in grids])[ids] for a in range(3)], -1)
    nmax = np.array([gr.data.shape[::-1] for gr in grids])[ids] - 1.5
    near = (np.abs(u - 0.5) < 1e-4).any(-1) | (np.abs(u - nmax) < 1e-4).any(-1)
    keep = ~near
    inf_r = np.isinf(phi_r)
    assert np.array_equal(np.isinf(phi)[keep], inf_r[keep])
    fin = keep & ~inf_r
    assert np.abs(phi[fin] - phi_r[fin]).max(initial=0) <= DEPTH_ATOL
    assert np.abs(grad[fin] - grad_r[fin]).max(initial=0) <= 1e-4 * max(1.0, np.abs(grad_r[fin]).max(initial=0))
    assert not grad[keep & inf_r].any()
    assert tacsl.check_errors() == 0


def test_sdf_query_bad_id_sets_flag(orc):
    grids = [synth.bake(synth.Shape("sphere", (5e-3,)), 32, 0.5e-3)]
    pts = np.zeros((64, 3), np.float32)
    ids = np.zeros(64, np.int32)
    ids[5], ids[9] = 1, -3
    phi, grad = tacsl.sdf_query(tacsl.SdfSet.from_grids(grids), dev(pts), dev(ids))
    phi = phi.cpu().numpy()
    assert np.isnan(phi[5]) and np.isnan(phi[9]) and np.isfinite(phi[0])
    assert tacsl.check_errors() == tacsl.DEVERR_BAD_OBJ_ID
    assert tacsl.check_errors() == 0


# ---------------------------------------------------------------------------
# Force field
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("E,seed", [(1, 1), (64, 2)])
def test_penalty_forces_sphere_pad(orc, E, seed):
    sc = synth.scene_sphere_pad(seed=seed, E=E, with_images=False)
    sc.pad_twist[..., 3:] = np.random.default_rng(seed).normal(0, 1.0, size=(E, 1, 3))   # spin too
    d = scene_to_device(sc)
    depth, fn, ft, wr = tacsl.penalty_forces(d["sdfs"], d["params"], d["taxels"], d["obj_id"], d["pose"], d["twist"])
    _check_forces(sc, _oracle_forces(orc, sc), depth, fn, ft, wr)


@pytest.mark.parametrize("T_shape", [(1, 7), (20, 25), (23, 23), (40, 50)])
def test_penalty_forces_objects(orc, T_shape):
    sc = synth.scene_objects(seed=3, E=96, P=2, ny=T_shape[0], nx=T_shape[1], n=64, depth_maps="none")
    sc.k_d[:] = np.random.default_rng(4).uniform(0, 50, size=sc.E).astype(np.float32)
    d = scene_to_device(sc)
    depth, fn, ft, wr = tacsl.penalty_forces(d["sdfs"], d["params"], d["taxels"], d["obj_id"], d["pose"], d["twist"])
    _check_forces(sc, _oracle_forces(orc, sc), depth, fn, ft, wr)


def test_penalty_forces_largest_pad(orc):
    """T = 65536 taxels, the library's limit per pad (256 x 256 at 0.1 mm pitch)."""
    sc = synth.scene_objects(seed=9, E=2, P=1, ny=256, nx=256, pitch=0.1e-3, n=64, depth_maps="none")
    assert sc.T == tacsl.MAX_TAXELS
    d = scene_to_device(sc)
    depth, fn, ft, wr = tacsl.penalty_forces(d["sdfs"], d["params"], d["taxels"], d["obj_id"], d["pose"], d["twist"])
    ref = _oracle_forces(orc, sc)
    assert (ref["depth"] > 0).sum() > 100
    _check_forces(sc, ref, depth, fn, ft, wr)


def test_penalty_forces_bad_obj_id(orc):
    sc = synth.scene_objects(seed=5, E=8, P=2, n=48, depth_maps="none")
    ids = sc.obj_id.copy()
    ids[3] = 100
    d = scene_to_device(sc)
    depth, fn, ft, wr = tacsl.penalty_forces(d["sdfs"], d["params"], d["taxels"], dev(ids), d["pose"], d["twist"])
    ref = _oracle_forces(orc, sc, obj_id=ids)
    _check_forces(sc, ref, depth, fn, ft, wr)
    assert tacsl.check_errors() == tacsl.DEVERR_BAD_OBJ_ID


def test_pad_wrench_parity_and_determinism(orc):
    g = np.random.default_rng(7)
    taxels = synth.taxel_grid(20, 25, 1e-3)
    fn = g.normal(0, 3, size=(300, 500, 3)).astype(np.float32)
    ft = g.normal(0, 1, size=(300, 500, 3)).astype(np.float32)
    fn[::7] = 0
    ref = orc.pad_wrench(taxels, fn, ft)
    w1 = tacsl.pad_wrench(dev(taxels), dev(fn), dev(ft))
    w2 = tacsl.pad_wrench(dev(taxels), dev(fn), dev(ft))
    assert torch.equal(w1, w2)
    f = fn.astype(np.float64) + ft.astype(np.float64)
    assert_wrench_close(w1.cpu().numpy(), ref, wrench_scale(taxels, f))


def test_chunked_launches_match_single_launch():
    """Env sharding: the batch split into chunks gives bitwise the same per-pad results."""
    sc = synth.scene_objects(seed=8, E=200, P=2, n=48, H=24, W=32)
    d = scene_to_device(sc)
    full = tacsl.penalty_forces(d["sdfs"], d["params"], d["taxels"], d["obj_id"], d["pose"], d["twist"])
    rgb_full = tacsl.shade_image(d["shading"], d["sensor_id"], d["depth_map"])
    k_n, k_d, k_t, mu = (dev(v) for v in (sc.k_n, sc.k_d, sc.k_t, sc.mu))
    for lo, hi in [(0, 37), (37, 150), (150, 200)]:
        prm = tacsl.ContactParams(k_n[lo:hi].contiguous(), k_d[lo:hi].contiguous(), k_t[lo:hi].contiguous(),
                                  mu[lo:hi].contiguous())
        part = tacsl.penalty_forces(d["sdfs"], prm, d["taxels"], d["obj_id"][lo:hi].contiguous(),
                                    d["pose"][lo:hi].contiguous(), d["twist"][lo:hi].contiguous())
        for a, b in zip(part, full):
            assert torch.equal(a, b[lo:hi])
        rgb = tacsl.shade_image(d["shading"], d["sensor_id"][2 * lo:2 * hi].contiguous(),
                                d["depth_map"][lo:hi].contiguous())
        assert torch.equal(rgb, rgb_full[2 * lo:2 * hi])


# ---------------------------------------------------------------------------
# Tactile image
# ---------------------------------------------------------------------------

def _shade_case(orc, B, H, W, S, seed, sensor_id=None, rgb_offset=0):
    g = np.random.default_rng(seed)
    coeffs = synth.shading_coeffs(S, H, W, seed + 100)
    base = synth.D0 - np.maximum(0, g.uniform(-1e-3, 1.5e-3, size=(B, 1, 1)))
    bumps = 8e-4 * np.sin(np.arange(W)[None, None, :] * g.uniform(0.05, 0.4, size=(B, 1, 1))) \
        * np.cos(np.arange(H)[None, :, None] * g.uniform(0.05, 0.4, size=(B, 1, 1)))
    depth = (base + bumps + 2e-5 * g.standard_normal((B, H, W))).astype(np.float32)
    sid = g.integers(0, S, size=B).astype(np.int32) if sensor_id is None else sensor_id
    px, py = 0.075e-3, 0.079e-3
    ref_rgb, ref_I, bad = orc.shade(coeffs, px, py, sid, depth, with_intensity=True)
    sh = tacsl.Shading(dev(coeffs), px, py)
    if rgb_offset:
        buf = torch.full((B * H * W * 3 + rgb_offset,), 7, dtype=torch.uint8, device="cuda")
        out = buf[rgb_offset:].view(B, H, W, 3)
        rgb = tacsl.shade_image(sh, dev(sid), dev(depth), rgb=out)
    else:
        rgb = tacsl.shade_image(sh, dev(sid), dev(depth))
    return rgb.cpu().numpy(), ref_rgb, ref_I, bad


@pytest.mark.parametrize("B,H,W,S", [
    (1, 120, 160, 1),      # config-1 image
    (64, 240, 320, 2),     # config-2 images, mixed sensors
    (5, 37, 52, 3),        # single partial tile, HW % 16 != 0
    (9, 1, 64, 1),         # one row: no y derivative
    (11, 6, 4, 2),         # minimum width
    (3, 480, 640, 2),      # largest configured image (many tiles, wide halo)
    (1200, 8, 16, 1),      # more images than one run holds
    (2, 6, 4096, 1),       # widest image the shared-memory ring takes (2 stages)
    (1, 2048, 8, 1),       # tall and narrow: a tile spans many rows
])
def test_shade_image_parity(orc, B, H, W, S):
    rgb, ref_rgb, ref_I, bad = _shade_case(orc, B, H, W, S, seed=B * 31 + H)
    assert bad == 0
    assert_rgb_close(rgb, ref_rgb, ref_I)
    assert tacsl.check_errors() == 0


@pytest.mark.parametrize("offset", [1, 4, 16])
def test_shade_image_unaligned_output(orc, offset):
    """An RGB buffer at any byte offset (byte stores at 1, word stores at 4 and 16) gives the
    same bytes."""
    rgb, ref_rgb, ref_I, _ = _shade_case(orc, 7, 24, 32, 2, seed=offset, rgb_offset=offset)
    assert_rgb_close(rgb, ref_rgb, ref_I)


def test_shade_image_bad_sensor_untouched(orc):
    H, W = 16, 32
    coeffs = synth.shading_coeffs(2, H, W, 5)
    depth = np.full((4, H, W), synth.D0, np.float32)
    sid = np.array([0, 7, 1, -1], np.int32)
    out = torch.full((4, H, W, 3), 9, dtype=torch.uint8, device="cuda")
    tacsl.shade_image(tacsl.Shading(dev(coeffs), 1e-4, 1e-4), dev(sid), dev(depth), rgb=out)
    o = out.cpu().numpy()
    assert (o[1] == 9).all() and (o[3] == 9).all()
    ref, _ = orc.shade(coeffs, 1e-4, 1e-4, sid, depth, rgb_init=np.full((4, H, W, 3), 9, np.uint8))
    assert np.array_equal(o, ref)
    assert tacsl.check_errors() == tacsl.DEVERR_BAD_SENSOR_ID


# ---------------------------------------------------------------------------
# Fused tactile step
# ---------------------------------------------------------------------------

def _step(d, **kw):
    return tacsl.tactile_step(d["sdfs"], d["params"], d["taxels"], d["obj_id"], d["pose"], d["twist"],
                              d.get("shading"), d.get("sensor_id"), d.get("depth_map"), **kw)


def test_tactile_step_config1(orc):
    sc = synth.scene_sphere_pad(seed=1)
    d = scene_to_device(sc)
    depth, fn, ft, wr, rgb = _step(d)
    _check_forces(sc, _oracle_forces(orc, sc), depth, fn, ft, wr)
    ref_rgb, ref_I, _ = orc.shade(sc.coeffs, sc.pitch_x, sc.pitch_y, sc.sensor_id, sc.depth_map,
                                  with_intensity=True)
    assert_rgb_close(rgb.cpu().numpy(), ref_rgb, ref_I)


@pytest.mark.parametrize("E,ny,nx,H,W", [(37, 20, 25, 24, 32), (300, 3, 171, 60, 80)])
def test_tactile_step_matches_separate_calls(orc, E, ny, nx, H, W):
    sc = synth.scene_objects(seed=11, E=E, P=2, ny=ny, nx=nx, n=48, H=H, W=W)
    d = scene_to_device(sc)
    depth, fn, ft, wr, rgb = _step(d)
    _check_forces(sc, _oracle_forces(orc, sc), depth, fn, ft, wr)
    ref_rgb, ref_I, _ = orc.shade(sc.coeffs, sc.pitch_x, sc.pitch_y, sc.sensor_id, sc.depth_map,
                                  with_intensity=True)
    assert_rgb_close(rgb.cpu().numpy(), ref_rgb, ref_I)
    # same per-taxel and per-pixel arithmetic as the separate entry points: identical bits
    d2, fn2, ft2, wr2 = tacsl.penalty_forces(d["sdfs"], d["params"], d["taxels"], d["obj_id"], d["pose"], d["twist"])
    rgb2 = tacsl.shade_image(d["shading"], d["sensor_id"], d["depth_map"])
    assert torch.equal(depth, d2) and torch.equal(fn, fn2) and torch.equal(ft, ft2) and torch.equal(wr, wr2)
    assert torch.equal(rgb, rgb2.view_as(rgb))


def test_tactile_step_full_workload(orc):
    """4096 envs x 2 pads x 20x25 taxels, eight 128^3 objects, 8192 images of 320x240, in
    the launch configuration the benchmark times.  Every taxel is checked, and every one
    of the 8192 images: the oracle shades each distinct (depth map, sensor) pair of the
    launch once, and each image slot is compared byte by byte with the oracle image of
    its own pair (within 1 LSB, and only at rounding ties)."""
    sc = synth.scene_objects(seed=2, E=4096, P=2, depth_maps="cycled", n_distinct_maps=256)
    d = scene_to_device(sc)
    depth, fn, ft, wr, rgb = _step(d)
    torch.cuda.synchronize()
    _check_forces(sc, _oracle_forces(orc, sc), depth, fn, ft, wr)
    B = sc.E * sc.P
    nd = sc.meta["distinct_depth_maps"]
    dm = sc.depth_map.reshape(B, sc.H, sc.W)
    # slot b holds depth map b % nd (the generator cycles through the distinct maps)
    src_map = np.arange(B) % nd
    assert all(np.array_equal(dm[b], dm[src_map[b]]) for b in range(0, B, 97))
    pairs, slot_pair = np.unique(np.stack([src_map, sc.sensor_id]), axis=1, return_inverse=True)
    ref_rgb, ref_I, bad = orc.shade(sc.coeffs, sc.pitch_x, sc.pitch_y, pairs[1].astype(np.int32),
                                    dm[pairs[0]], with_intensity=True)
    assert bad == 0
    ref_rgb_d = torch.as_tensor(ref_rgb).cuda()
    # the intensity's distance from a rounding tie, where a 1-LSB difference is allowed
    Ic = np.clip(ref_I, 0, 255)
    near_tie = torch.as_tensor(np.abs(Ic - np.floor(Ic) - 0.5) < RGB_TIE_BAND).cuda()
    slot_pair_d = torch.as_tensor(slot_pair.reshape(-1)).cuda()
    n_diff = 0
    for b0 in range(0, B, 1024):
        idx = slot_pair_d[b0:b0 + 1024]
        diff = (rgb[b0:b0 + 1024].to(torch.int16) - ref_rgb_d[idx].to(torch.int16)).abs()
        assert int(diff.max()) <= 1
        off = diff > 0
        assert bool(near_tie[idx][off].all()), "1-LSB differences away from a rounding tie"
        n_diff += int(off.sum())
    assert tacsl.check_errors() == 0
