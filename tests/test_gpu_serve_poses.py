"""GPU tests of the batched depth render (tacsl_batch_render) and of the server's pose
requests (tacsl_server_submit_poses), which carry only poses, twists and contact
parameters: the server renders each image's depth map on the device, shades it and
computes the force field, and returns only the outputs asked for.

Checked: every rendered map is bit for bit tacsl_render_depth of that pad with its
model's camera (which is checked against the FP64 oracle's column march elsewhere); a
bad object id poisons only its pad; a pose request gets the same bytes alone and mixed
with others, and the same bytes as tacsl_batch_render followed by tacsl_batch_step; its
forces match the FP64 oracle and its images match the oracle's shading of the maps it
rendered; outputs not asked for stay untouched; argument errors are refused."""
import numpy as np
import pytest
import torch

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import batch as tb
from paper_2408_06506_b300 import serve as sv
from paper_2408_06506_b300 import synth

from batch_common import Dev, check_pad, oracle_pad, small_scene
from gpu_common import assert_rgb_close, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06506_b300 import build
    build.build()
    tacsl.load()
    tacsl.check_errors(clear=True)


def cameras_for(sc, z_max=3e-3):
    """One orthographic camera per sensor model: the model's size and pixel pitch, centred
    on the pad, the undeformed gel at synth.D0."""
    cams = []
    for co, px, py in sc.models:
        H, W = co.shape[2], co.shape[3]
        cams.append(tacsl.Camera(H, W, px, py, -px * W / 2 + 0.5 * px, -py * H / 2 + 0.5 * py, synth.D0, z_max))
    return cams


@pytest.fixture(scope="module")
def scene():
    sc = small_scene(seed=31, E=26, no_image=0.15)
    return sc, tacsl.SdfSet.from_grids(sc.grids), tb.SensorSet([(dev(co), px, py) for co, px, py in sc.models]), \
        dev(sc.taxels), cameras_for(sc)


def _image_of(plan, sc, maps, b):
    co = sc.models[sc.sensor[b]][0]
    H, W = co.shape[2], co.shape[3]
    q = int(plan.pixel_offset[b])
    return maps[q:q + H * W].reshape(H, W)


def test_batch_render_equals_render_depth(scene):
    sc, sdfs, sensors, taxels, cams = scene
    d = Dev(sc)
    maps = d.plan.render(sdfs, cams, d.pose)
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    n_img = 0
    for b in range(sc.n_pad):
        if sc.sensor[b] < 0:
            continue
        n_img += 1
        ref = tacsl.render_depth(sdfs, cams[sc.sensor[b]], dev(sc.obj_id[b:b + 1]),
                                 d.pose[b].reshape(1, 1, 7).contiguous())
        assert torch.equal(_image_of(d.plan, sc, maps, b), ref.reshape(ref.shape[-2:])), f"pad {b}"
    assert n_img > 5
    # some pads touch their object: their maps read below d0 somewhere
    assert bool((maps < synth.D0).any())


def test_batch_render_bad_object_and_arguments(scene):
    sc, sdfs, sensors, taxels, cams = scene
    n_sdf = 3
    d = Dev(sc, n_sdf=n_sdf)
    maps = torch.zeros(max(d.plan.n_pixel_out, 4), device="cuda")
    d.plan.render(d.sdfs, cams, d.pose, depth_map=maps)
    flags = tacsl.check_errors(clear=True)
    bad = [b for b in range(sc.n_pad) if sc.sensor[b] >= 0 and sc.obj_id[b] >= n_sdf]
    good = [b for b in range(sc.n_pad) if sc.sensor[b] >= 0 and sc.obj_id[b] < n_sdf]
    assert bad and good
    assert flags == tacsl.DEVERR_BAD_OBJ_ID
    for b in bad:
        assert bool(torch.isnan(_image_of(d.plan, sc, maps, b)).all())
    for b in good:
        assert not bool(torch.isnan(_image_of(d.plan, sc, maps, b)).any())
    # a camera whose size differs from its sensor model is refused before any launch
    wrong = list(cams)
    m = int(sc.sensor[good[0]])
    c = cams[m].c
    wrong[m] = tacsl.Camera(c.H + 4, c.W, c.pitch_x, c.pitch_y, c.x0, c.y0, c.d0, c.z_max)
    with pytest.raises(tacsl.TacslError):
        d.plan.render(d.sdfs, wrong, d.pose, depth_map=maps)
    with pytest.raises(tacsl.TacslError):
        d.plan.render(d.sdfs, [], d.pose, depth_map=maps)


def _server(scene, **kw):
    sc, sdfs, sensors, taxels, cams = scene
    cfg = dict(hbm_budget_bytes=2 << 30, max_pads=1 << 20, n_streams=1, batch_timeout_ms=30000)
    cfg.update(kw)
    srv = sv.Server(sdfs, sensors, taxels, sc.layout_first, sc.layout_count, **cfg)
    srv.set_cameras(cams)
    return srv


def _pose_request(sc, pads):
    pads = np.asarray(pads)
    return dict(obj_id=sc.obj_id[pads], layout=sc.layout[pads], sensor=sc.sensor[pads], pad_pose=sc.pad_pose[pads],
                pad_twist=sc.pad_twist[pads], k_n=sc.k_n[pads], k_d=sc.k_d[pads], k_t=sc.k_t[pads], mu=sc.mu[pads])


ALL = ("wrench", "depth", "f_n", "f_t", "rgb", "depth_map")


def _submit(srv, r, want=ALL):
    out = srv.pose_outputs_for(r["layout"], r["sensor"], want=want)
    return srv.submit_poses(out=out, **r), out


def _clone(out):
    return {k: (v.clone() if v is not None else None) for k, v in out.items()}


def _equal(a, b, npx, keys=ALL):
    """Equal outputs (the image arrays compared over their npx pixels: a request without
    images leaves its one-pixel placeholders unwritten)."""
    return all(torch.equal(a[k][:npx], b[k][:npx]) if k in ("rgb", "depth_map") else torch.equal(a[k], b[k])
               for k in keys)


def _env_ranges(sizes):
    out, e = [], 0
    for n in sizes:
        out.append(np.arange(2 * e, 2 * (e + n)))
        e += n
    return out


def test_pose_requests_equal_alone_and_mixed(scene):
    sc = scene[0]
    groups = _env_ranges([1, 3, 2, 4, 1, 3])
    srv = _server(scene)
    alone = []
    for pads in groups:
        rid, out = _submit(srv, _pose_request(sc, pads))
        assert srv.wait(rid)[0] == 0
        alone.append(_clone(out))
    # mixed: a large pose request holds the only stream while the others queue, so they
    # are then served together in one batch; the small requests and their output buffers
    # are built before the large one goes in, so that they queue within its run time
    big = _pose_request(sc, np.tile(np.arange(sc.n_pad), 1000))
    small = [_pose_request(sc, pads) for pads in groups]
    outs = [srv.pose_outputs_for(r["layout"], r["sensor"], want=ALL) for r in small]
    big_out = srv.pose_outputs_for(big["layout"], big["sensor"], want=("wrench",))
    ids = [(srv.submit_poses(out=big_out, **big), big_out)]
    ids += [(srv.submit_poses(out=o, **r), o) for r, o in zip(small, outs)]
    for rid, _ in ids:
        assert srv.wait(rid)[0] == 0
    assert srv.stats()["max_batch_requests"] >= len(groups)
    for (rid, out), ref, pads in zip(ids[1:], alone, groups):
        npx = srv.sizes_of(sc.layout[pads], sc.sensor[pads])[1]
        assert _equal(out, ref, npx), f"request {rid} differs alone and mixed"
    srv.close()
    assert tacsl.check_errors() == 0


def test_pose_request_equals_render_then_step(scene):
    sc, sdfs, sensors, taxels, cams = scene
    pads = np.arange(sc.n_pad)
    srv = _server(scene)
    rid, out = _submit(srv, _pose_request(sc, pads))
    assert srv.wait(rid)[0] == 0
    srv.close()
    d = Dev(sc)
    maps = d.plan.render(sdfs, cams, d.pose)
    ref = d.plan.step(d.sdfs, d.params, d.taxels, d.pose, d.twist, maps)
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    npx = d.plan.n_pixel_out
    assert torch.equal(out["depth_map"][:npx], maps[:npx].cpu())
    assert torch.equal(out["rgb"][:npx], ref["rgb"][:npx].cpu())
    for k in ("depth", "f_n", "f_t", "wrench"):
        assert torch.equal(out[k], ref[k].cpu()), k


def test_pose_request_matches_oracle(orc, scene):
    """Forces against the FP64 oracle pad by pad; each image against the oracle's shading
    of the depth map the server rendered for it."""
    sc = scene[0]
    pads = np.arange(sc.n_pad)
    srv = _server(scene)
    rid, out = _submit(srv, _pose_request(sc, pads))
    assert srv.wait(rid)[0] == 0
    srv.close()
    t0 = q0 = 0
    for b in pads:
        T = int(sc.layout_count[sc.layout[b]])
        check_pad(sc, b, oracle_pad(orc, sc, b), out["depth"][t0:t0 + T], out["f_n"][t0:t0 + T],
                  out["f_t"][t0:t0 + T], out["wrench"][b])
        t0 += T
        if sc.sensor[b] >= 0:
            co, px, py = sc.models[sc.sensor[b]]
            H, W = co.shape[2], co.shape[3]
            dm = out["depth_map"][q0:q0 + H * W].numpy().reshape(1, H, W)
            ref_rgb, ref_i, bad = orc.shade(co[None], px, py, [0], dm, with_intensity=True)
            assert bad == 0
            assert_rgb_close(out["rgb"][q0:q0 + H * W].numpy().reshape(H, W, 3), ref_rgb[0], ref_i[0])
            q0 += H * W
    assert tacsl.check_errors() == 0


def test_pose_request_optional_outputs_and_refusals(scene):
    """Outputs not asked for are not written back; a pose request with images needs the
    cameras; cameras must match the sensor models."""
    sc, sdfs, sensors, taxels, cams = scene
    pads = np.arange(2 * 5)
    srv = _server(scene)
    rid, full = _submit(srv, _pose_request(sc, pads))
    assert srv.wait(rid)[0] == 0
    rid, only = _submit(srv, _pose_request(sc, pads), want=("wrench",))
    assert srv.wait(rid)[0] == 0
    assert all(only[k] is None for k in ALL if k != "wrench")
    assert torch.equal(only["wrench"], full["wrench"])
    # the image-free forces of the same pads, with the images dropped (sensor -1)
    r = _pose_request(sc, pads)
    r["sensor"] = -np.ones(len(pads), np.int32)
    rid, noimg = _submit(srv, r, want=("wrench", "depth", "f_n", "f_t"))
    assert srv.wait(rid)[0] == 0
    for k in ("wrench", "depth", "f_n", "f_t"):
        assert torch.equal(noimg[k], full[k]), k
    with pytest.raises(tacsl.TacslError):
        srv.set_cameras(cams[:-1])
    srv.close()
    bare = sv.Server(sdfs, sensors, taxels, sc.layout_first, sc.layout_count, hbm_budget_bytes=1 << 30)
    with pytest.raises(tacsl.TacslError):
        _submit(bare, _pose_request(sc, pads))
    bare.close()
    assert tacsl.check_errors() == 0
