"""GPU parity of the batched step (uneven pads, objects and images) against the FP64
oracle, bit-equality with the uniform entry points and across launch configurations,
CUDA-graph replay, and the device-side checks.  Tolerances as in the uniform tests:
depth abs 1e-6 m; forces rel 1e-4 with floors; wrench rel 1e-4 of sum |terms|; RGB
within 1 LSB and only at rounding ties."""
import numpy as np
import pytest
import torch

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import batch as tb
from paper_2408_06506_b300 import synth

from batch_common import Dev, check_image, check_pad, layout_taxels, oracle_pad, small_scene
from gpu_common import dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06506_b300 import build
    build.build()
    tacsl.load()
    tacsl.check_errors(clear=True)


def test_batch_step_matches_oracle(orc):
    sc = small_scene()
    d = Dev(sc)
    out = d.step()
    assert tacsl.check_errors() == 0
    assert d.plan.plan.n_image < sc.n_pad and d.plan.plan.n_image > 0
    for b in range(sc.n_pad):
        depth, fn, ft, img = d.views(out, b)
        check_pad(sc, b, oracle_pad(orc, sc, b), depth, fn, ft, out["wrench"][b])
        if img is not None:
            check_image(orc, sc, b, img)


def test_batch_equals_uniform_entry_points():
    """Per pad and per image the batch does exactly the arithmetic of
    tacsl_penalty_forces / tacsl_shade_image: the outputs are bit-for-bit equal."""
    sc = small_scene(seed=12, E=12)
    d = Dev(sc)
    out = d.step()
    for b in range(sc.n_pad):
        depth, fn, ft, img = d.views(out, b)
        l = sc.layout[b]
        params = tacsl.ContactParams(*[dev(v[b:b + 1]) for v in (sc.k_n, sc.k_d, sc.k_t, sc.mu)])
        r = tacsl.penalty_forces(d.sdfs, params, dev(layout_taxels(sc, b)), dev(sc.obj_id[b:b + 1]),
                                 d.pose[b].reshape(1, 1, 7).contiguous(), d.twist[b].reshape(1, 1, 6).contiguous())
        assert torch.equal(r[0].reshape(-1), depth)
        assert torch.equal(r[1].reshape(-1, 3), fn)
        assert torch.equal(r[2].reshape(-1, 3), ft)
        assert torch.equal(r[3].reshape(6), out["wrench"][b])
        if img is not None:
            co, px, py = sc.models[sc.sensor[b]]
            rgb = tacsl.shade_image(tacsl.Shading(dev(co[None]), px, py), dev(np.zeros(1, np.int32)),
                                    dev(sc.depth_maps[b]))
            assert torch.equal(rgb[0], img), f"image of pad {b}"


def _snapshot(out):
    return {k: v.clone() for k, v in out.items() if v is not None}


def _same(a, b):
    return all(torch.equal(a[k], b[k]) for k in a)


def test_launch_configurations_are_bitwise_identical():
    sc = small_scene(seed=13, E=40)
    d = Dev(sc)
    base = _snapshot(d.step())
    for np_ in (2, 4):
        for dyn in (0, 1):
            for blk, ns in ((0, 0), (32, 2), (64, 3), (1024, 12)):
                d.plan.set_config(img_block=blk, n_stages=ns, force_np=np_, force_dynamic=dyn)
                out = d.plan.outputs()
                for v in out.values():
                    if v is not None:
                        v.fill_(0x55 if v.dtype == torch.uint8 else float("nan"))
                for _ in range(2):   # twice: the pad counter must be back at zero
                    d.step(out)
                assert _same(base, out), d.plan.config()
    assert tacsl.check_errors() == 0


def test_autotune_then_graph_replay():
    sc = small_scene(seed=14, E=40)
    d = Dev(sc)
    base = _snapshot(d.step())
    out = d.plan.outputs()
    ms = d.plan.autotune(d.sdfs, d.params, d.taxels, d.pose, d.twist, d.depth_map, out=out, reps=2)
    cfg = d.plan.config()
    assert ms > 0 and cfg["force_np"] in (2, 4) and cfg["force_dynamic"] in (0, 1)
    assert cfg["img_block"] in [1 << k for k in range(4, 11)] and 2 <= cfg["n_stages"] <= 12
    assert _same(base, _snapshot(d.step(out)))
    g = d.plan.graph(d.sdfs, d.params, d.taxels, d.pose, d.twist, d.depth_map, out)
    for _ in range(3):
        for v in out.values():
            if v is not None:
                v.zero_()
        g.launch()
        torch.cuda.synchronize()
        assert _same(base, out)
    g.close()
    assert tacsl.check_errors() == 0


def test_bad_object_id_poisons_only_its_pads(orc):
    sc = small_scene(seed=15, E=16, no_image=0.0)
    d = Dev(sc, n_sdf=3)          # objects 3 and 4 of the plan are missing from the SDF set
    out = d.step()
    assert tacsl.check_errors() & tacsl.DEVERR_BAD_OBJ_ID
    bad = sc.obj_id >= 3
    assert bad.any() and (~bad).any()
    for b in range(sc.n_pad):
        depth, fn, ft, img = d.views(out, b)
        if bad[b]:
            assert torch.isnan(depth).all() and torch.isnan(fn).all() and torch.isnan(out["wrench"][b]).all()
        else:
            check_pad(sc, b, oracle_pad(orc, sc, b), depth, fn, ft, out["wrench"][b])
        check_image(orc, sc, b, img)   # images do not depend on the SDF


def test_batch_without_images_and_empty_batch(orc):
    sc = small_scene(seed=16, E=8, no_image=1.0)
    d = Dev(sc)
    assert d.sensors is None and d.plan.plan.n_image == 0
    out = d.plan.forces(d.sdfs, d.params, d.taxels, d.pose, d.twist)
    for b in range(sc.n_pad):
        depth, fn, ft, _ = d.views(out, b)
        check_pad(sc, b, oracle_pad(orc, sc, b), depth, fn, ft, out["wrench"][b])
    empty = tb.BatchPlan([], [], [], [0], [1], None)
    o = empty.outputs()
    one = tacsl.ContactParams(*[dev(v[:1]) for v in (sc.k_n, sc.k_d, sc.k_t, sc.mu)])
    empty.step(d.sdfs, one, d.taxels, d.pose[:0], d.twist[:0], d.depth_map, out=o)
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0


def test_uneven_workload_full_size_sampled(orc):
    """16384 envs x 2 pads with resolutions 10x12..40x50, a pool of 32 grids of 32^3 to
    256^3 and 16 image size classes (160x120..640x480), in the tuned launch
    configuration and through a CUDA graph; sampled pads and images against the oracle,
    and every image's undeformed pixels against the background the oracle gives."""
    grids = synth.grid_pool(4, 32, 32, 256)
    sc = synth.scene_batch(seed=3, E=16384, P=2, grids=grids, depth_maps="cycled", n_distinct_maps=2)
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    params = tacsl.ContactParams(dev(sc.k_n), dev(sc.k_d), dev(sc.k_t), dev(sc.mu))
    sensors = tb.SensorSet([(dev(co), px, py) for co, px, py in sc.models])
    plan = tb.BatchPlan(sc.obj_id, sc.layout, sc.sensor, sc.layout_first, sc.layout_count, sensors)
    depth_map = torch.empty(plan.n_pixel_out, dtype=torch.float32, device="cuda")
    uploaded = {}
    for b in range(sc.n_pad):
        m = sc.depth_maps[b]
        if m is None:
            continue
        key = id(m)
        if key not in uploaded:
            uploaded[key] = dev(m.reshape(-1))
        q = int(plan.pixel_offset[b])
        depth_map[q:q + m.size].copy_(uploaded[key])
    taxels, pose, twist = dev(sc.taxels), dev(sc.pad_pose), dev(sc.pad_twist)
    out = plan.outputs()
    plan.autotune(sdfs, params, taxels, pose, twist, depth_map, out=out, reps=1)
    g = plan.graph(sdfs, params, taxels, pose, twist, depth_map, out)
    g.launch()
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    g.close()
    d = Dev.__new__(Dev)
    d.sc, d.plan = sc, plan
    rng = np.random.default_rng(0)
    T = sc.layout_count[sc.layout]
    picks = set(rng.choice(sc.n_pad, 48, replace=False).tolist())
    picks |= {int(np.argmax(T)), int(np.argmin(T))}
    for b in sorted(picks):
        depth, fn, ft, img = d.views(out, b)
        check_pad(sc, b, oracle_pad(orc, sc, b), depth, fn, ft, out["wrench"][b])
    for m in range(len(sc.models)):          # one image of every model
        b = int(np.flatnonzero(sc.sensor == m)[rng.integers(0, (sc.sensor == m).sum())])
        check_image(orc, sc, b, d.views(out, b)[3])
