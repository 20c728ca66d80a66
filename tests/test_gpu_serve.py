"""GPU tests of the continuous-batching server (include/tacsl_serve.h): every request's
result is bit-for-bit the same alone and mixed with others into one batch; served
results match the FP64 oracle; admission keeps the arena within the HBM budget under
concurrent submitters; and both bounded waits (a caller's deadline, a batch's time
limit) return TACSL_ERR_TIMEOUT without losing the work."""
import threading

import numpy as np
import pytest
import torch

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import batch as tb
from paper_2408_06506_b300 import serve as sv
from paper_2408_06506_b300 import synth

from batch_common import check_image, check_pad, oracle_pad, small_scene
from gpu_common import assert_forces_close, assert_rgb_close, dev

pytestmark = pytest.mark.gpu
TIMEOUT = 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06506_b300 import build
    build.build()
    tacsl.load()
    tacsl.check_errors(clear=True)


@pytest.fixture(scope="module")
def scene():
    sc = small_scene(seed=21, E=30, no_image=0.1)
    return sc, tacsl.SdfSet.from_grids(sc.grids), tb.SensorSet([(dev(co), px, py) for co, px, py in sc.models]), \
        dev(sc.taxels)


def _request(sc, pads):
    pads = np.asarray(pads)
    maps = [sc.depth_maps[b].reshape(-1) for b in pads if sc.sensor[b] >= 0]
    return dict(obj_id=sc.obj_id[pads], layout=sc.layout[pads], sensor=sc.sensor[pads], pad_pose=sc.pad_pose[pads],
                pad_twist=sc.pad_twist[pads], k_n=sc.k_n[pads], k_d=sc.k_d[pads], k_t=sc.k_t[pads], mu=sc.mu[pads],
                depth_map=np.concatenate(maps) if maps else None)


def _requests(sc, sizes, seed=0):
    """Consecutive env ranges of the given sizes (2 pads per env) as requests."""
    out, e = [], 0
    for n in sizes:
        out.append((np.arange(2 * e, 2 * (e + n)), _request(sc, np.arange(2 * e, 2 * (e + n)))))
        e += n
    return out


def _blocker(sc, repeat):
    """A large request (every pad of the scene, repeated) that keeps a stream busy."""
    pads = np.tile(np.arange(sc.n_pad), repeat)
    return _request(sc, pads)


def _server(scene, **kw):
    sc, sdfs, sensors, taxels = scene
    cfg = dict(hbm_budget_bytes=4 << 30, max_pads=1 << 20, n_streams=1, batch_timeout_ms=30000)
    cfg.update(kw)
    return sv.Server(sdfs, sensors, taxels, sc.layout_first, sc.layout_count, **cfg)


def _submit(srv, r):
    out = srv.outputs_for(r["layout"], r["sensor"])
    return srv.submit(out=out, **r), out


def _clone(out):
    return {k: v.clone() for k, v in out.items()}


def _equal(a, b):
    return all(torch.equal(a[k], b[k]) for k in a)


def test_results_equal_alone_and_mixed(scene):
    sc = scene[0]
    reqs = _requests(sc, [1, 3, 2, 5, 1, 4, 2])
    srv = _server(scene)
    alone = []
    for _, r in reqs:
        rid, out = _submit(srv, r)
        assert srv.wait(rid)[0] == 0
        alone.append(_clone(out))
    # mixed: a large request holds the only stream while the others queue, so they are
    # then served together in one batch
    big = _blocker(sc, 300)
    ids = [_submit(srv, big)]
    ids += [_submit(srv, r) for _, r in reqs]
    for rid, _ in ids:
        assert srv.wait(rid)[0] == 0
    st = srv.stats()
    assert st["max_batch_requests"] >= len(reqs)
    for (rid, out), ref in zip(ids[1:], alone):
        assert _equal(out, ref), f"request {rid} differs alone and mixed"
    srv.close()
    assert tacsl.check_errors() == 0


def test_served_results_match_oracle(orc, scene):
    sc = scene[0]
    reqs = _requests(sc, [4, 7, 3])
    srv = _server(scene, n_streams=2)
    sub = [(pads, _submit(srv, r)) for pads, r in reqs]
    for pads, (rid, out) in sub:
        assert srv.wait(rid)[0] == 0
        t = q = 0
        for b in pads:
            T = int(sc.layout_count[sc.layout[b]])
            i = int(np.flatnonzero(pads == b)[0])
            check_pad(sc, b, oracle_pad(orc, sc, b), out["depth"][t:t + T], out["f_n"][t:t + T],
                      out["f_t"][t:t + T], out["wrench"][i])
            t += T
            if sc.sensor[b] >= 0:
                co = sc.models[sc.sensor[b]][0]
                H, W = co.shape[2], co.shape[3]
                check_image(orc, sc, b, out["rgb"][q:q + H * W].reshape(H, W, 3))
                q += H * W
    srv.close()


def test_admission_within_budget_concurrent_submitters(scene):
    sc = scene[0]
    sizes = [1, 2, 3, 1, 2, 1, 3, 2, 1, 2, 3, 1]
    reqs = _requests(sc, sizes)
    # references: each request alone through the batch entry point
    refs = []
    sdfs, sensors, taxels = scene[1], scene[2], scene[3]
    for pads, _ in reqs:
        plan = tb.BatchPlan(sc.obj_id[pads], sc.layout[pads], sc.sensor[pads], sc.layout_first, sc.layout_count,
                            sensors, n_points=sc.taxels.shape[0])
        maps = [sc.depth_maps[b].reshape(-1) for b in pads if sc.sensor[b] >= 0]
        dm = dev(np.concatenate(maps)) if maps else torch.zeros(4, device="cuda")
        params = tacsl.ContactParams(*[dev(v[pads]) for v in (sc.k_n, sc.k_d, sc.k_t, sc.mu)])
        o = plan.step(sdfs, params, taxels, dev(sc.pad_pose[pads]), dev(sc.pad_twist[pads]), dm)
        refs.append({k: v.cpu() for k, v in o.items() if v is not None})
    budget = 3 << 20          # room for a few of these requests at a time
    srv = _server(scene, hbm_budget_bytes=budget, n_streams=3)
    results = {}
    lock = threading.Lock()

    def worker(idx):
        for i in idx:
            rid, out = _submit(srv, reqs[i][1])
            st, _ = srv.wait(rid)
            with lock:
                results[i] = (st, out)

    th = [threading.Thread(target=worker, args=(list(range(k, len(reqs), 3)),)) for k in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["arena_peak_bytes"] <= budget
    for i, ref in enumerate(refs):
        status, out = results[i]
        assert status == 0
        npx = ref["rgb"].shape[0]
        assert torch.equal(out["depth"], ref["depth"]) and torch.equal(out["f_n"], ref["f_n"])
        assert torch.equal(out["f_t"], ref["f_t"]) and torch.equal(out["wrench"], ref["wrench"])
        assert torch.equal(out["rgb"][:npx], ref["rgb"])
    # a request that could never fit is refused at submission
    with pytest.raises(tacsl.TacslError) as ei:
        _submit(srv, _blocker(sc, 40))
    assert ei.value.code == 2
    srv.close()


def test_bounded_waits_time_out_without_losing_work(scene):
    sc = scene[0]
    big = _blocker(sc, 300)
    # reference outputs of the large request
    srv = _server(scene)
    rid, ref = _submit(srv, big)
    # the caller's deadline: not finished after 0 ms, finished when waited for
    with pytest.raises(tacsl.TacslError) as ei:
        srv.wait(rid, timeout_ms=0)
    assert ei.value.code == TIMEOUT
    status, lat = srv.wait(rid)
    assert status == 0 and lat > 0
    srv.close()
    # the batch's time limit: the request fails with a timeout, the GPU still finishes it
    srv = _server(scene, batch_timeout_ms=1)
    rid, out = _submit(srv, big)
    status, _ = srv.wait(rid)
    assert status == TIMEOUT
    srv.close()                 # returns once every batch has finished
    assert _equal(out, ref)
    assert tacsl.check_errors() == 0


def test_full_size_request_sampled(orc):
    """A request of 2048 envs (the serving workload's largest) with uneven pads and
    images up to 640x480, served next to small ones; sampled pads and images against the
    oracle."""
    w = synth.serve_workload(seed=9, n_templates=3, env_range=(2048, 2048), n_grid=8, grid_sides=(64, 128))
    sdfs = tacsl.SdfSet.from_grids(w.grids)
    sensors = tb.SensorSet([(dev(co), px, py) for co, px, py in w.models])
    srv = sv.Server(sdfs, sensors, dev(w.taxels), w.layout_first, w.layout_count, hbm_budget_bytes=32 << 30,
                    max_pads=1 << 16, n_streams=2)
    keys = ("obj_id", "layout", "sensor", "pad_pose", "pad_twist", "k_n", "k_d", "k_t", "mu", "depth_map")
    t = w.templates[0]
    out = srv.outputs_for(t["layout"], t["sensor"])
    rid = srv.submit(out=out, **{k: t[k] for k in keys})
    assert srv.wait(rid)[0] == 0
    srv.close()
    T = w.layout_count[t["layout"]]
    toff = np.concatenate([[0], np.cumsum(T)[:-1]])
    hw = np.array([m[0].shape[2] * m[0].shape[3] for m in w.models])
    px = np.where(t["sensor"] >= 0, hw[np.maximum(t["sensor"], 0)], 0)
    poff = np.concatenate([[0], np.cumsum(px)[:-1]])
    rng = np.random.default_rng(3)
    for b in rng.choice(len(t["obj_id"]), 24, replace=False):
        l = t["layout"][b]
        tax = w.taxels[w.layout_first[l]:w.layout_first[l] + w.layout_count[l]]
        ref = orc.penalty_forces(w.grids, tax, t["obj_id"][b:b + 1], t["pad_pose"][b][None, None],
                                 t["pad_twist"][b][None, None], t["k_n"][b], t["k_d"][b], t["k_t"][b], t["mu"][b])
        s0, n = int(toff[b]), int(T[b])
        d = out["depth"][s0:s0 + n].numpy()
        assert np.abs(d - ref["depth"][0, 0]).max() <= 1e-6
        fl = 2e-8 * float(t["k_n"][b]) + 2e-7 * float(t["k_t"][b])
        assert_forces_close(out["f_n"][s0:s0 + n].numpy()[None, None], ref["f_n"], "f_n", fl)
        assert_forces_close(out["f_t"][s0:s0 + n].numpy()[None, None], ref["f_t"], "f_t", fl)
        co, ppx, ppy = w.models[t["sensor"][b]]
        H, W = co.shape[2], co.shape[3]
        q = int(poff[b])
        dm = t["depth_map"][q:q + H * W].reshape(1, H, W)
        ref_rgb, ref_i, bad = orc.shade(co[None], ppx, ppy, [0], dm, with_intensity=True)
        assert_rgb_close(out["rgb"][q:q + H * W].numpy().reshape(H, W, 3), ref_rgb[0], ref_i[0])
