"""GPU tests of tacsl_tactile_step_host (the step from and to host memory, pipelined in
chunks over internal streams): bit for bit the results of tacsl_tactile_step on device
buffers, for ragged, single-env and oversized chunks, shared and per-env parameters, and
without images."""
import numpy as np
import pytest
import torch

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import synth

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


@pytest.fixture(scope="module")
def scene():
    return synth.scene_objects(seed=31, E=37, P=2, ny=7, nx=9, n=40, H=24, W=32, depth_maps="exact")


def _pinned(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).pin_memory()


@pytest.mark.parametrize("chunk,shared_params,images", [(8, False, True), (1, False, True), (64, False, True),
                                                         (5, True, True), (6, False, False)])
def test_host_step_equals_device_step(scene, chunk, shared_params, images):
    sc = scene
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    prm = [sc.k_n, sc.k_d, sc.k_t, sc.mu]
    if shared_params:
        prm = [v[:1] for v in prm]
    params = tacsl.ContactParams(*[dev(v) for v in prm])
    taxels = dev(sc.taxels)
    shading = tacsl.Shading(dev(sc.coeffs), sc.pitch_x, sc.pitch_y) if images else None
    ref = tacsl.tactile_step(sdfs, params, taxels, dev(sc.obj_id), dev(sc.pad_pose), dev(sc.pad_twist), shading,
                             dev(sc.sensor_id) if images else None, dev(sc.depth_map) if images else None)
    out = tacsl.tactile_step_host(sdfs, params, taxels, _pinned(sc.obj_id), _pinned(sc.pad_pose),
                                  _pinned(sc.pad_twist), shading, _pinned(sc.sensor_id) if images else None,
                                  _pinned(sc.depth_map.reshape(-1, sc.H, sc.W)) if images else None,
                                  chunk_envs=chunk)
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    for k in range(4):
        assert torch.equal(out[k], ref[k].cpu()), k
    if images:
        assert torch.equal(out[4], ref[4].cpu())
