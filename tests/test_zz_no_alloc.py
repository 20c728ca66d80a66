"""tacsl_batch_forces_static: the batched force field for callers that cannot give the
library device memory (a real-time loop where cudaMalloc would stall the device, a
plug-in whose host application owns all device allocations).  It keeps its pad
schedule in a fixed array inside the library instead of a caller workspace.

The test calls it through the C ABI twice in a row, on two different batches, and
checks each result against tacsl_batch_forces (which uses a caller workspace) at the
force tolerances of the other GPU tests, and the second batch pad by pad against the
FP64 oracle as well.  A call on a stream that is being captured into a CUDA graph is
refused.  It builds everything it needs itself, so it passes alone in a fresh process
as well as after the rest of the suite."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import batch as tb
from paper_2408_06506_b300 import build, synth

from batch_common import check_pad, oracle_pad
from gpu_common import (DEPTH_ATOL, PHI_F32_ERR, VT_F32_ERR, assert_forces_close, assert_wrench_close,
                        wrench_scale)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def _check_against(sc, plan, out, ref):
    """Pad by pad, the tolerances of the other GPU tests with the workspace entry point's
    result as the reference."""
    o = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items() if v is not None}
    r = {k: v.cpu().numpy().astype(np.float64) for k, v in ref.items() if v is not None}
    for b in range(sc.n_pad):
        l = sc.layout[b]
        T = int(sc.layout_count[l])
        s = slice(int(plan.taxel_offset[b]), int(plan.taxel_offset[b]) + T)
        assert np.abs(o["depth"][s] - r["depth"][s]).max() <= DEPTH_ATOL
        floor = PHI_F32_ERR * float(sc.k_n[b]) + VT_F32_ERR * float(sc.k_t[b])
        assert_forces_close(o["f_n"][s][None], r["f_n"][s][None], f"f_n pad {b}", floor)
        assert_forces_close(o["f_t"][s][None], r["f_t"][s][None], f"f_t pad {b}", floor)
        tax = sc.taxels[sc.layout_first[l]:sc.layout_first[l] + T]
        n_contact = int((r["depth"][s] > 0).sum())
        arm = np.linalg.norm(tax, axis=-1).max()
        assert_wrench_close(o["wrench"][b], r["wrench"][b], wrench_scale(tax, r["f_n"][s] + r["f_t"][s]),
                            f"wrench pad {b}", abs_floor=n_contact * floor * np.array([1, 1, 1, arm, arm, arm]))


@pytest.mark.gpu
def test_static_scratch_forces_match_workspace_forces(orc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    lib = tb._lib()
    f = lib.tacsl_batch_forces_static
    f.restype = C.c_int
    f.argtypes = [C.POINTER(tb._BatchDesc), C.POINTER(tacsl._SdfSet), C.POINTER(tacsl._Params),
                  C.POINTER(tb._BatchIO), C.c_void_p]
    tacsl.check_errors(clear=True)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    grids = synth.grid_pool(31, 4, sides=[16, 24, 40, 32])
    for seed, E in ((31, 20), (32, 7)):        # two calls in a row, different batches
        sc = synth.scene_batch(seed=seed, E=E, P=2, grids=grids, res_y=(1, 40), res_x=(1, 50), depth_maps="none",
                               width=(8, 16), n_size_class=1)
        sdfs = tacsl.SdfSet.from_grids(sc.grids)
        params = tacsl.ContactParams(_dev(sc.k_n), _dev(sc.k_d), _dev(sc.k_t), _dev(sc.mu))
        taxels, pose, twist = _dev(sc.taxels), _dev(sc.pad_pose), _dev(sc.pad_twist)
        no_img = -np.ones(sc.n_pad, np.int32)
        plan = tb.BatchPlan(sc.obj_id, sc.layout, no_img, sc.layout_first, sc.layout_count, None)
        ref = plan.forces(sdfs, params, taxels, pose, twist)
        out = plan.outputs(with_images=False)
        for v in out.values():
            v.fill_(float("nan"))
        io = plan._io(taxels, pose, twist, out)
        rc = f(C.byref(plan.desc), C.byref(sdfs.c), C.byref(params.c), C.byref(io), stream)
        assert rc == 0, lib.tacsl_last_error().decode()
        torch.cuda.synchronize()
        assert tacsl.check_errors() == 0
        _check_against(sc, plan, out, ref)
    # the second batch on its own terms: every pad against the FP64 oracle
    for b in range(sc.n_pad):
        o = int(plan.taxel_offset[b])
        T = int(sc.layout_count[sc.layout[b]])
        check_pad(sc, b, oracle_pad(orc, sc, b), out["depth"][o:o + T], out["f_n"][o:o + T], out["f_t"][o:o + T],
                  out["wrench"][b])

    # a call on a stream that is being captured is refused before it enqueues anything
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        g.capture_begin()
        try:
            rc = f(C.byref(plan.desc), C.byref(sdfs.c), C.byref(params.c), C.byref(io), C.c_void_p(side.cuda_stream))
        finally:
            g.capture_end()
    assert rc == 2 and "captured" in lib.tacsl_last_error().decode()
    torch.cuda.synchronize()

    # beyond the array's capacity: refused on the host, nothing launched
    n = 65529
    ids, first, count = np.zeros(n, np.int32), np.zeros(1, np.int64), np.ones(1, np.int32)
    desc = tb._BatchDesc(n, ids.ctypes.data, ids.ctypes.data, None, 1, first.ctypes.data, count.ctypes.data, 1)
    rc = f(C.byref(desc), None, None, None, stream)
    assert rc == 1  # io is NULL: invalid before anything else
    io = tb._BatchIO()
    rc = f(C.byref(desc), None, None, C.byref(io), stream)
    assert rc == 2 and "65528" in lib.tacsl_last_error().decode()
