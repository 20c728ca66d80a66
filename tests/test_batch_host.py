"""CPU checks of the batched interface (include/tacsl_batch.h): the plan's sizes and
offsets, the packed workspace (pad schedule, image list), argument validation before
any CUDA call, and that the Python mirror of the C structs has the C layout."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import batch as tb
from paper_2408_06506_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INVALID, UNSUPPORTED = 1, 2
FAKE = 0x7F0000001000


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tb._lib()


def test_struct_layout_matches_c(tmp_path):
    fields = [f[0] for f in tb._Plan._fields_]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "tacsl_batch.h"', "int main(void) {",
           '  printf("%zu\\n", sizeof(tacsl_batch_plan));']
    src += [f'  printf("%zu\\n", offsetof(tacsl_batch_plan, {f}));' for f in fields]
    for st, py in (("tacsl_batch_desc", tb._BatchDesc), ("tacsl_batch_io", tb._BatchIO),
                   ("tacsl_sensor_model", tb._SensorModel), ("tacsl_sensor_set", tb._SensorSet)):
        src.append(f'  printf("%zu\\n", sizeof({st}));')
    src.append("  return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == C.sizeof(tb._Plan)
    for f, off in zip(fields, vals[1:1 + len(fields)]):
        assert getattr(tb._Plan, f).offset == off, f
    assert vals[1 + len(fields):] == [C.sizeof(tb._BatchDesc), C.sizeof(tb._BatchIO), C.sizeof(tb._SensorModel),
                                      C.sizeof(tb._SensorSet)]


def _batch(seed=0, n_pad=50, n_layout=6, sizes=((12, 16), (120, 160), (60, 100)), no_image=0.2):
    g = np.random.default_rng(seed)
    counts = g.integers(1, 3000, size=n_layout).astype(np.int32)
    first = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    obj = g.integers(0, 8, size=n_pad)
    layout = g.integers(0, n_layout, size=n_pad)
    sensor = g.integers(0, len(sizes), size=n_pad)
    sensor[g.random(n_pad) < no_image] = -1
    return obj, layout, sensor, first, counts, tb.SensorSet.sizes_only(sizes)


def test_plan_sizes_and_offsets(lib):
    obj, layout, sensor, first, counts, ss = _batch()
    bp = tb.BatchPlan(obj, layout, sensor, first, counts, ss, device=None)
    T = counts[layout].astype(np.int64)
    assert bp.plan.n_taxel_out == T.sum()
    assert np.array_equal(bp.taxel_offset, np.concatenate([[0], np.cumsum(T)[:-1]]))
    hw = np.array([h * w for h, w in ss.sizes], np.int64)
    px = np.where(sensor >= 0, hw[np.maximum(sensor, 0)], 0)
    assert bp.plan.n_pixel_out == px.sum()
    starts = np.concatenate([[0], np.cumsum(px)[:-1]])
    assert np.array_equal(bp.pixel_offset, np.where(sensor >= 0, starts, -1))
    assert bp.plan.n_image == (sensor >= 0).sum()
    assert bp.plan.workspace_bytes % 256 == 0
    assert bp.plan.workspace_bytes >= 256 + 32 * len(obj) + 8 * bp.plan.n_image
    assert bp.config() == {"img_block": 0, "n_stages": 0, "force_np": 4, "force_dynamic": 1}


def test_pack_schedule_and_image_list(lib):
    obj, layout, sensor, first, counts, ss = _batch(seed=1)
    bp = tb.BatchPlan(obj, layout, sensor, first, counts, ss, device=None)
    ws = bp.pack()
    assert not ws[:256].any(), "counters must start at zero"
    n = len(obj)
    sched = np.frombuffer(ws[bp.plan.off_sched:bp.plan.off_sched + 32 * n].tobytes(),
                          dtype=[("pad", "<i4"), ("T", "<i4"), ("obj", "<i4"), ("unused", "<i4"),
                                 ("first", "<i8"), ("out", "<i8")])
    T = counts[layout]
    # grouped by object, largest first within an object, ties in pad order
    assert np.array_equal(sched["pad"], np.lexsort((np.arange(n), -T, obj)))
    b = sched["pad"]
    assert np.array_equal(sched["T"], T[b])
    assert np.array_equal(sched["obj"], obj[b])
    assert np.array_equal(sched["first"], first[layout[b]])
    assert np.array_equal(sched["out"], bp.taxel_offset[b])
    img = np.frombuffer(ws[bp.plan.off_images:bp.plan.off_images + 8 * bp.plan.n_image].tobytes(), dtype="<i8")
    want = np.concatenate([bp.pixel_offset[np.flatnonzero(sensor == m)] for m in range(len(ss.sizes))])
    assert np.array_equal(img, want)
    begins = np.concatenate([[0], np.cumsum([(sensor == m).sum() for m in range(len(ss.sizes))])])
    assert list(bp.plan.model_img_begin[:len(begins)]) == list(begins)


def test_batch_without_images_needs_no_sensor_set(lib):
    obj, layout, _, first, counts, _ = _batch(seed=2)
    bp = tb.BatchPlan(obj, layout, -np.ones(len(obj)), first, counts, None, device=None)
    assert bp.plan.n_image == 0 and bp.plan.n_pixel_out == 0
    assert (bp.pixel_offset == -1).all()


def test_empty_batch(lib):
    bp = tb.BatchPlan([], [], [], [5], [3], None, device=None)
    assert bp.plan.n_pad == 0 and bp.plan.n_taxel_out == 0
    assert len(bp.pack()) == bp.plan.workspace_bytes


@pytest.mark.parametrize("case,code", [
    ("obj_range", INVALID), ("layout_range", INVALID), ("sensor_range", INVALID), ("count_zero", INVALID),
    ("count_big", INVALID), ("h_not_mult4", INVALID), ("w_not_mult4", INVALID), ("no_sensor_set", INVALID),
    ("too_many_models", INVALID), ("too_wide", UNSUPPORTED), ("negative_first", INVALID),
    ("past_pool", INVALID),
])
def test_plan_rejects(lib, case, code):
    obj, layout, sensor, first, counts, ss = _batch(seed=3, no_image=0.0)
    sizes = [(12, 16), (120, 160), (60, 100)]
    if case == "obj_range":
        obj[4] = tacsl.MAX_SDF
    elif case == "layout_range":
        layout[2] = len(counts)
    elif case == "sensor_range":
        sensor[0] = 3
    elif case == "count_zero":
        counts[1] = 0
    elif case == "count_big":
        counts[1] = 65537
    elif case == "h_not_mult4":
        ss = tb.SensorSet.sizes_only([(13, 16)] + sizes[1:])
    elif case == "w_not_mult4":
        ss = tb.SensorSet.sizes_only([(12, 18)] + sizes[1:])
    elif case == "no_sensor_set":
        ss = None
    elif case == "too_many_models":
        ss = tb.SensorSet.sizes_only([(12, 16)] * (tb.MAX_MODEL + 1))
    elif case == "too_wide":
        ss = tb.SensorSet.sizes_only([(8, 40000)] + sizes[1:])
    elif case == "negative_first":
        first[0] = -1
    n_points = int((first + counts).max()) - (1 if case == "past_pool" else 0)
    with pytest.raises(tacsl.TacslError) as ei:
        tb.BatchPlan(obj, layout, sensor, first, counts, ss, device=None, n_points=n_points)
    assert ei.value.code == code


def test_pack_rejects_other_description(lib):
    obj, layout, sensor, first, counts, ss = _batch(seed=4)
    bp = tb.BatchPlan(obj, layout, sensor, first, counts, ss, device=None)
    bp._h["obj_id"][0] ^= 1           # the description changed after planning
    with pytest.raises(tacsl.TacslError) as ei:
        bp.pack()
    assert ei.value.code == INVALID and "differs" in str(ei.value)


def _io(**kw):
    vals = dict(taxels=FAKE, pad_pose=FAKE, pad_twist=FAKE, depth=FAKE, f_n=FAKE, f_t=FAKE, wrench=FAKE,
                depth_map=FAKE, rgb=FAKE)
    vals.update(kw)
    return tb._BatchIO(**vals)


def test_step_entry_points_reject_before_cuda(lib):
    obj, layout, sensor, first, counts, ss = _batch(seed=5)
    bp = tb.BatchPlan(obj, layout, sensor, first, counts, ss, device=None)
    sdf = tacsl._Sdf()
    sdf.n[0] = sdf.n[1] = sdf.n[2] = 8
    sdf.voxel = 1e-3
    sdf.data = FAKE
    arr = (tacsl._Sdf * 1)(sdf)
    st = tacsl._SdfSet(C.cast(arr, C.POINTER(tacsl._Sdf)), 1)
    prm = tacsl._Params(FAKE, FAKE, FAKE, FAKE, 1)
    P = C.byref(bp.plan)
    # workspace missing / misaligned
    assert lib.tacsl_batch_forces(P, None, C.byref(st), C.byref(prm), C.byref(_io()), None) == INVALID
    assert lib.tacsl_batch_forces(P, FAKE + 16, C.byref(st), C.byref(prm), C.byref(_io()), None) == INVALID
    # a NULL taxel pool, a misaligned wrench
    assert lib.tacsl_batch_forces(P, FAKE, C.byref(st), C.byref(prm), C.byref(_io(taxels=None)), None) == INVALID
    assert lib.tacsl_batch_forces(P, FAKE, C.byref(st), C.byref(prm), C.byref(_io(wrench=FAKE + 2)), None) == INVALID
    # params count must be 1 or n_pad
    prm3 = tacsl._Params(FAKE, FAKE, FAKE, FAKE, 3)
    assert lib.tacsl_batch_forces(P, FAKE, C.byref(st), C.byref(prm3), C.byref(_io()), None) == INVALID
    # images: depth map alignment, model sizes must match the plan, bad launch settings
    assert lib.tacsl_batch_shade(P, FAKE, C.byref(ss.c), C.byref(_io(depth_map=FAKE + 4)), None) == INVALID
    other = tb.SensorSet.sizes_only([(12, 16), (120, 160), (60, 104)])
    assert lib.tacsl_batch_shade(P, FAKE, C.byref(other.c), C.byref(_io()), None) == INVALID
    bp.plan.img_block = 3
    assert lib.tacsl_batch_shade(P, FAKE, C.byref(ss.c), C.byref(_io()), None) == INVALID
    bp.plan.img_block = 0
    bp.plan.n_stages = 13
    assert lib.tacsl_batch_step(P, FAKE, C.byref(st), C.byref(prm), C.byref(ss.c), C.byref(_io()), None) == INVALID
    bp.plan.n_stages = 0
    bp.plan.force_np = 3
    assert lib.tacsl_batch_step(P, FAKE, C.byref(st), C.byref(prm), C.byref(ss.c), C.byref(_io()), None) == INVALID
    bp.plan.force_np = 4
    assert lib.tacsl_batch_autotune(P, FAKE, C.byref(st), C.byref(prm), C.byref(ss.c), C.byref(_io()), 0, None,
                                    None) == INVALID


def test_graph_handles(lib):
    assert lib.tacsl_graph_launch(None, None) == INVALID
    assert lib.tacsl_graph_destroy(None) == 0
    h = C.c_void_p()
    assert lib.tacsl_batch_graph_create(None, None, None, None, None, None, C.byref(h)) == INVALID
    assert not h.value
