"""Shared helpers of the batch and serving GPU tests: small uneven scenes on the device
and per-pad / per-image comparisons with the FP64 oracle at the stated tolerances."""
import numpy as np
import torch

import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import batch as tb
from paper_2408_06506_b300 import synth

from gpu_common import (DEPTH_ATOL, PHI_F32_ERR, VT_F32_ERR, assert_forces_close, assert_rgb_close,
                        assert_wrench_close, dev, wrench_scale)


def small_scene(seed=11, E=24, no_image=0.15):
    """Uneven batch spanning the edge cases: layouts from 1 taxel up (ragged against the
    warp's 32 x 4 taxels in flight), grids of different sides, image models from below one
    1920-pixel tile to several tiles with a ragged last one, pads without image."""
    grids = synth.grid_pool(seed, 5, sides=[12, 20, 33, 48, 24])
    return synth.scene_batch(seed=seed, E=E, P=2, grids=grids, res_y=(1, 40), res_x=(1, 50), width=(8, 200),
                             n_size_class=4, no_image_frac=no_image)


class Dev:
    """The scene on the device, with its plan and packed depth maps."""

    def __init__(self, sc, n_sdf=None):
        self.sc = sc
        grids = sc.grids if n_sdf is None else sc.grids[:n_sdf]
        self.sdfs = tacsl.SdfSet.from_grids(grids)
        self.params = tacsl.ContactParams(dev(sc.k_n), dev(sc.k_d), dev(sc.k_t), dev(sc.mu))
        has_img = (sc.sensor >= 0).any()
        self.sensors = tb.SensorSet([(dev(co), px, py) for co, px, py in sc.models]) if has_img else None
        self.plan = tb.BatchPlan(sc.obj_id, sc.layout, sc.sensor, sc.layout_first, sc.layout_count, self.sensors)
        self.taxels = dev(sc.taxels)
        self.pose = dev(sc.pad_pose)
        self.twist = dev(sc.pad_twist)
        maps = [m.reshape(-1) for m in sc.depth_maps if m is not None]
        self.depth_map = dev(np.concatenate(maps)) if maps else torch.zeros(4, device="cuda")

    def step(self, out=None):
        return self.plan.step(self.sdfs, self.params, self.taxels, self.pose, self.twist, self.depth_map, out=out)

    def views(self, out, b):
        """(depth, f_n, f_t) of pad b and its RGB image (or None)."""
        sc, p = self.sc, self.plan
        T = int(sc.layout_count[sc.layout[b]])
        o = int(p.taxel_offset[b])
        img = None
        if sc.sensor[b] >= 0:
            co = sc.models[sc.sensor[b]][0]
            H, W = co.shape[2], co.shape[3]
            q = int(p.pixel_offset[b])
            img = out["rgb"][q:q + H * W].reshape(H, W, 3)
        return out["depth"][o:o + T], out["f_n"][o:o + T], out["f_t"][o:o + T], img


def layout_taxels(sc, b):
    l = sc.layout[b]
    return sc.taxels[sc.layout_first[l]:sc.layout_first[l] + sc.layout_count[l]]


def oracle_pad(orc, sc, b):
    return orc.penalty_forces(sc.grids, layout_taxels(sc, b), sc.obj_id[b:b + 1], sc.pad_pose[b][None, None],
                              sc.pad_twist[b][None, None], sc.k_n[b], sc.k_d[b], sc.k_t[b], sc.mu[b])


def check_pad(sc, b, ref, depth, fn, ft, wr):
    depth = depth.cpu().numpy()[None, None]
    fn = fn.cpu().numpy()[None, None]
    ft = ft.cpu().numpy()[None, None]
    nan = np.isnan(ref["depth"])
    assert np.array_equal(np.isnan(depth), nan)
    assert np.abs(np.where(nan, 0, depth - ref["depth"])).max(initial=0) <= DEPTH_ATOL
    floor = PHI_F32_ERR * float(sc.k_n[b]) + VT_F32_ERR * float(sc.k_t[b])
    assert_forces_close(fn, ref["f_n"], f"f_n pad {b}", floor)
    assert_forces_close(ft, ref["f_t"], f"f_t pad {b}", floor)
    out = (ref["depth"] == 0) & (depth == 0)
    assert not fn[out].any() and not ft[out].any()
    if wr is not None:
        tax = layout_taxels(sc, b)
        f = np.where(np.isnan(ref["f_n"]), 0, ref["f_n"] + ref["f_t"])
        arm = np.linalg.norm(tax, axis=-1).max()
        n_contact = ((np.nan_to_num(ref["depth"]) > 0) | (np.nan_to_num(depth) > 0)).sum()
        wfloor = n_contact * floor * np.array([1, 1, 1, arm, arm, arm])
        assert_wrench_close(wr.cpu().numpy()[None, None], ref["wrench"], wrench_scale(tax, f), f"wrench pad {b}",
                            abs_floor=wfloor)


def check_image(orc, sc, b, img):
    co, px, py = sc.models[sc.sensor[b]]
    ref_rgb, ref_i, bad = orc.shade(co[None], px, py, [0], sc.depth_maps[b][None], with_intensity=True)
    assert bad == 0
    assert_rgb_close(img.cpu().numpy(), ref_rgb[0], ref_i[0])


