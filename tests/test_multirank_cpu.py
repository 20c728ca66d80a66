"""Multi-rank path on CPU: world_size-2 gloo ranks shard the envs, each runs the step
(here the FP64 oracle, standing in for the per-rank GPU work) on its own shard with no
data exchange, and the gathered shards equal the single-process result bit for bit; the
timed-region reduction takes the max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2408_06506_b300.dist import env_shard, max_over_ranks


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_env_shard_covers_and_balances():
    for n in (0, 1, 7, 4096, 4097):
        for w in (1, 2, 3, 8):
            ranges = [env_shard(n, r, w) for r in range(w)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        env_shard(5, 2, 2)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_2408_06506_b300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = synth.scene_objects(seed=9, E=7, P=2, n=32, depth_maps="exact", H=8, W=12)
    lo, hi = env_shard(sc.E, rank, world)
    r = oracle.penalty_forces(sc.grids, sc.taxels, sc.obj_id[lo:hi], sc.pad_pose[lo:hi], sc.pad_twist[lo:hi],
                              sc.k_n[lo:hi], sc.k_d[lo:hi], sc.k_t[lo:hi], sc.mu[lo:hi], nthreads=1)
    rgb, _ = oracle.shade(sc.coeffs, sc.pitch_x, sc.pitch_y, sc.sensor_id[2 * lo:2 * hi],
                          sc.depth_map[lo:hi], nthreads=1)
    dist.barrier()
    t = max_over_ranks(0.5 + rank, dist)   # a per-rank "duration"
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), lo=lo, hi=hi, tmax=t, rgb=rgb,
             **{k: r[k] for k in ("depth", "f_n", "f_t", "wrench")})
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_without_exchange(tmp_path, orc):
    import oracle
    from paper_2408_06506_b300 import synth
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn",
                       join=True)
    sc = synth.scene_objects(seed=9, E=7, P=2, n=32, depth_maps="exact", H=8, W=12)
    full = oracle.penalty_forces(sc.grids, sc.taxels, sc.obj_id, sc.pad_pose, sc.pad_twist,
                                 sc.k_n, sc.k_d, sc.k_t, sc.mu, nthreads=1)
    rgb_full, _ = oracle.shade(sc.coeffs, sc.pitch_x, sc.pitch_y, sc.sensor_id, sc.depth_map, nthreads=1)
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    assert parts[0]["hi"] == parts[1]["lo"] and parts[1]["hi"] == sc.E
    for k in ("depth", "f_n", "f_t", "wrench"):
        np.testing.assert_array_equal(np.concatenate([p[k] for p in parts]), full[k])
    np.testing.assert_array_equal(np.concatenate([p["rgb"] for p in parts]), rgb_full)
    assert all(float(p["tmax"]) == 1.5 for p in parts)


def _grad_worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from oracle import grad as G
    from paper_2408_06506_b300 import synth
    from paper_2408_06506_b300.dist import env_shard, sum_shared_grads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = synth.scene_objects(seed=21, E=5, P=2, n=32, depth_maps="exact", H=8, W=12)
    target = np.random.default_rng(22).uniform(0, 255, size=(sc.E * sc.P, sc.H, sc.W, 3))
    lo, hi = env_shard(sc.E, rank, world)
    r = G.shade_mse(sc.coeffs, sc.pitch_x, sc.pitch_y, sc.sensor_id[2 * lo:2 * hi],
                    sc.depth_map[lo:hi].reshape(-1, sc.H, sc.W), target[2 * lo:2 * hi])
    own = r["coeffs"].copy()
    gc = torch.from_numpy(r["coeffs"].copy())
    gl = torch.from_numpy(r["loss_map"].copy())
    sum_shared_grads([gc, None, gl], dist)
    np.savez(os.path.join(out_dir, f"grad{rank}.npz"), own=own, summed=gc.numpy(), loss=gl.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_the_shared_coefficient_gradient(tmp_path):
    """The calibration's one exchange: each rank differentiates the image loss of its own
    shard (the oracle's float64 gradient standing in for the GPU adjoint); summing the
    shading-coefficient gradients over the ranks gives the gradient of the whole batch."""
    from oracle import grad as G
    from paper_2408_06506_b300 import synth
    world = 2
    mp.start_processes(_grad_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    sc = synth.scene_objects(seed=21, E=5, P=2, n=32, depth_maps="exact", H=8, W=12)
    target = np.random.default_rng(22).uniform(0, 255, size=(sc.E * sc.P, sc.H, sc.W, 3))
    full = G.shade_mse(sc.coeffs, sc.pitch_x, sc.pitch_y, sc.sensor_id, sc.depth_map.reshape(-1, sc.H, sc.W),
                       target)
    parts = [np.load(tmp_path / f"grad{r}.npz") for r in range(world)]
    scale = np.abs(full["coeffs"]).max()
    for p in parts:
        # each shard alone is not the whole gradient; the sum is, to float64 rounding
        assert np.abs(p["own"] - full["coeffs"]).max() > 1e-3 * scale
        np.testing.assert_allclose(p["summed"], full["coeffs"], rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(p["loss"], full["loss_map"], rtol=1e-12, atol=0)
    np.testing.assert_array_equal(parts[0]["summed"], parts[1]["summed"])
