"""Helpers for the gradient tests: which taxels lie far enough from every kink of the
force law that float32 (GPU) and float64 (oracle) take the same branch, and scenes for
the calibration workload."""
import numpy as np
import torch

from oracle import grad as G
from paper_2408_06506_b300 import synth


def safe_taxels(grid, taxels, pose, twist, kn, kd, kt, mu, phi_margin=1e-6, face_margin=2e-3, rel_margin=2e-3):
    """Bool [T]: taxels whose decisions (domain, contact, interpolation cell of the
    centre and the +-h/2 points, unilateral clamp, stick/slip, v_t = 0) hold with a
    margin, evaluated in float64."""
    with torch.no_grad():
        gt = G.grid_tensors(grid)
        data, origin, h = gt
        R = G.rotation(torch.tensor(np.asarray(pose[3:7], np.float64)))
        tax = torch.tensor(np.asarray(taxels, np.float64))
        x = tax @ R.T + torch.tensor(np.asarray(pose[:3], np.float64))
        u = ((x - origin) / h).numpy()
        n = np.array([data.shape[2], data.shape[1], data.shape[0]])
        inside = np.all((u >= 0.5) & (u <= n - 1.5), axis=1)
        edge = np.minimum(np.abs(u - 0.5), np.abs(u - (n - 1.5))).min(axis=1)
        ok = edge > face_margin
        phi, g, _ = G.sdf_eval(gt, x)
        phi = phi.numpy()
        ok &= ~(inside & (np.abs(phi) < phi_margin))
        con = inside & (phi < 0)
        for off in (0.0, 0.5, -0.5):
            fr = u + off
            ok &= ~(con & (np.abs(fr - np.rint(fr)) < face_margin).any(axis=1))
        tw = np.asarray(twist, np.float64)
        xd = tw[:3] + np.cross(np.broadcast_to(tw[3:], x.shape), x.numpy())
        gg = g.numpy()
        gn = np.linalg.norm(gg, axis=1)
        nn = gg / np.maximum(gn, 1e-300)[:, None]
        ddot = (nn * xd).sum(1)
        mag = (-kn + kd * ddot) * phi
        vt = xd - ddot[:, None] * nn
        s = np.linalg.norm(vt, axis=1)
        cap, lim = kt * s, mu * np.maximum(mag, 0)
        bad = con & ((np.abs(mag) < rel_margin * kn * np.abs(phi)) | (s < 1e-5) |
                     (np.abs(cap - lim) < rel_margin * np.maximum(cap, lim)))
        ok &= ~bad
    return ok


def calibration_scene(seed=7, E=24, P=2, ny=10, nx=12, n=48, pitch=1e-3):
    """Objects indenting pads (the calibration workload's layout at a test size), with a
    nonzero damping coefficient so every parameter has a gradient."""
    grids = synth.object_set(seed, n_obj=4, n=n)
    sc = synth.scene_objects(seed=seed, E=E, P=P, ny=ny, nx=nx, pitch=pitch, grids=grids, depth_maps="none")
    sc.k_d = np.random.default_rng(seed).uniform(1.0, 5.0, size=E).astype(np.float32)
    return sc


def upstream(sc, seed=0, wrench=True):
    """Seeded upstream gradients, zero on taxels near a kink (and no wrench gradient on a
    pad that has one, since the wrench sums every taxel)."""
    rng = np.random.default_rng(seed)
    E, P, T = sc.E, sc.P, sc.T
    mask = np.zeros((E, P, T), bool)
    for e in range(E):
        for p in range(P):
            mask[e, p] = safe_taxels(sc.grids[sc.obj_id[e]], sc.taxels, sc.pad_pose[e, p], sc.pad_twist[e, p],
                                     float(sc.k_n[e]), float(sc.k_d[e]), float(sc.k_t[e]), float(sc.mu[e]))
    gd = rng.normal(size=(E, P, T)) * mask * 1e3
    gfn = rng.normal(size=(E, P, T, 3)) * mask[..., None]
    gft = rng.normal(size=(E, P, T, 3)) * mask[..., None]
    gw = rng.normal(size=(E, P, 6)) * mask.all(axis=2)[..., None] if wrench else np.zeros((E, P, 6))
    return [a.astype(np.float32) for a in (gd, gfn, gft, gw)], mask
