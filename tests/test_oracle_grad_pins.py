"""Pins of the FP64 gradient oracle (oracle/grad.py), CPU only.

The gradient oracle restates the force law and the shading in float64 torch ops and
lets autograd differentiate them.  It is pinned to things other than itself:
  * its forward equals the C oracle's (which the other pin files fix);
  * its gradients equal float64 central differences of the C oracle, h = 1e-6 (Sec. III-C
    force law; the differentiated step of the calibration workload), on pads whose
    taxels all lie away from kinks;
  * the depth maps' gradient w.r.t. the pad pose equals central differences of the C
    oracle's render (t: h = 1e-5, q: h = 1e-3) and, for a tilted half-space, the closed
    form d D/d t = -n / (n . R e_z); grazing columns carry none;
  * closed forms: d f_n/d k_n = depth n; in stick d f_t/d k_t = f_t/k_t and in slip
    d f_t/d mu = f_t/mu; a half-space whose SDF is exactly linear; d I/d A_k = m_k; on an
    undeformed gel d I(q)/d D(q +- 1) = +-A_1(q)/(2 pitch_x), d I(q)/d D(q +- W) =
    +-A_2(q)/(2 pitch_y);
  * planted mistakes in a copy of the module fail at least one of the checks above.
"""
import importlib.util

import numpy as np
import pytest
import torch

import oracle
from oracle import grad as G0
from paper_2408_06506_b300 import synth

H_FD = 1e-6


# ---------------------------------------------------------------------------
# scenes and kink margins
# ---------------------------------------------------------------------------

def _scene(seed=3):
    grids = synth.object_set(seed, n_obj=3, n=40)
    sc = synth.scene_objects(seed=seed, E=12, P=2, ny=6, nx=7, pitch=1.5e-3, grids=grids, depth_maps="none",
                             vel_sigma=0.05)
    sc.k_d = np.full(sc.E, 3.0, np.float32)     # exercise the damping term
    return sc


def _margins_ok(G, grid, taxels, pose, twist, kn, kd, kt, mu):
    """True when every taxel of the pad is away from every kink by more than an FD step
    moves it: contact on/off, the domain boundary, interpolation cell faces (centre and
    the +-h/2 points), the unilateral clamp, stick/slip, v_t = 0."""
    with torch.no_grad():
        gt = G.grid_tensors(grid)
        R = G.rotation(torch.tensor(pose[3:7], dtype=torch.float64))
        tax = torch.tensor(taxels, dtype=torch.float64)
        x = tax @ R.T + torch.tensor(pose[:3], dtype=torch.float64)
        data, origin, h = gt
        u = ((x - origin) / h).numpy()
        n = np.array([data.shape[2], data.shape[1], data.shape[0]])
        inside = np.all((u >= 0.5) & (u <= n - 1.5), axis=1)
        edge = np.minimum(np.abs(u - 0.5), np.abs(u - (n - 1.5))).min(axis=1)
        if np.any(edge < 0.05):
            return False
        phi, g, _ = G.sdf_eval(gt, x)
        phi = phi.numpy()
        if np.any(inside & (np.abs(phi) < 2e-5)):
            return False
        con = inside & (phi < 0)
        for off in (0.0, 0.5, -0.5):
            fr = u[con] + off
            if np.any(np.abs(fr - np.rint(fr)) < 0.03):
                return False
        if con.any():
            xd = torch.tensor(twist[:3], dtype=torch.float64) + torch.cross(
                torch.tensor(twist[3:], dtype=torch.float64).expand_as(x), x, dim=1)
            gg = g.numpy()[con]
            nn = gg / np.linalg.norm(gg, axis=1, keepdims=True)
            xdc = xd.numpy()[con]
            ddot = (nn * xdc).sum(1)
            mag = (-kn + kd * ddot) * phi[con]
            if np.any(mag < 1e-3 * kn * np.abs(phi[con])):
                return False
            vt = xdc - ddot[:, None] * nn
            s = np.linalg.norm(vt, axis=1)
            if np.any(s < 1e-4):
                return False
            cap, lim = kt * s, mu * mag
            if np.any(np.abs(cap - lim) < 1e-3 * np.maximum(cap, lim)):
                return False
    return True


def _clean_pads(G, sc, want=4):
    out = []
    for e in range(sc.E):
        for p in range(sc.P):
            args = (sc.grids[sc.obj_id[e]], sc.taxels, sc.pad_pose[e, p], sc.pad_twist[e, p], float(sc.k_n[e]),
                    float(sc.k_d[e]), float(sc.k_t[e]), float(sc.mu[e]))
            if _margins_ok(G, *args):
                # keep pads in contact (otherwise every gradient is zero)
                with torch.no_grad():
                    d = G.pad_forces(G.grid_tensors(args[0]), torch.tensor(sc.taxels, dtype=torch.float64),
                                     torch.tensor(args[2], dtype=torch.float64),
                                     torch.tensor(args[3], dtype=torch.float64), *[torch.tensor(v) for v in args[4:]])[0]
                if (d > 0).sum() >= 3:
                    out.append((e, p))
        if len(out) >= want:
            break
    return out


def _weights(rng, T):
    return rng.normal(size=T), rng.normal(size=(T, 3)), rng.normal(size=(T, 3)), rng.normal(size=6)


def _c_loss(sc, e, p, pose, twist, prm, w):
    r = oracle.penalty_forces(sc.grids, sc.taxels, sc.obj_id[e:e + 1], pose[None, None], twist[None, None], *prm)
    return (np.sum(w[0] * r["depth"][0, 0]) + np.sum(w[1] * r["f_n"][0, 0]) + np.sum(w[2] * r["f_t"][0, 0]) +
            np.sum(w[3] * r["wrench"][0, 0]))


def _fd(f, x, j, h=H_FD):
    """Central difference of f at float32 vector x along component j; the step is the
    exact difference of the two float32 arguments."""
    xp, xm = x.copy(), x.copy()
    xp[j] = np.float32(x[j] + h)
    xm[j] = np.float32(x[j] - h)
    return (f(xp) - f(xm)) / (float(xp[j]) - float(xm[j]))


# ---------------------------------------------------------------------------
# checks (take the module under test, so planted mistakes can be run through them)
# ---------------------------------------------------------------------------

def check_forward_matches_c_oracle(G):
    sc = _scene()
    rng = np.random.default_rng(0)
    T = sc.T
    z = np.zeros((sc.E, sc.P, T, 3))
    out = G.force_gradients(sc.grids, sc.taxels, sc.obj_id, sc.pad_pose, sc.pad_twist, sc.k_n, sc.k_d, sc.k_t,
                            sc.mu, rng.normal(size=(sc.E, sc.P, T)), z, z)
    ref = oracle.penalty_forces(sc.grids, sc.taxels, sc.obj_id, sc.pad_pose, sc.pad_twist, sc.k_n, sc.k_d, sc.k_t,
                                sc.mu)
    assert (ref["depth"] > 0).sum() > 20
    for k in ("depth", "f_n", "f_t", "wrench"):
        scale = np.abs(ref[k]).max() + 1e-30
        assert np.abs(out[k] - ref[k]).max() <= 1e-12 * scale, k


def check_intensity_matches_c_oracle(G):
    rng = np.random.default_rng(1)
    H, W, S, B = 9, 12, 2, 3
    co = synth.shading_coeffs(S, H, W, 5)
    dm = (synth.D0 + 2e-4 * rng.normal(size=(B, H, W))).astype(np.float32)
    sid = np.array([0, 1, 1], np.int32)
    out = G.shade_gradients(co, 1e-4, 1.5e-4, sid, dm, np.zeros((B, H, W, 3)))
    _, inten, bad = oracle.shade(co, 1e-4, 1.5e-4, sid, dm, with_intensity=True)
    assert bad == 0
    assert np.abs(out["intensity"] - np.clip(inten, 0, 255)).max() <= 1e-9


def check_force_gradients_match_central_differences(G):
    sc = _scene()
    pads = _clean_pads(G, sc, want=3)
    assert len(pads) >= 2
    rng = np.random.default_rng(2)
    T = sc.T
    for e, p in pads:
        w = _weights(rng, T)
        gd = np.zeros((1, 1, T)); gd[0, 0] = w[0]
        gfn = np.zeros((1, 1, T, 3)); gfn[0, 0] = w[1]
        gft = np.zeros((1, 1, T, 3)); gft[0, 0] = w[2]
        gw = w[3][None, None]
        prm = [np.array([v[e]], np.float32) for v in (sc.k_n, sc.k_d, sc.k_t, sc.mu)]
        got = G.force_gradients(sc.grids, sc.taxels, sc.obj_id[e:e + 1], sc.pad_pose[e:e + 1, p:p + 1],
                                sc.pad_twist[e:e + 1, p:p + 1], *prm, gd, gfn, gft, gw)
        pose, tw = sc.pad_pose[e, p].copy(), sc.pad_twist[e, p].copy()
        fd_pose = np.array([_fd(lambda x: _c_loss(sc, e, p, x, tw, prm, w), pose, j) for j in range(7)])
        fd_tw = np.array([_fd(lambda x: _c_loss(sc, e, p, pose, x, prm, w), tw, j) for j in range(6)])
        fd_prm = []
        for i in range(4):
            def f(x, i=i):
                pr = list(prm)
                pr[i] = x
                return _c_loss(sc, e, p, pose, tw, pr, w)
            fd_prm.append(_fd(f, prm[i].copy(), 0, h=H_FD * max(1.0, abs(float(prm[i][0])))))
        for name, a, b in (("pose", got["pose"][0, 0], fd_pose), ("twist", got["twist"][0, 0], fd_tw),
                           ("params", np.array([got[k][0] for k in ("k_n", "k_d", "k_t", "mu")]), np.array(fd_prm))):
            assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max() + 1e-9, (name, a, b)


def check_closed_forms_kn_kt_mu(G):
    sc = _scene()
    rng = np.random.default_rng(3)
    T = sc.T
    seen_stick = seen_slip = False
    for e in range(sc.E):
        for p in range(sc.P):
            prm = [np.array([v[e]], np.float32) for v in (sc.k_n, sc.k_d, sc.k_t, sc.mu)]
            wfn = rng.normal(size=(1, 1, T, 3))
            z1, z3 = np.zeros((1, 1, T)), np.zeros((1, 1, T, 3))
            a = G.force_gradients(sc.grids, sc.taxels, sc.obj_id[e:e + 1], sc.pad_pose[e:e + 1, p:p + 1],
                                  sc.pad_twist[e:e + 1, p:p + 1], *prm, z1, wfn, z3)
            fn = a["f_n"][0, 0]
            mag = np.linalg.norm(fn, axis=1)
            on = mag > 0
            if not on.any():
                continue
            # d f_n / d k_n = depth * n  (d mag / d k_n = -phi = depth)
            want = np.sum(wfn[0, 0][on] * (a["depth"][0, 0][on, None] * fn[on] / mag[on, None]))
            assert abs(a["k_n"][0] - want) <= 1e-9 * (abs(want) + 1e-12)
            # shear: stick -> f_t = -u k_t |v_t| (d/dk_t = f_t/k_t), slip -> f_t = -u mu |f_n| (d/dmu = f_t/mu)
            wft = rng.normal(size=(1, 1, T, 3))
            b = G.force_gradients(sc.grids, sc.taxels, sc.obj_id[e:e + 1], sc.pad_pose[e:e + 1, p:p + 1],
                                  sc.pad_twist[e:e + 1, p:p + 1], *prm, z1, z3, wft)
            ft = b["f_t"][0, 0]
            ftn = np.linalg.norm(ft, axis=1)
            slip = on & (np.abs(ftn - float(prm[3][0]) * mag) <= 1e-9 * (mag + 1e-30))
            stick = on & (ftn > 0) & ~slip
            seen_slip |= slip.any()
            seen_stick |= stick.any()
            want_kt = np.sum(wft[0, 0][stick] * ft[stick]) / float(prm[2][0])
            want_mu = np.sum(wft[0, 0][slip] * ft[slip]) / float(prm[3][0])
            assert abs(b["k_t"][0] - want_kt) <= 1e-9 * (abs(want_kt) + 1e-12)
            assert abs(b["mu"][0] - want_mu) <= 1e-9 * (abs(want_mu) + 1e-12)
    assert seen_stick and seen_slip


def check_half_space(G):
    """phi = z baked on a grid (trilinear and its differences are exact for a linear
    field); an unrotated pad at depth delta with normal velocity v_z:
    F_z = T (k_n - k_d v_z) delta, so dF_z/dt_z = -T (k_n - k_d v_z), dF_z/dv_z = -T k_d delta,
    dF_z/dk_n = T delta, dF_z/dt_x = dF_z/dt_y = 0, and a rotation about z does not change F_z."""
    n, h = 24, 5e-4
    grid = synth.bake_field(lambda x, y, z: z, (n, n, n), h, [-(n - 1) * h / 2] * 3)
    tax = synth.taxel_grid(3, 4, 1e-3)
    T = tax.shape[0]
    delta, vz, kn, kd = 7.25e-4, 0.03, 1.0e4, 5.0
    pose = np.array([[[0.0, 0.0, -delta, 1.0, 0.0, 0.0, 0.0]]], np.float32)
    twist = np.array([[[0.0, 0.0, vz, 0.0, 0.0, 0.0]]], np.float32)
    gw = np.array([[[0.0, 0.0, 1.0, 0.0, 0.0, 0.0]]])       # L = F_z
    z1, z3 = np.zeros((1, 1, T)), np.zeros((1, 1, T, 3))
    r = G.force_gradients([grid], tax, [0], pose, twist, kn, kd, 100.0, 0.5, z1, z3, z3, gw)
    d, v = float(np.float32(delta)), float(np.float32(vz))
    assert abs(r["wrench"][0, 0, 2] - T * (kn - kd * v) * d) <= 1e-9 * kn * d * T
    g = r["pose"][0, 0]
    assert abs(g[2] - (-T * (kn - kd * v))) <= 1e-9 * kn * T
    assert abs(g[0]) <= 1e-9 * kn and abs(g[1]) <= 1e-9 * kn
    assert abs(g[6]) <= 1e-9 * kn          # q_z at the identity: rotation about the normal
    assert abs(r["twist"][0, 0, 2] - (-T * kd * d)) <= 1e-9 * kd * d * T
    assert abs(r["k_n"][0] - T * d) <= 1e-12 * T


def check_shading_closed_forms(G):
    rng = np.random.default_rng(4)
    H, W = 7, 9
    px, py = 1e-4, 2e-4
    co = synth.shading_coeffs(1, H, W, 9)
    # d L / d A_k[c, q] = sum_b g[b, q, c] m_k(b, q) with the C oracle's normals
    dm = (synth.D0 + 1e-4 * rng.normal(size=(2, H, W))).astype(np.float32)
    gI = rng.normal(size=(2, H, W, 3))
    out = G.shade_gradients(co, px, py, [0, 0], dm, gI)
    _, inten, _ = oracle.shade(co, px, py, [0, 0], dm, with_intensity=True)
    want = np.zeros((6, 3, H, W))
    for b in range(2):
        nrm = oracle.depth_normals(dm[b], px, py)
        m = np.stack([np.ones((H, W)), nrm[..., 0], nrm[..., 1], nrm[..., 0] ** 2, nrm[..., 1] ** 2,
                      nrm[..., 0] * nrm[..., 1]])
        live = (inten[b] > 0) & (inten[b] < 255)                  # [H, W, 3]
        for c in range(3):
            want[:, c] += m * np.where(live[..., c], gI[b, ..., c], 0.0)
    assert np.abs(out["coeffs"][0] - want).max() <= 1e-9 * np.abs(want).max()
    # undeformed gel, one-hot upstream gradient at an interior pixel q, channel c
    flat = np.full((1, H, W), synth.D0, np.float32)
    qy, qx, c = 3, 4, 1
    g1 = np.zeros((1, H, W, 3))
    g1[0, qy, qx, c] = 1.0
    gd = G.shade_gradients(co, px, py, [0], flat, g1)["depth"][0]
    A1, A2 = float(co[0, 1, c, qy, qx]), float(co[0, 2, c, qy, qx])
    px, py = float(np.float32(px)), float(np.float32(py))       # the pitches the images carry
    want = np.zeros((H, W))
    want[qy, qx + 1], want[qy, qx - 1] = A1 / (2 * px), -A1 / (2 * px)
    want[qy + 1, qx], want[qy - 1, qx] = A2 / (2 * py), -A2 / (2 * py)
    assert np.abs(gd - want).max() <= 1e-9 * np.abs(want).max()


# ---------------------------------------------------------------------------
# depth maps w.r.t. the pad pose (implicit function theorem at each column's hit)
# ---------------------------------------------------------------------------

CAM = dict(H=9, W=11, pitch_x=0.5e-3, pitch_y=0.5e-3, d0=0.02, z_max=3e-3)


def _cam(H, W, pitch_x, pitch_y, d0, z_max):
    return dict(H=H, W=W, pitch_x=pitch_x, pitch_y=pitch_y, x0=-(W - 1) / 2 * pitch_x, y0=-(H - 1) / 2 * pitch_y,
                d0=d0, z_max=z_max)


def _columns(c):
    """float64 pad-frame (x, y) of every pixel, as the float32 camera defines them."""
    f = np.float32
    xs = float(f(c["x0"])) + np.arange(c["W"]) * float(f(c["pitch_x"]))
    ys = float(f(c["y0"])) + np.arange(c["H"]) * float(f(c["pitch_y"]))
    return np.meshgrid(ys, xs, indexing="ij")[::-1]


def _quat_rot(q):
    q = np.asarray(q, np.float64)
    return synth.quat_to_matrix(q / np.linalg.norm(q))


def _half_space(nrm, n=64, h=0.5e-3):
    """phi(x) = nrm . x baked on a grid centred at the origin: trilinear interpolation is
    exact for a linear field, so the column's hit is z = -nrm.(R p0 + t) / (nrm . R e_z)."""
    nrm = np.asarray(nrm, np.float64) / np.linalg.norm(nrm)
    return synth.bake_field(lambda x, y, z: nrm[0] * x + nrm[1] * y + nrm[2] * z, (n, n, n), h,
                            [-(n - 1) * h / 2] * 3), nrm


def _z_closed(nrm, pose, xx, yy):
    R = _quat_rot(pose[3:7])
    p0 = np.stack([xx, yy, np.zeros_like(xx)], -1) @ R.T + np.asarray(pose[:3], np.float64)
    return -(p0 @ nrm) / (nrm @ R[:, 2])


def check_render_tilted_half_space(G):
    """Closed form of d D / d pose for a half-space tilted against the pad (every column
    hits it): d D / d t = -nrm / (nrm . R e_z) per column; d D / d q is the central
    difference (float64, h = 1e-7) of the closed-form hit depth itself."""
    grid, nrm = _half_space([0.3, -0.2, 1.0])
    q = synth.quat_multiply(synth.quat_multiply([0.0, 1.0, 0.0, 0.0], synth.quat_from_axis_angle([1.0, 0.5, 0.0], 0.1)),
                            synth.quat_from_axis_angle([0.0, 0.0, 1.0], 0.7))
    R = _quat_rot(q)
    pose = np.concatenate([-1.5e-3 * nrm + R @ np.array([0.3e-3, -0.2e-3, 0.0]), q]).astype(np.float32)
    c = _cam(**CAM)
    xx, yy = _columns(c)
    zc = _z_closed(nrm, pose.astype(np.float64), xx, yy)
    assert zc.max() < -1e-4 and zc.min() > -c["z_max"] + 1e-4       # every column hits inside the range
    rng = np.random.default_rng(8)
    g = rng.uniform(0.5, 1.5, size=(1, 1, c["H"], c["W"]))
    r = G.render_gradients([grid], [0], pose[None, None], g_depth=g, **c)
    got = r["pose"][0, 0]
    nd = nrm @ _quat_rot(pose[3:7].astype(np.float64))[:, 2]
    want_t = -g.sum() * nrm / nd
    assert np.abs(got[:3] - want_t).max() <= 1e-9 * np.abs(want_t).max()
    want_q = np.zeros(4)
    for j in range(4):
        pp, pm = pose.astype(np.float64), pose.astype(np.float64)
        pp[3 + j] += 1e-7
        pm[3 + j] -= 1e-7
        want_q[j] = np.sum(g[0, 0] * (_z_closed(nrm, pp, xx, yy) - _z_closed(nrm, pm, xx, yy))) / 2e-7
    # the march resolves each hit to voxel * 2^-16, which moves p_z (and so d D / d q) by as much
    assert np.abs(got[3:] - want_q).max() <= 1e-5 * np.abs(want_q).max()
    assert np.abs(want_q).min() > 1e-3 * np.abs(want_q).max()        # every quaternion component is exercised
    # grazing columns carry no derivative: the same half-space nearly along the column
    # (|d phi / dz| = 0.04) gives an exactly zero gradient although the columns hit
    q2 = synth.quat_multiply([0.0, 1.0, 0.0, 0.0], synth.quat_from_axis_angle([1.0, 0.0, 0.0], np.arccos(0.04)))
    grid2, _ = _half_space([0.0, 0.0, 1.0])
    pose2 = np.concatenate([[0.0, 0.0, -0.5e-3], q2]).astype(np.float32)
    r2 = G.render_gradients([grid2], [0], pose2[None, None], g_depth=g, **c)
    D2 = r2["depth"][0, 0]
    assert ((D2 < np.float32(0.02)) & (D2 > np.float32(0.02 - 3e-3))).sum() >= 5
    assert not r2["pose"].any()


def check_render_central_differences(G):
    """d(sum g D)/d pose against central differences of the C oracle's render (t: h = 1e-5 m,
    q: h = 1e-3) on a sphere under a tilted pad, over columns whose hit points stay away
    from interpolation cell faces by more than a step moves them.  Each rendered hit lies
    within voxel * 2^-16 above the root, so a difference errs by at most
    sum|g| voxel 2^-16 / (2 h) beyond its O(h^2) term."""
    Rs, h = 5e-3, 0.5e-3
    shape = synth.Shape("sphere", (Rs,))
    grid = synth.bake(shape, 32, h)
    q = synth.quat_multiply(synth.quat_from_axis_angle([0.3, 1.0, 0.0], 0.5), synth.quat_from_axis_angle([0, 0, 1], 1.1))
    pose = synth.place_pad(shape, q, 1.6e-3, (0.3e-3, -0.4e-3)).astype(np.float32)
    c = _cam(H=15, W=17, pitch_x=0.4e-3, pitch_y=0.4e-3, d0=0.02, z_max=3e-3)
    D, _ = oracle.render_depth([grid], [0], pose[None, None], **c)
    xx, yy = _columns(c)
    z = D[0, 0] - float(np.float32(c["d0"]))
    R = _quat_rot(pose[3:7])
    sel = np.zeros(z.shape, bool)
    for j in range(c["H"]):
        for i in range(c["W"]):
            if not (-c["z_max"] + 2e-4 < z[j, i] < -2e-4):
                continue
            x = R @ np.array([xx[j, i], yy[j, i], z[j, i]]) + pose[:3].astype(np.float64)
            u = (x - np.asarray(grid.origin, np.float64)) / grid.voxel
            if np.any(np.abs(u - np.rint(u)) < 0.12):
                continue
            dz = 1e-6
            pz = (oracle.column_phi(grid, pose, xx[j, i], yy[j, i], z[j, i] + dz) -
                  oracle.column_phi(grid, pose, xx[j, i], yy[j, i], z[j, i] - dz)) / (2 * dz)
            sel[j, i] = abs(pz) > 0.3
    assert sel.sum() >= 25, sel.sum()
    rng = np.random.default_rng(12)
    g = np.where(sel, rng.uniform(0.5, 1.5, size=sel.shape), 0.0)
    got = G.render_gradients([grid], [0], pose[None, None], g_depth=g[None, None], **c)["pose"][0, 0]

    def L(pz):
        return float(np.sum(g * oracle.render_depth([grid], [0], pz[None, None], **c)[0][0, 0]))

    eps = grid.voxel / 65536
    for j in range(7):
        hh = 1e-5 if j < 3 else 1e-3
        fd = _fd(L, pose, j, hh)
        tol = 1.2 * g.sum() * eps / (2 * hh) + 2e-3 * abs(got[j]) + 1e-9
        assert abs(got[j] - fd) <= tol, (j, got[j], fd, tol)


def check_shade_mse(G):
    """The image loss: its per-pixel map equals sum_b sum_c (I - T)^2 from the C oracle's
    float64 intensities; its gradient w.r.t. sampled coefficients (L is quadratic in them
    away from the clamp, so a central difference is exact up to rounding) and sampled
    depth pixels equals central differences of that C-oracle loss."""
    rng = np.random.default_rng(14)
    H, W, S, B = 6, 8, 2, 4
    px, py = 2e-4, 3e-4
    co = synth.shading_coeffs(S, H, W, 21)
    dm = (synth.D0 + 2e-5 * rng.normal(size=(B, H, W))).astype(np.float32)
    sid = np.array([0, 1, 1, 0], np.int32)
    _, inten, _ = oracle.shade(co, px, py, sid, dm, with_intensity=True)
    tgt = inten + rng.normal(0, 20, size=inten.shape)
    live = (inten > 0) & (inten < 255)
    assert live.mean() > 0.5
    r = G.shade_mse(co, px, py, sid, dm, tgt)
    want = np.zeros((S, H, W))
    for b in range(B):
        want[sid[b]] += ((inten[b] - tgt[b]) ** 2).sum(-1)
    assert np.abs(r["loss_map"] - want).max() <= 1e-9 * want.max()

    def L(c, d):
        _, i2, _ = oracle.shade(c, px, py, sid, d, with_intensity=True)
        return float(((i2 - tgt) ** 2).sum())

    checked = 0
    for _ in range(12):
        s_, k, c, y, x = rng.integers(S), rng.integers(6), rng.integers(3), rng.integers(H), rng.integers(W)
        if not live[sid == s_][..., c][:, y, x].all() or checked == 4:
            continue
        checked += 1
        h = 0.05
        cp, cm = co.copy(), co.copy()
        cp[s_, k, c, y, x] += np.float32(h)
        cm[s_, k, c, y, x] -= np.float32(h)
        fd = (L(cp, dm) - L(cm, dm)) / (float(cp[s_, k, c, y, x]) - float(cm[s_, k, c, y, x]))
        got = r["coeffs"][s_, k, c, y, x]
        assert abs(got - fd) <= 1e-6 * max(abs(fd), 1.0), (got, fd)
    assert checked == 4
    for _ in range(4):
        b, y, x = rng.integers(B), rng.integers(H), rng.integers(W)
        dp, dmn = dm.copy(), dm.copy()
        dp[b, y, x] += np.float32(2e-7)
        dmn[b, y, x] -= np.float32(2e-7)
        fd = (L(co, dp) - L(co, dmn)) / (float(dp[b, y, x]) - float(dmn[b, y, x]))
        got = r["depth"][b, y, x]
        assert abs(got - fd) <= 2e-3 * max(abs(fd), 1e-3 * np.abs(r["depth"]).max()), (got, fd)


def check_shade_slopes(G):
    """The pixel slopes (dL/dD_x, dL/dD_y): on a flat gel (D_x = D_y = 0, so n = 0 and
    dn/d(D_x, D_y) is the identity) they are sum_c g_c A[1, c] and sum_c g_c A[2, c] over
    the unclamped channels, g = g_intensity or 2 (I - T); on a relief their image under
    the transposed derivative stencils (built column by column from numpy.gradient:
    central inside, one-sided on the border) is the depth gradient of shade_gradients and
    shade_mse; an image with a bad sensor id keeps zero slopes."""
    rng = np.random.default_rng(15)
    H, W, S, B = 5, 8, 2, 3
    px, py = 2e-4, 3e-4
    co = synth.shading_coeffs(S, H, W, 22)
    sid = np.array([1, 0, 1], np.int32)
    flat = np.full((B, H, W), synth.D0, np.float32)
    gI = rng.normal(size=(B, H, W, 3))
    got = G.shade_slopes(co, px, py, sid, flat, g_intensity=gI)
    _, inten, _ = oracle.shade(co, px, py, sid, flat, with_intensity=True)
    live = (inten > 0) & (inten < 255)
    assert live.mean() > 0.5
    tgt = inten + rng.normal(0, 20, size=inten.shape)
    got_mse = G.shade_slopes(co, px, py, sid, flat, target=tgt)
    for b in range(B):
        A = co[sid[b]].astype(np.float64)                       # [6, 3, H, W]
        g = np.where(live[b], gI[b], 0.0)                       # [H, W, 3]
        e = np.where(live[b], 2 * (inten[b] - tgt[b]), 0.0)
        for axis in (0, 1):
            want = (g * np.moveaxis(A[1 + axis], 0, -1)).sum(-1)
            assert np.abs(got[b, :, :, axis] - want).max() <= 1e-9 * np.abs(want).max()
            want = (e * np.moveaxis(A[1 + axis], 0, -1)).sum(-1)
            assert np.abs(got_mse[b, :, :, axis] - want).max() <= 1e-9 * np.abs(want).max()
    dm = (synth.D0 + 2e-5 * rng.normal(size=(B, H, W))).astype(np.float32)
    _, inten, _ = oracle.shade(co, px, py, sid, dm, with_intensity=True)
    tgt = inten + rng.normal(0, 20, size=inten.shape)

    def transpose_stencil(sl):
        out = np.zeros((H, W))
        for y in range(H):
            for x in range(W):
                e = np.zeros((H, W))
                e[y, x] = 1.0
                # the pitches as the kernels and the oracle take them: float32 values
                out[y, x] = (sl[..., 0] * np.gradient(e, float(np.float32(px)), axis=1)).sum() + \
                    (sl[..., 1] * np.gradient(e, float(np.float32(py)), axis=0)).sum()
        return out

    sl = G.shade_slopes(co, px, py, sid, dm, g_intensity=gI)
    sl_mse = G.shade_slopes(co, px, py, sid, dm, target=tgt)
    gd = G.shade_gradients(co, px, py, sid, dm, gI)["depth"]
    gd_mse = G.shade_mse(co, px, py, sid, dm, tgt)["depth"]
    for b in range(B):
        assert np.abs(transpose_stencil(sl[b]) - gd[b]).max() <= 1e-9 * np.abs(gd[b]).max()
        assert np.abs(transpose_stencil(sl_mse[b]) - gd_mse[b]).max() <= 1e-9 * np.abs(gd_mse[b]).max()
    bad = G.shade_slopes(co, px, py, np.array([1, -1, 2], np.int32), dm, g_intensity=gI)
    assert np.array_equal(bad[0], sl[0]) and not bad[1].any() and not bad[2].any()


CHECKS = [check_forward_matches_c_oracle, check_intensity_matches_c_oracle,
          check_force_gradients_match_central_differences, check_closed_forms_kn_kt_mu, check_half_space,
          check_shading_closed_forms, check_render_tilted_half_space, check_render_central_differences,
          check_shade_mse, check_shade_slopes]


@pytest.mark.parametrize("check", CHECKS, ids=[c.__name__ for c in CHECKS])
def test_gradient_oracle(orc, check):
    check(G0)


# ---------------------------------------------------------------------------
# planted mistakes
# ---------------------------------------------------------------------------

MUTATIONS = {
    "omega_cross_order": ("torch.cross(w.expand_as(x), x, dim=1)", "torch.cross(x, w.expand_as(x), dim=1)"),
    "pose_transposed": ("x = taxels @ R.T + pose[0:3]", "x = taxels @ R + pose[0:3]"),
    "output_not_rotated_back": ("fn_pad = fn_all @ R  ", "fn_pad = fn_all @ R.T  "),
    "fd_step": ("e[a] = 0.5", "e[a] = 1.0"),
    "normal_edge_central": ("first = (sl(1, 2) - sl(0, 1)) / pitch", "first = (sl(1, 2) - sl(0, 1)) / (2 * pitch)"),
    "damping_sign": ("mraw = (-kn + kd * ddot) * ph", "mraw = (-kn - kd * ddot) * ph"),
    "friction_cap_max": ("torch.where(cap.detach() < lim.detach(), cap, lim)",
                         "torch.where(cap.detach() > lim.detach(), cap, lim)"),
    "intensity_unclamped": ("return torch.clamp(I, 0.0, 255.0).permute(1, 2, 0)", "return I.permute(1, 2, 0)"),
    "render_implicit_sign": ("dz = -phi / torch.where(", "dz = phi / torch.where("),
    "render_pose_transposed": ("x = pts @ R.T + pose[0:3]", "x = pts @ R + pose[0:3]"),
    "render_pixel_axes": ("torch.stack([torch.tensor(xx[hit], dtype=F64), torch.tensor(yy[hit], dtype=F64), z]",
                          "torch.stack([torch.tensor(yy[hit], dtype=F64), torch.tensor(xx[hit], dtype=F64), z]"),
    "render_grazing_kept": ("keep = inside & (phi_z.abs() >= GRAZING)", "keep = inside & (phi_z.abs() >= 0.0)"),
    "mse_target_sign": ("err = (shade_intensity(A[s], D, px, py) - T[b]) ** 2",
                        "err = (shade_intensity(A[s], D, px, py) + T[b]) ** 2"),
    "mse_map_sensor": ("loss_map[s] += err.detach().sum(dim=2).numpy()", "loss_map[0] += err.detach().sum(dim=2).numpy()"),
    "monomial_swap": ("m = torch.stack([torch.ones_like(nx), nx, ny, nx * nx, ny * ny, nx * ny])",
                      "m = torch.stack([torch.ones_like(nx), ny, nx, nx * nx, ny * ny, nx * ny])"),
}


def _load_variant(src, tmp_path, name):
    f = tmp_path / f"grad_{name}.py"
    f.write_text(src)
    spec = importlib.util.spec_from_file_location(f"grad_{name}", str(f))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_mutation_site_exists():
    src = open(G0.__file__).read()
    for name, (old, _) in MUTATIONS.items():
        assert src.count(old) == 1, name


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(orc, name, tmp_path):
    old, new = MUTATIONS[name]
    mod = _load_variant(open(G0.__file__).read().replace(old, new), tmp_path, name)
    caught = False
    for check in CHECKS:
        try:
            check(mod)
        except AssertionError:
            caught = True
            break
    assert caught, f"mutation {name} survived the gradient-oracle pins"
