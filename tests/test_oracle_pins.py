"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against a closed form, an invariant, a brute-force
construction or an independent library routine, chosen so that a dropped term,
a wrong sign or index, or a transposed operand in the oracle fails at least one.

Passages: Sec. III-C (SDF query, finite-difference normal, chain-rule d', penalty
normal force with d-scaled damping, friction-capped shear), Eq. 3 (unilateral
contact force), Sec. III-B (depth map -> RGB through a calibrated per-pixel map).
"""
import math

import numpy as np
import pytest

from paper_2408_06506_b300 import synth


# ---------------------------------------------------------------------------
# helpers (test-side closed forms only)
# ---------------------------------------------------------------------------

def _multilinear_grid(n, h, origin, coef):
    """Grid of a + b x + c y + d z + e xy + f yz + g zx + k xyz (all values exact in f32)."""
    a, b, c, d, e, f, g, k = coef
    return synth.bake_field(lambda x, y, z: a + b * x + c * y + d * z + e * x * y + f * y * z + g * z * x
                            + k * x * y * z, n, h, origin)


def _multilinear_value_grad(x, coef):
    a, b, c, d, e, f, g, k = coef
    X, Y, Z = x
    val = a + b * X + c * Y + d * Z + e * X * Y + f * Y * Z + g * Z * X + k * X * Y * Z
    grad = np.array([b + e * Y + g * Z + k * Y * Z, c + e * X + f * Z + k * X * Z,
                     d + f * Y + g * X + k * X * Y])
    return val, grad


def _pose(t, q):
    return np.concatenate([np.asarray(t, np.float64), np.asarray(q, np.float64)]).astype(np.float32)


def _run_forces(orc, grid, taxels, pose, twist, kn=1e4, kd=0.0, kt=1e2, mu=0.5):
    pose = np.asarray(pose, np.float32).reshape(1, 1, 7)
    twist = np.asarray(twist, np.float32).reshape(1, 1, 6)
    return orc.penalty_forces([grid], taxels, [0], pose, twist, [kn], [kd], [kt], [mu])


def _plane_grid(normal, n=40, h=0.5e-3):
    """Half-space n.x < 0 baked on a grid centred at the origin (linear field)."""
    nrm = np.asarray(normal, np.float64)
    nrm = nrm / np.linalg.norm(nrm)
    shape = synth.Shape("plane", (nrm[0], nrm[1], nrm[2], 0.0))
    return synth.bake(shape, n, h), nrm


def _pad_facing_plane(nrm, delta, q_spin, offset=(0.0, 0.0, 0.0)):
    """Pose whose +z axis is -nrm (facing the half-space) and whose plane cuts delta into it."""
    ez = np.array([0.0, 0.0, 1.0])
    target = -nrm
    axis = np.cross(ez, target)
    s = np.linalg.norm(axis)
    if s < 1e-12:
        q_align = np.array([1.0, 0, 0, 0]) if target[2] > 0 else np.array([0.0, 1.0, 0, 0])
    else:
        q_align = synth.quat_from_axis_angle(axis, math.atan2(s, ez @ target))
    q = synth.quat_multiply(q_align, q_spin)
    R = synth.quat_to_matrix(q)
    t = -delta * nrm + np.asarray(offset)
    return _pose(t, q), R


# ---------------------------------------------------------------------------
# SDF interpolation and gradient (Sec. III-C reading: trilinear + central FD, step h/2)
# ---------------------------------------------------------------------------

def test_trilinear_exact_on_multilinear_fields(orc):
    """Trilinear interpolation reproduces any multilinear polynomial exactly."""
    g = np.random.default_rng(11)
    coef = g.integers(-8, 9, size=8).astype(np.float64)
    grid = _multilinear_grid((6, 7, 5), 1.0, (-2.0, -3.0, -1.0), coef)
    for _ in range(200):
        u = g.uniform(0, [5, 6, 4])
        x = np.asarray(grid.origin, np.float64) + u
        got = orc.trilinear(grid, u)
        want, _ = _multilinear_value_grad(x, coef)
        assert got == pytest.approx(want, abs=1e-11)


def test_fd_gradient_exact_on_multilinear_fields(orc):
    """A central difference is exact for a field that is linear along the axis."""
    g = np.random.default_rng(12)
    coef = g.integers(-8, 9, size=8).astype(np.float64)
    h = 0.5
    grid = _multilinear_grid((9, 8, 7), h, (-2.0, -1.5, -1.0), coef)
    for _ in range(200):
        u = g.uniform(0.5, [7.5, 6.5, 5.5])
        x = np.asarray(grid.origin, np.float64) + u * h
        phi, grad, inside = orc.sdf_eval(grid, x)
        assert inside
        want_v, want_g = _multilinear_value_grad(x, coef)
        assert phi == pytest.approx(want_v, abs=1e-10)
        np.testing.assert_allclose(grad, want_g, atol=1e-10)


def test_trilinear_brute_force_2x2x2(orc):
    """On one cell, the interpolant is the unique multilinear function through the 8
    corner values: fit it by solving the 8x8 system and compare anywhere in the cell."""
    g = np.random.default_rng(13)
    for _ in range(20):
        vals = g.standard_normal((2, 2, 2)).astype(np.float32)          # [z][y][x]
        grid = synth.Grid(vals, np.zeros(3, np.float32), 1.0)
        rows, rhs = [], []
        for z in (0, 1):
            for y in (0, 1):
                for x in (0, 1):
                    rows.append([1, x, y, z, x * y, y * z, z * x, x * y * z])
                    rhs.append(float(vals[z, y, x]))
        coef = np.linalg.solve(np.array(rows, float), np.array(rhs))
        for _ in range(10):
            u = g.uniform(0, 1, size=3)
            want, _ = _multilinear_value_grad(u, coef)
            assert orc.trilinear(grid, u) == pytest.approx(want, abs=1e-12)


def test_gradient_at_nodes_is_grid_central_difference(orc):
    """At a node, the h/2 difference of the interpolant equals (g[i+1]-g[i-1]) / 2h."""
    g = np.random.default_rng(14)
    data = g.standard_normal((6, 7, 8)).astype(np.float32)
    h = 0.25
    grid = synth.Grid(data, np.array([0.1, -0.2, 0.3], np.float32), h)
    for (i, j, k) in [(1, 1, 1), (3, 2, 4), (6, 5, 4), (2, 4, 3)]:
        x = np.asarray(grid.origin, np.float64) + np.array([i, j, k]) * h
        phi, grad, inside = orc.sdf_eval(grid, x)
        assert inside
        assert phi == pytest.approx(float(data[k, j, i]), abs=1e-12)
        want = [(float(data[k, j, i + 1]) - float(data[k, j, i - 1])) / (2 * h),
                (float(data[k, j + 1, i]) - float(data[k, j - 1, i])) / (2 * h),
                (float(data[k + 1, j, i]) - float(data[k - 1, j, i])) / (2 * h)]
        np.testing.assert_allclose(grad, want, atol=1e-12)


def test_domain_rule(orc):
    """In domain iff 0.5 <= u <= n - 1.5 on every axis; outside: +inf and a zero gradient."""
    data = np.zeros((6, 5, 4), np.float32)
    grid = synth.Grid(data, np.zeros(3, np.float32), 1.0)
    for u, inside in [((0.5, 0.5, 0.5), True), ((2.5, 3.5, 4.5), True), ((0.49, 1, 1), False),
                      ((2.51, 1, 1), False), ((1, 3.51, 1), False), ((1, 1, 4.51), False),
                      ((1, 1, -1), False)]:
        phi, grad, ins = orc.sdf_eval(grid, np.array(u, float))
        assert ins == inside
        if not inside:
            assert phi == math.inf and not grad.any()


def test_batched_query_bad_id_and_thread_independence(orc):
    sc = synth.scene_sphere_pad(seed=3, with_images=False)
    g = np.random.default_rng(15)
    pts = g.uniform(-8e-3, 8e-3, size=(5000, 3)).astype(np.float32)
    ids = np.zeros(5000, np.int32)
    ids[7] = 3
    ids[9] = -1
    phi1, gr1, bad1 = orc.sdf_query(sc.grids, pts, ids, nthreads=1)
    phi4, gr4, bad4 = orc.sdf_query(sc.grids, pts, ids, nthreads=4)
    assert bad1 == bad4 == 2
    assert np.isnan(phi1[7]) and np.isnan(gr1[9]).all()
    np.testing.assert_array_equal(np.nan_to_num(phi1), np.nan_to_num(phi4))
    np.testing.assert_array_equal(np.nan_to_num(gr1), np.nan_to_num(gr4))


# ---------------------------------------------------------------------------
# Force field (Sec. III-C, Eq. 3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plane_indentation_closed_form(orc, seed):
    """A flat pad pressed delta into a half-space: every in-domain taxel reads depth delta,
    f_n = k_n delta along the plane normal, i.e. -k_n delta e_z in the pad frame; no shear at
    rest; F = T_in * f, tau = (sum of in-domain p_i) x f."""
    g = np.random.default_rng(100 + seed)
    nrm = g.standard_normal(3)
    grid, nrm = _plane_grid(nrm)
    spin = synth.quat_from_axis_angle([0, 0, 1], g.uniform(0, 2 * math.pi))
    delta = g.uniform(1e-4, 1e-3)
    kn = 1e4
    taxels = synth.taxel_grid(6, 7, 1e-3)
    pose, R = _pad_facing_plane(nrm, delta, spin)
    r = _run_forces(orc, grid, taxels, pose, np.zeros(6), kn=kn)
    dep, fn, ft, wr = r["depth"][0, 0], r["f_n"][0, 0], r["f_t"][0, 0], r["wrench"][0, 0]
    inside = dep > 0
    assert inside.all()   # the 5x6 mm pad stays inside the 20 mm grid
    np.testing.assert_allclose(dep, delta, atol=2e-9)
    np.testing.assert_allclose(fn, np.tile([0, 0, -kn * delta], (taxels.shape[0], 1)), atol=kn * 2e-9)
    assert not ft.any()
    np.testing.assert_allclose(wr[:3], [0, 0, -kn * delta * taxels.shape[0]], atol=1e-5)
    np.testing.assert_allclose(wr[3:], np.cross(taxels.astype(np.float64).sum(0), [0, 0, -kn * delta]), atol=1e-7)


def test_plane_offset_pad_torque(orc):
    """Same as above with the pad shifted so the wrench has a lever arm: tau = sum p_i x f."""
    grid, nrm = _plane_grid([0, 0, 1.0], n=40, h=0.5e-3)
    taxels = synth.taxel_grid(3, 4, 1e-3)
    # pad rotated 90 degrees about its normal; taxel plane 0.4 mm inside
    pose, R = _pad_facing_plane(nrm, 4e-4, synth.quat_from_axis_angle([0, 0, 1], math.pi / 2))
    r = _run_forces(orc, grid, taxels, pose, np.zeros(6), kn=2e4)
    f = np.array([0, 0, -2e4 * 4e-4])
    want_tau = sum(np.cross(p.astype(np.float64), f) for p in taxels)
    np.testing.assert_allclose(r["wrench"][0, 0, 3:], want_tau, atol=1e-9)
    # move the whole pad sideways: taxel positions in the pad frame do not change, so neither does tau
    pose2, _ = _pad_facing_plane(nrm, 4e-4, synth.quat_from_axis_angle([0, 0, 1], math.pi / 2), (2e-3, -1e-3, 0))
    r2 = _run_forces(orc, grid, taxels, pose2, np.zeros(6), kn=2e4)
    np.testing.assert_allclose(r2["wrench"], r["wrench"], atol=1e-9)


def test_out_of_contact_is_exact_zero(orc):
    grid, nrm = _plane_grid([0.3, -0.2, 1.0])
    taxels = synth.taxel_grid(5, 5, 1e-3)
    pose, _ = _pad_facing_plane(nrm, -1e-3, np.array([1.0, 0, 0, 0]))
    r = _run_forces(orc, grid, taxels, pose, [0.01, -0.02, 0.03, 0.5, 0.1, -0.2])
    for k in ("depth", "f_n", "f_t", "wrench"):
        assert not np.any(r[k]), k


def test_sphere_indentation_within_interpolation_bound(orc):
    """Sphere R indenting a flat pad by delta: exact depth at a taxel is R - |p - c| (when
    positive); trilinear interpolation of a smooth field errs by at most
    (h^2/8) sum_k |d2phi/dx_k^2| = (h^2/8)(2/r), about 3 um at h = 0.25 mm, r ~ 5 mm."""
    sc = synth.scene_sphere_pad(seed=4, E=6, with_images=False)
    r = orc.penalty_forces(sc.grids, sc.taxels, sc.obj_id, sc.pad_pose, sc.pad_twist,
                           sc.k_n, sc.k_d, sc.k_t, sc.mu)
    R, h = 5e-3, float(sc.grids[0].voxel)
    for e in range(sc.E):
        pose = sc.pad_pose[e, 0].astype(np.float64)
        # R(q) = I here, the sphere centre is at the object origin
        xo = sc.taxels.astype(np.float64) + pose[:3]
        dist = np.linalg.norm(xo, axis=1)
        exact = np.maximum(0.0, R - dist)
        bound = h * h / 8 * 2 / (R - 1.2e-3) + 1e-8
        got = r["depth"][e, 0]
        close = np.abs(exact) > bound
        np.testing.assert_array_less(np.abs(got - exact), bound + 1e-12)
        # the contact normal points radially out of the sphere: f_n || (p - c)
        fn = r["f_n"][e, 0]
        for i in np.nonzero(close & (exact > 0))[0]:
            nvec = fn[i] / np.linalg.norm(fn[i])
            assert nvec @ (xo[i] / dist[i]) > 0.999
            assert np.linalg.norm(fn[i]) == pytest.approx(sc.k_n[0] * got[i], rel=1e-12)


def test_normal_damping_closed_form(orc):
    """f_n = max((-k_n + k_d d') d, 0) n with d' = n . x' (chain rule): approaching adds
    force; a fast enough separation clamps it to zero (unilateral, Eq. 3)."""
    grid, nrm = _plane_grid([0, 0, 1.0])
    taxels = synth.taxel_grid(2, 2, 1e-3)
    delta, kn, kd = 5e-4, 1e4, 3e5
    pose, R = _pad_facing_plane(nrm, delta, np.array([1.0, 0, 0, 0]))
    for vn in (-0.02, 0.0, 0.01, 0.05):
        # pad moving along +z of the object frame (toward the free side of the plane) at vn
        r = _run_forces(orc, grid, taxels, pose, [0, 0, vn, 0, 0, 0], kn=kn, kd=kd)
        ddot = vn                     # n = +z in the object frame
        mag = max((-kn + kd * ddot) * (-delta), 0.0)
        want = R.T @ (mag * nrm)
        np.testing.assert_allclose(r["f_n"][0, 0], np.tile(want, (4, 1)), atol=1e-9 + 1e-7 * mag)
    assert not np.any(_run_forces(orc, grid, taxels, pose, [0, 0, 0.05, 0, 0, 0], kn=kn, kd=kd)["f_n"])


@pytest.mark.parametrize("speed", [0.001, 0.2])
def test_shear_opposes_sliding_stick_and_slip(orc, speed):
    """Pad sliding along the plane: f_t = -v_t/|v_t| min(k_t |v_t|, mu |f_n|), i.e. opposite
    to the relative tangential motion (the edge-test directionality) with the stick value
    k_t|v| at low speed and the slip cap mu k_n delta at high speed."""
    grid, nrm = _plane_grid([0, 0, 1.0])
    taxels = synth.taxel_grid(3, 3, 1e-3)
    delta, kn, kt, mu = 3e-4, 1e4, 1e2, 0.5
    pose, R = _pad_facing_plane(nrm, delta, synth.quat_from_axis_angle([0, 0, 1], 0.3))
    vdir = np.array([0.6, -0.8, 0.0])
    r = _run_forces(orc, grid, taxels, pose, np.concatenate([speed * vdir, [0, 0, 0]]), kn=kn, kt=kt, mu=mu)
    mag = min(kt * speed, mu * kn * delta)
    want = R.T @ (-mag * vdir)
    np.testing.assert_allclose(r["f_t"][0, 0], np.tile(want, (9, 1)), atol=1e-9)


def test_pure_normal_velocity_gives_no_shear(orc):
    grid, nrm = _plane_grid([0, 0, 1.0])
    taxels = synth.taxel_grid(3, 3, 1e-3)
    pose, R = _pad_facing_plane(nrm, 3e-4, np.array([1.0, 0, 0, 0]))
    r = _run_forces(orc, grid, taxels, pose, [0, 0, -0.03, 0, 0, 0])
    assert np.abs(r["f_t"]).max() < 1e-12


def test_spin_about_pad_normal_torque(orc):
    """Pad spinning at w about its own normal (twist about the object origin: v = -w x t).
    Each taxel slides at w x (R p); in the stick regime f_t = -k_t w x (R p), so the torque
    about the pad normal is -k_t w sum |p_i|^2 and the net shear force vanishes."""
    grid, nrm = _plane_grid([0, 0, 1.0], n=60, h=0.5e-3)
    taxels = synth.taxel_grid(4, 5, 1e-3)
    delta, kn, kt, mu = 5e-4, 1e4, 1e2, 0.5
    pose, R = _pad_facing_plane(nrm, delta, np.array([1.0, 0, 0, 0]), offset=(1e-3, 2e-3, 0))
    wz = 0.5
    w = R @ np.array([0, 0, wz])
    t = pose[:3].astype(np.float64)
    v = -np.cross(w, t)
    r = _run_forces(orc, grid, taxels, pose, np.concatenate([v, w]), kn=kn, kt=kt, mu=mu)
    p2 = (taxels.astype(np.float64) ** 2).sum()
    wr = r["wrench"][0, 0]
    np.testing.assert_allclose(wr[0:2], 0.0, atol=1e-7)
    assert wr[5] == pytest.approx(-kt * wz * p2, rel=1e-6)
    np.testing.assert_allclose(wr[3:5], 0.0, atol=1e-9)   # f_n uniform on a centred grid
    assert wr[2] == pytest.approx(-kn * delta * taxels.shape[0], rel=1e-6)


def test_friction_invariants_random(orc):
    """On random poses/twists against boxes, cylinders and hex prisms:
    |f_t| <= mu |f_n|; f_t . f_n = 0 (shear is tangential); zero where depth is zero."""
    sc = synth.scene_objects(seed=5, E=24, P=2, n=48, depth_maps="none")
    sc.pad_twist[..., 3:] = np.random.default_rng(16).normal(0, 2.0, size=sc.pad_twist[..., 3:].shape)
    r = orc.penalty_forces(sc.grids, sc.taxels, sc.obj_id, sc.pad_pose, sc.pad_twist,
                           sc.k_n, sc.k_d, sc.k_t, sc.mu)
    fn, ft, dep = r["f_n"], r["f_t"], r["depth"]
    mu = sc.mu[:, None, None]
    nfn = np.linalg.norm(fn, axis=-1)
    nft = np.linalg.norm(ft, axis=-1)
    assert (dep > 0).sum() > 100
    assert np.all(nft <= mu * nfn * (1 + 1e-12) + 1e-15)
    assert np.all(np.abs((fn * ft).sum(-1)) <= 1e-9 * (nfn * nft + 1e-30) + 1e-18)
    assert not fn[dep == 0].any() and not ft[dep == 0].any()


def test_quaternion_scale_invariance(orc):
    sc = synth.scene_objects(seed=6, E=4, P=2, n=48, depth_maps="none")
    a = orc.penalty_forces(sc.grids, sc.taxels, sc.obj_id, sc.pad_pose, sc.pad_twist,
                           sc.k_n, sc.k_d, sc.k_t, sc.mu)
    # scaling by 4 is exact in float32 and sqrt(4 s) = 2 sqrt(s) exactly: bitwise equal
    pose = sc.pad_pose.copy()
    pose[..., 3:] *= 4.0
    b = orc.penalty_forces(sc.grids, sc.taxels, sc.obj_id, pose, sc.pad_twist,
                           sc.k_n, sc.k_d, sc.k_t, sc.mu)
    for k in ("depth", "f_n", "f_t", "wrench"):
        np.testing.assert_array_equal(a[k], b[k])
    # scaling by 2.5 rounds the stored components: equal up to that float32 rounding
    pose[..., 3:] = sc.pad_pose[..., 3:] * np.float32(2.5)
    c = orc.penalty_forces(sc.grids, sc.taxels, sc.obj_id, pose, sc.pad_twist,
                           sc.k_n, sc.k_d, sc.k_t, sc.mu)
    for k in ("f_n", "f_t"):
        err = np.linalg.norm(c[k] - a[k], axis=-1)
        ref = np.linalg.norm(a[k], axis=-1)
        assert np.all(err <= 1e-4 * ref + 1e-5 * ref.max(axis=-1, keepdims=True) + 1e-12)


def test_rigid_motion_invariance(orc):
    """Moving the pad and the half-space together leaves the pad-frame outputs unchanged:
    a plane of normal n1 indented by delta gives the same field as one of normal n2."""
    taxels = synth.taxel_grid(4, 4, 1e-3)
    outs = []
    for nrm in ([0, 0, 1.0], [1.0, 2.0, -0.5], [-0.3, 0.1, -1.0]):
        grid, nv = _plane_grid(nrm)
        pose, R = _pad_facing_plane(nv, 6e-4, synth.quat_from_axis_angle([0, 0, 1], 0.7))
        # tangential sliding along pad x, expressed in the object frame
        v = R @ np.array([0.01, 0.0, 0.0])
        outs.append(_run_forces(orc, grid, taxels, pose, np.concatenate([v, [0, 0, 0]])))
    for o in outs[1:]:
        for k in ("depth", "f_n", "f_t", "wrench"):
            np.testing.assert_allclose(o[k], outs[0][k], atol=1e-6 * max(1.0, np.abs(outs[0][k]).max()))


def test_broadcast_params_equal_per_env(orc):
    sc = synth.scene_objects(seed=7, E=5, P=2, n=48, depth_maps="none")
    a = orc.penalty_forces(sc.grids, sc.taxels, sc.obj_id, sc.pad_pose, sc.pad_twist,
                           [2e4], [10.0], [80.0], [0.4])
    b = orc.penalty_forces(sc.grids, sc.taxels, sc.obj_id, sc.pad_pose, sc.pad_twist,
                           [2e4] * 5, [10.0] * 5, [80.0] * 5, [0.4] * 5)
    for k in ("depth", "f_n", "f_t", "wrench"):
        np.testing.assert_array_equal(a[k], b[k])


def test_bad_obj_id_gives_nan(orc):
    sc = synth.scene_objects(seed=8, E=3, P=2, n=48, depth_maps="none")
    ids = sc.obj_id.copy()
    ids[1] = 99
    r = orc.penalty_forces(sc.grids, sc.taxels, ids, sc.pad_pose, sc.pad_twist,
                           sc.k_n, sc.k_d, sc.k_t, sc.mu)
    assert r["bad"] == 2            # both pads of env 1
    assert np.isnan(r["f_n"][1]).all() and np.isnan(r["wrench"][1]).all()
    assert not np.isnan(r["f_n"][0]).any()


def test_standalone_wrench_matches_hand_sum(orc):
    """One taxel carries a force: the wrench is (f, p x f) exactly; others contribute zero."""
    taxels = synth.taxel_grid(3, 3, 2e-3)
    fn = np.zeros((2, 9, 3), np.float32)
    ft = np.zeros((2, 9, 3), np.float32)
    fn[0, 5] = [0.5, -1.0, 3.0]
    ft[0, 5] = [0.25, 0.25, 0.0]
    fn[1, 0] = [0.0, 0.0, -2.0]
    w = orc.pad_wrench(taxels, fn, ft)
    f = np.array([0.75, -0.75, 3.0])
    np.testing.assert_allclose(w[0], np.concatenate([f, np.cross(taxels[5].astype(float), f)]), atol=1e-15)
    np.testing.assert_allclose(w[1], np.concatenate([[0, 0, -2.0], np.cross(taxels[0].astype(float), [0, 0, -2.0])]),
                               atol=1e-15)


# ---------------------------------------------------------------------------
# Tactile image (Sec. III-B)
# ---------------------------------------------------------------------------

def test_normals_match_numpy_gradient(orc):
    """Depth-map gradient = numpy.gradient with edge_order=1 (central inside, one-sided at
    the borders); n = (D_x, D_y, -1) / sqrt(1 + D_x^2 + D_y^2)."""
    g = np.random.default_rng(20)
    H, W, sx, sy = 13, 17, 1e-4, 1.5e-4
    D = (0.02 + 1e-4 * g.standard_normal((H, W))).astype(np.float32)
    n = orc.depth_normals(D, sx, sy)
    dy, dx = np.gradient(D.astype(np.float64), float(np.float32(sy)), float(np.float32(sx)), edge_order=1)
    norm = np.sqrt(1 + dx ** 2 + dy ** 2)
    want = np.stack([dx / norm, dy / norm, -1 / norm], -1)
    np.testing.assert_allclose(n, want, atol=1e-12)


def test_flat_depth_shades_to_background(orc):
    coeffs = synth.shading_coeffs(2, 9, 12, seed=5)
    D = np.full((3, 9, 12), synth.D0, np.float32)
    rgb, bad = orc.shade(coeffs, 1e-4, 1e-4, [1, 0, 1], D)
    assert bad == 0
    for b, s in enumerate([1, 0, 1]):
        want = np.floor(np.clip(coeffs[s, 0].astype(np.float64), 0, 255) + 0.5).astype(np.uint8)
        np.testing.assert_array_equal(rgb[b], np.moveaxis(want, 0, -1))


def test_tilted_plane_shades_to_known_quadratic(orc):
    """D = D0 + a x + b y has the same normal at every pixel, borders included, so the
    image is A0 + A1 n_x + A2 n_y + A3 n_x^2 + A4 n_y^2 + A5 n_x n_y per pixel."""
    H, W, sx, sy = 10, 14, 2e-4, 1e-4
    a, b = 0.3, -0.45
    xs = np.arange(W) * sx
    ys = np.arange(H) * sy
    D = (synth.D0 + a * xs[None, :] + b * ys[:, None]).astype(np.float32)
    # the slopes the float32 map actually carries along each row/column
    coeffs = synth.shading_coeffs(1, H, W, seed=9).astype(np.float64)
    rgb, inten, bad = orc.shade(coeffs.astype(np.float32), sx, sy, [0], D[None], with_intensity=True)
    nx_, ny_ = a / math.sqrt(1 + a * a + b * b), b / math.sqrt(1 + a * a + b * b)
    m = np.array([1, nx_, ny_, nx_ * nx_, ny_ * ny_, nx_ * ny_])
    want = np.einsum("k,kchw->hwc", m, coeffs[0].astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(inten[0], want, atol=2e-3)   # f32 storage of D limits the slope to ~1e-5


@pytest.mark.parametrize("v,q", [(0.5, 1), (0.49999, 0), (254.5, 255), (254.49, 254), (-3.0, 0),
                                 (300.0, 255), (255.0, 255), (0.0, 0), (127.5, 128), (float("nan"), 0)])
def test_quantisation_hand_values(orc, v, q):
    assert orc.quantize(v) == q


def test_quantisation_through_shading(orc):
    """Background coefficients set to the hand values flow through unchanged to the bytes."""
    vals = np.array([0.5, 254.5, -3.0, 300.0, 12.25, 99.75], np.float32)
    coeffs = np.zeros((1, 6, 3, 1, 8), np.float32)
    coeffs[0, 0, :, 0, :6] = vals
    D = np.full((1, 1, 8), synth.D0, np.float32)
    rgb, _ = orc.shade(coeffs, 1e-4, 1e-4, [0], D)
    np.testing.assert_array_equal(rgb[0, 0, :6, 0], [1, 255, 0, 255, 12, 100])


def test_bad_sensor_id_leaves_image_untouched(orc):
    coeffs = synth.shading_coeffs(1, 4, 8, seed=1)
    D = np.full((2, 4, 8), synth.D0, np.float32)
    init = np.full((2, 4, 8, 3), 7, np.uint8)
    rgb, bad = orc.shade(coeffs, 1e-4, 1e-4, [0, 5], D, rgb_init=init)
    assert bad == 1
    assert (rgb[1] == 7).all() and not (rgb[0] == 7).all()


def test_single_row_and_column_maps(orc):
    """An axis of length 1 has no derivative (n_y = 0 for H = 1)."""
    # 2^-6 + k 2^-17 at pitch 2^-14 is exact in float32: slope 1/8 everywhere
    D = (2.0 ** -6 + np.arange(8) * 2.0 ** -17).astype(np.float32)[None, :]
    n = orc.depth_normals(D, 2.0 ** -14, 1e-4)
    assert not n[..., 1].any()
    np.testing.assert_allclose(n[0, :, 0], 0.125 / math.sqrt(1 + 0.125 ** 2), rtol=1e-15)


# ---------------------------------------------------------------------------
# Depth rendering (Sec. III-B: the in-sensor camera sees the indenting object)
# ---------------------------------------------------------------------------

def _render(orc, grid, pose, H=9, W=11, pitch=0.5e-3, d0=0.02, z_max=3e-3):
    x0, y0 = -(W - 1) / 2 * pitch, -(H - 1) / 2 * pitch
    D, bad = orc.render_depth([grid], [0], np.asarray(pose, np.float32).reshape(1, 1, 7), H, W, pitch, pitch,
                              x0, y0, d0, z_max)
    xs = x0 + np.arange(W) * pitch
    ys = y0 + np.arange(H) * pitch
    return D[0, 0], xs, ys, bad


def test_render_parallel_plane_closed_form(orc):
    """A half-space cut delta into the pad: every column meets it at z = -delta."""
    grid, nrm = _plane_grid([0.2, -0.3, 1.0], n=48, h=0.5e-3)
    pose, R = _pad_facing_plane(nrm, 4e-4, synth.quat_from_axis_angle([0, 0, 1], 0.4))
    D, xs, ys, bad = _render(orc, grid, pose)
    assert bad == 0
    # the march resolves z_hit to its bisection width voxel * 2^-16 (upper end of the bracket)
    np.testing.assert_allclose(D, 0.02 - 4e-4, atol=grid.voxel / 65536 + 2e-9)


def test_render_tilted_plane_closed_form(orc):
    """A half-space tilted against the pad: phi along a column is phi(0) + z (n . d), so
    the first point inside is z = -phi(0) / (n . d); this also pins the pixel order."""
    grid, nrm = _plane_grid([0.0, 0.0, 1.0], n=64, h=0.5e-3)
    q = synth.quat_multiply([0.0, 1.0, 0.0, 0.0], synth.quat_from_axis_angle([1.0, 0.5, 0.0], 0.3))
    R = synth.quat_to_matrix(q)
    pose = _pose(-3e-4 * np.array([0, 0, 1.0]) @ np.eye(3), q)    # pad origin 0.3 mm inside the plane
    D, xs, ys, bad = _render(orc, grid, pose)
    d = R[:, 2]
    assert nrm @ d < 0
    for j, y in enumerate(ys):
        for i, x in enumerate(xs):
            p0 = R @ np.array([x, y, 0.0]) + pose[:3].astype(np.float64)
            zh = -(nrm @ p0) / (nrm @ d)
            want = 0.02 - max(0.0, -zh) if zh >= -3e-3 else 0.02 - 3e-3
            assert D[j, i] == pytest.approx(want, abs=grid.voxel / 65536 + 3e-9)
    assert np.ptp(D[:, 0]) > 1e-5 and np.ptp(D[0, :]) > 1e-5    # varies along both image axes


def test_render_sphere_within_interpolation_bound(orc):
    """Sphere R indenting by delta: the column at radius r meets it at c - sqrt(R^2 - r^2)
    (pad frame); away from near-tangent columns the interpolation error h^2/(4 rho),
    divided by the column's |d phi/dz| >= 0.3, bounds the difference."""
    Rs, delta, h = 5e-3, 8e-4, 0.25e-3
    grid = synth.bake(synth.Shape("sphere", (Rs,)), 64, h)
    pose = synth.place_pad(synth.Shape("sphere", (Rs,)), np.array([1.0, 0, 0, 0]), delta, (0.4e-3, -0.7e-3))
    D, xs, ys, bad = _render(orc, grid, pose, H=21, W=25, pitch=0.2e-3)
    c = -pose[:3].astype(np.float64)          # sphere centre in the pad frame (R = I)
    bound = h * h / 8 * 2 / (Rs - 1e-3) / 0.3 + 1e-8
    checked = 0
    for j, y in enumerate(ys):
        for i, x in enumerate(xs):
            r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2
            if r2 >= Rs * Rs:
                continue
            zh = c[2] - np.sqrt(Rs * Rs - r2)
            if (c[2] - zh) / Rs < 0.3 or zh > -1e-6:
                continue
            assert abs(D[j, i] - (0.02 + zh)) <= bound
            checked += 1
    assert checked > 50
    assert D.min() == pytest.approx(0.02 - delta, abs=bound)


def test_render_miss_is_exactly_d0_and_deep_object_clamps(orc):
    grid, nrm = _plane_grid([0.0, 0.0, 1.0], n=48, h=0.5e-3)
    pose, R = _pad_facing_plane(nrm, -5e-4, np.array([1.0, 0, 0, 0]))     # 0.5 mm gap
    D, *_ = _render(orc, grid, pose)
    assert (D == np.float64(np.float32(0.02))).all()
    pose, R = _pad_facing_plane(nrm, 5e-3, np.array([1.0, 0, 0, 0]))      # 5 mm deep > z_max
    D, *_ = _render(orc, grid, pose, z_max=3e-3)
    np.testing.assert_allclose(D, np.float64(np.float32(0.02)) - np.float64(np.float32(3e-3)), atol=1e-12)
