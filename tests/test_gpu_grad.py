"""GPU parity of the adjoint kernels (include/tacsl_grad.h) against the FP64 gradient
oracle (torch autograd of the same definitions) and against float64 central
differences of the C oracle (h = 1e-6), to rel 1e-3, away from kinks; and of the
torch.autograd bindings against the direct calls."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from oracle import grad as G
import paper_2408_06506_b300 as tacsl
from paper_2408_06506_b300 import autograd as ta
from paper_2408_06506_b300 import synth

from gpu_common import dev
from grad_common import calibration_scene, safe_taxels, upstream

pytestmark = pytest.mark.gpu
RTOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_06506_b300 import build
    build.build()
    tacsl.load()
    tacsl.check_errors(clear=True)


def _adjoint(sc, gs, params_count_one=False):
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    prm = [sc.k_n, sc.k_d, sc.k_t, sc.mu]
    if params_count_one:
        prm = [np.array([v[0]], np.float32) for v in prm]
    params = tacsl.ContactParams(*[dev(v) for v in prm])
    E, P, T = sc.E, sc.P, sc.T
    gp = torch.empty(E, P, 7, device="cuda")
    gt = torch.empty(E, P, 6, device="cuda")
    gk = torch.empty(len(prm[0]), 4, device="cuda")
    lib = ta._lib()
    d = [dev(g) for g in gs]
    # device inputs held in names for the duration of the call (their pointers are passed)
    taxels, obj, pose, twist = dev(sc.taxels), dev(sc.obj_id), dev(sc.pad_pose), dev(sc.pad_twist)
    rc = lib.tacsl_penalty_forces_adjoint(C.byref(sdfs.c), C.byref(params.c), E, P, T, tacsl._ptr(taxels),
                                          tacsl._ptr(obj), tacsl._ptr(pose), tacsl._ptr(twist),
                                          *[tacsl._ptr(x) for x in d], tacsl._ptr(gp), tacsl._ptr(gt),
                                          tacsl._ptr(gk), None)
    assert rc == 0, lib.tacsl_last_error().decode()
    torch.cuda.synchronize()
    assert tacsl.check_errors() == 0
    return gp.cpu().numpy(), gt.cpu().numpy(), gk.cpu().numpy()


def _close(got, ref, what, floor_frac=1e-2):
    """Per row (pad or env): |got - ref|_inf <= 1e-3 max(|ref|_inf, floor_frac * max over rows)."""
    got = np.asarray(got, np.float64).reshape(ref.shape[0], -1)
    ref = np.asarray(ref, np.float64).reshape(ref.shape[0], -1)
    scale = np.maximum(np.abs(ref).max(axis=1), floor_frac * np.abs(ref).max()) + 1e-30
    err = np.abs(got - ref).max(axis=1)
    assert (err <= RTOL * scale).all(), f"{what}: worst {np.max(err / scale):.2e} of scale (row {np.argmax(err / scale)})"


@pytest.mark.parametrize("count_one", [False, True])
def test_force_adjoint_matches_oracle_gradient(count_one):
    sc = calibration_scene()
    if count_one:
        for k in ("k_n", "k_d", "k_t", "mu"):
            setattr(sc, k, np.full(sc.E, getattr(sc, k)[0], np.float32))
    gs, mask = upstream(sc)
    assert mask.mean() > 0.9
    gp, gt, gk = _adjoint(sc, gs, params_count_one=count_one)
    prm = [sc.k_n, sc.k_d, sc.k_t, sc.mu] if not count_one else [np.array([getattr(sc, k)[0]], np.float32)
                                                                  for k in ("k_n", "k_d", "k_t", "mu")]
    ref = G.force_gradients(sc.grids, sc.taxels, sc.obj_id, sc.pad_pose, sc.pad_twist, *prm, *gs)
    assert np.abs(ref["pose"]).max() > 0
    _close(gp.reshape(-1, 7), ref["pose"].reshape(-1, 7), "pose")
    _close(gt.reshape(-1, 6), ref["twist"].reshape(-1, 6), "twist")
    refk = np.stack([ref["k_n"], ref["k_d"], ref["k_t"], ref["mu"]], axis=1)
    for i, name in enumerate(("k_n", "k_d", "k_t", "mu")):
        _close(gk[:, i:i + 1], refk[:, i:i + 1], name)


def test_force_adjoint_matches_central_differences():
    """float64 central differences (h = 1e-6) of the C oracle's loss, for pads all of
    whose taxels are away from kinks."""
    sc = calibration_scene(seed=9, E=12)
    gs, mask = upstream(sc, seed=1)
    gp, gt, gk = _adjoint(sc, gs)
    clean = [(e, p) for e in range(sc.E) for p in range(sc.P) if mask[e, p].all() and gs[0][e, p].any()]
    assert len(clean) >= 2
    w = [np.asarray(g, np.float64) for g in gs]

    def loss(e, p, pose, twist, prm):
        r = oracle.penalty_forces(sc.grids, sc.taxels, sc.obj_id[e:e + 1], pose[None, None], twist[None, None], *prm)
        return (np.sum(w[0][e, p] * r["depth"][0, 0]) + np.sum(w[1][e, p] * r["f_n"][0, 0]) +
                np.sum(w[2][e, p] * r["f_t"][0, 0]) + np.sum(w[3][e, p] * r["wrench"][0, 0]))

    def fd(f, x, j, h=1e-6):
        xp, xm = x.copy(), x.copy()
        xp[j] = np.float32(x[j] + h)
        xm[j] = np.float32(x[j] - h)
        return (f(xp) - f(xm)) / (float(xp[j]) - float(xm[j]))

    for e, p in clean[:3]:
        prm = [np.array([v[e]], np.float32) for v in (sc.k_n, sc.k_d, sc.k_t, sc.mu)]
        pose, tw = sc.pad_pose[e, p].copy(), sc.pad_twist[e, p].copy()
        ref_pose = np.array([fd(lambda x: loss(e, p, x, tw, prm), pose, j) for j in range(7)])
        ref_tw = np.array([fd(lambda x: loss(e, p, pose, x, prm), tw, j) for j in range(6)])
        _close(gp[e, p][None], ref_pose[None], f"pose pad ({e},{p}) vs FD")
        _close(gt[e, p][None], ref_tw[None], f"twist pad ({e},{p}) vs FD")


def test_shade_intensity_and_adjoint_match_oracle():
    rng = np.random.default_rng(3)
    H, W, S, B = 24, 40, 2, 6
    px, py = 1.25e-4, 1e-4
    co = synth.shading_coeffs(S, H, W, 11)
    dm = np.full((B, H, W), synth.D0, np.float32)
    yy, xx = np.mgrid[0:H, 0:W]
    for b in range(B):                  # an indentation blob per image, plus flat gel around it
        cy, cx = rng.uniform(5, H - 5), rng.uniform(5, W - 5)
        dm[b] -= (4e-4 * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / 18.0)).astype(np.float32)
    sid = np.array([0, 1, 0, 1, 1, 0], np.int32)
    ref_fwd = G.shade_gradients(co, px, py, sid, dm, np.zeros((B, H, W, 3)))["intensity"]
    # upstream gradient, zero next to the clamp (I within 0.05 of 0 or 255)
    gI = rng.normal(size=(B, H, W, 3))
    gI[(ref_fwd < 0.05) | (ref_fwd > 254.95)] = 0.0
    gI = gI.astype(np.float32)
    ref = G.shade_gradients(co, px, py, sid, dm, gI)
    coeffs, depth = dev(co), dev(dm)
    sensor = dev(sid)
    inten = ta.shade_intensity(coeffs, depth, sensor, px, py)
    assert np.abs(inten.cpu().numpy() - ref_fwd).max() <= 2e-3
    c = coeffs.clone().requires_grad_(True)
    d = depth.clone().requires_grad_(True)
    I = ta.shade_intensity(c, d, sensor, px, py)
    I.backward(dev(gI))
    _close(c.grad.cpu().numpy().reshape(S, -1), ref["coeffs"].reshape(S, -1), "coefficients", floor_frac=1e-3)
    _close(d.grad.cpu().numpy().reshape(B, -1), ref["depth"].reshape(B, -1), "depth", floor_frac=1e-3)


def test_autograd_binding_matches_direct_adjoint():
    sc = calibration_scene(seed=5, E=8)
    gs, _ = upstream(sc, seed=2)
    gp, gt, gk = _adjoint(sc, gs)
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    pose = dev(sc.pad_pose).requires_grad_(True)
    twist = dev(sc.pad_twist).requires_grad_(True)
    ks = [dev(v).requires_grad_(True) for v in (sc.k_n, sc.k_d, sc.k_t, sc.mu)]
    depth, fn, ft, wr = ta.force_field(sdfs, dev(sc.taxels), dev(sc.obj_id), pose, twist, *ks)
    L = sum((o * dev(g)).sum() for o, g in zip((depth, fn, ft, wr), gs))
    L.backward()
    assert torch.equal(pose.grad.cpu(), torch.from_numpy(gp))
    assert torch.equal(twist.grad.cpu(), torch.from_numpy(gt))
    for i, k in enumerate(ks):
        assert torch.equal(k.grad.cpu(), torch.from_numpy(gk[:, i].copy()))


def test_calibration_step_reduces_the_loss():
    """A few gradient steps on k_n, k_t, mu from a perturbed start move the force field
    toward a target made with the true parameters."""
    sc = calibration_scene(seed=13, E=16)
    sdfs = tacsl.SdfSet.from_grids(sc.grids)
    taxels, obj = dev(sc.taxels), dev(sc.obj_id)
    pose, twist = dev(sc.pad_pose), dev(sc.pad_twist)
    kd = dev(sc.k_d)
    true = [dev(v) for v in (sc.k_n, sc.k_t, sc.mu)]
    with torch.no_grad():
        tgt = ta.force_field(sdfs, taxels, obj, pose, twist, true[0], kd, true[1], true[2])
    # parameters as relative offsets from a scale, started 20 % off
    delta = [torch.full_like(t, 0.2).requires_grad_(True) for t in true]
    opt = torch.optim.Adam(delta, lr=0.02)
    losses = []
    for _ in range(40):
        opt.zero_grad()
        ks = [t * (1 + d) for t, d in zip(true, delta)]
        _, fn, ft, _ = ta.force_field(sdfs, taxels, obj, pose, twist, ks[0], kd, ks[1], ks[2])
        loss = ((fn - tgt[1]) ** 2).sum() + ((ft - tgt[2]) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    assert losses[-1] < 0.2 * losses[0]


def test_force_adjoint_full_calibration_size_sampled():
    """1024 envs x 2 pads x 20x25 taxels against eight 128^3 grids (the calibration
    workload), in the bench's launch; the oracle gradient on 48 sampled pads."""
    sc = synth.scene_objects(seed=2, E=1024, P=2, depth_maps="none")
    sc.k_d = np.random.default_rng(2).uniform(1.0, 5.0, size=sc.E).astype(np.float32)
    rng = np.random.default_rng(7)
    picks = rng.choice(sc.E * sc.P, 48, replace=False)
    # upstream gradient on the sampled pads only (zero near kinks), zero elsewhere
    gs = [np.zeros((sc.E, sc.P, sc.T), np.float32), np.zeros((sc.E, sc.P, sc.T, 3), np.float32),
          np.zeros((sc.E, sc.P, sc.T, 3), np.float32), np.zeros((sc.E, sc.P, 6), np.float32)]
    for b in picks:
        e, p = divmod(int(b), sc.P)
        m = safe_taxels(sc.grids[sc.obj_id[e]], sc.taxels, sc.pad_pose[e, p], sc.pad_twist[e, p], float(sc.k_n[e]),
                        float(sc.k_d[e]), float(sc.k_t[e]), float(sc.mu[e]))
        gs[0][e, p] = rng.normal(size=sc.T) * m * 1e3
        gs[1][e, p] = rng.normal(size=(sc.T, 3)) * m[:, None]
        gs[2][e, p] = rng.normal(size=(sc.T, 3)) * m[:, None]
        if m.all():
            gs[3][e, p] = rng.normal(size=6)
    gp, gt, gk = _adjoint(sc, gs)
    for b in picks:
        e, p = divmod(int(b), sc.P)
        one = [g[e:e + 1, p:p + 1] for g in gs]
        prm = [np.array([v[e]], np.float32) for v in (sc.k_n, sc.k_d, sc.k_t, sc.mu)]
        ref = G.force_gradients(sc.grids, sc.taxels, sc.obj_id[e:e + 1], sc.pad_pose[e:e + 1, p:p + 1],
                                sc.pad_twist[e:e + 1, p:p + 1], *prm, *one)
        scale = max(np.abs(ref["pose"]).max(), 1e-30)
        assert np.abs(gp[e, p] - ref["pose"][0, 0]).max() <= RTOL * scale + 1e-9, (e, p)
        scale = max(np.abs(ref["twist"]).max(), 1e-30)
        assert np.abs(gt[e, p] - ref["twist"][0, 0]).max() <= RTOL * scale + 1e-9, (e, p)
