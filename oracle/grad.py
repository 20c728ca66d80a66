"""FP64 gradient oracle of the tactile step -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's baseline legs may import this
module; the product path (the CUDA library and its binding) never does.

The penalty force field with its per-pad wrench (Sec. III-C) and the shading of the
tactile image (Sec. III-B) are restated here in plain PyTorch CPU float64 operations,
so that torch.autograd differentiates exactly the definitions the C oracle evaluates:

  * SDF: trilinear interpolation of the grid (cell min(floor(u), n-2), clamped at 0), its
    gradient the central difference of that interpolant with step h/2 per axis, and the
    domain u in [0.5, n-1.5] per axis (readings c1-c3);
  * a tactile point p of a pad posed by (t, q) and moving with (v, w):
    x = R(q/|q|) p + t,  x' = v + w x x;
    where phi(x) < 0 and |grad phi| >= 1e-12:  n = grad phi/|grad phi|,  d' = n . x',
    f_n = max((-k_n + k_d d') phi, 0) n,  v_t = x' - d' n,
    f_t = -(v_t/|v_t|) min(k_t |v_t|, mu |f_n|)  (zero when v_t = 0);
    depth = -phi where phi < 0; both forces reported in the pad frame (R^T f);
  * wrench = (sum_i f_i, sum_i p_i x f_i), f = f_n + f_t, pad frame;
  * image: depth-map derivatives central inside and one-sided on the border (reading
    c10), n = (D_x, D_y, -1)/sqrt(1 + D_x^2 + D_y^2), m = (1, n_x, n_y, n_x^2, n_y^2,
    n_x n_y), I_c = sum_k A[k, c] m_k, clamped to [0, 255]: the continuous quantity the
    uint8 image rounds (reading c16), whose derivative is zero where it is clamped.

Decisions between pieces (in/out of contact, the unilateral clamp, stick/slip, the
interpolation cell, the intensity clamp) are taken on the values and carry no
derivative, so a gradient is that of the piece the point lies in: meaningful away
from the kinks between pieces, which the tests avoid.

The depth maps of the column camera are differentiated w.r.t. the pad pose by the
implicit function theorem at each column's first hit (render_gradients, reading c17).

Pinned by tests/test_oracle_grad_pins.py: the forward equals the C oracle's, the
gradients equal float64 central differences of the C oracle (h = 1e-6; h = 1e-5 for the
depth maps, whose hit search stops at voxel/65536), and closed forms (d f_n / d k_n =
depth n; stick and slip derivatives; a half-space whose field is exactly linear, for the
forces and for the depth maps; d I / d A_k = m_k; the flat-gel derivative of I w.r.t.
the depth).  The image loss (shade_mse) is pinned by its value from the C oracle's
intensities and by central differences of that value.  The pixel slopes (shade_slopes)
are pinned by their closed form on a flat gel and by the chain rule: their image under
the transposed derivative stencils is the (pinned) depth gradient.
"""
from __future__ import annotations

import itertools

import numpy as np
import torch

F64 = torch.float64


def _t(a, requires_grad=False):
    return torch.tensor(np.asarray(a, np.float64), dtype=F64, requires_grad=requires_grad)


def rotation(q):
    """R of the quaternion q = (w, x, y, z) after normalising it (pad -> object)."""
    q = q / torch.sqrt((q * q).sum())
    w, x, y, z = q[0], q[1], q[2], q[3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)]),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)]),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]),
    ])


def trilinear(data, u):
    """Trilinear interpolant of grid data [n2, n1, n0] at continuous indices u [N, 3]
    (x, y, z); cell min(floor(u), n - 2), clamped at 0."""
    n = torch.tensor([data.shape[2], data.shape[1], data.shape[0]])
    i = torch.minimum(torch.clamp(torch.floor(u.detach()).long(), min=0), n - 2)
    f = u - i.to(F64)
    acc = torch.zeros(u.shape[0], dtype=F64)
    for dz, dy, dx in itertools.product((0, 1), (0, 1), (0, 1)):
        w = ((f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) *
             (f[:, 2] if dz else 1 - f[:, 2]))
        acc = acc + w * data[i[:, 2] + dz, i[:, 1] + dy, i[:, 0] + dx]
    return acc


def sdf_eval(grid, x):
    """phi [N], its h/2 central-difference gradient [N, 3] and the domain mask at
    object-frame points x [N, 3]; grid = (data tensor, origin (3,), voxel h)."""
    data, origin, h = grid
    u = (x - origin) / h
    n = torch.tensor([data.shape[2], data.shape[1], data.shape[0]], dtype=F64)
    inside = ((u.detach() >= 0.5) & (u.detach() <= n - 1.5)).all(dim=1)
    phi = trilinear(data, u)
    g = []
    for a in range(3):
        e = torch.zeros(3, dtype=F64)
        e[a] = 0.5
        g.append((trilinear(data, u + e) - trilinear(data, u - e)) / h)
    return phi, torch.stack(g, dim=1), inside


def grid_tensors(g):
    """(data, origin, h) float64 tensors of a synth.Grid-like object."""
    return (torch.from_numpy(np.asarray(g.data, np.float64)), _t(np.asarray(g.origin, np.float64)),
            float(np.float32(g.voxel)))


def pad_forces(grid, taxels, pose, twist, kn, kd, kt, mu):
    """One pad: depth [T], f_n [T, 3], f_t [T, 3] (pad frame) and wrench [6].

    taxels [T, 3] float64 tensor; pose (7,), twist (6,) and the four parameters are
    float64 tensors that may require grad."""
    R = rotation(pose[3:7])
    x = taxels @ R.T + pose[0:3]
    v, w = twist[0:3], twist[3:6]
    xdot = v + torch.cross(w.expand_as(x), x, dim=1)
    phi, g, inside = sdf_eval(grid, x)
    T = taxels.shape[0]
    pen = inside & (phi.detach() < 0)
    gn = torch.sqrt((g.detach() ** 2).sum(dim=1))
    con = pen & (gn >= 1e-12)
    depth = torch.zeros(T, dtype=F64).index_put((pen.nonzero()[:, 0],), -phi[pen])
    ci = con.nonzero()[:, 0]
    gc, xd, ph = g[ci], xdot[ci], phi[ci]
    nrm = gc / torch.sqrt((gc * gc).sum(dim=1, keepdim=True))
    ddot = (nrm * xd).sum(dim=1)
    mraw = (-kn + kd * ddot) * ph
    mag = torch.where(mraw.detach() > 0, mraw, torch.zeros_like(mraw))
    fn = mag[:, None] * nrm
    vt = xd - ddot[:, None] * nrm
    s2 = (vt.detach() ** 2).sum(dim=1)
    sl = s2 > 0
    ft = torch.zeros_like(vt)
    if sl.any():
        vts = vt[sl]
        s = torch.sqrt((vts * vts).sum(dim=1))
        cap, lim = kt * s, mu * mag[sl]
        ftm = torch.where(cap.detach() < lim.detach(), cap, lim)
        ft = ft.index_put((sl.nonzero()[:, 0],), -(vts / s[:, None]) * ftm[:, None])
    fn_all = torch.zeros(T, 3, dtype=F64).index_put((ci,), fn)
    ft_all = torch.zeros(T, 3, dtype=F64).index_put((ci,), ft)
    fn_pad = fn_all @ R        # rows: R^T f
    ft_pad = ft_all @ R
    f = fn_pad + ft_pad
    wrench = torch.cat([f.sum(dim=0), torch.cross(taxels, f, dim=1).sum(dim=0)])
    return depth, fn_pad, ft_pad, wrench


def force_gradients(grids, taxels, obj_id, pad_pose, pad_twist, k_n, k_d, k_t, mu, g_depth, g_fn, g_ft,
                    g_wrench=None):
    """Gradient of L = sum(g_depth*depth) + sum(g_fn*f_n) + sum(g_ft*f_t) + sum(g_wrench*wrench)
    over E x P pads (shapes as the C oracle's penalty_forces; parameters of length 1 or E).

    Returns dict pose [E, P, 7], twist [E, P, 6], k_n, k_d, k_t, mu (length 1 or E), plus
    the forward outputs (depth, f_n, f_t, wrench) in float64."""
    pad_pose = np.asarray(pad_pose, np.float32)
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    tax = torch.from_numpy(np.asarray(taxels, np.float32).reshape(-1, 3).astype(np.float64))
    T = tax.shape[0]
    twist = np.asarray(pad_twist, np.float32).reshape(E, P, 6)
    prm = [np.atleast_1d(np.asarray(v, np.float32)).astype(np.float64) for v in (k_n, k_d, k_t, mu)]
    npar = prm[0].shape[0]
    gt = [torch.tensor(p, dtype=F64, requires_grad=True) for p in prm]
    gd = np.asarray(g_depth, np.float64).reshape(E, P, T)
    gfn = np.asarray(g_fn, np.float64).reshape(E, P, T, 3)
    gft = np.asarray(g_ft, np.float64).reshape(E, P, T, 3)
    gw = None if g_wrench is None else np.asarray(g_wrench, np.float64).reshape(E, P, 6)
    gt_grids = {}
    out = {k: np.zeros(s) for k, s in (("pose", (E, P, 7)), ("twist", (E, P, 6)), ("depth", (E, P, T)),
                                       ("f_n", (E, P, T, 3)), ("f_t", (E, P, T, 3)), ("wrench", (E, P, 6)))}
    for e in range(E):
        oid = int(np.asarray(obj_id).reshape(-1)[e])
        if oid not in gt_grids:
            gt_grids[oid] = grid_tensors(grids[oid])
        pi = 0 if npar == 1 else e
        for p in range(P):
            pose = _t(pad_pose[e, p].astype(np.float64), True)
            tw = _t(twist[e, p].astype(np.float64), True)
            depth, fn, ft, wr = pad_forces(gt_grids[oid], tax, pose, tw, gt[0][pi], gt[1][pi], gt[2][pi],
                                           gt[3][pi])
            L = ((depth * torch.from_numpy(gd[e, p])).sum() + (fn * torch.from_numpy(gfn[e, p])).sum() +
                 (ft * torch.from_numpy(gft[e, p])).sum())
            if gw is not None:
                L = L + (wr * torch.from_numpy(gw[e, p])).sum()
            if L.requires_grad:
                L.backward()
            out["pose"][e, p] = pose.grad.numpy() if pose.grad is not None else 0.0
            out["twist"][e, p] = tw.grad.numpy() if tw.grad is not None else 0.0
            out["depth"][e, p] = depth.detach().numpy()
            out["f_n"][e, p] = fn.detach().numpy()
            out["f_t"][e, p] = ft.detach().numpy()
            out["wrench"][e, p] = wr.detach().numpy()
    for name, t in zip(("k_n", "k_d", "k_t", "mu"), gt):
        out[name] = t.grad.numpy().copy() if t.grad is not None else np.zeros(npar)
    return out


def _axis_derivative(D, axis, pitch):
    """Derivative of D along `axis` (1: x / columns, 0: y / rows): central inside,
    one-sided on the border, zero along an axis of length 1."""
    n = D.shape[axis]
    if n < 2:
        return torch.zeros_like(D)
    sl = lambda a, b: D.narrow(axis, a, b - a)     # noqa: E731
    first = (sl(1, 2) - sl(0, 1)) / pitch
    last = (sl(n - 1, n) - sl(n - 2, n - 1)) / pitch
    if n == 2:
        return torch.cat([first, last], dim=axis)
    mid = (sl(2, n) - sl(0, n - 2)) / (2 * pitch)
    return torch.cat([first, mid, last], dim=axis)


def shade_intensity(coeffs, depth, pitch_x, pitch_y):
    """Clamped intensity [H, W, 3] of one image: coeffs [6, 3, H, W], depth [H, W]
    (float64 tensors, either may require grad)."""
    return _intensity_of_derivatives(coeffs, _axis_derivative(depth, 1, pitch_x), _axis_derivative(depth, 0, pitch_y))


def _intensity_of_derivatives(coeffs, dx, dy):
    """Clamped intensity [H, W, 3] from the depth derivatives dx = D_x, dy = D_y [H, W]."""
    inv = 1.0 / torch.sqrt(1.0 + dx * dx + dy * dy)
    nx, ny = dx * inv, dy * inv
    m = torch.stack([torch.ones_like(nx), nx, ny, nx * nx, ny * ny, nx * ny])       # [6, H, W]
    I = (coeffs * m[:, None]).sum(dim=0)                                            # [3, H, W]
    return torch.clamp(I, 0.0, 255.0).permute(1, 2, 0)


def shade_gradients(coeffs, pitch_x, pitch_y, sensor_id, depth, g_intensity):
    """Gradient of L = sum(g_intensity * I) over B images w.r.t. the coefficients
    [S, 6, 3, H, W] and the depth maps [B, H, W]; also returns the intensities."""
    coeffs = np.asarray(coeffs, np.float32)
    S, _, _, H, W = coeffs.shape
    depth = np.asarray(depth, np.float32).reshape(-1, H, W)
    B = depth.shape[0]
    gI = np.asarray(g_intensity, np.float64).reshape(B, H, W, 3)
    A = torch.tensor(coeffs.astype(np.float64), requires_grad=True)
    px, py = float(np.float32(pitch_x)), float(np.float32(pitch_y))
    g_depth = np.zeros((B, H, W))
    inten = np.zeros((B, H, W, 3))
    for b in range(B):
        s = int(np.asarray(sensor_id).reshape(-1)[b])
        D = torch.tensor(depth[b].astype(np.float64), requires_grad=True)
        I = shade_intensity(A[s], D, px, py)
        (I * torch.from_numpy(gI[b])).sum().backward()
        g_depth[b] = D.grad.numpy()
        inten[b] = I.detach().numpy()
    return {"coeffs": A.grad.numpy(), "depth": g_depth, "intensity": inten}



def shade_mse(coeffs, pitch_x, pitch_y, sensor_id, depth, target):
    """Squared error of the clamped intensities against target images [B, H, W, 3]:
    L = sum_s loss_map[s], loss_map[s, y, x] = sum over the images b of sensor s and the
    channels c of (clamp(I_c(b, y, x), 0, 255) - target[b, y, x, c])^2 (the image loss of
    sensor calibration, App. B and Sec. III-B, on the intensity of reading c16).  Returns dict
    loss_map [S, H, W], coeffs [S, 6, 3, H, W] and depth [B, H, W] (gradients of L)."""
    coeffs = np.asarray(coeffs, np.float32)
    S, _, _, H, W = coeffs.shape
    depth = np.asarray(depth, np.float32).reshape(-1, H, W)
    B = depth.shape[0]
    T = torch.from_numpy(np.asarray(target, np.float64).reshape(B, H, W, 3))
    A = torch.tensor(coeffs.astype(np.float64), requires_grad=True)
    px, py = float(np.float32(pitch_x)), float(np.float32(pitch_y))
    loss_map = np.zeros((S, H, W))
    g_depth = np.zeros((B, H, W))
    for b in range(B):
        s = int(np.asarray(sensor_id).reshape(-1)[b])
        D = torch.tensor(depth[b].astype(np.float64), requires_grad=True)
        err = (shade_intensity(A[s], D, px, py) - T[b]) ** 2
        loss_map[s] += err.detach().sum(dim=2).numpy()
        err.sum().backward()
        g_depth[b] = D.grad.numpy()
    return {"loss_map": loss_map, "coeffs": A.grad.numpy(), "depth": g_depth}


def shade_slopes(coeffs, pitch_x, pitch_y, sensor_id, depth, g_intensity=None, target=None):
    """Pixel slopes [B, H, W, 2]: at each pixel of each image, the gradient of that
    pixel's own term of L with respect to the two depth derivatives (D_x, D_y) its normal
    reads, the derivatives taken as independent variables.  L is sum(g_intensity * I)
    (g_intensity [B, H, W, 3]) or, with target [B, H, W, 3] instead, the squared error of
    shade_mse.  The depth gradient of L is the transpose of the derivative stencils
    applied to these slopes (chain rule through D -> (D_x, D_y)).  Images with a sensor id
    outside [0, S) are left at zero."""
    coeffs = np.asarray(coeffs, np.float32)
    S, _, _, H, W = coeffs.shape
    depth = np.asarray(depth, np.float32).reshape(-1, H, W)
    B = depth.shape[0]
    A = torch.tensor(coeffs.astype(np.float64))
    px, py = float(np.float32(pitch_x)), float(np.float32(pitch_y))
    out = np.zeros((B, H, W, 2))
    for b in range(B):
        s = int(np.asarray(sensor_id).reshape(-1)[b])
        if s < 0 or s >= S:
            continue
        D = torch.tensor(depth[b].astype(np.float64))
        dx = _axis_derivative(D, 1, px).requires_grad_(True)
        dy = _axis_derivative(D, 0, py).requires_grad_(True)
        I = _intensity_of_derivatives(A[s], dx, dy)
        if target is not None:
            T = torch.from_numpy(np.asarray(target, np.float64).reshape(B, H, W, 3)[b])
            ((I - T) ** 2).sum().backward()
        else:
            (I * torch.from_numpy(np.asarray(g_intensity, np.float64).reshape(B, H, W, 3)[b])).sum().backward()
        out[b, :, :, 0] = dx.grad.numpy()
        out[b, :, :, 1] = dy.grad.numpy()
    return out


GRAZING = 0.05   # |d phi / dz| below this: a grazing column, whose depth gradient is left out


def render_gradients(grids, obj_id, pad_pose, H, W, pitch_x, pitch_y, x0, y0, d0, z_max, g_depth, depth=None):
    """Gradient of L = sum(g_depth * D) w.r.t. the pad poses [E, P, 7], D [E, P, H, W] the
    depth maps of the column camera (the C oracle's render_depth, Sec. III-B).

    A column that meets the object at z_hit in (-z_max, 0) has D = d0 + z_hit, where z_hit
    solves phi(R p + t) = 0 for the pad-frame point p = (x_i, y_j, z_hit).  By the implicit
    function theorem d z_hit = -(d phi) / (d phi / dz) at the hit, with d phi / dz =
    grad phi . R e_z (reading c17); phi is the trilinear interpolant and its derivatives
    are taken by autograd at the hit point.  The columns are classified on the float32
    value of D, the precision of the maps the library carries: D >= d0 (no hit) and
    D <= d0 - z_max (the object reaches below the camera's range and D is clamped) carry
    no derivative, and neither do grazing columns (|d phi / dz| < GRAZING) nor hit points
    outside the grid's domain.

    depth: the maps whose hit points are differentiated (default: the C oracle's render).
    Returns dict pose [E, P, 7] (NaN for an env with a bad obj_id), depth [E, P, H, W] and
    phi_z [E, P, H, W] (d phi / dz at each column whose hit lies in the grid's domain,
    grazing or not; NaN elsewhere)."""
    import oracle as orc_c
    pad_pose = np.asarray(pad_pose, np.float32)
    E, P = pad_pose.shape[0], pad_pose.shape[1]
    obj_id = np.asarray(obj_id).reshape(-1)
    if depth is None:
        depth, _ = orc_c.render_depth(grids, obj_id, pad_pose, H, W, pitch_x, pitch_y, x0, y0, d0, z_max)
    depth = np.asarray(depth, np.float64).reshape(E, P, H, W)
    f32 = np.float32
    d0f, zf = float(f32(d0)), float(f32(z_max))
    top, bottom = f32(d0f), f32(f32(d0f) - f32(zf))
    xs = float(f32(x0)) + np.arange(W) * float(f32(pitch_x))
    ys = float(f32(y0)) + np.arange(H) * float(f32(pitch_y))
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    gd = np.asarray(g_depth, np.float64).reshape(E, P, H, W)
    out = np.zeros((E, P, 7))
    phi_z_map = np.full((E, P, H, W), np.nan)
    cache = {}
    for e in range(E):
        oid = int(obj_id[e])
        if oid < 0 or oid >= len(grids):
            out[e] = np.nan
            continue
        if oid not in cache:
            cache[oid] = grid_tensors(grids[oid])
        grid = cache[oid]
        for p in range(P):
            D = depth[e, p]
            D32 = D.astype(f32)
            hit = (D32 < top) & (D32 > bottom)
            if not hit.any():
                continue
            pose = _t(pad_pose[e, p].astype(np.float64), True)
            R = rotation(pose[3:7])
            z = torch.tensor(D[hit] - d0f, dtype=F64, requires_grad=True)
            pts = torch.stack([torch.tensor(xx[hit], dtype=F64), torch.tensor(yy[hit], dtype=F64), z], dim=1)
            x = pts @ R.T + pose[0:3]
            phi, _, inside = sdf_eval(grid, x)
            (phi_z,) = torch.autograd.grad(phi.sum(), z, retain_graph=True)
            keep = inside & (phi_z.abs() >= GRAZING)
            pz = phi_z.detach()
            dz = -phi / torch.where(keep, pz, torch.ones_like(pz))
            L = (torch.tensor(gd[e, p][hit], dtype=F64) * keep * dz).sum()
            L.backward()
            out[e, p] = pose.grad.numpy()
            pzm = np.where(inside.numpy(), pz.numpy(), np.nan)
            phi_z_map[e, p][hit] = pzm
    return {"pose": out, "depth": depth, "phi_z": phi_z_map}
