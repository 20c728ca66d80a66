"""Seeded synthetic inputs for the tactile step.

This module only *makes inputs*: analytic object shapes baked into signed-distance
grids, taxel templates, pad poses and twists, contact parameters, elastomer depth
maps and per-pixel shading coefficients.  It contains none of the tactile step's
own arithmetic (no SDF interpolation, no force law, no normal estimation, no
shading); both the CUDA library and the FP64 oracle consume what it produces.

Conventions shared by every consumer:

* SDF grid: float32 array ``[n2][n1][n0]`` (x fastest), node ``(i, j, k)`` at
  ``origin + (i, j, k) * voxel`` in the object frame; negative inside the object.
* Taxel template: float32 ``[T][3]`` in the pad frame, on the ``z = 0`` plane,
  row-major over ``ny`` rows by ``nx`` columns at ``pitch`` metres, centred.
  The pad's ``+z`` axis is the outward normal pointing toward the object.
* Pad pose: float32 ``[7]`` = ``(tx, ty, tz, qw, qx, qy, qz)``, the transform from
  pad frame to object frame, ``x_o = R(q) x_p + t``.
* Pad twist: float32 ``[6]`` = ``(vx, vy, vz, wx, wy, wz)``, the pad's velocity
  relative to the object in the object frame, referenced at the object origin:
  a pad-fixed point at ``x_o`` moves with ``v + w x x_o``.
* Depth map: float32 ``[H][W]``, camera-to-gel distance in metres; the
  undeformed gel reads the constant ``D0``.
* Shading coefficients: float32 ``[S][6][3][H][W]`` (term, channel, row, col).

Random streams use NumPy's PCG64 with the seeds stated by each function.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

D0 = 0.020  # undeformed camera-to-gel distance [m]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# Analytic shapes (object frame, centred at the origin, prism/cylinder axis = z)
# ---------------------------------------------------------------------------

@dataclass
class Shape:
    kind: str                 # "sphere" | "box" | "cylinder" | "hexprism" | "plane"
    dims: tuple               # sphere (R,), box (hx, hy, hz), cylinder (r, hz), hexprism (apothem, hz)
                              # plane (nx, ny, nz, offset): occupied where n.x < offset

    def extent(self) -> float:
        """Largest full dimension of the shape (for grid sizing)."""
        k, d = self.kind, self.dims
        if k == "sphere":
            return 2 * d[0]
        if k == "box":
            return 2 * max(d)
        if k == "cylinder":
            return 2 * max(d[0], d[1])
        if k == "hexprism":
            return 2 * max(2 * d[0] / math.sqrt(3.0), d[1])
        raise ValueError(k)

    def sdf(self, x: np.ndarray) -> np.ndarray:
        """Exact signed distance at points ``x[..., 3]`` (float64)."""
        k, d = self.kind, self.dims
        if k == "sphere":
            return np.linalg.norm(x, axis=-1) - d[0]
        if k == "plane":
            n = np.asarray(d[:3], dtype=np.float64)
            n = n / np.linalg.norm(n)
            return x @ n - d[3]
        if k == "box":
            q = np.abs(x) - np.asarray(d, dtype=np.float64)
            outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
            inside = np.minimum(q.max(axis=-1), 0.0)
            return outside + inside
        if k == "cylinder":
            r, hz = d
            q = np.stack([np.hypot(x[..., 0], x[..., 1]) - r, np.abs(x[..., 2]) - hz], -1)
            return np.linalg.norm(np.maximum(q, 0.0), axis=-1) + np.minimum(q.max(axis=-1), 0.0)
        if k == "hexprism":
            a, hz = d
            d2 = _hexagon_sdf(x[..., 0], x[..., 1], a)
            q = np.stack([d2, np.abs(x[..., 2]) - hz], -1)
            return np.linalg.norm(np.maximum(q, 0.0), axis=-1) + np.minimum(q.max(axis=-1), 0.0)
        raise ValueError(k)

    def support(self, dvec: np.ndarray) -> float:
        """max over points x of the shape of dvec . x (support function)."""
        k, d = self.kind, self.dims
        dvec = np.asarray(dvec, dtype=np.float64)
        if k == "sphere":
            return d[0] * float(np.linalg.norm(dvec))
        if k == "box":
            return float(np.abs(dvec) @ np.asarray(d, dtype=np.float64))
        if k == "cylinder":
            return d[0] * float(np.hypot(dvec[0], dvec[1])) + d[1] * abs(float(dvec[2]))
        if k == "hexprism":
            verts = _hexagon_vertices(d[0])
            return float(np.max(verts @ dvec[:2])) + d[1] * abs(float(dvec[2]))
        raise ValueError(k)


def _hexagon_vertices(apothem: float) -> np.ndarray:
    """Regular hexagon with flat sides at y = +-apothem: vertices at 0, 60, ... degrees."""
    rho = 2.0 * apothem / math.sqrt(3.0)
    ang = np.arange(6) * (math.pi / 3.0)
    return np.stack([rho * np.cos(ang), rho * np.sin(ang)], -1)


def _hexagon_sdf(px: np.ndarray, py: np.ndarray, apothem: float) -> np.ndarray:
    """Exact 2-D signed distance to the hexagon of ``_hexagon_vertices``.

    Fold by symmetry: first into the quadrant x, y >= 0, then mirror across the
    60-degree line through the centre, so the point lies in the wedge 60..120
    degrees that the top side (y = apothem, |x| <= apothem/sqrt 3) spans.  In that
    wedge the top side holds the nearest boundary point: inside, the distance is
    apothem - y; outside, it is the distance to the clamped point on the side.
    """
    x = np.abs(px)
    y = np.abs(py)
    ux, uy = 0.5, math.sqrt(3.0) / 2.0          # unit vector of the 60-degree line
    below = (ux * y - uy * x) < 0.0             # angle under 60 degrees
    pu = x * ux + y * uy
    x, y = np.where(below, 2 * pu * ux - x, x), np.where(below, 2 * pu * uy - y, y)
    half_side = apothem / math.sqrt(3.0)
    dx = x - np.clip(x, -half_side, half_side)
    dy = y - apothem
    return np.where(dy > 0.0, np.hypot(dx, dy), dy)


@dataclass
class Grid:
    data: np.ndarray          # float32 [n2][n1][n0]
    origin: np.ndarray        # float32 [3]
    voxel: float              # float32-representable
    shape: Shape | None = None

    @property
    def n(self) -> tuple:
        return (self.data.shape[2], self.data.shape[1], self.data.shape[0])


def bake(shape: Shape, n: int | tuple, voxel: float, origin=None) -> Grid:
    """Sample the shape's exact SDF at the grid nodes (float64 -> float32)."""
    if isinstance(n, int):
        n = (n, n, n)
    voxel = float(np.float32(voxel))
    if origin is None:
        origin = [-(n[a] - 1) * voxel / 2.0 for a in range(3)]
    origin = np.asarray(origin, dtype=np.float32)
    ax = [origin[a].astype(np.float64) + np.arange(n[a], dtype=np.float64) * voxel for a in range(3)]
    zz, yy, xx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    pts = np.stack([xx, yy, zz], -1)
    data = shape.sdf(pts).astype(np.float32)
    return Grid(np.ascontiguousarray(data), origin, voxel, shape)


def bake_extrusion(shape: Shape, n: int, voxel: float) -> Grid:
    """``bake`` for the shapes that are extrusions along z of a 2-D section (box,
    cylinder, hexagonal prism), at a fraction of the cost: the exact SDF of an
    extrusion is sqrt(max(d2, 0)^2 + max(dz, 0)^2) + min(max(d2, dz), 0) with d2 the
    section's 2-D distance and dz = |z| - hz, so d2 is evaluated on the n x n plane and
    dz on the n nodes of the z axis only (the same values as ``bake`` up to float64
    rounding)."""
    voxel = float(np.float32(voxel))
    origin = np.asarray([-(n - 1) * voxel / 2.0] * 3, dtype=np.float32)
    ax = [origin[a].astype(np.float64) + np.arange(n, dtype=np.float64) * voxel for a in range(3)]
    yy, xx = np.meshgrid(ax[1], ax[0], indexing="ij")
    k, d = shape.kind, shape.dims
    if k == "box":
        qx, qy = np.abs(xx) - d[0], np.abs(yy) - d[1]
        d2 = np.hypot(np.maximum(qx, 0.0), np.maximum(qy, 0.0)) + np.minimum(np.maximum(qx, qy), 0.0)
        hz = d[2]
    elif k == "cylinder":
        d2, hz = np.hypot(xx, yy) - d[0], d[1]
    elif k == "hexprism":
        d2, hz = _hexagon_sdf(xx, yy, d[0]), d[1]
    else:
        raise ValueError(f"{k} is not an extrusion along z")
    dz = (np.abs(ax[2]) - hz)[:, None, None]
    d2 = d2[None, :, :]
    out = np.hypot(np.maximum(d2, 0.0), np.maximum(dz, 0.0)) + np.minimum(np.maximum(d2, dz), 0.0)
    return Grid(np.ascontiguousarray(out.astype(np.float32)), origin, voxel, shape)


def bake_field(values_fn, n: tuple, voxel: float, origin) -> Grid:
    """Bake an arbitrary callable f(x, y, z) (float64 arrays) into a grid."""
    voxel = float(np.float32(voxel))
    origin = np.asarray(origin, dtype=np.float32)
    ax = [origin[a].astype(np.float64) + np.arange(n[a], dtype=np.float64) * voxel for a in range(3)]
    zz, yy, xx = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return Grid(np.ascontiguousarray(values_fn(xx, yy, zz).astype(np.float32)), origin, voxel, None)


# ---------------------------------------------------------------------------
# Rotations (input synthesis only)
# ---------------------------------------------------------------------------

def quat_to_matrix(q) -> np.ndarray:
    w, x, y, z = (float(v) for v in q)
    s = math.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / s, x / s, y / s, z / s
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def quat_multiply(a, b):
    aw, ax, ay, az = a
    bw, bx, by, bz = b
    return np.array([aw * bw - ax * bx - ay * by - az * bz,
                     aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx,
                     aw * bz + ax * by - ay * bx + az * bw])


def random_quaternion(g: np.random.Generator) -> np.ndarray:
    """Uniform on SO(3): a normalised 4-D Gaussian, sign fixed to qw >= 0."""
    q = g.standard_normal(4)
    q /= np.linalg.norm(q)
    return q if q[0] >= 0 else -q


def quat_from_axis_angle(axis, angle) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    return np.concatenate([[math.cos(angle / 2)], math.sin(angle / 2) * axis])


# ---------------------------------------------------------------------------
# Pads
# ---------------------------------------------------------------------------

def taxel_grid(ny: int, nx: int, pitch: float, pitch_y: float | None = None) -> np.ndarray:
    """Taxel template [ny*nx][3] (row-major, x fastest), centred, z = 0; rows are
    ``pitch_y`` apart (default ``pitch``)."""
    xs = (np.arange(nx) - (nx - 1) / 2.0) * pitch
    ys = (np.arange(ny) - (ny - 1) / 2.0) * (pitch if pitch_y is None else pitch_y)
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    return np.ascontiguousarray(np.stack([xx, yy, np.zeros_like(xx)], -1).reshape(-1, 3).astype(np.float32))


def place_pad(shape: Shape, q: np.ndarray, delta: float, offset_xy=(0.0, 0.0)) -> np.ndarray:
    """Pose whose pad plane cuts ``delta`` metres into the shape (negative = gap).

    The pad normal ``n = R e_z`` points toward the object; the object's point
    nearest the pad along ``n`` sits at ``n.x = -support(-n)``; the pad plane is
    put ``delta`` beyond it, and shifted in-plane by ``offset_xy`` (pad axes).
    """
    Rm = quat_to_matrix(q)
    n = Rm[:, 2]
    lowest = -shape.support(-n)
    t = (lowest + delta) * n + offset_xy[0] * Rm[:, 0] + offset_xy[1] * Rm[:, 1]
    return np.concatenate([t, q]).astype(np.float32)


# ---------------------------------------------------------------------------
# Depth maps and shading coefficients
# ---------------------------------------------------------------------------

def pixel_plane_points(H: int, W: int, extent_x: float, extent_y: float) -> np.ndarray:
    """Pad-frame points (pixel centres on z = 0) of an H x W image covering the pad."""
    xs = -extent_x / 2 + (np.arange(W) + 0.5) * (extent_x / W)
    ys = -extent_y / 2 + (np.arange(H) + 0.5) * (extent_y / H)
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([xx, yy, np.zeros_like(xx)], -1)


def depth_map(shape: Shape, pose: np.ndarray, H: int, W: int, extent_x: float, extent_y: float,
              d0: float = D0) -> np.ndarray:
    """Heightfield of the gel: D = D0 - max(0, -sdf(pixel point on the pad plane)).

    A synthetic stand-in for the in-sensor camera render; it gives a flat
    background with an indentation blob wherever the object cuts the pad plane.
    """
    P = pixel_plane_points(H, W, extent_x, extent_y).reshape(-1, 3)
    Rm = quat_to_matrix(pose[3:7])
    xo = P @ Rm.T + pose[:3].astype(np.float64)
    pen = np.maximum(0.0, -shape.sdf(xo))
    return (d0 - pen).reshape(H, W).astype(np.float32)


def shading_coeffs(n_sensor: int, H: int, W: int, seed: int) -> np.ndarray:
    """Per-pixel quadratic shading coefficients [S][6][3][H][W].

    Term 0 is the background: 90 + 60 (1 - r^2) plus a per-channel offset, with
    r the pixel's radius normalised to the image half-diagonal.  Terms 1-2 are
    drawn U(-120, 120), terms 3-5 U(-80, 80) at the four image corners and
    varied bilinearly across the image.
    """
    g = rng(seed)
    out = np.empty((n_sensor, 6, 3, H, W), dtype=np.float32)
    v = (np.arange(H) + 0.5) / H
    u = (np.arange(W) + 0.5) / W
    vv, uu = np.meshgrid(v, u, indexing="ij")
    r2 = ((uu - 0.5) ** 2 + (vv - 0.5) ** 2) / 0.5
    for s in range(n_sensor):
        offs = g.uniform(-20, 20, size=3)
        for c in range(3):
            out[s, 0, c] = 90.0 + 60.0 * (1.0 - r2) + offs[c]
        for k in range(1, 6):
            amp = 120.0 if k <= 2 else 80.0
            for c in range(3):
                cor = g.uniform(-amp, amp, size=4)  # (0,0) (0,1) (1,0) (1,1)
                out[s, k, c] = ((1 - vv) * (1 - uu) * cor[0] + (1 - vv) * uu * cor[1]
                                + vv * (1 - uu) * cor[2] + vv * uu * cor[3])
    return out


# ---------------------------------------------------------------------------
# Whole workloads
# ---------------------------------------------------------------------------

@dataclass
class Scene:
    """Everything one tactile step consumes (host numpy arrays)."""
    grids: list                       # list[Grid]
    taxels: np.ndarray                # [T][3] f32
    obj_id: np.ndarray                # [E] i32
    pad_pose: np.ndarray              # [E][P][7] f32
    pad_twist: np.ndarray             # [E][P][6] f32
    k_n: np.ndarray                   # [1] or [E] f32
    k_d: np.ndarray
    k_t: np.ndarray
    mu: np.ndarray
    H: int = 0
    W: int = 0
    pitch_x: float = 0.0
    pitch_y: float = 0.0
    coeffs: np.ndarray | None = None  # [S][6][3][H][W] f32
    sensor_id: np.ndarray | None = None   # [E*P] i32
    depth_map: np.ndarray | None = None   # [E][P][H][W] f32
    meta: dict = field(default_factory=dict)

    @property
    def E(self):
        return self.pad_pose.shape[0]

    @property
    def P(self):
        return self.pad_pose.shape[1]

    @property
    def T(self):
        return self.taxels.shape[0]


def scene_sphere_pad(seed: int = 1, E: int = 1, ny: int = 16, nx: int = 20, pitch: float = 1e-3,
                     R: float = 5e-3, n: int = 64, voxel: float = 0.25e-3, H: int = 120, W: int = 160,
                     vel_sigma: float = 0.02, with_images: bool = True) -> Scene:
    """One pad pressed by a sphere (R = 5 mm, 64^3 grid at 0.25 mm), per env.

    Indentation U(0, 1 mm), in-plane offset U(-3, 3 mm), twist v ~ N(0, 0.02 m/s)
    per axis with zero angular part; k_n = 1e4, k_d = 0, k_t = 1e2, mu = 0.5;
    a 160 x 120 depth map of the same contact and seeded shading coefficients
    (seed + 100).
    """
    g = rng(seed)
    shape = Shape("sphere", (R,))
    grid = bake(shape, n, voxel)
    taxels = taxel_grid(ny, nx, pitch)
    pose = np.zeros((E, 1, 7), np.float32)
    twist = np.zeros((E, 1, 6), np.float32)
    ext_x, ext_y = (nx - 1) * pitch, (ny - 1) * pitch
    dmaps = np.zeros((E, 1, H, W), np.float32) if with_images else None
    for e in range(E):
        delta = g.uniform(0.0, 1e-3)
        off = g.uniform(-3e-3, 3e-3, size=2)
        q = np.array([1.0, 0.0, 0.0, 0.0])
        pose[e, 0] = place_pad(shape, q, delta, off)
        twist[e, 0, :3] = g.normal(0.0, vel_sigma, size=3)
        if with_images:
            dmaps[e, 0] = depth_map(shape, pose[e, 0], H, W, ext_x, ext_y)
    sc = Scene([grid], taxels, np.zeros(E, np.int32), pose, twist,
               np.array([1e4], np.float32), np.array([0.0], np.float32),
               np.array([1e2], np.float32), np.array([0.5], np.float32))
    if with_images:
        sc.H, sc.W = H, W
        sc.pitch_x, sc.pitch_y = ext_x / W, ext_y / H
        sc.coeffs = shading_coeffs(1, H, W, seed + 100)
        sc.sensor_id = np.zeros(E, np.int32)
        sc.depth_map = dmaps
    return sc


def object_set(seed: int, n_obj: int = 8, n: int = 128, dims_mm=(5.0, 20.0)) -> list:
    """Cylinders, boxes and hexagonal prisms with seeded dimensions, baked at n^3.

    Kinds cycle 3 cylinders, 3 boxes, 2 hex prisms (for 8 objects); each full
    dimension is U(dims_mm) millimetres; the grid side is the largest dimension
    plus 6 mm, so the voxel is side / (n - 1).
    """
    g = rng(seed)
    kinds = (["cylinder"] * 3 + ["box"] * 3 + ["hexprism"] * 2)
    grids = []
    lo, hi = dims_mm[0] * 1e-3, dims_mm[1] * 1e-3
    for i in range(n_obj):
        kind = kinds[i % len(kinds)]
        if kind == "cylinder":
            shape = Shape(kind, (g.uniform(lo, hi) / 2, g.uniform(lo, hi) / 2))
        elif kind == "box":
            shape = Shape(kind, tuple(g.uniform(lo, hi, size=3) / 2))
        else:
            shape = Shape(kind, (g.uniform(lo, hi) / 2, g.uniform(lo, hi) / 2))
        side = shape.extent() + 6e-3
        grids.append(bake(shape, n, side / (n - 1)))
    return grids


def scene_objects(seed: int = 2, E: int = 4096, P: int = 2, ny: int = 20, nx: int = 25,
                  pitch: float = 1e-3, n_obj: int = 8, n: int = 128, H: int = 240, W: int = 320,
                  vel_sigma: float = 0.05, depth_maps: str = "exact", n_distinct_maps: int = 256,
                  grids: list | None = None) -> Scene:
    """E envs x P pads against one of ``n_obj`` objects each.

    Pad orientation uniform on SO(3); the pad plane cuts U(-2, 2) mm into the
    object's nearest point (about half the pads touch) with an in-plane offset
    U(-2, 2) mm; twist v ~ N(0, 0.05 m/s) per axis, zero angular part; obj_id
    U{0..n_obj-1}; contact parameters per env (k_n U(0.5e4, 1.5e4), k_d 0,
    k_t U(50, 150), mu U(0.3, 0.7)); pad slot p uses sensor model p.

    ``depth_maps``: "exact" renders every pad's own heightfield; "cycled" renders
    ``n_distinct_maps`` of them and fills the batch by cycling through those
    (each slot is still its own buffer); "none" skips images.
    """
    g = rng(seed)
    if grids is None:
        grids = object_set(seed, n_obj, n)
    taxels = taxel_grid(ny, nx, pitch)
    obj = g.integers(0, len(grids), size=E).astype(np.int32)
    pose = np.zeros((E, P, 7), np.float32)
    twist = np.zeros((E, P, 6), np.float32)
    for e in range(E):
        shape = grids[obj[e]].shape
        for p in range(P):
            q = random_quaternion(g)
            delta = g.uniform(-2e-3, 2e-3)
            off = g.uniform(-2e-3, 2e-3, size=2)
            pose[e, p] = place_pad(shape, q, delta, off)
            twist[e, p, :3] = g.normal(0.0, vel_sigma, size=3)
    k_n = g.uniform(0.5e4, 1.5e4, size=E).astype(np.float32)
    k_d = np.zeros(E, np.float32)
    k_t = g.uniform(50.0, 150.0, size=E).astype(np.float32)
    mu = g.uniform(0.3, 0.7, size=E).astype(np.float32)
    sc = Scene(grids, taxels, obj, pose, twist, k_n, k_d, k_t, mu)
    if depth_maps != "none":
        ext_x, ext_y = (nx - 1) * pitch, (ny - 1) * pitch
        sc.H, sc.W = H, W
        sc.pitch_x, sc.pitch_y = ext_x / W, ext_y / H
        sc.coeffs = shading_coeffs(P, H, W, seed + 100)
        sc.sensor_id = np.tile(np.arange(P, dtype=np.int32), E)
        B = E * P
        dm = np.empty((E, P, H, W), np.float32)
        flat = dm.reshape(B, H, W)
        nd = B if depth_maps == "exact" else min(B, n_distinct_maps)
        for b in range(nd):
            e, p = divmod(b, P)
            flat[b] = depth_map(grids[obj[e]].shape, pose[e, p], H, W, ext_x, ext_y)
        for b in range(nd, B):
            flat[b] = flat[b % nd]
        sc.depth_map = dm
        sc.meta["distinct_depth_maps"] = nd
    return sc


# ---------------------------------------------------------------------------
# Uneven batches: every pad with its own resolution, object and sensor model
# ---------------------------------------------------------------------------

def log_uniform_int(g: np.random.Generator, lo: int, hi: int, size=None) -> np.ndarray:
    """Integers log-uniform on [lo, hi] (rounded from a log-uniform real)."""
    return np.rint(np.exp(g.uniform(np.log(lo), np.log(hi), size=size))).astype(np.int64)


def grid_pool(seed: int, n_grid: int = 32, n_lo: int = 32, n_hi: int = 256, dims_mm=(5.0, 20.0),
              sides=None) -> list:
    """``n_grid`` objects (cylinders, boxes, hex prisms in turn, dimensions U(dims_mm))
    baked at cubic grids of side log-uniform in [n_lo, n_hi] (or the given ``sides``);
    grid extent = largest dimension + 6 mm."""
    g = rng(seed)
    kinds = ["cylinder", "box", "hexprism"]
    lo, hi = dims_mm[0] * 1e-3, dims_mm[1] * 1e-3
    if sides is None:
        sides = log_uniform_int(g, n_lo, n_hi, size=n_grid)
    grids = []
    for i, n in enumerate(sides):
        kind = kinds[i % 3]
        if kind == "box":
            shape = Shape(kind, tuple(g.uniform(lo, hi, size=3) / 2))
        else:
            shape = Shape(kind, (g.uniform(lo, hi) / 2, g.uniform(lo, hi) / 2))
        side = shape.extent() + 6e-3
        grids.append(bake_extrusion(shape, int(n), side / (int(n) - 1)))
    return grids


@dataclass
class BatchScene:
    """An uneven batch (host numpy arrays).  Pad b of env e = b // P uses object
    obj_id[b], taxel layout layout[b] (points layout_first[l] .. + layout_count[l] of
    ``taxels``) and sensor model sensor[b] (-1: no image); its depth map is the
    ``depth_maps[b]`` array of the model's size (None without image)."""
    grids: list
    taxels: np.ndarray                # [n_points][3] taxel pool
    layout_first: np.ndarray          # [n_layout] i64
    layout_count: np.ndarray          # [n_layout] i32
    layout_shape: list                # [(ny, nx)]
    obj_id: np.ndarray                # [n_pad] i32
    layout: np.ndarray                # [n_pad] i32
    sensor: np.ndarray                # [n_pad] i32
    pad_pose: np.ndarray              # [n_pad][7] f32
    pad_twist: np.ndarray             # [n_pad][6] f32
    k_n: np.ndarray                   # [n_pad] f32
    k_d: np.ndarray
    k_t: np.ndarray
    mu: np.ndarray
    models: list                      # [(coeffs [6][3][H][W] f32, pitch_x, pitch_y)]
    depth_maps: list                  # [n_pad] of [H][W] f32 or None
    meta: dict = field(default_factory=dict)

    @property
    def n_pad(self):
        return self.obj_id.shape[0]


PAD_EXTENT = (24e-3, 19e-3)   # taxel-grid extent (x, y) of every pad, metres


def scene_batch(seed: int = 3, E: int = 16384, P: int = 2, grids: list | None = None, n_grid: int = 32,
                grid_sides=(32, 256), res_y=(10, 40), res_x=(12, 50), width=(160, 640), n_size_class: int = 16,
                vel_sigma: float = 0.05, depth_maps: str = "exact", n_distinct_maps: int = 8,
                no_image_frac: float = 0.0) -> BatchScene:
    """E envs x P pads, every env drawing its own pad resolution (ny log-uniform in
    res_y, nx in res_x; the taxels span PAD_EXTENT at pitch extent/(n-1)), its object
    from a pool of ``n_grid`` SDF grids (sides log-uniform in grid_sides) and an image
    size class (W log-uniform in ``width``, stratified over the classes, rounded to a
    multiple of 4; H = 3/4 W rounded to a multiple of 4); pad slot p of size class c uses sensor model
    P*c + p, each with its own seeded coefficients.  Poses, twists and contact
    parameters follow ``scene_objects``; parameters are drawn per env and repeated per
    pad.  A fraction ``no_image_frac`` of the pads has no image.

    ``depth_maps``: "exact" renders each pad's heightfield; "cycled" renders
    ``n_distinct_maps`` per sensor model and hands them out in turn; "none" makes no
    depth maps (the pads keep their sensor models)."""
    g = rng(seed)
    if grids is None:
        grids = grid_pool(seed + 1, n_grid, *grid_sides)
    # image size classes
    # class c's width is log-uniform within the c-th of n_size_class equal slices of
    # [log width[0], log width[1]] (stratified, so the classes span the whole range)
    u = (np.arange(n_size_class) + g.random(n_size_class)) / n_size_class
    ws = np.exp(np.log(width[0]) + u * (np.log(width[1]) - np.log(width[0])))
    ws = np.maximum(4, 4 * np.rint(ws / 4.0).astype(np.int64))
    hs = np.maximum(4, 4 * np.rint(0.75 * ws / 4.0).astype(np.int64))
    models = []
    for c in range(n_size_class):
        H, W = int(hs[c]), int(ws[c])
        for p in range(P):
            co = shading_coeffs(1, H, W, seed * 1000 + P * c + p)[0]
            models.append((co, PAD_EXTENT[0] / W, PAD_EXTENT[1] / H))
    # per env draws
    ny = log_uniform_int(g, res_y[0], res_y[1], size=E)
    nx = log_uniform_int(g, res_x[0], res_x[1], size=E)
    obj_env = g.integers(0, len(grids), size=E)
    cls_env = g.integers(0, n_size_class, size=E)
    layouts, pool, first, count, shapes = {}, [], [], [], []
    n_points = 0
    lay_env = np.empty(E, np.int32)
    for e in range(E):
        key = (int(ny[e]), int(nx[e]))
        if key not in layouts:
            t = taxel_grid(key[0], key[1], PAD_EXTENT[0] / max(key[1] - 1, 1), PAD_EXTENT[1] / max(key[0] - 1, 1))
            layouts[key] = len(first)
            first.append(n_points)
            count.append(t.shape[0])
            shapes.append(key)
            pool.append(t)
            n_points += t.shape[0]
        lay_env[e] = layouts[key]
    n_pad = E * P
    obj = np.repeat(obj_env, P).astype(np.int32)
    layout = np.repeat(lay_env, P).astype(np.int32)
    sensor = (P * np.repeat(cls_env, P) + np.tile(np.arange(P), E)).astype(np.int32)
    if no_image_frac > 0:
        sensor[g.random(n_pad) < no_image_frac] = -1
    pose = np.zeros((n_pad, 7), np.float32)
    twist = np.zeros((n_pad, 6), np.float32)
    for b in range(n_pad):
        q = random_quaternion(g)
        delta = g.uniform(-2e-3, 2e-3)
        off = g.uniform(-2e-3, 2e-3, size=2)
        pose[b] = place_pad(grids[obj[b]].shape, q, delta, off)
        twist[b, :3] = g.normal(0.0, vel_sigma, size=3)
    k_n = np.repeat(g.uniform(0.5e4, 1.5e4, size=E), P).astype(np.float32)
    k_d = np.zeros(n_pad, np.float32)
    k_t = np.repeat(g.uniform(50.0, 150.0, size=E), P).astype(np.float32)
    mu = np.repeat(g.uniform(0.3, 0.7, size=E), P).astype(np.float32)
    maps = [None] * n_pad
    made = {}
    for b in range(n_pad):
        m = int(sensor[b])
        if m < 0 or depth_maps == "none":
            continue
        H, W = models[m][0].shape[2], models[m][0].shape[3]
        if depth_maps == "exact":
            maps[b] = depth_map(grids[obj[b]].shape, pose[b], H, W, *PAD_EXTENT)
        else:
            lst = made.setdefault(m, [])
            if len(lst) < n_distinct_maps:
                lst.append(depth_map(grids[obj[b]].shape, pose[b], H, W, *PAD_EXTENT))
                maps[b] = lst[-1]
            else:
                maps[b] = lst[(b // P) % n_distinct_maps]
    sc = BatchScene(grids, np.ascontiguousarray(np.concatenate(pool).astype(np.float32)),
                    np.asarray(first, np.int64), np.asarray(count, np.int32), shapes, obj, layout, sensor, pose,
                    twist, k_n, k_d, k_t, mu, models, maps)
    sc.meta.update(E=E, P=P, n_layout=len(first), n_model=len(models), depth_maps=depth_maps)
    return sc


# ---------------------------------------------------------------------------
# Request streams for the server
# ---------------------------------------------------------------------------

@dataclass
class ServeWorkload:
    """Resident state (grids, sensor models, taxel-layout pool) and request templates.

    Each template is a dict with per-pad obj_id, layout, sensor, pad_pose, pad_twist,
    k_n, k_d, k_t, mu (float32 / int32 arrays), the packed depth maps of its pads with an
    image (pad order) and n_env."""
    grids: list
    models: list                      # [(coeffs [6][3][H][W], pitch_x, pitch_y)]
    taxels: np.ndarray                # pool [n_points][3]
    layout_first: np.ndarray
    layout_count: np.ndarray
    templates: list


def serve_workload(seed: int = 5, n_templates: int = 16, env_range=(1, 2048), P: int = 2, n_grid: int = 32,
                   grid_sides=(64, 256), res_y=(10, 40), res_x=(12, 50), width=(160, 640), n_size_class: int = 16,
                   maps_per_model: int = 2, vel_sigma: float = 0.05) -> ServeWorkload:
    """Requests of log-uniform env counts in env_range (P pads per env), each env drawing
    its pad resolution, object (from a resident pool of n_grid grids, sides log-uniform
    in grid_sides) and image size class as in scene_batch; every resolution in the
    res_y x res_x box is a resident layout.  Depth maps: maps_per_model heightfields per
    sensor model (of a pad indenting a pool object), handed out in turn."""
    g = rng(seed)
    grids = grid_pool(seed + 1, n_grid, *grid_sides)
    u = (np.arange(n_size_class) + g.random(n_size_class)) / n_size_class
    ws = np.exp(np.log(width[0]) + u * (np.log(width[1]) - np.log(width[0])))
    ws = np.maximum(4, 4 * np.rint(ws / 4.0).astype(np.int64))
    hs = np.maximum(4, 4 * np.rint(0.75 * ws / 4.0).astype(np.int64))
    models = []
    for c in range(n_size_class):
        H, W = int(hs[c]), int(ws[c])
        for p in range(P):
            co = shading_coeffs(1, H, W, seed * 1000 + P * c + p)[0]
            models.append((co, PAD_EXTENT[0] / W, PAD_EXTENT[1] / H))
    # every resolution of the box is resident
    keys = [(ny, nx) for ny in range(res_y[0], res_y[1] + 1) for nx in range(res_x[0], res_x[1] + 1)]
    index, pool, first, count = {}, [], [], []
    n_points = 0
    for key in keys:
        t = taxel_grid(key[0], key[1], PAD_EXTENT[0] / (key[1] - 1), PAD_EXTENT[1] / (key[0] - 1))
        index[key] = len(first)
        first.append(n_points)
        count.append(t.shape[0])
        pool.append(t)
        n_points += t.shape[0]
    maps = {}
    for m, (co, _, _) in enumerate(models):
        H, W = co.shape[2], co.shape[3]
        lst = []
        for k in range(maps_per_model):
            obj = int(g.integers(0, len(grids)))
            pose = place_pad(grids[obj].shape, random_quaternion(g), g.uniform(0.5e-3, 2e-3), g.uniform(-2e-3, 2e-3, 2))
            lst.append(depth_map(grids[obj].shape, pose, H, W, *PAD_EXTENT).reshape(-1))
        maps[m] = lst
    templates = []
    for _ in range(n_templates):
        E = int(log_uniform_int(g, env_range[0], env_range[1]))
        ny = log_uniform_int(g, res_y[0], res_y[1], size=E)
        nx = log_uniform_int(g, res_x[0], res_x[1], size=E)
        obj_env = g.integers(0, len(grids), size=E)
        cls_env = g.integers(0, n_size_class, size=E)
        n = E * P
        obj = np.repeat(obj_env, P).astype(np.int32)
        layout = np.repeat([index[(int(a), int(b))] for a, b in zip(ny, nx)], P).astype(np.int32)
        sensor = (P * np.repeat(cls_env, P) + np.tile(np.arange(P), E)).astype(np.int32)
        pose = np.zeros((n, 7), np.float32)
        twist = np.zeros((n, 6), np.float32)
        for b in range(n):
            pose[b] = place_pad(grids[obj[b]].shape, random_quaternion(g), g.uniform(-2e-3, 2e-3),
                                g.uniform(-2e-3, 2e-3, size=2))
            twist[b, :3] = g.normal(0.0, vel_sigma, size=3)
        k_n = np.repeat(g.uniform(0.5e4, 1.5e4, size=E), P).astype(np.float32)
        k_t = np.repeat(g.uniform(50.0, 150.0, size=E), P).astype(np.float32)
        mu = np.repeat(g.uniform(0.3, 0.7, size=E), P).astype(np.float32)
        dm = np.concatenate([maps[int(s)][b % maps_per_model] for b, s in enumerate(sensor)])
        templates.append(dict(n_env=E, obj_id=obj, layout=layout, sensor=sensor, pad_pose=pose, pad_twist=twist,
                              k_n=k_n, k_d=np.zeros(n, np.float32), k_t=k_t, mu=mu, depth_map=dm))
    return ServeWorkload(grids, models, np.ascontiguousarray(np.concatenate(pool).astype(np.float32)),
                         np.asarray(first, np.int64), np.asarray(count, np.int32), templates)
