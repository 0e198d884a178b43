"""Seeded synthetic scenes, camera walk-throughs and pixel samples.

This module only *makes inputs*: triangle/sphere arrays, per-primitive albedo,
a light, base cameras along a walk-through, and seeded pixel subsets. It holds
none of the rendering method's arithmetic (no camera displacement, no ray
tracing, no shading), so both the CUDA path and the FP64 oracle can be fed from
it without sharing any of the method's code.

The paper (Recursive Camera Painting, §6) renders textured "infinite sphere"
scenes and Unreal user scenes whose assets are not available. The procedural
scenes here stand in for them; they are shaped like the paper's street and
forest walk-throughs (Figs. 3-5): a terrain with box "buildings", and a forest
of cone-canopy trees. Sizes:

* ``tiny``   -- 3 spheres on a 2-triangle ground quad, point light.
* ``mid``    -- 256x256-quad fBm terrain (131,072 tris) + 200 boxes (2,400 tris).
* ``forest`` -- 181x181-quad ground (65,522 tris) + 2,000 trees x 500 tris.
* ``terrain_scene(grid)`` -- terrain + 200 boxes of a chosen grid size
  (221, 706, 1224, 1580 give 0.1M, 1M, 3M, 5M triangles).
* ``forest_scene(n_trees)`` -- the forest with any tree count (25,000 for the
  12.57M-triangle stress scene).

Arrays are float32, C-contiguous: ``tris`` (T, 9) = v0 v1 v2, ``spheres``
(S, 4) = centre, radius, ``albedo`` (T+S, 3) with triangles first. Primitive
ids are 0..T-1 for triangles and T..T+S-1 for spheres.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

LIGHT_POINT = 0
LIGHT_DIRECTIONAL = 1


@dataclass
class Camera:
    """Base pinhole camera: eye, look-at point, up vector, vertical FOV (deg)."""

    eye: tuple
    look_at: tuple
    up: tuple = (0.0, 1.0, 0.0)
    fov_y_deg: float = 60.0

    def as_array(self) -> np.ndarray:
        return np.array([*self.eye, *self.look_at, *self.up, self.fov_y_deg], dtype=np.float64)


@dataclass
class Light:
    type: int
    v: tuple  # point: position; directional: unit direction towards the light
    ambient: float = 0.1


@dataclass
class Scene:
    name: str
    tris: np.ndarray  # (T, 9) float32
    spheres: np.ndarray  # (S, 4) float32
    albedo: np.ndarray  # (T+S, 3) float32
    light: Light
    poses: list = field(default_factory=list)  # list[Camera]
    sway_amp: np.ndarray | None = None  # (T, 3) per triangle-vertex sway amplitude (forest)
    sway_phase: np.ndarray | None = None  # (T,) per triangle sway phase (forest)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_spheres(self) -> int:
        return int(self.spheres.shape[0])

    @property
    def n_prims(self) -> int:
        return self.n_tris + self.n_spheres

    def diameter(self) -> float:
        """Diagonal of the axis-aligned box around every primitive.

        Used by the workload definitions to scale the displacement strength k
        and the focal distance f (e.g. k = 0.05 * diameter)."""
        lo = np.full(3, np.inf)
        hi = np.full(3, -np.inf)
        if self.n_tris:
            v = self.tris.reshape(-1, 3).astype(np.float64)
            lo = np.minimum(lo, v.min(0))
            hi = np.maximum(hi, v.max(0))
        if self.n_spheres:
            s = self.spheres.astype(np.float64)
            lo = np.minimum(lo, (s[:, :3] - s[:, 3:4]).min(0))
            hi = np.maximum(hi, (s[:, :3] + s[:, 3:4]).max(0))
        if not np.all(np.isfinite(lo)):
            return 0.0
        return float(np.linalg.norm(hi - lo))


# --------------------------------------------------------------------------
# procedural building blocks
# --------------------------------------------------------------------------

def _smoothstep(t):
    return t * t * (3.0 - 2.0 * t)


class ValueNoiseFBM:
    """fBm of seeded lattice value noise with smoothstep interpolation.

    ``octaves`` layers; octave o has ``base_freq * lacunarity**o`` cycles over
    ``extent`` world units and weight ``gain**o``; the sum is scaled by
    ``amplitude``. Lattice values are uniform in [-1, 1]."""

    def __init__(self, rng, extent, octaves=5, base_freq=4.0, lacunarity=2.0, gain=0.5, amplitude=20.0):
        self.extent = float(extent)
        self.layers = []
        for o in range(octaves):
            cycles = base_freq * lacunarity ** o
            n = int(np.ceil(cycles)) + 2
            lattice = rng.uniform(-1.0, 1.0, size=(n, n))
            self.layers.append((cycles, gain ** o, lattice))
        self.amplitude = float(amplitude)

    def __call__(self, x, z, x0, z0):
        """Height at world (x, z); (x0, z0) is the terrain's min corner."""
        x = np.asarray(x, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        h = np.zeros(np.broadcast(x, z).shape)
        for cycles, w, lat in self.layers:
            fx = (x - x0) / self.extent * cycles
            fz = (z - z0) / self.extent * cycles
            ix = np.clip(np.floor(fx).astype(np.int64), 0, lat.shape[0] - 2)
            iz = np.clip(np.floor(fz).astype(np.int64), 0, lat.shape[1] - 2)
            tx = _smoothstep(np.clip(fx - ix, 0.0, 1.0))
            tz = _smoothstep(np.clip(fz - iz, 0.0, 1.0))
            a = lat[ix, iz] * (1 - tx) + lat[ix + 1, iz] * tx
            b = lat[ix, iz + 1] * (1 - tx) + lat[ix + 1, iz + 1] * tx
            h += w * (a * (1 - tz) + b * tz)
        return self.amplitude * h


def _grid_mesh(n, lo, hi, height_fn):
    """n x n quads over [lo, hi]^2 in x/z, two triangles per quad, y from height_fn."""
    xs = np.linspace(lo, hi, n + 1)
    X, Z = np.meshgrid(xs, xs, indexing="ij")
    Y = height_fn(X, Z)
    V = np.stack([X, Y, Z], axis=-1)  # (n+1, n+1, 3)
    v00 = V[:-1, :-1].reshape(-1, 3)
    v10 = V[1:, :-1].reshape(-1, 3)
    v11 = V[1:, 1:].reshape(-1, 3)
    v01 = V[:-1, 1:].reshape(-1, 3)
    t1 = np.concatenate([v00, v10, v11], axis=1)
    t2 = np.concatenate([v00, v11, v01], axis=1)
    tris = np.empty((2 * n * n, 9))
    tris[0::2] = t1
    tris[1::2] = t2
    return tris


def _box_tris(cx, cz, sx, sz, y0, y1):
    """12 triangles of an axis-aligned box with footprint centred on (cx, cz)."""
    x0, x1 = cx - sx / 2, cx + sx / 2
    z0, z1 = cz - sz / 2, cz + sz / 2
    c = np.array([
        [x0, y0, z0], [x1, y0, z0], [x1, y0, z1], [x0, y0, z1],
        [x0, y1, z0], [x1, y1, z0], [x1, y1, z1], [x0, y1, z1],
    ])
    faces = [
        (0, 2, 1), (0, 3, 2),  # bottom
        (4, 5, 6), (4, 6, 7),  # top
        (0, 1, 5), (0, 5, 4),  # z0 side
        (3, 7, 6), (3, 6, 2),  # z1 side
        (0, 4, 7), (0, 7, 3),  # x0 side
        (1, 2, 6), (1, 6, 5),  # x1 side
    ]
    return np.array([np.concatenate([c[a], c[b], c[d]]) for a, b, d in faces])


def _tree_template(cone_segments=200, trunk_segments=50):
    """Unit tree (scale 1, base at the origin).

    Canopy: cone of radius 2, height 6, base at y=2 -> 200 side + 200 base
    triangles. Trunk: open cylinder radius 0.3, height 2 -> 100 side triangles.
    Returns (canopy_tris (400, 9), trunk_tris (100, 9))."""
    a = np.linspace(0.0, 2 * np.pi, cone_segments + 1)
    ring = np.stack([2.0 * np.cos(a), np.full_like(a, 2.0), 2.0 * np.sin(a)], axis=1)
    apex = np.array([0.0, 8.0, 0.0])
    centre = np.array([0.0, 2.0, 0.0])
    side = np.concatenate([ring[:-1], ring[1:], np.broadcast_to(apex, (cone_segments, 3))], axis=1)
    base = np.concatenate([ring[1:], ring[:-1], np.broadcast_to(centre, (cone_segments, 3))], axis=1)
    canopy = np.concatenate([side, base], axis=0)
    b = np.linspace(0.0, 2 * np.pi, trunk_segments + 1)
    lo = np.stack([0.3 * np.cos(b), np.zeros_like(b), 0.3 * np.sin(b)], axis=1)
    hi = lo + np.array([0.0, 2.0, 0.0])
    t1 = np.concatenate([lo[:-1], lo[1:], hi[1:]], axis=1)
    t2 = np.concatenate([lo[:-1], hi[1:], hi[:-1]], axis=1)
    trunk = np.empty((2 * trunk_segments, 9))
    trunk[0::2] = t1
    trunk[1::2] = t2
    return canopy, trunk


def catmull_rom_centripetal(points, n_samples):
    """Samples uniform in the parameter of a centripetal (alpha = 0.5)
    Catmull-Rom spline through ``points`` (the first and last point only
    shape the end segments). Returns (positions (n,2), tangents (n,2))."""
    P = np.asarray(points, dtype=np.float64)
    nseg = len(P) - 3
    pos = np.empty((n_samples, P.shape[1]))
    tan = np.empty((n_samples, P.shape[1]))
    for i in range(n_samples):
        s = nseg * i / n_samples
        j = min(int(s), nseg - 1)
        u = s - j
        p0, p1, p2, p3 = P[j:j + 4]
        t0 = 0.0
        t1 = t0 + np.linalg.norm(p1 - p0) ** 0.5
        t2 = t1 + np.linalg.norm(p2 - p1) ** 0.5
        t3 = t2 + np.linalg.norm(p3 - p2) ** 0.5

        def curve(t):
            a1 = (t1 - t) / (t1 - t0) * p0 + (t - t0) / (t1 - t0) * p1
            a2 = (t2 - t) / (t2 - t1) * p1 + (t - t1) / (t2 - t1) * p2
            a3 = (t3 - t) / (t3 - t2) * p2 + (t - t2) / (t3 - t2) * p3
            b1 = (t2 - t) / (t2 - t0) * a1 + (t - t0) / (t2 - t0) * a2
            b2 = (t3 - t) / (t3 - t1) * a2 + (t - t1) / (t3 - t1) * a3
            return (t2 - t) / (t2 - t1) * b1 + (t - t1) / (t2 - t1) * b2

        t = t1 + u * (t2 - t1)
        h = 1e-4 * (t2 - t1)
        pos[i] = curve(t)
        d = curve(t + h) - curve(t - h)
        tan[i] = d / max(np.linalg.norm(d), 1e-12)
    return pos, tan


def _walkthrough(rng, height_fn, span, n_poses=64, eye_height=2.0, pitch_deg=-10.0, fov=60.0):
    ctrl = rng.uniform(-span, span, size=(8, 2))
    pos, tan = catmull_rom_centripetal(ctrl, n_poses)
    pitch = np.deg2rad(pitch_deg)
    poses = []
    for (x, z), (tx, tz) in zip(pos, tan):
        y = float(height_fn(np.array(x), np.array(z))) + eye_height
        fwd = np.array([np.cos(pitch) * tx, np.sin(pitch), np.cos(pitch) * tz])
        eye = np.array([x, y, z])
        poses.append(Camera(tuple(eye.tolist()), tuple((eye + fwd).tolist()), (0.0, 1.0, 0.0), fov))
    return poses


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def tiny_scene(seed: int = 1) -> Scene:
    """3 unit spheres (centres U([-3,3]x[1,2]x[-3,3]), albedo U[0.2,0.9]^3) on a
    2-triangle ground quad [-10,10]^2 at y=0 (albedo 0.5), point light at
    (5,8,5); camera eye (0,3,10) looking at (0,1,0), FOV 60 degrees."""
    rng = np.random.default_rng(seed)
    centres = np.stack([rng.uniform(-3, 3, 3), rng.uniform(1, 2, 3), rng.uniform(-3, 3, 3)], axis=1)
    spheres = np.concatenate([centres, np.ones((3, 1))], axis=1)
    sph_albedo = rng.uniform(0.2, 0.9, size=(3, 3))
    g = 10.0
    tris = np.array([
        [-g, 0, -g, g, 0, g, g, 0, -g],
        [-g, 0, -g, -g, 0, g, g, 0, g],
    ])
    albedo = np.concatenate([np.full((2, 3), 0.5), sph_albedo], axis=0)
    cam = Camera((0.0, 3.0, 10.0), (0.0, 1.0, 0.0), (0.0, 1.0, 0.0), 60.0)
    return Scene("tiny", _f32(tris), _f32(spheres), _f32(albedo),
                 Light(LIGHT_POINT, (5.0, 8.0, 5.0), 0.1), [cam])


def terrain_scene(grid: int = 256, seed: int = 2, n_boxes: int = 200, n_poses: int = 64) -> Scene:
    """fBm terrain of grid x grid unit quads centred on the origin (5 octaves,
    4 base cycles over the extent, lacunarity 2, gain 0.5, amplitude 20) plus
    ``n_boxes`` boxes (footprint U[2,8]^2, height U[5,30], base at the lowest
    terrain height under the footprint); per-triangle albedo U[0.1,0.9]^3;
    directional light towards normalize(0.4, 0.8, 0.3); a 64-pose walk-through
    2 units above the terrain with -10 degree pitch."""
    rng = np.random.default_rng(seed)
    half = grid / 2.0
    fbm = ValueNoiseFBM(rng, extent=grid, octaves=5, base_freq=4.0, lacunarity=2.0, gain=0.5, amplitude=20.0)

    def height(x, z):
        return fbm(x, z, -half, -half)

    ground = _grid_mesh(grid, -half, half, height)
    boxes = []
    margin = 8.0
    for _ in range(n_boxes):
        cx, cz = rng.uniform(-half + margin, half - margin, 2)
        sx, sz = rng.uniform(2.0, 8.0, 2)
        hgt = rng.uniform(5.0, 30.0)
        xs = np.array([cx - sx / 2, cx + sx / 2, cx - sx / 2, cx + sx / 2, cx])
        zs = np.array([cz - sz / 2, cz - sz / 2, cz + sz / 2, cz + sz / 2, cz])
        y0 = float(np.min(height(xs, zs)))
        boxes.append(_box_tris(cx, cz, sx, sz, y0, y0 + hgt))
    tris = np.concatenate([ground] + boxes, axis=0)
    albedo = rng.uniform(0.1, 0.9, size=(tris.shape[0], 3))
    d = np.array([0.4, 0.8, 0.3])
    d /= np.linalg.norm(d)
    poses = _walkthrough(rng, height, span=0.75 * half, n_poses=n_poses)
    return Scene(f"terrain{grid}", _f32(tris), np.zeros((0, 4), np.float32), _f32(albedo),
                 Light(LIGHT_DIRECTIONAL, tuple(d.tolist()), 0.1), poses)


def mid_scene(seed: int = 2) -> Scene:
    """The 133,472-triangle street-like terrain (256 x 256 grid + 200 boxes)."""
    s = terrain_scene(256, seed)
    s.name = "mid"
    return s


def forest_scene(n_trees: int = 2000, seed: int = 3, extent: float | None = None,
                 n_poses: int = 64) -> Scene:
    """Ground of 181 x 181 quads (fBm amplitude 5) plus ``n_trees`` trees at
    seeded positions with scale U[0.7,1.3]. Each tree: a 400-triangle cone
    canopy (radius 2s, height 6s, base 2s above the ground) and a 100-triangle
    cylinder trunk (radius 0.3s, height 2s). Canopy albedo per tree
    U([0.05,0.2]x[0.3,0.7]x[0.05,0.2]), trunk U([0.3,0.5]x[0.2,0.3]x[0.1,0.15]).
    The ground spans [-200,200]^2 for 2,000 trees and grows with sqrt(n_trees)
    to keep the tree density. Walk-through eye 1 unit above the ground."""
    rng = np.random.default_rng(seed)
    if extent is None:
        extent = 400.0 * np.sqrt(max(n_trees, 1) / 2000.0)
    half = extent / 2.0
    fbm = ValueNoiseFBM(rng, extent=extent, octaves=5, base_freq=4.0, lacunarity=2.0, gain=0.5, amplitude=5.0)

    def height(x, z):
        return fbm(x, z, -half, -half)

    ground = _grid_mesh(181, -half, half, height)
    canopy, trunk = _tree_template()
    px = rng.uniform(-half * 0.95, half * 0.95, n_trees)
    pz = rng.uniform(-half * 0.95, half * 0.95, n_trees)
    sc = rng.uniform(0.7, 1.3, n_trees)
    base_y = height(px, pz)
    off = np.stack([px, base_y, pz], axis=1)  # (n, 3)
    tree = np.concatenate([canopy, trunk], axis=0).reshape(1, -1, 3, 3)  # (1, 500, 3, 3)
    verts = tree * sc.reshape(-1, 1, 1, 1) + off.reshape(-1, 1, 1, 3)
    tree_tris = verts.reshape(n_trees * 500, 9)
    can_alb = np.stack([rng.uniform(0.05, 0.2, n_trees), rng.uniform(0.3, 0.7, n_trees),
                        rng.uniform(0.05, 0.2, n_trees)], axis=1)
    trk_alb = np.stack([rng.uniform(0.3, 0.5, n_trees), rng.uniform(0.2, 0.3, n_trees),
                        rng.uniform(0.1, 0.15, n_trees)], axis=1)
    tree_alb = np.concatenate([np.repeat(can_alb[:, None, :], 400, axis=1),
                               np.repeat(trk_alb[:, None, :], 100, axis=1)], axis=1).reshape(-1, 3)
    ground_alb = rng.uniform(0.2, 0.5, size=(ground.shape[0], 3)) * np.array([0.8, 0.7, 0.4])
    tris = np.concatenate([ground, tree_tris], axis=0)
    albedo = np.concatenate([ground_alb, tree_alb], axis=0)
    d = np.array([0.4, 0.8, 0.3])
    d /= np.linalg.norm(d)
    poses = _walkthrough(rng, height, span=0.75 * half, n_poses=n_poses, eye_height=1.0, pitch_deg=-5.0)
    sc = Scene(f"forest{n_trees}", _f32(tris), np.zeros((0, 4), np.float32), _f32(albedo),
               Light(LIGHT_DIRECTIONAL, tuple(d.tolist()), 0.1), poses)
    # wind sway inputs: per triangle-vertex amplitude A * h_v / h_tree = 0.02 * h_v
    # (h_v = height above the tree's base; the ground does not move) and a
    # seeded phase per tree
    vert_h = (verts[..., 1] - base_y.reshape(-1, 1, 1)).reshape(n_trees * 500, 3)
    phase = rng.uniform(0.0, 2.0 * np.pi, n_trees)
    sc.sway_amp = _f32(np.concatenate([np.zeros((ground.shape[0], 3)), 0.02 * vert_h], axis=0))
    sc.sway_phase = _f32(np.concatenate([np.zeros(ground.shape[0]), np.repeat(phase, 500)]))
    return sc


def sway_vertices(base_tris, sway_amp, sway_phase, frame, fps=60.0, freq=0.5):
    """Wind sway of frame `frame` (numpy reference of the stress workload):
    x += a sin(2 pi f t + phi), z += a cos(2 pi f t + phi), t = frame / fps."""
    t = frame / fps
    ang = 2.0 * np.pi * freq * t + sway_phase.astype(np.float64)
    v = base_tris.reshape(-1, 3, 3).astype(np.float64).copy()
    v[:, :, 0] += sway_amp * np.sin(ang)[:, None]
    v[:, :, 2] += sway_amp * np.cos(ang)[:, None]
    return _f32(v.reshape(-1, 9))


def random_soup(n_tris: int, n_spheres: int = 0, seed: int = 0, extent: float = 10.0,
                tri_size: float = 1.0) -> Scene:
    """Random triangles and spheres in a cube (for builder and traversal tests)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(-extent, extent, size=(n_tris, 1, 3))
    v = c + rng.normal(0.0, tri_size, size=(n_tris, 3, 3))
    sph = np.concatenate([rng.uniform(-extent, extent, size=(n_spheres, 3)),
                          rng.uniform(0.2, 1.5, size=(n_spheres, 1))], axis=1)
    alb = rng.uniform(0.1, 0.9, size=(n_tris + n_spheres, 3))
    cam = Camera((0.0, 0.5 * extent, 3.0 * extent), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 60.0)
    return Scene(f"soup{n_tris}_{n_spheres}", _f32(v.reshape(n_tris, 9)), _f32(sph.reshape(n_spheres, 4)),
                 _f32(alb), Light(LIGHT_POINT, (extent, 3 * extent, extent), 0.1), [cam])


def blocks_scene(n: int = 32, n_cubes: int = 200, seed: int = 6,
                 offset: tuple = (0.0, 0.0, 0.0)) -> Scene:
    """Axis-aligned geometry on integer coordinates (for traversal edge cases):
    a flat n x n grid of unit quads at y = 0, each split into two triangles
    along the diagonal from (x, z) to (x+1, z+1), and unit cubes (12 triangles)
    on seeded grid cells, stacked up to 3 high. Every vertex coordinate is an
    integer plus `offset`, so boxes are flat or share faces exactly."""
    rng = np.random.default_rng(seed)
    tris = []
    for x in range(n):
        for z in range(n):
            a, b, c, d = (x, 0, z), (x + 1, 0, z), (x + 1, 0, z + 1), (x, 0, z + 1)
            tris += [a + c + b, a + d + c]
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], np.float64)
    faces = [(0, 1, 3, 2), (4, 6, 7, 5), (0, 4, 5, 1), (2, 3, 7, 6), (0, 2, 6, 4), (1, 5, 7, 3)]
    cells = rng.integers(0, n, size=(n_cubes, 2))
    heights = rng.integers(1, 4, size=n_cubes)
    for (cx, cz), h in zip(cells, heights):
        for level in range(int(h)):
            base = np.array([cx, level, cz], np.float64)
            for f in faces:
                q = [tuple(corners[i] + base) for i in f]
                tris += [q[0] + q[1] + q[2], q[0] + q[2] + q[3]]
    t = np.asarray(tris, np.float64) + np.tile(np.asarray(offset, np.float64), 3)
    alb = rng.uniform(0.1, 0.9, size=(len(t), 3))
    c = np.asarray(offset, np.float64) + np.array([n / 2, 0.0, n / 2])
    cam = Camera(tuple(c + np.array([0.0, n / 2, 1.5 * n])), tuple(c), (0.0, 1.0, 0.0), 60.0)
    d = np.array([0.4, 0.8, 0.3]) / np.linalg.norm([0.4, 0.8, 0.3])
    return Scene(f"blocks{n}_{n_cubes}", _f32(t), np.zeros((0, 4), np.float32), _f32(alb),
                 Light(LIGHT_DIRECTIONAL, tuple(d.tolist()), 0.1), [cam])


# --------------------------------------------------------------------------
# view sets and samples
# --------------------------------------------------------------------------

def batched_view_sizes(n_views: int = 64, seed: int = 3):
    """Uneven view sizes: W uniform in [256, 1920], H uniform in [256, 1080]."""
    rng = np.random.default_rng(seed + 1000)
    W = rng.integers(256, 1921, n_views)
    H = rng.integers(256, 1081, n_views)
    return [(int(w), int(h)) for w, h in zip(W, H)]


def pixel_subset(width: int, height: int, n: int, seed: int) -> np.ndarray:
    """Seeded sorted sample of distinct pixel indices (row-major y*W + x)."""
    P = width * height
    rng = np.random.default_rng(seed)
    if n >= P:
        return np.arange(P, dtype=np.int64)
    return np.sort(rng.choice(P, size=n, replace=False)).astype(np.int64)


def served_requests(n: int, n_scenes: int, n_poses: int, seed: int = 4):
    """Request mix: scene index, pose index, resolution, K in 1..8, k fraction in [0, 0.05]."""
    rng = np.random.default_rng(seed)
    res = [(1280, 720), (1920, 1080), (2560, 1440), (3840, 2160)]
    out = []
    for _ in range(n):
        w, h = res[int(rng.integers(0, 4))]
        out.append(dict(scene=int(rng.integers(0, n_scenes)), pose=int(rng.integers(0, n_poses)),
                        width=w, height=h, K=int(rng.integers(1, 9)), k_frac=float(rng.uniform(0.0, 0.05))))
    return out


def poisson_arrivals(rate: float, n: int, seed: int = 4) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed + int(rate * 1000))
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
