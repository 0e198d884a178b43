"""Pins for the FP64 oracle: facts fixed by the paper or by plain geometry.

Each ``check_*`` raises AssertionError on a wrong oracle. They take the path of
an oracle build so that ``test_oracle_mutants`` can run them against copies of
the oracle with a planted mistake and show that every mistake is caught.

None of these retypes the oracle's formulas: they use closed forms of the
pinhole geometry, a textbook quadratic or a linear solve, symmetries, and the
properties the paper states (§3: I_0 = 0.5 gives an ordinary ray-traced image,
mid-grey does not move rays, R moves right and G moves up in the camera frame).
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O

# camera looking down -z with +y up: right = +x, up = +y, forward = -z
CAM_Z = np.array([0.0, 0.0, 0.0, 0.0, 0.0, -1.0, 0.0, 1.0, 0.0, 60.0])


def _ray(cam, W, H, x, y, mapping, k, f, c=(0.5, 0.5, 0.5), z=0.0, z0=0.0, n=None, lp=None):
    o, d, _ = O.camera_ray(cam, W, H, x, y, mapping, k, f, c, z, z0, n=n, libpath=lp)
    return o, d


def _angle(a, b):
    return math.acos(max(-1.0, min(1.0, float(np.dot(a, b) / np.linalg.norm(a) / np.linalg.norm(b)))))


def _line_dist(p, o, d):
    w = p - o
    return float(np.linalg.norm(w - np.dot(w, d) * d))


# --------------------------------------------------------------------------- camera

def check_camera_centre(lp=None):
    """Odd W, H: the centre pixel looks exactly along look_at - eye."""
    cam = np.array([1.0, 2.0, 3.0, -4.0, 0.5, -2.0, 0.0, 1.0, 0.0, 50.0])
    fwd = cam[3:6] - cam[:3]
    fwd /= np.linalg.norm(fwd)
    for W, H in [(129, 65), (7, 7), (1, 1)]:
        for m in (O.MAP_EYE, O.MAP_TARGET):
            o, d = _ray(cam, W, H, W // 2, H // 2, m, 0.7, 3.0, lp=lp)
            assert np.allclose(d, fwd, atol=1e-14), (W, H, m, d, fwd)
            assert np.allclose(o, cam[:3], atol=1e-14)


def check_camera_fov(lp=None):
    """Pinhole angles: rays through the centres of the first and last row
    (column W//2) span 2 atan(tan(fov/2) (H-1)/H); first/last column (row H//2)
    span 2 atan(tan(fov/2) (W/H) (W-1)/W)."""
    for fov, W, H in [(60.0, 65, 33), (90.0, 129, 129), (30.0, 201, 101)]:
        cam = CAM_Z.copy()
        cam[9] = fov
        t = math.tan(math.radians(fov) / 2)
        _, dt = _ray(cam, W, H, W // 2, 0, O.MAP_EYE, 0.0, 1.0, lp=lp)
        _, db = _ray(cam, W, H, W // 2, H - 1, O.MAP_EYE, 0.0, 1.0, lp=lp)
        assert abs(_angle(dt, db) - 2 * math.atan(t * (H - 1) / H)) < 1e-12
        _, dl = _ray(cam, W, H, 0, H // 2, O.MAP_EYE, 0.0, 1.0, lp=lp)
        _, dr = _ray(cam, W, H, W - 1, H // 2, O.MAP_EYE, 0.0, 1.0, lp=lp)
        assert abs(_angle(dl, dr) - 2 * math.atan(t * (W / H) * (W - 1) / W)) < 1e-12


def check_camera_orientation(lp=None):
    """Row 0 is the top of the image and column W-1 its right side: for a
    camera looking down -z with +y up, the top-right pixel's ray has x > 0,
    y > 0; mirror pixels give mirrored rays."""
    W, H = 40, 30
    _, d = _ray(CAM_Z, W, H, W - 1, 0, O.MAP_EYE, 0.0, 1.0, lp=lp)
    assert d[0] > 0 and d[1] > 0 and d[2] < 0
    for x, y in [(3, 4), (0, 0), (17, 29)]:
        _, a = _ray(CAM_Z, W, H, x, y, O.MAP_EYE, 0.0, 1.0, lp=lp)
        _, b = _ray(CAM_Z, W, H, W - 1 - x, y, O.MAP_EYE, 0.0, 1.0, lp=lp)
        _, c = _ray(CAM_Z, W, H, x, H - 1 - y, O.MAP_EYE, 0.0, 1.0, lp=lp)
        assert np.allclose(a * [-1, 1, 1], b, atol=1e-15)
        assert np.allclose(a * [1, -1, 1], c, atol=1e-15)


def check_eye_mapping(lp=None):
    """EYE mapping: the eye moves by k (2c-1) along (right, up, forward) =
    (+x, +y, -z) here, and every ray still passes through the pixel's point on
    the focal plane z = -f (the point the undisplaced ray reaches there)."""
    W, H, k, f = 33, 21, 0.8, 5.0
    cases = {(1.0, 0.5, 0.5): (k, 0, 0), (0.5, 1.0, 0.5): (0, k, 0), (0.5, 0.5, 1.0): (0, 0, -k),
             (0.0, 0.0, 0.0): (-k, -k, k), (0.25, 0.75, 0.5): (-k / 2, k / 2, 0)}
    for c, off in cases.items():
        for x, y in [(0, 0), (16, 10), (32, 20), (5, 17)]:
            o, d = _ray(CAM_Z, W, H, x, y, O.MAP_EYE, k, f, c, lp=lp)
            assert np.allclose(o, off, atol=1e-14), (c, o, off)
            o0, d0 = _ray(CAM_Z, W, H, x, y, O.MAP_EYE, 0.0, f, lp=lp)
            P = o0 + d0 * (f / -d0[2])  # where the pinhole ray meets z = -f
            assert _line_dist(P, o, d) < 1e-12
            assert abs(np.linalg.norm(d) - 1) < 1e-15


def check_target_mapping(lp=None):
    """TARGET mapping (§3): with k equal to the focal-plane pixel pitch, R = 1
    moves a pixel's ray onto its right neighbour's, R = 0 onto the left one's,
    G = 1 onto the one above (row y-1) and G = 0 below; blue moves the target
    along the view axis only."""
    W, H, f = 31, 23, 4.0
    pitch = f * 2 * math.tan(math.radians(30.0)) / H
    for x, y in [(10, 10), (1, 1), (29, 21)]:
        for c, (dx, dy) in {(1.0, 0.5, 0.5): (1, 0), (0.0, 0.5, 0.5): (-1, 0),
                            (0.5, 1.0, 0.5): (0, -1), (0.5, 0.0, 0.5): (0, 1)}.items():
            o, d = _ray(CAM_Z, W, H, x, y, O.MAP_TARGET, pitch, f, c, lp=lp)
            o2, d2 = _ray(CAM_Z, W, H, x + dx, y + dy, O.MAP_TARGET, 0.0, f, lp=lp)
            assert np.allclose(o, [0, 0, 0], atol=1e-15)
            assert np.allclose(d, d2, atol=1e-13), (x, y, c)
    o, d = _ray(CAM_Z, W, H, W // 2, H // 2, O.MAP_TARGET, 0.3, f, (0.5, 0.5, 1.0), lp=lp)
    assert np.allclose(d, [0, 0, -1], atol=1e-15)


def check_grey_and_zero_k(lp=None):
    """Mid-grey does not move rays (§3), k = 0 moves nothing, and the centre
    ray of the EYE mapping stays on the axis for pure-blue colours."""
    W, H = 25, 19
    for m in (O.MAP_EYE, O.MAP_TARGET, O.MAP_DEPTH):
        for x, y in [(0, 0), (12, 9), (24, 18)]:
            o0, d0 = _ray(CAM_Z, W, H, x, y, m, 0.0, 3.0, (0.9, 0.1, 0.3), z=2.0, lp=lp)
            o1, d1 = _ray(CAM_Z, W, H, x, y, m, 1.5, 3.0, (0.5, 0.5, 0.5), z=2.0, lp=lp)
            o2, d2 = _ray(CAM_Z, W, H, x, y, m, 0.0, 3.0, lp=lp)
            assert np.array_equal(o0, o2) and np.array_equal(d0, d2)
            assert np.array_equal(o1, o2) and np.array_equal(d1, d2)
    for c in [(0.5, 0.5, 1.0), (0.5, 0.5, 0.0)]:
        _, d = _ray(CAM_Z, W, H, W // 2, H // 2, O.MAP_EYE, 0.9, 3.0, c, lp=lp)
        assert np.allclose(d, [0, 0, -1], atol=1e-15)


def check_depth_mapping(lp=None):
    """Depth mapping (§4): |z - z0| scales the TARGET displacement."""
    W, H, f = 21, 21, 3.0
    for c in [(1.0, 0.2, 0.7), (0.1, 0.9, 0.4)]:
        for z, z0, mul in [(5.0, 5.0, 0.0), (6.0, 5.0, 1.0), (1.0, 3.0, 2.0)]:
            _, d = _ray(CAM_Z, W, H, 4, 7, O.MAP_DEPTH, 0.25, f, c, z=z, z0=z0, lp=lp)
            _, e = _ray(CAM_Z, W, H, 4, 7, O.MAP_TARGET, 0.25 * mul, f, c, lp=lp)
            assert np.allclose(d, e, atol=1e-15)


# --------------------------------------------------------------------------- primitives

def check_triangle_closed_forms(lp=None):
    v0, v1, v2 = [0, 0, 0], [1, 0, 0], [0, 1, 0]
    assert abs(O.hit_triangle(v0, v1, v2, [0.25, 0.25, 1], [0, 0, -1], libpath=lp) - 1.0) < 1e-15
    assert abs(O.hit_triangle(v0, v1, v2, [0.5, 0.5, 2], [0, 0, -1], libpath=lp) - 2.0) < 1e-15  # on an edge
    assert abs(O.hit_triangle(v0, v1, v2, [0, 0, 3], [0, 0, -1], libpath=lp) - 3.0) < 1e-15  # on a vertex
    assert O.hit_triangle(v0, v1, v2, [0.6, 0.6, 1], [0, 0, -1], libpath=lp) is None
    assert O.hit_triangle(v0, v1, v2, [-0.01, 0.5, 1], [0, 0, -1], libpath=lp) is None
    assert O.hit_triangle(v0, v1, v2, [0.25, 0.25, -1], [0, 0, -1], libpath=lp) is None  # behind
    assert O.hit_triangle(v0, v1, v2, [0.25, 0.25, 1], [0, 0, -1], tmin=1.5, libpath=lp) is None
    assert O.hit_triangle(v0, v1, v2, [0.25, 0.25, 1], [0, 0, -1], tmax=0.5, libpath=lp) is None
    assert O.hit_triangle(v0, v1, v2, [-1, 0.2, 0], [1, 0, 0], libpath=lp) is None  # in-plane
    assert O.hit_triangle([0, 0, 0], [1, 1, 1], [2, 2, 2], [1, 1, 5], [0, 0, -1], libpath=lp) is None
    # random rays: t from a 3x3 linear solve of o + t d = v0 + a e1 + b e2
    rng = np.random.default_rng(7)
    n_hit = 0
    for _ in range(300):
        V = rng.normal(size=(3, 3))
        o = rng.normal(size=3) * 3
        target = V[0] + rng.uniform(-0.3, 1.0) * (V[1] - V[0]) + rng.uniform(-0.3, 1.0) * (V[2] - V[0])
        d = target - o
        d /= np.linalg.norm(d)
        A = np.stack([-d, V[1] - V[0], V[2] - V[0]], axis=1)
        t, a, b = np.linalg.solve(A, o - V[0])
        inside = a >= 0 and b >= 0 and a + b <= 1 and t > 0
        got = O.hit_triangle(V[0], V[1], V[2], o, d, libpath=lp)
        if min(a, b, 1 - a - b) > 1e-9 or min(a, b, 1 - a - b) < -1e-9:
            assert (got is not None) == inside, (a, b, t)
        if got is not None and inside:
            assert abs(got - t) < 1e-9 * max(1, abs(t))
            n_hit += 1
    assert n_hit > 50


def check_sphere_closed_forms(lp=None):
    c0 = [0, 0, 0]
    assert abs(O.hit_sphere(c0, 1.0, [0, 0, 10], [0, 0, -1], libpath=lp) - 9.0) < 1e-14
    assert abs(O.hit_sphere(c0, 1.0, [0, 0, 0], [0, 0, -1], libpath=lp) - 1.0) < 1e-14  # from inside
    assert abs(O.hit_sphere(c0, 1.0, [1, 0, 10], [0, 0, -1], libpath=lp) - 10.0) < 1e-14  # tangent
    assert O.hit_sphere(c0, 1.0, [1.01, 0, 10], [0, 0, -1], libpath=lp) is None
    assert O.hit_sphere(c0, 1.0, [0, 0, -10], [0, 0, -1], libpath=lp) is None  # behind
    assert abs(O.hit_sphere(c0, 1.0, [0, 0, 10], [0, 0, -1], tmin=9.5, libpath=lp) - 11.0) < 1e-14
    rng = np.random.default_rng(11)
    n_hit = 0
    for _ in range(300):
        c = rng.normal(size=3)
        r = rng.uniform(0.2, 2.0)
        o = rng.normal(size=3) * 4
        d = c + rng.normal(size=3) * r - o
        d /= np.linalg.norm(d)
        # |o + t d - c|^2 = r^2  ->  t^2 + 2 (d.(o-c)) t + |o-c|^2 - r^2 = 0
        roots = np.roots([1.0, 2 * np.dot(d, o - c), np.dot(o - c, o - c) - r * r])
        roots = sorted(float(x.real) for x in roots if abs(x.imag) < 1e-12 and x.real > 0)
        got = O.hit_sphere(c, r, o, d, libpath=lp)
        if roots:
            assert got is not None and abs(got - roots[0]) < 1e-8 * max(1, roots[0])
            n_hit += 1
        else:
            assert got is None
    assert n_hit > 50


# --------------------------------------------------------------------------- shading

def _scene(tris=(), spheres=(), albedo=(), light_type=O.LIGHT_DIRECTIONAL, light=(0, 1, 0), ambient=0.1, lp=None):
    t = np.array(tris, dtype=np.float32).reshape(-1, 9)
    s = np.array(spheres, dtype=np.float32).reshape(-1, 4)
    a = np.array(albedo, dtype=np.float32).reshape(-1, 3)
    return O.OracleScene(t, s, a, light_type, light, ambient, libpath=lp)


GROUND = [[-10, 0, -10, 10, 0, 10, 10, 0, -10], [-10, 0, -10, -10, 0, 10, 10, 0, 10]]


def check_lambert_and_shadow(lp=None):
    """Lambert + ambient with an unoccluded or blocked shadow ray."""
    alb = [0.2, 0.6, 0.9]
    sc = _scene(spheres=[[0, 0, 0, 1]], albedo=[alb], light=(0, 1, 0), lp=lp)
    rgb, prim, _ = sc.shade_ray([0, 5, 0], [0, -1, 0])  # top of the sphere, N = L
    assert prim == 0 and np.allclose(rgb[:3], alb, atol=1e-7) and abs(rgb[3] - 4.0) < 1e-12
    L = np.array([0, 1, 1]) / math.sqrt(2)
    sc = _scene(spheres=[[0, 0, 0, 1]], albedo=[alb], light=L, lp=lp)
    rgb, _, _ = sc.shade_ray([0, 5, 0], [0, -1, 0])  # N.L = cos 45
    assert np.allclose(rgb[:3], np.array(alb) * (0.1 + 0.9 / math.sqrt(2)), atol=1e-7)
    rgb, _, _ = sc.shade_ray([0, -5, 0], [0, 1, 0])  # bottom: N.L < 0 -> ambient only
    assert np.allclose(rgb[:3], np.array(alb) * 0.1, atol=1e-7)
    # sphere above the ground, light straight up: the spot below it is in shadow
    sc = _scene(tris=GROUND, spheres=[[0, 2, 0, 1]], albedo=[[0.5] * 3, [0.5] * 3, alb], light=(0, 1, 0), lp=lp)
    d = np.array([0, -0.5, -5.4])  # meets the ground at (0.3, 0, -0.4), below the sphere
    d /= np.linalg.norm(d)
    rgb, prim, flag = sc.shade_ray([0.3, 0.5, 5], d)
    assert prim in (0, 1) and np.allclose(rgb[:3], 0.05, atol=1e-7) and flag == 0
    rgb, prim, _ = sc.shade_ray([5, 3, 0.5], [0, -1, 0])
    assert prim in (0, 1) and np.allclose(rgb[:3], 0.5, atol=1e-7)
    assert abs(rgb[3] - 3.0) < 1e-12
    # ambient is a parameter
    sc = _scene(tris=GROUND, spheres=[[0, 2, 0, 1]], albedo=[[0.5] * 3, [0.5] * 3, alb], light=(0, 1, 0),
                ambient=0.3, lp=lp)
    rgb, _, _ = sc.shade_ray([0.3, 0.5, 5], d)
    assert np.allclose(rgb[:3], 0.15, atol=1e-7)


def check_point_light(lp=None):
    """Point light without distance falloff; the shadow ray stops at the light."""
    for h in (1.0, 7.0, 100.0):
        sc = _scene(tris=GROUND, albedo=[[0.4, 0.4, 0.4]] * 2, light_type=O.LIGHT_POINT, light=(1, h, 2), lp=lp)
        rgb, _, _ = sc.shade_ray([1, 5, 2.0001], [0, -1, 0])
        assert np.allclose(rgb[:3], 0.4, atol=1e-6), (h, rgb)
    # light at 45 degrees: N.L = cos 45
    sc = _scene(tris=GROUND, albedo=[[0.4, 0.4, 0.4]] * 2, light_type=O.LIGHT_POINT, light=(3, 3, 0), lp=lp)
    rgb, _, _ = sc.shade_ray([0, 5, 0.001], [0, -1, 0])
    assert np.allclose(rgb[:3], 0.4 * (0.1 + 0.9 / math.sqrt(2)), atol=1e-6)
    # an occluder beyond the light does not shadow; one between does
    tri_far = [-1, 6, -1, 1, 6, 1, 1, 6, -1]
    sc = _scene(tris=GROUND + [tri_far], albedo=[[0.4] * 3] * 3, light_type=O.LIGHT_POINT, light=(0.2, 4, 0.1), lp=lp)
    rgb, _, _ = sc.shade_ray([0.2, 2, 0.1], [0, -1, 0])
    assert np.allclose(rgb[:3], 0.4, atol=1e-6)
    sc = _scene(tris=GROUND + [tri_far], albedo=[[0.4] * 3] * 3, light_type=O.LIGHT_POINT, light=(0.2, 8, 0.1), lp=lp)
    rgb, _, _ = sc.shade_ray([0.2, 2, 0.1], [0, -1, 0])
    assert np.allclose(rgb[:3], 0.04, atol=1e-6)


def check_sky_and_clamp(lp=None):
    sc = _scene(tris=GROUND, albedo=[[2.0, 0.5, -1.0]] * 2, light=(0, 1, 0), lp=lp)
    rgb, prim, _ = sc.shade_ray([0, 5, 0], [0, 1, 0])
    assert prim == -1 and np.allclose(rgb, [0.5, 0.7, 1.0, -1.0])
    rgb, prim, _ = sc.shade_ray([0, 5, 0], [1, 0, 0])
    assert prim == -1 and np.allclose(rgb[:3], [0.75, 0.85, 1.0])
    rgb, prim, _ = sc.shade_ray([0, -5, 0], [0, -1, 0])
    assert prim == -1 and np.allclose(rgb[:3], [1.0, 1.0, 1.0])
    rgb, prim, _ = sc.shade_ray([1, 5, 0.5], [0, -1, 0])
    assert prim in (0, 1) and np.allclose(rgb[:3], [1.0, 0.5, 0.0])


def check_two_sided(lp=None):
    """Seen from below, the ground's normal faces down; a light above gives
    ambient only. A light below lights it fully."""
    sc = _scene(tris=GROUND, albedo=[[0.5] * 3] * 2, light=(0, 1, 0), lp=lp)
    rgb, _, _ = sc.shade_ray([1, -3, 0.5], [0, 1, 0])
    assert np.allclose(rgb[:3], 0.05)
    sc = _scene(tris=GROUND, albedo=[[0.5] * 3] * 2, light=(0, -1, 0), lp=lp)
    rgb, _, _ = sc.shade_ray([1, -3, 0.5], [0, 1, 0])
    assert np.allclose(rgb[:3], 0.5)


# --------------------------------------------------------------------------- closest hit

def check_closest_and_ties(lp=None):
    near = [-1, -1, 0, 1, -1, 0, 0, 1, 0]
    far = [-1, -1, -1, 1, -1, -1, 0, 1, -1]
    for tris, want in [([near, far], 0), ([far, near], 1)]:
        sc = _scene(tris=tris, albedo=[[0.5] * 3] * 2, lp=lp)
        t, p, f = sc.trace_closest([0, 0, 5], [0, 0, -1], 1e-6)
        assert p == want and abs(t - 5) < 1e-14 and f == 0
    sc = _scene(tris=[far, near, near], albedo=[[0.5] * 3] * 3, lp=lp)
    t, p, f = sc.trace_closest([0, 0, 5], [0, 0, -1], 1e-6)
    assert p == 1 and f == O.FLAG_ID  # exact depth tie -> lower id, flagged (same plane: point well defined)
    sc = _scene(tris=[near], spheres=[[0, 0, -1, 1]], albedo=[[0.5] * 3] * 2, lp=lp)
    t, p, f = sc.trace_closest([0, 0, 5], [0, 0, -1], 1e-6)
    assert p == 0 and f == O.FLAG_ID  # sphere top touches the triangle at t = 5
    t, p, f = sc.trace_closest([0, 0, 5], [0, 0, -1], 5.5)
    assert p == 1 and abs(t - 7.0) < 1e-14  # t_min skips the triangle; far root of the sphere
    sc = _scene(spheres=[[0, 0, 0, 1], [0, 0, -3, 1]], albedo=[[0.5] * 3] * 2, lp=lp)
    t, p, f = sc.trace_closest([0, 0, 5], [0, 0, -1], 1e-6)
    assert p == 0 and abs(t - 4) < 1e-14 and f == 0


def check_flags(lp=None):
    sc = _scene(tris=GROUND, albedo=[[0.5] * 3] * 2, lp=lp)
    _, p, f = sc.trace_closest([3, 5, -6], [0, -1, 0], 1e-6)
    assert p in (0, 1) and f == 0
    _, p, f = sc.trace_closest([2, 5, 2], [0, -1, 0], 1e-6)  # on the shared diagonal
    assert f == 1
    band = O.TOL * (5 + math.sqrt(4 + 25 + 100))  # t + |o|
    _, p, f = sc.trace_closest([10 + 0.3 * band, 5, 10], [0, -1, 0], 1e-6)  # just outside a corner
    assert f == 1 and p == -1
    _, p, f = sc.trace_closest([10 + 3 * band, 5, 0], [0, -1, 0], 1e-6)
    assert f == 0 and p == -1
    sc = _scene(spheres=[[0, 0, 0, 1]], albedo=[[0.5] * 3], lp=lp)
    _, p, f = sc.trace_closest([1.0, 0, 10], [0, 0, -1], 1e-6)  # grazing the silhouette: hit point ill-conditioned
    assert p == 0 and f == O.FLAG_ID | O.FLAG_POINT
    _, p, f = sc.trace_closest([1.0 + 1e-9, 0, 10], [0, 0, -1], 1e-6)  # just outside: a miss, id ambiguous
    assert p == -1 and f == O.FLAG_ID
    _, p, f = sc.trace_closest([0.5, 0, 10], [0, 0, -1], 1e-6)
    assert f == 0 and p == 0
    t, p, f = sc.trace_closest([0.0, 0.0, 0.0], [0, 0, -1], 1.0 - 1e-9)  # from the centre: the root at t_min
    assert p == 0 and t == 1.0 and f == O.FLAG_ID | O.FLAG_POINT
    # the flag bits of a shaded ray: the ground point (1, 0, -2) seen from
    # straight above is clear of the sphere, but its shadow ray towards
    # L = (0, 1, 1)/sqrt(2) is tangent to the sphere (distance 1 from (0, 2, 0))
    sc = _scene(tris=GROUND, spheres=[[0, 2, 0, 1]], albedo=[[0.5] * 3] * 3, light=(0, 1, 1), lp=lp)
    _, p, f = sc.shade_ray([1, 10, -2], [0, -1, 0])
    assert p in (0, 1) and f == O.FLAG_SHADOW
    _, p, f = sc.shade_ray([1, 10, -2.5], [0, -1, 0])  # clear of the tangent: nothing ambiguous
    assert p in (0, 1) and f == 0


def check_any_hit(lp=None):
    """Any-hit: occluded exactly when some primitive is hit at t in the open
    interval (t_min, t_max); a hit at t_max itself does not occlude. On random
    rays it agrees with 'the closest hit lies before t_max'."""
    sc = _scene(tris=GROUND, spheres=[[0, 2, 0, 1]], albedo=[[0.5] * 3] * 3, lp=lp)
    o, d = [0.3, 10, 0.2], [0, -1, 0]
    t_sph, p, _ = sc.trace_closest(o, d, 0.0)  # the sphere's top, at t = 10 - (2 + sqrt(1 - 0.13))
    assert p == 2 and abs(t_sph - (8 - math.sqrt(1 - 0.13))) < 1e-12
    occ, _ = sc.trace_any(o, d, 0.0, np.inf)
    assert occ == 1
    occ, f = sc.trace_any(o, d, 0.0, t_sph)  # t_max exactly at the hit: free
    assert occ == 0 and f == 1  # ... and flagged: the hit sits on the interval's end
    occ, _ = sc.trace_any(o, d, 0.0, t_sph * (1 + 1e-9))
    assert occ == 1
    occ, _ = sc.trace_any(o, d, 9.0, 9.5)  # interval past the sphere and before the ground
    assert occ == 0
    occ, _ = sc.trace_any(o, d, 9.0, 10.5)  # reaches the ground at t = 10
    assert occ == 1
    occ, _ = sc.trace_any([5, 10, 5], [0, 1, 0], 0.0, np.inf)  # upwards: nothing
    assert occ == 0
    occ, f = sc.trace_any([5, 10, 5], [0, -1, 0], 0.0, 10.0)  # t_max exactly at the ground: free
    assert occ == 0 and f == 1
    occ, _ = sc.trace_any([5, 10, 5], [0, -1, 0], 0.0, 10.0 * (1 + 1e-9))
    assert occ == 1
    rng = np.random.default_rng(12)
    soup = rng.uniform(-3, 3, size=(40, 9))
    sph = np.concatenate([rng.uniform(-3, 3, size=(5, 3)), rng.uniform(0.2, 0.8, size=(5, 1))], 1)
    sc = _scene(tris=soup, spheres=sph, albedo=[[0.5] * 3] * 45, lp=lp)
    n_occ = 0
    for _ in range(3000):
        o = rng.uniform(-5, 5, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        tmax = rng.uniform(0.5, 8.0)
        t, p, f1 = sc.trace_closest(o, d, 1e-6)
        occ, f2 = sc.trace_any(o, d, 1e-6, tmax)
        if f1 or f2:
            continue
        assert occ == (1 if (p >= 0 and t < tmax) else 0), (o, d, tmax, t, p)
        n_occ += occ
    assert 200 < n_occ < 2800


def check_scene_diam(lp=None):
    """The scene diameter (which sets t_min and the shadow offset) is the
    diagonal of the box around every triangle vertex and every sphere."""
    tri = [[1, 2, 3, 4, -1, 0, 2, 2, 7]]
    sph = [[-2, 0, 1, 0.5], [0, 5, 0, 2]]
    sc = _scene(tris=tri, spheres=sph, albedo=[[0.5] * 3] * 3, lp=lp)
    # per axis: the three vertices, then each sphere's centre -/+ radius
    lo = np.array([min(1, 4, 2, -2.5, -2), min(2, -1, 2, -0.5, 3), min(3, 0, 7, 0.5, -2)])
    hi = np.array([max(1, 4, 2, -1.5, 2), max(2, -1, 2, 0.5, 7), max(3, 0, 7, 1.5, 2)])
    assert abs(sc.diam - float(np.linalg.norm(hi - lo))) < 1e-12
    assert abs(_scene(tris=GROUND, albedo=[[0.5] * 3] * 2, lp=lp).diam - math.sqrt(800)) < 1e-12


# --------------------------------------------------------------------------- passes

def _tiny(lp=None):
    rng = np.random.default_rng(1)
    cen = np.stack([rng.uniform(-3, 3, 3), rng.uniform(1, 2, 3), rng.uniform(-3, 3, 3)], 1)
    sph = np.concatenate([cen, np.ones((3, 1))], 1)
    alb = np.concatenate([np.full((2, 3), 0.5), rng.uniform(0.2, 0.9, (3, 3))])
    return _scene(tris=GROUND, spheres=sph, albedo=alb, light_type=O.LIGHT_POINT, light=(5, 8, 5), lp=lp)


TINY_CAM = np.array([0.0, 3.0, 10.0, 0.0, 1.0, 0.0, 0.0, 1.0, 0.0, 60.0])


def check_first_pass_is_pinhole(lp=None):
    """I_0 = 0.5 gives an ordinary ray-traced image (§3): pass 1 from grey
    equals an explicit grey input, and with k = 0 every pass equals pass 1."""
    sc = _tiny(lp)
    W, H = 24, 16
    k = 0.05 * sc.diam
    a, pa, _ = sc.render_pass(TINY_CAM, W, H, O.MAP_EYE, k, 6.0)
    grey = np.full((H, W, 4), 0.5, np.float32)
    b, pb, _ = sc.render_pass(TINY_CAM, W, H, O.MAP_EYE, k, 6.0, in_rgbz=grey)
    assert np.array_equal(a[:, :3], b[:, :3]) and np.array_equal(pa, pb)
    for K in (2, 6):
        c, pc, _ = sc.render(TINY_CAM, W, H, K, O.MAP_EYE, 0.0, 6.0)
        assert np.array_equal(a[:, :3], c[:, :3]) and np.array_equal(pa, pc)
    # k > 0 does change later passes
    d, _, _ = sc.render(TINY_CAM, W, H, 3, O.MAP_EYE, k, 6.0)
    assert np.abs(d[:, :3] - a[:, :3]).max() > 0.05


def check_chain_and_subset(lp=None):
    """Each pixel's chain depends only on its own previous colour (§3): K
    chained passes equal the K-pass render, on the full image and on a subset."""
    sc = _tiny(lp)
    W, H, K = 20, 14, 3
    k = 0.05 * sc.diam
    full, pf, ff = sc.render(TINY_CAM, W, H, K, O.MAP_EYE, k, 6.0)
    img = None
    flags = np.zeros(W * H, bool)
    for _ in range(K):
        out, pr, fl = sc.render_pass(TINY_CAM, W, H, O.MAP_EYE, k, 6.0, in_rgbz=img)
        flags |= fl.astype(bool)
        img = out.reshape(H, W, 4).astype(np.float32)
    # the chained passes round colours to float32 in between; away from
    # ambiguous rays that changes nothing above the rounding level
    ok = ~flags & (ff == 0)
    assert ok.mean() > 0.9
    assert np.abs(out[ok, :3] - full[ok, :3]).max() < 1e-5
    assert np.array_equal(pr[ok], pf[ok])
    pix = np.array([0, 7, 55, W * H - 1])
    sub, ps, _ = sc.render(TINY_CAM, W, H, K, O.MAP_EYE, k, 6.0, pix=pix)
    assert np.array_equal(sub, full[pix]) and np.array_equal(ps, pf[pix])


def check_sphere_silhouette_image(lp=None):
    """A unit sphere at distance 10 on the axis covers exactly the pixels whose
    pinhole ray makes an angle below asin(1/10) with the axis."""
    sc = _scene(spheres=[[0, 0, -10, 1]], albedo=[[0.3, 0.3, 0.3]], lp=lp)
    W, H = 41, 31
    rgbz, prim, flag = sc.render_pass(CAM_Z, W, H, O.MAP_EYE, 0.0, 1.0)
    lim = math.asin(0.1)
    n = 0
    for p in range(W * H):
        _, d = _ray(CAM_Z, W, H, p % W, p // W, O.MAP_EYE, 0.0, 1.0, lp=lp)
        ang = _angle(d, np.array([0, 0, -1.0]))
        if abs(ang - lim) < 1e-9:
            continue
        assert (prim[p] == 0) == (ang < lim), p
        n += prim[p] == 0
        if prim[p] == 0:
            # depth: the near root of the textbook quadratic
            b = np.dot(d, [0, 0, 10.0])  # d . (o - c)
            t = -b - math.sqrt(b * b - 99.0)
            assert abs(rgbz[p, 3] - t * -d[2]) < 1e-9  # z-depth along the view axis (0, 0, -1)
    assert n > 20


def check_permutation(lp=None):
    """The closest hit does not depend on primitive order (ids follow)."""
    rng = np.random.default_rng(5)
    T = 40
    c = rng.uniform(-3, 3, (T, 1, 3))
    tris = (c + rng.normal(0, 1.0, (T, 3, 3))).reshape(T, 9)
    alb = rng.uniform(0.1, 0.9, (T, 3))
    perm = rng.permutation(T)
    a = _scene(tris=tris, albedo=alb, light=(0.3, 0.9, 0.2), lp=lp)
    b = _scene(tris=tris[perm], albedo=alb[perm], light=(0.3, 0.9, 0.2), lp=lp)
    cam = np.array([0.0, 2.0, 12.0, 0, 0, 0, 0, 1, 0, 50.0])
    ra, pa, fa = a.render_pass(cam, 32, 24, O.MAP_EYE, 0.0, 1.0)
    rb, pb, fb = b.render_pass(cam, 32, 24, O.MAP_EYE, 0.0, 1.0)
    inv = np.empty(T, np.int64)
    inv[perm] = np.arange(T)
    ok = (fa == 0) & (fb == 0)
    assert ok.mean() > 0.9
    pb_mapped = np.where(pb >= 0, perm[np.maximum(pb, 0)], -1)
    assert np.array_equal(pa[ok], pb_mapped[ok])
    assert np.allclose(ra[ok], rb[ok], atol=1e-12)


def check_ground_plane_image(lp=None):
    """Looking straight down on the lit ground: every pixel's colour is
    albedo (a + (1-a) L_y) and its z-depth (along the view axis, §4) is the
    camera's height above the plane, whatever the pixel; the hit distance
    along the ray is h / |d_y|."""
    L = np.array([0.3, 0.8, 0.2])
    L /= np.linalg.norm(L)
    sc = _scene(tris=GROUND, albedo=[[0.6, 0.4, 0.2]] * 2, light=L, lp=lp)
    cam = np.array([0.3, 4.0, 0.2, 0.3, 0.0, 0.2, 0.0, 0.0, -1.0, 40.0])
    W, H = 16, 12
    rgbz, prim, flag = sc.render_pass(cam, W, H, O.MAP_EYE, 0.0, 1.0)
    want = np.array([0.6, 0.4, 0.2]) * (0.1 + 0.9 * L[1])
    for p in range(W * H):
        if flag[p]:
            continue
        o, d = _ray(cam, W, H, p % W, p // W, O.MAP_EYE, 0.0, 1.0, lp=lp)
        assert np.allclose(rgbz[p, :3], want, atol=1e-12)
        assert abs(rgbz[p, 3] - 4.0) < 1e-12
        rgbt, _, _ = sc.shade_ray(o, d)
        assert abs(rgbt[3] - 4.0 / -d[1]) < 1e-12
    # EYE mapping: a blue displacement moves each pixel's eye along the view
    # axis by k (2b - 1), so the plane's z-depth becomes 4 - k (2b - 1)
    prev = np.zeros((H, W, 4), np.float32)
    prev[..., :3] = (0.5, 0.5, 0.9)
    rgbz, _, flag = sc.render_pass(cam, W, H, O.MAP_EYE, 0.5, 1.0, in_rgbz=prev)
    ok = flag == 0
    assert ok.mean() > 0.9
    assert np.allclose(rgbz[ok, 3], 4.0 - 0.5 * (2 * np.float32(0.9) - 1), atol=1e-9)


# --------------------------------------------------------------------------- image space (§6, §6.1)

def check_mirror_rule(lp=None):
    """Reflection without repeating the edge pixel, repeated for big offsets."""
    n = 5
    got = [O.mirror_index(i, n, libpath=lp) for i in range(-12, 17)]
    want = []
    for i in range(-12, 17):
        j = i
        while j < 0 or j >= n:
            j = -j - 1 if j < 0 else 2 * n - 1 - j
        want.append(j)
    assert got == want
    assert [O.mirror_index(i, 5, libpath=lp) for i in (-1, -2, 5, 6, 10)] == [0, 1, 4, 3, 0]
    assert O.mirror_index(7, 1, libpath=lp) == 0


def _ramp(W, H):
    # every pixel carries its own coordinates, so a gather is readable
    b = np.zeros((H, W, 4), np.float32)
    b[..., 0] = np.arange(W)[None, :]
    b[..., 1] = np.arange(H)[:, None]
    b[..., 2] = 7.0
    b[..., 3] = np.arange(W * H).reshape(H, W)
    return b


def check_imagespace_shifts(lp=None):
    """Grey and pure blue do not move; R=1 samples k pixels to the right, R=0
    to the left, G=1 k rows up (towards row 0), G=0 down; edges mirror."""
    W, H, k = 11, 7, 3.0
    base = _ramp(W, H)

    def run(c, kk=k):
        prev = np.empty((H, W, 4), np.float32)
        prev[...] = c
        return O.imagespace_pass(base, prev, W, H, kk, libpath=lp).reshape(H, W, 4)

    for c in [(0.5, 0.5, 0.5, 0.0), (0.5, 0.5, 1.0, 2.0), (0.5, 0.5, 0.0, 9.0)]:
        assert np.array_equal(run(c), base)
    mx = lambda i: O.mirror_index(i, W, libpath=lp)
    my = lambda i: O.mirror_index(i, H, libpath=lp)
    for (c, fx, fy) in [((1.0, 0.5, 0.5, 0), lambda x: mx(x + 3), lambda y: y),
                        ((0.0, 0.5, 0.5, 0), lambda x: mx(x - 3), lambda y: y),
                        ((0.5, 1.0, 0.5, 0), lambda x: x, lambda y: my(y - 3)),
                        ((0.5, 0.0, 0.5, 0), lambda x: x, lambda y: my(y + 3)),
                        ((1.0, 1.0, 0.5, 0), lambda x: mx(x + 3), lambda y: my(y - 3))]:
        out = run(c)
        for y in range(H):
            for x in range(W):
                assert out[y, x, 0] == fx(x) and out[y, x, 1] == fy(y), (c, x, y)
                assert out[y, x, 2] == 7.0 and out[y, x, 3] == fy(y) * W + fx(x)


def check_imagespace_rounding(lp=None):
    """The nearest pixel is taken; halves round up (towards +x / +y)."""
    W, H = 9, 5
    base = _ramp(W, H)
    prev = np.full((H, W, 4), 0.5, np.float32)
    prev[..., 0] = 1.0
    for kk, shift, at_half in [(1.4, 1, 0), (1.6, 2, 0), (0.5, 1, 1), (0.49, 0, 0), (2.5, 3, 1)]:
        out, fl = O.imagespace_pass(base, prev, W, H, kk, libpath=lp, want_flag=True)
        out = out.reshape(H, W, 4)
        assert out[2, 3, 0] == 3 + shift, (kk, out[2, 3, 0])
        assert fl.reshape(H, W)[2, 3] == at_half, kk  # a sample exactly between two pixels is flagged
    prev[..., 0] = 0.0
    out = O.imagespace_pass(base, prev, W, H, 0.5, libpath=lp).reshape(H, W, 4)
    assert out[2, 3, 0] == 3  # x - 0.5 rounds half up to x
    sub = O.imagespace_pass(base, prev, W, H, 2.0, pix=np.array([0, 13, 44]), libpath=lp)
    full = O.imagespace_pass(base, prev, W, H, 2.0, libpath=lp)
    assert np.array_equal(sub, full[[0, 13, 44]])


# --------------------------------------------------------------------------- normal mapping (§5, Eq. 8)

def check_imagespace_band(lp=None):
    """The flag marks exactly the samples within IMG_TOL (x + k + 1) of a
    half-integer: just inside the band flagged, just outside not, and a
    displacement that lands near an integer (a pixel centre) never flagged."""
    W, H, x, y = 64, 3, 40, 1
    base = _ramp(W, H)
    prev = np.full((H, W, 4), 0.5, np.float32)
    prev[..., 0] = 1.0  # sx = x + k exactly
    for frac, want in [(0.5, 1), (0.5 + 0.5 * O.IMG_TOL * 48, 1), (0.5 - 0.9 * O.IMG_TOL * 48, 1),
                       (0.5 + 1.5 * O.IMG_TOL * 48, 0), (0.0, 0), (0.999999, 0), (0.25, 0)]:
        k = 6.0 + frac  # x + k + 1 = 47 + frac ~ 47.5
        _, fl = O.imagespace_pass(base, prev, W, H, k, libpath=lp, want_flag=True)
        assert fl.reshape(H, W)[y, x] == want, (frac, want)
    # the row coordinate has its own band (y - k (2g - 1))
    prev[..., 0] = 0.5
    prev[..., 1] = 0.0  # sy = y + k
    _, fl = O.imagespace_pass(base, prev, W, H, 0.5, libpath=lp, want_flag=True)
    assert fl.reshape(H, W)[y, x] == 1
    _, fl = O.imagespace_pass(base, prev, W, H, 0.7, libpath=lp, want_flag=True)
    assert fl.reshape(H, W)[y, x] == 0


def check_normal_mapping_camera(lp=None):
    """V_p = k (C x N): for the centre ray C = (0,0,-1) and N = +y the target
    moves by +k along x (right); N along C does not move it; no normal (as in
    I_0, or after a miss) gives the pinhole ray."""
    W, H, k, f = 21, 21, 0.7, 4.0
    x, y = W // 2, H // 2
    _, d0 = _ray(CAM_Z, W, H, x, y, O.MAP_TARGET, 0.0, f, lp=lp)
    o, d = _ray(CAM_Z, W, H, x, y, O.MAP_NORMAL, k, f, n=[0.0, 1.0, 0.0], lp=lp)
    P = o + d * (f / -d[2])  # where the ray meets the focal plane z = -f
    assert np.allclose(P, [k, 0.0, -f], atol=1e-12)
    o, d = _ray(CAM_Z, W, H, x, y, O.MAP_NORMAL, k, f, n=[1.0, 0.0, 0.0], lp=lp)
    P = o + d * (f / -d[2])  # C x (+x) = (0,0,-1) x (1,0,0) = (0,-1,0): down
    assert np.allclose(P, [0.0, -k, -f], atol=1e-12)
    _, d = _ray(CAM_Z, W, H, x, y, O.MAP_NORMAL, k, f, n=[0.0, 0.0, 1.0], lp=lp)
    assert np.allclose(d, d0, atol=1e-15)
    for n in (None, [0.0, 0.0, 0.0]):
        _, d = _ray(CAM_Z, W, H, 3, 5, O.MAP_NORMAL, k, f, n=n, lp=lp)
        _, e = _ray(CAM_Z, W, H, 3, 5, O.MAP_TARGET, 0.0, f, lp=lp)
        assert np.array_equal(d, e)


def check_normal_mapping_render(lp=None):
    """Pass 1 is pinhole (I_0 has no normal) and outputs each hit's normal
    facing its ray (the ground seen from above: +y; a miss: zero); a ground
    plane seen straight on from above has N parallel to C at the centre, so
    the centre pixel keeps its colour in pass 2."""
    L = np.array([0.3, 0.8, 0.2])
    sc = _scene(tris=GROUND, albedo=[[0.6, 0.4, 0.2]] * 2, light=L, lp=lp)
    cam = np.array([0.3, 4.0, 0.2, 0.3, 0.0, 0.2, 0.0, 0.0, -1.0, 40.0])
    W, H = 9, 7
    a, pa, _, na = sc.render_pass(cam, W, H, O.MAP_NORMAL, 0.5, 1.0, want_normal=True)
    b, pb, _ = sc.render_pass(cam, W, H, O.MAP_TARGET, 0.0, 1.0)
    assert np.array_equal(a, b) and np.array_equal(pa, pb)
    assert np.array_equal(na, np.tile([0.0, 1.0, 0.0], (W * H, 1)))
    c2, _, _ = sc.render_pass(cam, W, H, O.MAP_NORMAL, 0.5, 1.0, in_rgbz=O.rgbz_to_image(a), in_normal=na)
    centre = (H // 2) * W + W // 2
    assert np.allclose(c2[centre, :3], a[centre, :3], atol=1e-12)
    sky = _scene(spheres=[[30, -50, 0, 1]], albedo=[[0.5] * 3], lp=lp)  # out of view
    _, p, _, n = sky.render_pass(cam, 3, 3, O.MAP_NORMAL, 0.5, 1.0, want_normal=True)
    assert np.all(p == -1) and not n.any()


def check_normal_chain(lp=None):
    """The K-pass normal-mapping render carries each pass's hit normal into the
    next pass's camera: it equals passes chained by hand with the normals
    handed over, and differs from a chain that drops them."""
    sc = _tiny(lp)
    W, H, K, k = 18, 12, 3, 0.8
    full, pf, ff, nf = sc.render(TINY_CAM, W, H, K, O.MAP_NORMAL, k, 6.0, want_normal=True)
    img, nrm = None, None
    for _ in range(K):
        out, pr, fl, nrm = sc.render_pass(TINY_CAM, W, H, O.MAP_NORMAL, k, 6.0, in_rgbz=img, in_normal=nrm,
                                          want_normal=True)
        img = O.rgbz_to_image(out)
    ok = ff == 0
    assert ok.mean() > 0.9
    assert np.abs(out[ok, :3] - full[ok, :3]).max() < 1e-5 and np.array_equal(pr[ok], pf[ok])
    assert np.abs(nrm[ok] - nf[ok]).max() < 1e-9
    lost, _, _ = sc.render_pass(TINY_CAM, W, H, O.MAP_NORMAL, k, 6.0, in_rgbz=img)  # no normals: pinhole
    pin, _, _ = sc.render_pass(TINY_CAM, W, H, O.MAP_TARGET, 0.0, 6.0)
    assert np.array_equal(lost[:, :3], pin[:, :3])
    assert np.abs(full[ok, :3] - pin[ok, :3]).max() > 0.01


# --------------------------------------------------------------------------- multi-sample passes (§2 jitter)

def check_ms_centre_is_single(lp=None):
    """One sample at the pixel centre, or several identical ones, is the
    single-sample pass bit for bit (with I_0 and with a previous image)."""
    sc = _tiny(lp)
    W, H, k = 20, 14, 1.4
    ref, pref, _ = sc.render_pass(TINY_CAM, W, H, O.MAP_EYE, k, 6.0)
    img = O.rgbz_to_image(ref).reshape(H, W, 4)
    for jit in ([[0.5, 0.5]], [[0.5, 0.5]] * 4):
        a, pa, _ = sc.render_pass_ms(TINY_CAM, W, H, O.MAP_EYE, k, 6.0, jit)
        assert np.array_equal(a, ref) and np.array_equal(pa, pref)
        b, _, _ = sc.render_pass_ms(TINY_CAM, W, H, O.MAP_EYE, k, 6.0, jit, in_rgbz=img)
        c, _, _ = sc.render_pass(TINY_CAM, W, H, O.MAP_EYE, k, 6.0, in_rgbz=img)
        assert np.array_equal(b, c)
    full, _ = sc.render_ms(TINY_CAM, W, H, 3, O.MAP_EYE, k, 6.0, [[0.5, 0.5]])
    chain, _, _ = sc.render(TINY_CAM, W, H, 3, O.MAP_EYE, k, 6.0)
    assert np.array_equal(full, chain)
    # the normal mapping: a centre sample reads its own pixel's normal
    full, _, nf = sc.render_ms(TINY_CAM, W, H, 3, O.MAP_NORMAL, k, 6.0, [[0.5, 0.5]], want_normal=True)
    chain, _, _, nc = sc.render(TINY_CAM, W, H, 3, O.MAP_NORMAL, k, 6.0, want_normal=True)
    assert np.array_equal(full, chain) and np.array_equal(nf, nc)


def check_bilinear_reads(lp=None):
    """Bilinear reads reproduce a linear ramp exactly inside the image and
    clamp to the edge pixels outside; the normal code lane is the nearest
    pixel's."""
    W, H = 8, 6
    img = np.zeros((H, W, 4), np.float32)
    img[..., 0] = 0.1 * np.arange(W)[None, :]
    img[..., 1] = 0.05 * np.arange(H)[:, None]
    img[..., 3] = 0.01 * np.arange(W * H).reshape(H, W)
    for px, py in [(1.5, 1.5), (3.25, 2.75), (6.9, 4.1), (4.0, 3.0)]:
        c = O.sample_image(img, W, H, px, py, libpath=lp)
        assert abs(c[0] - 0.1 * (px - 0.5)) < 1e-7 and abs(c[1] - 0.05 * (py - 0.5)) < 1e-7
    c = O.sample_image(img, W, H, 0.1, 0.2, libpath=lp)
    assert np.allclose(c[:2], img[0, 0, :2])
    c = O.sample_image(img, W, H, W + 3.0, H + 0.4, libpath=lp)
    assert np.allclose(c[:2], img[H - 1, W - 1, :2])
    c = O.sample_image(img, W, H, 2.5, 1.5, libpath=lp)  # a pixel centre: that pixel, all four lanes
    assert np.allclose(c, img[1, 2], atol=1e-7)
    # the nearest pixel (where a sample reads a normal): the one whose square holds the point
    assert O.nearest_pixel(W, H, 3.9, 2.2, libpath=lp) == 2 * W + 3
    assert O.nearest_pixel(W, H, 4.0, 3.0, libpath=lp) == 3 * W + 4
    assert O.nearest_pixel(W, H, -2.0, H + 5.0, libpath=lp) == (H - 1) * W


def check_ms_sphere_coverage(lp=None):
    """A unit sphere at distance 10, lit from behind (ambient only): each pixel
    is the mean over its samples of the sphere's ambient colour (sample inside
    the silhouette angle asin(1/10)) or the sky seen along that sample."""
    alb = np.array([0.6, 0.3, 0.9])
    sc = _scene(spheres=[[0, 0, -10, 1]], albedo=[alb], light=(0.0, 0.0, -1.0), lp=lp)
    W, H = 31, 23
    jit = np.array([[0.125, 0.375], [0.625, 0.125], [0.375, 0.875], [0.875, 0.625]], np.float32)
    rgbz, _, flag = sc.render_pass_ms(CAM_Z, W, H, O.MAP_EYE, 0.0, 1.0, jit)
    lim = math.asin(0.1)
    n_mixed = 0
    for p in range(W * H):
        x, y = p % W, p // W
        want = np.zeros(3)
        hits = 0
        for jx, jy in jit:
            _, d, _ = O.camera_ray_at(CAM_Z, W, H, x + float(jx), y + float(jy), O.MAP_EYE, 0.0, 1.0, libpath=lp)
            if _angle(d, np.array([0, 0, -1.0])) < lim:
                want += 0.1 * alb
                hits += 1
            else:
                sv = 0.5 * (d[1] + 1)
                want += (1 - sv) * np.ones(3) + sv * np.array([0.5, 0.7, 1.0])
        if flag[p]:
            continue
        assert np.allclose(rgbz[p, :3], want / 4, atol=1e-12), (x, y)
        n_mixed += 0 < hits < 4
    assert n_mixed > 4


ALL_CHECKS = [v for k, v in sorted(globals().items()) if k.startswith("check_")]
