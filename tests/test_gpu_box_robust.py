"""The BVH walk against brute force on rays chosen to break a box test that is
not conservative: axis-aligned geometry on integer coordinates (flat boxes,
shared faces), rays parallel to the axes, rays in or starting on a box plane,
rays through shared edges and vertices (equal-t ties), rays from far away,
and the same scene moved to 1e4 (large |origin| against small box sizes).
Closest hits must agree bit for bit (id and t); any-hit must agree on
occlusion, also with t_max exactly at and just past the closest hit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu

N_GRID = 32


def _rays(off, seed):
    """Seeded adversarial rays for blocks_scene(N_GRID, offset=off)."""
    rng = np.random.default_rng(seed)
    o, d = [], []
    off = np.asarray(off, np.float64)
    half = np.arange(0, 2 * N_GRID + 1) / 2.0  # integer and half-integer grid lines
    # A: straight down onto vertices, edges and quad diagonals; B: straight up
    # from the floor plane (t = 0 excluded) and from below it
    for x in half[::3]:
        for z in half[::3]:
            o.append((x, 5.0, z)), d.append((0.0, -1.0, 0.0))
            o.append((x, 0.0, z)), d.append((0.0, 1.0, 0.0))
            o.append((x, -1.0, z)), d.append((0.0, 1.0, 0.0))
    # C, D: along +-x and +-z in the floor plane, through cube faces, edges and tops
    for y in (0.0, 0.5, 1.0, 2.0, 3.0):
        for w in half[::2]:
            o.append((-2.0, y, w)), d.append((1.0, 0.0, 0.0))
            o.append((N_GRID + 2.0, y, w)), d.append((-1.0, 0.0, 0.0))
            o.append((w, y, -2.0)), d.append((0.0, 0.0, 1.0))
            o.append((w, y, N_GRID + 2.0)), d.append((0.0, 0.0, -1.0))
    # E: oblique with one zero component, from integer points
    s = 1.0 / np.sqrt(2.0)
    for _ in range(3000):
        p = rng.integers(0, N_GRID + 1, size=3).astype(np.float64)
        p[1] = rng.integers(0, 5)
        k = rng.integers(0, 6)
        dirs = [(s, -s, 0.0), (-s, -s, 0.0), (0.0, -s, s), (0.0, -s, -s), (s, 0.0, s), (-s, 0.0, s)]
        o.append(tuple(p)), d.append(dirs[k])
    # F: from far away towards grid vertices and cube corners
    for _ in range(3000):
        target = rng.integers(0, N_GRID + 1, size=3).astype(np.float64)
        target[1] = rng.integers(0, 4)
        src = target + rng.normal(size=3) * 1000.0
        src[1] = abs(src[1]) + 10.0
        v = target - src
        o.append(tuple(src)), d.append(tuple(v / np.linalg.norm(v)))
    # G: random rays in and around the grid
    for _ in range(3000):
        src = rng.uniform(-4, N_GRID + 4, size=3)
        src[1] = rng.uniform(-1, 6)
        v = rng.normal(size=3)
        o.append(tuple(src)), d.append(tuple(v / np.linalg.norm(v)))
    o = np.asarray(o) + off
    d = np.asarray(d)
    ot = np.zeros((len(o), 4), np.float32)
    dt = np.zeros((len(o), 4), np.float32)
    ot[:, :3] = o
    dt[:, :3] = d
    dt[:, 3] = np.inf
    return ot, dt


def _trace(g, ot, dt, any_hit, brute):
    n = len(ot)
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    p = torch.empty(n, dtype=torch.int32, device="cuda")
    rcp.rcp_debug_trace(g, n, torch.from_numpy(ot).cuda(), torch.from_numpy(dt).cuda(), any_hit, brute, t, p)
    torch.cuda.synchronize()
    return t.cpu().numpy(), p.cpu().numpy()


@pytest.mark.parametrize("collapse", [rcp.RCP_COLLAPSE_AREA, rcp.RCP_COLLAPSE_SAH])
@pytest.mark.parametrize("offset", [(0.0, 0.0, 0.0), (1e4, 0.0, 1e4), (-3e3, 50.0, 7e3)])
def test_closest_and_any_hit_equal_brute_force(offset, collapse):
    sc = scenes.blocks_scene(N_GRID, offset=offset)
    g = U.gpu_scene(sc, collapse)
    try:
        ot, dt = _rays(offset, seed=31)
        tb, pb = _trace(g, ot, dt, 0, 1)
        tw, pw = _trace(g, ot, dt, 0, 0)
        assert (pb >= 0).sum() >= len(pb) // 4
        bad = np.nonzero((pb != pw) | (tb.view(np.uint32) != tw.view(np.uint32)))[0]
        assert len(bad) == 0, (len(bad), ot[bad[:5]], dt[bad[:5]], pb[bad[:5]], pw[bad[:5]])
        # any hit, unbounded and with t_max at / just past the closest hit
        hit = pb >= 0
        for tmax in (np.inf, "at", "past"):
            d2 = dt.copy()
            if tmax == "at":
                d2[hit, 3] = tb[hit]
            elif tmax == "past":
                d2[hit, 3] = np.nextafter(tb[hit], np.float32(np.inf))
            _, ob = _trace(g, ot, d2, 1, 1)
            _, ow = _trace(g, ot, d2, 1, 0)
            assert np.array_equal(ob, ow), (tmax, int((ob != ow).sum()))
            if tmax == "past":
                assert np.all(ow[hit] == 1)
    finally:
        rcp.rcp_scene_destroy(g)


def test_tmin_on_the_hit():
    """Origins exactly on the floor with t_min = 0 and t_min just above 0."""
    sc = scenes.blocks_scene(N_GRID)
    g = U.gpu_scene(sc)
    try:
        rng = np.random.default_rng(8)
        n = 4000
        ot = np.zeros((n, 4), np.float32)
        dt = np.zeros((n, 4), np.float32)
        ot[:, 0] = rng.integers(0, 2 * N_GRID + 1, n) / 2.0
        ot[:, 2] = rng.integers(0, 2 * N_GRID + 1, n) / 2.0
        v = rng.normal(size=(n, 3))
        dt[:, :3] = v / np.linalg.norm(v, axis=1, keepdims=True)
        dt[:, 3] = np.inf
        for tmin in (0.0, 1e-6, 0.25):
            ot[:, 3] = tmin
            tb, pb = _trace(g, ot, dt, 0, 1)
            tw, pw = _trace(g, ot, dt, 0, 0)
            assert np.array_equal(pb, pw) and np.array_equal(tb.view(np.uint32), tw.view(np.uint32)), tmin
    finally:
        rcp.rcp_scene_destroy(g)
