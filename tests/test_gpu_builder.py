"""GPU tests of the BVH builder's parts: radix sort, Morton codes, tree
validity, and BVH traversal against brute force over every primitive."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n", [0, 1, 2, 3839, 3840, 3841, 100_003, 1_000_000])
@pytest.mark.parametrize("bits", [30, 32])
def test_radix_sort_matches_stable_sort(n, bits):
    rng = np.random.default_rng(n + bits)
    hi = 1 << bits
    keys = rng.integers(0, hi, size=n, dtype=np.uint64).astype(np.uint32)
    if n > 10:
        keys[: n // 3] = keys[0]  # many duplicates: stability matters
        rng.shuffle(keys)
    vals = np.arange(n, dtype=np.uint32)
    dk, dv = _dev(keys.view(np.int32)), _dev(vals.view(np.int32))
    rcp.rcp_debug_sort_pairs(dk, dv, n, bits)
    torch.cuda.synchronize()
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(dk.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(dv.cpu().numpy().view(np.uint32), vals[order])


def _morton_ref(p, lo, hi):
    """Interleaved 10-bit cells of each axis, all axes scaled by the largest
    extent of the box (a cube with corner lo)."""
    ext = float(np.max(hi - lo))
    q = np.clip(((p - lo) / ext * 1024.0).astype(np.int64), 0, 1023)
    code = np.zeros(len(p), np.int64)
    for b in range(10):
        for a in range(3):
            code |= ((q[:, a] >> b) & 1) << (3 * b + (2 - a))
    return code.astype(np.uint32)


def _codes(p, lo, hi):
    codes = torch.empty(len(p), dtype=torch.int32, device="cuda")
    rcp.rcp_debug_morton(_dev(p), len(p), lo, hi, codes)
    return codes.cpu().numpy().view(np.uint32)


def test_morton_codes():
    rng = np.random.default_rng(3)
    p = rng.uniform(-5, 7, size=(50_000, 3)).astype(np.float32)
    lo = np.array([-5, -5, -5], np.float32)
    hi = np.array([7, 7, 7], np.float32)
    got = _codes(p, lo, hi)
    want = _morton_ref(p.astype(np.float32), lo, hi)
    # the kernel normalises in float32; allow codes to differ only where a
    # coordinate sits on a cell boundary
    diff = got != want
    assert diff.mean() < 1e-3
    # corners
    corners = np.array([[-5, -5, -5], [7 - 1e-4, 7 - 1e-4, 7 - 1e-4]], np.float32)
    c = _codes(corners, lo, hi)
    assert c[0] == 0 and c[1] == (1 << 30) - 1


def test_morton_flat_box_keeps_thin_axis_low():
    """A slab 256 x 8 x 256: y spans 8/256 of the cube, i.e. cells 0..31, so
    its bits never reach the top 5 interleaved levels; x and z use all 10."""
    rng = np.random.default_rng(4)
    lo = np.array([-128, 0, -128], np.float32)
    hi = np.array([128, 8, 128], np.float32)
    p = (lo + rng.uniform(0, 1, size=(20_000, 3)) * (hi - lo)).astype(np.float32)
    got = _codes(p, lo, hi)
    assert (got != _morton_ref(p, lo, hi)).mean() < 1e-3
    y_bits = sum(1 << (3 * b + 1) for b in range(10))
    assert np.all((got & y_bits) < (1 << 14))  # y bits 5..9 (positions 16..28) are zero
    top = np.array([[127.999, 7.999, 127.999]], np.float32)
    assert _codes(top, lo, hi)[0] == _morton_ref(top, lo, hi)[0]


SCENES = {
    "one_tri": lambda: scenes.random_soup(1, 0, seed=1),
    "two_tris": lambda: scenes.random_soup(2, 0, seed=2),
    "three_prims": lambda: scenes.random_soup(2, 1, seed=3),
    "sphere_only": lambda: scenes.random_soup(0, 5, seed=4),
    "tiny": lambda: scenes.tiny_scene(),
    "soup_10k": lambda: scenes.random_soup(10_000, 50, seed=5),
    "soup_dupes": lambda: _dupes(),
    "mid": lambda: scenes.mid_scene(),
}


def _dupes():
    sc = scenes.random_soup(3000, 0, seed=9, extent=1.0, tri_size=0.01)
    sc.tris[1000:2000] = sc.tris[0]  # identical centroids -> identical Morton codes
    return sc


COLLAPSE = [rcp.RCP_COLLAPSE_AREA, rcp.RCP_COLLAPSE_SAH]
# (collapse policy, references per triangle at most)
BUILDS = [(rcp.RCP_COLLAPSE_AREA, 0), (rcp.RCP_COLLAPSE_SAH, 0), (rcp.RCP_COLLAPSE_SAH, 8), (rcp.RCP_COLLAPSE_AREA, 4)]


@pytest.mark.parametrize("build", BUILDS, ids=lambda b: f"c{b[0]}s{b[1]}")
@pytest.mark.parametrize("name", sorted(SCENES))
def test_bvh_valid(name, build):
    collapse, split = build
    sc = SCENES[name]()
    g = U.gpu_scene(sc, collapse, split)
    try:
        rcp.rcp_scene_validate(g)
        info = rcp.rcp_scene_get_info(g)
        assert info.collapse == collapse and info.split_max == max(split, 1)
        assert sc.n_prims <= info.n_records <= sc.n_prims * max(split, 1)
        if split <= 1:
            assert info.n_records == sc.n_prims
        assert info.n_tris == sc.n_tris and info.n_spheres == sc.n_spheres
        assert 1 <= info.max_leaf <= 3
        assert info.depth >= 1 and info.n_nodes >= 1
        assert abs(info.diam - sc.diameter()) <= 1e-5 * sc.diameter() + 1e-6
    finally:
        rcp.rcp_scene_destroy(g)


@pytest.mark.parametrize("build", BUILDS, ids=lambda b: f"c{b[0]}s{b[1]}")
@pytest.mark.parametrize("name", ["tiny", "soup_10k", "soup_dupes", "three_prims", "sphere_only", "mid"])
@pytest.mark.parametrize("any_hit", [0, 1])
def test_bvh_equals_brute_force(name, any_hit, build):
    collapse, split = build
    """The BVH walk returns exactly what testing every primitive returns:
    same primitive ids, bit-identical distances (the box test is conservative
    and ties go to the lower id in both)."""
    sc = SCENES[name]()
    g = U.gpu_scene(sc, collapse, split)
    try:
        ext = max(sc.diameter() / 4, 1.0)
        n = 20_000 if name != "mid" else 4_000
        ot, dt = U.random_rays(n, seed=17, extent=ext, towards=(0, 0, 0))
        if any_hit:
            dt[:, 3] = np.random.default_rng(1).uniform(0.1, 4 * ext, n).astype(np.float32)
        res = []
        for brute in (0, 1):
            t = torch.empty(n, dtype=torch.float32, device="cuda")
            p = torch.empty(n, dtype=torch.int32, device="cuda")
            rcp.rcp_debug_trace(g, n, _dev(ot), _dev(dt), any_hit, brute, t, p)
            res.append((t.cpu().numpy(), p.cpu().numpy()))
        assert np.array_equal(res[0][1], res[1][1])
        assert np.array_equal(res[0][0], res[1][0])
        if not any_hit:
            assert (res[0][1] >= 0).sum() >= 100  # enough hits to mean something
    finally:
        rcp.rcp_scene_destroy(g)


def test_refit_after_vertex_update():
    """Moving vertices and refitting keeps the BVH valid and its walk equal to
    brute force on the moved geometry, and equal to a fresh build."""
    sc = scenes.random_soup(20_000, 0, seed=21)
    g = U.gpu_scene(sc)
    try:
        rng = np.random.default_rng(4)
        moved = sc.tris + rng.normal(0, 0.3, size=sc.tris.shape).astype(np.float32)
        rcp.rcp_scene_update_vertices(g, moved)
        rcp.rcp_scene_validate(g)
        fresh_sc = scenes.Scene("moved", moved, sc.spheres, sc.albedo, sc.light, sc.poses)
        f = U.gpu_scene(fresh_sc)
        try:
            n = 20_000
            ot, dt = U.random_rays(n, seed=5, extent=10.0, towards=(0, 0, 0))
            out = []
            for scene, brute in ((g, 0), (g, 1), (f, 0)):
                t = torch.empty(n, dtype=torch.float32, device="cuda")
                p = torch.empty(n, dtype=torch.int32, device="cuda")
                rcp.rcp_debug_trace(scene, n, _dev(ot), _dev(dt), 0, brute, t, p)
                out.append((t.cpu().numpy(), p.cpu().numpy()))
            assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][0], out[1][0])
            assert np.array_equal(out[0][1], out[2][1]) and np.array_equal(out[0][0], out[2][0])
            # device-array variant
            d = torch.from_numpy(sc.tris.copy()).cuda()
            rcp.rcp_scene_update_vertices_device(g, d)
            torch.cuda.synchronize()
            rcp.rcp_scene_validate(g)
        finally:
            rcp.rcp_scene_destroy(f)
    finally:
        rcp.rcp_scene_destroy(g)


def test_unknown_collapse_rejected():
    sc = scenes.tiny_scene()
    with pytest.raises(rcp.RcpError):
        U.gpu_scene(sc, 7)
    for bad in (-1, rcp.RCP_SPLIT_MAX + 1):
        with pytest.raises(rcp.RcpError):
            U.gpu_scene(sc, rcp.RCP_COLLAPSE_AREA, bad)


def _cone_rays(sc, n, seed):
    """Rays aimed at the forest's triangle vertices (cone apexes included) and
    at points on their edges, from random points around them."""
    rng = np.random.default_rng(seed)
    v = sc.tris.reshape(-1, 3, 3).astype(np.float64)
    pick = rng.integers(0, len(v), n)
    a, b = rng.integers(0, 3, n), rng.integers(0, 3, n)
    w = rng.choice([0.0, 0.5, 0.25, 1.0], n)[:, None]
    target = (1 - w) * v[pick, a] + w * v[pick, b]
    src = target + rng.normal(size=(n, 3)) * 20.0
    d = target - src
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ot = np.zeros((n, 4), np.float32)
    dt = np.zeros((n, 4), np.float32)
    ot[:, :3] = src
    dt[:, :3] = d
    dt[:, 3] = np.inf
    return ot, dt


def _walk_and_brute(g, ot, dt, any_hit):
    res = []
    for brute in (0, 1):
        t = torch.empty(len(ot), dtype=torch.float32, device="cuda")
        p = torch.empty(len(ot), dtype=torch.int32, device="cuda")
        rcp.rcp_debug_trace(g, len(ot), _dev(ot), _dev(dt), any_hit, brute, t, p)
        res.append((t.cpu().numpy(), p.cpu().numpy()))
    return res


@pytest.mark.parametrize("split", [0, 4, 8])
def test_split_references_equal_brute_force(split):
    """Triangles split into clipped references (and unsplit trees): the walk
    returns exactly what testing every primitive returns, also on rays aimed
    at vertices (the cone apexes, where all split pieces meet, and where two
    triangles tie at equal t) and at edges."""
    sc = scenes.forest_scene(60, seed=3)
    g = U.gpu_scene(sc, rcp.RCP_COLLAPSE_SAH, split)
    try:
        info = rcp.rcp_scene_get_info(g)
        if split > 1:
            assert info.n_records > 1.3 * sc.n_prims  # the cones' sides are split
        rcp.rcp_scene_validate(g)
        ot, dt = _cone_rays(sc, 30_000, seed=4 + split)
        for any_hit in (0, 1):
            (tw, pw), (tb, pb) = _walk_and_brute(g, ot, dt, any_hit)
            assert np.array_equal(pw, pb), (any_hit, int((pw != pb).sum()))
            if not any_hit:
                assert np.array_equal(tw.view(np.uint32), tb.view(np.uint32))
                assert (pb >= 0).mean() > 0.5
    finally:
        rcp.rcp_scene_destroy(g)


@pytest.mark.parametrize("motion", ["sway", "jitter"])
def test_split_scene_refit_stays_exact(motion):
    """A refit bounds each split reference by its part of the moved triangle:
    under the stress workload's sway (a translation per triangle) and under
    independent random moves of every vertex (which shear and scale each
    triangle), the refitted tree validates and its walk equals brute force
    bit for bit, twice in a row (parts are kept relative to the build)."""
    sc = scenes.forest_scene(40, seed=5)
    g = U.gpu_scene(sc, rcp.RCP_COLLAPSE_SAH, 8)
    rng = np.random.default_rng(19)
    try:
        for frame in (37, 90):
            if motion == "sway":
                moved = scenes.sway_vertices(sc.tris, sc.sway_amp, sc.sway_phase, frame)
            else:
                moved = (sc.tris + rng.normal(scale=0.4, size=sc.tris.shape)).astype(np.float32)
            rcp.rcp_scene_update_vertices(g, moved)
            rcp.rcp_scene_validate(g)
            msc = scenes.Scene("moved", moved, sc.spheres, sc.albedo, sc.light, sc.poses)
            ot, dt = _cone_rays(msc, 20_000, seed=11 + frame)
            for any_hit in (0, 1):
                (tw, pw), (tb, pb) = _walk_and_brute(g, ot, dt, any_hit)
                assert np.array_equal(pw, pb), (motion, frame, any_hit, int((pw != pb).sum()))
                if not any_hit:
                    assert np.array_equal(tw.view(np.uint32), tb.view(np.uint32))
    finally:
        rcp.rcp_scene_destroy(g)


def test_split_refit_keeps_the_clipped_boxes():
    """A refit with the build's own vertices leaves a split tree about as
    tight as the build made it (the parts' boxes equal the clipped boxes up
    to rounding and the pad), far tighter than the same tree bounded by whole
    triangles (the unsplit tree's triangle-test count stands in for that)."""
    sc = scenes.forest_scene(40, seed=5)
    d = sc.diameter()
    p = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    cam = rcp.camera_from(sc.poses[3])
    tests = {}
    for split in (0, 8):
        g = U.gpu_scene(sc, rcp.RCP_COLLAPSE_SAH, split)
        try:
            tests[split] = rcp.rcp_count_pass(g, cam, 320, 180, p).tri_tests
            if split:
                rcp.rcp_scene_update_vertices(g, sc.tris)
                tests["refit"] = rcp.rcp_count_pass(g, cam, 320, 180, p).tri_tests
        finally:
            rcp.rcp_scene_destroy(g)
    assert tests[8] < 0.6 * tests[0], tests
    assert tests["refit"] <= 1.02 * tests[8], tests


@pytest.mark.parametrize("name", ["mid", "forest"])
def test_collapse_policies_render_identical_images(name):
    """The collapse policies and triangle splitting walk different trees over
    the same primitives; ties go to the lower id, so the images are
    bit-identical."""
    sc = scenes.mid_scene() if name == "mid" else scenes.forest_scene()
    d = sc.diameter()
    p = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    imgs = []
    for collapse, split in [(rcp.RCP_COLLAPSE_AREA, 0), (rcp.RCP_COLLAPSE_SAH, 0), (rcp.RCP_COLLAPSE_SAH, 8)]:
        g = U.gpu_scene(sc, collapse, split)
        try:
            imgs.append([rcp.rcp_render(g, rcp.camera_from(sc.poses[i]), 480, 270, 6, p) for i in (3, 40)])
        finally:
            rcp.rcp_scene_destroy(g)
    for other in imgs[1:]:
        for a, b in zip(imgs[0], other):
            assert np.array_equal(a, b)
