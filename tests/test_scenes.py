"""The seeded workload generators: sizes, determinism and shape."""
import numpy as np

from paper_2312_12392_gb300 import scenes


def test_sizes_match_the_workloads():
    assert scenes.tiny_scene().n_prims == 5
    assert scenes.mid_scene().n_tris == 256 * 256 * 2 + 200 * 12 == 133_472
    f = scenes.forest_scene()
    assert f.n_tris == 181 * 181 * 2 + 2000 * 500 == 1_065_522
    for grid, n in [(221, 100_082), (706, 999_272)]:
        assert scenes.terrain_scene(grid, seed=4).n_tris == n


def test_deterministic():
    a, b = scenes.mid_scene(), scenes.mid_scene()
    assert np.array_equal(a.tris, b.tris) and np.array_equal(a.albedo, b.albedo)
    assert [p.eye for p in a.poses] == [p.eye for p in b.poses]
    assert not np.array_equal(scenes.terrain_scene(64, seed=1).tris, scenes.terrain_scene(64, seed=2).tris)


def test_arrays_and_ranges():
    t = scenes.tiny_scene()
    assert t.tris.dtype == np.float32 and t.tris.flags["C_CONTIGUOUS"] and t.tris.shape == (2, 9)
    c = t.spheres[:, :3]
    assert np.all(np.abs(c[:, [0, 2]]) <= 3) and np.all((c[:, 1] >= 1) & (c[:, 1] <= 2))
    assert np.all((t.albedo[2:] >= 0.2) & (t.albedo[2:] <= 0.9))
    assert abs(t.diameter() - np.linalg.norm([20, c[:, 1].max() + 1, 20])) < 1e-6
    m = scenes.mid_scene()
    assert len(m.poses) == 64 and m.light.type == scenes.LIGHT_DIRECTIONAL
    assert np.all((m.albedo >= 0.1) & (m.albedo <= 0.9))


def test_catmull_rom_passes_through_control_points():
    P = np.array([[0, 0], [1, 0], [2, 1], [3, 3], [5, 3]], float)
    pos, tan = scenes.catmull_rom_centripetal(P, 4)
    # samples at the start of each of the 2 segments hit P1 and P2
    assert np.allclose(pos[0], P[1]) and np.allclose(pos[2], P[2])
    assert np.allclose(np.linalg.norm(tan, axis=1), 1.0)


def test_pixel_subset_and_requests():
    s = scenes.pixel_subset(1920, 1080, 4096, seed=3)
    assert len(s) == len(np.unique(s)) == 4096 and s.min() >= 0 and s.max() < 1920 * 1080
    assert np.array_equal(s, scenes.pixel_subset(1920, 1080, 4096, seed=3))
    assert len(scenes.pixel_subset(4, 3, 100, seed=0)) == 12
    reqs = scenes.served_requests(200, 4, 64)
    assert {r["K"] for r in reqs} <= set(range(1, 9)) and all(0 <= r["k_frac"] <= 0.05 for r in reqs)
    sizes = scenes.batched_view_sizes(64)
    assert all(256 <= w <= 1920 and 256 <= h <= 1080 for w, h in sizes)
    arr = scenes.poisson_arrivals(50.0, 1000)
    assert abs(np.mean(np.diff(arr)) - 1 / 50.0) < 0.2 / 50.0


def test_blocks_scene_integer_grid():
    a = scenes.blocks_scene(8, n_cubes=10, seed=3)
    b = scenes.blocks_scene(8, n_cubes=10, seed=3)
    assert np.array_equal(a.tris, b.tris)
    # 2 triangles per floor quad, 12 per stacked unit cube
    assert (a.n_tris - 2 * 8 * 8) % 12 == 0 and a.n_tris > 2 * 8 * 8
    assert np.array_equal(a.tris, np.round(a.tris))
    floor = a.tris[: 2 * 8 * 8].reshape(-1, 3, 3)
    assert np.all(floor[:, :, 1] == 0.0)
    off = scenes.blocks_scene(8, n_cubes=10, seed=3, offset=(1e4, 0.0, -5e3))
    assert np.array_equal(off.tris - np.tile(np.float32([1e4, 0.0, -5e3]), 3), a.tris)
