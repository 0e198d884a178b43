"""Per-frame refit under wind sway (the stress workload at reduced size): after
every swayed frame the refitted BVH is valid, its walk equals brute force over
every primitive, and a rendered pass matches the oracle on the moved scene."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_oracle_golden as G  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("collapse,split", [(None, 0), (rcp.RCP_COLLAPSE_SAH, 8)])
def test_swaying_forest_refit_parity(collapse, split):
    """Unsplit trees, and the stress workload's build (surface-area collapse,
    split references refitted by their parts of the moved triangles)."""
    sc = scenes.forest_scene(60, seed=5)
    g = U.gpu_scene(sc, collapse, split)
    try:
        d = sc.diameter()
        W, H = 320, 180
        for frame in (1, 17, 45):
            moved = scenes.sway_vertices(sc.tris, sc.sway_amp, sc.sway_phase, frame)
            rcp.rcp_scene_update_vertices(g, moved)
            rcp.rcp_scene_validate(g)
            n = 8000
            ot, dt = U.random_rays(n, seed=frame, extent=d / 6, towards=(0, 2, 0))
            res = []
            for brute in (0, 1):
                t = torch.empty(n, dtype=torch.float32, device="cuda")
                p = torch.empty(n, dtype=torch.int32, device="cuda")
                rcp.rcp_debug_trace(g, n, torch.from_numpy(ot).cuda(), torch.from_numpy(dt).cuda(), 0, brute, t, p)
                res.append((t.cpu().numpy(), p.cpu().numpy()))
            assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][0], res[1][0])
            moved_sc = scenes.Scene("moved", moved, sc.spheres, sc.albedo, sc.light, sc.poses)
            pix = scenes.pixel_subset(W, H, 1500, seed=frame)
            rep = U.per_pass_parity(moved_sc, sc.poses[frame % 64], W, H, 2, rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d,
                                    pix=pix, g=g)
            rep.assert_ok(f"sway frame {frame}")
    finally:
        rcp.rcp_scene_destroy(g)


def test_served_two_copy_stream_equals_single_stream():
    """The stress workload's serving path (two copies of a swaying scene,
    refitted in turn while the other renders) delivers the same frames as one
    stream that refits and renders frame after frame."""
    sc = scenes.forest_scene(40, seed=5)
    d = sc.diameter()
    W, H, K = 320, 180, 3
    p = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    frames = [0, 7, 13, 29, 30]
    g = U.gpu_scene(sc)
    g2 = U.gpu_scene(sc)
    srv = rcp.rcp_server_create(1 << 30, 4)
    try:
        single = []
        for f in frames:
            rcp.rcp_scene_update_vertices(g, scenes.sway_vertices(sc.tris, sc.sway_amp, sc.sway_phase, f))
            single.append(rcp.rcp_render(g, rcp.camera_from(sc.poses[f]), W, H, K, p))
        copies, outs, tickets = [g, g2], [np.zeros((H, W, 3), np.float32) for _ in frames], []
        for i, f in enumerate(frames):
            if i >= 2:
                rcp.rcp_server_wait(srv, tickets[i - 2], 60.0)
            rcp.rcp_scene_update_vertices(copies[i % 2], scenes.sway_vertices(sc.tris, sc.sway_amp, sc.sway_phase, f))
            tickets.append(rcp.rcp_server_submit(srv, copies[i % 2], rcp.camera_from(sc.poses[f]), W, H, K, p,
                                                 outs[i]))
        for tk in tickets:
            rcp.rcp_server_wait(srv, tk, 60.0)
        for a, b in zip(single, outs):
            assert np.array_equal(a, b)
    finally:
        rcp.rcp_server_destroy(srv)
        rcp.rcp_scene_destroy(g2)
        rcp.rcp_scene_destroy(g)


def _vertex_rays(tris, n, seed, dist):
    """Rays from random points at distance ~dist aimed at triangle vertices and
    at points on their edges (where split references meet)."""
    rng = np.random.default_rng(seed)
    v = tris.reshape(-1, 3, 3).astype(np.float64)
    pick = rng.integers(0, len(v), n)
    a, b = rng.integers(0, 3, n), rng.integers(0, 3, n)
    w = rng.choice([0.0, 0.5, 0.25, 1.0], n)[:, None]
    target = (1 - w) * v[pick, a] + w * v[pick, b]
    src = target + rng.normal(size=(n, 3)) * dist
    src[:, 1] = np.abs(src[:, 1] - target[:, 1]) + target[:, 1]  # from above
    d = target - src
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ot = np.zeros((n, 4), np.float32)
    dt = np.zeros((n, 4), np.float32)
    ot[:, :3] = src
    dt[:, :3] = d
    dt[:, 3] = np.inf
    return ot, dt


def test_full_size_stress_parity():
    """The stress workload at full size in the bench's build: 25,000 swaying
    cone trees (12.57M triangles), surface-area collapse with split <= 8,
    refitted to a swayed frame. The refitted tree validates; its walk equals
    brute force over every record on rays aimed at vertices and edges; and
    4,096 sampled pixels of a 3840x2160, K=8 chain match the oracle pass by
    pass (values the oracle wrote beforehand, tests/golden/make_oracle_golden.py:
    the brute-force oracle needs about ten minutes of the host's cores for
    them)."""
    gd, meta = G.load("stress")
    sc = scenes.forest_scene(25_000, seed=5)
    g = U.gpu_scene(sc, rcp.RCP_COLLAPSE_SAH, 8)
    try:
        info = rcp.rcp_scene_get_info(g)
        assert info.n_tris == 12_565_522 and info.n_records > 4 * info.n_tris
        frame = 123
        assert meta["poses"] == [frame % len(sc.poses)]
        moved = scenes.sway_vertices(sc.tris, sc.sway_amp, sc.sway_phase, frame)
        rcp.rcp_scene_update_vertices(g, moved)
        rcp.rcp_scene_validate(g)
        n = 4096
        ot, dt = _vertex_rays(moved, n, seed=frame, dist=20.0)
        res = []
        for brute in (0, 1):
            t = torch.empty(n, dtype=torch.float32, device="cuda")
            p = torch.empty(n, dtype=torch.int32, device="cuda")
            rcp.rcp_debug_trace(g, n, torch.from_numpy(ot).cuda(), torch.from_numpy(dt).cuda(), 0, brute, t, p)
            res.append((t.cpu().numpy(), p.cpu().numpy()))
        assert (res[1][1] >= 0).sum() > n // 2
        assert np.array_equal(res[0][1], res[1][1])
        assert np.array_equal(res[0][0].view(np.uint32), res[1][0].view(np.uint32))
        W, H, K = meta["W"], meta["H"], meta["K"]
        cam_o = sc.poses[meta["poses"][0]].as_array().astype(np.float32).astype(np.float64)
        pix = gd["pix_0"]
        k, f = G.params_of(dict(diam=sc.diameter()))
        assert G.input_hash(moved, sc.albedo, [cam_o], [pix], (k, f)) == meta["inputs"], "stress golden inputs differ"
        params = rcp.make_params(rcp.RCP_MAP_EYE, k, f)
        cam = rcp.camera_from(sc.poses[meta["poses"][0]])
        rep = U.PassReport()
        img = None
        for n in range(K):
            prim = np.empty(H * W, np.int32)
            out = rcp.rcp_render_pass(g, cam, W, H, params, in_rgbz=img, out_prim=prim)
            o_rgbz = gd["rgbz_0"][n].astype(np.float64)
            rep.add(out.reshape(-1, 4)[pix], prim[pix], o_rgbz, gd["prim_0"][n], gd["flag_0"][n])
            img = U.next_image(out, pix, o_rgbz, rcp.RCP_MAP_EYE).reshape(H, W, 4)
        print(rep.assert_ok(f"stress frame {frame}"))
    finally:
        rcp.rcp_scene_destroy(g)
