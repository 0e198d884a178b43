"""Per-frame refit under wind sway (the stress workload at reduced size): after
every swayed frame the refitted BVH is valid, its walk equals brute force over
every primitive, and a rendered pass matches the oracle on the moved scene."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu


def test_swaying_forest_refit_parity():
    sc = scenes.forest_scene(60, seed=5)
    g = U.gpu_scene(sc)
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
