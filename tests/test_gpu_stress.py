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
