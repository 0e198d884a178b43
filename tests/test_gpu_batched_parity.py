"""Many views of uneven size in one persistent launch per pass, against the
FP64 oracle (§2: every (u,v) of every image gets its own camera; the launch's
tile queue spans all views, and each view's pixels must come out exactly as
the oracle computes them for that view's camera and size).

Per pass: each pass is one batched launch (rcp_render_batch_device, K = 1)
whose per-view inputs carry the oracle's previous values on the sampled
pixels. End to end: one K = 6 batched render from I_0 (the captured K-pass
graph) against the oracle's chains, by PSNR.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu


def _views(sc, n_views, seed):
    sizes = scenes.batched_view_sizes(n_views, seed=seed)
    poses = [(7 * i + 3) % len(sc.poses) for i in range(n_views)]
    return sizes, poses


def _batched_parity(sc, g, n_views, samples, K_pass, K_e2e, seed):
    d = sc.diameter()
    k, f = U.f32(0.02 * d), U.f32(0.1 * d)
    params = rcp.make_params(rcp.RCP_MAP_EYE, k, f)
    o = U.oracle_scene(sc)
    sizes, poses = _views(sc, n_views, seed)
    assert len({w * h for w, h in sizes}) == n_views  # uneven
    cams = [rcp.camera_from(sc.poses[p]) for p in poses]
    camo = [U.cam_f32(sc.poses[p]) for p in poses]
    Ws, Hs = [w for w, _ in sizes], [h for _, h in sizes]
    pixs = [scenes.pixel_subset(w, h, samples, seed=seed * 100 + i) for i, (w, h) in enumerate(sizes)]
    reps = [U.PassReport() for _ in sizes]
    ins = [None] * n_views
    for n in range(K_pass):
        outs = [torch.empty((h, w, 4), dtype=torch.float32, device="cuda") for w, h in sizes]
        prims = [torch.empty((h, w), dtype=torch.int32, device="cuda") for w, h in sizes]
        rcp.rcp_render_batch_device(g, cams, Ws, Hs, 1, params, outs, torch.cuda.current_stream(),
                                    d_ins=[None if x is None else torch.from_numpy(x).cuda() for x in ins],
                                    d_prims=prims)
        torch.cuda.synchronize()
        for i, (w, h) in enumerate(sizes):
            out = outs[i].cpu().numpy()
            prim = prims[i].cpu().numpy().reshape(-1)
            o_rgbz, o_prim, o_flag = o.render_pass(camo[i], w, h, rcp.RCP_MAP_EYE, k, f, in_rgbz=ins[i],
                                                   pix=pixs[i])
            reps[i].add(out.reshape(-1, 4)[pixs[i]], prim[pixs[i]], o_rgbz, o_prim, o_flag)
            ins[i] = U.next_image(out, pixs[i], o_rgbz, rcp.RCP_MAP_EYE).reshape(h, w, 4)
    for i, (w, h) in enumerate(sizes):
        print(reps[i].assert_ok(f"{sc.name} view {i} {w}x{h} pose {poses[i]}"))
    # end to end: one batched K-pass render from I_0
    outs = [torch.empty((h, w, 4), dtype=torch.float32, device="cuda") for w, h in sizes]
    rcp.rcp_render_batch_device(g, cams, Ws, Hs, K_e2e, params, outs, torch.cuda.current_stream())
    torch.cuda.synchronize()
    for i, (w, h) in enumerate(sizes):
        ref, _, fl = o.render(camo[i], w, h, K_e2e, rcp.RCP_MAP_EYE, k, f, pix=pixs[i])
        p = U.psnr(outs[i].cpu().numpy().reshape(-1, 4)[pixs[i], :3], ref[:, :3])
        print(f"{sc.name} view {i} {w}x{h}: K={K_e2e} PSNR {p:.1f} dB, flagged chains {float((fl != 0).mean()):.4f}")
        assert p >= U.PSNR_MIN


def test_mid_batched_views():
    sc = scenes.mid_scene()
    g = U.gpu_scene(sc)
    try:
        _batched_parity(sc, g, n_views=8, samples=2048, K_pass=6, K_e2e=6, seed=3)
    finally:
        rcp.rcp_scene_destroy(g)


def test_forest_batched_views():
    """The forest in the benchmark's build (surface-area collapse, split <= 8)."""
    sc = scenes.forest_scene()
    g = U.gpu_scene(sc, rcp.RCP_COLLAPSE_SAH, 8)
    try:
        _batched_parity(sc, g, n_views=6, samples=384, K_pass=4, K_e2e=6, seed=5)
    finally:
        rcp.rcp_scene_destroy(g)
