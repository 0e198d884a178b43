"""Jittered multi-sample passes (§2: any number of samples per pixel at jittered
(u,v)) and temporal feedback (a frame's pass continues from the previous
frame's image, Eq. 1 with S(n) a time step), on the GPU against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu

JIT4 = np.array([[0.125, 0.375], [0.625, 0.125], [0.375, 0.875], [0.875, 0.625]], np.float32)


def test_centre_sample_is_the_single_sample_path():
    sc = scenes.tiny_scene()
    g = U.gpu_scene(sc)
    try:
        cam = rcp.camera_from(sc.poses[0])
        W, H = 96, 64
        a = rcp.rcp_render(g, cam, W, H, 4, rcp.make_params(rcp.RCP_MAP_EYE, 1.4, 6.0))
        b = rcp.rcp_render(g, cam, W, H, 4, rcp.make_params(rcp.RCP_MAP_EYE, 1.4, 6.0, jitter=[[0.5, 0.5]]))
        assert np.array_equal(a, b)
        c = rcp.rcp_render(g, cam, W, H, 4, rcp.make_params(rcp.RCP_MAP_EYE, 1.4, 6.0, jitter=[[0.5, 0.5]] * 4))
        assert np.abs(c - a).max() <= 1e-6
    finally:
        rcp.rcp_scene_destroy(g)


def _ms_parity(sc, cam, W, H, K, mapping, k, f, jit, pix=None):
    g = U.gpu_scene(sc)
    o = U.oracle_scene(sc)
    k, f = U.f32(k), U.f32(f)
    params = rcp.make_params(mapping, k, f, jitter=jit)
    rep = U.PassReport()
    idx = np.arange(W * H) if pix is None else np.asarray(pix)
    img = None
    try:
        for _ in range(K):
            prim = np.empty(W * H, np.int32)
            out = rcp.rcp_render_pass(g, rcp.camera_from(cam), W, H, params, in_rgbz=img, out_prim=prim)
            o_rgbz, o_prim, o_flag, o_n = o.render_pass_ms(U.cam_f32(cam), W, H, mapping, k, f, jit, in_rgbz=img,
                                                           pix=pix, in_normal=U.oracle_normals(img, mapping),
                                                           want_normal=True)
            rep.add(out.reshape(-1, 4)[idx], prim[idx], o_rgbz, o_prim, o_flag)
            # samples read their neighbours: the next input is the GPU's whole
            # image with the oracle's values on the compared pixels
            img = U.next_image(out, idx, o_rgbz, mapping, o_n).reshape(H, W, 4)
    finally:
        rcp.rcp_scene_destroy(g)
    return rep


def test_tiny_per_pass_parity():
    sc = scenes.tiny_scene()
    rep = _ms_parity(sc, sc.poses[0], 96, 72, 4, rcp.RCP_MAP_EYE, 0.05 * sc.diameter(), 6.0, JIT4)
    print(rep.assert_ok("tiny 4 spp"))


def test_mid_per_pass_parity_sample():
    sc = scenes.mid_scene()
    d = sc.diameter()
    W, H = 960, 540
    pix = scenes.pixel_subset(W, H, 1024, seed=9)
    rep = _ms_parity(sc, sc.poses[30], W, H, 3, rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d, JIT4, pix=pix)
    print(rep.assert_ok("mid 4 spp"))


@pytest.mark.parametrize("mapping", [rcp.RCP_MAP_EYE, rcp.RCP_MAP_NORMAL])
def test_tiny_end_to_end_psnr(mapping):
    sc = scenes.tiny_scene()
    g = U.gpu_scene(sc)
    o = U.oracle_scene(sc)
    try:
        W, H, K = 64, 48, 4
        k = U.f32(0.05 * sc.diameter())
        out = rcp.rcp_render(g, rcp.camera_from(sc.poses[0]), W, H, K, rcp.make_params(mapping, k, 6.0, jitter=JIT4))
        ref, flag = o.render_ms(U.cam_f32(sc.poses[0]), W, H, K, mapping, k, 6.0, JIT4)
        p = U.psnr(out.reshape(-1, 3), ref[:, :3])
        print(f"tiny 4 spp K={K} mapping {mapping}: PSNR {p:.1f} dB, flagged {float((flag != 0).mean()):.4f}")
        assert p >= U.PSNR_MIN
    finally:
        rcp.rcp_scene_destroy(g)


def test_temporal_feedback_chain():
    """Frames that each run one pass from the previous frame's image equal one
    K-pass render when the camera does not move; with a moving camera every
    frame continues from the last one (device path, in place)."""
    sc = scenes.mid_scene()
    g = U.gpu_scene(sc)
    try:
        d = sc.diameter()
        W, H = 320, 180
        p = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
        cam = rcp.camera_from(sc.poses[4])
        buf = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        rcp.rcp_render_device(g, cam, W, H, 1, p, None, buf, None, torch.cuda.current_stream())
        for _ in range(4):
            rcp.rcp_render_device(g, cam, W, H, 1, p, buf, buf, None, torch.cuda.current_stream())
        torch.cuda.synchronize()
        five = rcp.rcp_render(g, cam, W, H, 5, p)
        assert np.array_equal(buf.cpu().numpy()[..., :3], five)
        prev = None
        for i in range(3):  # walk-through frames
            c = rcp.camera_from(sc.poses[10 + i])
            host = rcp.rcp_render_pass(g, c, W, H, p, in_rgbz=prev)
            dev_in = None if prev is None else torch.from_numpy(prev).cuda()
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
            rcp.rcp_render_device(g, c, W, H, 1, p, dev_in, out, None, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert np.array_equal(out.cpu().numpy(), host)
            prev = host
    finally:
        rcp.rcp_scene_destroy(g)


def test_in_place_one_pass_multisample_rejected():
    sc = scenes.tiny_scene()
    g = U.gpu_scene(sc)
    try:
        buf = torch.zeros((8, 8, 4), dtype=torch.float32, device="cuda")
        p = rcp.make_params(rcp.RCP_MAP_EYE, 1.0, 6.0, jitter=JIT4)
        with pytest.raises(rcp.RcpError):
            rcp.rcp_render_device(g, rcp.camera_from(sc.poses[0]), 8, 8, 1, p, buf, buf, None,
                                  torch.cuda.current_stream())
    finally:
        rcp.rcp_scene_destroy(g)


def test_bad_jitter_rejected():
    sc = scenes.tiny_scene()
    g = U.gpu_scene(sc)
    try:
        cam = rcp.camera_from(sc.poses[0])
        with pytest.raises(rcp.RcpError):
            rcp.rcp_render(g, cam, 8, 8, 1, rcp.make_params(rcp.RCP_MAP_EYE, 1.0, 6.0, jitter=[[1.0, 0.5]]))
        with pytest.raises(rcp.RcpError):
            rcp.rcp_render(g, cam, 8, 8, 2, rcp.make_params(rcp.RCP_MAP_IMAGE, 1.0, 6.0, jitter=[[0.5, 0.5]]))
    finally:
        rcp.rcp_scene_destroy(g)
