"""The image-space reduction (§6, §6.1) on the GPU against the oracle.

A gather decides a pixel index from float32 arithmetic, which both sides do in
the same precision and order, so every comparison here is bit-exact, except
the end-to-end one, whose first pass is traced (FP32 against FP64)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu


def _images(W, H, seed):
    rng = np.random.default_rng(seed)
    base = rng.uniform(0, 1, size=(H, W, 4)).astype(np.float32)
    prev = rng.uniform(0, 1, size=(H, W, 4)).astype(np.float32)
    prev[: H // 5] = rng.choice([0.0, 0.5, 1.0], size=(H // 5, W, 4))  # exact extremes and mid-grey
    return base, prev


@pytest.mark.parametrize("W,H", [(1, 1), (7, 3), (257, 131), (1920, 1080)])
@pytest.mark.parametrize("k_px", [0.0, 1.0, 3.7, 50.0, 3000.0])
def test_pass_bit_exact(W, H, k_px):
    base, prev = _images(W, H, seed=W + H)
    db, dp = torch.from_numpy(base).cuda(), torch.from_numpy(prev).cuda()
    out = torch.empty_like(db)
    rcp.rcp_imagespace_pass_device(db, dp, out, W, H, k_px)
    torch.cuda.synchronize()
    want = O.imagespace_pass(base, prev, W, H, k_px).reshape(H, W, 4)
    assert np.array_equal(out.cpu().numpy(), want)


def test_render_chain_bit_exact():
    """K-pass render with RCP_MAP_IMAGE = traced pass 1, then K-1 gathers of it."""
    sc = scenes.tiny_scene()
    g = U.gpu_scene(sc)
    try:
        W, H, K, kpx = 160, 120, 6, 4.0
        cam = rcp.camera_from(sc.poses[0])
        p = rcp.make_params(rcp.RCP_MAP_IMAGE, kpx, 6.0)
        traced = rcp.rcp_render_pass(g, cam, W, H, rcp.make_params(rcp.RCP_MAP_TARGET, 0.0, 6.0))
        out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        rcp.rcp_render_device(g, cam, W, H, K, p, None, out, None, torch.cuda.current_stream())
        torch.cuda.synchronize()
        img = traced
        for _ in range(K - 1):
            img = O.imagespace_pass(traced, img, W, H, kpx).reshape(H, W, 4)
        assert np.array_equal(out.cpu().numpy(), img)
        host = rcp.rcp_render(g, cam, W, H, K, p)
        assert np.array_equal(host, img[..., :3])
        # batched views with the image mapping equal the single-view renders
        outs = [torch.empty((h, w, 4), dtype=torch.float32, device="cuda") for w, h in [(W, H), (97, 61)]]
        rcp.rcp_render_batch_device(g, [cam, cam], [W, 97], [H, 61], K, p, outs)
        torch.cuda.synchronize()
        assert np.array_equal(outs[0].cpu().numpy(), img)
        assert np.array_equal(outs[1].cpu().numpy()[..., :3], rcp.rcp_render(g, cam, 97, 61, K, p))
        with pytest.raises(rcp.RcpError):
            rcp.rcp_render_pass(g, cam, W, H, p)
    finally:
        rcp.rcp_scene_destroy(g)


def test_end_to_end_against_fp64_oracle():
    sc = scenes.mid_scene()
    g = U.gpu_scene(sc)
    o = U.oracle_scene(sc)
    try:
        W, H, K, kpx = 480, 270, 6, 6.0
        d = sc.diameter()
        cam = sc.poses[9]
        f = U.f32(0.1 * d)
        out = rcp.rcp_render(g, rcp.camera_from(cam), W, H, K, rcp.make_params(rcp.RCP_MAP_IMAGE, kpx, f))
        traced, _, _ = o.render_pass(U.cam_f32(cam), W, H, O.MAP_TARGET, 0.0, f)
        traced = traced.astype(np.float32).reshape(H, W, 4)
        img = traced
        for _ in range(K - 1):
            img = O.imagespace_pass(traced, img, W, H, kpx).reshape(H, W, 4)
        p = U.psnr(out, img[..., :3])
        print(f"image-space mid {W}x{H} K={K}: PSNR {p:.1f} dB")
        assert p >= U.PSNR_MIN
    finally:
        rcp.rcp_scene_destroy(g)


def test_argument_checks():
    a = torch.zeros((4, 4, 4), dtype=torch.float32, device="cuda")
    b = torch.zeros_like(a)
    with pytest.raises(rcp.RcpError):
        rcp.rcp_imagespace_pass_device(a, b, a, 4, 4, 1.0)  # out aliases base
    with pytest.raises(rcp.RcpError):
        rcp.rcp_imagespace_pass_device(a, b, torch.zeros_like(a), 4, 4, -1.0)
    with pytest.raises(rcp.RcpError):
        rcp.rcp_imagespace_pass_device(a, b, torch.zeros_like(a), 0, 4, 1.0)
