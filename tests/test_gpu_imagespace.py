"""The image-space reduction (§6, §6.1) on the GPU against the oracle.

The oracle evaluates the gather's displaced coordinate in double and flags
samples within its rounding band of a half-integer (where a float32 evaluation
may take the neighbouring pixel). Off the flag every gathered pixel is the
oracle's, bit for bit; on it, the GPU's pixel is the oracle's or an adjacent
one. The end-to-end test compares against the FP64 chain by PSNR (its first
pass is traced)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu


def _images(W, H, seed):
    """base: each pixel holds its own column and row (so a gathered value names
    its source pixel) and two random lanes; prev: random colours, a fifth of
    the rows exact extremes and mid-grey."""
    rng = np.random.default_rng(seed)
    base = rng.uniform(0, 1, size=(H, W, 4)).astype(np.float32)
    base[..., 0] = np.arange(W, dtype=np.float32)[None, :]
    base[..., 1] = np.arange(H, dtype=np.float32)[:, None]
    prev = rng.uniform(0, 1, size=(H, W, 4)).astype(np.float32)
    prev[: H // 5] = rng.choice([0.0, 0.5, 1.0], size=(H // 5, W, 4))
    return base, prev


def _check_gather(got, want, flag, label):
    """Bit-exact off the flag; on it, the source pixel is the oracle's or adjacent."""
    got, want = got.reshape(-1, 4), want.reshape(-1, 4)
    fl = flag.astype(bool)
    assert np.array_equal(got[~fl].view(np.uint32), want[~fl].view(np.uint32)), label
    near = (np.abs(got[fl, 0] - want[fl, 0]) <= 1) & (np.abs(got[fl, 1] - want[fl, 1]) <= 1)
    assert near.all(), label
    return float(fl.mean())


@pytest.mark.parametrize("W,H", [(1, 1), (7, 3), (257, 131), (1920, 1080)])
@pytest.mark.parametrize("k_px", [0.0, 1.0, 3.7, 50.0, 3000.0])
def test_pass_against_oracle(W, H, k_px):
    base, prev = _images(W, H, seed=W + H)
    db, dp = torch.from_numpy(base).cuda(), torch.from_numpy(prev).cuda()
    out = torch.empty_like(db)
    rcp.rcp_imagespace_pass_device(db, dp, out, W, H, k_px)
    torch.cuda.synchronize()
    want, flag = O.imagespace_pass(base, prev, W, H, k_px, want_flag=True)
    frac = _check_gather(out.cpu().numpy(), want, flag, f"{W}x{H} k={k_px}")
    assert frac <= 0.02 or flag.sum() <= 2, frac  # a band of a few 1e-3 pixels per axis


def test_render_chain():
    """The K-pass device render with RCP_MAP_IMAGE is its traced pass 1 followed
    by K-1 gathers of it; each gather, given the oracle's traced image and the
    oracle's previous pass, matches the oracle's gather."""
    sc = scenes.tiny_scene()
    g = U.gpu_scene(sc)
    o = U.oracle_scene(sc)
    try:
        W, H, K, kpx = 160, 120, 6, 4.0
        cam = rcp.camera_from(sc.poses[0])
        p = rcp.make_params(rcp.RCP_MAP_IMAGE, kpx, 6.0)
        # (a) the render path is the traced image followed by gathers of it
        traced_g = torch.from_numpy(rcp.rcp_render_pass(g, cam, W, H, rcp.make_params(rcp.RCP_MAP_TARGET, 0.0, 6.0)))
        traced_g = traced_g.cuda()
        chain = traced_g.clone()
        for _ in range(K - 1):
            nxt = torch.empty_like(chain)
            rcp.rcp_imagespace_pass_device(traced_g, chain, nxt, W, H, kpx)
            chain = nxt
        out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        rcp.rcp_render_device(g, cam, W, H, K, p, None, out, None, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.equal(out, chain)
        host = rcp.rcp_render(g, cam, W, H, K, p)
        assert np.array_equal(host, chain.cpu().numpy()[..., :3])
        # batched views with the image mapping equal the single-view renders
        outs = [torch.empty((h, w, 4), dtype=torch.float32, device="cuda") for w, h in [(W, H), (97, 61)]]
        rcp.rcp_render_batch_device(g, [cam, cam], [W, 97], [H, 61], K, p, outs)
        torch.cuda.synchronize()
        assert torch.equal(outs[0], chain)
        assert np.array_equal(outs[1].cpu().numpy()[..., :3], rcp.rcp_render(g, cam, 97, 61, K, p))
        with pytest.raises(rcp.RcpError):
            rcp.rcp_render_pass(g, cam, W, H, p)
        # (b) per pass against the oracle, on the oracle's own traced image
        traced, _, _ = o.render_pass(U.cam_f32(sc.poses[0]), W, H, O.MAP_TARGET, 0.0, 6.0)
        traced = traced.astype(np.float32).reshape(H, W, 4)
        db = torch.from_numpy(traced).cuda()
        img = traced
        for n in range(K - 1):
            nxt = torch.empty_like(db)
            rcp.rcp_imagespace_pass_device(db, torch.from_numpy(img).cuda(), nxt, W, H, kpx)
            torch.cuda.synchronize()
            want, flag = O.imagespace_pass(traced, img, W, H, kpx, want_flag=True)
            got = nxt.cpu().numpy()
            fl = flag.astype(bool)
            assert np.array_equal(got.reshape(-1, 4)[~fl], want[~fl]), f"gather {n + 2}"
            assert fl.mean() <= 0.02
            img = want.reshape(H, W, 4)
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
