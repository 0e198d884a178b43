"""rcp_render's host output. On a device that reads and writes pageable host
memory coherently, the last pass may write the caller's RGB straight into host
memory while it traces (rcp_set_host_output: always, never, or for buffers
written that way recently); otherwise, and for the image-space mapping, a pack
kernel and a copy deliver it. Every way the host image must equal the device
path's image (its RGB lanes) bit for bit: every mapping, jittered samples,
ragged sizes, K = 1, fresh buffers and a reused one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [
    # (mapping, k as a fraction of the diameter (IMAGE: pixels), jitter samples, W, H, K)
    (rcp.RCP_MAP_EYE, 0.03, 0, 97, 61, 6),
    (rcp.RCP_MAP_EYE, 0.03, 0, 64, 48, 1),
    (rcp.RCP_MAP_TARGET, 0.05, 0, 128, 72, 3),
    (rcp.RCP_MAP_DEPTH, 0.02, 0, 81, 33, 4),
    (rcp.RCP_MAP_NORMAL, 0.02, 0, 50, 70, 3),
    (rcp.RCP_MAP_EYE, 0.03, 4, 67, 45, 3),
    (rcp.RCP_MAP_IMAGE, 6.0, 0, 96, 64, 3),
]


@pytest.fixture(scope="module")
def mid_g():
    sc = scenes.mid_scene()
    g = U.gpu_scene(sc)
    yield sc, g
    rcp.rcp_scene_destroy(g)


def _params(sc, mapping, kf, spp):
    d = sc.diameter()
    k = kf if mapping == rcp.RCP_MAP_IMAGE else kf * d
    jitter = None
    if spp:
        jitter = np.random.default_rng(spp).random((spp, 2))
    return rcp.make_params(mapping, k, 0.1 * d, jitter=jitter)


@pytest.fixture(params=[rcp.RCP_HOST_OUTPUT_AUTO, rcp.RCP_HOST_OUTPUT_DIRECT, rcp.RCP_HOST_OUTPUT_COPY])
def host_mode(request):
    rcp.rcp_set_host_output(request.param)
    yield request.param
    rcp.rcp_set_host_output(rcp.RCP_HOST_OUTPUT_AUTO)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_host_image_equals_device_image(mid_g, case, host_mode):
    sc, g = mid_g
    mapping, kf, spp, W, H, K = CASES[case]
    p = _params(sc, mapping, kf, spp)
    cam = rcp.camera_from(sc.poses[case % len(sc.poses)])
    d_out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    rcp.rcp_render_device(g, cam, W, H, K, p, None, d_out, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref = np.ascontiguousarray(d_out[..., :3].cpu().numpy())
    host = rcp.rcp_render(g, cam, W, H, K, p)  # a fresh, never-touched buffer
    assert host.shape == (H, W, 3)
    assert np.array_equal(host.view(np.uint32), ref.view(np.uint32))


def test_reused_buffer_is_overwritten(mid_g, host_mode):
    """One buffer through renders of different sizes' worth of poses: every
    call leaves exactly its own image, no pixel of the previous one."""
    sc, g = mid_g
    W, H = 160, 90
    p = _params(sc, rcp.RCP_MAP_EYE, 0.03, 0)
    buf = np.full((H, W, 3), np.nan, np.float32)
    for i in range(3):
        cam = rcp.camera_from(sc.poses[5 * i])
        d_out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        rcp.rcp_render_device(g, cam, W, H, 6, p, None, d_out, None, torch.cuda.current_stream())
        torch.cuda.synchronize()
        ref = d_out[..., :3].cpu().numpy()
        out = rcp.rcp_render(g, cam, W, H, 6, p, buf)
        assert out is buf
        assert np.array_equal(buf, ref)


def test_page_locked_buffer(mid_g):
    """A page-locked buffer is written directly by the last pass (through the
    GPU's page tables) under every policy but COPY, with the same image."""
    sc, g = mid_g
    W, H = 131, 77
    p = _params(sc, rcp.RCP_MAP_EYE, 0.03, 0)
    cam = rcp.camera_from(sc.poses[9])
    d_out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    rcp.rcp_render_device(g, cam, W, H, 4, p, None, d_out, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref = d_out[..., :3].cpu().numpy()
    buf = torch.full((H, W, 3), float("nan"), dtype=torch.float32, pin_memory=True).numpy()
    for mode in (rcp.RCP_HOST_OUTPUT_AUTO, rcp.RCP_HOST_OUTPUT_COPY):
        rcp.rcp_set_host_output(mode)
        try:
            buf[...] = np.nan
            assert rcp.rcp_render(g, cam, W, H, 4, p, buf) is buf
            assert np.array_equal(buf, ref)
        finally:
            rcp.rcp_set_host_output(rcp.RCP_HOST_OUTPUT_AUTO)
