"""Invariants of the CUDA path that hold bit-exactly (no oracle needed):
k = 0 and mid-grey (§3) leave every pass equal to the pinhole pass; launch
shapes, the fused/separate camera kernel, batching and graph replay do not
change any pixel; degenerate inputs and argument errors behave."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny_g():
    sc = scenes.tiny_scene()
    g = U.gpu_scene(sc)
    yield sc, g
    rcp.rcp_scene_destroy(g)


def _render(g, cam, W, H, K, params):
    return rcp.rcp_render(g, cam, W, H, K, params)


def test_zero_k_every_pass_is_pinhole(tiny_g):
    sc, g = tiny_g
    cam = rcp.camera_from(sc.poses[0])
    one = _render(g, cam, 128, 128, 1, rcp.make_params(rcp.RCP_MAP_EYE, 0.0, 6.0))
    six = _render(g, cam, 128, 128, 6, rcp.make_params(rcp.RCP_MAP_EYE, 0.0, 6.0))
    assert np.array_equal(one, six)
    k1 = _render(g, cam, 128, 128, 1, rcp.make_params(rcp.RCP_MAP_EYE, 1.4, 6.0))
    assert np.array_equal(one, k1)  # pass 1 from I_0 = 0.5 is pinhole whatever k


def test_mid_grey_does_not_move_rays(tiny_g):
    sc, g = tiny_g
    cam = rcp.camera_from(sc.poses[0])
    p = rcp.make_params(rcp.RCP_MAP_EYE, 1.4, 6.0)
    grey = np.full((96, 128, 4), 0.5, np.float32)
    a = rcp.rcp_render_pass(g, cam, 128, 96, p, in_rgbz=None)
    b = rcp.rcp_render_pass(g, cam, 128, 96, p, in_rgbz=grey)
    assert np.array_equal(a, b)


def test_launch_shapes_identical(tiny_g):
    sc = scenes.mid_scene()
    g = U.gpu_scene(sc)
    try:
        cam = rcp.camera_from(sc.poses[3])
        d = sc.diameter()
        p = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
        ref = None
        for block in (64, 128, 256):
            for fused in (0, 1):
                for chunk in (32, 64):
                    rcp.rcp_set_tuning(g, rcp.rcp_tuning(block, 0, chunk, fused, 0, 3))
                    out = _render(g, cam, 640, 360, 3, p)
                    if ref is None:
                        ref = out
                    assert np.array_equal(out, ref), (block, fused, chunk)
        # shorter shared stacks (the deeper levels spill to global memory), and
        # the previous-hit hints off, on for primary or shadow rays only
        for stack, hints in ((4, 3), (2, 3), (1, 3), (0, 0), (0, 1), (0, 2)):
            rcp.rcp_set_tuning(g, rcp.rcp_tuning(128, 0, 32, 1, stack, hints))
            assert np.array_equal(_render(g, cam, 640, 360, 3, p), ref), (stack, hints)
    finally:
        rcp.rcp_scene_destroy(g)


def test_short_stack_spills_identical():
    """The forest in the benchmark's build (13 levels): a 4-entry shared stack
    spills twelve levels to global memory and renders the same image, also
    batched and with the separate camera kernel."""
    sc = scenes.forest_scene()
    g = U.gpu_scene(sc, rcp.RCP_COLLAPSE_SAH, 8)
    try:
        assert rcp.rcp_scene_get_info(g).depth > 8
        cam = rcp.camera_from(sc.poses[20])
        d = sc.diameter()
        p = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
        ref = _render(g, cam, 480, 270, 4, p)
        for t in (rcp.rcp_tuning(128, 0, 32, 1, 4, 3), rcp.rcp_tuning(256, 0, 64, 0, 8, 0),
                  rcp.rcp_tuning(64, 0, 32, 1, 1, 3)):
            rcp.rcp_set_tuning(g, t)
            assert np.array_equal(_render(g, cam, 480, 270, 4, p), ref), (t.block, t.stack_entries)
    finally:
        rcp.rcp_scene_destroy(g)


def _full(g, cam, W, H, K, p, d_in=None, d_out=None):
    """The device path's whole output: rgb + z-depth (or normal code) bits and hit ids."""
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda") if d_out is None else d_out
    prim = torch.empty((H, W), dtype=torch.int32, device="cuda")
    rcp.rcp_render_device(g, cam, W, H, K, p, d_in, out, prim, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).copy(), prim.cpu().numpy()


@pytest.mark.parametrize("name", ["mid", "forest"])
def test_chained_passes_identical(name):
    """All K passes in one launch (each warp carrying its tile's pixels from
    pass to pass in registers) give the per-pass launches' output bit for bit:
    colours, z-depths, normal codes and hit ids, for every mapping that reads
    only the pixel's own previous value, every block size, a short stack that
    spills, hints off, a ragged image, a given first image rendered in place,
    and a batch of views; a chained render reports one launch."""
    sc = scenes.mid_scene() if name == "mid" else scenes.forest_scene()
    g = U.gpu_scene(sc) if name == "mid" else U.gpu_scene(sc, rcp.RCP_COLLAPSE_SAH, 8)
    try:
        cam = rcp.camera_from(sc.poses[5])
        d = sc.diameter()
        W, H, K = 643, 361, 5  # ragged in both directions
        for mapping in (rcp.RCP_MAP_EYE, rcp.RCP_MAP_TARGET, rcp.RCP_MAP_DEPTH, rcp.RCP_MAP_NORMAL):
            p = rcp.make_params(mapping, 0.02 * d, 0.1 * d, z0=0.1 * d if mapping == rcp.RCP_MAP_DEPTH else 0.0)
            rcp.rcp_set_tuning(g, rcp.rcp_tuning(128, 0, 32, 1, 0, 3, 0))
            ref = _full(g, cam, W, H, K, p)
            assert len(rcp.rcp_last_pass_times(g)) == K
            for t in (rcp.rcp_tuning(128, 0, 32, 1, 0, 3, 1), rcp.rcp_tuning(64, 0, 32, 1, 0, 3, 1),
                      rcp.rcp_tuning(256, 0, 64, 1, 0, 3, 1), rcp.rcp_tuning(128, 0, 32, 1, 2, 3, 1),
                      rcp.rcp_tuning(64, 0, 64, 1, 1, 0, 1)):
                rcp.rcp_set_tuning(g, t)
                got = _full(g, cam, W, H, K, p)
                key = (mapping, t.block, t.chunk, t.stack_entries, t.hints)
                assert len(rcp.rcp_last_pass_times(g)) == 1, key
                assert np.array_equal(got[0], ref[0]), key
                assert np.array_equal(got[1], ref[1]), key
        # a given first image, rendered in place (d_in == d_out)
        p = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
        first = torch.from_numpy(np.random.default_rng(4).random((H, W, 4), dtype=np.float32)).cuda()
        res = []
        for chain in (0, 1):
            rcp.rcp_set_tuning(g, rcp.rcp_tuning(128, 0, 32, 1, 0, 3, chain))
            buf = first.clone()
            res.append(_full(g, cam, W, H, 3, p, d_in=buf, d_out=buf))
        assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
        # a batch of views of several sizes, all passes in one launch
        sizes = [(97, 33), (256, 144), (31, 7), (400, 300)]
        cams = [rcp.camera_from(sc.poses[i * 9 + 1]) for i in range(len(sizes))]
        res = {}
        for chain in (0, 1):
            rcp.rcp_set_tuning(g, rcp.rcp_tuning(128, 0, 32, 1, 0, 3, chain))
            outs = [torch.empty((h, w, 4), dtype=torch.float32, device="cuda") for w, h in sizes]
            rcp.rcp_render_batch_device(g, cams, [w for w, _ in sizes], [h for _, h in sizes], 6, p, outs)
            torch.cuda.synchronize()
            res[chain] = [o.cpu().numpy().view(np.uint32) for o in outs]
        for a, b in zip(res[0], res[1]):
            assert np.array_equal(a, b)
    finally:
        rcp.rcp_scene_destroy(g)


def test_device_path_and_graph_replay(tiny_g):
    sc, g = tiny_g
    d = sc.diameter()
    p = rcp.make_params(rcp.RCP_MAP_EYE, 0.05 * d, 6.0)
    W, H = 200, 120
    outs = []
    cams = [sc.poses[0], scenes.Camera((3.0, 4.0, 9.0), (0.0, 1.0, 0.0))]
    for cam in cams:  # same shape: the second call replays the captured graph
        out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        rcp.rcp_render_device(g, rcp.camera_from(cam), W, H, 4, p, None, out, None, torch.cuda.current_stream())
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    for cam, out in zip(cams, outs):
        host = rcp.rcp_render(g, rcp.camera_from(cam), W, H, 4, p)
        assert np.array_equal(out[..., :3], host)
    assert not np.array_equal(outs[0], outs[1])
    # in-place: d_in == d_out
    buf = torch.from_numpy(outs[0].copy()).cuda()
    rcp.rcp_render_device(g, rcp.camera_from(cams[0]), W, H, 1, p, buf, buf, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    want = rcp.rcp_render_pass(g, rcp.camera_from(cams[0]), W, H, p, in_rgbz=outs[0])
    assert np.array_equal(buf.cpu().numpy(), want)


def test_batch_equals_single_views():
    sc = scenes.mid_scene()
    g = U.gpu_scene(sc)
    try:
        d = sc.diameter()
        p = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
        sizes = scenes.batched_view_sizes(6, seed=3)
        sizes = [(w // 4 + 1, h // 4 + 3) for w, h in sizes]
        cams = [rcp.camera_from(sc.poses[i * 7]) for i in range(len(sizes))]
        outs = [torch.empty((h, w, 4), dtype=torch.float32, device="cuda") for w, h in sizes]
        rcp.rcp_render_batch_device(g, cams, [w for w, _ in sizes], [h for _, h in sizes], 6, p, outs)
        torch.cuda.synchronize()
        for cam, (w, h), out in zip(cams, sizes, outs):
            single = _render(g, cam, w, h, 6, p)
            assert np.array_equal(out.cpu().numpy()[..., :3], single)
    finally:
        rcp.rcp_scene_destroy(g)


def test_empty_and_degenerate_scenes():
    light = rcp.make_light(rcp.RCP_LIGHT_DIRECTIONAL, (0.0, 1.0, 0.0))
    cam = rcp.make_camera((0, 0, 5), (0, 0, 0))
    p = rcp.make_params(rcp.RCP_MAP_EYE, 0.1, 2.0)
    g = rcp.rcp_scene_create(np.zeros((0, 9)), None, np.zeros((0, 3)), light)
    try:
        out = rcp.rcp_render(g, cam, 16, 8, 3, p)
        assert np.all(out[..., 2] == 1.0)  # sky only (its colour follows the moved rays)
        p0 = rcp.make_params(rcp.RCP_MAP_EYE, 0.0, 2.0)
        assert np.array_equal(rcp.rcp_render(g, cam, 16, 8, 3, p0), rcp.rcp_render(g, cam, 16, 8, 1, p0))
        info = rcp.rcp_scene_get_info(g)
        assert info.n_nodes == 0
    finally:
        rcp.rcp_scene_destroy(g)
    # a zero-area triangle is never hit; the valid one is
    tris = np.array([[-1, -1, 0, 1, -1, 0, 0, 1, 0], [0, 0, 1, 1, 1, 1, 2, 2, 1]], np.float32)
    g = rcp.rcp_scene_create(tris, None, np.full((2, 3), 0.5), light)
    try:
        prim = np.empty(32 * 32, np.int32)
        rcp.rcp_render_pass(g, cam, 32, 32, p, out_prim=prim)
        assert set(np.unique(prim)) <= {-1, 0} and (prim == 0).any()
        rcp.rcp_scene_validate(g)
    finally:
        rcp.rcp_scene_destroy(g)


def test_argument_errors(tiny_g):
    sc, g = tiny_g
    cam = rcp.camera_from(sc.poses[0])
    p = rcp.make_params(rcp.RCP_MAP_EYE, 1.0, 6.0)
    for W, H, K in [(0, 5, 1), (5, 0, 1), (8193, 5, 1), (5, 5, 0), (5, 5, 17)]:
        with pytest.raises(rcp.RcpError) as e:
            rcp.rcp_render(g, cam, W, H, K, p, out_rgb=np.empty(W * H * 3, np.float32))
        assert e.value.status == rcp.RCP_ERR_ARG
    for bad in [rcp.make_params(rcp.RCP_MAP_EYE, -1.0, 6.0), rcp.make_params(rcp.RCP_MAP_EYE, 1.0, 0.0),
                rcp.make_params(7, 1.0, 6.0)]:
        with pytest.raises(rcp.RcpError):
            rcp.rcp_render(g, cam, 4, 4, 1, bad)
    with pytest.raises(rcp.RcpError):
        rcp.rcp_render(g, rcp.make_camera((0, 0, 0), (0, 0, 0)), 4, 4, 1, p)
    bad_tris = np.array([[0, 0, np.nan, 1, 0, 0, 0, 1, 0]], np.float32)
    with pytest.raises(rcp.RcpError):
        rcp.rcp_scene_create(bad_tris, None, np.full((1, 3), 0.5), rcp.make_light(0, (1, 1, 1)))


def test_max_size_single_pass(tiny_g):
    sc, g = tiny_g
    cam = rcp.camera_from(sc.poses[0])
    p = rcp.make_params(rcp.RCP_MAP_EYE, 1.4, 6.0)
    W = H = 8192
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    rcp.rcp_render_device(g, cam, W, H, 1, p, None, out, None, torch.cuda.current_stream())
    torch.cuda.synchronize()
    # spot-check a few pixels against the oracle
    o = U.oracle_scene(sc)
    pix = scenes.pixel_subset(W, H, 256, seed=1)
    rgbz, prim, flag = o.render_pass(U.cam_f32(sc.poses[0]), W, H, 0, U.f32(1.4), 6.0, pix=pix)
    got = out.reshape(-1, 4)[torch.from_numpy(pix).cuda()].cpu().numpy()
    ok = flag == 0
    assert np.abs(got[ok, :3] - rgbz[ok, :3]).max() <= U.COLOUR_TOL
    del out


def test_max_size_max_k_chained(tiny_g):
    """The largest image and the most passes at once (8192 x 8192, K = 16):
    the chained launch equals one launch per pass on every pixel (compared on
    the device), and sampled pixels match the oracle's 16-pass chains."""
    sc, g = tiny_g
    cam = rcp.camera_from(sc.poses[0])
    d = sc.diameter()
    p = rcp.make_params(rcp.RCP_MAP_EYE, U.f32(0.05 * d), 6.0)
    W = H = 8192
    outs = []
    try:
        for chain in (1, 0):
            rcp.rcp_set_tuning(g, rcp.rcp_tuning(128, 0, 32, 1, 0, 3, chain))
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
            rcp.rcp_render_device(g, cam, W, H, 16, p, None, out, None, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert len(rcp.rcp_last_pass_times(g)) == (1 if chain else 16)
            outs.append(out)
        assert torch.equal(outs[0].view(torch.int32), outs[1].view(torch.int32))
        o = U.oracle_scene(sc)
        pix = scenes.pixel_subset(W, H, 128, seed=2)
        ref, _, _ = o.render(U.cam_f32(sc.poses[0]), W, H, 16, rcp.RCP_MAP_EYE, U.f32(0.05 * d), 6.0, pix=pix)
        got = outs[0].reshape(-1, 4)[torch.from_numpy(pix).cuda()].cpu().numpy()
        assert U.psnr(got[:, :3], ref[:, :3]) >= U.PSNR_MIN
    finally:
        rcp.rcp_set_tuning(g, rcp.rcp_tuning(128, 0, 32, 1, 0, 3, 1))
        del outs


def test_ray_counts_and_counters(tiny_g):
    sc, g = tiny_g
    cam = rcp.camera_from(sc.poses[0])
    p = rcp.make_params(rcp.RCP_MAP_EYE, 1.4, 6.0)
    out = rcp.rcp_render(g, cam, 128, 128, 6, p)
    prim, shadow = rcp.rcp_last_ray_counts(g)
    assert prim == 128 * 128 * 6 and 0 < shadow < prim
    c = rcp.rcp_count_pass(g, cam, 128, 128, p)
    assert c.primary_rays == 128 * 128 and c.rays == c.primary_rays + c.shadow_rays
    assert c.nodes > 0 and c.box_tests >= c.nodes and c.tri_tests + c.sphere_tests > 0
    assert out.shape == (128, 128, 3)


def test_autotune_cache(tmp_path):
    """The autotuner searches block, chunk, camera kernel and shared stack
    depth (mid: 7 levels, so 8 or 4 entries), and the cache returns its pick."""
    sc = scenes.mid_scene()
    g = U.gpu_scene(sc)
    try:
        cam = rcp.camera_from(sc.poses[0])
        d = sc.diameter()
        p = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
        path = str(tmp_path / "tune.json")
        ref = _render(g, cam, 320, 180, 3, p)
        t = rcp.rcp_autotune(g, cam, 320, 180, p, path)
        assert t.block in (64, 128, 256) and t.chunk in (32, 64) and t.stack_entries in (0, 4) and t.hints in (0, 3)
        assert np.array_equal(_render(g, cam, 320, 180, 3, p), ref)
        t2 = rcp.rcp_autotune(g, cam, 320, 180, p, path)  # from the cache
        assert (t2.block, t2.chunk, t2.fused_camera, t2.stack_entries, t2.hints) == (
            t.block, t.chunk, t.fused_camera, t.stack_entries, t.hints)
        assert "depth7" in open(path).read()
    finally:
        rcp.rcp_scene_destroy(g)
