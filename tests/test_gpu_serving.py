"""The continuous-batching server: every request's image is identical alone
and in a mix of scenes, sizes and K (each pixel's chain is deterministic and
independent of the other work in the launch), memory admission holds, and the
statistics add up."""
import time

import numpy as np
import pytest

from paper_2312_12392_gb300 import rcp, scenes
import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def two_scenes():
    a = scenes.tiny_scene()
    b = scenes.terrain_scene(64, seed=4, n_boxes=20)
    ga, gb = U.gpu_scene(a), U.gpu_scene(b)
    yield (a, ga), (b, gb)
    rcp.rcp_scene_destroy(ga)
    rcp.rcp_scene_destroy(gb)


def _requests(two_scenes, n=24, seed=0, ms_every=0):
    """ms_every > 0: every ms_every-th request takes 4 jittered samples per pixel."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        sc, g = two_scenes[int(rng.integers(0, 2))]
        W = int(rng.integers(8, 300))
        H = int(rng.integers(8, 200))
        K = int(rng.integers(1, 9))
        cam = sc.poses[int(rng.integers(0, len(sc.poses)))]
        d = sc.diameter()
        f = U.f32(6.0 if sc.name == "tiny" else 0.1 * d)
        k = U.f32(float(rng.uniform(0, 0.05)) * d)
        jit = rng.random((4, 2)) if ms_every and i % ms_every == ms_every - 1 else None
        p = rcp.make_params(rcp.RCP_MAP_EYE, k, f, jitter=jit)
        out.append(dict(sc=sc, g=g, cam=cam, W=W, H=H, K=K, k=k, f=f, p=p))
    return out


def _serve(reqs, slots=8, max_chain=None, step_pixels=None):
    srv = rcp.rcp_server_create(4 << 30, slots)
    try:
        if max_chain is not None:
            rcp.rcp_server_set_max_chain(srv, max_chain)
        if step_pixels is not None:
            rcp.rcp_server_set_step_pixels(srv, step_pixels)
        outs, tickets = [], []
        for i, r in enumerate(reqs):
            o = np.full((r["H"], r["W"], 3), -1.0, np.float32)
            outs.append(o)
            tickets.append(rcp.rcp_server_submit(srv, r["g"], rcp.camera_from(r["cam"]), r["W"], r["H"], r["K"],
                                                 r["p"], o))
            if i % 5 == 4:
                time.sleep(0.002)  # arrivals while others are in flight
        for t in tickets:
            rcp.rcp_server_wait(srv, t, 60.0)
            assert rcp.rcp_server_poll(srv, t)
        return outs, rcp.rcp_server_stats_get(srv)
    finally:
        rcp.rcp_server_destroy(srv)


@pytest.mark.parametrize("mode", [rcp.RCP_HOST_OUTPUT_AUTO, rcp.RCP_HOST_OUTPUT_DIRECT])
def test_alone_equals_in_mix(two_scenes, mode):
    """Served images equal the same requests rendered alone, bit for bit, with
    images delivered by pack-and-copy (fresh buffers under AUTO) or written by
    the last pass (DIRECT)."""
    rcp.rcp_set_host_output(mode)
    try:
        _alone_equals_in_mix(two_scenes)
    finally:
        rcp.rcp_set_host_output(rcp.RCP_HOST_OUTPUT_AUTO)


def _alone_equals_in_mix(two_scenes):
    reqs = _requests(two_scenes)
    alone = [rcp.rcp_render(r["g"], rcp.camera_from(r["cam"]), r["W"], r["H"], r["K"], r["p"]) for r in reqs]
    outs, st = _serve(reqs)
    for a, o in zip(alone, outs):
        assert np.array_equal(a, o)
    assert st.completed == len(reqs) and st.rejected == 0 and st.in_flight == 0 and st.queued == 0
    assert st.p99_ms >= st.p50_ms > 0 and st.frames_per_s > 0 and st.mrays_per_s > 0
    assert st.steps >= 1
    assert st.device_bytes_in_use == 0 and st.device_bytes_peak > 0


@pytest.mark.parametrize("max_chain,step_pixels,ms_every", [(1, None, 0), (3, 60_000, 0), (16, 0, 0),
                                                            (16, None, 5)])
def test_step_shapes_equal_alone(two_scenes, max_chain, step_pixels, ms_every):
    """However a step is shaped -- one pass per request per step, short chains
    under a small pixel-pass budget, every admitted request chained to the end,
    or per-pass steps forced by multi-sample requests in the mix -- every
    served image equals the request rendered alone, bit for bit."""
    reqs = _requests(two_scenes, n=20, seed=7, ms_every=ms_every)
    alone = [rcp.rcp_render(r["g"], rcp.camera_from(r["cam"]), r["W"], r["H"], r["K"], r["p"]) for r in reqs]
    outs, st = _serve(reqs, max_chain=max_chain, step_pixels=step_pixels)
    for i, (a, o) in enumerate(zip(alone, outs)):
        assert np.array_equal(a, o), i
    if max_chain == 1 and not ms_every:
        assert st.steps >= max(r["K"] for r in reqs)
    with pytest.raises(rcp.RcpError):
        srv = rcp.rcp_server_create(1 << 20, 1)
        try:
            rcp.rcp_server_set_max_chain(srv, 0)
        finally:
            rcp.rcp_server_destroy(srv)


def test_mix_against_oracle(two_scenes):
    """Every request of a mixed run (two scenes, uneven sizes, K from 1 to 8,
    arrivals while others are in flight) against the FP64 oracle's K-pass
    chains on a seeded pixel sample of its own image."""
    reqs = _requests(two_scenes, n=24, seed=1)
    outs, _ = _serve(reqs)
    oscenes = {}
    worst = np.inf
    for i, (r, out) in enumerate(zip(reqs, outs)):
        o = oscenes.setdefault(r["sc"].name, U.oracle_scene(r["sc"]))
        pix = scenes.pixel_subset(r["W"], r["H"], 512, seed=i)
        ref, _, fl = o.render(U.cam_f32(r["cam"]), r["W"], r["H"], r["K"], rcp.RCP_MAP_EYE, r["k"], r["f"], pix=pix)
        p = U.psnr(out.reshape(-1, 3)[pix], ref[:, :3])
        worst = min(worst, p)
        assert p >= U.PSNR_MIN, (i, r["sc"].name, r["W"], r["H"], r["K"], p)
    print(f"{len(reqs)} served requests against the oracle: worst PSNR {worst:.1f} dB")


def test_memory_admission(two_scenes):
    (sc, g), _ = two_scenes
    cam = rcp.camera_from(sc.poses[0])
    p = rcp.make_params(rcp.RCP_MAP_EYE, 1.0, 6.0)
    W, H = 256, 256
    per_req = W * H * 52 + 1024  # two rgbz images, hit hints and RGB staging (the larger, copy-out form)
    srv = rcp.rcp_server_create(2 * per_req + 100, 16)  # room for two at a time
    try:
        outs = [np.empty((H, W, 3), np.float32) for _ in range(6)]
        ts = [rcp.rcp_server_submit(srv, g, cam, W, H, 3, p, o) for o in outs]
        big = np.empty((1024, 1024, 3), np.float32)
        tb = rcp.rcp_server_submit(srv, g, cam, 1024, 1024, 1, p, big)  # never fits
        for t in ts:
            rcp.rcp_server_wait(srv, t, 60.0)
        with pytest.raises(rcp.RcpError) as e:
            rcp.rcp_server_wait(srv, tb, 60.0)
        assert e.value.status == rcp.RCP_ERR_OOM
        st = rcp.rcp_server_stats_get(srv)
        assert st.device_bytes_peak <= 2 * per_req + 100
        assert st.completed == 6 and st.rejected == 1
        ref = rcp.rcp_render(g, cam, W, H, 3, p)
        for o in outs:
            assert np.array_equal(o, ref)
    finally:
        rcp.rcp_server_destroy(srv)


def test_wait_timeout_and_unknown_ticket(two_scenes):
    srv = rcp.rcp_server_create(1 << 30, 4)
    try:
        with pytest.raises(rcp.RcpError) as e:
            rcp.rcp_server_wait(srv, 12345, 0.01)
        assert e.value.status == rcp.RCP_ERR_ARG
    finally:
        rcp.rcp_server_destroy(srv)
