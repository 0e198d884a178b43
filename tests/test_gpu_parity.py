"""Parity of the CUDA path with the FP64 oracle (per pass and end to end).

Workloads (seeded, see paper_2312_12392_gb300.scenes):
  * tiny: 3 spheres + ground quad, point light, 128x128, K=6, EYE mapping,
    k = 0.05 * diameter, f = 6 -- compared on every pixel;
  * mid: 133,472-triangle terrain + boxes, 1920x1080, K=6, k = 0.02 * diameter,
    f = 0.1 * diameter -- a seeded 16,384-pixel sample on each of 3 poses (each
    pixel's chain depends only on its own previous value, so a sample is
    exact), the oracle run live;
  * forest: 1,065,522 triangles, 1920x1080, K=6, in the benchmark's build
    (surface-area collapse, split <= 8) -- 16,384 pixels on each of 3 poses,
    against values the oracle wrote beforehand
    (tests/golden/make_oracle_golden.py: the brute-force oracle needs about
    ten minutes of the host's cores for them);
  * the TARGET, DEPTH and NORMAL mappings, and ragged image sizes.
"""
import os
import sys

import numpy as np
import pytest

from paper_2312_12392_gb300 import rcp, scenes
import gpu_util as U

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_oracle_golden as G  # noqa: E402

pytestmark = pytest.mark.gpu

MID_SAMPLE = 16384


@pytest.fixture(scope="module")
def tiny():
    return scenes.tiny_scene()


@pytest.fixture(scope="module")
def mid():
    return scenes.mid_scene()


def test_tiny_per_pass_full_frame(tiny):
    d = tiny.diameter()
    rep = U.per_pass_parity(tiny, tiny.poses[0], 128, 128, 6, rcp.RCP_MAP_EYE, 0.05 * d, 6.0)
    print(rep.assert_ok("tiny EYE 128x128 K=6"))


def test_tiny_end_to_end_psnr(tiny):
    d = tiny.diameter()
    p, fl = U.end_to_end_psnr(tiny, tiny.poses[0], 128, 128, 6, rcp.RCP_MAP_EYE, 0.05 * d, 6.0)
    print(f"tiny K=6 PSNR {p:.1f} dB, flagged chains {fl:.4f}")
    assert p >= U.PSNR_MIN


@pytest.mark.parametrize("mapping", [rcp.RCP_MAP_TARGET, rcp.RCP_MAP_DEPTH])
def test_tiny_other_mappings(tiny, mapping):
    d = tiny.diameter()
    k = 0.02 * d if mapping == rcp.RCP_MAP_TARGET else 0.002 * d
    rep = U.per_pass_parity(tiny, tiny.poses[0], 96, 80, 4, mapping, k, 6.0, z0=10.0)
    print(rep.assert_ok(f"tiny mapping {mapping}"))
    p, _ = U.end_to_end_psnr(tiny, tiny.poses[0], 96, 80, 4, mapping, k, 6.0, z0=10.0)
    assert p >= U.PSNR_MIN


@pytest.mark.parametrize("W,H", [(1, 1), (7, 3), (13, 9), (130, 61)])
def test_ragged_sizes(tiny, W, H):
    d = tiny.diameter()
    rep = U.per_pass_parity(tiny, tiny.poses[0], W, H, 3, rcp.RCP_MAP_EYE, 0.05 * d, 6.0)
    rep.assert_ok(f"tiny {W}x{H}")


@pytest.fixture(scope="module")
def mid_gpu(mid):
    g = U.gpu_scene(mid)
    yield g
    rcp.rcp_scene_destroy(g)


@pytest.mark.parametrize("pose", [0, 21, 42])
def test_mid_per_pass_sample(mid, mid_gpu, pose):
    d = mid.diameter()
    W, H = 1920, 1080
    pix = scenes.pixel_subset(W, H, MID_SAMPLE, seed=100 + pose)
    rep = U.per_pass_parity(mid, mid.poses[pose], W, H, 6, rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d, pix=pix, g=mid_gpu)
    print(rep.assert_ok(f"mid pose {pose}"))


def test_mid_end_to_end_psnr(mid, mid_gpu):
    d = mid.diameter()
    W, H = 1920, 1080
    pix = scenes.pixel_subset(W, H, MID_SAMPLE, seed=7)
    p, fl = U.end_to_end_psnr(mid, mid.poses[5], W, H, 6, rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d, pix=pix, g=mid_gpu)
    print(f"mid K=6 PSNR {p:.1f} dB, flagged chains {fl:.4f}")
    assert p >= U.PSNR_MIN


@pytest.mark.parametrize("mapping", [rcp.RCP_MAP_TARGET, rcp.RCP_MAP_DEPTH])
def test_mid_other_mappings(mid, mid_gpu, mapping):
    """The TARGET (§3) and DEPTH (§4, z0 at the focal distance) mappings at
    the bench's size and parameters (1920x1080, K=6, k = 0.02 diam, f = 0.1
    diam): per pass on 4,096 sampled pixels, and end to end by PSNR."""
    d = mid.diameter()
    W, H = 1920, 1080
    k, f = 0.02 * d, 0.1 * d
    z0 = f if mapping == rcp.RCP_MAP_DEPTH else 0.0
    pix = scenes.pixel_subset(W, H, 4096, seed=300 + mapping)
    rep = U.per_pass_parity(mid, mid.poses[9], W, H, 6, mapping, k, f, pix=pix, z0=z0, g=mid_gpu)
    print(rep.assert_ok(f"mid mapping {mapping}"))
    p, fl = U.end_to_end_psnr(mid, mid.poses[9], W, H, 6, mapping, k, f, pix=pix, z0=z0, g=mid_gpu)
    print(f"mid mapping {mapping} K=6 PSNR {p:.1f} dB, flagged chains {fl:.4f}")
    assert p >= U.PSNR_MIN


@pytest.fixture(scope="module")
def forest_golden():
    sc = scenes.forest_scene()
    d, meta = G.load("forest")
    cams = [sc.poses[p].as_array().astype(np.float32).astype(np.float64) for p in meta["poses"]]
    pixs = [d[f"pix_{i}"] for i in range(len(meta["poses"]))]
    k, f = G.params_of(dict(diam=sc.diameter()))
    assert G.input_hash(sc.tris, sc.albedo, cams, pixs, (k, f)) == meta["inputs"], "forest golden inputs differ"
    g = U.gpu_scene(sc, rcp.RCP_COLLAPSE_SAH, 8)
    yield sc, g, d, meta
    rcp.rcp_scene_destroy(g)


@pytest.mark.parametrize("i", [0, 1, 2])
def test_forest_per_pass_sample(forest_golden, i):
    """The forest in the benchmark's build, 16,384 pixels of one pose, each
    pass from the oracle's previous values."""
    sc, g, d, meta = forest_golden
    W, H, K = meta["W"], meta["H"], meta["K"]
    pose = meta["poses"][i]
    params = rcp.make_params(rcp.RCP_MAP_EYE, meta["k"], meta["f"])
    cam = rcp.camera_from(sc.poses[pose])
    pix = d[f"pix_{i}"]
    rep = U.PassReport()
    img = None
    for n in range(K):
        prim = np.empty(H * W, np.int32)
        out = rcp.rcp_render_pass(g, cam, W, H, params, in_rgbz=img, out_prim=prim)
        o_rgbz = d[f"rgbz_{i}"][n].astype(np.float64)
        rep.add(out.reshape(-1, 4)[pix], prim[pix], o_rgbz, d[f"prim_{i}"][n], d[f"flag_{i}"][n])
        img = U.next_image(out, pix, o_rgbz, rcp.RCP_MAP_EYE).reshape(H, W, 4)
    print(rep.assert_ok(f"forest pose {pose}"))


def test_forest_end_to_end_psnr(forest_golden):
    sc, g, d, meta = forest_golden
    i = int(d["e2e_index"])
    W, H, K = meta["W"], meta["H"], meta["K"]
    out = rcp.rcp_render(g, rcp.camera_from(sc.poses[meta["poses"][i]]), W, H, K,
                         rcp.make_params(rcp.RCP_MAP_EYE, meta["k"], meta["f"]))
    p = U.psnr(out.reshape(-1, 3)[d[f"pix_{i}"]], d["e2e_rgb"])
    print(f"forest K={K} PSNR {p:.1f} dB, flagged chains {float((d['e2e_flag'] != 0).mean()):.4f}")
    assert p >= U.PSNR_MIN


@pytest.mark.parametrize("scene_name", ["tiny", "mid"])
def test_normal_mapping(scene_name, tiny, mid):
    """§5, Eq. 8 (V_p = k C x N): per-pass parity, the normal handed to both
    sides being the oracle's previous normal in the ABI's code; the normals
    the GPU writes decode to the oracle's within the code's resolution."""
    sc = tiny if scene_name == "tiny" else mid
    d = sc.diameter()
    if scene_name == "tiny":
        W, H, pix, f = 128, 96, None, 6.0
    else:
        W, H, f = 1920, 1080, 0.1 * d
        pix = scenes.pixel_subset(W, H, 4096, seed=77)
    rep = U.per_pass_parity(sc, sc.poses[0], W, H, 4, rcp.RCP_MAP_NORMAL, 0.03 * d, f, pix=pix)
    print(rep.assert_ok(f"{scene_name} NORMAL"))
    assert rep.normal_err > 0  # the normals were compared
    g_rgbz, o_rgbz, o_flag, g_prim, o_prim = rep.last
    miss = (o_prim < 0) & (g_prim < 0)
    assert np.all(g_rgbz[miss, 3].view(np.uint32) == 0)  # a miss carries no normal
    p, _ = U.end_to_end_psnr(sc, sc.poses[0], W, H, 4, rcp.RCP_MAP_NORMAL, 0.03 * d, f, pix=pix)
    print(f"{scene_name} NORMAL K=4 PSNR {p:.1f} dB")
    assert p >= U.PSNR_MIN
