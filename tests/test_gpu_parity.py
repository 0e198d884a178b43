"""Parity of the CUDA path with the FP64 oracle (per pass and end to end).

Workloads (seeded, see paper_2312_12392_gb300.scenes):
  * tiny: 3 spheres + ground quad, point light, 128x128, K=6, EYE mapping,
    k = 0.05 * diameter, f = 6 -- compared on every pixel;
  * mid: 133,472-triangle terrain + boxes, 1920x1080, K=6, k = 0.02 * diameter,
    f = 0.1 * diameter -- compared on a seeded 4,096-pixel sample (each pixel's
    chain depends only on its own previous value, so a sample is exact);
  * forest: 1,065,522 triangles, 1920x1080, K=6 -- 1,024-pixel sample;
  * the TARGET and DEPTH mappings on tiny, and ragged image sizes.
"""
import numpy as np
import pytest

from paper_2312_12392_gb300 import rcp, scenes
import gpu_util as U

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("pose", [0, 21, 42])
def test_mid_per_pass_sample(mid, pose):
    d = mid.diameter()
    W, H = 1920, 1080
    pix = scenes.pixel_subset(W, H, 4096, seed=100 + pose)
    rep = U.per_pass_parity(mid, mid.poses[pose], W, H, 6, rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d, pix=pix)
    print(rep.assert_ok(f"mid pose {pose}"))


def test_mid_end_to_end_psnr(mid):
    d = mid.diameter()
    W, H = 1920, 1080
    pix = scenes.pixel_subset(W, H, 4096, seed=7)
    p, fl = U.end_to_end_psnr(mid, mid.poses[5], W, H, 6, rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d, pix=pix)
    print(f"mid K=6 PSNR {p:.1f} dB, flagged chains {fl:.4f}")
    assert p >= U.PSNR_MIN


def test_forest_per_pass_and_psnr():
    """The forest in the bench's build (surface-area collapse, split <= 8)."""
    sc = scenes.forest_scene()
    d = sc.diameter()
    W, H = 1920, 1080
    pix = scenes.pixel_subset(W, H, 1024, seed=3)
    g = U.gpu_scene(sc, rcp.RCP_COLLAPSE_SAH, 8)
    o = U.oracle_scene(sc)
    try:
        rep = U.per_pass_parity(sc, sc.poses[10], W, H, 6, rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d, pix=pix, g=g, o=o)
        print(rep.assert_ok("forest pose 10"))
        p, fl = U.end_to_end_psnr(sc, sc.poses[10], W, H, 6, rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d, pix=pix, g=g, o=o)
        print(f"forest K=6 PSNR {p:.1f} dB, flagged chains {fl:.4f}")
        assert p >= U.PSNR_MIN
    finally:
        rcp.rcp_scene_destroy(g)


@pytest.mark.parametrize("scene_name", ["tiny", "mid"])
def test_normal_mapping(scene_name, tiny, mid):
    """§5, Eq. 8 (V_p = k C x N): per-pass parity, and the normal codes the GPU
    writes decode to the oracle's normals within the code's resolution."""
    import oracle as O
    sc = tiny if scene_name == "tiny" else mid
    d = sc.diameter()
    if scene_name == "tiny":
        W, H, pix, f = 128, 96, None, 6.0
    else:
        W, H, f = 1920, 1080, 0.1 * d
        pix = scenes.pixel_subset(W, H, 2048, seed=77)
    rep = U.per_pass_parity(sc, sc.poses[0], W, H, 4, rcp.RCP_MAP_NORMAL, 0.03 * d, f, pix=pix)
    print(rep.assert_ok(f"{scene_name} NORMAL"))
    g_rgbz, o_rgbz, o_flag, g_prim, o_prim = rep.last
    ok = (o_flag == 0) & (o_prim >= 0) & (g_prim == o_prim)
    codes_g = g_rgbz[:, 3].view(np.uint32)
    worst = 0.0
    for cg, co in zip(codes_g[ok], o_rgbz[ok, 3].astype(np.uint64)):
        ng, okg = O.normal_decode(int(cg))
        no, oko = O.normal_decode(int(co))
        assert okg and oko
        worst = max(worst, float(np.linalg.norm(ng - no)))
    assert worst < 2e-4, worst
    assert np.all(codes_g[o_prim < 0] == 0) or not (o_prim < 0).any()
    p, _ = U.end_to_end_psnr(sc, sc.poses[0], W, H, 4, rcp.RCP_MAP_NORMAL, 0.03 * d, f, pix=pix)
    print(f"{scene_name} NORMAL K=4 PSNR {p:.1f} dB")
    assert p >= U.PSNR_MIN
