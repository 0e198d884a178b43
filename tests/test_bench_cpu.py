"""Host-side arithmetic of bench.py, without a GPU: the tuning string, the
roofline's sharing of counted work over launches (one per pass, or one per
chained frame), and the rule that ties a committed ncu record to the kernel
sources and to the kind of launch it was taken on."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_parse_tuning_fields_and_defaults():
    t = bench.parse_tuning("64,32,1,4,3,1")
    assert (t.block, t.blocks_per_sm, t.chunk, t.fused_camera, t.stack_entries, t.hints, t.chain_passes) == \
        (64, 0, 32, 1, 4, 3, 1)
    t = bench.parse_tuning("128,64,0")
    assert (t.stack_entries, t.hints, t.chain_passes) == (0, 3, 0)
    assert bench.tuning_dict(t)["chain_passes"] == 0


def _work(frames):
    # per frame: 1000 box tests, 100 triangle tests, 10 nodes, 20 primary rays, 35 rays
    return dict(box=1000 * frames, tri=100 * frames, sph=0, nodes=10 * frames, prim_rays=20 * frames,
                rays=35 * frames, frames=frames)


@pytest.mark.parametrize("per_frame", [1, 6])
def test_roofline_shares_work_over_launches(per_frame):
    frames = 4
    launch_ms = 2.0 / per_frame  # the same frame time either way
    pass_ms = [launch_ms] * (frames * per_frame)
    r = bench.roofline(_work(frames), pass_ms, frames, "none", None, 152)
    ops_frame = bench.OPS_BOX * 1000 + bench.OPS_TRI * 100 + bench.OPS_PIXEL * 20
    assert r["launches_per_frame"] == per_frame
    assert r["algorithmic_ops_per_launch"] == pytest.approx(ops_frame / per_frame)
    # achieved = ops per launch / launch time: the same rate whichever way the frame was launched
    assert r["achieved"] == pytest.approx(ops_frame / 2e-3 / 1e12)
    _, mhz, _ = bench.measured_peaks()
    assert r["peak"] == pytest.approx(152 * 128 * mhz * 1e6 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert ("all K passes" in r["kernel"]) == (per_frame == 1)
    assert r["per_ray"]["nodes"] == pytest.approx(10 / 35)


def test_ncu_record_matches_sources_and_launch_kind(tmp_path, monkeypatch):
    rec = {"mid": {"csrc_hash": bench.csrc_hash(), "chained": True, "dram_bytes_per_launch": 1.0},
           "forest": {"csrc_hash": "0" * 16, "chained": True, "dram_bytes_per_launch": 2.0}}
    os.makedirs(tmp_path / "profiles")
    (tmp_path / "profiles" / "k_trace_ncu.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "csrc_hash", lambda: rec["mid"]["csrc_hash"])
    assert bench.profiled("mid", True)["dram_bytes_per_launch"] == 1.0
    assert bench.profiled("mid", False) is None  # taken on chained launches, not per pass
    assert bench.profiled("forest", True) is None  # taken on other kernel sources
    assert bench.profiled("stress", True) is None  # no record


def test_committed_ncu_record_is_for_the_current_sources():
    """The committed record names the kernel sources it was taken on; while
    they hash the same, the bench reports its traffic."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "k_trace_ncu.json")))
    for name in ("mid", "forest"):
        assert rec[name]["chained"] is True
        assert len(rec[name]["csrc_hash"]) == 16
        assert rec[name]["dram_bytes_per_launch"] > 0
