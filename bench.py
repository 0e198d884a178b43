#!/usr/bin/env python
"""Benchmark of the recursive-camera-painting hot path on GB300.

Default workload (one JSON line on stdout): the 133,472-triangle fBm terrain +
200 boxes, 1920x1080, K = 6 passes, EYE mapping with k = 0.02 * diameter and
f = 0.1 * diameter, cycling through its 64-pose walk-through. One step = one
frame = K passes (camera + primary ray + shadow ray + shading for every pixel),
replayed from the library's captured CUDA graph with the scene resident in HBM.
L2 is flushed (a 256 MB write) between steps, outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload mid|forest|batched|served|stress|imagespace]
                    [--collapse auto|area|sah] [--tuning auto|block,chunk,fused]

The other workloads print their own line: the 1.07M-triangle forest, 64
batched forest views in one persistent launch, Poisson-arrival serving
against the plain per-request path, the 12.57M-triangle swaying forest at 4K
with per-frame refit (device-only, one stream and the serving path end to
end), and the image-space gather passes. --collapse auto builds the forests'
BVHs with the surface-area slot assignment and the terrains' with the
largest-area rule (the faster for each, as measured); the choice is printed in
each line's config.

With N > 1 (torchrun) every rank renders its own poses (replicas, no
collective on the data path); the time is the max over ranks.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
pixel sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

W_IMG, H_IMG, K_PASSES = 1920, 1080, 6
L2_FLUSH_BYTES = 256 << 20
# FP32 lane-operations per unit of work: a child-box test is 6 FMAs, 4 min/max
# and the compare and mask update; a Moller-Trumbore test 34; a sphere test 20;
# a pixel's camera and shading 40.
OPS_BOX, OPS_TRI, OPS_SPH, OPS_PIXEL = 14, 34, 20, 40
BYTES_NODE, BYTES_PRIM, BYTES_PIXEL_PASS = 208, 48, 32


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


FOREST_WORKLOADS = ("forest", "batched", "stress")


def collapse_for(args, workload):
    """BVH collapse policy: --collapse, or by scene kind ('auto'): the surface-
    area dynamic program for the forests (measured +11 % frames/s there), the
    largest-area greedy for the terrains (measured +1.2 % there)."""
    from paper_2312_12392_gb300 import rcp
    name = args.collapse
    if name == "auto":
        name = "sah" if workload in FOREST_WORKLOADS else "area"
    return (rcp.RCP_COLLAPSE_SAH if name == "sah" else rcp.RCP_COLLAPSE_AREA), name


def split_for(args, workload):
    """References per triangle at most: --split, or by scene kind ('auto'):
    early split clipping for the forests (long thin cone triangles; the stress
    forest's refits keep each reference bounded by its part of the moved
    triangle), none for the terrains."""
    if args.split != "auto":
        return int(args.split)
    return 8 if workload in FOREST_WORKLOADS else 0


def csrc_hash():
    """Hash of the CUDA/C++ sources with comments and whitespace removed, so
    that a recorded ncu figure stays tied to the code it was taken on."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2312_12392_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        src = open(os.path.join(d, f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(f.encode() + b"\0" + " ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload):
    """DRAM bytes per trace launch from the committed ncu summary, if it was
    taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "trace_dram_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(workload)
    if not e or e.get("csrc_hash") != csrc_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard_poses(rank, world, steps, n_poses):
    """Pose indices rendered by one rank: each rank takes its own run of
    `steps` consecutive poses of the walk-through (weak scaling, replicas)."""
    return [(rank * steps + i) % n_poses for i in range(steps)]


def max_over_ranks(value, device=None):
    """Max of a float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


def physical_gpu(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [x for x in vis.split(",") if x.strip()]
        if local < len(ids) and ids[local].strip().isdigit():
            return int(ids[local])
    return local


# ------------------------------------------------------------------ workloads

def make_workload(name):
    from paper_2312_12392_gb300 import scenes
    if name in ("mid", "served"):
        sc = scenes.mid_scene()
        desc = ("mid: 133,472-tri fBm terrain (256x256 quads) + 200 boxes, 1920x1080, K=6, EYE mapping "
                "k=0.02*diam, f=0.1*diam, directional light + shadow rays, 64-pose Catmull-Rom walk-through")
    elif name in ("forest", "batched"):
        sc = scenes.forest_scene()
        desc = ("forest: 1,065,522 tris (2,000 cone trees + 65k-tri ground), 1920x1080, K=6, EYE mapping "
                "k=0.02*diam, f=0.1*diam, directional light + shadow rays, 64-pose walk-through")
    else:
        raise SystemExit(f"unknown workload {name}")
    return sc, desc


def cpu_oracle_sample(sc, poses, target_s, nthreads=0, min_px=64, max_px=8192):
    """Time the FP64 oracle on seeded pixel samples (full K-pass chains) of the
    given poses; return (frames/s extrapolated, Mrays/s, pixels, seconds)."""
    import oracle as O
    from paper_2312_12392_gb300 import scenes
    o = O.OracleScene(sc.tris, sc.spheres, sc.albedo, sc.light.type,
                      np.asarray(sc.light.v, np.float32).astype(np.float64), float(np.float32(sc.light.ambient)))
    d = sc.diameter()
    k, f = float(np.float32(0.02 * d)), float(np.float32(0.1 * d))
    cam = poses[0].as_array().astype(np.float32).astype(np.float64)
    # size the sample from a probe long enough that thread start-up and load
    # imbalance over the host cores do not dominate it
    m = min_px
    while True:
        pix = scenes.pixel_subset(W_IMG, H_IMG, m, seed=11)
        t0 = time.perf_counter()
        o.render(cam, W_IMG, H_IMG, K_PASSES, O.MAP_EYE, k, f, pix=pix, nthreads=nthreads)
        t1 = time.perf_counter() - t0
        if t1 >= min(1.0, 0.1 * target_s * len(poses)) or m * 4 > max_px:
            break
        m *= 4
    n = int(min(max_px, max(min_px, m * target_s / max(t1, 1e-6))))
    total_px, total_t = 0, 0.0
    for i, pose in enumerate(poses):
        pix = scenes.pixel_subset(W_IMG, H_IMG, n, seed=12 + i)
        cam = pose.as_array().astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        o.render(cam, W_IMG, H_IMG, K_PASSES, O.MAP_EYE, k, f, pix=pix, nthreads=nthreads)
        total_t += time.perf_counter() - t0
        total_px += n
    fps = total_px / (total_t * W_IMG * H_IMG)
    return fps, total_px, total_t


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import torch

    from paper_2312_12392_gb300 import build as B
    from paper_2312_12392_gb300 import rcp
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    B.build()
    sc, desc = make_workload(args.workload)
    d = sc.diameter()
    params = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    collapse, collapse_name = collapse_for(args, args.workload)
    split = split_for(args, args.workload)
    t0 = time.perf_counter()
    g = rcp.scene_from(sc, collapse, split)
    build_s = time.perf_counter() - t0
    info = rcp.rcp_scene_get_info(g)
    log(f"[rank {rank}] scene {sc.name}: {info.n_tris} tris, {info.n_nodes} nodes, depth {info.depth}, "
        f"device build {info.build_ms:.1f} ms (host call {build_s:.2f} s)")
    if args.tuning == "auto":
        t = rcp.rcp_autotune(g, rcp.camera_from(sc.poses[0]), W_IMG, H_IMG, params,
                             os.path.join(ROOT, "paper_2312_12392_gb300", "tuning_cache.json"))
    else:
        b, c, fz = (int(x) for x in args.tuning.split(","))
        t = rcp.rcp_tuning(b, 0, c, fz)
        rcp.rcp_set_tuning(g, t)
    log(f"[rank {rank}] tuning block={t.block} chunk={t.chunk} fused_camera={t.fused_camera}")
    poses = [sc.poses[i] for i in shard_poses(rank, world, args.steps, len(sc.poses))]
    cams = [rcp.camera_from(p) for p in poses]
    stream = torch.cuda.current_stream()
    out = torch.empty((H_IMG, W_IMG, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for i in range(args.warmup):
        rcp.rcp_render_device(g, cams[i % len(cams)], W_IMG, H_IMG, K_PASSES, params, None, out, None, stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(physical_gpu(local))
    clocks.start()
    time.sleep(0.3)
    step_ms, pass_ms = [], []
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        s, e = evs[i]
        s.record(stream)
        rcp.rcp_render_device(g, cams[i], W_IMG, H_IMG, K_PASSES, params, None, out, None, stream)
        e.record(stream)
        e.synchronize()
        step_ms.append(s.elapsed_time(e))
        pass_ms.extend(rcp.rcp_last_pass_times(g))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = float(sum(step_ms))
    tmax = max_over_ranks(total_ms, "cuda")

    # rays traced per timed frame (deterministic per pose): replay each frame once more
    rays = 0
    for c in cams:
        rcp.rcp_render_device(g, c, W_IMG, H_IMG, K_PASSES, params, None, out, None, stream)
        torch.cuda.synchronize()
        p_, s_ = rcp.rcp_last_ray_counts(g)
        rays += p_ + s_
    rays = sum_over_ranks(rays, "cuda")

    # algorithmic work of a launch: chained counted passes over a few poses
    n_cnt = min(args.count_poses, len(cams))
    tot = dict(box=0, tri=0, sph=0, nodes=0, prim_rays=0, rays=0)
    a = torch.empty_like(out)
    b = torch.empty_like(out)
    for c in cams[:n_cnt]:
        prev = None
        for n in range(K_PASSES):
            dst = a if n % 2 == 0 else b
            cnt = rcp.rcp_count_pass(g, c, W_IMG, H_IMG, params, prev, dst)
            tot["box"] += cnt.box_tests
            tot["tri"] += cnt.tri_tests
            tot["sph"] += cnt.sphere_tests
            tot["nodes"] += cnt.nodes
            tot["prim_rays"] += cnt.primary_rays
            tot["rays"] += cnt.rays
            prev = dst
    n_launch_cnt = n_cnt * K_PASSES
    ops_launch = (OPS_BOX * tot["box"] + OPS_TRI * tot["tri"] + OPS_SPH * tot["sph"] +
                  OPS_PIXEL * tot["prim_rays"]) / n_launch_cnt
    bytes_launch = (BYTES_NODE * tot["nodes"] + BYTES_PRIM * (tot["tri"] + tot["sph"]) +
                    BYTES_PIXEL_PASS * tot["prim_rays"]) / n_launch_cnt
    launch_s = statistics.mean(pass_ms) / 1000.0
    hbm_gbs, sm_max_mhz, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = sms * 128 * sm_max_mhz * 1e6  # FP32 lanes x clock (ops/s)
    # The kernel is bound by arithmetic issue (ncu: integer/logic and FMA pipes
    # busy, DRAM idle because the BVH and images stay in L2), so the roofline
    # is the FP32-lane one. The byte view (every node and primitive fetch
    # charged at HBM peak) is reported beside it.
    roof = {"bound": "alu", "achieved": ops_launch / launch_s / 1e12, "peak": alu_peak / 1e12,
            "unit": "Tops/s (algorithmic FP32 lane-ops)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = profiled_traffic(args.workload)
    roof["kernel"] = "k_trace (camera + primary + shadow + shade, one launch per pass)"
    roof["launch_ms"] = launch_s * 1e3
    roof["algorithmic_ops_per_launch"] = ops_launch
    roof["algorithmic_bytes_per_launch"] = bytes_launch
    roof["peak_source"] = f"{sms} SMs x 128 FP32 lanes x {sm_max_mhz:.0f} MHz (max SM clock)"
    roof["hbm_view"] = {"achieved_gbs": bytes_launch / launch_s / 1e9, "peak_gbs": hbm_gbs,
                        "frac": bytes_launch / launch_s / 1e9 / hbm_gbs, "peak_source": peak_src,
                        "note": "algorithmic node/primitive/image bytes charged at HBM peak; they are served "
                                "from L1/L2 (see traffic)"}
    if clk and clk.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = roof["frac"] * sm_max_mhz / clk["sm_mhz"]
    roof["per_ray"] = {"nodes": tot["nodes"] / max(tot["rays"], 1), "box_tests": tot["box"] / max(tot["rays"], 1),
                       "tri_tests": tot["tri"] / max(tot["rays"], 1)}

    # end to end through the host API (host output buffer, copies timed)
    e2e_steps = max(3, min(args.steps, 16))
    host = np.empty((H_IMG, W_IMG, 3), np.float32)
    e2e_t = 0.0
    for i in range(e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rcp.rcp_render(g, cams[i % len(cams)], W_IMG, H_IMG, K_PASSES, params, host)
        if i > 0:
            e2e_t += time.perf_counter() - t0
    e2e_fps = world * e2e_steps / max_over_ranks(e2e_t, "cuda")

    frames = args.steps * world
    value = frames / (tmax / 1000.0)
    res = {
        "metric": "frames_per_s (1080p, K=6 passes per frame)",
        "value": value,
        "unit": "frames/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tmax / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded procedural scene and walk-through)",
        "config": {"workload": desc, "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "bvh_collapse": collapse_name, "bvh_split_max": max(split, 1),
                   "tuning": {"block": t.block, "chunk": t.chunk, "fused_camera": t.fused_camera},
                   "parallelism": f"replicas x{world} (poses split across ranks, no collective on the data path)"},
        "mrays_per_s": rays / (tmax / 1000.0) / 1e6,
        "rays_per_frame": rays / frames,
        "roofline": roof,
        "e2e": {"value": e2e_fps, "unit": "frames/s", "h2d_bytes_per_step": rcp.rcp_render_h2d_bytes(1, K_PASSES),
                "d2h_bytes_per_step": W_IMG * H_IMG * 3 * 4 + 4,  # the RGB image and the status word
                "api": "rcp_render (host RGB output; view descriptors H2D, RGB device-to-host inside the timed call: written into host memory by the last pass where the device reads pageable memory coherently, else packed and copied)"},
        "gpu_launches": args.steps * K_PASSES * (1 if t.fused_camera else 2),
        "clocks": clk,
        "wall_s": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fps, npx, secs = cpu_oracle_sample(sc, poses[:2], target_s=args.cpu_seconds / 2)
        res["cpu_baseline"] = {"value": fps, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"{npx} seeded pixels (full K=6 chains) over 2 poses in {secs:.1f} s, "
                                         f"extrapolated to 1920x1080 frames"}
    if args.extra_forest and args.workload == "mid" and world == 1:
        res["forest"] = forest_extra(args)
    rcp.rcp_scene_destroy(g)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        dist.destroy_process_group()


def forest_extra(args):
    """The 1.07M-triangle forest at 1080p K=6 over its whole 64-pose walk-through
    (same protocol as the headline: L2 flushed between frames, CUDA events)."""
    import torch

    from paper_2312_12392_gb300 import rcp
    sc, desc = make_workload("forest")
    d = sc.diameter()
    params = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    collapse, collapse_name = collapse_for(args, "forest")
    split = split_for(args, "forest")
    g = rcp.scene_from(sc, collapse, split)
    try:
        cams = [rcp.camera_from(p) for p in sc.poses]
        stream = torch.cuda.current_stream()
        out = torch.empty((H_IMG, W_IMG, 4), dtype=torch.float32, device="cuda")
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        for c in cams[:3]:
            rcp.rcp_render_device(g, c, W_IMG, H_IMG, K_PASSES, params, None, out, None, stream)
        torch.cuda.synchronize()
        ms, rays = [], 0
        for c in cams:
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            rcp.rcp_render_device(g, c, W_IMG, H_IMG, K_PASSES, params, None, out, None, stream)
            e.record(stream)
            e.synchronize()
            ms.append(s.elapsed_time(e))
            p_, s_ = rcp.rcp_last_ray_counts(g)
            rays += p_ + s_
        tot = sum(ms) / 1000.0
        info = rcp.rcp_scene_get_info(g)
        return {"workload": desc, "frames_per_s": len(cams) / tot, "mrays_per_s": rays / tot / 1e6,
                "ms_per_frame": 1000 * tot / len(cams), "bvh_build_ms": info.build_ms, "nodes": info.n_nodes,
                "depth": info.depth, "bvh_collapse": collapse_name, "bvh_split_max": max(split, 1),
                "records": info.n_records}
    finally:
        rcp.rcp_scene_destroy(g)


# ------------------------------------------------------------------ reference arm (the oracle)

def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    sc, desc = make_workload(args.workload)
    import oracle as O
    from paper_2312_12392_gb300 import scenes
    o = O.OracleScene(sc.tris, sc.spheres, sc.albedo, sc.light.type,
                      np.asarray(sc.light.v, np.float32).astype(np.float64), float(np.float32(sc.light.ambient)))
    d = sc.diameter()
    k, f = float(np.float32(0.02 * d)), float(np.float32(0.1 * d))
    # size each step's pixel sample so the whole run takes about 2.5 minutes
    probe = scenes.pixel_subset(W_IMG, H_IMG, 32, seed=1)
    t0 = time.perf_counter()
    o.render(sc.poses[0].as_array(), W_IMG, H_IMG, K_PASSES, O.MAP_EYE, k, f, pix=probe)
    per_px = (time.perf_counter() - t0) / 32
    per_step_s = 150.0 / max(args.steps + args.warmup, 1)
    n = int(max(32, min(16384, per_step_s / max(per_px, 1e-9))))
    times = []
    for i in range(args.warmup + args.steps):
        pix = scenes.pixel_subset(W_IMG, H_IMG, n, seed=1000 + i)
        cam = sc.poses[i % len(sc.poses)].as_array().astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        o.render(cam, W_IMG, H_IMG, K_PASSES, O.MAP_EYE, k, f, pix=pix)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    fps = args.steps * n / (tot * W_IMG * H_IMG)
    res = {
        "impl": "reference",
        "metric": "frames_per_s (1080p, K=6 passes per frame)",
        "value": fps,
        "unit": "frames/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1000.0 / fps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded procedural scene and walk-through)",
        "config": {"workload": desc},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{n} seeded pixels per step (full K=6 chains), {args.steps} steps, "
                                   f"extrapolated to 1920x1080 frames"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res), flush=True)


# ------------------------------------------------------------------ batched and served modes

def run_batched(args):
    """64 views of uneven size (W in [256,1920], H in [256,1080], seeded) of the
    1.07M-triangle forest, K = 6: one persistent launch per pass over all views
    (graph-captured, autotuned), against rendering the same views one after
    another with the single-view device path."""
    import torch

    from paper_2312_12392_gb300 import build as B
    from paper_2312_12392_gb300 import rcp, scenes
    torch.cuda.set_device(0)
    B.build()
    sc, _ = make_workload("forest")
    d = sc.diameter()
    params = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    collapse, collapse_name = collapse_for(args, "batched")
    split = split_for(args, "batched")
    g = rcp.scene_from(sc, collapse, split)
    sizes = scenes.batched_view_sizes(64, seed=3)
    cams = [rcp.camera_from(sc.poses[i % len(sc.poses)]) for i in range(len(sizes))]
    t = rcp.rcp_autotune(g, cams[0], 960, 540, params,
                         os.path.join(ROOT, "paper_2312_12392_gb300", "tuning_cache.json"))
    outs = [torch.empty((h, w, 4), dtype=torch.float32, device="cuda") for w, h in sizes]
    Ws, Hs = [w for w, _ in sizes], [h for _, h in sizes]
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def batch_once():
        rcp.rcp_render_batch_device(g, cams, Ws, Hs, K_PASSES, params, outs, stream)

    def plain_once():
        for c, (w, h), o in zip(cams, sizes, outs):
            rcp.rcp_render_device(g, c, w, h, K_PASSES, params, None, o, None, stream)

    res = {}
    for name, fn in (("batched", batch_once), ("plain", plain_once)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            fn()
            e.record(stream)
            e.synchronize()
            ms.append(s.elapsed_time(e))
        res[name] = statistics.mean(ms)
    pix = sum(w * h for w, h in sizes)
    batch_once()
    torch.cuda.synchronize()
    p_, s_ = rcp.rcp_last_ray_counts(g)
    out = {
        "metric": "views_per_s (64 uneven views, K=6 each, one launch per pass)",
        "value": len(sizes) / (res["batched"] / 1000.0),
        "unit": "views/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": res["batched"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"forest 1.07M tris, 64 views ({pix / 1e6:.1f} Mpixel total), K=6, graph-captured",
                   "bvh_collapse": collapse_name, "bvh_split_max": max(split, 1),
                   "l2": "flushed between steps", "tuning": {"block": t.block, "chunk": t.chunk,
                                                             "fused_camera": t.fused_camera}},
        "mrays_per_s": (p_ + s_) / (res["batched"] / 1000.0) / 1e6,
        "plain_ms_per_step": res["plain"],
        "plain_views_per_s": len(sizes) / (res["plain"] / 1000.0),
        "speedup_vs_plain": res["plain"] / res["batched"],
        "gpu_launches": args.steps * K_PASSES,
    }
    rcp.rcp_scene_destroy(g)
    print(json.dumps(out), flush=True)


def run_served(args):
    """Poisson arrivals over 4 resident terrain scenes (0.1M, 1M, 3M, 5M tris);
    each request: a walk-through pose, 720p/1080p/1440p/2160p, K in 1..8,
    k in [0, 0.05] * diameter. The continuous-batching server against the plain
    path (one request at a time, FIFO, each its own launch sequence), same
    arrivals. Reports frames/s and p50/p99 latency per arrival rate."""
    import threading

    import torch

    from paper_2312_12392_gb300 import build as B
    from paper_2312_12392_gb300 import rcp, scenes
    torch.cuda.set_device(0)
    B.build()
    grids = [221, 706, 1224, 1580]
    scs = [scenes.terrain_scene(gsz, seed=4) for gsz in grids]
    collapse, collapse_name = collapse_for(args, "served")
    gs = [rcp.scene_from(s, collapse) for s in scs]
    n_req = args.steps
    reqs = scenes.served_requests(n_req, len(scs), 64, seed=4)
    diams = [s.diameter() for s in scs]
    # one output buffer per request, allocated and touched before any timing
    outs = [np.zeros((r["height"], r["width"], 3), np.float32) for r in reqs]

    def buf(i):
        return outs[i]

    def params_of(r):
        d = diams[r["scene"]]
        return rcp.make_params(rcp.RCP_MAP_EYE, r["k_frac"] * d, 0.1 * d)

    def cam_of(r):
        return rcp.camera_from(scs[r["scene"]].poses[r["pose"]])

    prepared = [(cam_of(r), params_of(r)) for r in reqs]

    # warm both paths: every request once through the plain path (render
    # contexts and graphs), a short burst through a server (memory pool)
    for i, r in enumerate(reqs):
        rcp.rcp_render(gs[r["scene"]], prepared[i][0], r["width"], r["height"], r["K"], prepared[i][1], buf(i))
    srv = rcp.rcp_server_create(int(args.serve_budget_gb * (1 << 30)), args.serve_slots)
    tks = [rcp.rcp_server_submit(srv, gs[r["scene"]], prepared[i][0], r["width"], r["height"], r["K"],
                                 prepared[i][1], buf(i)) for i, r in enumerate(reqs[:16])]
    for tk in tks:
        rcp.rcp_server_wait(srv, tk, 600.0)
    rcp.rcp_server_destroy(srv)
    rates = [float(x) for x in args.rates.split(",")]
    table = []
    for lam in rates:
        arr = scenes.poisson_arrivals(lam, n_req, seed=4)
        # -- plain: FIFO worker, one request at a time
        lat = [0.0] * n_req
        t0 = time.perf_counter()

        def plain_worker():
            for i, r in enumerate(reqs):
                wait = arr[i] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                rcp.rcp_render(gs[r["scene"]], prepared[i][0], r["width"], r["height"], r["K"], prepared[i][1],
                               buf(i))
                lat[i] = time.perf_counter() - t0 - arr[i]

        th = threading.Thread(target=plain_worker)
        th.start()
        th.join()
        plain_span = time.perf_counter() - t0
        plain = {"frames_per_s": n_req / plain_span, "p50_ms": 1000 * float(np.percentile(lat, 50)),
                 "p99_ms": 1000 * float(np.percentile(lat, 99))}
        # -- server: submit at the arrival times
        srv = rcp.rcp_server_create(int(args.serve_budget_gb * (1 << 30)), args.serve_slots)
        t0 = time.perf_counter()
        tickets = []
        for i, r in enumerate(reqs):
            wait = arr[i] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            tickets.append(rcp.rcp_server_submit(srv, gs[r["scene"]], prepared[i][0], r["width"], r["height"],
                                                 r["K"], prepared[i][1], buf(i)))
        for tk in tickets:
            rcp.rcp_server_wait(srv, tk, 600.0)
        st = rcp.rcp_server_stats_get(srv)
        rcp.rcp_server_destroy(srv)
        served = {"frames_per_s": st.frames_per_s, "p50_ms": st.p50_ms, "p99_ms": st.p99_ms,
                  "mrays_per_s": st.mrays_per_s, "steps": st.steps, "peak_gb": st.device_bytes_peak / 2 ** 30}
        table.append({"rate_req_s": lam, "served": served, "plain": plain})
        log(f"lambda={lam}: served {served} | plain {plain}")
    best = max(table, key=lambda r: r["served"]["frames_per_s"])
    out = {
        "metric": "served frames_per_s and p50/p99 latency vs the plain per-request path",
        "value": best["served"]["frames_per_s"], "unit": "frames/s",
        "n_gpus": 1, "steps": n_req, "warmup": 1, "ms_per_step": 1000.0 / best["served"]["frames_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"bvh_collapse": collapse_name,
                   "workload": "4 resident terrain scenes (100,082 / 999,272 / 2,998,752 / 4,995,200 tris); "
                               "720p-2160p, K in 1..8, Poisson arrivals",
                   "requests_per_rate": n_req, "slots": args.serve_slots, "budget_gb": args.serve_budget_gb},
        "sweep": table,
    }
    for g in gs:
        rcp.rcp_scene_destroy(g)
    print(json.dumps(out), flush=True)


def run_stress(args):
    """25,000-tree forest (12.57M triangles), 3840x2160, K=8: every frame the
    wind sways the trees (input generated on the device with torch), the BVH is
    refitted (rcp_scene_update_vertices_device) and the frame is rendered."""
    import torch

    from paper_2312_12392_gb300 import build as B
    from paper_2312_12392_gb300 import rcp, scenes
    torch.cuda.set_device(0)
    B.build()
    t0 = time.perf_counter()
    sc = scenes.forest_scene(25_000, seed=5)
    gen_s = time.perf_counter() - t0
    W, H, K = 3840, 2160, 8
    d = sc.diameter()
    params = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    collapse, collapse_name = collapse_for(args, "stress")
    split = split_for(args, "stress")
    g = rcp.scene_from(sc, collapse, split)
    info = rcp.rcp_scene_get_info(g)
    base = torch.from_numpy(sc.tris).cuda().reshape(-1, 3, 3)
    amp = torch.from_numpy(sc.sway_amp).cuda()
    phase = torch.from_numpy(sc.sway_phase).cuda()
    moved = torch.empty_like(base)
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    cams = [rcp.camera_from(sc.poses[i % len(sc.poses)]) for i in range(args.steps + args.warmup)]

    def sway(frame):
        ang = 2.0 * np.pi * 0.5 * (frame / 60.0) + phase
        moved.copy_(base)
        moved[:, :, 0] += amp * torch.sin(ang)[:, None]
        moved[:, :, 2] += amp * torch.cos(ang)[:, None]

    for i in range(args.warmup):
        sway(i)
        rcp.rcp_scene_update_vertices_device(g, moved, stream)
        rcp.rcp_render_device(g, cams[i], W, H, K, params, None, out, None, stream)
    torch.cuda.synchronize()
    refit_ms, render_ms, frame_ms, rays = [], [], [], 0
    for i in range(args.warmup, args.warmup + args.steps):
        sway(i)  # input generation, outside the timed events
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        rcp.rcp_scene_update_vertices_device(g, moved, stream)
        e1.record(stream)
        rcp.rcp_render_device(g, cams[i], W, H, K, params, None, out, None, stream)
        e2.record(stream)
        e2.synchronize()
        refit_ms.append(e0.elapsed_time(e1))
        render_ms.append(e1.elapsed_time(e2))
        frame_ms.append(e0.elapsed_time(e2))
        p_, s_ = rcp.rcp_last_ray_counts(g)
        rays += p_ + s_
    rcp.rcp_scene_validate(g)
    tot = sum(frame_ms) / 1000.0

    # End to end, every frame's RGB delivered to host memory, the same frames:
    # (1) one stream: sway, refit, render, copy out, frame after frame;
    # (2) the serving path with two copies of the scene used in turn, so that
    #     frame f's sway and refit overlap frame f-1's render and copy-out (a
    #     copy is refitted only once the request two frames back, its last
    #     user, is done). Three host buffers rotate (at most two in flight).
    n = args.steps
    frames = [args.warmup + i for i in range(n)]
    bufs = {k: [np.zeros((H, W, 3), np.float32) for _ in range(3)] for k in ("single", "served")}
    t0 = time.perf_counter()
    for i, f in enumerate(frames):
        sway(f)
        rcp.rcp_scene_update_vertices_device(g, moved, stream)
        torch.cuda.synchronize()  # the render runs on the library's stream
        rcp.rcp_render(g, cams[f], W, H, K, params, bufs["single"][i % 3])
    single_s = time.perf_counter() - t0
    g2 = rcp.scene_from(sc, collapse, split)
    copies = [g, g2]
    budget = int(args.serve_budget_gb * (1 << 30))
    # warm the device memory pool with one request per copy on a server of its
    # own, so that the timed server's latency figures hold the timed frames only
    srv = rcp.rcp_server_create(budget, args.serve_slots)
    for j in range(2):
        rcp.rcp_server_wait(srv, rcp.rcp_server_submit(srv, copies[j], cams[0], W, H, K, params,
                                                       bufs["served"][j]), 600.0)
    rcp.rcp_server_destroy(srv)
    srv = rcp.rcp_server_create(budget, args.serve_slots)
    tickets = []
    t0 = time.perf_counter()
    for i, f in enumerate(frames):
        if i >= 2:
            rcp.rcp_server_wait(srv, tickets[i - 2], 600.0)
        sway(f)
        rcp.rcp_scene_update_vertices_device(copies[i % 2], moved, stream)
        torch.cuda.synchronize()
        tickets.append(rcp.rcp_server_submit(srv, copies[i % 2], cams[f], W, H, K, params, bufs["served"][i % 3]))
    for tk in tickets[-2:]:
        rcp.rcp_server_wait(srv, tk, 600.0)
    served_s = time.perf_counter() - t0
    st = rcp.rcp_server_stats_get(srv)
    rcp.rcp_server_destroy(srv)
    same_last = bool(np.array_equal(bufs["single"][(n - 1) % 3], bufs["served"][(n - 1) % 3]))
    rcp.rcp_scene_destroy(g2)
    out_bytes = H * W * 3 * 4
    res = {
        "metric": "frames_per_s (3840x2160, K=8, per-frame refit)",
        "value": args.steps / tot, "unit": "frames/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"bvh_collapse": collapse_name, "bvh_split_max": split, "records": info.n_records,
                   "workload": f"stress: {info.n_tris:,} tris (25,000 swaying cone trees), 3840x2160, K=8, "
                               "wind sway A=0.02*h_tree at 0.5 Hz, refit every frame",
                   "scene_generation_s": gen_s, "bvh_build_ms": info.build_ms, "nodes": info.n_nodes,
                   "depth": info.depth},
        "refit_ms": statistics.mean(refit_ms), "render_ms": statistics.mean(render_ms),
        "mrays_per_s": rays / tot / 1e6, "gpu_launches_per_step": K + 2 + info.depth,
        "e2e": {"value": n / single_s, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": out_bytes,
                "api": "single stream: rcp_scene_update_vertices_device + rcp_render (host RGB) per frame"},
        "served_e2e": {"value": n / served_s, "unit": "frames/s", "p50_ms": st.p50_ms, "p99_ms": st.p99_ms,
                       "d2h_bytes_per_step": out_bytes, "last_frame_identical_to_single_stream": same_last,
                       "api": "rcp_server_submit (host RGB), two scene copies refitted in turn"},
    }
    rcp.rcp_scene_destroy(g)
    print(json.dumps(res), flush=True)


def run_imagespace(args):
    """The image-space reduction (§6): mid terrain at 3840x2160, K=6; pass 1 is
    traced, passes 2..6 gather from it (k = 8 pixels, mirrored edges). The
    gather kernel's roofline is HBM: 48 bytes per pixel (read I_{n-1} and the
    traced image, write I_n), 398 MB per pass at 4K (above the 129 MB L2)."""
    import torch

    from paper_2312_12392_gb300 import build as B
    from paper_2312_12392_gb300 import rcp
    torch.cuda.set_device(0)
    B.build()
    sc, _ = make_workload("mid")
    W, H, K, kpx = 3840, 2160, 6, 8.0
    d = sc.diameter()
    params = rcp.make_params(rcp.RCP_MAP_IMAGE, kpx, 0.1 * d)
    collapse, collapse_name = collapse_for(args, "imagespace")
    g = rcp.scene_from(sc, collapse)
    stream = torch.cuda.current_stream()
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    cams = [rcp.camera_from(sc.poses[i % len(sc.poses)]) for i in range(args.steps + args.warmup)]
    for i in range(args.warmup):
        rcp.rcp_render_device(g, cams[i], W, H, K, params, None, out, None, stream)
    torch.cuda.synchronize()
    frame_ms, trace_ms, gather_ms = [], [], []
    for i in range(args.warmup, args.warmup + args.steps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        rcp.rcp_render_device(g, cams[i], W, H, K, params, None, out, None, stream)
        e.record(stream)
        e.synchronize()
        frame_ms.append(s.elapsed_time(e))
        pt = rcp.rcp_last_pass_times(g)
        trace_ms.append(pt[0])
        gather_ms.extend(pt[1:])
    hbm_gbs, _, peak_src = measured_peaks()
    g_s = statistics.mean(gather_ms) / 1000.0
    bytes_launch = 48.0 * W * H
    tot = sum(frame_ms) / 1000.0
    res = {
        "metric": "frames_per_s (image-space reduction, 3840x2160, K=6)",
        "value": args.steps / tot, "unit": "frames/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"bvh_collapse": collapse_name,
                   "workload": "mid terrain 133k tris, 3840x2160, K=6, RCP_MAP_IMAGE k=8 px: 1 traced pass + 5 "
                               "gather passes", "l2": "flushed between steps"},
        "trace_pass_ms": statistics.mean(trace_ms),
        "roofline": {"bound": "hbm", "kernel": "k_imagespace (one gather pass)", "launch_ms": g_s * 1e3,
                     "achieved": bytes_launch / g_s / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                     "frac": bytes_launch / g_s / 1e9 / hbm_gbs, "traffic": None,
                     "algorithmic_bytes_per_launch": bytes_launch, "peak_source": peak_src},
        "gpu_launches": args.steps * K,
    }
    rcp.rcp_scene_destroy(g)
    print(json.dumps(res), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="mid", choices=["mid", "forest", "batched", "served", "stress", "imagespace"])
    ap.add_argument("--tuning", default="128,32,1", help="'auto' or block,chunk,fused_camera")
    ap.add_argument("--collapse", default="auto", choices=["auto", "area", "sah"],
                    help="BVH collapse policy; auto: sah for the forest workloads, area for the terrains")
    ap.add_argument("--split", default="auto", choices=["auto"] + [str(i) for i in range(9)],
                    help="references per triangle at most (early split clipping); auto: 8 for the forests "
                         "(static and swaying), 0 for the terrains")
    ap.add_argument("--count-poses", type=int, default=4)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-forest", dest="extra_forest", action="store_false")
    ap.add_argument("--rates", default="10,25,50,100,200,400", help="served: arrival rates (req/s)")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-budget-gb", type=float, default=24.0)
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        log("warmup raised to 3 (timing rule)")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    elif args.workload == "stress":
        run_stress(args)
    elif args.workload == "imagespace":
        run_imagespace(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
