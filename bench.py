#!/usr/bin/env python
"""Benchmark of the recursive-camera-painting hot path on GB300.

Default workload (one JSON line on stdout): the 133,472-triangle fBm terrain +
200 boxes, 1920x1080, K = 6 passes, EYE mapping with k = 0.02 * diameter and
f = 0.1 * diameter, cycling through its 64-pose walk-through. One step = one
frame = K passes (camera + primary ray + shadow ray + shading for every pixel),
replayed from the library's captured CUDA graph with the scene resident in HBM
(by default one launch runs the K passes, chained).
L2 is flushed (a 256 MB write) between steps, outside the timed events.

At one GPU the same line also carries the other workloads, each measured in
this run: "forest" (the 1.07M-triangle forest, 1080p K=6 over its 64-pose
walk-through, with its own roofline, end-to-end figure and clock record),
"batched" (64 uneven forest views in one launch, against per-view renders),
"served" (Poisson arrivals over four resident terrains of 0.1-5M triangles,
the continuous-batching server against the plain per-request path, 1,000
requests per rate), "stress" (the 12.57M-triangle swaying forest at 4K, K=8,
refit and render per frame) and "mappings" (the terrain under the TARGET,
DEPTH and NORMAL mappings and with 4 jittered samples per pixel).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload mid|forest|batched|served|stress|mappings|imagespace]
                    [--collapse auto|area|sah] [--tuning auto|block,chunk,fused[,stack[,hints[,chain]]]]
                    [--no-extras]

--workload prints one workload's line alone. --collapse auto builds the
forests' BVHs with the surface-area slot assignment and the terrains' with the
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


TRACE_SOURCES = ("rcp_internal.cuh", "trace.cu", "trace.cuh")  # everything the k_trace kernel compiles from


def csrc_hash():
    """Hash of the trace kernel's sources with comments and whitespace
    removed, so that a recorded ncu figure stays tied to the code it was taken
    on (edits elsewhere, the server or the ABI, do not invalidate it)."""
    import re
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2312_12392_gb300", "csrc")
    for f in TRACE_SOURCES:
        src = open(os.path.join(d, f), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(f.encode() + b"\0" + " ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled(workload, chained):
    """The committed ncu record of the trace kernel on this workload (DRAM
    bytes per launch, issue and pipe utilisation, L1 hit rate), if it was taken
    on the current kernel sources and on the same kind of launch (all passes
    chained, or one launch per pass); else None."""
    p = os.path.join(ROOT, "profiles", "k_trace_ncu.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get(workload)
    if not e or e.get("csrc_hash") != csrc_hash() or bool(e.get("chained")) != chained:
        return None
    return e


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


# ------------------------------------------------------------------ measurement helpers

def parse_tuning(spec):
    from paper_2312_12392_gb300 import rcp
    v = [int(x) for x in spec.split(",")]
    return rcp.rcp_tuning(v[0], 0, v[1], v[2], v[3] if len(v) > 3 else 0, v[4] if len(v) > 4 else 3,
                          v[5] if len(v) > 5 else 0)


def tuning_dict(t):
    return {"block": t.block, "chunk": t.chunk, "fused_camera": t.fused_camera, "stack_entries": t.stack_entries,
            "hints": t.hints, "chain_passes": t.chain_passes}


def time_frames(g, cams, W, H, K, params, stream, flush):
    """Render one frame per camera (K passes each) through the device path,
    L2 flushed before each (outside the events). Returns per-frame ms, per-
    launch ms and the rays traced. A frame's time is its captured graph's
    device time, from the CUDA events the library records on the launching
    stream around the graph's launches (rcp_last_pass_times, summed): events
    recorded by this loop around the call would also count any wait of the
    idle GPU for this host thread between the two records. The per-frame
    outer events are kept in time_frames.outer_ms (their excess over the
    graph's time: the descriptor upload and such waits)."""
    import torch

    from paper_2312_12392_gb300 import rcp
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    step_ms, pass_ms, rays, outer = [], [], 0, []
    for c in cams:
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        rcp.rcp_render_device(g, c, W, H, K, params, None, out, None, stream)
        e.record(stream)
        e.synchronize()
        outer.append(s.elapsed_time(e))
        pt = rcp.rcp_last_pass_times(g)
        step_ms.append(float(sum(pt)))
        pass_ms.extend(pt)
        p_, s_ = rcp.rcp_last_ray_counts(g)
        rays += p_ + s_
    time_frames.outer_ms = outer
    return step_ms, pass_ms, rays


def count_work(g, cams, W, H, K, params, sizes=None, frames=None):
    """The algorithmic work of the timed frames: an instrumented copy of the
    trace kernel run over the same cameras, K passes each, each reading the
    previous one's image. sizes: one (W, H) per camera (else W x H for all);
    frames: how many timed frames the cameras make up (default one each)."""
    import torch

    from paper_2312_12392_gb300 import rcp
    tot = dict(box=0, tri=0, sph=0, nodes=0, prim_rays=0, rays=0, frames=len(cams) if frames is None else frames)
    sizes = sizes or [(W, H)] * len(cams)
    for c, (W, H) in zip(cams, sizes):
        a = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        b = torch.empty_like(a)
        prev = None
        for n in range(K):
            dst = a if n % 2 == 0 else b
            cnt = rcp.rcp_count_pass(g, c, W, H, params, prev, dst)
            tot["box"] += cnt.box_tests
            tot["tri"] += cnt.tri_tests
            tot["sph"] += cnt.sphere_tests
            tot["nodes"] += cnt.nodes
            tot["prim_rays"] += cnt.primary_rays
            tot["rays"] += cnt.rays
            prev = dst
    return tot


def roofline(work, pass_ms, frames, workload, clk, sms):
    """The trace kernel's roofline: algorithmic FP32 lane-operations per launch
    over the mean launch time, against SMs x 128 lanes x the maximum SM clock
    (the kernel is bound by instruction issue and the ALU pipe, ncu); the byte
    view charges every node, primitive and image fetch at the measured HBM
    peak; the ncu view (issue, pipes, L1) comes from the committed profile when
    it was taken on the current sources. A launch is one pass, or all K passes
    of a frame when they ran chained: pass_ms holds the launches of `frames`
    timed frames, and the counted work (over the same cameras) is shared out
    over as many launches."""
    hbm_gbs, sm_max_mhz, peak_src = measured_peaks()
    per_frame = len(pass_ms) / max(frames, 1)
    n = max(work["frames"] * per_frame, 1)
    ops = (OPS_BOX * work["box"] + OPS_TRI * work["tri"] + OPS_SPH * work["sph"] + OPS_PIXEL * work["prim_rays"]) / n
    byts = (BYTES_NODE * work["nodes"] + BYTES_PRIM * (work["tri"] + work["sph"]) +
            BYTES_PIXEL_PASS * work["prim_rays"]) / n
    launch_s = statistics.mean(pass_ms) / 1000.0
    peak = sms * 128 * sm_max_mhz * 1e6
    prof = profiled(workload, per_frame == 1)
    roof = {"bound": "alu", "achieved": ops / launch_s / 1e12, "peak": peak / 1e12,
            "unit": "Tops/s (algorithmic FP32 lane-ops)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = prof.get("dram_bytes_per_launch") if prof else None
    roof["kernel"] = ("k_trace (camera + primary + shadow + shade, " +
                      ("one launch per pass)" if per_frame > 1 else "all K passes in one launch)"))
    roof["launch_ms"] = launch_s * 1e3
    roof["launches_per_frame"] = per_frame
    roof["launches_counted"] = n
    roof["algorithmic_ops_per_launch"] = ops
    roof["algorithmic_bytes_per_launch"] = byts
    roof["peak_source"] = f"{sms} SMs x 128 FP32 lanes x {sm_max_mhz:.0f} MHz (max SM clock)"
    roof["hbm_view"] = {"achieved_gbs": byts / launch_s / 1e9, "peak_gbs": hbm_gbs,
                        "frac": byts / launch_s / 1e9 / hbm_gbs, "peak_source": peak_src,
                        "note": "algorithmic node/primitive/image bytes charged at HBM peak; they are served "
                                "from L1/L2 (see traffic)"}
    if prof:
        roof["ncu_view"] = {k: prof[k] for k in ("issue_active_pct", "alu_pipe_pct", "fma_pipe_pct",
                                                 "l1tex_throughput_pct", "l1_hit_pct", "dram_throughput_pct",
                                                 "warp_lanes_active")
                            if k in prof}
        roof["ncu_view"]["source"] = "profiles/k_trace_ncu.json (" + prof.get("command", "") + ")"
    if clk and clk.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = roof["frac"] * sm_max_mhz / clk["sm_mhz"]
    r = max(work["rays"], 1)
    roof["per_ray"] = {"nodes": work["nodes"] / r, "box_tests": work["box"] / r, "tri_tests": work["tri"] / r}
    return roof


def e2e_host(g, cams, W, H, K, params, flush, n):
    """Frames/s through rcp_render with a host RGB buffer: the per-call
    view-descriptor upload and the image's delivery to host memory are inside
    the timed call. One untimed call first, then n timed calls; with n =
    len(cams) every camera is timed once."""
    import torch

    from paper_2312_12392_gb300 import rcp
    host = np.empty((H, W, 3), np.float32)
    t = 0.0
    for i in range(n + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rcp.rcp_render(g, cams[i % len(cams)], W, H, K, params, host)
        if i > 0:
            t += time.perf_counter() - t0
    return n / t, t


def e2e_record(value, t_unit, W, H, K, chained):
    """chained: the passes ran in one launch (one view descriptor uploaded, not K)."""
    from paper_2312_12392_gb300 import rcp
    return {"value": value, "unit": t_unit, "h2d_bytes_per_step": rcp.rcp_render_h2d_bytes(1, 1 if chained else K),
            "d2h_bytes_per_step": W * H * 3 * 4 + 4,  # the RGB image and the status word
            "api": "rcp_render (host RGB output; view descriptors H2D, RGB device-to-host inside the timed call: "
                   "written into host memory by the last pass where the device reads pageable memory "
                   "coherently, else packed and copied)"}


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
        t = parse_tuning(args.tuning)
        rcp.rcp_set_tuning(g, t)
    log(f"[rank {rank}] tuning {tuning_dict(t)}")
    poses = [sc.poses[i] for i in shard_poses(rank, world, args.steps, len(sc.poses))]
    cams = [rcp.camera_from(p) for p in poses]
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    time_frames(g, [cams[i % len(cams)] for i in range(args.warmup)], W_IMG, H_IMG, K_PASSES, params, stream, flush)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(physical_gpu(local))
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    step_ms, pass_ms, rays = time_frames(g, cams, W_IMG, H_IMG, K_PASSES, params, stream, flush)
    outer_ms = list(time_frames.outer_ms)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = float(sum(step_ms))
    tmax = max_over_ranks(total_ms, "cuda")
    rays = sum_over_ranks(rays, "cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # algorithmic work of the timed launches: the same poses, counted
    roof = roofline(count_work(g, cams, W_IMG, H_IMG, K_PASSES, params), pass_ms, len(cams), args.workload, clk,
                    sms)
    # end to end over the same poses as the device-timed frames
    e2e_fps, e2e_t = e2e_host(g, cams, W_IMG, H_IMG, K_PASSES, params, flush, len(cams))
    e2e_fps = world * len(cams) / max_over_ranks(e2e_t, "cuda")
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
        "step_timing": {"source": "CUDA events the library records on the launching stream around the graph's "
                                  "launches, summed per frame",
                        "call_bracket_ms_per_step": statistics.mean(outer_ms),
                        "call_bracket_note": "events recorded by the bench before and after each rcp_render_device "
                                             "call: also the descriptor upload and any wait of the GPU for the "
                                             "host between them"},
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded procedural scene and walk-through)",
        "config": {"workload": desc, "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "bvh_collapse": collapse_name, "bvh_split_max": max(split, 1),
                   "tuning": tuning_dict(t),
                   "tuning_source": "rcp_autotune (block x chunk x fused camera x shared stack depth x hints x chained passes)"
                   if args.tuning == "auto" else "fixed by --tuning",
                   "parallelism": f"replicas x{world} (poses split across ranks, no collective on the data path)"},
        "mrays_per_s": rays / (tmax / 1000.0) / 1e6,
        "rays_per_frame": rays / frames,
        "roofline": roof,
        "e2e": e2e_record(e2e_fps, "frames/s", W_IMG, H_IMG, K_PASSES,
                          roof["launches_per_frame"] == 1),
        "gpu_launches": len(pass_ms) * (1 if t.fused_camera else 2),  # trace launches (+ camera kernels)
        "clocks": clk,
        "wall_s": wall,
    }
    rcp.rcp_scene_destroy(g)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        fps, npx, secs = cpu_oracle_sample(sc, poses[:2], target_s=args.cpu_seconds / 2)
        res["cpu_baseline"] = {"value": fps, "unit": "frames/s", "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"{npx} seeded pixels (full K=6 chains) over 2 poses in {secs:.1f} s, "
                                         f"extrapolated to 1920x1080 frames"}
    if args.extras and args.workload == "mid" and world == 1:
        for name, fn in (("forest", forest_summary), ("batched", batched_summary), ("served", served_summary),
                         ("stress", stress_summary), ("mappings", mappings_summary)):
            t1 = time.perf_counter()
            res[name] = fn(args)
            res[name]["bench_wall_s"] = time.perf_counter() - t1
            log(f"{name}: {json.dumps(res[name])[:400]}")
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        dist.destroy_process_group()


def forest_summary(args):
    """The 1.07M-triangle forest at 1080p K=6 over its whole 64-pose
    walk-through (same protocol as the headline: L2 flushed between frames,
    CUDA events), with its own clock record, roofline (work counted on the same
    64 poses) and end-to-end figure through rcp_render with host output."""
    import torch

    from paper_2312_12392_gb300 import rcp
    sc, desc = make_workload("forest")
    d = sc.diameter()
    params = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    collapse, collapse_name = collapse_for(args, "forest")
    split = split_for(args, "forest")
    g = rcp.scene_from(sc, collapse, split)
    try:
        cams = [rcp.camera_from(p) for p in sc.poses[: max(1, args.forest_poses)]]
        if args.tuning == "auto":
            t = rcp.rcp_autotune(g, cams[0], W_IMG, H_IMG, params,
                                 os.path.join(ROOT, "paper_2312_12392_gb300", "tuning_cache.json"))
        else:
            t = parse_tuning(args.tuning)
            rcp.rcp_set_tuning(g, t)
        stream = torch.cuda.current_stream()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        time_frames(g, cams[:3], W_IMG, H_IMG, K_PASSES, params, stream, flush)
        torch.cuda.synchronize()
        clocks = ClockSampler(physical_gpu(0))
        clocks.start()
        time.sleep(0.3)
        ms, pass_ms, rays = time_frames(g, cams, W_IMG, H_IMG, K_PASSES, params, stream, flush)
        clk = clocks.stop()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        roof = roofline(count_work(g, cams, W_IMG, H_IMG, K_PASSES, params), pass_ms, len(cams), "forest", clk,
                        sms)
        e2e_fps, _ = e2e_host(g, cams, W_IMG, H_IMG, K_PASSES, params, flush, len(cams))
        tot = sum(ms) / 1000.0
        info = rcp.rcp_scene_get_info(g)
        return {"workload": desc, "frames_per_s": len(cams) / tot, "mrays_per_s": rays / tot / 1e6,
                "ms_per_frame": 1000 * tot / len(cams), "frames": len(cams), "roofline": roof,
                "e2e": e2e_record(e2e_fps, "frames/s", W_IMG, H_IMG, K_PASSES,
                          roof["launches_per_frame"] == 1), "clocks": clk,
                "tuning": tuning_dict(t), "bvh_build_ms": info.build_ms, "nodes": info.n_nodes,
                "depth": info.depth, "bvh_collapse": collapse_name, "bvh_split_max": max(split, 1),
                "records": info.n_records, "gpu_launches": len(pass_ms)}
    finally:
        rcp.rcp_scene_destroy(g)


def mappings_summary(args):
    """The mid terrain at 1080p K=6 under every camera mapping of the paper,
    each autotuned, timed and counted like the headline over the first 16
    poses: EYE (the headline's), TARGET (§3), DEPTH (§4, z0 at the focal
    distance), NORMAL (§5), and EYE with 4 jittered samples per pixel per
    pass (§2; one launch per pass, the samples reading the previous image
    bilinearly)."""
    import torch

    from paper_2312_12392_gb300 import rcp
    sc, _ = make_workload("mid")
    d = sc.diameter()
    k, f = 0.02 * d, 0.1 * d
    g = rcp.scene_from(sc, collapse_for(args, "mid")[0])
    jitter = np.random.default_rng(11).random((4, 2))
    variants = [("eye", rcp.make_params(rcp.RCP_MAP_EYE, k, f)),
                ("target", rcp.make_params(rcp.RCP_MAP_TARGET, k, f)),
                ("depth", rcp.make_params(rcp.RCP_MAP_DEPTH, k, f, z0=f)),
                ("normal", rcp.make_params(rcp.RCP_MAP_NORMAL, k, f)),
                ("eye_4spp", rcp.make_params(rcp.RCP_MAP_EYE, k, f, jitter=jitter))]
    try:
        cams = [rcp.camera_from(p) for p in sc.poses[:16]]
        stream = torch.cuda.current_stream()
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        out = {}
        for name, params in variants:
            t = rcp.rcp_autotune(g, cams[0], W_IMG, H_IMG, params,
                                 os.path.join(ROOT, "paper_2312_12392_gb300", "tuning_cache.json"))
            time_frames(g, cams[:3], W_IMG, H_IMG, K_PASSES, params, stream, flush)
            torch.cuda.synchronize()
            clocks = ClockSampler(physical_gpu(0))
            clocks.start()
            time.sleep(0.3)
            ms, pass_ms, rays = time_frames(g, cams, W_IMG, H_IMG, K_PASSES, params, stream, flush)
            clk = clocks.stop()
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            roof = roofline(count_work(g, cams, W_IMG, H_IMG, K_PASSES, params), pass_ms, len(cams),
                            "mid_" + name, clk, sms)
            tot = sum(ms) / 1000.0
            out[name] = {"frames_per_s": len(cams) / tot, "mrays_per_s": rays / tot / 1e6,
                         "ms_per_frame": 1000 * tot / len(cams), "roofline_frac": roof["frac"],
                         "launch_ms": roof["launch_ms"], "launches_per_frame": roof["launches_per_frame"],
                         "tuning": tuning_dict(t), "clocks": clk}
        return {"workload": "mid terrain 133k tris, 1920x1080, K=6, 16 poses of the walk-through; k=0.02*diam, "
                            "f=0.1*diam, DEPTH z0=f, 4 jittered samples from a seeded table",
                "frames": len(cams), "variants": out}
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


# ------------------------------------------------------------------ batched, served and stress workloads

def one_line(metric, value, unit, args, steps, extra):
    out = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": steps, "warmup": args.warmup,
           "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic"}
    out.update(extra)
    return out


def batched_summary(args):
    """64 views of uneven size (W in [256,1920], H in [256,1080], seeded) of the
    1.07M-triangle forest, K = 6: one persistent launch over all views (all
    passes chained, or one launch per pass, as tuned; graph-captured,
    autotuned), against rendering the same views one after another with the
    single-view device path. The roofline counts the batch's work over its
    launches."""
    import torch

    from paper_2312_12392_gb300 import rcp, scenes
    sc, _ = make_workload("forest")
    d = sc.diameter()
    params = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    collapse, collapse_name = collapse_for(args, "batched")
    split = split_for(args, "batched")
    g = rcp.scene_from(sc, collapse, split)
    try:
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

        steps = max(3, min(args.steps, 20))
        res, batch_launch_ms = {}, []
        clocks = ClockSampler(physical_gpu(0))
        for name, fn in (("batched", batch_once), ("plain", plain_once)):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            if name == "batched":
                clocks.start()
            ms = []
            for _ in range(steps):
                flush.zero_()
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record(stream)
                fn()
                e.record(stream)
                e.synchronize()
                ms.append(s.elapsed_time(e))
                if name == "batched":
                    batch_launch_ms.extend(rcp.rcp_last_pass_times(g))
            if name == "batched":
                clk = clocks.stop()
            res[name] = statistics.mean(ms)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        roof = roofline(count_work(g, cams, 0, 0, K_PASSES, params, sizes=sizes, frames=1), batch_launch_ms,
                        steps, "batched", clk, sms)
        pix = sum(w * h for w, h in sizes)
        batch_once()
        torch.cuda.synchronize()
        p_, s_ = rcp.rcp_last_ray_counts(g)
        launches = len(rcp.rcp_last_pass_times(g))
        return {"views_per_s": len(sizes) / (res["batched"] / 1000.0), "ms_per_batch": res["batched"],
                "plain_views_per_s": len(sizes) / (res["plain"] / 1000.0), "plain_ms_per_batch": res["plain"],
                "speedup_vs_plain": res["plain"] / res["batched"],
                "mrays_per_s": (p_ + s_) / (res["batched"] / 1000.0) / 1e6, "steps": steps,
                "workload": f"forest 1.07M tris, 64 views ({pix / 1e6:.1f} Mpixel total), K=6, " +
                            ("one launch per pass" if launches > 1 else "one launch for all passes") +
                            " over all views, graph-captured",
                "bvh_collapse": collapse_name, "bvh_split_max": max(split, 1), "tuning": tuning_dict(t),
                "l2": "flushed between steps", "gpu_launches": steps * launches, "roofline": roof, "clocks": clk}
    finally:
        rcp.rcp_scene_destroy(g)


def pinned_array(shape):
    """A float32 numpy array in page-locked host memory (torch's pinned
    allocator): the GPU writes it through its own page tables."""
    import torch
    return torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy()


class BufferPool:
    """Page-locked host output buffers, `per_shape` per resolution, handed out
    round robin: request i of a resolution writes into buffer (i mod
    per_shape). Both paths of the served comparison use the same pool, as a
    frame server hands its renderer page-locked frame buffers: the last pass
    writes them directly through the GPU's page tables, whereas pageable
    buffers the GPU has not written recently cost address-translation misses
    on every page (measured on the served mix: both paths several times
    slower)."""

    def __init__(self, per_shape):
        self.per_shape = per_shape
        self.bufs = {}
        self.owner = {}
        self.waits = 0

    def get(self, i, w, h, wait=None):
        pool = self.bufs.setdefault((w, h), [pinned_array((h, w, 3)) for _ in range(self.per_shape)])
        n = self.owner.setdefault((w, h), [0, [None] * self.per_shape])
        j = n[0] % self.per_shape
        n[0] += 1
        prev = n[1][j]
        if prev is not None and wait is not None and wait(prev):
            self.waits += 1
        n[1][j] = i
        return pool[j]

    def release_all(self):
        """Every request that used a buffer is done."""
        for k in self.owner:
            self.owner[k][1] = [None] * self.per_shape

    def all_buffers(self):
        for (w, h), v in self.bufs.items():
            for b in v:
                yield w, h, b


def served_summary(args):
    """Poisson arrivals over 4 resident terrain scenes (0.1M, 1M, 3M, 5M tris);
    each request: a walk-through pose, 720p/1080p/1440p/2160p, K in 1..8,
    k in [0, 0.05] * diameter. The continuous-batching server against the plain
    path (one request at a time, FIFO, each its own render: all K passes
    chained in one launch, the scenes' default tuning), same arrivals, at each
    rate."""
    import threading

    from paper_2312_12392_gb300 import rcp, scenes
    grids = [221, 706, 1224, 1580]
    scs = [scenes.terrain_scene(gsz, seed=4) for gsz in grids]
    collapse, collapse_name = collapse_for(args, "served")
    gs = [rcp.scene_from(s, collapse) for s in scs]
    try:
        n_req = args.served_requests
        reqs = scenes.served_requests(n_req, len(scs), 64, seed=4)
        diams = [s.diameter() for s in scs]
        prepared = [(rcp.camera_from(scs[r["scene"]].poses[r["pose"]]),
                     rcp.make_params(rcp.RCP_MAP_EYE, r["k_frac"] * diams[r["scene"]], 0.1 * diams[r["scene"]]))
                    for r in reqs]
        pool = BufferPool(24)
        # warm both paths: every distinct request shape once through the plain
        # path (its render contexts and graphs), every pool buffer written once
        # by a render, a burst through a server
        seen = set()
        for i, r in enumerate(reqs):
            key = (r["scene"], r["width"], r["height"], r["K"])
            if key not in seen:
                seen.add(key)
                rcp.rcp_render(gs[r["scene"]], prepared[i][0], r["width"], r["height"], r["K"], prepared[i][1],
                               pool.get(i, r["width"], r["height"]))
        for j in range(pool.per_shape):
            for r in ({"width": w, "height": h} for w, h in {(q["width"], q["height"]) for q in reqs}):
                rcp.rcp_render(gs[0], prepared[0][0], r["width"], r["height"], 1, prepared[0][1],
                               pool.get(j, r["width"], r["height"]))
        pool.release_all()
        srv = rcp.rcp_server_create(int(args.serve_budget_gb * (1 << 30)), args.serve_slots)
        # the device writes each request's RGB into its buffer during the last
        # pass: every buffer stays alive until its request is done
        warm_bufs = [np.zeros((r["height"], r["width"], 3), np.float32) for r in reqs[:16]]
        tks = [rcp.rcp_server_submit(srv, gs[r["scene"]], prepared[i][0], r["width"], r["height"], r["K"],
                                     prepared[i][1], warm_bufs[i])
               for i, r in enumerate(reqs[:16])]
        for tk in tks:
            rcp.rcp_server_wait(srv, tk, 600.0)
        rcp.rcp_server_destroy(srv)
        del warm_bufs
        table = []
        for lam in [float(x) for x in args.rates.split(",")]:
            arr = scenes.poisson_arrivals(lam, n_req, seed=4)
            # -- plain: FIFO worker, one request at a time (synchronous: every
            #    buffer is free again when the next request starts)
            lat = [0.0] * n_req
            t0 = time.perf_counter()

            def plain_worker():
                for i, r in enumerate(reqs):
                    wait = arr[i] - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(wait)
                    rcp.rcp_render(gs[r["scene"]], prepared[i][0], r["width"], r["height"], r["K"],
                                   prepared[i][1], pool.get(i, r["width"], r["height"]))
                    lat[i] = time.perf_counter() - t0 - arr[i]

            th = threading.Thread(target=plain_worker)
            th.start()
            th.join()
            plain_span = time.perf_counter() - t0
            plain = {"frames_per_s": n_req / plain_span, "p50_ms": 1000 * float(np.percentile(lat, 50)),
                     "p99_ms": 1000 * float(np.percentile(lat, 99))}
            # -- server: submit at the arrival times (latency from submit to the
            #    image in the caller's buffer; late submits are reported)
            srv = rcp.rcp_server_create(int(args.serve_budget_gb * (1 << 30)), args.serve_slots)
            rcp.rcp_server_set_max_chain(srv, args.serve_max_chain)
            if args.serve_step_pixels is not None:
                rcp.rcp_server_set_step_pixels(srv, args.serve_step_pixels)
            pool.release_all()
            pool.waits = 0
            tickets, late, t_sub = [], 0.0, []

            def wait_if_busy(j):
                if rcp.rcp_server_poll(srv, tickets[j]):
                    return False
                rcp.rcp_server_wait(srv, tickets[j], 600.0)
                return True

            t0 = time.perf_counter()
            for i, r in enumerate(reqs):
                wait = arr[i] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                # a buffer still in use by an earlier request (only under
                # overload) is waited for before it is handed out again
                buf = pool.get(i, r["width"], r["height"], wait_if_busy)
                t_sub.append(time.perf_counter() - t0)
                late = max(late, t_sub[-1] - arr[i])
                tickets.append(rcp.rcp_server_submit(srv, gs[r["scene"]], prepared[i][0], r["width"], r["height"],
                                                     r["K"], prepared[i][1], buf))
            for tk in tickets:
                rcp.rcp_server_wait(srv, tk, 600.0)
            st = rcp.rcp_server_stats_get(srv)
            # latency from arrival, as for the plain path: any wait before the
            # submit plus the request's submit-to-done time
            lat_s = [1000.0 * (t_sub[i] - arr[i]) + rcp.rcp_server_latency(srv, tk) for i, tk in enumerate(tickets)]
            rcp.rcp_server_destroy(srv)
            span = st.frames_per_s and st.completed / st.frames_per_s
            served = {"frames_per_s": st.frames_per_s, "p50_ms": float(np.percentile(lat_s, 50)),
                      "p99_ms": float(np.percentile(lat_s, 99)), "p50_ms_from_submit": st.p50_ms,
                      "p99_ms_from_submit": st.p99_ms,
                      "mrays_per_s": st.mrays_per_s, "steps": st.steps, "peak_gb": st.device_bytes_peak / 2 ** 30,
                      "device_busy_frac": st.device_busy_ms / 1000.0 / span if span else None,
                      "max_submit_late_ms": 1000.0 * late, "buffer_waits": pool.waits}
            table.append({"rate_req_s": lam, "served": served, "plain": plain})
            log(f"lambda={lam}: served {served} | plain {plain}")
        return {"requests_per_rate": n_req, "slots": args.serve_slots, "budget_gb": args.serve_budget_gb,
                "max_chain": args.serve_max_chain, "step_pixel_passes": args.serve_step_pixels,
                "bvh_collapse": collapse_name,
                "workload": "4 resident terrain scenes (100,082 / 999,272 / 2,998,752 / 4,995,200 tris); "
                            "720p-2160p, K in 1..8, k in [0, 0.05]*diam, Poisson arrivals; latency from arrival "
                            "to the image in the caller's host buffer",
                "plain_path": "one rcp_render per request (host output, the K passes chained in one launch), "
                              "FIFO, one worker thread",
                "sweep": table}
    finally:
        for g in gs:
            rcp.rcp_scene_destroy(g)


def stress_summary(args):
    """25,000-tree forest (12.57M triangles), 3840x2160, K=8: every frame the
    wind sways the trees (input generated on the device with torch), the BVH is
    refitted (rcp_scene_update_vertices_device) and the frame is rendered."""
    import torch

    from paper_2312_12392_gb300 import rcp, scenes
    t0 = time.perf_counter()
    sc = scenes.forest_scene(25_000, seed=5)
    gen_s = time.perf_counter() - t0
    W, H, K = 3840, 2160, 8
    d = sc.diameter()
    params = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * d, 0.1 * d)
    collapse, collapse_name = collapse_for(args, "stress")
    split = split_for(args, "stress")
    g = rcp.scene_from(sc, collapse, split)
    g2 = None
    try:
        info = rcp.rcp_scene_get_info(g)
        base = torch.from_numpy(sc.tris).cuda().reshape(-1, 3, 3)
        amp = torch.from_numpy(sc.sway_amp).cuda()
        phase = torch.from_numpy(sc.sway_phase).cuda()
        moved = torch.empty_like(base)
        out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
        stream = torch.cuda.current_stream()
        steps = max(3, args.stress_steps)
        cams = [rcp.camera_from(sc.poses[i % len(sc.poses)]) for i in range(steps + args.warmup)]

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
        refit_ms, render_ms, frame_ms, rays, launch_ms = [], [], [], 0, []
        work = None
        clocks = ClockSampler(physical_gpu(0))
        clocks.start()
        for i in range(args.warmup, args.warmup + steps):
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
            launch_ms.extend(rcp.rcp_last_pass_times(g))
            # this frame's work on this frame's tree, counted outside the events
            w = count_work(g, [cams[i]], W, H, K, params)
            work = w if work is None else {k: work[k] + w[k] for k in work}
        clk = clocks.stop()
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        roof = roofline(work, launch_ms, steps, "stress", clk, sms)
        rcp.rcp_scene_validate(g)
        tot = sum(frame_ms) / 1000.0
        # End to end, every frame's RGB delivered to host memory, the same frames:
        # (1) one stream: sway, refit, render, copy out, frame after frame;
        # (2) the serving path with two copies of the scene used in turn, so that
        #     frame f's sway and refit overlap frame f-1's render and copy-out (a
        #     copy is refitted only once the request two frames back, its last
        #     user, is done). Three host buffers rotate (at most two in flight).
        frames = [args.warmup + i for i in range(steps)]
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
            tickets.append(rcp.rcp_server_submit(srv, copies[i % 2], cams[f], W, H, K, params,
                                                 bufs["served"][i % 3]))
        for tk in tickets[-2:]:
            rcp.rcp_server_wait(srv, tk, 600.0)
        served_s = time.perf_counter() - t0
        st = rcp.rcp_server_stats_get(srv)
        rcp.rcp_server_destroy(srv)
        same_last = bool(np.array_equal(bufs["single"][(steps - 1) % 3], bufs["served"][(steps - 1) % 3]))
        out_bytes = H * W * 3 * 4
        return {"frames_per_s": steps / tot, "ms_per_frame": 1000 * tot / steps, "frames": steps,
                "refit_ms": statistics.mean(refit_ms), "render_ms": statistics.mean(render_ms),
                "mrays_per_s": rays / tot / 1e6,
                "workload": f"stress: {info.n_tris:,} tris (25,000 swaying cone trees), 3840x2160, K=8, wind sway "
                            "A=0.02*h_tree at 0.5 Hz, refit every frame",
                "bvh_collapse": collapse_name, "bvh_split_max": split, "records": info.n_records,
                "scene_generation_s": gen_s, "bvh_build_ms": info.build_ms, "nodes": info.n_nodes,
                "depth": info.depth, "gpu_launches_per_step": len(launch_ms) // steps + 2 + info.depth,
                "roofline": roof, "clocks": clk,
                "e2e": {"value": steps / single_s, "unit": "frames/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": out_bytes,
                        "api": "single stream: rcp_scene_update_vertices_device + rcp_render (host RGB) per frame"},
                "served_e2e": {"value": steps / served_s, "unit": "frames/s", "p50_ms": st.p50_ms, "p99_ms": st.p99_ms,
                               "d2h_bytes_per_step": out_bytes, "last_frame_identical_to_single_stream": same_last,
                               "api": "rcp_server_submit (host RGB), two scene copies refitted in turn"}}
    finally:
        if g2:
            rcp.rcp_scene_destroy(g2)
        rcp.rcp_scene_destroy(g)


def run_workload_line(args, name):
    """One workload's own line (--workload forest|batched|served|stress|mappings)."""
    import torch

    from paper_2312_12392_gb300 import build as B
    torch.cuda.set_device(0)
    B.build()
    if name == "forest":
        r = forest_summary(args)
        out = one_line("frames_per_s (forest, 1080p, K=6)", r["frames_per_s"], "frames/s", args, r["frames"], r)
        out.update(ms_per_step=r["ms_per_frame"], e2e=r["e2e"], roofline=r["roofline"], clocks=r["clocks"])
    elif name == "batched":
        r = batched_summary(args)
        out = one_line("views_per_s (64 uneven views, K=6 each, one persistent launch over all views)",
                       r["views_per_s"], "views/s", args, r["steps"], r)
        out["ms_per_step"] = r["ms_per_batch"]
    elif name == "mappings":
        r = mappings_summary(args)
        v = r["variants"]["eye_4spp"]
        out = one_line("frames_per_s (mid 1080p K=6, 4 jittered samples per pixel; every mapping alongside)",
                       v["frames_per_s"], "frames/s", args, r["frames"], r)
        out["ms_per_step"] = v["ms_per_frame"]
    elif name == "served":
        r = served_summary(args)
        best = max(r["sweep"], key=lambda x: x["served"]["frames_per_s"])
        out = one_line("served frames_per_s and p50/p99 latency vs the plain per-request path",
                       best["served"]["frames_per_s"], "frames/s", args, r["requests_per_rate"], r)
        out["ms_per_step"] = 1000.0 / best["served"]["frames_per_s"]
    else:
        r = stress_summary(args)
        out = one_line("frames_per_s (3840x2160, K=8, per-frame refit)", r["frames_per_s"], "frames/s", args,
                       r["frames"], r)
        out.update(ms_per_step=r["ms_per_frame"], e2e=r["e2e"])
    print(json.dumps(out), flush=True)


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
    ap.add_argument("--workload", default="mid",
                    choices=["mid", "forest", "batched", "served", "stress", "mappings", "imagespace"])
    ap.add_argument("--tuning", default="auto",
                    help="'auto' (the library's autotuner, cached per GPU, scene size, tree depth and view) or "
                         "block,chunk,fused_camera[,stack_entries[,hints[,chain_passes]]] (stack 0 = one entry per "
                         "tree level; hints: bit 0 primary, bit 1 shadow, default 3; chain_passes 1 = all K passes "
                         "in one launch)")
    ap.add_argument("--collapse", default="auto", choices=["auto", "area", "sah"],
                    help="BVH collapse policy; auto: sah for the forest workloads, area for the terrains")
    ap.add_argument("--split", default="auto", choices=["auto"] + [str(i) for i in range(9)],
                    help="references per triangle at most (early split clipping); auto: 8 for the forests "
                         "(static and swaying), 0 for the terrains")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="the headline line without the forest, batched, served, stress and mappings summaries")
    ap.add_argument("--rates", default="100,200,400", help="served: arrival rates (req/s)")
    ap.add_argument("--served-requests", type=int, default=1000, help="served: requests per rate")
    ap.add_argument("--stress-steps", type=int, default=20, help="stress: timed frames")
    ap.add_argument("--forest-poses", type=int, default=64, help="forest: walk-through poses timed (all 64)")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-max-chain", type=int, default=16,
                    help="served: passes a request may advance by in one server step (1 = one pass per step)")
    ap.add_argument("--serve-budget-gb", type=float, default=24.0)
    ap.add_argument("--serve-step-pixels", type=int, default=None,
                    help="served: pixel-passes per server step (default: the library's; 0 = unbounded)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        log("warmup raised to 3 (timing rule)")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("forest", "batched", "served", "stress", "mappings"):
        run_workload_line(args, args.workload)
    elif args.workload == "imagespace":
        run_imagespace(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
