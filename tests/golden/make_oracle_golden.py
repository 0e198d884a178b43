"""Write the oracle's expected values for the full-size parity samples that
take the brute-force oracle too long to recompute inside a test run.

    python tests/golden/make_oracle_golden.py [forest] [stress] [--threads N]

Only ``oracle`` computes here; ``paper_2312_12392_gb300.scenes`` generates the
seeded inputs (scene, walk-through, wind sway, pixel sample) and holds none of
the method's arithmetic. Nothing from the CUDA path is read.

For each workload and pose the file holds a per-pass chain over a seeded pixel
sample, exactly as the GPU test replays it: pass 1 from I_0, and before every
later pass each sampled pixel's previous value is the oracle's own output of
the pass before, rounded to float32 (each pixel's chain depends only on its own
previous value, §3, so the unsampled pixels do not matter). Stored per pass:
colour and z-depth (float32), hit id, ORC_FLAG_* bits. The forest file also
holds one pose's end-to-end K-pass chain (carried in double) for the PSNR test.

Each file records a hash of the oracle's source (comments and layout ignored)
and of the inputs, so a test can tell when it is stale.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import re
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2312_12392_gb300 import scenes  # noqa: E402

W_MID, H_MID = 1920, 1080


def oracle_source_hash() -> str:
    """sha256 of the oracle's C source and header, comments and whitespace removed."""
    h = hashlib.sha256()
    for name in ("rcp_oracle.c", "rcp_oracle.h"):
        src = open(os.path.join(ROOT, "oracle", name), encoding="utf-8").read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(name.encode() + b"\0" + " ".join(src.split()).encode())
    return h.hexdigest()[:16]


def input_hash(tris, albedo, cams, pix_list, extra=()) -> str:
    h = hashlib.sha256()
    for a in (tris, albedo, *cams, *pix_list):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(repr(tuple(extra)).encode())
    return h.hexdigest()[:16]


def forest_spec():
    sc = scenes.forest_scene()
    return dict(name="forest", scene=sc, W=W_MID, H=H_MID, K=6, poses=[10, 31, 52], n=16384, seed0=300,
                e2e_pose=10, diam=sc.diameter())


def stress_spec():
    base = scenes.forest_scene(25_000, seed=5)
    frame = 123
    moved = scenes.sway_vertices(base.tris, base.sway_amp, base.sway_phase, frame)
    sc = scenes.Scene("stress moved", moved, base.spheres, base.albedo, base.light, base.poses)
    # the k and f of the workload come from the unmoved scene's diameter
    return dict(name="stress", scene=sc, W=3840, H=2160, K=8, poses=[frame % len(base.poses)], n=4096,
                seed0=frame, e2e_pose=None, diam=base.diameter(), frame=frame)


SPECS = {"forest": forest_spec, "stress": stress_spec}


def path_of(name: str) -> str:
    return os.path.join(HERE, f"oracle_{name}.npz")


def sample_of(spec, i):
    return scenes.pixel_subset(spec["W"], spec["H"], spec["n"], seed=spec["seed0"] + i)


def params_of(spec):
    f32 = lambda x: float(np.float32(x))
    return f32(0.02 * spec["diam"]), f32(0.1 * spec["diam"])


def generate(name: str, nthreads: int = 0) -> str:
    spec = SPECS[name]()
    sc = spec["scene"]
    W, H, K = spec["W"], spec["H"], spec["K"]
    k, f = params_of(spec)
    o = O.OracleScene(sc.tris, sc.spheres, sc.albedo, sc.light.type,
                      np.asarray(sc.light.v, np.float32).astype(np.float64), float(np.float32(sc.light.ambient)))
    out = {}
    cams, pixs = [], []
    for i, pose in enumerate(spec["poses"]):
        pix = sample_of(spec, i)
        cam = sc.poses[pose].as_array().astype(np.float32).astype(np.float64)
        cams.append(cam)
        pixs.append(pix)
        img = np.zeros((H * W, 4), np.float32)
        rgbz, prim, flag = [], [], []
        t0 = time.perf_counter()
        for n in range(K):
            r, p, fl = o.render_pass(cam, W, H, O.MAP_EYE, k, f, in_rgbz=None if n == 0 else img, pix=pix,
                                     nthreads=nthreads)
            rgbz.append(r.astype(np.float32))
            prim.append(p)
            flag.append(fl)
            img[pix] = r.astype(np.float32)
            print(f"{name} pose {pose} pass {n + 1}/{K}: {time.perf_counter() - t0:.0f} s", flush=True)
        out[f"pix_{i}"] = pix
        out[f"rgbz_{i}"] = np.stack(rgbz)
        out[f"prim_{i}"] = np.stack(prim)
        out[f"flag_{i}"] = np.stack(flag)
        if pose == spec["e2e_pose"]:
            r, _, fl = o.render(cam, W, H, K, O.MAP_EYE, k, f, pix=pix, nthreads=nthreads)
            out["e2e_rgb"] = r[:, :3].astype(np.float32)
            out["e2e_flag"] = fl
            out["e2e_index"] = np.int64(i)
    meta = dict(workload=name, W=W, H=H, K=K, k=k, f=f, poses=spec["poses"], n=spec["n"],
                oracle=oracle_source_hash(),
                inputs=input_hash(sc.tris, sc.albedo, cams, pixs, (k, f)))
    out["meta"] = np.array(repr(meta))
    path = path_of(name)
    np.savez_compressed(path, **out)
    return path


def load(name: str):
    """The stored values and their metadata; raises if the oracle's source has
    changed since they were written."""
    import ast
    d = np.load(path_of(name))
    meta = ast.literal_eval(str(d["meta"]))
    if meta["oracle"] != oracle_source_hash():
        raise RuntimeError(f"{path_of(name)} was written by another oracle version: rerun "
                           f"tests/golden/make_oracle_golden.py {name}")
    return d, meta


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("names", nargs="*", default=sorted(SPECS))
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args(argv)
    for name in a.names:
        t0 = time.perf_counter()
        p = generate(name, a.threads)
        print(f"wrote {p} ({os.path.getsize(p) / 1e6:.1f} MB) in {time.perf_counter() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
