"""The ABI's storage format of a hit normal, as include/rcp.h defines it for
RCP_MAP_NORMAL images: a 32-bit octahedral code in the fourth float of each
rgbz pixel. The tests use it to hand the oracle's FP64 normals to the CUDA path
and to read the normals the CUDA path writes back; the oracle itself carries
normals as double-precision vectors and never sees a code.

Vectorised numpy, written from the header's description:
  p = (n.x, n.y) / (|n.x| + |n.y| + |n.z|), folded for n.z < 0 to
  ((1 - |p.y|) sgn p.x, (1 - |p.x|) sgn p.y), sgn 0 = +1;
  q = round(32767 p); code = (q.x + 32768) | (q.y + 32768) << 16; 0 = none.
"""
from __future__ import annotations

import numpy as np

ROUND_TRIP_TOL = 1e-4  # the header's bound on |decode(encode(n)) - n|


def _sgn(x):
    return np.where(x >= 0, 1.0, -1.0)


def normal_encode(n) -> np.ndarray:
    """(m, 3) unit vectors (zero rows = no normal) -> (m,) uint32 codes."""
    n = np.asarray(n, np.float64).reshape(-1, 3)
    s = np.abs(n).sum(axis=1)
    ok = s > 0
    ss = np.where(ok, s, 1.0)
    px, py = n[:, 0] / ss, n[:, 1] / ss
    fold = n[:, 2] < 0
    fx = (1.0 - np.abs(py)) * _sgn(px)
    fy = (1.0 - np.abs(px)) * _sgn(py)
    px, py = np.where(fold, fx, px), np.where(fold, fy, py)
    # round half away from zero, as C's round()
    qx = np.trunc(px * 32767.0 + np.where(px >= 0, 0.5, -0.5)).astype(np.int64)
    qy = np.trunc(py * 32767.0 + np.where(py >= 0, 0.5, -0.5)).astype(np.int64)
    code = ((qx + 32768) | ((qy + 32768) << 16)).astype(np.uint32)
    return np.where(ok, code, np.uint32(0)).astype(np.uint32)


def normal_decode(codes):
    """(m,) uint32 codes -> ((m, 3) unit vectors, (m,) bool valid); code 0 decodes to zero, invalid."""
    c = np.asarray(codes).astype(np.uint32).reshape(-1)
    valid = c != 0
    px = ((c & 0xFFFF).astype(np.float64) - 32768.0) / 32767.0
    py = ((c >> 16).astype(np.float64) - 32768.0) / 32767.0
    z = 1.0 - np.abs(px) - np.abs(py)
    fold = z < 0
    x = np.where(fold, (1.0 - np.abs(py)) * _sgn(px), px)
    y = np.where(fold, (1.0 - np.abs(px)) * _sgn(py), py)
    v = np.stack([x, y, z], axis=1)
    ln = np.linalg.norm(v, axis=1, keepdims=True)
    v = v / np.where(ln > 0, ln, 1.0)
    v[~valid] = 0.0
    return v, valid


def codes_to_lane(codes) -> np.ndarray:
    """uint32 codes -> the float32 values whose bits they are (the image's fourth lane)."""
    return np.asarray(codes, np.uint32).view(np.float32)


def lane_to_codes(lane) -> np.ndarray:
    return np.ascontiguousarray(lane, np.float32).view(np.uint32)
