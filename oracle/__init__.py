"""FP64 brute-force CPU oracle for Recursive Camera Painting (arXiv 2312.12392).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this package to check and time the CUDA path;
the CUDA library and its Python binding never import it. It shares no code with
the CUDA path: ``rcp_oracle.c`` is plain C, compiled here with gcc.

Images exchanged with the oracle are (H, W, 4) float32 arrays: RGB in [0, 1]
and the z-depth of the primary hit along the camera's view axis (0 on a miss)
in the fourth lane. The normal mapping's previous hit normals travel beside
the image as (H, W, 3) float64 unit vectors (zero = no normal).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rcp_oracle.c")
_HDR = os.path.join(_HERE, "rcp_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

MAP_EYE, MAP_TARGET, MAP_DEPTH, MAP_NORMAL = 0, 1, 2, 4
LIGHT_POINT, LIGHT_DIRECTIONAL = 0, 1
FLAG_ID, FLAG_SHADOW, FLAG_POINT = 1, 2, 4
TOL = 1e-5
IMG_TOL = 2.0 ** -21


def build(force: bool = False, extra_flags=()) -> str:
    """Compile the oracle with gcc (-O2, no fast-math: IEEE double throughout)."""
    os.makedirs(_BUILD, exist_ok=True)
    out = _LIB if not extra_flags else os.path.join(_BUILD, "liborc_" + "_".join(
        f.strip("-").replace("=", "") for f in extra_flags) + ".so")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = out + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
               *extra_flags, _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, out)
    return out


def _bind(lib):
    d, i64, i32 = C.c_double, C.c_int64, C.c_int
    fp = C.POINTER(C.c_float)
    dp = C.POINTER(C.c_double)
    lp = C.POINTER(C.c_int64)
    ip = C.POINTER(C.c_int32)
    up = C.POINTER(C.c_uint8)
    lib.orc_scene_new.restype = C.c_void_p
    lib.orc_scene_new.argtypes = [fp, i64, fp, i64, fp, i32, dp, d]
    lib.orc_scene_free.argtypes = [C.c_void_p]
    lib.orc_scene_diam.restype = d
    lib.orc_scene_diam.argtypes = [C.c_void_p]
    lib.orc_camera_ray.restype = i32
    lib.orc_camera_ray.argtypes = [dp, i32, i32, i32, i32, i32, d, d, d, dp, d, dp, dp, dp]
    lib.orc_hit_triangle.argtypes = [dp, dp, dp, dp, dp, d, d, dp]
    lib.orc_hit_sphere.argtypes = [dp, d, dp, dp, d, d, dp]
    lib.orc_trace_closest.argtypes = [C.c_void_p, dp, dp, d, d, dp, lp, C.POINTER(C.c_int)]
    lib.orc_trace_any.argtypes = [C.c_void_p, dp, dp, d, d, d, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.orc_shade_ray.argtypes = [C.c_void_p, dp, dp, dp, dp, lp, C.POINTER(C.c_int)]
    lib.orc_render_pass.restype = i32
    lib.orc_render_pass.argtypes = [C.c_void_p, dp, i32, i32, i32, d, d, d, fp, dp, lp, i64, dp, dp, ip, up, i32]
    lib.orc_imagespace_pass.restype = i32
    lib.orc_imagespace_pass.argtypes = [fp, fp, i32, i32, d, lp, i64, fp, up]
    lib.orc_mirror_index.restype = i64
    lib.orc_mirror_index.argtypes = [i64, i64]
    lib.orc_render_pass_ms.restype = i32
    lib.orc_render_pass_ms.argtypes = [C.c_void_p, dp, i32, i32, i32, d, d, d, i32, fp, fp, dp, lp, i64, dp, dp, ip,
                                       up, i32]
    lib.orc_render_ms.restype = i32
    lib.orc_render_ms.argtypes = [C.c_void_p, dp, i32, i32, i32, i32, d, d, d, i32, fp, dp, dp, up, i32]
    lib.orc_sample_image.restype = i32
    lib.orc_sample_image.argtypes = [fp, i32, i32, d, d, dp]
    lib.orc_nearest_pixel.restype = i64
    lib.orc_nearest_pixel.argtypes = [i32, i32, d, d]
    lib.orc_camera_ray_at.restype = i32
    lib.orc_camera_ray_at.argtypes = [dp, i32, i32, d, d, i32, d, d, d, dp, d, dp, dp, dp]
    lib.orc_render.restype = i32
    lib.orc_render.argtypes = [C.c_void_p, dp, i32, i32, i32, i32, d, d, d, lp, i64, dp, dp, ip, up, i32]
    return lib


def lib(path: str | None = None):
    """The loaded oracle library (built on first use)."""
    global _lib
    with _lock:
        if path is not None:
            return _bind(C.CDLL(path))
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
        return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))


class OracleScene:
    """An oracle-side copy of a scene (arrays are copied into the C library)."""

    def __init__(self, tris, spheres, albedo, light_type, light_v, ambient=0.1, libpath=None):
        self._lib = lib(libpath)
        self.tris = np.ascontiguousarray(tris, dtype=np.float32).reshape(-1, 9)
        self.spheres = np.ascontiguousarray(spheres, dtype=np.float32).reshape(-1, 4)
        self.albedo = np.ascontiguousarray(albedo, dtype=np.float32).reshape(-1, 3)
        lv = _vec(light_v)
        self.h = self._lib.orc_scene_new(
            self.tris.ctypes.data_as(C.POINTER(C.c_float)), self.tris.shape[0],
            self.spheres.ctypes.data_as(C.POINTER(C.c_float)), self.spheres.shape[0],
            self.albedo.ctypes.data_as(C.POINTER(C.c_float)), int(light_type), _dp(lv), float(ambient))
        if not self.h:
            raise ValueError("orc_scene_new rejected the scene")

    @classmethod
    def from_scene(cls, sc, libpath=None):
        return cls(sc.tris, sc.spheres, sc.albedo, sc.light.type, sc.light.v, sc.light.ambient, libpath)

    def __del__(self):
        if getattr(self, "h", None):
            self._lib.orc_scene_free(self.h)
            self.h = None

    @property
    def diam(self) -> float:
        return self._lib.orc_scene_diam(self.h)

    # -- single rays
    def trace_closest(self, o, d, tmin, tmax=np.inf):
        t = C.c_double()
        p = C.c_int64()
        f = C.c_int()
        self._lib.orc_trace_closest(self.h, _dp(_vec(o)), _dp(_vec(d)), tmin, tmax, C.byref(t), C.byref(p), C.byref(f))
        return t.value, p.value, f.value

    def trace_any(self, o, d, tmin, tmax, extra=0.0):
        occ = C.c_int()
        f = C.c_int()
        self._lib.orc_trace_any(self.h, _dp(_vec(o)), _dp(_vec(d)), tmin, tmax, extra, C.byref(occ), C.byref(f))
        return occ.value, f.value

    def shade_ray(self, o, d, want_normal=False):
        """(rgbt, prim, flag[, unit normal facing the ray]) of one primary ray."""
        out = np.zeros(4)
        nrm = np.zeros(3)
        p = C.c_int64()
        f = C.c_int()
        self._lib.orc_shade_ray(self.h, _dp(_vec(o)), _dp(_vec(d)), _dp(out), _dp(nrm), C.byref(p), C.byref(f))
        return (out, p.value, f.value, nrm) if want_normal else (out, p.value, f.value)

    # -- passes
    def render_pass(self, cam, W, H, mapping, k, f, in_rgbz=None, pix=None, z0=0.0, nthreads=0, in_normal=None,
                    want_normal=False):
        """One pass; returns (rgbz (n,4) float64, prim (n,) int32, flag (n,) uint8[, normal (n,3)]).
        in_normal: the previous pass's hit normals, (H, W, 3) float64 (normal mapping)."""
        cam = _vec(cam)
        n = W * H if pix is None else len(pix)
        out = np.zeros((n, 4))
        nrm = np.zeros((n, 3))
        prim = np.zeros(n, np.int32)
        flag = np.zeros(n, np.uint8)
        inp = _img_f32(in_rgbz, W, H)
        inn = _normals(in_normal, W, H)
        pp = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
        rc = self._lib.orc_render_pass(
            self.h, _dp(cam), W, H, mapping, k, f, z0, _fp(inp), None if inn is None else _dp(inn),
            None if pp is None else pp.ctypes.data_as(C.POINTER(C.c_int64)), n, _dp(out), _dp(nrm),
            prim.ctypes.data_as(C.POINTER(C.c_int32)), flag.ctypes.data_as(C.POINTER(C.c_uint8)), nthreads)
        if rc != 0:
            raise ValueError("orc_render_pass rejected its arguments")
        return (out, prim, flag, nrm) if want_normal else (out, prim, flag)

    def render_pass_ms(self, cam, W, H, mapping, k, f, jitter, in_rgbz=None, pix=None, z0=0.0, nthreads=0,
                       in_normal=None, want_normal=False):
        """Multi-sample pass; jitter (spp, 2) offsets in [0,1). Returns (rgbz, prim of sample 0, flag[, normal])."""
        cam = _vec(cam)
        jit = np.ascontiguousarray(jitter, dtype=np.float32).reshape(-1)
        n = W * H if pix is None else len(pix)
        out = np.zeros((n, 4))
        nrm = np.zeros((n, 3))
        prim = np.zeros(n, np.int32)
        flag = np.zeros(n, np.uint8)
        inp = _img_f32(in_rgbz, W, H)
        inn = _normals(in_normal, W, H)
        pp = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
        rc = self._lib.orc_render_pass_ms(
            self.h, _dp(cam), W, H, mapping, k, f, z0, jit.size // 2, _fp(jit), _fp(inp),
            None if inn is None else _dp(inn), None if pp is None else pp.ctypes.data_as(C.POINTER(C.c_int64)), n,
            _dp(out), _dp(nrm), prim.ctypes.data_as(C.POINTER(C.c_int32)), flag.ctypes.data_as(C.POINTER(C.c_uint8)),
            nthreads)
        if rc != 0:
            raise ValueError("orc_render_pass_ms rejected its arguments")
        return (out, prim, flag, nrm) if want_normal else (out, prim, flag)

    def render_ms(self, cam, W, H, K, mapping, k, f, jitter, z0=0.0, nthreads=0, want_normal=False):
        """K multi-sample passes over the whole image: (rgbz (W*H, 4), OR of flags[, normal (W*H, 3)])."""
        cam = _vec(cam)
        jit = np.ascontiguousarray(jitter, dtype=np.float32).reshape(-1)
        out = np.zeros((W * H, 4))
        nrm = np.zeros((W * H, 3))
        flag = np.zeros(W * H, np.uint8)
        rc = self._lib.orc_render_ms(self.h, _dp(cam), W, H, K, mapping, k, f, z0, jit.size // 2, _fp(jit), _dp(out),
                                     _dp(nrm), flag.ctypes.data_as(C.POINTER(C.c_uint8)), nthreads)
        if rc != 0:
            raise ValueError("orc_render_ms rejected its arguments")
        return (out, flag, nrm) if want_normal else (out, flag)

    def render(self, cam, W, H, K, mapping, k, f, pix=None, z0=0.0, nthreads=0, want_normal=False):
        """K passes from I_0; returns (rgbz of the last pass, prim of the last pass, OR of flags[, normal])."""
        cam = _vec(cam)
        n = W * H if pix is None else len(pix)
        out = np.zeros((n, 4))
        nrm = np.zeros((n, 3))
        prim = np.zeros(n, np.int32)
        flag = np.zeros(n, np.uint8)
        pp = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
        rc = self._lib.orc_render(
            self.h, _dp(cam), W, H, K, mapping, k, f, z0,
            None if pp is None else pp.ctypes.data_as(C.POINTER(C.c_int64)), n, _dp(out), _dp(nrm),
            prim.ctypes.data_as(C.POINTER(C.c_int32)), flag.ctypes.data_as(C.POINTER(C.c_uint8)), nthreads)
        if rc != 0:
            raise ValueError("orc_render rejected its arguments")
        return (out, prim, flag, nrm) if want_normal else (out, prim, flag)


def _fp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_float))


def _img_f32(img, W, H):
    if img is None:
        return None
    a = np.ascontiguousarray(img, dtype=np.float32).reshape(-1)
    if a.size != W * H * 4:
        raise ValueError("images must be H*W*4 floats")
    return a


def _normals(nrm, W, H):
    if nrm is None:
        return None
    a = np.ascontiguousarray(nrm, dtype=np.float64).reshape(-1)
    if a.size != W * H * 3:
        raise ValueError("normals must be H*W*3 doubles")
    return a


def camera_ray(cam, W, H, x, y, mapping, k, f, c=(0.5, 0.5, 0.5), z=0.0, z0=0.0, n=None, libpath=None):
    """Per-pixel camera of the oracle: returns (origin, unit direction, degenerate).
    n: the previous hit normal (normal mapping), None = no normal."""
    L = lib(libpath)
    o = np.zeros(3)
    d = np.zeros(3)
    rc = L.orc_camera_ray(_dp(_vec(cam)), W, H, x, y, mapping, k, f, z0, _dp(_vec(c)), z,
                          None if n is None else _dp(_vec(n)), _dp(o), _dp(d))
    return o, d, rc


def camera_ray_at(cam, W, H, px, py, mapping, k, f, c=(0.5, 0.5, 0.5), z=0.0, z0=0.0, n=None, libpath=None):
    o = np.zeros(3)
    d = np.zeros(3)
    rc = lib(libpath).orc_camera_ray_at(_dp(_vec(cam)), W, H, float(px), float(py), mapping, k, f, z0, _dp(_vec(c)),
                                        z, None if n is None else _dp(_vec(n)), _dp(o), _dp(d))
    return o, d, rc


def hit_triangle(v0, v1, v2, o, d, tmin=0.0, tmax=np.inf, libpath=None):
    t = C.c_double()
    ok = lib(libpath).orc_hit_triangle(_dp(_vec(v0)), _dp(_vec(v1)), _dp(_vec(v2)), _dp(_vec(o)), _dp(_vec(d)),
                                       tmin, tmax, C.byref(t))
    return (t.value if ok else None)


def hit_sphere(c, r, o, d, tmin=0.0, tmax=np.inf, libpath=None):
    t = C.c_double()
    ok = lib(libpath).orc_hit_sphere(_dp(_vec(c)), r, _dp(_vec(o)), _dp(_vec(d)), tmin, tmax, C.byref(t))
    return (t.value if ok else None)


def mirror_index(i, n, libpath=None):
    return lib(libpath).orc_mirror_index(int(i), int(n))


def imagespace_pass(base, prev, W, H, k_px, pix=None, libpath=None, want_flag=False):
    """One image-space pass: returns (n, 4) float32 (n = W*H or len(pix)), and
    with want_flag the (n,) uint8 rounding-band flags."""
    b = np.ascontiguousarray(base, dtype=np.float32).reshape(-1)
    p = np.ascontiguousarray(prev, dtype=np.float32).reshape(-1)
    if b.size != W * H * 4 or p.size != W * H * 4:
        raise ValueError("base and prev must be H*W*4 floats")
    n = W * H if pix is None else len(pix)
    out = np.zeros((n, 4), np.float32)
    flag = np.zeros(n, np.uint8)
    pp = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
    rc = lib(libpath).orc_imagespace_pass(_fp(b), _fp(p), W, H, float(k_px),
                                          None if pp is None else pp.ctypes.data_as(C.POINTER(C.c_int64)), n,
                                          _fp(out), flag.ctypes.data_as(C.POINTER(C.c_uint8)))
    if rc != 0:
        raise ValueError("orc_imagespace_pass rejected its arguments")
    return (out, flag) if want_flag else out


def rgbz_to_image(rgbz):
    """Oracle pass output (n, 4) float64 -> float32 image rows."""
    return np.asarray(rgbz, dtype=np.float32).copy()


def sample_image(img, W, H, px, py, libpath=None):
    a = np.ascontiguousarray(img, dtype=np.float32).reshape(-1)
    out = np.zeros(4)
    rc = lib(libpath).orc_sample_image(_fp(a), W, H, float(px), float(py), _dp(out))
    if rc != 0:
        raise ValueError("orc_sample_image rejected its arguments")
    return out


def nearest_pixel(W, H, px, py, libpath=None):
    return int(lib(libpath).orc_nearest_pixel(W, H, float(px), float(py)))
