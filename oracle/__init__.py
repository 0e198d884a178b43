"""FP64 brute-force CPU oracle for Recursive Camera Painting (arXiv 2312.12392).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this package to check and time the CUDA path;
the CUDA library and its Python binding never import it. It shares no code with
the CUDA path: ``rcp_oracle.c`` is plain C, compiled here with gcc.

Images exchanged with the oracle are (H, W, 4) float32 arrays: RGB in [0, 1]
and the hit distance (0 on a miss) in the fourth lane.
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
TOL = 1e-5


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
    lib.orc_camera_ray.argtypes = [dp, i32, i32, i32, i32, i32, d, d, d, dp, d, dp, dp]
    lib.orc_hit_triangle.argtypes = [dp, dp, dp, dp, dp, d, d, dp]
    lib.orc_hit_sphere.argtypes = [dp, d, dp, dp, d, d, dp]
    lib.orc_trace_closest.argtypes = [C.c_void_p, dp, dp, d, d, dp, lp, C.POINTER(C.c_int)]
    lib.orc_trace_any.argtypes = [C.c_void_p, dp, dp, d, d, d, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    lib.orc_shade_ray.argtypes = [C.c_void_p, dp, dp, dp, lp, C.POINTER(C.c_int)]
    lib.orc_render_pass.restype = i32
    lib.orc_render_pass.argtypes = [C.c_void_p, dp, i32, i32, i32, d, d, d, fp, lp, i64, dp, ip, up, i32]
    lib.orc_imagespace_pass.restype = i32
    lib.orc_imagespace_pass.argtypes = [fp, fp, i32, i32, C.c_float, lp, i64, fp]
    lib.orc_mirror_index.restype = i64
    lib.orc_mirror_index.argtypes = [i64, i64]
    lib.orc_normal_encode.restype = C.c_uint32
    lib.orc_normal_encode.argtypes = [dp]
    lib.orc_normal_decode.restype = i32
    lib.orc_normal_decode.argtypes = [C.c_uint32, dp]
    lib.orc_render_pass_ms.restype = i32
    lib.orc_render_pass_ms.argtypes = [C.c_void_p, dp, i32, i32, i32, d, d, d, i32, fp, fp, lp, i64, dp, ip, up, i32]
    lib.orc_render_ms.restype = i32
    lib.orc_render_ms.argtypes = [C.c_void_p, dp, i32, i32, i32, i32, d, d, d, i32, fp, dp, up, i32]
    lib.orc_sample_image.restype = i32
    lib.orc_sample_image.argtypes = [fp, i32, i32, d, d, i32, dp]
    lib.orc_camera_ray_at.restype = i32
    lib.orc_camera_ray_at.argtypes = [dp, i32, i32, d, d, i32, d, d, d, dp, d, dp, dp]
    lib.orc_render.restype = i32
    lib.orc_render.argtypes = [C.c_void_p, dp, i32, i32, i32, i32, d, d, d, lp, i64, dp, ip, up, i32]
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

    def shade_ray(self, o, d):
        out = np.zeros(4)
        p = C.c_int64()
        f = C.c_int()
        self._lib.orc_shade_ray(self.h, _dp(_vec(o)), _dp(_vec(d)), _dp(out), C.byref(p), C.byref(f))
        return out, p.value, f.value

    # -- passes
    def render_pass(self, cam, W, H, mapping, k, f, in_rgbz=None, pix=None, z0=0.0, nthreads=0):
        """One pass; returns (rgbz (n,4) float64, prim (n,) int32, flag (n,) uint8)."""
        cam = _vec(cam)
        n = W * H if pix is None else len(pix)
        out = np.zeros((n, 4))
        prim = np.zeros(n, np.int32)
        flag = np.zeros(n, np.uint8)
        inp = None
        if in_rgbz is not None:
            inp = np.ascontiguousarray(in_rgbz, dtype=np.float32).reshape(H * W * 4)
        pp = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
        rc = self._lib.orc_render_pass(
            self.h, _dp(cam), W, H, mapping, k, f, z0,
            None if inp is None else inp.ctypes.data_as(C.POINTER(C.c_float)),
            None if pp is None else pp.ctypes.data_as(C.POINTER(C.c_int64)), n, _dp(out),
            prim.ctypes.data_as(C.POINTER(C.c_int32)), flag.ctypes.data_as(C.POINTER(C.c_uint8)), nthreads)
        if rc != 0:
            raise ValueError("orc_render_pass rejected its arguments")
        return out, prim, flag

    def render_pass_ms(self, cam, W, H, mapping, k, f, jitter, in_rgbz=None, pix=None, z0=0.0, nthreads=0):
        """Multi-sample pass; jitter (spp, 2) offsets in [0,1). Returns (rgbz, prim of sample 0, flag)."""
        cam = _vec(cam)
        jit = np.ascontiguousarray(jitter, dtype=np.float32).reshape(-1)
        n = W * H if pix is None else len(pix)
        out = np.zeros((n, 4))
        prim = np.zeros(n, np.int32)
        flag = np.zeros(n, np.uint8)
        inp = None if in_rgbz is None else np.ascontiguousarray(in_rgbz, dtype=np.float32).reshape(-1)
        pp = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
        fptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
        rc = self._lib.orc_render_pass_ms(
            self.h, _dp(cam), W, H, mapping, k, f, z0, jit.size // 2, fptr(jit), None if inp is None else fptr(inp),
            None if pp is None else pp.ctypes.data_as(C.POINTER(C.c_int64)), n, _dp(out),
            prim.ctypes.data_as(C.POINTER(C.c_int32)), flag.ctypes.data_as(C.POINTER(C.c_uint8)), nthreads)
        if rc != 0:
            raise ValueError("orc_render_pass_ms rejected its arguments")
        return out, prim, flag

    def render_ms(self, cam, W, H, K, mapping, k, f, jitter, z0=0.0, nthreads=0):
        """K multi-sample passes over the whole image: (rgbz (W*H, 4), OR of flags)."""
        cam = _vec(cam)
        jit = np.ascontiguousarray(jitter, dtype=np.float32).reshape(-1)
        out = np.zeros((W * H, 4))
        flag = np.zeros(W * H, np.uint8)
        rc = self._lib.orc_render_ms(self.h, _dp(cam), W, H, K, mapping, k, f, z0, jit.size // 2,
                                     jit.ctypes.data_as(C.POINTER(C.c_float)), _dp(out),
                                     flag.ctypes.data_as(C.POINTER(C.c_uint8)), nthreads)
        if rc != 0:
            raise ValueError("orc_render_ms rejected its arguments")
        return out, flag

    def render(self, cam, W, H, K, mapping, k, f, pix=None, z0=0.0, nthreads=0):
        """K passes from I_0; returns (rgbz of the last pass, prim of the last pass, OR of flags)."""
        cam = _vec(cam)
        n = W * H if pix is None else len(pix)
        out = np.zeros((n, 4))
        prim = np.zeros(n, np.int32)
        flag = np.zeros(n, np.uint8)
        pp = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
        rc = self._lib.orc_render(
            self.h, _dp(cam), W, H, K, mapping, k, f, z0,
            None if pp is None else pp.ctypes.data_as(C.POINTER(C.c_int64)), n, _dp(out),
            prim.ctypes.data_as(C.POINTER(C.c_int32)), flag.ctypes.data_as(C.POINTER(C.c_uint8)), nthreads)
        if rc != 0:
            raise ValueError("orc_render rejected its arguments")
        return out, prim, flag


def camera_ray(cam, W, H, x, y, mapping, k, f, c=(0.5, 0.5, 0.5), z=0.0, z0=0.0, libpath=None):
    """Per-pixel camera of the oracle: returns (origin, unit direction, degenerate)."""
    L = lib(libpath)
    o = np.zeros(3)
    d = np.zeros(3)
    rc = L.orc_camera_ray(_dp(_vec(cam)), W, H, x, y, mapping, k, f, z0, _dp(_vec(c)), z, _dp(o), _dp(d))
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


def imagespace_pass(base, prev, W, H, k_px, pix=None, libpath=None):
    """One image-space pass: returns (n, 4) float32 (n = W*H or len(pix))."""
    b = np.ascontiguousarray(base, dtype=np.float32).reshape(-1)
    p = np.ascontiguousarray(prev, dtype=np.float32).reshape(-1)
    if b.size != W * H * 4 or p.size != W * H * 4:
        raise ValueError("base and prev must be H*W*4 floats")
    n = W * H if pix is None else len(pix)
    out = np.zeros((n, 4), np.float32)
    pp = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
    fptr = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
    rc = lib(libpath).orc_imagespace_pass(fptr(b), fptr(p), W, H, float(np.float32(k_px)),
                                          None if pp is None else pp.ctypes.data_as(C.POINTER(C.c_int64)), n,
                                          fptr(out))
    if rc != 0:
        raise ValueError("orc_imagespace_pass rejected its arguments")
    return out


def normal_encode(n, libpath=None):
    return int(lib(libpath).orc_normal_encode(_dp(_vec(n))))


def normal_decode(code, libpath=None):
    out = np.zeros(3)
    ok = lib(libpath).orc_normal_decode(int(code) & 0xffffffff, _dp(out))
    return out, bool(ok)


def rgbz_to_image(rgbz, mapping):
    """Oracle pass output (n, 4) float64 -> float32 image rows; for the normal
    mapping the fourth lane's value is the 32-bit normal code, stored as bits."""
    out = np.asarray(rgbz, dtype=np.float32).copy()
    if mapping == MAP_NORMAL:
        out[:, 3] = np.asarray(rgbz[:, 3], dtype=np.uint64).astype(np.uint32).view(np.float32)
    return out


def sample_image(img, W, H, px, py, mapping=MAP_EYE, libpath=None):
    a = np.ascontiguousarray(img, dtype=np.float32).reshape(-1)
    out = np.zeros(4)
    rc = lib(libpath).orc_sample_image(a.ctypes.data_as(C.POINTER(C.c_float)), W, H, float(px), float(py), mapping,
                                       _dp(out))
    if rc != 0:
        raise ValueError("orc_sample_image rejected its arguments")
    return out


def camera_ray_at(cam, W, H, px, py, mapping, k, f, c=(0.5, 0.5, 0.5), z=0.0, z0=0.0, libpath=None):
    o = np.zeros(3)
    d = np.zeros(3)
    rc = lib(libpath).orc_camera_ray_at(_dp(_vec(cam)), W, H, float(px), float(py), mapping, k, f, z0, _dp(_vec(c)),
                                        z, _dp(o), _dp(d))
    return o, d, rc
