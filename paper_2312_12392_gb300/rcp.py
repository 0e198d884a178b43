"""Python binding of the C ABI in include/rcp.h (ctypes; argument marshalling only).

Every function has the C name and forwards to librcp.so; all rendering work
runs in the library's CUDA kernels. Host arrays are numpy arrays; device
buffers may be torch CUDA tensors or integer device pointers; streams may be a
torch.cuda.Stream, an integer cudaStream_t or None (legacy default stream).
A failed call raises RcpError carrying the status and rcp_last_error().

If librcp.so has not been built this module raises on first use: there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "librcp.so")

RCP_OK, RCP_ERR_ARG, RCP_ERR_OOM, RCP_ERR_CUDA, RCP_ERR_STACK, RCP_ERR_TIMEOUT, RCP_ERR_STATE = 0, -1, -2, -3, -4, -5, -6
RCP_LIGHT_POINT, RCP_LIGHT_DIRECTIONAL = 0, 1
RCP_MAP_EYE, RCP_MAP_TARGET, RCP_MAP_DEPTH, RCP_MAP_IMAGE, RCP_MAP_NORMAL = 0, 1, 2, 3, 4
RCP_COLLAPSE_AREA, RCP_COLLAPSE_SAH = 0, 1
RCP_HOST_OUTPUT_AUTO, RCP_HOST_OUTPUT_DIRECT, RCP_HOST_OUTPUT_COPY = 0, 1, 2
RCP_SPLIT_MAX = 8


class RcpError(RuntimeError):
    def __init__(self, status, func, msg):
        super().__init__(f"{func} failed with status {status}: {msg}")
        self.status = status


class rcp_light(C.Structure):
    _fields_ = [("type", C.c_int32), ("v", C.c_float * 3), ("ambient", C.c_float)]


class rcp_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look_at", C.c_float * 3), ("up", C.c_float * 3), ("fov_y_deg", C.c_float)]


RCP_MAX_SPP = 16


class rcp_params(C.Structure):
    _fields_ = [("mapping", C.c_int32), ("k", C.c_float), ("focal_dist", C.c_float), ("z0", C.c_float),
                ("spp", C.c_int32), ("jitter", C.c_float * (2 * RCP_MAX_SPP))]


class rcp_scene_info(C.Structure):
    _fields_ = [("n_tris", C.c_int64), ("n_spheres", C.c_int64), ("n_nodes", C.c_int64), ("depth", C.c_int32),
                ("max_leaf", C.c_int32), ("device_bytes", C.c_int64), ("diam", C.c_float), ("build_ms", C.c_float),
                ("collapse", C.c_int32), ("split_max", C.c_int32), ("n_records", C.c_int64)]


class rcp_build_options(C.Structure):
    _fields_ = [("collapse", C.c_int32), ("split_max", C.c_int32)]


class rcp_tuning(C.Structure):
    _fields_ = [("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("chunk", C.c_int32),
                ("fused_camera", C.c_int32), ("stack_entries", C.c_int32), ("hints", C.c_int32),
                ("chain_passes", C.c_int32)]


class rcp_counters(C.Structure):
    _fields_ = [("rays", C.c_int64), ("primary_rays", C.c_int64), ("shadow_rays", C.c_int64), ("nodes", C.c_int64),
                ("box_tests", C.c_int64), ("tri_tests", C.c_int64), ("sphere_tests", C.c_int64)]


class rcp_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("rejected", C.c_int64),
                ("in_flight", C.c_int64), ("queued", C.c_int64), ("steps", C.c_int64), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("frames_per_s", C.c_double), ("mrays_per_s", C.c_double),
                ("device_bytes_in_use", C.c_int64), ("device_bytes_peak", C.c_int64), ("device_busy_ms", C.c_double)]


_lock = threading.Lock()
_lib = None

_vp = C.c_void_p
_SIGS = {
    "rcp_scene_create": [_vp, C.c_int64, _vp, C.c_int64, _vp, C.POINTER(rcp_light), C.POINTER(_vp)],
    "rcp_scene_create_ex": [_vp, C.c_int64, _vp, C.c_int64, _vp, C.POINTER(rcp_light), C.POINTER(rcp_build_options),
                            C.POINTER(_vp)],
    "rcp_scene_update_vertices": [_vp, _vp],
    "rcp_scene_update_vertices_device": [_vp, _vp, _vp],
    "rcp_scene_get_info": [_vp, C.POINTER(rcp_scene_info)],
    "rcp_scene_validate": [_vp],
    "rcp_scene_destroy": [_vp],
    "rcp_render": [_vp, C.POINTER(rcp_camera), C.c_int, C.c_int, C.c_int, C.POINTER(rcp_params), _vp],
    "rcp_render_pass": [_vp, C.POINTER(rcp_camera), C.c_int, C.c_int, C.POINTER(rcp_params), _vp, _vp, _vp],
    "rcp_render_device": [_vp, C.POINTER(rcp_camera), C.c_int, C.c_int, C.c_int, C.POINTER(rcp_params), _vp, _vp,
                          _vp, _vp],
    "rcp_render_batch_device": [_vp, C.c_int, C.POINTER(rcp_camera), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.c_int, C.POINTER(rcp_params), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), _vp],
    "rcp_get_tuning": [_vp, C.POINTER(rcp_tuning)],
    "rcp_set_tuning": [_vp, C.POINTER(rcp_tuning)],
    "rcp_autotune": [_vp, C.POINTER(rcp_camera), C.c_int, C.c_int, C.POINTER(rcp_params), C.c_char_p,
                     C.POINTER(rcp_tuning)],
    "rcp_last_ray_counts": [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "rcp_count_pass": [_vp, C.POINTER(rcp_camera), C.c_int, C.c_int, C.POINTER(rcp_params), _vp, _vp,
                       C.POINTER(rcp_counters)],
    "rcp_last_pass_times": [_vp, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)],
    "rcp_render_h2d_bytes": [C.c_int, C.c_int],
    "rcp_debug_trace": [_vp, C.c_int64, _vp, _vp, C.c_int, C.c_int, _vp, _vp, C.c_int, _vp],
    "rcp_debug_sort_pairs": [_vp, _vp, C.c_int64, C.c_int, _vp],
    "rcp_debug_morton": [_vp, C.c_int64, _vp, _vp, _vp, _vp],
    "rcp_debug_sort_lookback_timeout": [C.c_int64, _vp],
    "rcp_imagespace_pass_device": [_vp, _vp, _vp, C.c_int, C.c_int, C.c_float, _vp],
    "rcp_sort_pairs_static": [_vp, _vp, C.c_int64, C.c_int, _vp],
    "rcp_sort_static_capacity": [],
    "rcp_server_create": [C.c_int64, C.c_int, C.POINTER(_vp)],
    "rcp_server_submit": [_vp, _vp, C.POINTER(rcp_camera), C.c_int, C.c_int, C.c_int, C.POINTER(rcp_params), _vp,
                          C.POINTER(C.c_int64)],
    "rcp_server_poll": [_vp, C.c_int64, C.POINTER(C.c_int)],
    "rcp_server_set_step_pixels": [_vp, C.c_int64],
    "rcp_server_set_max_chain": [_vp, C.c_int],
    "rcp_server_wait": [_vp, C.c_int64, C.c_double],
    "rcp_server_latency": [_vp, C.c_int64, C.POINTER(C.c_double)],
    "rcp_server_stats_get": [_vp, C.POINTER(rcp_server_stats)],
    "rcp_server_destroy": [_vp],
    "rcp_last_error": [],
    "rcp_version": [],
    "rcp_set_host_output": [C.c_int],
    "rcp_get_host_output": [],
}


def lib():
    """Load librcp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2312_12392_gb300.build` (no CPU fallback exists)")
            L = C.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = C.c_int
            L.rcp_last_error.restype = C.c_char_p
            L.rcp_version.restype = C.c_char_p
            L.rcp_render_h2d_bytes.restype = C.c_int64
            L.rcp_sort_static_capacity.restype = C.c_int64
            L.rcp_scene_destroy.restype = None
            L.rcp_server_destroy.restype = None
            _lib = L
        return _lib


def _check(status, func):
    if status != RCP_OK:
        raise RcpError(status, func, lib().rcp_last_error().decode())
    return status


def _ptr(x):
    """Pointer of a numpy array, torch tensor or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _host(a, dtype, n=None):
    a = np.ascontiguousarray(a, dtype=dtype)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} elements, got {a.size}")
    return a


def make_camera(eye, look_at, up=(0.0, 1.0, 0.0), fov_y_deg=60.0) -> rcp_camera:
    return rcp_camera((C.c_float * 3)(*eye), (C.c_float * 3)(*look_at), (C.c_float * 3)(*up), float(fov_y_deg))


def make_params(mapping=RCP_MAP_EYE, k=0.0, focal_dist=1.0, z0=0.0, jitter=None) -> rcp_params:
    """jitter: None (one sample at the pixel centre) or (spp, 2) offsets in [0,1)."""
    p = rcp_params(int(mapping), float(k), float(focal_dist), float(z0), 0)
    if jitter is not None:
        j = np.asarray(jitter, dtype=np.float32).reshape(-1, 2)
        if not 1 <= len(j) <= RCP_MAX_SPP:
            raise ValueError("1..16 samples per pixel")
        p.spp = len(j)
        for i, v in enumerate(j.reshape(-1)):
            p.jitter[i] = float(v)
    return p


def make_light(type_, v, ambient=0.1) -> rcp_light:
    return rcp_light(int(type_), (C.c_float * 3)(*v), float(ambient))


# ------------------------------------------------------------------ scenes

def rcp_scene_create(tri_xyz, spheres, albedo, light: rcp_light):
    tri = _host(tri_xyz, np.float32).reshape(-1)
    sph = _host(spheres if spheres is not None else np.zeros(0), np.float32).reshape(-1)
    alb = _host(albedo, np.float32).reshape(-1)
    T, S = tri.size // 9, sph.size // 4
    if tri.size != 9 * T or sph.size != 4 * S or alb.size != 3 * (T + S):
        raise ValueError("tri_xyz must be T*9, spheres S*4 and albedo (T+S)*3 floats")
    out = C.c_void_p()
    _check(lib().rcp_scene_create(_ptr(tri) if T else None, T, _ptr(sph) if S else None, S,
                                  _ptr(alb) if T + S else None, C.byref(light), C.byref(out)), "rcp_scene_create")
    return out.value


def rcp_scene_create_ex(tri_xyz, spheres, albedo, light: rcp_light, collapse=RCP_COLLAPSE_AREA, split_max=0):
    tri = _host(tri_xyz, np.float32).reshape(-1)
    sph = _host(spheres if spheres is not None else np.zeros(0), np.float32).reshape(-1)
    alb = _host(albedo, np.float32).reshape(-1)
    T, S = tri.size // 9, sph.size // 4
    if tri.size != 9 * T or sph.size != 4 * S or alb.size != 3 * (T + S):
        raise ValueError("tri_xyz must be T*9, spheres S*4 and albedo (T+S)*3 floats")
    opt = rcp_build_options(int(collapse), int(split_max))
    out = C.c_void_p()
    _check(lib().rcp_scene_create_ex(_ptr(tri) if T else None, T, _ptr(sph) if S else None, S,
                                     _ptr(alb) if T + S else None, C.byref(light), C.byref(opt), C.byref(out)),
           "rcp_scene_create_ex")
    return out.value


def rcp_scene_update_vertices(scene, tri_xyz):
    tri = _host(tri_xyz, np.float32).reshape(-1)
    _check(lib().rcp_scene_update_vertices(scene, _ptr(tri)), "rcp_scene_update_vertices")


def rcp_scene_update_vertices_device(scene, d_tri_xyz, stream=None):
    _check(lib().rcp_scene_update_vertices_device(scene, _ptr(d_tri_xyz), _stream(stream)),
           "rcp_scene_update_vertices_device")


def rcp_scene_get_info(scene) -> rcp_scene_info:
    info = rcp_scene_info()
    _check(lib().rcp_scene_get_info(scene, C.byref(info)), "rcp_scene_get_info")
    return info


def rcp_scene_validate(scene):
    _check(lib().rcp_scene_validate(scene), "rcp_scene_validate")


def rcp_scene_destroy(scene):
    if scene:
        lib().rcp_scene_destroy(scene)


# ------------------------------------------------------------------ renders

def rcp_render(scene, cam: rcp_camera, width, height, K, params: rcp_params, out_rgb=None):
    if out_rgb is None:
        out_rgb = np.empty((height, width, 3), np.float32)
    if out_rgb.dtype != np.float32 or out_rgb.size != width * height * 3 or not out_rgb.flags["C_CONTIGUOUS"]:
        raise ValueError("out_rgb must be a contiguous float32 array of height*width*3")
    _check(lib().rcp_render(scene, C.byref(cam), width, height, K, C.byref(params), _ptr(out_rgb)), "rcp_render")
    return out_rgb


def rcp_render_pass(scene, cam: rcp_camera, width, height, params: rcp_params, in_rgbz=None, out_rgbz=None,
                    out_prim=None):
    if in_rgbz is not None:
        in_rgbz = _host(in_rgbz, np.float32, width * height * 4)
    if out_rgbz is None:
        out_rgbz = np.empty((height, width, 4), np.float32)
    _check(lib().rcp_render_pass(scene, C.byref(cam), width, height, C.byref(params), _ptr(in_rgbz),
                                 _ptr(out_rgbz), _ptr(out_prim)), "rcp_render_pass")
    return out_rgbz


def rcp_render_device(scene, cam: rcp_camera, width, height, K, params: rcp_params, d_in, d_out, d_prim=None,
                      stream=None):
    _check(lib().rcp_render_device(scene, C.byref(cam), width, height, K, C.byref(params), _ptr(d_in), _ptr(d_out),
                                   _ptr(d_prim), _stream(stream)), "rcp_render_device")


def rcp_render_batch_device(scene, cams, widths, heights, K, params: rcp_params, d_outs, stream=None, d_ins=None,
                            d_prims=None):
    """d_ins / d_prims: None, or one entry per view (a device buffer or None)."""
    n = len(cams)
    ca = (rcp_camera * n)(*cams)
    wa = (C.c_int * n)(*[int(w) for w in widths])
    ha = (C.c_int * n)(*[int(h) for h in heights])
    oa = (C.c_void_p * n)(*[_ptr(o) for o in d_outs])
    ia = None if d_ins is None else (C.c_void_p * n)(*[_ptr(x) for x in d_ins])
    pa = None if d_prims is None else (C.c_void_p * n)(*[_ptr(x) for x in d_prims])
    _check(lib().rcp_render_batch_device(scene, n, ca, wa, ha, K, C.byref(params), ia, oa, pa, _stream(stream)),
           "rcp_render_batch_device")


def rcp_imagespace_pass_device(d_base, d_prev, d_out, width, height, k_px, stream=None):
    _check(lib().rcp_imagespace_pass_device(_ptr(d_base), _ptr(d_prev), _ptr(d_out), width, height, float(k_px),
                                            _stream(stream)), "rcp_imagespace_pass_device")


def rcp_get_tuning(scene) -> rcp_tuning:
    t = rcp_tuning()
    _check(lib().rcp_get_tuning(scene, C.byref(t)), "rcp_get_tuning")
    return t


def rcp_set_tuning(scene, t: rcp_tuning):
    _check(lib().rcp_set_tuning(scene, C.byref(t)), "rcp_set_tuning")


def rcp_autotune(scene, cam: rcp_camera, width, height, params: rcp_params, cache_path=None) -> rcp_tuning:
    t = rcp_tuning()
    _check(lib().rcp_autotune(scene, C.byref(cam), width, height, C.byref(params),
                              cache_path.encode() if cache_path else None, C.byref(t)), "rcp_autotune")
    return t


def rcp_last_ray_counts(scene):
    p, s = C.c_int64(), C.c_int64()
    _check(lib().rcp_last_ray_counts(scene, C.byref(p), C.byref(s)), "rcp_last_ray_counts")
    return p.value, s.value


def rcp_count_pass(scene, cam: rcp_camera, width, height, params: rcp_params, d_in=None,
                   d_out=None) -> rcp_counters:
    c = rcp_counters()
    _check(lib().rcp_count_pass(scene, C.byref(cam), width, height, C.byref(params), _ptr(d_in), _ptr(d_out),
                                C.byref(c)), "rcp_count_pass")
    return c


def rcp_render_h2d_bytes(n_views, K):
    """Bytes one rcp_render call copies host to device (view descriptors)."""
    return int(lib().rcp_render_h2d_bytes(int(n_views), int(K)))


def rcp_last_pass_times(scene, max_passes=16):
    ms = (C.c_float * max_passes)()
    n = C.c_int()
    _check(lib().rcp_last_pass_times(scene, ms, max_passes, C.byref(n)), "rcp_last_pass_times")
    return list(ms)[: n.value]


def rcp_debug_trace(scene, n, orig_tmin, dir_tmax, any_hit, brute, t_out, prim_out, stream=None, stack_entries=0):
    _check(lib().rcp_debug_trace(scene, n, _ptr(orig_tmin), _ptr(dir_tmax), int(any_hit), int(brute), _ptr(t_out),
                                 _ptr(prim_out), int(stack_entries), _stream(stream)), "rcp_debug_trace")


def rcp_debug_sort_pairs(keys, values, n, bits, stream=None):
    _check(lib().rcp_debug_sort_pairs(_ptr(keys), _ptr(values), n, bits, _stream(stream)), "rcp_debug_sort_pairs")


def rcp_debug_morton(xyz, n, lo, hi, codes, stream=None):
    lo = _host(lo, np.float32, 3)
    hi = _host(hi, np.float32, 3)
    _check(lib().rcp_debug_morton(_ptr(xyz), n, _ptr(lo), _ptr(hi), _ptr(codes), _stream(stream)),
           "rcp_debug_morton")


def rcp_debug_sort_lookback_timeout(spin_limit, stream=None):
    _check(lib().rcp_debug_sort_lookback_timeout(int(spin_limit), _stream(stream)), "rcp_debug_sort_lookback_timeout")


def rcp_sort_static_capacity() -> int:
    """The largest n rcp_sort_pairs_static accepts, as the library was built."""
    return int(lib().rcp_sort_static_capacity())


def rcp_sort_pairs_static(keys, values, n, bits, stream=None):
    """Allocation-free radix sort (device arrays, n <= rcp_sort_static_capacity())."""
    _check(lib().rcp_sort_pairs_static(_ptr(keys), _ptr(values), n, bits, _stream(stream)), "rcp_sort_pairs_static")


# ------------------------------------------------------------------ serving

def rcp_server_create(mem_budget_bytes, max_slots):
    out = C.c_void_p()
    _check(lib().rcp_server_create(int(mem_budget_bytes), int(max_slots), C.byref(out)), "rcp_server_create")
    return out.value


def rcp_server_submit(srv, scene, cam: rcp_camera, width, height, K, params: rcp_params, out_rgb):
    if out_rgb.dtype != np.float32 or out_rgb.size != width * height * 3 or not out_rgb.flags["C_CONTIGUOUS"]:
        raise ValueError("out_rgb must be a contiguous float32 array of height*width*3")
    t = C.c_int64()
    _check(lib().rcp_server_submit(srv, scene, C.byref(cam), width, height, K, C.byref(params), _ptr(out_rgb),
                                   C.byref(t)), "rcp_server_submit")
    return t.value


def rcp_server_set_step_pixels(srv, pixels):
    _check(lib().rcp_server_set_step_pixels(srv, int(pixels)), "rcp_server_set_step_pixels")


def rcp_server_set_max_chain(srv, passes):
    _check(lib().rcp_server_set_max_chain(srv, int(passes)), "rcp_server_set_max_chain")


def rcp_server_poll(srv, ticket):
    d = C.c_int()
    _check(lib().rcp_server_poll(srv, ticket, C.byref(d)), "rcp_server_poll")
    return bool(d.value)


def rcp_server_wait(srv, ticket, timeout_s=60.0):
    _check(lib().rcp_server_wait(srv, ticket, float(timeout_s)), "rcp_server_wait")


def rcp_server_latency(srv, ticket) -> float:
    """Submit-to-done latency (ms) of a finished request."""
    ms = C.c_double()
    _check(lib().rcp_server_latency(srv, ticket, C.byref(ms)), "rcp_server_latency")
    return ms.value


def rcp_server_stats_get(srv) -> rcp_server_stats:
    s = rcp_server_stats()
    _check(lib().rcp_server_stats_get(srv, C.byref(s)), "rcp_server_stats_get")
    return s


def rcp_server_destroy(srv):
    if srv:
        lib().rcp_server_destroy(srv)


def rcp_set_host_output(mode):
    _check(lib().rcp_set_host_output(int(mode)), "rcp_set_host_output")


def rcp_get_host_output() -> int:
    return int(lib().rcp_get_host_output())


def rcp_last_error() -> str:
    return lib().rcp_last_error().decode()


def rcp_version() -> str:
    return lib().rcp_version().decode()


# ------------------------------------------------------------------ helpers

def scene_from(sc, collapse=None, split_max=0):
    """Create a library scene from a scenes.Scene (collapse: an RCP_COLLAPSE_*
    build policy, None = the library default; split_max: references per
    triangle at most, 0 or 1 = no splitting)."""
    light = make_light(sc.light.type, sc.light.v, sc.light.ambient)
    if collapse is None and split_max <= 1:
        return rcp_scene_create(sc.tris, sc.spheres, sc.albedo, light)
    return rcp_scene_create_ex(sc.tris, sc.spheres, sc.albedo, light,
                               RCP_COLLAPSE_AREA if collapse is None else collapse, split_max)


def camera_from(cam):
    """rcp_camera from a scenes.Camera."""
    return make_camera(cam.eye, cam.look_at, cam.up, cam.fov_y_deg)
