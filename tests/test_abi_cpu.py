"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point include/rcp.h declares. Only calls that fail argument
checks before touching the GPU are made here."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2312_12392_gb300 import build, rcp

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rcp.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rcp_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return rcp.lib()


def test_header_declares_the_abi():
    names = declared()
    for must in ["rcp_scene_create", "rcp_render", "rcp_render_pass", "rcp_render_device",
                 "rcp_render_batch_device", "rcp_server_submit", "rcp_autotune", "rcp_last_error"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    for n in declared():
        assert hasattr(rcp, n), n


def test_version_and_error_strings(lib):
    assert "sm_103a" in rcp.rcp_version()
    assert isinstance(rcp.rcp_last_error(), str)


def test_argument_errors_without_gpu(lib):
    out = C.c_void_p()
    light = rcp.make_light(rcp.RCP_LIGHT_POINT, (0, 1, 0))
    assert lib.rcp_scene_create(None, 5, None, 0, None, C.byref(light), C.byref(out)) == rcp.RCP_ERR_ARG
    assert "NULL" in rcp.rcp_last_error()
    assert lib.rcp_scene_create(None, -1, None, 0, None, C.byref(light), C.byref(out)) == rcp.RCP_ERR_ARG
    bad = rcp.make_light(7, (0, 1, 0))
    t = np.zeros(9, np.float32)
    a = np.zeros(3, np.float32)
    assert lib.rcp_scene_create(t.ctypes.data, 1, None, 0, a.ctypes.data, C.byref(bad),
                                C.byref(out)) == rcp.RCP_ERR_ARG
    cam = rcp.make_camera((0, 0, 1), (0, 0, 0))
    p = rcp.make_params()
    assert lib.rcp_render(None, C.byref(cam), 4, 4, 1, C.byref(p), None) == rcp.RCP_ERR_ARG
    assert lib.rcp_server_create(0, 4, C.byref(out)) == rcp.RCP_ERR_ARG
    assert lib.rcp_set_tuning(None, None) == rcp.RCP_ERR_ARG
    assert lib.rcp_set_host_output(7) == rcp.RCP_ERR_ARG
    assert rcp.rcp_get_host_output() == rcp.RCP_HOST_OUTPUT_AUTO


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(rcp, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(rcp, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        rcp.lib()


def test_render_h2d_bytes(lib):
    """The per-call host-to-device bytes of rcp_render (view descriptors): K
    descriptors per view, and -1 outside the valid ranges. Host logic only."""
    one = rcp.rcp_render_h2d_bytes(1, 1)
    assert one > 0 and one % 8 == 0
    assert rcp.rcp_render_h2d_bytes(1, 6) == 6 * one
    assert rcp.rcp_render_h2d_bytes(64, 6) == 64 * 6 * one
    assert rcp.rcp_render_h2d_bytes(0, 6) == -1
    assert rcp.rcp_render_h2d_bytes(1, 0) == -1
    assert rcp.rcp_render_h2d_bytes(1, 17) == -1


def test_static_sort_capacity_matches_header(lib):
    """The allocation-free sort's capacity as built equals the header's
    RCP_SORT_STATIC_MAX_PAIRS, so neither the binding nor the error message can
    go stale (a constant returned without touching the GPU)."""
    m = re.search(r"#define\s+RCP_SORT_STATIC_MAX_PAIRS\s+(\d+)", open(HEADER).read())
    assert m and rcp.rcp_sort_static_capacity() == int(m.group(1))
    assert lib.rcp_sort_pairs_static(None, None, -1, 30, None) == rcp.RCP_ERR_ARG
