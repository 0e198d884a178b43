"""Failure paths reached without faulting the GPU: every wait in the kernels is
bounded and every overflow is reported as a status the host reads.

  * the radix sort's look-back wait: a pass whose earlier tile never publishes
    its counts gives up after a short poll limit and the call returns
    RCP_ERR_TIMEOUT; the device stays usable;
  * the traversal stack: a walk given fewer stack entries than the tree needs
    drops the deeper groups, ends, and the call returns RCP_ERR_STACK.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp, scenes  # noqa: E402
import gpu_util as U  # noqa: E402

pytestmark = pytest.mark.gpu


def test_lookback_wait_times_out_and_device_stays_usable():
    for limit in (1, 1000):
        with pytest.raises(rcp.RcpError) as e:
            rcp.rcp_debug_sort_lookback_timeout(limit)
        assert e.value.status == rcp.RCP_ERR_TIMEOUT and "ran out" in str(e.value)
    # a real sort right after it
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 1 << 30, size=50_000, dtype=np.uint64).astype(np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32)
    dk = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    dv = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    rcp.rcp_debug_sort_pairs(dk, dv, keys.size, 30)
    torch.cuda.synchronize()
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(dk.cpu().numpy().view(np.uint32), keys[order])
    with pytest.raises(rcp.RcpError) as e:
        rcp.rcp_debug_sort_lookback_timeout(0)
    assert e.value.status == rcp.RCP_ERR_ARG


def test_stack_overflow_is_reported():
    sc = scenes.mid_scene()
    g = U.gpu_scene(sc)
    try:
        depth = rcp.rcp_scene_get_info(g).depth
        assert depth >= 4
        n = 4096
        ot, dt = U.random_rays(n, seed=3, extent=sc.diameter() / 4, towards=(0, 0, 0))
        o, d = torch.from_numpy(ot).cuda(), torch.from_numpy(dt).cuda()
        t = torch.empty(n, dtype=torch.float32, device="cuda")
        p = torch.empty(n, dtype=torch.int32, device="cuda")
        with pytest.raises(rcp.RcpError) as e:
            rcp.rcp_debug_trace(g, n, o, d, 0, 0, t, p, stack_entries=1)
        assert e.value.status == rcp.RCP_ERR_STACK
        # enough entries: no error, and the walk equals brute force
        rcp.rcp_debug_trace(g, n, o, d, 0, 0, t, p, stack_entries=depth)
        tb = torch.empty_like(t)
        pb = torch.empty_like(p)
        rcp.rcp_debug_trace(g, n, o, d, 0, 1, tb, pb)
        torch.cuda.synchronize()
        assert torch.equal(p, pb) and torch.equal(t, tb)
        # renders after the overflow are unaffected
        cam = rcp.camera_from(sc.poses[0])
        prm = rcp.make_params(rcp.RCP_MAP_EYE, 0.02 * sc.diameter(), 0.1 * sc.diameter())
        a = rcp.rcp_render(g, cam, 64, 48, 2, prm)
        assert np.isfinite(a).all()
        with pytest.raises(rcp.RcpError):
            rcp.rcp_debug_trace(g, n, o, d, 0, 0, t, p, stack_entries=65)
    finally:
        rcp.rcp_scene_destroy(g)
