"""The allocation-free sort entry point against the allocating one.

rcp_sort_pairs_static serves callers that cannot allocate device memory when
they sort: real-time loops that must not allocate once they are running, and
hosts that own all device memory and give the library no allocator. Its
scratch is a fixed array compiled into the library. It must give exactly what
rcp_debug_sort_pairs gives (integer work: bit-exact), on consecutive calls
that reuse the same array, allocate no device memory, and refuse sizes beyond
its capacity. This file is collected last so a failure here leaves every other
test already run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2312_12392_gb300 import rcp  # noqa: E402

pytestmark = pytest.mark.gpu


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 1 << 30, size=n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 4] = keys[0]  # duplicates, so stability is checked too
    rng.shuffle(keys)
    vals = rng.permutation(n).astype(np.uint32)
    return keys, vals


def _dev(a):
    return torch.from_numpy(a.view(np.int32).copy()).cuda()


@pytest.mark.parametrize("n,bits", [(300_001, 30), ("capacity", 32)])
def test_static_sort_matches_allocating_sort_twice(n, bits):
    if n == "capacity":
        n = rcp.rcp_sort_static_capacity()
    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        keys, vals = _pairs(n, seed=100 * call + bits)
        rk, rv = _dev(keys), _dev(vals)
        rcp.rcp_debug_sort_pairs(rk, rv, n, bits)
        sk, sv = _dev(keys), _dev(vals)
        rcp.rcp_sort_pairs_static(sk, sv, n, bits, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.equal(sk, rk), f"keys differ on call {call}"
        assert torch.equal(sv, rv), f"values differ on call {call}"


def test_static_sort_allocates_nothing():
    """After a first call (which looks up the array's address), a call leaves
    the device's free memory exactly as it was."""
    n = 200_003
    keys, vals = _pairs(n, seed=3)
    sk, sv = _dev(keys), _dev(vals)
    rcp.rcp_sort_pairs_static(sk, sv, n, 30)
    torch.cuda.synchronize()
    sk, sv = _dev(keys), _dev(vals)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rcp.rcp_sort_pairs_static(sk, sv, n, 30)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(sk.cpu().numpy().view(np.uint32), keys[order])


def test_static_sort_small_and_limits():
    keys, vals = _pairs(5, seed=1)
    sk, sv = _dev(keys), _dev(vals)
    rcp.rcp_sort_pairs_static(sk, sv, 5, 30)
    torch.cuda.synchronize()
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(sk.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(sv.cpu().numpy().view(np.uint32), vals[order])
    cap = rcp.rcp_sort_static_capacity()
    n = cap + 1
    big = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(rcp.RcpError) as e:
        rcp.rcp_sort_pairs_static(big, big.clone(), n, 30)
    assert e.value.status == rcp.RCP_ERR_ARG and "capacity" in str(e.value) and str(cap) in str(e.value)
