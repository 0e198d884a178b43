"""Pins of the test-side codec of the ABI's normal code (no GPU): round trip
within the header's bound, exact axes, the reserved code 0, the fold of the
lower hemisphere, and decoding of hand-built codes."""
import numpy as np

import abi_codec as A


def test_round_trip_within_bound():
    rng = np.random.default_rng(8)
    n = rng.normal(size=(20000, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    c = A.normal_encode(n)
    m, ok = A.normal_decode(c)
    assert ok.all() and (c != 0).all()
    err = np.linalg.norm(m - n, axis=1).max()
    assert err < A.ROUND_TRIP_TOL, err
    assert np.allclose(np.linalg.norm(m, axis=1), 1.0, atol=1e-12)


def test_axes_and_reserved_code():
    ax = np.vstack([np.eye(3), -np.eye(3)])
    m, ok = A.normal_decode(A.normal_encode(ax))
    assert ok.all() and np.allclose(m, ax, atol=1e-12)
    m, ok = A.normal_decode(np.array([0], np.uint32))
    assert not ok[0] and not m.any()
    assert A.normal_encode(np.zeros((1, 3)))[0] == 0


def test_hand_built_codes():
    # +z: p = (0, 0) -> fields 32768, 32768
    assert A.normal_encode([[0.0, 0.0, 1.0]])[0] == 32768 | (32768 << 16)
    # +x: p = (1, 0) -> q = (32767, 0)
    assert A.normal_encode([[1.0, 0.0, 0.0]])[0] == (32767 + 32768) | (32768 << 16)
    # -z folds to the corner (+1, +1) (sgn 0 = +1)
    assert A.normal_encode([[0.0, 0.0, -1.0]])[0] == (32767 + 32768) | ((32767 + 32768) << 16)
    # a lower-hemisphere normal and its mirror above differ only by the fold
    n = np.array([[0.3, -0.2, 0.5], [0.3, -0.2, -0.5]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    m, _ = A.normal_decode(A.normal_encode(n))
    assert m[0, 2] > 0 > m[1, 2] and np.allclose(m[:, :2], n[:, :2], atol=1e-4)


def test_lane_bits():
    c = np.array([1, 0xFFFFFFFF, 32768 | (32768 << 16)], np.uint32)
    assert np.array_equal(A.lane_to_codes(A.codes_to_lane(c)), c)
