"""The rule the GPU parity tests use to accept a membership that differs from
the oracle's (tests/parity.py), checked on hand-made cases without a GPU: an
exact tie between centers the oracle and the kernel both hold exactly must be
decided alike; a near-tie on rounded values may go either way; a clear
difference is always rejected."""
import numpy as np

import oracle
from parity import all_exact, exact_sq, unexplained_flips


def pack(rgb):
    rgb = np.asarray(rgb, np.uint32)
    return (rgb[:, 0] << 16) | (rgb[:, 1] << 8) | rgb[:, 2]


def test_exact_distances():
    x = np.array([[10.0, 20.0, 30.0]])
    assert exact_sq(x, np.array([[3.0, 250.0, 0.0]]))[0]
    assert exact_sq(x, np.array([[10.125, 19.875, 30.5]]))[0]
    third = float(np.float32(1.0 / 3.0))
    assert not exact_sq(x, np.array([[third, 0.0, 0.0]]))[0]
    assert all_exact(np.array([[0.0, 255.0, 12.375]]))
    assert not all_exact(np.array([[0.1, 0.0, 0.0]]))


def test_an_exact_tie_must_follow_the_visit_order():
    # color (10, 0, 0) is exactly between centers 0 (5, 0, 0) and 2 (15, 0, 0)
    colors = pack([[10, 0, 0]])
    c = np.array([[5.0, 0, 0], [200.0, 200, 200], [15.0, 0, 0]])
    lab = np.zeros(1, np.int32)
    ref, _, _ = oracle.assign(colors, c, lab)
    other = 2 if ref[0] == 0 else 0
    assert unexplained_flips(colors, c, c, lab, np.array([other]), ref).size == 1
    assert unexplained_flips(colors, c, c, lab, ref.copy(), ref).size == 0


def test_duplicate_centers_are_an_exact_tie():
    colors = pack([[100, 50, 25]])
    third = float(np.float32(1.0 / 3.0))
    c = np.array([[90.0 + third, 50, 25], [0.0, 0, 0], [90.0 + third, 50, 25]])
    lab = np.ones(1, np.int32)
    ref, _, _ = oracle.assign(colors, c, lab)
    other = 2 if ref[0] == 0 else 0
    assert unexplained_flips(colors, c, c, lab, np.array([other]), ref).size == 1


def test_a_near_tie_on_rounded_values_may_flip():
    colors = pack([[10, 0, 0]])
    third = float(np.float32(1.0 / 3.0))
    # the color is almost exactly between the two centers (far within the
    # 1e-3 gap), and neither
    # distance is computed exactly in FP32
    d = 4.0 + third
    c = np.array([[10.0 - d, 0, 0], [200.0, 200, 200], [10.0 + d + 1e-6, 0, 0]])
    c32 = c.astype(np.float32).astype(np.float64)
    lab = np.zeros(1, np.int32)
    ref, _, _ = oracle.assign(colors, c, lab)
    best, second, _ = oracle.exhaustive(colors, c)
    assert second[0] - best[0] <= 1e-3
    other = 2 if ref[0] == 0 else 0
    assert unexplained_flips(colors, c, c32, lab, np.array([other]), ref).size == 0


def test_a_clear_difference_is_rejected():
    colors = pack([[10, 0, 0], [199, 201, 200]])
    third = float(np.float32(1.0 / 3.0))
    c = np.array([[5.0 + third, 0, 0], [200.0 + third, 200, 200], [30.0, 0, 0]])
    lab = np.zeros(2, np.int32)
    ref, _, _ = oracle.assign(colors, c, lab)
    got = ref.copy()
    got[1] = 2
    bad = unexplained_flips(colors, c, c.astype(np.float32).astype(np.float64), lab, got, ref)
    assert bad.tolist() == [1]
