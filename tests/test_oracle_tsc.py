"""Pins of the oracle's mass assignment kernels (Sec. 3.5 uses TSC) that do
not restate the weight formulas: partition of unity, exact reproduction of
linear fields, the constant second moment of the quadratic B-spline, the
values at a node, and mass conservation of the Q32.32 deposit."""
import numpy as np
import pytest

from oracle import mesh as om


@pytest.mark.parametrize("assign", [0, 1, 2])
def test_partition_of_unity(assign):
    u = np.random.default_rng(1).uniform(0, 64, 5000)
    _, w = om.axis_nodes(u, 64, assign)
    np.testing.assert_allclose(w.sum(1), 1.0, rtol=0, atol=1e-15)
    assert np.all(w >= 0)


@pytest.mark.parametrize("assign", [1, 2])
def test_linear_fields_reproduced(assign):
    # away from the wrap, node indices are the unwrapped node positions
    u = np.random.default_rng(2).uniform(4, 60, 5000)
    idx, w = om.axis_nodes(u, 64, assign)
    np.testing.assert_allclose((w * idx).sum(1), u, rtol=0, atol=1e-12)


def test_tsc_second_moment_is_a_quarter():
    """For the quadratic B-spline sampled at unit nodes, sum_j w_j (x_j - u)^2
    is 1/4 wherever the point sits."""
    u = np.random.default_rng(3).uniform(4, 60, 5000)
    idx, w = om.axis_nodes(u, 64, 2)
    np.testing.assert_allclose((w * (idx - u[:, None]) ** 2).sum(1), 0.25, rtol=0, atol=1e-13)


def test_tsc_point_on_a_node():
    idx, w = om.axis_nodes(np.array([10.0]), 64, 2)
    assert idx.tolist() == [[9, 10, 11]]
    np.testing.assert_array_equal(w, [[0.125, 0.75, 0.125]])


def test_tsc_deposit_conserves_mass_and_wraps():
    rng = np.random.default_rng(4)
    L, N = 50.0, 16
    pts = rng.uniform(0, L, (300, 3))
    pts[:5] = [[0.0, 0.0, 0.0], [L - 1e-9, 1.0, 2.0], [0.2, L - 0.1, 7.0], [25.0, 25.0, 25.0], [3.1, 49.9, 0.01]]
    w = rng.uniform(0.5, 2.0, 300)
    mesh = om.deposit(pts, w, L, N, 2)
    # 27 roundings of at most 1/2 ulp of Q32.32 per point
    assert abs(int(mesh.sum()) - w.sum() * 2 ** 32) <= 27 * 300
    zs, ys, xs, k = om.node_weights(pts, L, N, 2)
    assert zs.shape == (300, 27) and zs.min() >= 0 and zs.max() < N
    np.testing.assert_allclose(k.sum(1), 1.0, atol=1e-14)
