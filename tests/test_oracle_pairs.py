"""Pins of the oracle's positions, pair enumeration and pair counts."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import pairs as op
from paper_1705_03464_gb300 import synth


def test_wrap_and_rsd_shift():
    L = 100.0
    pos = np.array([[-1.0, 101.0, 50.0], [99.999, 0.0, 99.0]])
    vel = np.array([[0.0, 0.0, 500.0], [0.0, 0.0, -200.0]], dtype=np.float32)
    x = op.transform_positions(pos, None, L, 0.0)
    assert np.allclose(x[0], [99.0, 1.0, 50.0])
    f = 0.01
    y = op.transform_positions(pos, vel, L, f)
    # eq. RSD: only the line-of-sight (z) coordinate moves, by v_z / H
    assert np.allclose(y[:, :2], x[:, :2])
    assert np.isclose(y[0, 2], 55.0) and np.isclose(y[1, 2], 97.0)
    z = op.transform_positions(np.array([[1.0, 1.0, 99.0]]), np.array([[0, 0, 300.0]], np.float32), L, f)
    assert np.isclose(z[0, 2], 2.0)  # 99 + 3 wraps to 2
    assert np.all((y >= 0) & (y < L))


def test_pair_counts_match_kdtree():
    """Cumulative pair counts equal scipy's periodic k-d tree counts exactly."""
    L = 64.0
    cat = synth.make_catalogue_box(L, 1500, seed=3)
    edges = (0.0, 0.5, 1.0, 2.0, 3.5, 5.0, 7.0)
    pr = op.find_pairs(cat.pos, None, L, edges, 1)
    dd, _ = op.pair_counts(pr, len(edges) - 1, 1)
    tree = cKDTree(cat.pos, boxsize=L)
    n = cat.n
    cum = [(tree.count_neighbors(tree, r) - n) // 2 for r in edges[1:]]
    ours = np.cumsum(dd)
    # count_neighbors uses d <= r, the oracle d < r: equal with continuous positions
    assert list(ours) == cum


def test_triplet_gives_three_pairs_and_midpoints():
    L = 50.0
    pos = np.array([[1.0, 1.0, 1.0], [2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [30.0, 30.0, 30.0]])
    pr = op.find_pairs(pos, None, L, (0.0, 5.0), 1)
    assert pr["i"].size == 3
    # min-image midpoint across the periodic boundary
    pos2 = np.array([[49.5, 10.0, 10.0], [0.5, 10.0, 10.0]])
    pr2 = op.find_pairs(pos2, None, L, (0.0, 5.0), 1)
    assert np.allclose(pr2["mid"][0], [0.0, 10.0, 10.0])


def test_midpoints_equidistant():
    L = 64.0
    cat = synth.make_catalogue_box(L, 800, seed=5)
    pr = op.find_pairs(cat.pos, None, L, (0.0, 6.0), 1)
    x = cat.pos
    di = op.min_image(pr["mid"] - x[pr["i"]], L)
    dj = op.min_image(pr["mid"] - x[pr["j"]], L)
    s = np.linalg.norm(op.min_image(x[pr["j"]] - x[pr["i"]], L), axis=1)
    assert np.allclose(np.linalg.norm(di, axis=1), s / 2, atol=1e-9)
    assert np.allclose(di, -dj, atol=1e-9)


def test_mu_bins_los_and_transverse():
    L = 50.0
    pos = np.array([[10, 10, 10], [10, 10, 13],      # along LOS: mu = 1 -> last bin
                    [20, 20, 20], [23, 20, 20],      # transverse: mu = 0
                    [30, 30, 30], [30, 31, 31]], float)  # mu = 1/sqrt2
    pr = op.find_pairs(pos, None, L, (0.0, 4.0), 4)
    got = {(int(i), int(j)): int(m) for i, j, m in zip(pr["i"], pr["j"], pr["mubin"])}
    assert got[(0, 1)] == 3 and got[(2, 3)] == 0 and got[(4, 5)] == 2


def test_poisson_dd_matches_rr():
    """Uniform catalogue: DD agrees with the exact RR within 4 sigma (eq. 2PCF_d_collapsed)."""
    L = 100.0
    pos = synth.make_uniform(L, 6000, seed=1)
    edges = (2.0, 4.0, 6.0, 8.0)
    n_mu = 2
    pr = op.find_pairs(pos, None, L, edges, n_mu)
    dd, ddq = op.pair_counts(pr, 3, n_mu)
    xi, rr = op.xi_ss(ddq, None, pos.shape[0], L, edges, n_mu)
    assert np.all(np.abs(dd - rr) < 4 * np.sqrt(rr))
    assert np.all(np.abs(xi) < 4 / np.sqrt(rr))


def test_weighted_counts_exact():
    L = 40.0
    rng = np.random.default_rng(2)
    pos = rng.random((300, 3)) * L
    w = synth.make_weights(300, 4)
    pr = op.find_pairs(pos, w, L, (0.0, 3.0, 6.0), 1)
    _, ddq = op.pair_counts(pr, 2, 1)
    wd = w.astype(np.float64)
    for b in range(2):
        sel = pr["sbin"] == b
        exact = sum(int(np.rint(wd[i] * wd[j] * 2.0 ** 32)) for i, j in zip(pr["i"][sel], pr["j"][sel]))
        assert ddq[b] == exact
    # weights all one: RR is N(N-1)/2 times the volume fraction
    _, rr = op.xi_ss(np.zeros(1, np.int64), np.ones(300, np.float32), 300, L, (0.0, 3.0), 1)
    assert math.isclose(rr[0], 300 * 299 / 2 * (4 / 3 * math.pi * 27) / L ** 3)


def test_kdtree_pairs_equal_brute_force():
    L = 80.0
    cat = synth.make_catalogue_box(L, 1500, seed=12)
    w = synth.make_weights(cat.n, 3)
    edges = (0.0, 1.0, 2.5, 4.0, 6.0)
    a = op.find_pairs(cat.pos, w, L, edges, 3)
    b = op.find_pairs_kdtree(cat.pos, w, L, edges, 3)
    oa = np.lexsort((a["j"], a["i"]))
    for k in ("i", "j", "sbin", "mubin", "mid", "weight"):
        np.testing.assert_array_equal(a[k][oa], b[k])
