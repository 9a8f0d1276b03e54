"""Pins of the oracle's smooth-W estimator (eq. bpg_final with the
Gauss-sigmoid W of eq. weighting) against what the mathematics and the
paper fix, not against its own formulas."""
import numpy as np
import pytest

from oracle import correlate as oc
from oracle import mesh as om
from oracle import pipeline
from oracle import smooth as sm
from paper_1705_03464_gb300 import synth


def test_convolution_equals_direct_sum():
    """G(x) = sum_r W(r) delta(x - r) summed over all mesh offsets by hand."""
    rng = np.random.default_rng(0)
    N, L = 8, 40.0
    f = rng.uniform(0.2, 2.0, (N, N, N))
    Wm = sm.weight_mesh(L, N, sm.WParams(9.0, 6.0, 0.7, 4.0))
    G = sm.convolve(f, Wm)
    delta = f - f.mean()
    ref = np.zeros_like(f)
    for rz in range(N):
        for ry in range(N):
            for rx in range(N):
                ref += Wm[rz, ry, rx] * np.roll(delta, (rz, ry, rx), axis=(0, 1, 2))
    np.testing.assert_allclose(G, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_b_pg_is_one_when_pairs_are_the_galaxies():
    rng = np.random.default_rng(1)
    N, L = 16, 64.0
    pts = rng.uniform(0, L, (400, 3))
    w = rng.uniform(0.5, 1.5, 400)
    for assign in (0, 1, 2):
        G = sm.convolve(oc.field(om.deposit(pts, w, L, N, assign)), sm.weight_mesh(L, N, sm.W_DP10))
        g = sm.interpolate(G, pts, L, N, assign)
        assert sm.ratio_of_means(g, w, g, w) == 1.0


def test_xi_dw_of_a_plane_wave():
    """delta = A cos(2 pi m x / L) has C(r) = (A^2/2) cos(2 pi m r_x / L)
    exactly on the mesh, so eq. xi_dw must equal the W-weighted ratio of
    that closed form."""
    N, L, A, m = 32, 128.0, 0.3, 3
    x = np.arange(N) * (L / N)
    f = 1.0 + A * np.cos(2 * np.pi * m * x / L)[None, None, :] * np.ones((N, N, 1))
    q = np.rint(f * 2 ** 32).astype(np.int64)
    C = oc.correlate_mesh(q, q)
    o = sm.offsets(N, L)
    c_closed = np.broadcast_to(0.5 * A * A * np.cos(2 * np.pi * m * o / L)[None, None, :], (N, N, N))
    np.testing.assert_allclose(C, c_closed, atol=1e-9)
    Wm = sm.weight_mesh(L, N, sm.WParams(20.0, 14.0, 0.8, 6.0))
    ref = np.sum(Wm * c_closed ** 2) / np.sum(Wm * c_closed)
    assert sm.xi_dw(C, Wm) == pytest.approx(ref, rel=1e-8)


@pytest.mark.parametrize("prm", [sm.W_DP10, sm.W_DP30])
def test_weight_jump_at_the_cut_is_small(prm):
    """Sec. 3.6 chooses the parameters so that W jumps only a little at
    r_cut (Table tab:weightings); a sign error in the sigmoid breaks this."""
    r = np.linspace(0.0, 200.0, 20001)
    W = sm.weight(r, 0.0, prm)
    jump = sm.weight(prm.r_cut, 0.0, prm)
    assert 0.0 < jump < 1e-3 * W.max()
    assert np.all(sm.weight(np.linspace(0, prm.r_cut - 1e-9, 50), 3.0, prm) == 0.0)
    assert r[np.argmax(W)] > prm.r_cut


def test_estimate_runs_and_uses_every_pair_bin():
    cat = synth.make_catalogue_box(64.0, 600, seed=2)
    p = pipeline.Params(64.0, 32, 2, (0.0, 2.0, 4.0), 2, (6.0, 10.0), 1)
    out = sm.estimate(p, sm.WParams(12.0, 9.0, 0.8, 4.0), cat.pos)
    assert np.all(out["dd"] > 0) and np.all(np.isfinite(out["b_pg"]))
    assert np.isfinite(out["den"]) and np.isfinite(out["xi_dw"])
