"""Pins of the oracle's reverse-mode gradient of the smooth-W estimator:
central finite differences of its forward in single galaxy weights (h = 1e-3
relative, well above the Q32.32 rounding of the deposit), for a real-space
CIC and a redshift-space TSC case, and on the (d_perp, d_par) grid. Dropping
the xi(d_w) term, the RR normalisation or the galaxy-mean term changes the
gradient by 2 to 30 % of its largest component, far above these bounds."""
import numpy as np
import pytest

from oracle import pipeline
from oracle import smooth as sm
from oracle import smooth_adjoint as sa
from paper_1705_03464_gb300 import synth


def _case(assign, rsd, grid):
    L, N = 64.0, 32
    cat = synth.make_catalogue_box(L, 400, seed=3)
    w = synth.make_weights(cat.n, 3).astype(np.float64)
    if grid:
        p = pipeline.Params(L, N, assign, (0.0, 1.5, 3.0), 2, (6.0, 9.0), 1, rsd, 0.0, (0.0, 1.5, 3.5))
    else:
        p = pipeline.Params(L, N, assign, (0.0, 2.0, 4.0), 2, (6.0, 9.0), 1, rsd)
    return p, sm.WParams(8.0, 6.0, 0.8, 3.0), cat, w


@pytest.mark.parametrize("assign,rsd,grid", [(1, 0.0, False), (2, 0.011, False), (1, 0.011, True)])
def test_smooth_gradient_matches_central_differences(assign, rsd, grid):
    p, prm, cat, w = _case(assign, rsd, grid)
    st = sa.forward_state(p, prm, cat.pos, cat.vel, w)
    rng = np.random.default_rng(5)
    out = sa.outputs(st)
    gbar = {k: rng.standard_normal(np.asarray(out[k]).shape) for k in sa.OUTPUT_KEYS}
    g = sa.grad_weights(st, gbar)
    scale = np.max(np.abs(g))
    for i in rng.choice(cat.n, 5, replace=False):
        h = 1e-3 * w[i]
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (sa.loss(sa.forward_state(p, prm, cat.pos, cat.vel, wp), gbar)
              - sa.loss(sa.forward_state(p, prm, cat.pos, cat.vel, wm), gbar)) / (2 * h)
        assert abs(fd - g[i]) <= 2e-5 * abs(g[i]) + 1e-8 * scale, (i, fd, g[i])


def test_smooth_forward_state_matches_the_estimator():
    # the differentiable forward is the same estimator as oracle/smooth.py (the
    # two compute f and C_gg in different rounding orders)
    p, prm, cat, w = _case(2, 0.011, False)
    w32 = w.astype(np.float32)
    st = sa.forward_state(p, prm, cat.pos, cat.vel, w32.astype(np.float64))
    a = sa.outputs(st)
    b = sm.estimate(p, prm, cat.pos, cat.vel, w32)
    for k in ("num", "b_pg", "q_eff", "xi_ss"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(a["den"][0], b["den"], rtol=1e-8)
    np.testing.assert_allclose(a["xi_dw"][0], b["xi_dw"], rtol=1e-8)
