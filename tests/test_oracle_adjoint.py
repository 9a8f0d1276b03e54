"""Pins of the oracle's reverse-mode gradient: central finite differences of
the oracle forward (h = 1e-3 relative, above the Q32.32 rounding)."""
import numpy as np
import pytest

from oracle import adjoint as oa, pipeline
from paper_1705_03464_gb300 import synth


def _setup(assign, rsd, cut):
    L, N = 64.0, 32
    cat = synth.make_catalogue_box(L, 400, seed=3)
    w = synth.make_weights(cat.n, 3).astype(np.float64)
    p = pipeline.Params(L, N, assign, (0.0, 2.0, 4.0), 2, (6.0, 9.0, 13.0), 2, rsd, cut)
    st = oa.forward_state(p, cat.pos, cat.vel, w)
    rng = np.random.default_rng(assign + 7)
    o = oa.outputs(st)
    gbar = {k: rng.standard_normal(np.asarray(o[k]).shape) for k in oa.OUTPUT_KEYS}
    return p, cat, w, st, gbar, rng


@pytest.mark.parametrize("assign,rsd,cut", [(0, 0.0, 0.0), (1, 0.011, 3.0)])
def test_gradient_matches_central_differences(assign, rsd, cut):
    p, cat, w, st, gbar, rng = _setup(assign, rsd, cut)
    g = oa.grad_weights(st, gbar)
    for i in rng.choice(cat.n, 3, replace=False):
        h = 1e-3 * w[i]
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (oa.loss(oa.forward_state(p, cat.pos, cat.vel, wp), gbar)
              - oa.loss(oa.forward_state(p, cat.pos, cat.vel, wm), gbar)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(g[i]) + 1e-9


def test_directional_derivative():
    p, cat, w, st, gbar, rng = _setup(1, 0.0, 0.0)
    g = oa.grad_weights(st, gbar)
    v = rng.standard_normal(cat.n) * w
    h = 1e-3
    fd = (oa.loss(oa.forward_state(p, cat.pos, None, w + h * v), gbar)
          - oa.loss(oa.forward_state(p, cat.pos, None, w - h * v), gbar)) / (2 * h)
    assert abs(fd - g @ v) <= 1e-5 * abs(g @ v)
