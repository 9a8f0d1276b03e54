"""Pins of the oracle's soft HOD weights: eq. hod special values, the weight
derivatives against central differences, and dL/dtheta of the whole oracle
forward against central differences in theta."""
import math

import numpy as np

from oracle import adjoint as oa, hod, pipeline
from paper_1705_03464_gb300 import synth

TH = np.array(synth.HOD_Z09, dtype=np.float64)


def test_hod_special_values():
    mcut = 10.0 ** TH[0]
    # at M = M_cut the central occupation is 1/2; far above it is 1
    w = hod.weights(TH, [mcut, 1e16, 1e10], [0, 0, 0], [1, 1, 1])
    assert math.isclose(w[0], 0.5) and w[1] > 0.999999 and w[2] < 1e-6
    # satellites: zero below kappa M_cut, ((M - M_cut)/M_1)^alpha / K above
    m1 = 10.0 ** TH[1]
    s = hod.weights(TH, [0.5 * mcut, mcut + m1], [1, 1], [1, 2])
    assert s[0] == 0.0 and math.isclose(s[1], 0.5)


def test_weight_derivatives_central_differences():
    rng = np.random.default_rng(0)
    M = 10.0 ** rng.uniform(12.5, 15.0, 200)
    kind = rng.integers(0, 2, 200).astype(np.int32)
    kh = rng.integers(1, 5, 200).astype(np.float32)
    d = hod.dweights(TH, M, kind, kh)
    for k in range(5):
        h = 1e-6
        tp, tm = TH.copy(), TH.copy()
        tp[k] += h
        tm[k] -= h
        fd = (hod.weights(tp, M, kind, kh) - hod.weights(tm, M, kind, kh)) / (2 * h)
        assert np.allclose(fd, d[:, k], rtol=1e-5, atol=1e-9)


def test_dL_dtheta_central_differences():
    """alpha = 1.1: the satellite weight is then continuously differentiable at
    M = kappa M_cut (with alpha = 1 it has a kink there, and central
    differences across the kink are biased)."""
    th0 = TH.copy()
    th0[3] = 1.1
    L = 64.0
    cand = synth.make_candidates(L, 300, seed=4)
    p = pipeline.Params(L, 32, 1, (0.0, 2.0, 4.0), 2, (6.0, 9.0, 13.0), 2)
    rng = np.random.default_rng(1)

    def state(th):
        return oa.forward_state(p, cand.pos, None, hod.weights(th, cand.mass, cand.kind, cand.kh))

    st = state(th0)
    o = oa.outputs(st)
    gbar = {k: rng.standard_normal(np.asarray(o[k]).shape) for k in ("b_pg", "q_eff", "xi_pg", "xi_gg")}
    wbar = oa.grad_weights(st, gbar)
    g = hod.grad_theta(th0, cand.mass, cand.kind, cand.kh, wbar)
    def cd(k, h):
        tp, tm = th0.copy(), th0.copy()
        tp[k] += h
        tm[k] -= h
        return (oa.loss(state(tp), gbar) - oa.loss(state(tm), gbar)) / (2 * h)

    for k in range(5):
        # parameters that move the satellite threshold M = kappa M_cut get a small
        # step (the satellite weight's second derivative is singular there); sigma
        # only enters the smooth central weight and takes 1e-3, well above the
        # Q32.32 rounding of the meshes
        fd = cd(k, 1e-3 if k == 2 else 1e-4)
        assert abs(fd - g[k]) <= 1e-4 * abs(g[k]) + 1e-6, (k, fd, g[k])
