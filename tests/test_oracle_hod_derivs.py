"""Pins of the exact HOD-parameter derivatives of the pair-count statistics
(oracle/hod_derivs.py) and of the soft weights' second derivatives: central
differences of the oracle's own xi(s, mu), xi(d_perp, d_par) and w(d_perp)
(oracle/pairs.py, pinned by brute force elsewhere), and the Taylor
structure of the second-order emulator (eq. 2pf_emulate_2nd)."""
import numpy as np
import pytest

from oracle import hod, hod_derivs as hd, pairs as op
from paper_1705_03464_gb300 import synth

TH = np.array(synth.HOD_Z09, dtype=np.float64)


def test_second_weight_derivatives_central_differences():
    rng = np.random.default_rng(3)
    th = TH.copy()
    th[3] = 1.3
    M = 10.0 ** rng.uniform(12.5, 15.0, 300)
    kind = rng.integers(0, 2, 300).astype(np.int32)
    kh = rng.integers(1, 5, 300).astype(np.float32)
    # keep satellites away from the threshold M = kappa M_cut, where the
    # second derivative of x^alpha is singular for alpha < 2
    mc = 10.0 ** th[0] * th[4]
    keep = (kind == 0) | (np.abs(M / mc - 1.0) > 0.05)
    M, kind, kh = M[keep], kind[keep], kh[keep]
    H = hod.d2weights(th, M, kind, kh)
    assert np.allclose(H, np.transpose(H, (0, 2, 1)))
    for k in range(5):
        h = 1e-6
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (hod.dweights(tp, M, kind, kh) - hod.dweights(tm, M, kind, kh)) / (2 * h)
        assert np.allclose(fd, H[:, :, k], rtol=1e-5, atol=1e-7), k
    # alpha = 1: the satellite weight is linear in x, so f_xx vanishes
    th1 = TH.copy()
    H1 = hod.d2weights(th1, M, kind, kh)
    s = (kind == 1) & (M > 10.0 ** th1[0] * th1[4])
    x = (M[s] - th1[4] * 10.0 ** th1[0]) / 10.0 ** th1[1]
    assert np.allclose(H1[s, 1, 1], x * np.log(10.0) ** 2 / kh[s])


def _candidates(L, n, seed, th):
    cand = synth.make_candidates(L, n, seed=seed)
    mc = 10.0 ** th[0] * th[4]
    keep = (cand.kind == 0) | (np.abs(cand.mass / mc - 1.0) > 0.05)
    return (cand.pos[keep], cand.mass[keep], cand.kind[keep], cand.kh[keep])


def _xi_of(th, pos, mass, kind, kh, L, s_edges, n_mu, par_edges=None):
    w = hod.weights(th, mass, kind, kh)
    pr = op.find_pairs(pos, None, L, s_edges, n_mu, par_edges=par_edges)
    b = pr["sbin"] * n_mu + pr["mubin"]
    DD = np.bincount(b, weights=w[pr["i"]] * w[pr["j"]], minlength=(len(s_edges) - 1) * n_mu)
    RR = 0.5 * (w.sum() ** 2 - np.sum(w * w)) * op.pair_volumes(s_edges, n_mu, par_edges) / L ** 3
    return DD / RR - 1.0


@pytest.mark.parametrize("grid", [False, True])
def test_xi_and_w_perp_derivatives_central_differences(grid):
    th = TH.copy()
    th[3] = 1.2
    L = 60.0
    pos, mass, kind, kh = _candidates(L, 500, 7, th)
    if grid:
        s_edges, par, n_mu = (0.0, 2.0, 4.0, 6.0), (0.0, 3.0, 6.0), 2
    else:
        s_edges, par, n_mu = (0.0, 2.0, 4.0, 6.0), None, 2
    w = hod.weights(th, mass, kind, kh)
    d = hd.derivs(pos, w, hod.dweights(th, mass, kind, kh), hod.d2weights(th, mass, kind, kh),
                  L, s_edges, n_mu, par)
    # the value against the oracle's own xi from its Q32.32 pair counts
    pr = op.find_pairs(pos, w.astype(np.float32), L, s_edges, n_mu, par_edges=par)
    _, ddq = op.pair_counts(pr, len(s_edges) - 1, n_mu)
    xs, _ = op.xi_ss(ddq, w.astype(np.float32), pos.shape[0], L, s_edges, n_mu, par)
    assert np.allclose(d["xi"], xs, rtol=1e-6, atol=1e-6)
    for k in range(5):
        h = 1e-5
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (_xi_of(tp, pos, mass, kind, kh, L, s_edges, n_mu, par)
              - _xi_of(tm, pos, mass, kind, kh, L, s_edges, n_mu, par)) / (2 * h)
        assert np.allclose(fd, d["dxi"][:, k], rtol=1e-5, atol=1e-6 * np.max(np.abs(fd))), k
        # second derivatives: central differences of the first
        wp, wm = hod.weights(tp, mass, kind, kh), hod.weights(tm, mass, kind, kh)
        dp = hd.derivs(pos, wp, hod.dweights(tp, mass, kind, kh), hod.d2weights(tp, mass, kind, kh),
                       L, s_edges, n_mu, par)
        dm = hd.derivs(pos, wm, hod.dweights(tm, mass, kind, kh), hod.d2weights(tm, mass, kind, kh),
                       L, s_edges, n_mu, par)
        fd2 = (dp["dxi"] - dm["dxi"]) / (2 * h)
        assert np.allclose(fd2, d["d2xi"][:, :, k], rtol=1e-4, atol=1e-5 * np.max(np.abs(fd2))), k
        if grid:
            fdw = (op.w_perp(_xi_of(tp, pos, mass, kind, kh, L, s_edges, n_mu, par), par)
                   - op.w_perp(_xi_of(tm, pos, mass, kind, kh, L, s_edges, n_mu, par), par)) / (2 * h)
            assert np.allclose(fdw, d["dw_perp"][:, k], rtol=1e-5, atol=1e-6 * np.max(np.abs(fdw)))
            assert np.allclose((dp["dw_perp"] - dm["dw_perp"]) / (2 * h), d["d2w_perp"][:, :, k],
                               rtol=1e-4, atol=1e-5 * np.max(np.abs(d["d2w_perp"])))
    if grid:
        assert np.allclose(d["w_perp"], op.w_perp(d["xi"], par))


def test_second_order_emulator_is_a_taylor_series():
    """eq. 2pf_emulate_2nd with the exact derivatives: the emulator's error at
    a parameter offset t*dp falls as t^3 (second order) where the linear
    emulator of eq. 2pf_emulate_1st falls as t^2. A factor other than 1/2 on
    the second-order term would leave a t^2 residual."""
    th = TH.copy()
    th[3] = 1.2
    L = 60.0
    pos, mass, kind, kh = _candidates(L, 500, 9, th)
    s_edges, par, n_mu = (0.0, 2.0, 4.0, 6.0), (0.0, 3.0, 6.0), 2
    w = hod.weights(th, mass, kind, kh)
    d = hd.derivs(pos, w, hod.dweights(th, mass, kind, kh), hod.d2weights(th, mass, kind, kh),
                  L, s_edges, n_mu, par)
    J, H = d["dw_perp"][:, :4], d["d2w_perp"][:, :4, :4]
    dp = np.array([0.02, -0.03, 0.04, 0.05])
    e1, e2 = [], []
    for t in (1.0, 0.5):
        tt = th.copy()
        tt[:4] += t * dp
        true = op.w_perp(_xi_of(tt, pos, mass, kind, kh, L, s_edges, n_mu, par), par)
        e1.append(np.max(np.abs(hd.emulate(d["w_perp"], J, None, t * dp) - true)))
        e2.append(np.max(np.abs(hd.emulate(d["w_perp"], J, H, t * dp) - true)))
    assert 3.0 < e1[0] / e1[1] < 5.0          # O(t^2)
    assert e2[0] / e2[1] > 6.0                # O(t^3)
    assert e2[0] < 0.2 * e1[0]
