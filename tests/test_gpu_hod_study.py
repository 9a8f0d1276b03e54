"""GPU HOD-derivative workflows (Sec. 5): the soft weights' second
derivatives, the exact emulator coefficients (eqs. 2pf_emulate_1st/2nd) and
delta Q_eff against the oracle on the same seeded inputs, and the emulator
against central differences of the GPU forward at 512^3."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import hod, hod_derivs as hd, pairs as op, pipeline  # noqa: E402
from oracle import smooth as sm  # noqa: E402
from paper_1705_03464_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def pg():
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import pairgal
    return pairgal


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _theta(alpha):
    th = np.array(synth.HOD_Z09, dtype=np.float64)
    th[3] = alpha
    return th


def _cand(L, n, seed, th):
    """Candidates with no satellite halo within 5 % of M = kappa M_cut, where
    the satellite weight is not twice differentiable."""
    c = synth.make_candidates(L, n, seed=seed)
    mc = 10.0 ** th[0] * th[4]
    keep = (c.kind == 0) | (np.abs(c.mass / mc - 1.0) > 0.05)
    return (np.ascontiguousarray(c.pos[keep]), np.ascontiguousarray(c.vel[keep]),
            np.ascontiguousarray(c.mass[keep]), np.ascontiguousarray(c.kind[keep]),
            np.ascontiguousarray(c.kh[keep]))


def _close(got, ref, rel):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    ok = np.isfinite(ref)
    assert np.array_equal(ok, np.isfinite(got))
    scale = np.max(np.abs(ref[ok])) if ok.any() else 1.0
    assert np.max(np.abs(got[ok] - ref[ok])) <= rel * scale, np.max(np.abs(got[ok] - ref[ok])) / scale


def test_hod_weights2_match_oracle(pg):
    th = _theta(1.2)
    pos, vel, mass, kind, kh = _cand(64.0, 400, 5, th)
    w, dw, d2w = pg.pg_hod_weights2(dev(mass), dev(kind), dev(kh), th)
    assert np.allclose(w.cpu().numpy(), hod.weights(th, mass, kind, kh).astype(np.float32), rtol=2e-7, atol=1e-12)
    _close(dw.cpu().numpy(), hod.dweights(th, mass, kind, kh), 1e-12)
    _close(d2w.cpu().numpy(), hod.d2weights(th, mass, kind, kh), 1e-12)
    # the first-order entry point gives the same weights and derivatives
    w1, dw1 = pg.pg_hod_weights(dev(mass), dev(kind), dev(kh), th)
    assert torch.equal(w1, w) and torch.equal(dw1, dw)


@pytest.mark.parametrize("grid,rsd", [(False, 0.0), (True, 0.0), (True, 0.011)])
def test_pair_derivs_match_oracle(pg, grid, rsd):
    th = _theta(1.2)
    L = 60.0
    pos, vel, mass, kind, kh = _cand(L, 500, 7, th)
    s_edges, n_mu = (0.0, 2.0, 4.0, 6.0), 2
    par = (0.0, 3.0, 6.0) if grid else None
    plan = pg.Plan(L, 32, 1, s_edges, n_mu, (8.0, 12.0), 1, rsd_factor=rsd, par_edges=par)
    w, dw, d2w = pg.pg_hod_weights2(dev(mass), dev(kind), dev(kh), th)
    got = pg.pg_hod_pair_derivs(plan, dev(pos), dev(vel) if rsd else None, w, dw, d2w)
    x = op.transform_positions(pos, vel, L, rsd)
    ref = hd.derivs(x, w.cpu().numpy().astype(np.float64), dw.cpu().numpy(), d2w.cpu().numpy(),
                    L, s_edges, n_mu, par)
    for k in ("xi", "dxi", "d2xi"):
        _close(got[k], ref[k], 1e-11)
    if grid:
        for k in ("w_perp", "dw_perp", "d2w_perp"):
            _close(got[k], ref[k], 1e-11)
    else:
        assert np.all(np.isnan(got["w_perp"]))
    # the value agrees with the forward path's own xi(s, mu) (Q32.32 counts)
    fwd = pg.pg_forward(plan, dev(pos), dev(vel) if rsd else None, w)
    _close(got["xi"], fwd["xi_ss"], 1e-8)


def test_delta_q_eff_matches_oracle(pg):
    """delta Q_eff and delta xi from three smooth-W forwards (FP64 plan, TSC,
    redshift space, the (d_perp, d_par) grid) against the oracle's smooth
    estimator at the same three HODs."""
    from paper_1705_03464_gb300 import hod_study as hs
    th0 = _theta(1.0)
    thp, thm = _theta(1.05), _theta(0.95)
    thp[1] += 0.02
    thm[1] -= 0.02
    L = 96.0
    pos, vel, mass, kind, kh = _cand(L, 1500, 11, th0)
    perp, par = (0.0, 2.0, 4.0, 6.0), (0.0, 3.0, 6.0)
    wprm = (14.0, 10.0, 0.5, 5.0)
    plan = pg.Plan(L, 32, 2, perp, 2, (8.0, 12.0), 1, rsd_factor=synth.RSD_FACTOR_Z05, precision=1,
                   par_edges=par)
    dq, dx, _ = hs.delta_q_eff(plan, wprm, dev(pos), dev(vel), dev(mass), dev(kind), dev(kh), thp, thm, th0)
    p = pipeline.Params(L, 32, 2, perp, 2, (8.0, 12.0), 1, synth.RSD_FACTOR_Z05, 0.0, par)
    ref = []
    for th in (th0, thp, thm):
        w = pg.pg_hod_weights(dev(mass), dev(kind), dev(kh), th, with_grad=False)[0].cpu().numpy()
        ref.append(sm.estimate(p, sm.WParams(*wprm), pos, vel, w))
    rq = (ref[1]["q_eff"] - ref[2]["q_eff"]) / ref[0]["q_eff"]
    rx = (ref[1]["xi_ss"] - ref[2]["xi_ss"]) / ref[0]["xi_ss"]
    _close(dq, rq, 1e-7)
    _close(dx, rx, 1e-9)


@pytest.mark.slow
def test_emulator_against_gpu_forward_512(pg):
    """A 512^3 box of about 18000 halos' candidates on a (d_perp, d_par) grid
    to 20 Mpc/h: the exact first derivatives of w(d_perp) against central
    differences in theta of the GPU forward's w(d_perp), and the second-order
    emulator (eq. 2pf_emulate_2nd) against the forward at alpha = 1.05,
    closer than the first-order one (eq. 2pf_emulate_1st)."""
    from paper_1705_03464_gb300 import hod_study as hs
    th0 = _theta(1.0)
    L = 512.0
    pos, vel, mass, kind, kh = _cand(L, 18000, 0, th0)
    perp, par = tuple(np.linspace(0.0, 20.0, 11)), tuple(np.linspace(0.0, 20.0, 5))
    plan = pg.Plan(L, 512, 1, perp, len(par) - 1, (30.0, 40.0), 1, precision=1, par_edges=par)
    P, M, K, H = dev(pos), dev(mass), dev(kind), dev(kh)
    em = hs.emulator(plan, P, None, M, K, H, th0)

    def w_of(th):
        w, _ = pg.pg_hod_weights(M, K, H, th, with_grad=False)
        return np.asarray(pg.pg_forward(plan, P, None, w)["w_perp"])

    w0 = w_of(th0)
    _close(em["w0"], w0, 1e-7)
    for k in range(4):
        h = 1e-3 if k == 2 else 2e-4
        tp, tm = th0.copy(), th0.copy()
        tp[k] += h
        tm[k] -= h
        fd = (w_of(tp) - w_of(tm)) / (2 * h)
        _close(em["J"][:, k], fd, 1e-4)
    th = th0.copy()
    th[3] = 1.05
    true = w_of(th)
    e1 = np.max(np.abs(hs.emulate(em, th, order=1) - true))
    e2 = np.max(np.abs(hs.emulate(em, th, order=2) - true))
    print(f"512^3 emulator at alpha = 1.05: first-order error {e1:.3e}, second-order {e2:.3e}")
    assert e2 < 0.25 * e1
