"""Host logic of the HOD-derivative workflows (no GPU): the emulator
expansion and the alpha-constrained fit with the paper's error model."""
import numpy as np
import pytest

pytest.importorskip("scipy")


def _study():
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import hod_study
    return hod_study


def test_emulate_is_the_taylor_series_of_a_quadratic():
    hs = _study()
    rng = np.random.default_rng(0)
    J = rng.standard_normal((6, 4))
    A = rng.standard_normal((6, 4, 4))
    H = A + np.transpose(A, (0, 2, 1))
    w0 = rng.standard_normal(6)
    th0 = np.array([13.35, 13.8, 0.85, 1.0, 1.0])
    em = {"theta0": th0, "w0": w0, "J": J, "H": H, "xi0": w0, "Jxi": J, "Hxi": H}
    dp = np.array([0.1, -0.2, 0.05, 0.3])
    th = th0.copy()
    th[:4] += dp
    exact = w0 + J @ dp + 0.5 * np.array([dp @ H[i] @ dp for i in range(6)])
    np.testing.assert_allclose(hs.emulate(em, th), exact, rtol=1e-13)
    np.testing.assert_allclose(hs.emulate(em, th, order=1), w0 + J @ dp, rtol=1e-13)
    th[4] = 7.0   # kappa is not emulated
    np.testing.assert_allclose(hs.emulate(em, th), exact, rtol=1e-13)


def test_chi2_sigma_matches_the_paper_error_model():
    hs = _study()
    e = np.array([0.0, 2.0, 4.0, 6.0])
    s2 = hs.chi2_sigma2(e, 10.0)
    c = np.array([1.0, 3.0, 5.0])
    np.testing.assert_allclose(s2, np.sqrt(100.0 - c * c) / c)
    assert hs.chi2_sigma2(np.array([8.0, 12.0]), 10.0)[0] == 0.0


def test_fit_at_alpha_recovers_a_planted_degeneracy():
    """A linear-plus-quadratic w(p) built so that moving alpha is exactly
    compensated by a known move of (log M_cut, log M_1, sigma): the fit at
    the new alpha finds that move, with chi^2 at zero."""
    hs = _study()
    rng = np.random.default_rng(3)
    n = 12
    B = rng.standard_normal((n, 3))
    comp = np.array([0.04, -0.07, 0.02])      # d(t0, t1, sigma) per unit d(alpha)
    J = np.concatenate([B, -(B @ comp)[:, None]], axis=1)
    # the quadratic term vanishes along the compensating direction
    v = np.concatenate([comp, [1.0]])
    Pm = np.eye(4) - np.outer(v, v) / (v @ v)
    H = np.stack([Pm @ (M + M.T) @ Pm for M in rng.standard_normal((n, 4, 4)) * 0.1])
    th0 = np.array([13.35, 13.8, 0.85, 1.0, 1.0])
    em = {"theta0": th0, "w0": rng.standard_normal(n), "J": J, "H": H}
    edges = np.linspace(0.0, 24.0, n + 1)
    th, chi2, per = hs.fit_at_alpha(em, 1.05, edges, 30.0)
    assert chi2 < 1e-12
    np.testing.assert_allclose(th[:3], th0[:3] + 0.05 * comp, atol=1e-5)
    assert th[3] == 1.05 and th[4] == th0[4]
    assert set(per) == {"BFGS", "Powell", "Nelder-Mead"}
