"""The HOD-derivative workflows of Sec. 5, built on the library's calls.

* ``emulator``: the projected 2PCF w(d_perp) (and xi per pair bin) with its
  first and second derivatives in the HOD parameters p = (log10 M_cut,
  log10 M_1, sigma, alpha) around a design HOD, the coefficients of eqs.
  2pf_emulate_1st and 2pf_emulate_2nd. The paper solves for them from 14
  separate evaluations; here they are exact, from the soft weights'
  derivatives (pg_hod_weights2) and one pass over the pairs
  (pg_hod_pair_derivs). kappa is left out, as in the paper.
* ``emulate``: the first- or second-order prediction at p. The paper's sum
  over k >= j with a factor 1/2 is the Taylor series when its off-diagonal
  coefficients are twice the mixed second derivatives, so the prediction
  is w0 + J dp + dp^T H dp / 2 with H the symmetric matrix of second
  derivatives.
* ``fit_at_alpha``: alpha fixed (the paper takes alpha0 +- 5 %), the other
  parameters that best reproduce the design w(d_perp): chi^2 of the
  emulated w against the design, with the paper's error model
  sigma_i^2 = sqrt(d_p,max^2 - d_perp,i^2) / d_perp,i for even d_perp bins,
  minimised from several starting points by BFGS, Powell and Nelder-Mead
  (the paper's three methods); the best minimum is kept.
* ``delta_q_eff``: delta Q_eff = [Q_eff(theta+) - Q_eff(theta-)] / Q_eff(theta0)
  per pair bin (and the same ratio for xi(d_p)), from three forwards of the
  smooth-W estimator on the GPU, as in the paper's redshift-space maps.

Every statistic comes from the library's kernels; this module only chains
the calls and runs the small host-side fit over four parameters.
"""
from __future__ import annotations

import time

import numpy as np

from . import pairgal as pg

N_EMU = 4   # emulated parameters: log10 M_cut, log10 M_1, sigma, alpha


def emulator(plan, pos, vel, mass, kind, kh, theta0, stream=None):
    """Design values and derivatives around theta0 (5 HOD parameters):
    {"theta0", "w0", "J" [n_s, 4], "H" [n_s, 4, 4], "xi0", "Jxi" [P, 4],
    "Hxi" [P, 4, 4], "ms"}. The plan must bin pairs on the (d_perp, d_par)
    grid for the w(d_perp) entries (else they are NaN)."""
    import torch
    t0 = time.perf_counter()
    w, dw, d2w = pg.pg_hod_weights2(mass, kind, kh, theta0, stream)
    d = pg.pg_hod_pair_derivs(plan, pos, vel, w, dw, d2w, stream)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    k = N_EMU
    return {"theta0": np.asarray(theta0, np.float64).copy(),
            "w0": d["w_perp"], "J": d["dw_perp"][:, :k], "H": d["d2w_perp"][:, :k, :k],
            "xi0": d["xi"], "Jxi": d["dxi"][:, :k], "Hxi": d["d2xi"][:, :k, :k], "ms": ms}


def emulate(em, theta, order=2, which="w"):
    """eq. 2pf_emulate_1st (order 1) or eq. 2pf_emulate_2nd (order 2) at the
    HOD parameters theta (5 values; kappa is not emulated)."""
    dp = np.asarray(theta, np.float64)[:N_EMU] - em["theta0"][:N_EMU]
    v0, J, H = (em["w0"], em["J"], em["H"]) if which == "w" else (em["xi0"], em["Jxi"], em["Hxi"])
    out = v0 + J @ dp
    if order >= 2:
        out = out + 0.5 * np.einsum("itu,t,u->i", H, dp, dp)
    return out


def chi2_sigma2(perp_edges, dp_max):
    """sigma_i^2 = sqrt(d_p,max^2 - d_perp,i^2) / d_perp,i at the d_perp bin
    centres (the paper's error on delta w_i, scaling with the inverse sample
    volume of a sphere of diameter d_p,max in pair-separation space)."""
    e = np.asarray(perp_edges, np.float64)
    c = 0.5 * (e[1:] + e[:-1])
    return np.sqrt(np.maximum(dp_max * dp_max - c * c, 0.0)) / c


def fit_at_alpha(em, alpha, perp_edges, dp_max, starts=None):
    """HOD parameters with alpha fixed that minimise the emulated chi^2
    sum_i (w_i(p) - w_i(p0))^2 / sigma_i^2 (bins with sigma_i = 0 left
    out). Returns (theta [5], chi2, {method: chi2})."""
    from scipy.optimize import minimize
    th0 = em["theta0"]
    s2 = chi2_sigma2(perp_edges, dp_max)
    use = s2 > 0
    target = em["w0"]

    def theta_of(x):
        t = th0.copy()
        t[0], t[1], t[2] = x
        t[3] = alpha
        return t

    def chi2(x):
        r = emulate(em, theta_of(x))[use] - target[use]
        return float(np.sum(r * r / s2[use]))

    if starts is None:
        base = th0[:3]
        starts = [base] + [base + d for d in ((0.1, 0.0, 0.0), (0.0, 0.1, 0.0), (0.0, 0.0, 0.1),
                                              (-0.1, -0.1, 0.0), (0.05, -0.05, -0.05))]
    best, best_x, per = np.inf, None, {}
    for method in ("BFGS", "Powell", "Nelder-Mead"):
        for x0 in starts:
            r = minimize(chi2, np.asarray(x0, np.float64), method=method,
                         options={"maxiter": 4000} if method != "BFGS" else {"gtol": 1e-12})
            per[method] = min(per.get(method, np.inf), float(r.fun))
            if r.fun < best:
                best, best_x = float(r.fun), r.x
    return theta_of(best_x), best, per


def delta_q_eff(plan, w_params, pos, vel, mass, kind, kh, theta_plus, theta_minus, theta0, stream=None):
    """delta Q_eff = [Q_eff(theta+) - Q_eff(theta-)] / Q_eff(theta0) and
    delta xi = [xi(theta+) - xi(theta-)] / xi(theta0) per pair bin (the
    paper's redshift-space maps on the (d_perp, d_par) grid), from the
    smooth-W estimator at the three HODs. Returns (dq [P], dxi [P], outputs
    at theta0, theta+, theta-)."""
    outs = []
    for th in (theta0, theta_plus, theta_minus):
        w, _ = pg.pg_hod_weights(mass, kind, kh, th, with_grad=False, stream=stream)
        outs.append(pg.pg_forward_smooth(plan, w_params, pos, vel, w, stream))
    o0, op_, om_ = outs
    with np.errstate(invalid="ignore", divide="ignore"):
        dq = (np.asarray(op_["q_eff"]) - np.asarray(om_["q_eff"])) / np.asarray(o0["q_eff"])
        dx = (np.asarray(op_["xi_ss"]) - np.asarray(om_["xi_ss"])) / np.asarray(o0["xi_ss"])
    return dq, dx, outs
