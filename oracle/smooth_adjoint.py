"""Reverse-mode gradient of the smooth-W estimator with respect to the galaxy
weights (oracle, FP64, test-only).

The forward is the one of oracle/smooth.py (Sec. 2.1 eq. bpg_final with the
W of Sec. 3.6 eq. weighting, eqs. xi_dw, Qeff_notsq, 2PCF_d_collapsed), held
here with FP64 weights so that it can be differentiated and finite-differenced:

    rho = deposit of w_j,  Q = sum rho,  f = rho N^3 / Q,  delta = f - 1
    G = W * delta (k = 0 removed),  g_p = G at pair midpoints, g_j at galaxies
    num_b = sum_{p in b} w_p g_p / sum_{p in b} w_p,  den = sum_j w_j g_j / sum_j w_j
    b_b = num_b / den,  xi_b = DD_b / RR_b - 1 (DD_b = sum w_p, RR_b from sum w, sum w^2)
    C = (1/N^3) sum_x delta(x) delta(x + r),  xi_w = sum W C^2 / sum W C
    q_b = eq. Qeff_notsq(b_b, xi_b, xi_w),  w_p = w_i w_j

The reverse sweep takes these steps backwards: ratio outputs -> num, den, xi,
xi_w -> the pair and galaxy weights directly and, through the means, adjoint
weights at the points -> their deposit (the transpose of the interpolation)
-> the convolution with W (self-adjoint: W is real and even) -> the term of
xi_w, delta_bar += (2/N^3) Cbar * delta -> the rho / Q normalisation -> w.
The deposit's Q32.32 rounding is treated as exact (differences are taken at
steps well above it).
"""
from __future__ import annotations

import numpy as np

from . import correlate as oc
from . import dft
from . import mesh as om
from . import pairs as op
from . import smooth as sm

OUTPUT_KEYS = ("num", "den", "b_pg", "q_eff", "xi_ss", "xi_dw")


def _auto_corr(f):
    """C(r) = N^-6 IDFT[|DFT f|^2] with k = 0 removed."""
    N = f.shape[0]
    F = dft.dft3(np.asarray(f, dtype=np.complex128), -1)
    P = F * np.conj(F)
    P[0, 0, 0] = 0.0
    return dft.dft3(P, +1).real / float(N) ** 6


def _scatter(points, vals, L, N, assign):
    """The transpose of sm.interpolate: sum of vals times the node weights."""
    zs, ys, xs, k = om.node_weights(points, L, N, assign)
    out = np.zeros(N * N * N)
    np.add.at(out, ((zs * N + ys) * N + xs).reshape(-1), (k * np.asarray(vals)[:, None]).reshape(-1))
    return out.reshape(N, N, N)


def forward_state(p, prm, pos, vel, w):
    L, N = p.box_L, p.mesh_n
    x = op.transform_positions(pos, vel, L, p.rsd_factor)
    wt = np.asarray(w, dtype=np.float64)
    pr = op.find_pairs(x, None, L, p.s_edges, p.n_mu, par_edges=p.par_edges)
    pr["weight"] = wt[pr["i"]] * wt[pr["j"]]
    n_s = len(p.s_edges) - 1
    P = n_s * p.n_mu
    rho = om.deposit(x, wt, L, N, p.assign).astype(np.float64) / 2.0 ** 32
    Qs = rho.sum()
    f = rho * N ** 3 / Qs
    Wm = sm.weight_mesh(L, N, prm)
    G = sm.convolve(f, Wm)
    gj = sm.interpolate(G, x, L, N, p.assign)
    pb = pr["sbin"] * p.n_mu + pr["mubin"]
    gp = sm.interpolate(G, pr["mid"], L, N, p.assign) if pb.size else np.zeros(0)
    Wb = np.bincount(pb, weights=pr["weight"], minlength=P)
    Nb = np.bincount(pb, weights=pr["weight"] * gp, minlength=P)
    C = _auto_corr(f)
    S1, S2 = float(np.sum(Wm * C)), float(np.sum(Wm * C * C))
    sw, sw2 = wt.sum(), (wt * wt).sum()
    vb = op.pair_volumes(p.s_edges, p.n_mu, p.par_edges)
    return {"p": p, "prm": prm, "x": x, "w": wt, "pairs": pr, "pb": pb, "P": P, "rho": rho, "Q": Qs,
            "f": f, "W": Wm, "G": G, "gj": gj, "gp": gp, "Wb": Wb, "Nb": Nb, "C": C, "S1": S1, "S2": S2,
            "sw": sw, "sw2": sw2, "vb": vb}


def outputs(st):
    p = st["p"]
    with np.errstate(invalid="ignore", divide="ignore"):
        num = np.where(st["Wb"] > 0, st["Nb"] / st["Wb"], np.nan)
        den = float(np.sum(st["w"] * st["gj"]) / st["sw"])
        npairs = 0.5 * (st["sw"] ** 2 - st["sw2"])
        rr = npairs * st["vb"] / p.box_L ** 3
        xs = st["Wb"] / rr - 1.0
        xw = st["S2"] / st["S1"]
        b = num / den
        q = oc.q_eff_notsq(b, xs, xw)
    return {"num": num, "den": np.array([den]), "b_pg": b, "q_eff": q, "xi_ss": xs, "xi_dw": np.array([xw])}


def loss(st, gbar):
    out = outputs(st)
    tot = 0.0
    for k, g in gbar.items():
        v = np.asarray(out[k], float)
        g = np.asarray(g, float).reshape(v.shape)
        m = np.isfinite(v)
        tot += float(np.sum(g[m] * v[m]))
    return tot


def grad_weights(st, gbar):
    """dL/dw_j for L = sum_k sum gbar[k] * outputs[k] (non-finite outputs skipped)."""
    p, P = st["p"], st["P"]
    L, N = p.box_L, p.mesh_n
    out = outputs(st)
    gz = {}
    for k in OUTPUT_KEYS:
        v = np.asarray(out[k], float)
        g = np.asarray(gbar.get(k, np.zeros(v.shape)), float).reshape(v.shape)
        gz[k] = np.where(np.isfinite(v), g, 0.0)
    num, den, b, xs = out["num"], float(out["den"][0]), out["b_pg"], out["xi_ss"]
    xw = float(out["xi_dw"][0])
    npairs = 0.5 * (st["sw"] ** 2 - st["sw2"])
    rr = npairs * st["vb"] / L ** 3
    # ---- ratio outputs -> b, xi, xi_w (eq. Qeff_notsq) ----
    bbar = gz["b_pg"].copy()
    xsbar = gz["xi_ss"].copy()
    xwbar = float(gz["xi_dw"][0])
    for k in range(P):
        if gz["q_eff"][k] == 0.0:
            continue
        x, bb = xs[k], b[k]
        D = 2.0 * x + 1.5 * xw
        n = (1.0 + x) * bb - 2.0 - xw / (2.0 * x)
        gq = gz["q_eff"][k]
        bbar[k] += gq * (1.0 + x) / D
        xsbar[k] += gq * ((bb + xw / (2.0 * x * x)) / D - 2.0 * n / (D * D))
        xwbar += gq * ((-1.0 / (2.0 * x)) / D - 1.5 * n / (D * D))
    # ---- b = num / den ----
    fin = np.isfinite(num)
    numbar = np.where(fin, gz["num"] + bbar / den, 0.0)
    denbar = float(gz["den"][0]) - float(np.sum(np.where(fin, bbar * num, 0.0)) / den ** 2)
    # ---- means, xi = DD / RR - 1 ----
    wt, pr, pb = st["w"], st["pairs"], st["pb"]
    wp = pr["weight"]
    Wb = st["Wb"]
    wbar = np.zeros(wt.size)
    wpbar = np.zeros(wp.size)
    gpbar = np.zeros(wp.size)
    if wp.size:
        inb = Wb[pb] > 0
        wpbar += np.where(inb, numbar[pb] * (st["gp"] - np.nan_to_num(num[pb])) / np.where(inb, Wb[pb], 1.0), 0.0)
        gpbar = np.where(inb, numbar[pb] * wp / np.where(inb, Wb[pb], 1.0), 0.0)
        wpbar += np.where(rr[pb] > 0, xsbar[pb] / rr[pb], 0.0)
    wbar += denbar * (st["gj"] - den) / st["sw"]
    gjbar = denbar * wt / st["sw"]
    npb = float(np.sum(np.where(rr > 0, -xsbar * Wb / rr ** 2, 0.0) * st["vb"] / L ** 3))
    wbar += npb * (st["sw"] - wt)
    # ---- G at the points -> G mesh -> delta (convolution with W) ----
    Gbar = _scatter(st["x"], gjbar, L, N, p.assign)
    if wp.size:
        Gbar += _scatter(pr["mid"], gpbar, L, N, p.assign)
    fbar = sm.convolve(Gbar, st["W"])
    # ---- xi_w = S2 / S1 -> C -> delta ----
    Cbar = xwbar * st["W"] * (2.0 * st["C"] / st["S1"] - st["S2"] / st["S1"] ** 2)
    fbar += (2.0 / float(N) ** 3) * sm.convolve(st["f"], Cbar)
    # ---- f = rho N^3 / Q ----
    fj = sm.interpolate(fbar, st["x"], L, N, p.assign)
    T = float(np.sum(wt * fj))
    Qs = st["Q"]
    wbar += (float(N) ** 3 / Qs) * (fj - T / Qs)
    # ---- pair weights w_p = w_i w_j ----
    np.add.at(wbar, pr["i"], wpbar * wt[pr["j"]])
    np.add.at(wbar, pr["j"], wpbar * wt[pr["i"]])
    return wbar


__all__ = ["OUTPUT_KEYS", "forward_state", "outputs", "loss", "grad_weights"]
