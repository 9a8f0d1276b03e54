"""Reverse-mode gradient of the outputs with respect to per-galaxy weights
(oracle, FP64, test-only).

The forward quantities follow ``pipeline`` (Sec. 2.1-2.2, 3.4-3.5). With
galaxy weights w_i, a pair p = (i, j) carries w_p = w_i w_j; the pair mesh of
bin b is rho_b(y) = sum_p w_p K(y - m_p) (K: CIC or NGP node weights), the
galaxy mesh rho_g(y) = sum_j w_j K(y - x_j), f = rho * N^3 / Q with
Q = sum_x rho, and

    C_b(r)  = (1/N^3) sum_x f_g(x) f_b(x + r) - 1,
    C_gg(r) = (1/N^3) sum_x f_g(x) f_g(x + r) - 1.

Bin sums S[b][q] = sum_{r in q} C_b(r), G[q], G2[q] = sum C_gg^2 feed the
ratio outputs (eqs. xi_dw, Qeff, Qeff_notsq), and xi(s, mu) = DD/RR - 1
with DD = sum_p w_p and RR from ((sum w)^2 - sum w^2)/2 (eq. 2PCF_d_collapsed).

Given upstream gradients gbar on the outputs, ``grad_weights`` returns
dL/dw_i for L = sum gbar * outputs, written out step by step in reverse:
ratios -> bin sums -> correlation cells -> f fields (real-space
correlations, evaluated with np.roll, no FFT) -> rho (normalisation) ->
w_p and w_j (gather with the same node weights) -> w_i. The Q32.32
rounding of the forward meshes is treated as the identity.
"""
from __future__ import annotations

import numpy as np

from . import correlate as oc
from . import mesh as om
from . import pairs as op

OUTPUT_KEYS = ("xi_pg", "xi_gg", "b_pg", "q_eff", "q_eff_sq", "xi_dw", "b_pg_agg", "q_eff_agg",
               "xi_dw_agg", "xi_ss", "dd_w")
# on the (d_perp, d_par) pair grid the projected w(d_perp) is an output too
GRID_OUTPUT_KEYS = OUTPUT_KEYS + ("w_perp",)


def _node_weights(points, L, N, assign):
    """Nodes (iz, iy, ix) and unrounded weights K of each point: [n, k] arrays."""
    return om.node_weights(points, L, N, assign)


def _gather(field, nodes):
    z, y, x, k = nodes
    return np.sum(field[z, y, x] * k, axis=1)


def _window_offsets(w):
    o = np.arange(-w, w + 1)
    c, b, a = np.meshgrid(o, o, o, indexing="ij")
    return c.reshape(-1), b.reshape(-1), a.reshape(-1)


def _corr_window(fa, fb, w):
    """C_ab over the window: (1/N^3) sum_x fb(x) fa(x + r) - 1, flat [W^3]."""
    N = fa.shape[0]
    oz, oy, ox = _window_offsets(w)
    out = np.empty(oz.size)
    for t in range(oz.size):
        out[t] = np.sum(fb * np.roll(fa, (-oz[t], -oy[t], -ox[t]), axis=(0, 1, 2))) / N ** 3 - 1.0
    return out


def _sum_shift(cbar, f, w, sign):
    """(1/N^3) sum_r cbar(r) f(y + sign * r) as a mesh."""
    N = f.shape[0]
    oz, oy, ox = _window_offsets(w)
    out = np.zeros_like(f)
    for t in np.nonzero(cbar)[0]:
        # np.roll(f, s)[y] = f[y - s]
        out += cbar[t] * np.roll(f, (-sign * oz[t], -sign * oy[t], -sign * ox[t]), axis=(0, 1, 2))
    return out / N ** 3


def forward_state(p, pos, vel, w):
    """Forward quantities in FP64 with the real-space correlation."""
    L, N = p.box_L, p.mesh_n
    x = op.transform_positions(pos, vel, L, p.rsd_factor)
    # weights taken in FP64 as given (FP32 inputs convert exactly), so that
    # finite differences of this forward are not rounded to FP32
    wt = np.asarray(w, dtype=np.float64)
    pr = op.find_pairs(x, None, L, p.s_edges, p.n_mu, par_edges=getattr(p, "par_edges", None))
    pr["weight"] = wt[pr["i"]] * wt[pr["j"]]
    n_s = len(p.s_edges) - 1
    P = n_s * p.n_mu
    Q = (len(p.r_edges) - 1) * p.n_mur
    wh = oc.window_half(N, L, p.r_edges[-1])
    bins, agg = oc.cell_bins(N, L, p.r_edges, p.n_mur, p.r_perp_cut, wh)
    rho_g = om.deposit(x, wt, L, N, p.assign).astype(np.float64) / 2.0 ** 32
    f_g = rho_g * N ** 3 / rho_g.sum()
    cgg = _corr_window(f_g, f_g, wh)
    pb = pr["sbin"] * p.n_mu + pr["mubin"]
    st = {"p": p, "x": x, "w": wt, "pairs": pr, "pb": pb, "P": P, "Q": Q, "wh": wh, "bins": bins,
          "agg": agg, "rho_g": rho_g, "f_g": f_g, "cgg": cgg, "f_b": {}, "rho_b": {}, "cb": {}}
    S = np.full((P, Q + 1), np.nan)
    for b in range(P):
        sel = pb == b
        if not np.any(sel):
            continue
        rho = om.deposit(pr["mid"][sel], pr["weight"][sel], L, N, p.assign).astype(np.float64) / 2.0 ** 32
        fb = rho * N ** 3 / rho.sum()
        cb = _corr_window(fb, f_g, wh)
        st["f_b"][b], st["rho_b"][b], st["cb"][b] = fb, rho, cb
        S[b, :Q] = np.bincount(bins[bins >= 0], weights=cb[bins >= 0], minlength=Q)
        S[b, Q] = cb[agg].sum()
    G = np.append(np.bincount(bins[bins >= 0], weights=cgg[bins >= 0], minlength=Q), cgg[agg].sum())
    G2 = np.append(np.bincount(bins[bins >= 0], weights=cgg[bins >= 0] ** 2, minlength=Q),
                   (cgg[agg] ** 2).sum())
    n = np.append(np.bincount(bins[bins >= 0], minlength=Q), np.count_nonzero(agg)).astype(float)
    dd_w = np.bincount(pb, weights=pr["weight"], minlength=P)
    sw, sw2 = wt.sum(), (wt * wt).sum()
    vb = op.pair_volumes(p.s_edges, p.n_mu, getattr(p, "par_edges", None))
    st.update({"S": S, "G": G, "G2": G2, "n": n, "dd_w": dd_w, "sw": sw, "sw2": sw2, "vb": vb})
    return st


def outputs(st):
    """The differentiable outputs (same definitions as correlate.ratios)."""
    p, Q = st["p"], st["Q"]
    S, G, G2, n = st["S"], st["G"], st["G2"], st["n"]
    npairs = 0.5 * (st["sw"] ** 2 - st["sw2"])
    rr = npairs * st["vb"] / p.box_L ** 3
    xs = st["dd_w"] / rr - 1.0
    with np.errstate(invalid="ignore", divide="ignore"):
        bb = S[:, :Q] / G[None, :Q]
        xw = G2[:Q] / G[:Q]
        b_agg = S[:, Q] / G[Q]
        xw_agg = G2[Q] / G[Q]
        return {"xi_pg": S[:, :Q] / n[None, :Q], "xi_gg": G[:Q] / n[:Q], "b_pg": bb,
                "q_eff": oc.q_eff_notsq(bb, xs[:, None], xw[None, :]),
                "q_eff_sq": oc.q_eff_sq(bb, xs[:, None]), "xi_dw": xw, "b_pg_agg": b_agg,
                "q_eff_agg": oc.q_eff_notsq(b_agg, xs, xw_agg), "xi_dw_agg": np.array([xw_agg]),
                "xi_ss": xs, "dd_w": st["dd_w"], "w_perp": _w_perp(p, xs)}


def _w_perp(p, xs):
    """w(d_perp) on the (d_perp, d_par) grid, NaN for (s, mu) bins."""
    pe = getattr(p, "par_edges", None)
    if pe is None:
        return np.full(len(p.s_edges) - 1, np.nan)
    return op.w_perp(xs, pe)


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
    """dL/dw_i for L = sum_k sum gbar[k] * outputs[k] (non-finite outputs skipped)."""
    p, P, Q = st["p"], st["P"], st["Q"]
    L, N, wh = p.box_L, p.mesh_n, st["wh"]
    S, G, G2, n = st["S"], st["G"], st["G2"], st["n"]
    out = outputs(st)
    gz = {k: np.zeros_like(np.asarray(out[k], float)) for k in GRID_OUTPUT_KEYS}
    for k, g in gbar.items():
        v = np.asarray(out[k], float)
        gz[k] = np.where(np.isfinite(v), np.asarray(g, float).reshape(v.shape), 0.0)
    npairs = 0.5 * (st["sw"] ** 2 - st["sw2"])
    rr = npairs * st["vb"] / L ** 3
    xs = st["dd_w"] / rr - 1.0
    # ---- ratios -> bin sums (quotient rule on each output) ----
    Sb = np.zeros((P, Q + 1))
    Gb = np.zeros(Q + 1)
    G2b = np.zeros(Q + 1)
    xsb = gz["xi_ss"].copy()
    pe = getattr(p, "par_edges", None)
    if pe is not None:   # w(d_perp) = sum_m 2 (l_hi - l_lo) xi(d_perp, d_par)
        dl2 = 2.0 * (np.asarray(pe, float)[1:] - np.asarray(pe, float)[:-1])
        xsb += (gz["w_perp"][:, None] * dl2[None, :]).reshape(-1)
    valid = np.isfinite(S[:, 0])
    for b in np.nonzero(valid)[0]:
        x = xs[b]
        for q in range(Q):
            bb = S[b, q] / G[q]
            xw = G2[q] / G[q]
            den = 2 * x + 1.5 * xw
            num = (1 + x) * bb - 2 - xw / (2 * x)
            g_q, g_s = gz["q_eff"][b, q], gz["q_eff_sq"][b, q]
            d_bb = gz["b_pg"][b, q] + g_q * (1 + x) / den + g_s * (1 + x) / (2 * x)
            d_x = g_q * ((bb + xw / (2 * x * x)) / den - 2 * num / den ** 2) \
                + g_s * (bb / (2 * x) - ((1 + x) * bb - 2) / (2 * x * x))
            d_xw = g_q * (-1 / (2 * x) / den - 1.5 * num / den ** 2)
            Sb[b, q] += gz["xi_pg"][b, q] / n[q] + d_bb / G[q]
            Gb[q] += -d_bb * S[b, q] / G[q] ** 2 - d_xw * G2[q] / G[q] ** 2
            G2b[q] += d_xw / G[q]
            xsb[b] += d_x
        ba = S[b, Q] / G[Q]
        xwa = G2[Q] / G[Q]
        den = 2 * x + 1.5 * xwa
        num = (1 + x) * ba - 2 - xwa / (2 * x)
        g_a = gz["q_eff_agg"][b]
        d_ba = gz["b_pg_agg"][b] + g_a * (1 + x) / den
        d_xa = g_a * ((ba + xwa / (2 * x * x)) / den - 2 * num / den ** 2)
        d_xwa = g_a * (-1 / (2 * x) / den - 1.5 * num / den ** 2)
        Sb[b, Q] += d_ba / G[Q]
        Gb[Q] += -d_ba * S[b, Q] / G[Q] ** 2 - d_xwa * G2[Q] / G[Q] ** 2
        G2b[Q] += d_xwa / G[Q]
        xsb[b] += d_xa
    for q in range(Q):
        Gb[q] += gz["xi_gg"][q] / n[q] - gz["xi_dw"][q] * G2[q] / G[q] ** 2
        G2b[q] += gz["xi_dw"][q] / G[q]
    Gb[Q] += -gz["xi_dw_agg"][0] * G2[Q] / G[Q] ** 2
    G2b[Q] += gz["xi_dw_agg"][0] / G[Q]
    ddb = gz["dd_w"] + np.where(valid | (st["dd_w"] > 0), xsb / rr, 0.0)
    rrb = -xsb * st["dd_w"] / rr ** 2
    npb = np.sum(rrb * st["vb"] / L ** 3)
    swb, sw2b = npb * st["sw"], -0.5 * npb
    # ---- bin sums -> correlation cells ----
    bins, agg = st["bins"], st["agg"]
    inb = bins >= 0

    def cell_grad(vals_bar, agg_bar):
        c = np.zeros(bins.size)
        c[inb] = vals_bar[bins[inb]]
        c[agg] += agg_bar
        return c

    cgg = st["cgg"]
    cggb = cell_grad(Gb[:Q], Gb[Q]) + 2.0 * cgg * cell_grad(G2b[:Q], G2b[Q])
    f_g = st["f_g"]
    # ---- cells -> f fields (real-space correlations) ----
    fgb = _sum_shift(cggb, f_g, wh, -1) + _sum_shift(cggb, f_g, wh, +1)
    wbar = np.zeros(st["x"].shape[0])
    pr, pb = st["pairs"], st["pb"]
    for b in st["f_b"]:
        cbb = cell_grad(Sb[b, :Q], Sb[b, Q])
        fbb = _sum_shift(cbb, f_g, wh, -1)            # (1/N^3) sum_r cbar(r) f_g(y - r)
        fgb += _sum_shift(cbb, st["f_b"][b], wh, +1)  # (1/N^3) sum_r cbar(r) f_b(x + r)
        rho = st["rho_b"][b]
        Qb = rho.sum()
        rhob = (N ** 3 / Qb) * (fbb - np.sum(fbb * st["f_b"][b]) / N ** 3)
        sel = np.nonzero(pb == b)[0]
        wp_bar = _gather(rhob, _node_weights(pr["mid"][sel], L, N, p.assign)) + ddb[b]
        np.add.at(wbar, pr["i"][sel], wp_bar * st["w"][pr["j"][sel]])
        np.add.at(wbar, pr["j"][sel], wp_bar * st["w"][pr["i"][sel]])
    Qg = st["rho_g"].sum()
    rhogb = (N ** 3 / Qg) * (fgb - np.sum(fgb * f_g) / N ** 3)
    wbar += _gather(rhogb, _node_weights(st["x"], L, N, p.assign))
    wbar += swb + 2.0 * st["w"] * sw2b
    return wbar
