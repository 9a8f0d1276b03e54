"""The whole forward path for one catalogue (oracle, FP64, test-only).

Steps in the paper's order: positions (Sec. 3.2, eq. RSD) -> pairs binned by
(s, mu) (or on the (d_perp, d_par) grid) with midpoints (Sec. 2.1, Sec. 3.3)
-> pair counts and xi(s, mu) (Sec. 3.4; on the grid also w(d_perp)) -> mass assignment of pair midpoints per bin and of galaxies
(Sec. 3.5) -> cross-correlation with the galaxy mesh and binning by
(r, mu_r) (Sec. 2.1, eqs. bpg_initial / bpg_intermediate with a shell W) ->
b_pg, xi(d_w), Q_eff (Sec. 2.2, eqs. xi_dw, Qeff, Qeff_notsq).

``form='mesh'`` correlates through the oracle's own DFT; ``form='direct'``
sums over (pair, galaxy) corner combinations. ``pair_bins`` restricts the
pair-galaxy correlation to a subset of (s, mu) bins (the rest are NaN).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import correlate as oc
from . import direct as od
from . import mesh as om
from . import pairs as op


@dataclasses.dataclass
class Params:
    box_L: float
    mesh_n: int
    assign: int
    s_edges: tuple
    n_mu: int
    r_edges: tuple
    n_mur: int
    rsd_factor: float = 0.0
    r_perp_cut: float = 0.0
    par_edges: tuple = None   # (d_perp, d_par) pair grid: s_edges are then the d_perp edges

    @classmethod
    def of(cls, wl):
        return cls(wl.box_L, wl.mesh_n, wl.assign, tuple(wl.s_edges), wl.n_mu,
                   tuple(wl.r_edges), wl.n_mur, wl.rsd_factor, wl.r_perp_cut)


def run(p: Params, pos, vel=None, w=None, form="mesh", pair_bins=None):
    L, N = p.box_L, p.mesh_n
    n_s = len(p.s_edges) - 1
    n_pb = n_s * p.n_mu
    n_r = len(p.r_edges) - 1
    n_rb = n_r * p.n_mur
    x = op.transform_positions(pos, vel, L, p.rsd_factor)
    wt = None if w is None else np.asarray(w, dtype=np.float32).astype(np.float64)
    pr = op.find_pairs(x, w, L, p.s_edges, p.n_mu, par_edges=p.par_edges)
    dd, ddq = op.pair_counts(pr, n_s, p.n_mu)
    xi_ss, rr = op.xi_ss(ddq, w, x.shape[0], L, p.s_edges, p.n_mu, p.par_edges)
    wh = oc.window_half(N, L, p.r_edges[-1])
    bins, agg = oc.cell_bins(N, L, p.r_edges, p.n_mur, p.r_perp_cut, wh)
    r_max = p.r_edges[-1]

    def cwin_of(pts_a, w_a, mesh_a, same):
        if form == "mesh":
            if same:
                C = oc.correlate_mesh(mesh_g, mesh_g)
            else:
                C = oc.correlate_mesh(mesh_a, mesh_g)
            return None if C is None else oc.window_of(C, wh)
        return od.window_C(pts_a, w_a, x, wt, L, N, p.assign, wh, r_max)

    mesh_g = om.deposit(x, wt, L, N, p.assign) if form == "mesh" else None
    cg = cwin_of(x, wt, None, True)
    s1, s2, n, a1, a2, na = oc.bin_sums(cg, bins, agg, n_rb)
    sg = {"s1": s1, "s2": s2, "n": n, "a1": a1, "a2": a2, "na": na}
    sp1 = np.full((n_pb, n_rb), np.nan)
    spa = np.full(n_pb, np.nan)
    pb = pr["sbin"] * p.n_mu + pr["mubin"]
    todo = range(n_pb) if pair_bins is None else pair_bins
    for b in todo:
        sel = pb == b
        if not np.any(sel):
            continue
        mid = pr["mid"][sel]
        wp = pr["weight"][sel]
        mesh_p = om.deposit(mid, wp, L, N, p.assign) if form == "mesh" else None
        cp = cwin_of(mid, wp, mesh_p, False)
        if cp is None:
            continue
        t1, _, _, u1, _, _ = oc.bin_sums(cp, bins, agg, n_rb)
        sp1[b] = t1
        spa[b] = u1
    out = oc.ratios({"s1": sp1, "a1": spa}, sg, xi_ss)
    out.update({
        "dd": dd, "ddq": ddq, "xi_ss": xi_ss, "rr": rr,
        "n_cells": n, "n_cells_agg": na,
        "sum_pg": sp1, "sum_pg_agg": spa,
        "sum_gg": s1, "sum2_gg": s2, "sum_gg_agg": a1, "sum2_gg_agg": a2,
        "pairs": pr, "pos": x, "window_half": wh,
        "w_perp": (op.w_perp(xi_ss, p.par_edges) if p.par_edges is not None
                   else np.full(n_s, np.nan)),
    })
    return out
