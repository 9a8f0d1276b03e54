"""Positions, pair enumeration and pair counts (oracle, FP64, test-only).

Follows:
* Sec. 3.2, eq. RSD: the line-of-sight coordinate (z here) of each galaxy is
  shifted by its LOS velocity over H(z); ``rsd_factor`` carries 1/H in
  Mpc/h per km/s.
* Sec. 2.1 (eq. delta_pi_x and the text before it): a pair is an object at
  the middle of its two galaxies; in the periodic box that is the
  minimum-image midpoint.
* Sec. 3.3 (pair catalogue): every pair closer than the maximum separation is
  kept, so a close triplet gives three pairs.
* Sec. 3.4, eq. 2PCF_d_collapsed: xi = (pair count) / (expected count) - 1,
  with the expected count written exactly as ((sum w)^2 - sum w^2)/2 times
  the bin volume over the box volume.
* Sec. 3.4, eq. 2PCF_los_integrated_explicit and the (d_perp, d_par) maps of
  Sec. 5: on the pair grid d_perp = sqrt(dx^2 + dy^2) and d_par = |dz| (line
  of sight z) are binned instead of (s, mu); a grid cell's volume is the
  annulus pi (p_hi^2 - p_lo^2) times 2 (l_hi - l_lo) (both signs of d_par),
  and w(d_perp) is the integral of xi over d_par, sum over the d_par bins of
  2 (l_hi - l_lo) xi(d_perp, d_par), with d_par,max the last d_par edge.

All arithmetic is IEEE FP64 with one rounding per operation (numpy does not
contract a*b+c), in the order written below.
"""
from __future__ import annotations

import math

import numpy as np

TWO32 = float(2 ** 32)


def wrap(x: np.ndarray, L: float) -> np.ndarray:
    """x - L*floor(x/L), and a result equal to L (from rounding) becomes 0."""
    y = x - L * np.floor(x / L)
    return np.where(y >= L, 0.0, y)


def transform_positions(pos, vel, L, rsd_factor):
    """Wrap into [0, L); with RSD, z <- wrap(z + rsd_factor * v_z)."""
    p = wrap(np.asarray(pos, dtype=np.float64), L)
    if rsd_factor != 0.0 and vel is not None:
        v = np.asarray(vel, dtype=np.float32).astype(np.float64)
        p[:, 2] = wrap(p[:, 2] + rsd_factor * v[:, 2], L)
    return p


def min_image(d: np.ndarray, L: float) -> np.ndarray:
    """One correction by +-L for separations of already-wrapped positions."""
    h = 0.5 * L
    d = np.where(d > h, d - L, d)
    return np.where(d < -h, d + L, d)


def _bin_pairs(d, s_edges, n_mu):
    """(s bin, mu bin, valid) for separation vectors d [m, 3]."""
    e = np.asarray(s_edges, dtype=np.float64)
    e2 = e * e
    s2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    k = np.searchsorted(e2, s2, side="right") - 1
    valid = (k >= 0) & (k < len(e2) - 1)
    s = np.sqrt(s2)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(s > 0.0, np.abs(d[:, 2]) / s, 0.0)
    m = np.minimum(n_mu - 1, np.floor(n_mu * mu).astype(np.int64))
    return k, m, valid


def _bin_pairs_grid(d, perp_edges, par_edges):
    """(d_perp bin, d_par bin, valid) for separation vectors d [m, 3]:
    d_perp^2 = dx^2 + dy^2 against the squared d_perp edges, d_par = |dz|
    against the d_par edges, bins half-open."""
    e = np.asarray(perp_edges, dtype=np.float64)
    e2 = e * e
    pe = np.asarray(par_edges, dtype=np.float64)
    p2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
    l = np.abs(d[:, 2])
    k = np.searchsorted(e2, p2, side="right") - 1
    m = np.searchsorted(pe, l, side="right") - 1
    valid = (k >= 0) & (k < len(e2) - 1) & (m >= 0) & (m < len(pe) - 1)
    return k, m, valid


def max_separation(s_edges, par_edges=None):
    """The largest pair separation a binning keeps: s_max, or on the grid
    the corner sqrt(d_perp,max^2 + d_par,max^2) of its cylinder."""
    if par_edges is None:
        return float(s_edges[-1])
    return math.sqrt(float(s_edges[-1]) ** 2 + float(par_edges[-1]) ** 2)


def _bin(d, s_edges, n_mu, par_edges):
    if par_edges is None:
        return _bin_pairs(d, s_edges, n_mu)
    return _bin_pairs_grid(d, s_edges, par_edges)


def find_pairs(pos, w, L, s_edges, n_mu, chunk=2048, par_edges=None):
    """All unordered pairs i < j with s in [s_edges[0], s_edges[-1]) (with
    par_edges: d_perp in [s_edges[0], s_edges[-1]) and d_par in
    [par_edges[0], par_edges[-1]), bins 'sbin' = d_perp bin, 'mubin' = d_par bin).

    Returns a dict of arrays over pairs: i, j (input indices), sbin, mubin,
    mid [m, 3] (wrapped midpoint x_i + d/2, d = min-image x_j - x_i) and
    weight w_i * w_j (FP64).
    """
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    wt = None if w is None else np.asarray(w, dtype=np.float32).astype(np.float64)
    out = {k: [] for k in ("i", "j", "sbin", "mubin", "mid", "weight")}
    for a0 in range(0, n, chunk):
        a1 = min(n, a0 + chunk)
        ia = np.arange(a0, a1)
        for b0 in range(a0, n, chunk):
            b1 = min(n, b0 + chunk)
            jb = np.arange(b0, b1)
            I, J = np.meshgrid(ia, jb, indexing="ij")
            keep = J > I
            I = I[keep]
            J = J[keep]
            d = min_image(pos[J] - pos[I], L)
            k, m, valid = _bin(d, s_edges, n_mu, par_edges)
            I, J, d, k, m = I[valid], J[valid], d[valid], k[valid], m[valid]
            mid = wrap(pos[I] + 0.5 * d, L)
            out["i"].append(I)
            out["j"].append(J)
            out["sbin"].append(k)
            out["mubin"].append(m)
            out["mid"].append(mid)
            out["weight"].append(np.ones(I.size) if wt is None else wt[I] * wt[J])
    res = {k: (np.concatenate(v) if v else np.zeros(0)) for k, v in out.items()}
    if res["mid"].size == 0:
        res["mid"] = np.zeros((0, 3))
    for k in ("i", "j", "sbin", "mubin"):
        res[k] = res[k].astype(np.int64)
    return res


def pair_counts(pairs, n_s, n_mu):
    """DD per (s, mu) bin: integer count and exact Q32.32 weight sum."""
    b = pairs["sbin"] * n_mu + pairs["mubin"]
    count = np.bincount(b, minlength=n_s * n_mu).astype(np.int64)
    q = np.rint(pairs["weight"] * TWO32).astype(np.int64)
    ddq = np.zeros(n_s * n_mu, dtype=np.int64)
    np.add.at(ddq, b, q)
    return count, ddq


def pair_volumes(s_edges, n_mu, par_edges=None):
    """Volume of every pair bin (index s bin * n_mu + mu bin): the shell
    (4 pi / 3)(s_hi^3 - s_lo^3) / n_mu, or on the grid the annulus
    pi (p_hi^2 - p_lo^2) times 2 (l_hi - l_lo)."""
    e = np.asarray(s_edges, dtype=np.float64)
    if par_edges is None:
        vshell = (4.0 * math.pi / 3.0) * (e[1:] ** 3 - e[:-1] ** 3)
        return np.repeat(vshell / n_mu, n_mu)
    pe = np.asarray(par_edges, dtype=np.float64)
    ann = math.pi * (e[1:] ** 2 - e[:-1] ** 2)
    return (ann[:, None] * (2.0 * (pe[1:] - pe[:-1]))[None, :]).reshape(-1)


def w_perp(xi, par_edges):
    """w(d_perp) = sum over the d_par bins of 2 (l_hi - l_lo) xi(d_perp, d_par)
    (eq. 2PCF_los_integrated_explicit, first line, on the grid); xi is
    [n_perp * n_par] in bin order."""
    pe = np.asarray(par_edges, dtype=np.float64)
    n_par = len(pe) - 1
    x = np.asarray(xi, dtype=np.float64).reshape(-1, n_par)
    return np.sum(x * (2.0 * (pe[1:] - pe[:-1]))[None, :], axis=1)


def xi_ss(ddq, w, n_gal, L, s_edges, n_mu, par_edges=None):
    """xi(s, mu) = DD / RR - 1 (eq. 2PCF_d_collapsed, exact pair normalisation).

    RR = ((sum w)^2 - sum w^2) / 2 * V_bin / L^3 with V_bin from pair_volumes
    ((s, mu) shells or (d_perp, d_par) cells).
    """
    if w is None:
        sw = float(n_gal)
        sw2 = float(n_gal)
    else:
        wd = np.asarray(w, dtype=np.float32).astype(np.float64)
        sw = float(np.sum(wd))
        sw2 = float(np.sum(wd * wd))
    npairs = 0.5 * (sw * sw - sw2)
    rr = npairs * pair_volumes(s_edges, n_mu, par_edges) / L ** 3
    dd = ddq.astype(np.float64) / TWO32
    with np.errstate(invalid="ignore", divide="ignore"):
        return dd / rr - 1.0, rr


def find_pairs_kdtree(pos, w, L, s_edges, n_mu, par_edges=None):
    """find_pairs for large catalogues: the candidate pairs i < j closer than
    s_max come from scipy's periodic k-d tree (a library neighbour search,
    slightly enlarged radius); binning, midpoints and weights are then the
    same definitions as find_pairs. Output sorted by (i, j)."""
    from scipy.spatial import cKDTree
    pos = np.asarray(pos, dtype=np.float64)
    wt = None if w is None else np.asarray(w, dtype=np.float32).astype(np.float64)
    tree = cKDTree(pos, boxsize=L)
    cand = tree.query_pairs(max_separation(s_edges, par_edges) * (1.0 + 1e-9), output_type="ndarray")
    if cand.size == 0:
        cand = np.zeros((0, 2), dtype=np.int64)
    I = np.minimum(cand[:, 0], cand[:, 1]).astype(np.int64)
    J = np.maximum(cand[:, 0], cand[:, 1]).astype(np.int64)
    o = np.lexsort((J, I))
    I, J = I[o], J[o]
    d = min_image(pos[J] - pos[I], L)
    k, m, valid = _bin(d, s_edges, n_mu, par_edges)
    I, J, d, k, m = I[valid], J[valid], d[valid], k[valid], m[valid]
    return {"i": I, "j": J, "sbin": k.astype(np.int64), "mubin": m.astype(np.int64),
            "mid": wrap(pos[I] + 0.5 * d, L),
            "weight": np.ones(I.size) if wt is None else wt[I] * wt[J]}
