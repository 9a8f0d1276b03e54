"""Mesh cross-correlation, (r, mu_r) binning and the ratio outputs (oracle).

Sec. 2.1, eq. bpg_initial: b_pg is a W-weighted k-space average of
Re(delta_g^* delta_p) over one of delta_g^* delta_g; eq. bpg_intermediate
shows it equals a real-space sum of (W * delta_g) at the pair positions, W
even and real. Taking W as the indicator of one (r, mu_r) shell makes both
numerator and denominator the shell sums of the mesh correlation

    C_ab(r) = (1/N^3) sum_x delta_b(x) delta_a(x + r),

computed here as N^-6 * IDFT[F_a conj(F_b)] with the k = 0 mode set to zero
(Sec. 2.1: the DC term does not contribute). delta = rho / rho_bar - 1 with
rho_bar the mesh mean (eq. delta_pi_x).

Outputs (Sec. 2.2): xi_pg = mean of C_pg over a bin, xi_gg likewise,
b_pg = xi_pg / xi_gg; xi(d_w) = sum C_gg^2 / sum C_gg over the bin (eq.
xi_dw with the measured xi_gg as the 2PCF and the bin indicator as W);
Q_eff from eq. Qeff_notsq and the strict-squeezed Q_eff_sq from eq. Qeff,
with xi(d_p) = xi(s, mu) from the pair counts.
"""
from __future__ import annotations

import math

import numpy as np

from . import dft

TWO32 = float(2 ** 32)


def window_half(N, L, r_max):
    """Half-size w of the offset window: every |r| < r_max has |r_i| <= w."""
    dx = L / N
    w = int(math.ceil(r_max / dx))
    if 2 * w + 1 > N or w >= N // 2:
        raise ValueError("r_max must be below L/2")
    return w


def cell_bins(N, L, r_edges, n_mur, r_perp_cut, w):
    """Bin of every offset in the window cube [-w, w]^3 (z, y, x order).

    Offsets (a, b, c) along (x, y, z); R2 = a^2 + b^2 + c^2 (integer),
    r^2 = R2 * dx^2 tested against the squared edges, mu_r = |c| / sqrt(R2)
    (0 at R2 = 0), mu_r bin = min(n_mur - 1, floor(n_mur * mu_r)).
    Returns (bin [W^3] int64, -1 outside every bin; agg [W^3] bool).
    """
    dx = L / N
    dx2 = dx * dx
    e = np.asarray(r_edges, dtype=np.float64)
    e2 = e * e
    o = np.arange(-w, w + 1, dtype=np.int64)
    c = o[:, None, None]
    b = o[None, :, None]
    a = o[None, None, :]
    R2 = (a * a + b * b + c * c).astype(np.int64)
    r2 = R2.astype(np.float64) * dx2
    k = np.searchsorted(e2, r2.reshape(-1), side="right").reshape(r2.shape) - 1
    inr = (k >= 0) & (k < len(e2) - 1)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(R2 > 0, np.abs(c) / np.sqrt(R2.astype(np.float64)), 0.0)
    m = np.minimum(n_mur - 1, np.floor(n_mur * mu).astype(np.int64))
    bins = np.where(inr, k * n_mur + m, -1)
    agg = inr.copy()
    if r_perp_cut > 0.0:
        rp2 = (a * a + b * b).astype(np.float64) * dx2
        agg &= np.broadcast_to(rp2 >= r_perp_cut * r_perp_cut, agg.shape)
    return bins.reshape(-1), agg.reshape(-1)


def field(mesh_q):
    """f = rho / rho_bar as FP64 (the -1 of delta only touches k = 0)."""
    q = np.asarray(mesh_q)
    N3 = q.size
    Q = int(q.sum())
    if Q == 0:
        return None
    return q.astype(np.float64) * (float(N3) / float(Q))


def correlate_mesh(qa, qb):
    """C_ab(r) on the full offset grid [N, N, N] (z, y, x), FP64."""
    fa = field(qa)
    fb = field(qb)
    if fa is None or fb is None:
        return None
    N = qa.shape[0]
    Fa = dft.dft3(fa, -1)
    Fb = Fa if qa is qb else dft.dft3(fb, -1)
    P = Fa * np.conj(Fb)
    P[0, 0, 0] = 0.0
    C = dft.dft3(P, +1).real / float(N) ** 6
    return C


def window_of(C, w):
    """Extract offsets [-w, w]^3 from a full offset grid, flat [W^3]."""
    N = C.shape[0]
    o = np.arange(-w, w + 1) % N
    return C[np.ix_(o, o, o)].reshape(-1)


def bin_sums(cwin, bins, agg, n_bins):
    """Per-bin sum C, sum C^2, cell count, and the same over the aggregate."""
    sel = bins >= 0
    s1 = np.bincount(bins[sel], weights=cwin[sel], minlength=n_bins)
    s2 = np.bincount(bins[sel], weights=cwin[sel] ** 2, minlength=n_bins)
    n = np.bincount(bins[sel], minlength=n_bins).astype(np.int64)
    a1 = float(np.sum(cwin[agg]))
    a2 = float(np.sum(cwin[agg] ** 2))
    return s1, s2, n, a1, a2, int(np.count_nonzero(agg))


def q_eff_notsq(b, xi_p, xi_w):
    """eq. Qeff_notsq: ((1+xi)b - 2 - xi_w/(2 xi)) / (2 xi + 1.5 xi_w)."""
    return ((1.0 + xi_p) * b - 2.0 - xi_w / (2.0 * xi_p)) / (2.0 * xi_p + 1.5 * xi_w)


def q_eff_sq(b, xi_p):
    """eq. Qeff: ((1+xi)b - 2) / (2 xi)."""
    return ((1.0 + xi_p) * b - 2.0) / (2.0 * xi_p)


def b_pg_notsq(q, xi_p, xi_w):
    """eq. bpg_notsq_dw: b_pg from Q_eff, xi(d_p) and xi(d_w)."""
    return (2.0 + xi_w / (2.0 * xi_p) + q * (2.0 * xi_p + 1.5 * xi_w)) / (1.0 + xi_p)


def ratios(sp, sg, xi_ss_b):
    """All outputs from pair and galaxy bin sums.

    sp: dict of per-pair-bin arrays s1 [nb, nr], a1 [nb]; sg: s1, s2, n, a1,
    a2, na for the galaxy auto-correlation; xi_ss_b: xi(s, mu) per pair bin.
    """
    with np.errstate(invalid="ignore", divide="ignore"):
        n = sg["n"].astype(np.float64)
        nn = np.where(sg["n"] > 0, n, np.nan)
        xi_gg = sg["s1"] / nn
        xi_pg = sp["s1"] / nn[None, :]
        b = xi_pg / xi_gg[None, :]
        xi_dw = sg["s2"] / sg["s1"]
        xs = xi_ss_b[:, None]
        out = {
            "xi_gg": xi_gg,
            "xi_pg": xi_pg,
            "b_pg": b,
            "xi_dw": xi_dw,
            "q_eff": q_eff_notsq(b, xs, xi_dw[None, :]),
            "q_eff_sq": q_eff_sq(b, xs),
        }
        b_agg = sp["a1"] / sg["a1"]
        xi_dw_agg = sg["a2"] / sg["a1"]
        out["b_pg_agg"] = b_agg
        out["xi_dw_agg"] = xi_dw_agg
        out["q_eff_agg"] = q_eff_notsq(b_agg, xi_ss_b, xi_dw_agg)
    return out
