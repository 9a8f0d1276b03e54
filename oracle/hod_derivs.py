"""Exact first and second derivatives of the pair-count statistics with
respect to the HOD parameters, and the emulators built on them (oracle,
test-only).

Sec. 5 (eqs. 2pf_emulate_1st and 2pf_emulate_2nd) models the projected
2PCF w(d_perp) around a design HOD by a Taylor expansion in the HOD
parameters, whose first and second derivatives the paper solves for from 14
separate evaluations. With the soft occupation weights of eq. hod on fixed
candidates, the pair counts DD_b (the sum over the pairs of bin b of
w_i w_j, Sec. 3.4) and the pair normalisation R = ((sum w)^2 - sum w^2) / 2
are polynomials in the weights, so their derivatives in theta follow exactly
from dw/dtheta and d2w/dtheta2 by the product rule. Then
xi_b = DD_b / (R V_b / L^3) - 1 (eq. 2PCF_d_collapsed) by the quotient rule,
and w(d_perp)_i = sum_m 2 (l_hi - l_lo) xi_{i,m} (eq.
2PCF_los_integrated_explicit, the d_par bins of one d_perp bin) by
linearity. All sums are FP64 products of the weights (no Q32.32 rounding).

Reading of eq. 2pf_emulate_2nd: the paper's sum runs over k >= j with a
factor 1/2; with the exact second derivatives H_jk that expansion is the
Taylor series when its off-diagonal coefficients are 2 H_jk, so
``emulate`` evaluates w0 + J dp + dp^T H dp / 2 (H symmetric).
"""
from __future__ import annotations

import numpy as np

from . import pairs as op


def pair_sums(pairs, w, dw, d2w, n_bins):
    """DD [P], dDD [P, T] and d2DD [P, T, T] over the pairs of each bin
    (pairs: input indices 'i', 'j' and flat bin index 'bin'):
    DD = sum w_i w_j; d/dt_j = sum (w_i' w_j + w_i w_j'); second
    derivatives sum (w_i'' w_j + w_i' w_j'^T + w_j' w_i'^T + w_i w_j'')."""
    w = np.asarray(w, np.float64)
    i, j, b = pairs["i"], pairs["j"], pairs["bin"]
    T = dw.shape[1]
    DD = np.bincount(b, weights=w[i] * w[j], minlength=n_bins)
    dDD = np.zeros((n_bins, T))
    d2DD = np.zeros((n_bins, T, T))
    for a in range(T):
        dDD[:, a] = np.bincount(b, weights=dw[i, a] * w[j] + w[i] * dw[j, a], minlength=n_bins)
        for c in range(T):
            v = (d2w[i, a, c] * w[j] + dw[i, a] * dw[j, c] + dw[i, c] * dw[j, a]
                 + w[i] * d2w[j, a, c])
            d2DD[:, a, c] = np.bincount(b, weights=v, minlength=n_bins)
    return DD, dDD, d2DD


def norm_sums(w, dw, d2w):
    """R = ((sum w)^2 - sum w^2) / 2 with its first and second derivatives."""
    w = np.asarray(w, np.float64)
    S1, dS1, d2S1 = w.sum(), dw.sum(axis=0), d2w.sum(axis=0)
    S2 = np.sum(w * w)
    dS2 = 2.0 * (w @ dw)
    d2S2 = 2.0 * (dw.T @ dw + np.einsum("n,njk->jk", w, d2w))
    R = 0.5 * (S1 * S1 - S2)
    dR = S1 * dS1 - 0.5 * dS2
    d2R = np.outer(dS1, dS1) + S1 * d2S1 - 0.5 * d2S2
    return R, dR, d2R


def xi_derivs(DD, dDD, d2DD, R, dR, d2R, vol, L):
    """xi_b = DD_b / E_b - 1 with E_b = R V_b / L^3 (q = DD / E):
    dq_j = (dDD_j - q dE_j) / E and
    d2q_jk = (d2DD_jk - dq_j dE_k - dq_k dE_j - q d2E_jk) / E."""
    c = np.asarray(vol, np.float64) / L ** 3
    E = R * c
    dE = c[:, None] * dR[None, :]
    d2E = c[:, None, None] * d2R[None, :, :]
    q = DD / E
    dq = (dDD - q[:, None] * dE) / E[:, None]
    d2q = (d2DD - dq[:, :, None] * dE[:, None, :] - dq[:, None, :] * dE[:, :, None]
           - q[:, None, None] * d2E) / E[:, None, None]
    return q - 1.0, dq, d2q


def derivs(pos, w, dw, d2w, L, s_edges, n_mu, par_edges=None):
    """xi per pair bin and, on the (d_perp, d_par) grid, w(d_perp), each with
    its first [., T] and second [., T, T] derivatives in the parameters."""
    pr = op.find_pairs(pos, None, L, s_edges, n_mu, par_edges=par_edges)
    n_s = len(s_edges) - 1
    P = n_s * n_mu
    pr = dict(pr)
    pr["bin"] = pr["sbin"] * n_mu + pr["mubin"]
    DD, dDD, d2DD = pair_sums(pr, w, dw, d2w, P)
    R, dR, d2R = norm_sums(w, dw, d2w)
    vol = op.pair_volumes(s_edges, n_mu, par_edges)
    xi, dxi, d2xi = xi_derivs(DD, dDD, d2DD, R, dR, d2R, vol, L)
    out = {"xi": xi, "dxi": dxi, "d2xi": d2xi, "dd": DD}
    if par_edges is not None:
        pe = np.asarray(par_edges, np.float64)
        cm = 2.0 * (pe[1:] - pe[:-1])
        T = dw.shape[1]
        out["w_perp"] = xi.reshape(n_s, n_mu) @ cm
        out["dw_perp"] = np.einsum("smt,m->st", dxi.reshape(n_s, n_mu, T), cm)
        out["d2w_perp"] = np.einsum("smtu,m->stu", d2xi.reshape(n_s, n_mu, T, T), cm)
    return out


def emulate(v0, J, H, dp):
    """First-order (H None, eq. 2pf_emulate_1st) or second-order (eq.
    2pf_emulate_2nd) prediction at parameter offsets dp."""
    dp = np.asarray(dp, np.float64)
    out = v0 + J @ dp
    if H is not None:
        out = out + 0.5 * np.einsum("itu,t,u->i", H, dp, dp)
    return out
