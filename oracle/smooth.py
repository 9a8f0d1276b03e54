"""The paper's own estimator with the smooth Gauss-sigmoid W (oracle, FP64,
test-only).

Sec. 2.1, eq. bpg_final: b_pg = [(1/n_p) sum_i (W * delta_g)(x_p,i)] /
[(1/n_g) sum_j (W * delta_g)(x_g,j)]: one convolution of the galaxy
overdensity with W, evaluated at the pair midpoints of each (s, mu) bin and at
the galaxies. Sec. 3.6, eq. weighting: W(r_perp, r_par) = N sigmoid(s0 (r_perp
- r_s)) exp(-(r_perp^2 + r_par^2) / (2 sigma^2)) for r_perp >= r_cut and 0
inside that cylinder around the line of sight (z); the normalisation N
cancels and is 1 here. Q_eff follows eq. Qeff_notsq with xi(d_p) = DD/RR - 1
of the pair bin and xi(d_w) from eq. xi_dw, sum_r W C_gg^2 / sum_r W C_gg over
the mesh offsets, C_gg the measured galaxy auto-correlation.

Steps, in the paper's order: mass assignment of the galaxies (mesh.deposit),
f = rho / rho_bar, delta_g = f - 1 (its k = 0 mode), the convolution by DFT
(the oracle's own dft3: G = N^-3 IDFT[DFT(W) DFT(f)] with k = 0 set to zero,
i.e. G(x) = sum_r W(r) delta_g(x - r)), interpolation of G at points with
the assignment weights, weighted means (pair weight w_i w_j, galaxy weight
w_j; a mean over the points times the volume is the sum over points divided
by the number density), their ratio, and eq. Qeff_notsq.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import correlate as oc
from . import dft
from . import mesh as om
from . import pairs as op


@dataclasses.dataclass(frozen=True)
class WParams:
    sigma: float      # Mpc/h
    r_s: float        # Mpc/h
    s0: float         # h/Mpc
    r_cut: float      # Mpc/h


# Table tab:weightings: d_p,max = 10 Mpc (real space) and 30 Mpc (redshift space)
W_DP10 = WParams(30.0, 20.0, 0.8, 10.0)
W_DP30 = WParams(50.0, 35.0, 0.5, 20.0)


def weight(r_perp, r_par, prm: WParams):
    """eq. weighting with N = 1."""
    r_perp = np.asarray(r_perp, dtype=np.float64)
    r_par = np.asarray(r_par, dtype=np.float64)
    sig = 1.0 / (1.0 + np.exp(-prm.s0 * (r_perp - prm.r_s)))
    g = np.exp(-0.5 * (r_perp * r_perp + r_par * r_par) / (prm.sigma * prm.sigma))
    return np.where(r_perp >= prm.r_cut, sig * g, 0.0)


def offsets(N, L):
    """Signed mesh offsets along one axis: i for i <= N/2, i - N above."""
    i = np.arange(N)
    return np.where(i <= N // 2, i, i - N) * (L / N)


def weight_mesh(L, N, prm: WParams):
    """W at every mesh offset r (minimum image), [z, y, x]; LOS = z."""
    o = offsets(N, L)
    rz, ry, rx = np.meshgrid(o, o, o, indexing="ij")
    return weight(np.sqrt(rx * rx + ry * ry), np.abs(rz), prm)


def convolve(f, Wm):
    """G(x) = sum_r W(r) (f - <f>)(x - r) by the oracle's DFT, k = 0 zeroed."""
    N = f.shape[0]
    P = dft.dft3(np.asarray(f, dtype=np.complex128), -1) * dft.dft3(np.asarray(Wm, dtype=np.complex128), -1)
    P[0, 0, 0] = 0.0
    return dft.dft3(P, +1).real / float(N) ** 3


def interpolate(G, points, L, N, assign):
    """G at points with the assignment weights (unrounded)."""
    zs, ys, xs, k = om.node_weights(points, L, N, assign)
    return np.sum(k * G[zs, ys, xs], axis=1)


def ratio_of_means(gp, wp, gg, wg):
    """(sum wp gp / sum wp) / (sum wg gg / sum wg): eq. bpg_final."""
    return (np.sum(wp * gp) / np.sum(wp)) / (np.sum(wg * gg) / np.sum(wg))


def xi_dw(C, Wm):
    """eq. xi_dw on the mesh offsets: sum W C^2 / sum W C."""
    return float(np.sum(Wm * C * C) / np.sum(Wm * C))


def estimate(p, prm: WParams, pos, vel=None, w=None):
    """The smooth-W estimator for every (s, mu) pair bin of Params p (the
    correlation bins of p are not used). Returns dd, ddq, xi_ss, num (the
    weighted mean of G over each bin's pair midpoints, NaN for an empty bin),
    den (over the galaxies), b_pg = num / den, xi_dw, q_eff."""
    L, N = p.box_L, p.mesh_n
    n_s = len(p.s_edges) - 1
    n_pb = n_s * p.n_mu
    x = op.transform_positions(pos, vel, L, p.rsd_factor)
    wt = np.ones(x.shape[0]) if w is None else np.asarray(w, dtype=np.float32).astype(np.float64)
    pr = op.find_pairs(x, w, L, p.s_edges, p.n_mu, par_edges=p.par_edges)
    dd, ddq = op.pair_counts(pr, n_s, p.n_mu)
    xi_ss, _ = op.xi_ss(ddq, w, x.shape[0], L, p.s_edges, p.n_mu, p.par_edges)
    mq = om.deposit(x, wt, L, N, p.assign)
    f = oc.field(mq)
    Wm = weight_mesh(L, N, prm)
    G = convolve(f, Wm)
    gg = interpolate(G, x, L, N, p.assign)
    den = float(np.sum(wt * gg) / np.sum(wt))
    num = np.full(n_pb, np.nan)
    pb = pr["sbin"] * p.n_mu + pr["mubin"]
    if pr["mid"].shape[0]:
        gp = interpolate(G, pr["mid"], L, N, p.assign)
        for b in range(n_pb):
            sel = pb == b
            if np.any(sel):
                num[b] = np.sum(pr["weight"][sel] * gp[sel]) / np.sum(pr["weight"][sel])
    C = oc.correlate_mesh(mq, mq)
    xdw = xi_dw(C, Wm)
    b = num / den
    with np.errstate(invalid="ignore", divide="ignore"):
        q = oc.q_eff_notsq(b, xi_ss, xdw)
    return {"dd": dd, "ddq": ddq, "xi_ss": xi_ss, "num": num, "den": den, "b_pg": b,
            "xi_dw": xdw, "q_eff": q, "G": G, "W": Wm}


__all__ = ["WParams", "W_DP10", "W_DP30", "weight", "offsets", "weight_mesh", "convolve",
           "interpolate", "ratio_of_means", "xi_dw", "estimate"]
