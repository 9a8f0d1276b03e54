"""Soft HOD occupation weights and their parameter derivatives (oracle,
test-only).

Sec. 3.3, eq. hod: <n_cen> = erfc[ln(M_cut/M) / (sqrt(2) sigma)] / 2 and
<n_sat> = ((M - kappa M_cut) / M_1)^alpha (zero for M <= kappa M_cut), with
theta = (log10 M_cut, log10 M_1, sigma, alpha, kappa). A central candidate
carries <n_cen>; each of the K satellite candidates of a halo carries
<n_sat> / K. Derivatives are written out by hand; ``grad_theta`` chains the
weight gradient of ``adjoint.grad_weights`` to theta.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc


def weights(theta, mass, kind, kh):
    t0, t1, sig, alpha, kappa = [float(v) for v in theta]
    mcut, m1 = 10.0 ** t0, 10.0 ** t1
    M = np.asarray(mass, dtype=np.float64)
    u = np.log(mcut / M) / (math.sqrt(2.0) * sig)
    cen = 0.5 * erfc(u)
    x = (M - kappa * mcut) / m1
    sat = np.where(x > 0, np.clip(x, 1e-300, None) ** alpha, 0.0) / np.asarray(kh, np.float64)
    return np.where(np.asarray(kind) == 0, cen, sat)


def dweights(theta, mass, kind, kh):
    """[n, 5] derivatives of ``weights`` with respect to theta."""
    t0, t1, sig, alpha, kappa = [float(v) for v in theta]
    ln10 = math.log(10.0)
    mcut, m1 = 10.0 ** t0, 10.0 ** t1
    M = np.asarray(mass, dtype=np.float64)
    K = np.asarray(kh, np.float64)
    d = np.zeros((M.size, 5))
    u = np.log(mcut / M) / (math.sqrt(2.0) * sig)
    dcu = -np.exp(-u * u) / math.sqrt(math.pi)        # d erfc(u)/2 / du
    c = np.asarray(kind) == 0
    d[c, 0] = dcu[c] * ln10 / (math.sqrt(2.0) * sig)
    d[c, 2] = dcu[c] * (-u[c] / sig)
    x = (M - kappa * mcut) / m1
    s = (~c) & (x > 0)
    xa = x[s] ** alpha
    dx = alpha * xa / x[s] / K[s]
    d[s, 0] = dx * (-kappa * mcut * ln10 / m1)
    d[s, 1] = dx * (-x[s] * ln10)
    d[s, 3] = xa * np.log(x[s]) / K[s]
    d[s, 4] = dx * (-mcut / m1)
    return d


def d2weights(theta, mass, kind, kh):
    """[n, 5, 5] second derivatives of ``weights`` with respect to theta
    (symmetric), from the chain rule through the same closed forms.

    Central: v = erfc(u)/2 with g = dv/du = -exp(-u^2)/sqrt(pi), dg/du =
    -2 u g; u depends on log10 M_cut (u_0 = ln10 / (sqrt(2) sigma)) and
    sigma (u_2 = -u / sigma), with u_00 = 0, u_02 = -u_0 / sigma and
    u_22 = 2 u / sigma^2, so v_jk = -2 u g u_j u_k + g u_jk.
    Satellite (x > 0): v = x^alpha / K, x = (M - kappa M_cut) / M_1, with
    x_0 = -kappa M_cut ln10 / M_1, x_1 = -x ln10, x_4 = -M_cut / M_1 and
    x_00 = x_0 ln10, x_01 = -x_0 ln10, x_04 = x_4 ln10, x_11 = x ln10^2,
    x_14 = -x_4 ln10, x_44 = 0; v_jk = (f_xx x_j x_k + f_x x_jk) / K for
    j, k in (0, 1, 4), v_j3 = f_xa x_j / K and v_33 = f_aa / K with
    f = x^alpha, f_x = alpha x^(alpha-1), f_xx = alpha (alpha-1) x^(alpha-2),
    f_xa = x^(alpha-1) (1 + alpha ln x), f_aa = x^alpha (ln x)^2."""
    t0, t1, sig, alpha, kappa = [float(v) for v in theta]
    ln10 = math.log(10.0)
    mcut, m1 = 10.0 ** t0, 10.0 ** t1
    M = np.asarray(mass, dtype=np.float64)
    K = np.asarray(kh, np.float64)
    h = np.zeros((M.size, 5, 5))
    c = np.asarray(kind) == 0
    u = np.log(mcut / M[c]) / (math.sqrt(2.0) * sig)
    g = -np.exp(-u * u) / math.sqrt(math.pi)
    gu = -2.0 * u * g
    u0 = ln10 / (math.sqrt(2.0) * sig)
    u2 = -u / sig
    h[c, 0, 0] = gu * u0 * u0
    h[c, 0, 2] = h[c, 2, 0] = gu * u0 * u2 + g * (-u0 / sig)
    h[c, 2, 2] = gu * u2 * u2 + g * (2.0 * u / (sig * sig))
    x = (M - kappa * mcut) / m1
    s = (~c) & (x > 0)
    xs = x[s]
    Ks = K[s]
    fx = alpha * xs ** (alpha - 1.0)
    fxx = alpha * (alpha - 1.0) * xs ** (alpha - 2.0)
    fxa = xs ** (alpha - 1.0) * (1.0 + alpha * np.log(xs))
    faa = xs ** alpha * np.log(xs) ** 2
    x0 = -kappa * mcut * ln10 / m1
    x4 = -mcut / m1
    xj = {0: np.full(xs.size, x0), 1: -xs * ln10, 4: np.full(xs.size, x4)}
    xjk = {(0, 0): np.full(xs.size, x0 * ln10), (0, 1): np.full(xs.size, -x0 * ln10),
           (0, 4): np.full(xs.size, x4 * ln10), (1, 1): xs * ln10 * ln10,
           (1, 4): np.full(xs.size, -x4 * ln10), (4, 4): np.zeros(xs.size)}
    for (j, k), v in xjk.items():
        h[s, j, k] = h[s, k, j] = (fxx * xj[j] * xj[k] + fx * v) / Ks
    for j in (0, 1, 4):
        h[s, j, 3] = h[s, 3, j] = fxa * xj[j] / Ks
    h[s, 3, 3] = faa / Ks
    return h


def grad_theta(theta, mass, kind, kh, wbar):
    return dweights(theta, mass, kind, kh).T @ np.asarray(wbar, np.float64)
