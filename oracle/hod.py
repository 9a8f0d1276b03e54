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


def grad_theta(theta, mass, kind, kh, wbar):
    return dweights(theta, mass, kind, kh).T @ np.asarray(wbar, np.float64)
