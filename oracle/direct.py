"""The correlation summed directly over mesh-corner pairs (oracle, test-only).

For meshes rho_a, rho_b holding point weights at their assignment nodes,

    D(r) = sum_x rho_b(x) rho_a(x + r)
         = sum over (corner of an a-point, corner of a b-point) of q_a q_b
           with node(a) - node(b) = r (mod N),

and C_ab(r) = N^3 D(r) / (Q_a Q_b) - 1 with Q the mesh totals: the same
quantity as the FFT form in ``correlate`` (Sec. 2.1, eq. bpg_intermediate:
the convolution evaluated at the pair positions), but summed over triplets
(pair, galaxy) instead of Fourier modes. Only point pairs closer than
r_max + 2 sqrt(3) dx can reach a window offset below r_max, so a periodic
k-d tree (scipy) limits the candidate list; offsets of |r| >= r_max are not
accumulated. With NGP and unit weights every term is an integer.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial import cKDTree

from . import mesh as omesh

TWO32 = float(2 ** 32)


def _signed(d, N):
    d = np.mod(d, N)
    return np.where(d > N // 2, d - N, d)


def window_D(pts_a, w_a, pts_b, w_b, L, N, assign, w, r_max, chunk=1 << 16):
    """D(r) over the window [-w, w]^3 (flat, z-y-x) for offsets |r| < r_max.

    Returns (D [W^3] as FP64 in units of 2^-64, Q_a, Q_b in units of 2^-32).
    """
    pa = np.asarray(pts_a, dtype=np.float64)
    pb = np.asarray(pts_b, dtype=np.float64)
    W = 2 * w + 1
    D = np.zeros(W ** 3)
    za, ya, xa, qa, _ = omesh.corners(pa, w_a, L, N, assign)
    zb, yb, xb, qb, _ = omesh.corners(pb, w_b, L, N, assign)
    Qa = float(qa.sum()) / TWO32
    Qb = float(qb.sum()) / TWO32
    na, nb = pa.shape[0], pb.shape[0]
    ka = za.size // max(na, 1)
    kb = zb.size // max(nb, 1)
    if na == 0 or nb == 0:
        return D, Qa, Qb
    dx = L / N
    rq = r_max + 2.0 * math.sqrt(3.0) * dx * 1.0001
    ta = cKDTree(pa, boxsize=L)
    tb = cKDTree(pb, boxsize=L)
    # 'ndarray' output keeps zero-distance pairs (including i == j).
    sm = ta.sparse_distance_matrix(tb, rq, output_type="ndarray")
    I = sm["i"].astype(np.int64)
    J = sm["j"].astype(np.int64)
    dx2 = dx * dx
    rmax2 = r_max * r_max
    for c0 in range(0, I.size, chunk):
        Ii = I[c0:c0 + chunk]
        Jj = J[c0:c0 + chunk]
        for ca in range(ka):
            ia = ca * na + Ii
            for cb in range(kb):
                ib = cb * nb + Jj
                oz = _signed(za[ia] - zb[ib], N)
                oy = _signed(ya[ia] - yb[ib], N)
                ox = _signed(xa[ia] - xb[ib], N)
                R2 = ox * ox + oy * oy + oz * oz
                keep = (R2.astype(np.float64) * dx2 < rmax2)
                keep &= (np.abs(ox) <= w) & (np.abs(oy) <= w) & (np.abs(oz) <= w)
                if not np.any(keep):
                    continue
                idx = ((oz[keep] + w) * W + (oy[keep] + w)) * W + (ox[keep] + w)
                val = (qa[ia[keep]].astype(np.float64) / TWO32) * (qb[ib[keep]].astype(np.float64) / TWO32)
                D += np.bincount(idx, weights=val, minlength=W ** 3)
    return D, Qa, Qb


def window_C(pts_a, w_a, pts_b, w_b, L, N, assign, w, r_max):
    """C_ab over the window (valid for |r| < r_max; other cells are -1)."""
    D, Qa, Qb = window_D(pts_a, w_a, pts_b, w_b, L, N, assign, w, r_max)
    if Qa == 0.0 or Qb == 0.0:
        return None
    return float(N) ** 3 * D / (Qa * Qb) - 1.0


def _window_D_chunk(args):
    return window_D(*args)[0]


def window_C_parallel(pts_a, w_a, pts_b, w_b, L, N, assign, w, r_max, workers=None):
    """window_C with the a-points split over a spawn-started process pool
    (D is a sum over a-points, so the chunks add). Safe to call from a
    process that already uses CUDA."""
    import multiprocessing as mp
    import os
    pa = np.asarray(pts_a, dtype=np.float64)
    na = pa.shape[0]
    workers = workers or max(1, min(16, os.cpu_count() or 1))
    if workers == 1 or na < 2000:
        return window_C(pts_a, w_a, pts_b, w_b, L, N, assign, w, r_max)
    bounds = np.linspace(0, na, workers * 2 + 1).astype(int)
    wa = None if w_a is None else np.asarray(w_a, dtype=np.float64)
    jobs = [(pa[b0:b1], None if wa is None else wa[b0:b1], pts_b, w_b, L, N, assign, w, r_max)
            for b0, b1 in zip(bounds[:-1], bounds[1:]) if b1 > b0]
    with mp.get_context("spawn").Pool(workers) as pool:
        parts = pool.map(_window_D_chunk, jobs)
    D = np.sum(parts, axis=0)
    _, _, _, qa, _ = omesh.corners(pa, w_a, L, N, assign)
    _, _, _, qb, _ = omesh.corners(np.asarray(pts_b, dtype=np.float64), w_b, L, N, assign)
    Qa = float(qa.sum()) / TWO32
    Qb = float(qb.sum()) / TWO32
    if Qa == 0.0 or Qb == 0.0:
        return None
    return float(N) ** 3 * D / (Qa * Qb) - 1.0
