"""Mass assignment onto the periodic mesh (oracle, FP64, test-only).

Sec. 3.5 assigns galaxies and pairs to an evenly spaced grid over the box
with the triangular-shaped cloud (TSC, 3 nodes per axis); nearest grid
point (NGP, 1 node) and cloud-in-cell (CIC, 2 nodes) are also provided.
Mesh node i sits at i * dx, dx = L / N.

Every node weight is stored as the integer llrint(w * wx * wy * wz * 2^32)
(Q32.32, round half to even), so a mesh is an exact int64 sum that does not
depend on the order of deposits. Layout: mesh[z, y, x].
"""
from __future__ import annotations

import numpy as np

TWO32 = float(2 ** 32)


def axis_nodes(u, N, assign):
    """Nodes and weights along one axis for positions u = x / dx: [n, k]
    arrays. NGP (assign 0): node floor(u + 1/2). CIC (1): floor(u) and the
    next node, weights 1 - f and f, f = u - floor(u). TSC (2): the nearest
    node c = floor(u + 1/2) and its two neighbours, weights (1/2)(1/2 - d)^2,
    3/4 - d^2, (1/2)(1/2 + d)^2 with d = u - c in [-1/2, 1/2). Node indices
    are taken mod N."""
    u = np.asarray(u, dtype=np.float64)
    if assign == 0:
        i = np.floor(u + 0.5)
        return (i.astype(np.int64) % N)[:, None], np.ones((u.size, 1))
    if assign == 1:
        i0 = np.floor(u)
        f = u - i0
        i0 = i0.astype(np.int64)
        return np.stack([i0 % N, (i0 + 1) % N], 1), np.stack([1.0 - f, f], 1)
    if assign == 2:
        c = np.floor(u + 0.5)
        d = u - c
        c = c.astype(np.int64)
        idx = np.stack([(c - 1) % N, c % N, (c + 1) % N], 1)
        wt = np.stack([0.5 * (0.5 - d) ** 2, 0.75 - d ** 2, 0.5 * (0.5 + d) ** 2], 1)
        return idx, wt
    raise ValueError("assign must be 0 (NGP), 1 (CIC) or 2 (TSC)")


def node_weights(points, L, N, assign):
    """Nodes (iz, iy, ix) and unrounded weights wx*wy*wz of each point's
    footprint: [n, k] arrays, k = 1, 8 or 27."""
    p = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    u = p / (L / N)
    (ix, wx), (iy, wy), (iz, wz) = (axis_nodes(u[:, a], N, assign) for a in range(3))
    n, m = p.shape[0], ix.shape[1]
    zs = np.repeat(iz, m * m, axis=1)
    ys = np.tile(np.repeat(iy, m, axis=1), (1, m))
    xs = np.tile(ix, (1, m * m))
    ks = np.repeat(wz, m * m, axis=1) * np.tile(np.repeat(wy, m, axis=1), (1, m)) * np.tile(wx, (1, m * m))
    return zs, ys, xs, ks


def corners(points, w, L, N, assign):
    """Mesh nodes and Q32.32 weights of each point's assignment footprint.

    Returns (iz, iy, ix, q, owner): flat arrays over (point, corner), owner
    being the point index. Node weights per axis as in axis_nodes; the Q32.32
    value is llrint of the product taken in the order ((w * wx) * wy) * wz
    (NGP: w), u = x / dx.
    """
    p = np.asarray(points, dtype=np.float64)
    n = p.shape[0]
    wt = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    dx = L / N
    u = p / dx
    if assign == 0:
        i = np.floor(u + 0.5).astype(np.int64) % N
        q = np.rint(wt * TWO32).astype(np.int64)
        return i[:, 2], i[:, 1], i[:, 0], q, np.arange(n)
    (ix, wx), (iy, wy), (iz, wz) = (axis_nodes(u[:, a], N, assign) for a in range(3))
    m = ix.shape[1]
    izs, iys, ixs, qs, own = [], [], [], [], []
    for cz in range(m):
        for cy in range(m):
            for cx in range(m):
                val = ((wt * wx[:, cx]) * wy[:, cy]) * wz[:, cz]
                qs.append(np.rint(val * TWO32).astype(np.int64))
                izs.append(iz[:, cz])
                iys.append(iy[:, cy])
                ixs.append(ix[:, cx])
                own.append(np.arange(n))
    return (np.concatenate(izs), np.concatenate(iys), np.concatenate(ixs),
            np.concatenate(qs), np.concatenate(own))


def deposit(points, w, L, N, assign):
    """Dense int64 mesh [N, N, N] (z, y, x) of Q32.32 node weights."""
    iz, iy, ix, q, _ = corners(points, w, L, N, assign)
    mesh = np.zeros(N * N * N, dtype=np.int64)
    np.add.at(mesh, (iz * N + iy) * N + ix, q)
    return mesh.reshape(N, N, N)
