"""Mass assignment onto the periodic mesh (oracle, FP64, test-only).

Sec. 3.5 assigns galaxies and pairs to an evenly spaced grid over the box;
the paper uses TSC, this build uses nearest-grid-point (NGP) and
cloud-in-cell (CIC) weights. Mesh node i sits at i * dx, dx = L / N.

Every node weight is stored as the integer llrint(w * wx * wy * wz * 2^32)
(Q32.32, round half to even), so a mesh is an exact int64 sum that does not
depend on the order of deposits. Layout: mesh[z, y, x].
"""
from __future__ import annotations

import numpy as np

TWO32 = float(2 ** 32)


def corners(points, w, L, N, assign):
    """Mesh nodes and Q32.32 weights of each point's assignment footprint.

    Returns (iz, iy, ix, q, owner): flat arrays over (point, corner), owner
    being the point index. NGP: node floor(u + 1/2) mod N. CIC: nodes
    i0 = floor(u) and i0 + 1 (mod N) with weights 1 - f and f, f = u - i0,
    u = x / dx. The product order is ((w * wx) * wy) * wz.
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
    i0 = np.floor(u)
    f = u - i0
    i0 = i0.astype(np.int64)
    izs, iys, ixs, qs, own = [], [], [], [], []
    for cz in (0, 1):
        wz = f[:, 2] if cz else 1.0 - f[:, 2]
        for cy in (0, 1):
            wy = f[:, 1] if cy else 1.0 - f[:, 1]
            for cx in (0, 1):
                wx = f[:, 0] if cx else 1.0 - f[:, 0]
                val = ((wt * wx) * wy) * wz
                qs.append(np.rint(val * TWO32).astype(np.int64))
                izs.append((i0[:, 2] + cz) % N)
                iys.append((i0[:, 1] + cy) % N)
                ixs.append((i0[:, 0] + cx) % N)
                own.append(np.arange(n))
    return (np.concatenate(izs), np.concatenate(iys), np.concatenate(ixs),
            np.concatenate(qs), np.concatenate(own))


def deposit(points, w, L, N, assign):
    """Dense int64 mesh [N, N, N] (z, y, x) of Q32.32 node weights."""
    iz, iy, ix, q, _ = corners(points, w, L, N, assign)
    mesh = np.zeros(N * N * N, dtype=np.int64)
    np.add.at(mesh, (iz * N + iy) * N + ix, q)
    return mesh.reshape(N, N, N)
