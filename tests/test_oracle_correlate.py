"""Pins of the oracle's correlation, binning and ratio outputs."""
import itertools
import math

import numpy as np
import pytest

from oracle import correlate as oc, direct as od, mesh as om, pairs as op, pipeline
from paper_1705_03464_gb300 import synth


def _triplet_counts(pp, gp, L, N, w, bins, n_rb):
    """Pure-Python NGP triplet counting: for every (pair, galaxy) the node
    offset pair - galaxy, binned. Exact integers."""
    dx = L / N
    node = lambda x: [int(math.floor(c / dx + 0.5)) % N for c in x]
    W = 2 * w + 1
    T = [0] * n_rb
    for p in pp:
        a = node(p)
        for g in gp:
            b = node(g)
            o = []
            for k in range(3):
                d = (a[k] - b[k]) % N
                o.append(d - N if d > N // 2 else d)
            if max(abs(v) for v in o) > w:
                continue
            idx = ((o[2] + w) * W + (o[1] + w)) * W + (o[0] + w)
            if bins[idx] >= 0:
                T[bins[idx]] += 1
    return np.array(T)


def test_mesh_correlation_equals_brute_force_triplets():
    L, N = 16.0, 16
    rng = np.random.default_rng(0)
    g = rng.random((40, 3)) * L
    p = rng.random((12, 3)) * L
    r_edges = (1.0, 2.5, 4.0, 6.0)
    n_mur = 2
    w = oc.window_half(N, L, r_edges[-1])
    bins, agg = oc.cell_bins(N, L, r_edges, n_mur, 0.0, w)
    nrb = 3 * n_mur
    T = _triplet_counts(p, g, L, N, w, bins, nrb)
    C = oc.correlate_mesh(om.deposit(p, None, L, N, 0), om.deposit(g, None, L, N, 0))
    s1, _, n, _, _, _ = oc.bin_sums(oc.window_of(C, w), bins, agg, nrb)
    # sum over a bin of C = N^3 T / (N_p N_g) - n_cells, exactly
    assert np.allclose(s1, N ** 3 * T / (12 * 40) - n, rtol=0, atol=1e-9)
    assert np.all(n > 0)


def test_raw_correlation_sign_convention():
    """C_ab(r) = (1/N^3) sum_x delta_b(x) delta_a(x + r): a single a-point at
    node A and b-point at node B peak at r = A - B."""
    L, N = 8.0, 8
    a = np.array([[3.0, 1.0, 5.0]])
    b = np.array([[1.0, 0.0, 2.0]])
    C = oc.correlate_mesh(om.deposit(a, None, L, N, 0), om.deposit(b, None, L, N, 0))
    peak = np.unravel_index(np.argmax(C), C.shape)
    assert peak == (3, 1, 2)  # (z, y, x) of A - B = (2, 1, 3)
    assert np.isclose(C[peak], N ** 3 - 1.0)


def test_mesh_and_direct_forms_agree_cic():
    L, N = 40.0, 32
    cat = synth.make_catalogue_box(L, 300, seed=7)
    rng = np.random.default_rng(8)
    pts = rng.random((25, 3)) * L
    wts = rng.random(25)
    r_max = 15.0
    w = oc.window_half(N, L, r_max)
    Cm = oc.window_of(oc.correlate_mesh(om.deposit(pts, wts, L, N, 1),
                                        om.deposit(cat.pos, None, L, N, 1)), w)
    Cd = od.window_C(pts, wts, cat.pos, None, L, N, 1, w, r_max)
    o = np.arange(-w, w + 1)
    R2 = (o[:, None, None] ** 2 + o[None, :, None] ** 2 + o[None, None, :] ** 2).reshape(-1)
    inside = R2 * (L / N) ** 2 < r_max ** 2
    assert np.max(np.abs(Cm[inside] - Cd[inside])) < 1e-10


def test_translation_by_whole_cells_is_exact_ngp():
    L, N = 32.0, 16
    dx = L / N
    cat = synth.make_catalogue_box(L, 200, seed=9)
    p = pipeline.Params(L, N, 0, (0.0, 2.0, 4.0), 1, (6.0, 9.0, 12.0), 2)
    a = pipeline.run(p, cat.pos, form="direct")
    b = pipeline.run(p, (cat.pos + np.array([3, 5, 7]) * dx) % L, form="direct")
    assert np.array_equal(a["dd"], b["dd"])
    np.testing.assert_array_equal(a["sum_gg"], b["sum_gg"])


def test_poisson_xi_consistent_with_zero():
    L, N = 64.0, 32
    pos = synth.make_uniform(L, 3000, seed=4)
    r_edges = (8.0, 12.0, 16.0, 20.0)
    w = oc.window_half(N, L, r_edges[-1])
    bins, agg = oc.cell_bins(N, L, r_edges, 1, 0.0, w)
    m = om.deposit(pos, None, L, N, 1)
    s1, _, n, _, _, _ = oc.bin_sums(oc.window_of(oc.correlate_mesh(m, m), w), bins, agg, 3)
    xi = s1 / n
    # Poisson sigma of a shell estimate ~ 1 / sqrt(expected pairs in the shell)
    npair = 3000 * 3000 / L ** 3 * np.array([4 / 3 * math.pi * (b ** 3 - a ** 3) for a, b in zip(r_edges[:-1], r_edges[1:])])
    assert np.all(np.abs(xi) < 5 / np.sqrt(npair))


def test_self_count_excess_inside_cavity():
    """Sec. 3.6(a): inside r < s_max/2 + 2 dx the pair field sees its own
    galaxies; far outside it does not."""
    L, N = 64.0, 64
    pos = synth.make_uniform(L, 3000, seed=6)
    p = pipeline.Params(L, N, 1, (0.0, 4.0), 1, (0.0, 2.0, 10.0, 14.0), 1)
    out = pipeline.run(p, pos, form="direct")
    xi = out["xi_pg"][0]
    assert xi[0] > 50 * abs(xi[2])


def test_b_pg_identically_one_when_pairs_are_galaxies():
    L, N = 48.0, 24
    cat = synth.make_catalogue_box(L, 400, seed=2)
    r_edges = (6.0, 10.0, 14.0)
    w = oc.window_half(N, L, r_edges[-1])
    bins, agg = oc.cell_bins(N, L, r_edges, 2, 0.0, w)
    m = om.deposit(cat.pos, None, L, N, 1)
    cg = oc.window_of(oc.correlate_mesh(m, m), w)
    cp = od.window_C(cat.pos, None, cat.pos, None, L, N, 1, w, r_edges[-1])
    s_g = oc.bin_sums(cg, bins, agg, 4)
    s_p = oc.bin_sums(cp, bins, agg, 4)
    sg = dict(zip(("s1", "s2", "n", "a1", "a2", "na"), s_g))
    out = oc.ratios({"s1": s_p[0][None, :], "a1": np.array([s_p[3]])}, sg, np.array([3.0]))
    assert np.allclose(out["b_pg"], 1.0, rtol=1e-9)
    # then eq. Qeff_notsq has the closed form (xi - 1 - xi_w/(2 xi)) / (2 xi + 1.5 xi_w)
    xw = out["xi_dw"]
    assert np.allclose(out["q_eff"][0], (3.0 - 1 - xw / 6.0) / (6.0 + 1.5 * xw), rtol=1e-9)


def test_q_eff_round_trip_and_limits():
    rng = np.random.default_rng(5)
    q = rng.uniform(0.2, 3.0, 50)
    xi = rng.uniform(0.1, 50.0, 50)
    xw = rng.uniform(0.0, 0.5, 50)
    b = oc.b_pg_notsq(q, xi, xw)              # eq. bpg_notsq_dw
    assert np.allclose(oc.q_eff_notsq(b, xi, xw), q, rtol=1e-12)   # eq. Qeff_notsq
    # xi(d_w) -> 0: eq. Qeff_notsq reduces to eq. Qeff, and b to eq. bpg_squeezed
    b0 = 2 * (1 + q * xi) / (1 + xi)
    assert np.allclose(oc.b_pg_notsq(q, xi, 0.0), b0)
    assert np.allclose(oc.q_eff_sq(b0, xi), q)
    assert np.allclose(oc.q_eff_notsq(b0, xi, 0.0), q)
    # xi(d_p) >> 1: Q_eff -> b_pg / 2
    assert np.isclose(oc.q_eff_sq(2.6, 1e9), 1.3, rtol=1e-8)


def test_cell_bins_counts_and_mu():
    N, L = 32, 32.0
    w = oc.window_half(N, L, 6.0)
    bins, agg = oc.cell_bins(N, L, (0.0, 6.0), 3, 0.0, w)
    o = np.arange(-w, w + 1)
    pts = list(itertools.product(o, o, o))
    inside = [(a, b, c) for (c, b, a) in pts if a * a + b * b + c * c < 36]
    assert np.count_nonzero(bins >= 0) == len(inside)
    W = 2 * w + 1
    at = lambda a, b, c: bins[((c + w) * W + (b + w)) * W + (a + w)]
    assert at(0, 0, 5) == 2 and at(5, 0, 0) == 0 and at(0, 0, 0) == 0
    _, agg2 = oc.cell_bins(N, L, (0.0, 6.0), 3, 2.0, w)
    assert not agg2[((5 + w) * W + w) * W + w] and agg2[(w * W + w) * W + w + 3]


def _ngp_node(x, L, N):
    dx = L / N
    return tuple(int(math.floor(c / dx + 0.5)) % N for c in x)


def _offset_counts(pa, pb, L, N):
    """Pure-Python D(r) for NGP unit weights: the number of (a, b) point
    pairs whose node offset node(a) - node(b) is r (mod N), keyed by the
    signed offset (ox, oy, oz) in (-N/2, N/2]."""
    D = {}
    nb = [_ngp_node(q, L, N) for q in pb]
    for p in pa:
        a = _ngp_node(p, L, N)
        for b in nb:
            o = []
            for k in range(3):
                d = (a[k] - b[k]) % N
                o.append(d - N if d > N // 2 else d)
            o = tuple(o)
            D[o] = D.get(o, 0) + 1
    return D


def _shell_sums_brute(D, n_a, n_b, L, N, w, r_edges, n_mur, r_perp_cut):
    """Per (r, mu_r) bin: sum C, sum C^2, cell count, and the same over the
    aggregate (r range, r_perp >= cut), with C(r) = N^3 D(r) / (n_a n_b) - 1
    per window cell, accumulated cell by cell in pure Python."""
    dx = L / N
    nrb = (len(r_edges) - 1) * n_mur
    s1, s2, n = [0.0] * nrb, [0.0] * nrb, [0] * nrb
    a1 = a2 = 0.0
    na = 0
    for oz in range(-w, w + 1):
        for oy in range(-w, w + 1):
            for ox in range(-w, w + 1):
                R2 = ox * ox + oy * oy + oz * oz
                r2 = R2 * dx * dx
                k = -1
                for i in range(len(r_edges) - 1):
                    if r_edges[i] ** 2 <= r2 < r_edges[i + 1] ** 2:
                        k = i
                if k < 0:
                    continue
                mu = abs(oz) / math.sqrt(R2) if R2 > 0 else 0.0
                m = min(n_mur - 1, int(math.floor(n_mur * mu)))
                c = N ** 3 * D.get((ox, oy, oz), 0) / (n_a * n_b) - 1.0
                b = k * n_mur + m
                s1[b] += c
                s2[b] += c * c
                n[b] += 1
                if (ox * ox + oy * oy) * dx * dx >= r_perp_cut ** 2:
                    a1 += c
                    a2 += c * c
                    na += 1
    return np.array(s1), np.array(s2), np.array(n), a1, a2, na


@pytest.mark.parametrize("r_perp_cut", [0.0, 2.0])
def test_shell_sum_of_squares_and_xi_dw_equal_brute_force(r_perp_cut):
    """eq. xi_dw with a shell W: xi(d_w) = sum C_gg^2 / sum C_gg over a bin.
    The squared sums (per bin and over the aggregate support, with and
    without the r_perp cut) are checked against C summed cell by cell from
    pure-Python NGP offset counts; the pipeline's xi_dw and xi_dw_agg follow."""
    L, N = 16.0, 16
    rng = np.random.default_rng(11)
    g = rng.random((36, 3)) * L
    # clustered galaxies, so that C_gg is far from constant inside a shell
    g[:12] = (g[0] + rng.normal(0.0, 1.2, (12, 3))) % L
    r_edges = (1.0, 2.5, 4.0, 6.0)
    n_mur = 2
    w = oc.window_half(N, L, r_edges[-1])
    D = _offset_counts(g, g, L, N)
    b1, b2, bn, ba1, ba2, bna = _shell_sums_brute(D, len(g), len(g), L, N, w, r_edges, n_mur,
                                                  r_perp_cut)
    bins, agg = oc.cell_bins(N, L, r_edges, n_mur, r_perp_cut, w)
    m = om.deposit(g, None, L, N, 0)
    s1, s2, n, a1, a2, na = oc.bin_sums(oc.window_of(oc.correlate_mesh(m, m), w), bins, agg,
                                        len(bn))
    assert n.tolist() == bn.tolist() and na == bna
    np.testing.assert_allclose(s1, b1, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(s2, b2, rtol=1e-12, atol=1e-9)
    assert abs(a1 - ba1) <= 1e-9 * max(1.0, abs(ba1))
    assert abs(a2 - ba2) <= 1e-12 * abs(ba2)
    # the shell sum of squares is not the square of the shell sum
    assert np.max(np.abs(b2 - b1 ** 2 / np.maximum(bn, 1))) > 1.0
    # through the whole forward path: xi_dw, xi_dw_agg and the raw sums
    p = pipeline.Params(L, N, 0, (0.0, 1.5, 3.0), 1, r_edges, n_mur, 0.0, r_perp_cut)
    out = pipeline.run(p, g, form="mesh")
    np.testing.assert_allclose(out["sum2_gg"], b2, rtol=1e-12, atol=1e-9)
    assert abs(out["sum2_gg_agg"] - ba2) <= 1e-12 * abs(ba2)
    np.testing.assert_allclose(out["xi_dw"], b2 / b1, rtol=1e-9)
    assert abs(out["xi_dw_agg"] - ba2 / ba1) <= 1e-9 * abs(ba2 / ba1)
    assert out["n_cells_agg"] == bna
