"""Pins of the oracle's (d_perp, d_par) pair grid (Sec. 3.4, eq.
2PCF_los_integrated_explicit; the b_pg / Q_eff maps of Sec. 5): brute force
on tiny catalogues, planted pairs with known separations, closed-form
volumes, a Poisson catalogue, and the projected w(d_perp) of a constant xi."""
import math

import numpy as np

from oracle import pairs as op


def _brute_grid(pos, L, pe_perp, pe_par):
    """Pair counts per grid cell by a plain double loop (sqrt of d_perp^2)."""
    n_p, n_l = len(pe_perp) - 1, len(pe_par) - 1
    cnt = np.zeros(n_p * n_l, dtype=np.int64)
    n = len(pos)
    for i in range(n):
        for j in range(i + 1, n):
            d = []
            for a in range(3):
                t = pos[j][a] - pos[i][a]
                if t > L / 2:
                    t -= L
                if t < -L / 2:
                    t += L
                d.append(t)
            dp = math.sqrt(d[0] ** 2 + d[1] ** 2)
            dl = abs(d[2])
            k = [b for b in range(n_p) if pe_perp[b] <= dp < pe_perp[b + 1]]
            m = [b for b in range(n_l) if pe_par[b] <= dl < pe_par[b + 1]]
            if k and m:
                cnt[k[0] * n_l + m[0]] += 1
    return cnt


def test_grid_counts_match_brute_force():
    rng = np.random.default_rng(5)
    L = 10.0
    pos = rng.random((70, 3)) * L
    perp = (0.0, 1.0, 2.0, 3.0)
    par = (0.0, 0.5, 1.5, 2.5)
    pr = op.find_pairs(pos, None, L, perp, 3, par_edges=par)
    cnt, _ = op.pair_counts(pr, 3, 3)
    assert cnt.tolist() == _brute_grid(pos.tolist(), L, perp, par).tolist()
    assert cnt.sum() > 20


def test_planted_pairs_land_in_their_cells():
    # isolated pairs 20 apart with chosen (d_perp, d_par), across the box edge too
    L = 100.0
    perp = (0.0, 1.0, 2.0, 4.0)
    par = (0.0, 1.0, 3.0)
    seps = [((0.6, 0.0), 0.5), ((0.0, 1.5), -2.0), ((2.0, 2.0), 0.2), ((0.3, -0.4), 2.9), ((3.0, 0.0), -0.9)]
    want = [0 * 2 + 0, 1 * 2 + 1, 2 * 2 + 0, 0 * 2 + 1, 2 * 2 + 0]
    pos = []
    for n, ((dx, dy), dz) in enumerate(seps):
        base = np.array([20.0 * n + 5.0, 50.0, 0.5 if n == 1 else 30.0])
        pos += [base, base + np.array([dx, dy, dz])]
    pos = op.wrap(np.array(pos), L)
    pr = op.find_pairs(pos, None, L, perp, 2, par_edges=par)
    got = sorted((pr["sbin"] * 2 + pr["mubin"]).tolist())
    assert got == sorted(want)


def test_cell_volumes_closed_form():
    perp = np.array([0.0, 1.0, 2.5, 4.0])
    par = np.array([0.0, 0.5, 2.0])
    v = op.pair_volumes(perp, 2, par)
    assert v.shape == (6,)
    # the whole grid is the cylinder pi p_max^2 * 2 l_max
    assert math.isclose(v.sum(), math.pi * 16.0 * 4.0, rel_tol=1e-14)
    # one cell: annulus 1 <= d_perp < 2.5 times |d_par| in [0.5, 2)
    assert math.isclose(v[1 * 2 + 1], math.pi * (2.5 ** 2 - 1.0) * 2 * 1.5, rel_tol=1e-14)


def test_poisson_grid_counts_match_volumes():
    rng = np.random.default_rng(17)
    L, n = 60.0, 2500
    pos = rng.random((n, 3)) * L
    perp = (0.0, 2.0, 4.0, 6.0)
    par = (0.0, 2.0, 4.0, 6.0)
    pr = op.find_pairs(pos, None, L, perp, 3, par_edges=par)
    dd, ddq = op.pair_counts(pr, 3, 3)
    xi, rr = op.xi_ss(ddq, None, n, L, perp, 3, par)
    assert np.all(np.abs(dd - rr) <= 5.0 * np.sqrt(rr))
    w = op.w_perp(xi, par)
    # noise of w: 2 dl sqrt(sum 1/RR) per row
    sig = 2 * 2.0 * np.sqrt(np.sum(1.0 / rr.reshape(3, 3), axis=1))
    assert np.all(np.abs(w) <= 5.0 * sig)


def test_w_perp_of_constant_xi_is_twice_the_depth():
    par = (0.0, 0.5, 2.0, 3.5)
    xi = np.full(4 * 3, 0.7)
    np.testing.assert_allclose(op.w_perp(xi, par), 2 * 3.5 * 0.7, rtol=1e-14)


def test_grid_and_shell_binnings_agree_inside_the_sphere():
    # pairs with s < R are the same set under both binnings when R <= p_max, l_max
    rng = np.random.default_rng(23)
    L = 30.0
    pos = rng.random((600, 3)) * L
    R = 3.0
    shell = op.find_pairs(pos, None, L, (0.0, R), 1)
    grid = op.find_pairs(pos, None, L, (0.0, 3.5), 1, par_edges=(0.0, 3.5))
    d = op.min_image(pos[grid["j"]] - pos[grid["i"]], L)
    inside = (d * d).sum(axis=1) < R * R
    a = sorted(zip(shell["i"].tolist(), shell["j"].tolist()))
    b = sorted(zip(grid["i"][inside].tolist(), grid["j"][inside].tolist()))
    assert a == b and len(a) > 50


def test_w_perp_gradient_matches_central_differences():
    # the oracle's reverse mode of w(d_perp) (through xi = DD/RR - 1 and the
    # weight sums of RR) against central differences in single weights
    from oracle import adjoint as oa, pipeline
    from paper_1705_03464_gb300 import synth
    L, N = 64.0, 32
    cat = synth.make_catalogue_box(L, 400, seed=3)
    w = synth.make_weights(cat.n, 3).astype(np.float64)
    p = pipeline.Params(L, N, 1, (0.0, 1.5, 3.0), 2, (6.0, 9.0), 1, 0.0, 0.0, (0.0, 1.5, 3.5))
    st = oa.forward_state(p, cat.pos, None, w)
    rng = np.random.default_rng(4)
    gbar = {"w_perp": rng.standard_normal(2), "xi_ss": rng.standard_normal(4)}
    g = oa.grad_weights(st, gbar)
    for i in rng.choice(cat.n, 4, replace=False):
        h = 1e-4 * w[i]
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (oa.loss(oa.forward_state(p, cat.pos, None, wp), gbar)
              - oa.loss(oa.forward_state(p, cat.pos, None, wm), gbar)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]) + 1e-9
