"""The smooth-W estimator (pg_forward_smooth, eq. bpg_final with the
Gauss-sigmoid W of eq. weighting) against the oracle on the same seeded
inputs: pair counts exact, xi(s, mu) to FP64 rounding, the convolved-field
means, b_pg, xi(d_w) and Q_eff within the FP32 / FP64 tolerances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import pipeline  # noqa: E402
from oracle import smooth as sm  # noqa: E402
from paper_1705_03464_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def pg():
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import pairgal
    return pairgal


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def close(got, ref, rel, abs_):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    ok = ~np.isnan(ref)
    assert np.all(np.abs(got[ok] - ref[ok]) <= np.maximum(rel * np.abs(ref[ok]), abs_)), (got, ref)


CASES = [
    # box, mesh, assign, galaxies, rsd, weights, W
    (96.0, 32, 2, 1500, 0.0, False, (14.0, 10.0, 0.8, 5.0)),
    (128.0, 64, 1, 3000, 0.011, True, (20.0, 14.0, 0.5, 7.0)),
    (128.0, 64, 0, 2500, 0.0, True, (20.0, 14.0, 0.8, 6.0)),
]


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_smooth_matches_oracle(pg, precision, case):
    L, N, assign, n, rsd, weighted, wprm = CASES[case]
    cat = synth.make_catalogue_box(L, n, seed=20 + case)
    w = synth.make_weights(cat.n, 20 + case) if weighted else None
    p = pipeline.Params(L, N, assign, (0.0, 2.0, 4.0, 6.0), 2, (8.0, 12.0), 1, rsd)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur,
                   rsd_factor=rsd, precision=precision)
    got = pg.pg_forward_smooth(plan, wprm, dev(cat.pos), dev(cat.vel) if rsd else None,
                               None if w is None else dev(w))
    ref = sm.estimate(p, sm.WParams(*wprm), cat.pos, cat.vel if rsd else None, w)
    assert got["dd"].tolist() == ref["dd"].tolist()
    close(got["xi_ss"], ref["xi_ss"], 1e-12, 1e-12)
    scale = max(abs(ref["den"]), np.nanmax(np.abs(ref["num"])))
    tol = 1e-9 if precision else 1e-5
    close(got["num"], ref["num"], tol, tol * scale)
    close([got["den"]], [ref["den"]], tol, tol * scale)
    close([got["xi_dw"]], [ref["xi_dw"]], 1e-9 if precision else 1e-4, 0.0)
    rr = 1e-9 if precision else 1e-4
    close(got["b_pg"], ref["b_pg"], rr, rr * np.nanmax(np.abs(ref["b_pg"])))
    close(got["q_eff"], ref["q_eff"], rr, rr * np.nanmax(np.abs(ref["q_eff"])))
    # a second call reuses W's spectrum; the pair list comes out of the
    # compacting pair kernel in a varying order, so the per-bin FP64 sums can
    # differ in the last bits
    again = pg.pg_forward_smooth(plan, wprm, dev(cat.pos), dev(cat.vel) if rsd else None,
                                 None if w is None else dev(w))
    for k in ("num", "b_pg", "q_eff"):
        np.testing.assert_allclose(again[k], got[k], rtol=1e-12, atol=0)


def test_smooth_rejects_bad_parameters(pg):
    plan = pg.Plan(64.0, 32, 1, (0.0, 2.0), 1, (6.0, 9.0), 1)
    pos = dev(synth.make_uniform(64.0, 100, 1))
    for bad in [(0.0, 10.0, 0.5, 2.0), (10.0, 10.0, 0.5, -1.0), (float("nan"), 1.0, 1.0, 1.0)]:
        with pytest.raises(pg.PairgalError) as e:
            pg.pg_forward_smooth(plan, bad, pos)
        assert e.value.status == pg.PG_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("wset", ["dp30", "dp10"])
def test_smooth_table_weightings_on_the_redshift_space_grid(pg, precision, wset):
    """The paper's two weightings of table tab:weightings (d_p,max = 30 Mpc/h:
    sigma = 50, r_s = 35, s0 = 0.5, r_cut = 20; d_p,max = 10 Mpc/h: 30, 20,
    0.8, 10) with TSC on redshift-space positions, pairs on a (d_perp, d_par)
    grid to 30 Mpc/h in each direction (the cylinder corner, 42.4 Mpc/h, stays
    below L/2), against the oracle's smooth estimator."""
    L, N = 160.0, 64
    cat = synth.make_catalogue_box(L, 2500, seed=41)
    perp = tuple(np.linspace(0.0, 30.0, 7))
    par = tuple(np.linspace(0.0, 30.0, 4))
    wprm = pg.W_DP30 if wset == "dp30" else pg.W_DP10
    p = pipeline.Params(L, N, 2, perp, len(par) - 1, (8.0, 12.0), 1, synth.RSD_FACTOR_Z05, 0.0, par)
    plan = pg.Plan(L, N, 2, perp, len(par) - 1, (8.0, 12.0), 1, rsd_factor=synth.RSD_FACTOR_Z05,
                   precision=precision, par_edges=par)
    got = pg.pg_forward_smooth(plan, wprm, dev(cat.pos), dev(cat.vel))
    ref = sm.estimate(p, sm.WParams(*wprm), cat.pos, cat.vel)
    assert got["dd"].tolist() == ref["dd"].tolist()
    assert int(np.sum(ref["dd"])) > 10000
    close(got["xi_ss"], ref["xi_ss"], 1e-12, 1e-12)
    scale = max(abs(ref["den"]), np.nanmax(np.abs(ref["num"])))
    tol = 1e-9 if precision else 1e-5
    close(got["num"], ref["num"], tol, tol * scale)
    close([got["den"]], [ref["den"]], tol, tol * scale)
    rr = 1e-9 if precision else 1e-4
    close([got["xi_dw"]], [ref["xi_dw"]], rr, 0.0)
    close(got["b_pg"], ref["b_pg"], rr, rr * np.nanmax(np.abs(ref["b_pg"])))
    close(got["q_eff"], ref["q_eff"], rr, rr * np.nanmax(np.abs(ref["q_eff"])))
