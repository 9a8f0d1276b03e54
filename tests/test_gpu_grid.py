"""GPU path on the (d_perp, d_par) pair grid (pair_grid = 1; the b_pg / Q_eff
maps of Sec. 5 and the projected w(d_perp) of eq.
2PCF_los_integrated_explicit) against the oracle on the same seeded inputs:
pair lists and counts bit-exact, the forward (xi, b_pg, Q_eff, w(d_perp)),
the smooth-W estimator and the adjoint within the usual tolerances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import adjoint as oa, pairs as op, pipeline  # noqa: E402
from oracle import smooth as sm  # noqa: E402
from paper_1705_03464_gb300 import synth  # noqa: E402

PERP = (0.0, 1.0, 2.5, 4.0)
PAR = (0.0, 1.0, 3.0, 6.0)


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
    err = np.abs(got[ok] - ref[ok])
    tol = np.maximum(rel * np.abs(ref[ok]), abs_)
    assert np.all(err <= tol), (err / tol).max()


def _params(L=128.0, N=64, assign=1, rsd=0.0):
    return pipeline.Params(L, N, assign, PERP, len(PAR) - 1, (8.0, 12.0, 17.0, 23.0), 2, rsd, 0.0, PAR)


def _plan(pg, p, precision, **kw):
    return pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur,
                   rsd_factor=p.rsd_factor, precision=precision, par_edges=p.par_edges, **kw)


def test_grid_pairs_bitexact(pg):
    L = 64.0
    cat = synth.make_catalogue_box(L, 2500, seed=31)
    w = synth.make_weights(cat.n, 31)
    x = op.transform_positions(cat.pos, None, L, 0.0)
    plan = pg.Plan(L, 32, 0, PERP, 3, (0.0, L / 4), 1, par_edges=PAR)
    out = pg.pg_find_pairs(plan, dev(x), dev(w))
    ref = op.find_pairs(x, w, L, PERP, 3, par_edges=PAR)
    dd, ddq = op.pair_counts(ref, 3, 3)
    assert out["dd"].cpu().numpy().tolist() == dd.tolist()
    assert out["ddq"].cpu().numpy().tolist() == ddq.tolist()
    assert out["n_pairs"] == len(ref["i"]) > 100
    gi = out["i"].cpu().numpy().astype(np.int64)
    gj = out["j"].cpu().numpy().astype(np.int64)
    og = np.lexsort((gj, gi))
    orf = np.lexsort((ref["j"], ref["i"]))
    assert np.array_equal(gi[og], ref["i"][orf]) and np.array_equal(gj[og], ref["j"][orf])
    assert np.array_equal(out["bin"].cpu().numpy()[og], (ref["sbin"] * 3 + ref["mubin"])[orf])
    assert np.array_equal(out["mid"].cpu().numpy()[og], ref["mid"][orf])


@pytest.mark.parametrize("precision", [1, 0])
def test_grid_forward_matches_oracle(pg, precision):
    p = _params(rsd=synth.RSD_FACTOR_Z05)
    cat = synth.make_catalogue_box(p.box_L, 3000, seed=8)
    w = synth.make_weights(cat.n, 8)
    got = pg.pg_forward(_plan(pg, p, precision, bins_per_batch=4), dev(cat.pos), dev(cat.vel), dev(w))
    ref = pipeline.run(p, cat.pos, cat.vel, w, form="mesh")
    assert got["dd"].tolist() == ref["dd"].tolist()
    close(got["xi_ss"], ref["xi_ss"], 1e-12, 1e-12)
    close(got["w_perp"], ref["w_perp"], 1e-12, 1e-12)
    rel, absx = (1e-9, 1e-12) if precision else (1e-5, 1e-7)
    close(got["xi_pg"], ref["xi_pg"], rel, absx)
    rr = 1e-9 if precision else 1e-4
    for k in ("b_pg", "q_eff", "b_pg_agg", "q_eff_agg"):
        close(got[k], ref[k], rr, rr * np.nanmax(np.abs(ref[k])))


def test_grid_w_perp_is_nan_on_shell_bins(pg):
    p = pipeline.Params(128.0, 64, 1, (0.0, 2.0, 4.0), 2, (8.0, 12.0), 1)
    cat = synth.make_catalogue_box(p.box_L, 1500, seed=2)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur)
    assert np.all(np.isnan(pg.pg_forward(plan, dev(cat.pos))["w_perp"]))


def test_grid_rejects_bad_edges(pg):
    with pytest.raises(Exception):
        pg.Plan(64.0, 32, 1, PERP, 2, (8.0, 12.0), 1, par_edges=(0.0, 2.0, 1.0))
    with pytest.raises(Exception):   # sqrt(4^2 + 31.9^2) >= L / 2
        pg.Plan(64.0, 32, 1, PERP, 1, (8.0, 12.0), 1, par_edges=(0.0, 31.9))


@pytest.mark.parametrize("precision", [1, 0])
def test_grid_smooth_matches_oracle(pg, precision):
    p = _params(L=128.0, N=64, assign=2)
    cat = synth.make_catalogue_box(p.box_L, 2500, seed=40)
    wprm = (20.0, 14.0, 0.8, 6.0)
    got = pg.pg_forward_smooth(_plan(pg, p, precision), wprm, dev(cat.pos))
    ref = sm.estimate(p, sm.WParams(*wprm), cat.pos)
    assert got["dd"].tolist() == ref["dd"].tolist()
    close(got["xi_ss"], ref["xi_ss"], 1e-12, 1e-12)
    rr = 1e-9 if precision else 1e-4
    close(got["b_pg"], ref["b_pg"], rr, rr * np.nanmax(np.abs(ref["b_pg"])))
    close(got["q_eff"], ref["q_eff"], rr, rr * np.nanmax(np.abs(ref["q_eff"])))


@pytest.mark.parametrize("precision", [1, 0])
def test_grid_backward_matches_oracle_gradient(pg, precision):
    p = pipeline.Params(64.0, 32, 1, (0.0, 1.5, 3.0), 2, (6.0, 9.0, 13.0), 2, 0.011, 0.0, (0.0, 1.5, 3.5))
    cat = synth.make_catalogue_box(p.box_L, 500, seed=3)
    w = synth.make_weights(cat.n, 3)
    plan = _plan(pg, p, precision)
    pg.pg_forward(plan, dev(cat.pos), dev(cat.vel), dev(w))
    st = oa.forward_state(p, cat.pos, cat.vel, w.astype(np.float64))
    rng = np.random.default_rng(13)
    o = oa.outputs(st)
    gbar = {k: rng.standard_normal(np.asarray(o[k]).shape) for k in oa.GRID_OUTPUT_KEYS}
    ref = oa.grad_weights(st, gbar)
    got = pg.pg_backward(plan, gbar, cat.n).cpu().numpy()
    scale = np.max(np.abs(ref))
    tol = 1e-9 if precision else 2e-4
    assert np.max(np.abs(got - ref)) <= tol * scale, np.max(np.abs(got - ref)) / scale
