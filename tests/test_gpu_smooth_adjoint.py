"""GPU adjoint of the smooth-W estimator (pg_backward_smooth) against the
oracle's reverse-mode gradient (oracle/smooth_adjoint.py, itself pinned by
finite differences) on the same seeded inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import pipeline  # noqa: E402
from oracle import smooth as sm  # noqa: E402
from oracle import smooth_adjoint as sa  # noqa: E402
from paper_1705_03464_gb300 import synth  # noqa: E402

WPRM = (8.0, 6.0, 0.8, 3.0)


@pytest.fixture(scope="module")
def pg():
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import pairgal
    return pairgal


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(assign, rsd, weighted, grid):
    L, N = 64.0, 32
    cat = synth.make_catalogue_box(L, 400, seed=3)
    w = synth.make_weights(cat.n, 3) if weighted else None
    if grid:
        p = pipeline.Params(L, N, assign, (0.0, 1.5, 3.0), 2, (6.0, 9.0), 1, rsd, 0.0, (0.0, 1.5, 3.5))
    else:
        p = pipeline.Params(L, N, assign, (0.0, 2.0, 4.0), 2, (6.0, 9.0), 1, rsd)
    return p, cat, w


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("assign,rsd,weighted,grid", [(1, 0.0, False, False), (2, 0.011, True, False),
                                                      (0, 0.011, True, True)])
def test_smooth_backward_matches_oracle_gradient(pg, precision, assign, rsd, weighted, grid):
    p, cat, w = _case(assign, rsd, weighted, grid)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur,
                   rsd_factor=rsd, precision=precision, par_edges=p.par_edges)
    pg.pg_forward_smooth(plan, WPRM, dev(cat.pos), dev(cat.vel) if rsd else None,
                         None if w is None else dev(w))
    w64 = np.ones(cat.n) if w is None else w.astype(np.float64)
    st = sa.forward_state(p, sm.WParams(*WPRM), cat.pos, cat.vel if rsd else None, w64)
    rng = np.random.default_rng(17)
    o = sa.outputs(st)
    gbar = {k: rng.standard_normal(np.asarray(o[k]).shape) for k in sa.OUTPUT_KEYS}
    ref = sa.grad_weights(st, gbar)
    got = pg.pg_backward_smooth(plan, gbar, cat.n).cpu().numpy()
    scale = np.max(np.abs(ref))
    # FP64: 1e-8 of the largest component (rounding through the ratio and
    # eq. Qeff_notsq chains reaches 1.4e-9 on these shot-noise boxes)
    tol = 1e-8 if precision else 2e-4
    assert np.max(np.abs(got - ref)) <= tol * scale, np.max(np.abs(got - ref)) / scale


def test_smooth_backward_needs_a_smooth_forward(pg):
    p, cat, _ = _case(1, 0.0, False, False)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur)
    with pytest.raises(Exception):
        pg.pg_backward_smooth(plan, {"num": np.ones(plan.P)}, cat.n)
    pg.pg_forward_smooth(plan, WPRM, dev(cat.pos))
    pg.pg_backward_smooth(plan, {"num": np.ones(plan.P)}, cat.n)
    pg.pg_forward(plan, dev(cat.pos))   # a shell-W forward reuses the plan's buffers
    with pytest.raises(Exception):
        pg.pg_backward_smooth(plan, {"num": np.ones(plan.P)}, cat.n)


@pytest.mark.parametrize("precision", [1, 0])
def test_hod_gradient_through_the_smooth_estimator(pg, precision):
    """dL/dtheta of the paper's own estimator for the five HOD parameters
    (Sec. 3.3 eq. hod): soft weights, pg_forward_smooth, pg_backward_smooth and
    the chain on the device, against the oracle's reverse mode composed with the
    oracle's dw/dtheta at the FP32 weights the GPU used."""
    from oracle import hod
    th = np.array(synth.HOD_Z09)
    th[3] = 1.1
    L = 64.0
    cand = synth.make_candidates(L, 300, seed=4)
    p = pipeline.Params(L, 32, 2, (0.0, 2.0, 4.0), 2, (6.0, 9.0), 1)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur, precision=precision)
    rng = np.random.default_rng(6)
    gbar = {"b_pg": rng.standard_normal(plan.P), "q_eff": rng.standard_normal(plan.P),
            "xi_dw": rng.standard_normal(1)}
    out, g = pg.hod_gradient_smooth(plan, WPRM, dev(cand.pos), None, dev(cand.mass), dev(cand.kind),
                                    dev(cand.kh), th, gbar)
    w, _ = pg.pg_hod_weights(dev(cand.mass), dev(cand.kind), dev(cand.kh), th)
    st = sa.forward_state(p, sm.WParams(*WPRM), cand.pos, None, w.cpu().numpy().astype(np.float64))
    wbar = sa.grad_weights(st, gbar)
    ref = hod.grad_theta(th, cand.mass, cand.kind, cand.kh, wbar)
    cond = np.abs(hod.dweights(th, cand.mass, cand.kind, cand.kh)).T @ np.abs(wbar)
    tol = 1e-8 if precision else 2e-4
    assert np.all(np.abs(np.asarray(g) - ref) <= tol * cond), (g, ref, cond)


@pytest.mark.slow
def test_smooth_backward_1024_directional_fd_and_fp32(pg):
    """The smooth-W adjoint's 1024^3 passes with the table's d_p,max = 10
    weighting and TSC, on a 12 000-galaxy 1024^3 box: the FP64 backward
    against central differences of the FP64 smooth forward along a random
    direction in weight space (0.5 % steps, exactly representable in FP32),
    and the FP32 backward against the FP64 one within 2e-4 of the largest
    component."""
    L = 1024.0
    cat = synth.make_catalogue_box(L, 12000, seed=22)
    w = synth.make_weights(cat.n, 22)
    pos = dev(cat.pos)
    keys = ("b_pg", "q_eff", "num", "xi_dw")
    args = (L, 1024, 2, (0.0, 5.0, 10.0), 2, (12.0, 20.0), 1)
    plan = pg.Plan(*args, precision=1)
    rng = np.random.default_rng(29)
    out = pg.pg_forward_smooth(plan, pg.W_DP10, pos, None, dev(w))
    gbar = {k: rng.standard_normal(np.asarray(out[k]).shape) for k in keys}
    g64 = pg.pg_backward_smooth(plan, gbar, cat.n).cpu().numpy()

    def loss(wv):
        o = pg.pg_forward_smooth(plan, pg.W_DP10, pos, None, dev(wv.astype(np.float32)))
        return sum(float(np.nansum(gbar[k] * np.asarray(o[k]))) for k in keys)

    v = (rng.standard_normal(cat.n) * 0.005 * w).astype(np.float32).astype(np.float64)
    wp = (w + v).astype(np.float32).astype(np.float64)
    wm = (w - v).astype(np.float32).astype(np.float64)
    fd = (loss(wp) - loss(wm)) / 2.0
    ad = g64 @ ((wp - wm) / 2.0)
    print(f"1024^3 smooth-W adjoint: directional FD {fd:.9e}, adjoint {ad:.9e}, rel {abs(fd - ad) / abs(fd):.2e}")
    assert abs(fd - ad) <= 2e-4 * abs(fd)
    plan.close()
    plan32 = pg.Plan(*args, precision=0)
    pg.pg_forward_smooth(plan32, pg.W_DP10, pos, None, dev(w))
    g32 = pg.pg_backward_smooth(plan32, gbar, cat.n).cpu().numpy()
    rel = np.max(np.abs(g32 - g64)) / np.max(np.abs(g64))
    print(f"1024^3 smooth-W adjoint: FP32 against FP64, max |diff| / max |g| = {rel:.2e}")
    assert rel <= 2e-4


@pytest.mark.parametrize("precision", [1, 0])
def test_smooth_backward_dp30_redshift_space_grid(pg, precision):
    """The adjoint of the paper's redshift-space configuration: the table's
    d_p,max = 30 Mpc/h weighting, TSC, positions displaced along z, weighted
    galaxies and pairs on a (d_perp, d_par) grid to 30 Mpc/h, against the
    oracle's reverse mode (1e-8 in FP64, 2e-4 in FP32, of the largest
    component)."""
    L, N = 160.0, 64
    cat = synth.make_catalogue_box(L, 1200, seed=43)
    w = synth.make_weights(cat.n, 43)
    perp = tuple(np.linspace(0.0, 30.0, 7))
    par = tuple(np.linspace(0.0, 30.0, 4))
    p = pipeline.Params(L, N, 2, perp, len(par) - 1, (8.0, 12.0), 1, synth.RSD_FACTOR_Z05, 0.0, par)
    plan = pg.Plan(L, N, 2, perp, len(par) - 1, (8.0, 12.0), 1, rsd_factor=synth.RSD_FACTOR_Z05,
                   precision=precision, par_edges=par)
    pg.pg_forward_smooth(plan, pg.W_DP30, dev(cat.pos), dev(cat.vel), dev(w))
    st = sa.forward_state(p, sm.WParams(*pg.W_DP30), cat.pos, cat.vel, w.astype(np.float64))
    rng = np.random.default_rng(31)
    o = sa.outputs(st)
    gbar = {k: rng.standard_normal(np.asarray(o[k]).shape) for k in sa.OUTPUT_KEYS}
    ref = sa.grad_weights(st, gbar)
    got = pg.pg_backward_smooth(plan, gbar, cat.n).cpu().numpy()
    scale = np.max(np.abs(ref))
    tol = 1e-8 if precision else 2e-4
    assert np.max(np.abs(got - ref)) <= tol * scale, np.max(np.abs(got - ref)) / scale
