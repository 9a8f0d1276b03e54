"""GPU adjoint (pg_backward) against the oracle's reverse-mode gradient and
against finite differences of the GPU forward."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import adjoint as oa, pipeline  # noqa: E402
from paper_1705_03464_gb300 import synth  # noqa: E402


@pytest.fixture(scope="module")
def pg():
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import pairgal
    return pairgal


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(assign, rsd, cut, seed=3):
    L, N = 64.0, 32
    cat = synth.make_catalogue_box(L, 500, seed=seed)
    w = synth.make_weights(cat.n, seed)
    p = pipeline.Params(L, N, assign, (0.0, 2.0, 4.0), 2, (6.0, 9.0, 13.0), 2, rsd, cut)
    return p, cat, w


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("assign,rsd,cut", [(0, 0.0, 0.0), (1, 0.011, 3.0)])
def test_backward_matches_oracle_gradient(pg, precision, assign, rsd, cut):
    p, cat, w = _case(assign, rsd, cut)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur,
                   rsd_factor=p.rsd_factor, r_perp_cut=p.r_perp_cut, precision=precision)
    out = pg.pg_forward(plan, dev(cat.pos), dev(cat.vel), dev(w))
    st = oa.forward_state(p, cat.pos, cat.vel, w.astype(np.float64))
    rng = np.random.default_rng(11)
    o = oa.outputs(st)
    gbar = {k: rng.standard_normal(np.asarray(o[k]).shape) for k in oa.OUTPUT_KEYS}
    ref = oa.grad_weights(st, gbar)
    got = pg.pg_backward(plan, gbar, cat.n).cpu().numpy()
    scale = np.max(np.abs(ref))
    tol = 1e-9 if precision else 2e-4
    assert np.max(np.abs(got - ref)) <= tol * scale, np.max(np.abs(got - ref)) / scale


def test_backward_directional_finite_difference(pg):
    p, cat, w = _case(1, 0.011, 0.0, seed=5)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur,
                   rsd_factor=p.rsd_factor, precision=1)
    rng = np.random.default_rng(2)
    keys = ("b_pg", "q_eff", "xi_pg", "b_pg_agg")
    out = pg.pg_forward(plan, dev(cat.pos), dev(cat.vel), dev(w))
    gbar = {k: rng.standard_normal(np.asarray(out[k]).shape) for k in keys}

    def loss(wv):
        o = pg.pg_forward(plan, dev(cat.pos), dev(cat.vel), dev(wv.astype(np.float32)))
        return sum(float(np.nansum(gbar[k] * np.asarray(o[k]))) for k in keys)

    pg.pg_forward(plan, dev(cat.pos), dev(cat.vel), dev(w))
    g = pg.pg_backward(plan, gbar, cat.n).cpu().numpy()
    # perturb along a direction exactly representable in FP32 around w
    # (a 0.5% step: the central-difference error is second order in the step)
    v = (rng.standard_normal(cat.n) * 0.005 * w).astype(np.float32).astype(np.float64)
    wp = (w + v).astype(np.float32).astype(np.float64)
    wm = (w - v).astype(np.float32).astype(np.float64)
    fd = (loss(wp) - loss(wm)) / 2.0
    assert abs(fd - g @ ((wp - wm) / 2.0)) <= 2e-4 * abs(fd) + 1e-9


def test_autograd_function(pg):
    p, cat, w = _case(1, 0.0, 0.0, seed=7)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur, precision=1)
    wt = dev(w).requires_grad_(True)
    outs = pg.PairGalFn.apply(wt, plan, dev(cat.pos))
    loss = torch.nansum(outs[0]) + 0.5 * torch.nansum(outs[1])
    loss.backward()
    st = oa.forward_state(p, cat.pos, None, w.astype(np.float64))
    o = oa.outputs(st)
    ref = oa.grad_weights(st, {"b_pg": np.ones_like(o["b_pg"]), "q_eff": 0.5 * np.ones_like(o["q_eff"])})
    got = wt.grad.double().cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
