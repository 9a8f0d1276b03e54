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
@pytest.mark.parametrize("assign,rsd,cut", [(0, 0.0, 0.0), (1, 0.011, 3.0), (2, 0.011, 0.0)])
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


@pytest.mark.parametrize("precision", [1, 0])
def test_backward_across_batches(pg, precision):
    """Pair meshes split over batches (4 meshes in one batch, in 3 + 1 and in
    2 + 2): the batched passes run the same transforms per column and A
    accumulates in the same order, so the gradients agree up to the order of
    the FP64 atomic adds of the pair chain. (The one-batch gradient is held
    to the oracle by the test above.)"""
    p, cat, w = _case(1, 0.011, 3.0, seed=9)
    rng = np.random.default_rng(12)
    gbar = None
    got = []
    for per_batch in (4, 3, 2):
        plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur,
                       rsd_factor=p.rsd_factor, r_perp_cut=p.r_perp_cut, precision=precision,
                       bins_per_batch=per_batch)
        out = pg.pg_forward(plan, dev(cat.pos), dev(cat.vel), dev(w))
        if gbar is None:
            gbar = {k: rng.standard_normal(np.asarray(out[k]).shape) for k in oa.OUTPUT_KEYS}
        got.append(pg.pg_backward(plan, gbar, cat.n).cpu().numpy())
    scale = np.max(np.abs(got[0]))
    for g in got[1:]:
        assert np.max(np.abs(g - got[0])) <= 1e-12 * scale


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


def _hod_grads(pg, plan, cand, th, keys, seed):
    pos, mass = dev(cand.pos), dev(cand.mass)
    kind, kh = dev(cand.kind), dev(cand.kh)
    w, _ = pg.pg_hod_weights(mass, kind, kh, th, with_grad=False)
    out = pg.pg_forward(plan, pos, None, w)
    rng = np.random.default_rng(seed)
    gbar = {k: rng.standard_normal(np.asarray(out[k]).shape) for k in keys}
    out, g = pg.hod_gradient(plan, pos, None, mass, kind, kh, th, gbar)

    def loss(t):
        wt, _ = pg.pg_hod_weights(mass, kind, kh, t, with_grad=False)
        o = pg.pg_forward(plan, pos, None, wt)
        return sum(float(np.nansum(gbar[k] * np.asarray(o[k]))) for k in keys)

    return gbar, g, loss


@pytest.mark.parametrize("precision", [1, 0])
def test_hod_gradient_matches_oracle(pg, precision):
    from oracle import hod
    th = np.array(synth.HOD_Z09)
    th[3] = 1.1
    L = 64.0
    cand = synth.make_candidates(L, 300, seed=4)
    p = pipeline.Params(L, 32, 1, (0.0, 2.0, 4.0), 2, (6.0, 9.0, 13.0), 2)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur, precision=precision)
    keys = ("b_pg", "q_eff", "xi_pg", "xi_gg")
    gbar, g, _ = _hod_grads(pg, plan, cand, th, keys, 1)
    # the weights themselves: device kernel against the oracle's eq. hod
    w, dw = pg.pg_hod_weights(dev(cand.mass), dev(cand.kind), dev(cand.kh), th)
    wo = hod.weights(th, cand.mass, cand.kind, cand.kh)
    assert np.allclose(w.cpu().numpy(), wo.astype(np.float32), rtol=2e-7, atol=1e-12)
    assert np.allclose(dw.cpu().numpy(), hod.dweights(th, cand.mass, cand.kind, cand.kh), rtol=1e-9, atol=1e-12)
    # dL/dtheta: oracle reverse mode at the FP32 weights the GPU used
    st = oa.forward_state(p, cand.pos, None, w.cpu().numpy().astype(np.float64))
    wbar = oa.grad_weights(st, gbar)
    ref = hod.grad_theta(th, cand.mass, cand.kind, cand.kh, wbar)
    # each component is a sum with cancellation: bound the error by the sum
    # of the magnitudes of its terms, sum_i |wbar_i dw_i/dtheta_k|
    cond = np.abs(hod.dweights(th, cand.mass, cand.kind, cand.kh)).T @ np.abs(wbar)
    tol = 1e-9 if precision else 2e-4
    assert np.all(np.abs(g - ref) <= tol * cond), (g, ref, cond)


@pytest.mark.slow
def test_hod_gradient_finite_differences_512(pg):
    """The 512^3 CIC gradient workload (about 40k candidates, 10 x 5 pair bins,
    10 x 5 correlation bins). log10 M_1, sigma and alpha leave the set of
    occupied satellites unchanged, so the loss is smooth in them and central
    differences in theta check dL/dtheta directly. log10 M_cut and kappa move
    the satellite threshold kappa M_cut, where w ~ x^alpha has an unbounded
    second derivative for alpha < 2, so there the check is a difference along
    dw/dtheta_k in weight space at FP32-representable points."""
    wl = synth.WORKLOADS["rsd_cic_512"]
    th = np.array(synth.HOD_Z09)
    th[3] = 1.1
    cand = synth.make_candidates(wl.box_L, 18000, seed=0, min_ncen=0.2)
    keys = ("b_pg_agg", "q_eff_agg", "xi_gg")
    plan64 = pg.Plan(wl.box_L, wl.mesh_n, 1, wl.s_edges, wl.n_mu, wl.r_edges, wl.n_mur, precision=1)
    gbar, g64, loss = _hod_grads(pg, plan64, cand, th, keys, 3)
    # the weights reach the plan rounded to FP32, a relative error of about
    # 2^-24 / h on each weight's difference: a step of 1e-3 keeps it small
    for k in (1, 2, 3):
        tp, tm = th.copy(), th.copy()
        tp[k] += 1e-3
        tm[k] -= 1e-3
        fd = (loss(tp) - loss(tm)) / 2e-3
        assert abs(fd - g64[k]) <= 1e-3 * abs(g64[k]) + 1e-6, (k, fd, g64[k])
    pos, mass = dev(cand.pos), dev(cand.mass)
    w, dw = pg.pg_hod_weights(mass, dev(cand.kind), dev(cand.kh), th)
    w, dw = w.cpu().numpy().astype(np.float64), dw.cpu().numpy()

    def loss_w(wv):
        o = pg.pg_forward(plan64, pos, None, dev(wv.astype(np.float32)))
        return sum(float(np.nansum(gbar[k] * np.asarray(o[k]))) for k in keys)

    pg.pg_forward(plan64, pos, None, dev(w.astype(np.float32)))
    wbar = pg.pg_backward(plan64, gbar, cand.n).cpu().numpy()
    for k in (0, 4):
        wp = (w + 1e-4 * dw[:, k]).astype(np.float32).astype(np.float64)
        wm = (w - 1e-4 * dw[:, k]).astype(np.float32).astype(np.float64)
        fd = (loss_w(wp) - loss_w(wm)) / 2.0
        # against the step actually taken, (wp - wm) / 2
        assert abs(fd - wbar @ ((wp - wm) / 2.0)) <= 1e-4 * abs(fd), (k, fd)
        # and the device chain against the same sum taken on the host
        assert abs(dw[:, k] @ wbar - g64[k]) <= 1e-10 * (np.abs(dw[:, k]) @ np.abs(wbar)), (k, g64[k])
    plan32 = pg.Plan(wl.box_L, wl.mesh_n, 1, wl.s_edges, wl.n_mu, wl.r_edges, wl.n_mur, precision=0)
    _, g32, _ = _hod_grads(pg, plan32, cand, th, keys, 3)
    cond = np.abs(dw).T @ np.abs(wbar)
    assert np.all(np.abs(g32 - g64) <= 2e-4 * cond), (g32, g64, cond)


@pytest.mark.slow
def test_backward_1024_directional_fd_and_fp32(pg):
    """The 1024^3 instantiations of the adjoint passes (the window-field x
    and y passes, the adjoint z pass with register-free twiddle tables at
    N1 = N2 = 32, the y inverse at the pair lines), on the 12 000-galaxy
    1024^3 case whose forward is held to the oracle elsewhere. FP64: the
    backward against central differences of the FP64 forward along a random
    direction in weight space (a 0.5 % step, exactly representable in FP32).
    FP32: the backward against the FP64 one, within 2e-4 of the largest
    component (the bar of the small-box oracle comparison)."""
    L = 1024.0
    p = pipeline.Params(L, 1024, 1, (0.0, 6.0, 12.0), 2, (4.0, 8.0, 12.0), 2, 0.0, 0.0)
    cat = synth.make_catalogue_box(L, 12000, seed=21)
    w = synth.make_weights(cat.n, 21)
    pos = dev(cat.pos)
    keys = ("b_pg", "q_eff", "xi_pg", "xi_gg", "b_pg_agg", "q_eff_agg")
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur, precision=1)
    rng = np.random.default_rng(23)
    out = pg.pg_forward(plan, pos, None, dev(w))
    gbar = {k: rng.standard_normal(np.asarray(out[k]).shape) for k in keys}
    g64 = pg.pg_backward(plan, gbar, cat.n).cpu().numpy()

    def loss(wv):
        o = pg.pg_forward(plan, pos, None, dev(wv.astype(np.float32)))
        return sum(float(np.nansum(gbar[k] * np.asarray(o[k]))) for k in keys)

    v = (rng.standard_normal(cat.n) * 0.005 * w).astype(np.float32).astype(np.float64)
    wp = (w + v).astype(np.float32).astype(np.float64)
    wm = (w - v).astype(np.float32).astype(np.float64)
    fd = (loss(wp) - loss(wm)) / 2.0
    ad = g64 @ ((wp - wm) / 2.0)
    print(f"1024^3 shell-W adjoint: directional FD {fd:.9e}, adjoint {ad:.9e}, rel {abs(fd - ad) / abs(fd):.2e}")
    assert abs(fd - ad) <= 2e-4 * abs(fd)
    plan.close()
    plan32 = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur, precision=0)
    pg.pg_forward(plan32, pos, None, dev(w))
    g32 = pg.pg_backward(plan32, gbar, cat.n).cpu().numpy()
    rel = np.max(np.abs(g32 - g64)) / np.max(np.abs(g64))
    print(f"1024^3 shell-W adjoint: FP32 against FP64, max |diff| / max |g| = {rel:.2e}")
    assert rel <= 2e-4


@pytest.mark.parametrize("r_max", [6.0, 12.0, 20.0])
def test_backward_pruned_window_transform_256(pg, r_max):
    """At N = 256 (N2 = 8) the adjoint z pass prunes the window column's z
    transform to its nonzero inputs: half-widths w = 6, 12 and 20 cells keep
    2, 4 and 8 of each 32-point DFT's inputs (w < 8, 16 and 32). The FP64
    backward against directional differences of the FP64 forward. With
    D(h) = (L(w + h v) - L(w - h v)) / 2 = h g.v + c h^3 + O(h^5), the
    Richardson combination (8 D(h/2) - D(h)) / 3 removes the h^3 term (on the
    w = 12 case the loss is curved enough that a plain 0.5 % step leaves a
    1e-2 truncation error); the adjoint's g.(actual half-steps) is combined
    the same way."""
    L = 256.0
    cat = synth.make_catalogue_box(L, 4000, seed=61)
    w = synth.make_weights(cat.n, 61)
    p = pipeline.Params(L, 256, 1, (0.0, 4.0, 8.0), 1, (0.25 * r_max, 0.5 * r_max, r_max), 2, 0.0, 0.0)
    plan = pg.Plan(p.box_L, p.mesh_n, p.assign, p.s_edges, p.n_mu, p.r_edges, p.n_mur, precision=1)
    keys = ("b_pg", "q_eff", "xi_pg", "xi_gg", "b_pg_agg")
    rng = np.random.default_rng(62)
    pos = dev(cat.pos)
    out = pg.pg_forward(plan, pos, None, dev(w))
    gbar = {k: rng.standard_normal(np.asarray(out[k]).shape) for k in keys}
    g = pg.pg_backward(plan, gbar, cat.n).cpu().numpy()

    def loss(wv):
        o = pg.pg_forward(plan, pos, None, dev(wv.astype(np.float32)))
        return sum(float(np.nansum(gbar[k] * np.asarray(o[k]))) for k in keys)

    u = rng.standard_normal(cat.n)
    fd, ad = [], []
    for h in (0.005, 0.0025):
        v = u * h * w
        wp = (w + v).astype(np.float32).astype(np.float64)
        wm = (w - v).astype(np.float32).astype(np.float64)
        fd.append((loss(wp) - loss(wm)) / 2.0)
        ad.append(g @ ((wp - wm) / 2.0))
    rf = (8.0 * fd[1] - fd[0]) / 3.0
    ra = (8.0 * ad[1] - ad[0]) / 3.0
    assert abs(rf - ra) <= 2e-4 * abs(ra), (rf, ra)
