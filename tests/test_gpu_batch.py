"""Many-mock batch (pg_run_batch), plans that share mesh scratch
(pg_plan_create_shared) and the batch-size autotuner, on the GPU. The
forward is deterministic, so a mock run in a batch or on a shared-scratch
plan must give exactly the outputs of its own standalone plan."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1705_03464_gb300 import synth  # noqa: E402

KEYS = ("dd", "dd_w", "xi_ss", "xi_pg", "xi_gg", "b_pg", "q_eff", "q_eff_sq", "b_pg_agg",
        "q_eff_agg", "sum_pg", "sum_gg", "sum2_gg", "n_cells")


@pytest.fixture(scope="module")
def pg():
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import pairgal
    return pairgal


def _same(a, b):
    for k in KEYS:
        np.testing.assert_array_equal(np.asarray(a[k]), np.asarray(b[k]), err_msg=k)


def _small_mocks():
    """Uneven mocks on two mesh sizes; mock 3 repeats mock 0's problem."""
    spec = [(96.0, 64, 1500, 0), (80.0, 32, 900, 1), (128.0, 64, 2500, 2), (96.0, 64, 1200, 3),
            (72.0, 32, 600, 4)]
    out = []
    for L, N, n, seed in spec:
        w = synth.Workload(f"m{seed}", L, N, 1, n, (0.0, 2.0, 4.0), 2, (6.0, 10.0, 15.0), 2, False, 0,
                           bins_per_batch=3)
        out.append((w, synth.make_catalogue(w, seed).pos))
    return out


def test_shared_scratch_plans_match_standalone(pg):
    mocks = _small_mocks()
    (w0, p0), (w2, p2) = mocks[0], mocks[2]   # both 64^3, different boxes
    a = pg.Plan.of(w0)
    b = pg.Plan.of(w2, share_with=a)
    ra, rb = pg.pg_forward_host(a, p0), pg.pg_forward_host(b, p2)
    ra2 = pg.pg_forward_host(a, p0)   # after b used the shared scratch
    _same(ra, ra2)
    _same(ra, pg.pg_forward_host(pg.Plan.of(w0), p0))
    _same(rb, pg.pg_forward_host(pg.Plan.of(w2), p2))
    with pytest.raises(pg.PairgalError):   # other mesh size: no sharing
        pg.Plan.of(mocks[1][0], share_with=a)


def test_run_batch_matches_standalone_plans(pg):
    mocks = _small_mocks()
    problems = [pg.Problem.of(w) for w, _ in mocks]
    outs, lat, st = pg.pg_run_batch(problems, [(p,) for _, p in mocks])
    assert st["n_plans"] == 4 and st["n_workspaces"] == 2
    assert np.all(np.isfinite(lat)) and np.all(lat > 0)
    assert st["p50_ms"] <= st["p99_ms"] and st["mocks_per_s"] > 0 and st["gpu_launches"] > 0
    for (w, pos), o in zip(mocks, outs):
        _same(o, pg.pg_forward_host(pg.Plan.of(w), pos))


def test_run_batch_reports_failures(pg):
    mocks = _small_mocks()[:2]
    bad = mocks[1][1].copy()
    bad[3, 0] = np.nan
    problems = [pg.Problem.of(w) for w, _ in mocks]
    with pytest.raises(pg.PairgalError) as e:
        pg.pg_run_batch(problems, [(mocks[0][1],), (bad,)])
    assert e.value.status == pg.PG_ERR_INVALID_ARG


def test_autotune_picks_a_candidate(pg):
    w, pos = _small_mocks()[2]
    best, ms = pg.pg_autotune(pg.Problem.of(w), pos, candidates=(1, 2, 4))
    assert best in (1, 2, 4) and set(ms) == {1, 2, 4}
    assert all(t > 0 for t in ms.values()) and ms[best] == min(ms.values())


@pytest.mark.parametrize("n_streams", [2, 3])
def test_run_batch_streams_matches_standalone_plans(pg, n_streams):
    """The work-queue driver: runners on their own streams, with their own
    plans and scratch, claim mocks; every mock's outputs equal its standalone
    plan's bit for bit, and a mock whose problem is invalid fails alone."""
    mocks = _small_mocks()
    problems = [pg.Problem.of(w) for w, _ in mocks]
    bad = mocks[1][0]
    problems.insert(2, pg.Problem(bad.box_L, bad.mesh_n, 1, bad.s_edges, bad.n_mu,
                                  (6.0, 10.0, 0.6 * bad.box_L), 1))   # r_max >= L/2
    cats = [(p,) for _, p in mocks]
    cats.insert(2, (mocks[1][1],))
    with pytest.raises(pg.PairgalError) as e:
        pg.pg_run_batch(problems, cats, n_streams=n_streams)
    assert e.value.status == pg.PG_ERR_INVALID_ARG
    good = [p for i, p in enumerate(problems) if i != 2]
    gcat = [c for i, c in enumerate(cats) if i != 2]
    outs, lat, st = pg.pg_run_batch(good, gcat, n_streams=n_streams)
    assert np.all(np.isfinite(lat)) and st["mocks_per_s"] > 0 and st["gpu_launches"] > 0
    assert st["n_workspaces"] <= 2 * n_streams
    for (w, p), o in zip(mocks, outs):
        _same(o, pg.pg_forward_host(pg.Plan.of(w), p))
