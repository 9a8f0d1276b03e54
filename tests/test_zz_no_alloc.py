"""The allocation-free pair-count entry point against the plan-based one.

pg_pair_counts_static serves callers that cannot allocate device memory (a
framework's caching allocator owns the budget, or a latency-critical thread
must not take cudaMalloc's device-wide synchronisation); its scratch is a
fixed array inside the library. This file is collected last so that a run
that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    from paper_1705_03464_gb300 import build_lib
    build_lib.build(verbose=False)
    from paper_1705_03464_gb300 import pairgal
    assert torch.cuda.is_available()
    return pairgal


def test_static_scratch_counts_equal_plan_counts_twice(pg):
    from paper_1705_03464_gb300 import synth
    L = 300.0
    cat = synth.make_catalogue_box(L, 60000, seed=31)
    w = synth.make_weights(cat.n, 31)
    edges = np.linspace(0.0, 12.0, 9)
    n_mu = 3
    pos = torch.from_numpy(np.ascontiguousarray(cat.pos)).cuda()
    wt = torch.from_numpy(w).cuda()
    plan = pg.Plan(L, 64, 1, edges, n_mu, (20.0, 40.0), 1)
    ref = pg.pg_find_pairs(plan, pos, wt, with_list=False)
    assert int(ref["dd"].sum()) > 1000
    for _ in range(2):   # two calls in a row share the scratch array
        dd, ddq = pg.pg_pair_counts_static(pos, wt, L, edges, n_mu)
        torch.cuda.synchronize()
        assert torch.equal(dd, ref["dd"]) and torch.equal(ddq, ref["ddq"])
    # unweighted, different binning, then a catalogue above the fixed limit
    dd, ddq = pg.pg_pair_counts_static(pos, None, L, edges[:5], 1)
    ref2 = pg.pg_find_pairs(pg.Plan(L, 64, 1, edges[:5], 1, (20.0, 40.0), 1), pos, None,
                            with_list=False)
    assert torch.equal(dd, ref2["dd"]) and torch.equal(ddq, ref2["ddq"])
    big = torch.zeros((131073, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(pg.PairgalError) as e:
        pg.pg_pair_counts_static(big, None, L, edges, n_mu)
    assert e.value.status == pg.PG_ERR_CAPACITY


def test_static_scratch_capped_cell_list_and_single_cell(pg):
    """Where L / s_max exceeds the fixed 40 cells per side the cell list is
    capped (cells larger than s_max, still complete); where s_max is just
    above L/3 the whole box is one cell. Both against the plan path."""
    from paper_1705_03464_gb300 import synth
    L = 1000.0
    cat = synth.make_catalogue_box(L, 100000, seed=33)
    w = synth.make_weights(cat.n, 33)
    edges = np.linspace(0.0, 10.0, 6)
    pos = torch.from_numpy(np.ascontiguousarray(cat.pos)).cuda()
    wt = torch.from_numpy(w).cuda()
    ref = pg.pg_find_pairs(pg.Plan(L, 64, 1, edges, 2, (20.0, 40.0), 1), pos, wt, with_list=False)
    assert int(ref["dd"].sum()) > 1000
    dd, ddq = pg.pg_pair_counts_static(pos, wt, L, edges, 2)
    torch.cuda.synchronize()
    assert torch.equal(dd, ref["dd"]) and torch.equal(ddq, ref["ddq"])
    # one cell: s_max = 12 in a box of 30 (fewer than 3 cells per side)
    L1 = 30.0
    small = synth.make_catalogue_box(L1, 800, seed=34)
    e1 = np.linspace(0.0, 12.0, 4)
    p1 = torch.from_numpy(np.ascontiguousarray(small.pos)).cuda()
    ref1 = pg.pg_find_pairs(pg.Plan(L1, 32, 1, e1, 3, (10.0, 12.0), 1), p1, None, with_list=False)
    dd1, ddq1 = pg.pg_pair_counts_static(p1, None, L1, e1, 3)
    torch.cuda.synchronize()
    assert torch.equal(dd1, ref1["dd"]) and torch.equal(ddq1, ref1["ddq"])


def test_static_scratch_refuses_non_finite_positions(pg):
    """A NaN or Inf coordinate is refused with PG_ERR_INVALID_ARG, and the
    next valid call still gives the plan path's counts."""
    from paper_1705_03464_gb300 import synth
    L = 200.0
    cat = synth.make_catalogue_box(L, 5000, seed=35)
    edges = np.linspace(0.0, 8.0, 5)
    good = torch.from_numpy(np.ascontiguousarray(cat.pos)).cuda()
    for bad_value in (float("nan"), float("inf")):
        bad = good.clone()
        bad[1234, 1] = bad_value
        with pytest.raises(pg.PairgalError) as e:
            pg.pg_pair_counts_static(bad, None, L, edges, 2)
        assert e.value.status == pg.PG_ERR_INVALID_ARG
    ref = pg.pg_find_pairs(pg.Plan(L, 64, 1, edges, 2, (10.0, 20.0), 1), good, None, with_list=False)
    dd, ddq = pg.pg_pair_counts_static(good, None, L, edges, 2)
    torch.cuda.synchronize()
    assert torch.equal(dd, ref["dd"]) and torch.equal(ddq, ref["ddq"])
