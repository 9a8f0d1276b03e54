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
