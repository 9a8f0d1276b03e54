"""The oracle still reproduces its stored fixture (regression guard)."""
import json
import os

import numpy as np

from oracle import pipeline
from paper_1705_03464_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "real_ngp_128_seed0.json")


def test_oracle_matches_stored_fixture():
    g = json.load(open(GOLD))
    wl = synth.WORKLOADS[g["workload"]]
    cat = synth.make_catalogue(wl, g["seed"])
    assert cat.n == g["n_gal"]
    out = pipeline.run(pipeline.Params.of(wl), cat.pos, form="direct")
    assert out["dd"].tolist() == g["dd"] and out["ddq"].tolist() == g["ddq"]
    assert out["n_cells"].tolist() == g["n_cells"]
    for k in ("xi_gg", "xi_pg", "sum_gg", "sum_pg", "xi_ss"):
        np.testing.assert_allclose(out[k], np.array(g[k], dtype=float), rtol=1e-12, atol=1e-12)
