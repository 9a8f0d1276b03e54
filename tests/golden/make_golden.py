"""Writes tests/golden/real_ngp_128_seed0.json from the FP64 oracle alone.

The workload is the 128^3 NGP real-space catalogue (L = 128 Mpc/h, ~1.2k
galaxies, s = 0-8 Mpc/h in 8 bins, r = 8-40 Mpc/h in 8 bins), seed 0. The
values are the oracle's mesh form (its own DFT), i.e. Sec. 2.1 eq.
bpg_initial with a shell W, Sec. 2.2 eq. Qeff_notsq and Sec. 3.4 eq.
2PCF_d_collapsed. Run: python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import pipeline  # noqa: E402
from paper_1705_03464_gb300 import synth  # noqa: E402


def main():
    wl = synth.WORKLOADS["real_ngp_128"]
    cat = synth.make_catalogue(wl, 0)
    out = pipeline.run(pipeline.Params.of(wl), cat.pos, form="mesh")
    keep = ["dd", "ddq", "xi_ss", "xi_gg", "xi_pg", "b_pg", "q_eff", "q_eff_sq",
            "xi_dw", "b_pg_agg", "q_eff_agg", "xi_dw_agg", "n_cells", "n_cells_agg",
            "sum_gg", "sum2_gg", "sum_pg"]
    js = {"workload": wl.name, "seed": 0, "n_gal": int(cat.n),
          "source": "oracle mesh form (oracle/pipeline.py)"}
    for k in keep:
        v = out[k]
        js[k] = v.tolist() if hasattr(v, "tolist") else v
    with open(os.path.join(HERE, "real_ngp_128_seed0.json"), "w") as f:
        json.dump(js, f, indent=0)


if __name__ == "__main__":
    main()
