#!/usr/bin/env python
"""Benchmark of the pair-galaxy cross-correlation path.

Metric: milliseconds per mock for the whole (s, mu) x (r, mu_r) grid of
b_pg / Q_eff (forward) on the paper-scale box: L = 1100 Mpc/h, 1024^3 CIC
mesh, n = 3e-4 (h/Mpc)^3 (~4e5 galaxies), 20 x 5 pair bins, 10 x 5
correlation bins; lower is better. One step = one full forward pass over one
synthetic mock (positions -> pairs -> 100 pair meshes + galaxy mesh -> FFT
correlation -> binning -> ratios). With N GPUs every rank processes its own
mock per step (weak scaling) and value = slowest rank's step time / N.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "ms per mock for b_pg/Q_eff grid, fwd and fwd+adjoint at 1024^3; % of HBM peak"
UNIT = "ms/mock"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="paper_1024")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=3,
                    help="timed forward+adjoint steps (0 = skip)")
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="timed steps of the plain per-bin FP64 form (0 = skip)")
    ap.add_argument("--smooth-steps", type=int, default=3,
                    help="timed steps of the paper's smooth-W estimator, TSC (0 = skip)")
    ap.add_argument("--many-mocks", type=int, default=64,
                    help="uneven mocks through the batch driver (0 = skip)")
    ap.add_argument("--many-mocks-fp64", type=int, default=3,
                    help="of those, mocks also run in the plain per-bin FP64 form")
    ap.add_argument("--hod-study", type=int, default=1,
                    help="the Sec. 5 HOD-derivative workflow at the paper-scale box (0 = skip)")
    ap.add_argument("--bins-per-batch", type=int, default=0,
                    help="pair meshes resident at once (0 = the plan's default)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            js = json.load(f)
        return float(js["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel_family, workload, algorithmic_bytes_per_launch):
    """DRAM bytes per launch of one kernel family, from the committed ncu
    summary (profiles/ncu_traffic.txt: 'family workload ratio:R source'): the
    measured dram read+write bytes over the algorithmic bytes of the captured
    launch, applied to this launch's algorithmic bytes. None if absent."""
    path = os.path.join(HERE, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 3 and parts[0] == kernel_family and parts[1] == workload:
            if parts[2].startswith("ratio:"):
                try:
                    return float(parts[2][6:]) * algorithmic_bytes_per_launch
                except ValueError:
                    return None
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def device_smi_index(torch, local):
    try:
        p = torch.cuda.get_device_properties(local)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return str(local)


# ---------------------------------------------------------------- oracle legs
def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(wl, cat, gal_fraction, max_bin_pairs=1500, workers=1):
    """Times the FP64 oracle (as it stands) on a bounded sample of one mock:
    the k-d tree pair search over the whole catalogue, the direct corner sums
    of one pair bin, and the galaxy auto-correlation of a random subsample of
    galaxy a-points. With workers > 1 the corner sums run through the
    oracle's own process pool (window_C_parallel) on `workers` cores, over a
    sample `workers` times larger; the pair search stays on one core.
    Returns (extrapolated ms per mock, description)."""
    import numpy as np
    from oracle import correlate as oc, direct as od, pairs as op
    if workers > 1:
        gal_fraction *= workers
        max_bin_pairs *= workers
    L, N = wl.box_L, wl.mesh_n
    t0 = time.perf_counter()
    x = op.transform_positions(cat.pos, cat.vel, L, wl.rsd_factor)
    pr = op.find_pairs_kdtree(x, None, L, wl.s_edges, wl.n_mu)
    t_pairs = time.perf_counter() - t0
    pb = pr["sbin"] * wl.n_mu + pr["mubin"]
    counts = np.bincount(pb, minlength=(len(wl.s_edges) - 1) * wl.n_mu)
    ok = np.nonzero((counts > 0) & (counts <= max_bin_pairs))[0]
    b = int(ok[np.argmax(counts[ok])]) if ok.size else int(np.argmin(np.where(counts > 0, counts, 1 << 60)))
    w = oc.window_half(N, L, wl.r_edges[-1])
    sel = pb == b
    t1 = time.perf_counter()
    if workers > 1:
        od.window_C_parallel(pr["mid"][sel], None, x, None, L, N, wl.assign, w, wl.r_edges[-1],
                             workers=workers)
    else:
        od.window_C(pr["mid"][sel], None, x, None, L, N, wl.assign, w, wl.r_edges[-1])
    t_bin = time.perf_counter() - t1
    rng = np.random.default_rng(1)
    ns = max(1, int(min(1.0, gal_fraction) * x.shape[0]))
    sub = x[rng.choice(x.shape[0], ns, replace=False)]
    t2 = time.perf_counter()
    if workers > 1:
        od.window_C_parallel(sub, None, x, None, L, N, wl.assign, w, wl.r_edges[-1], workers=workers)
    else:
        od.window_D(sub, None, x, None, L, N, wl.assign, w, wl.r_edges[-1])
    t_gg = time.perf_counter() - t2
    n_pairs = int(counts.sum())
    est = t_pairs + t_bin / max(1, int(counts[b])) * n_pairs + t_gg * x.shape[0] / ns
    desc = (f"oracle direct corner-sum form on {workers} core(s): k-d tree pairs of all "
            f"{x.shape[0]} galaxies ({n_pairs} pairs, one core), pair bin {b} "
            f"({int(counts[b])} pairs) scaled by pair count to all bins, galaxy "
            f"auto-correlation of {ns} sampled a-points scaled to all; "
            f"sample took {t_pairs + t_bin + t_gg:.1f} s")
    return est * 1e3, desc


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from paper_1705_03464_gb300 import synth
    wl = synth.WORKLOADS[args.workload]
    cat = synth.make_catalogue(wl, args.seed)
    cores = host_cores()
    vals = []
    desc = ""
    for k in range(args.warmup + args.steps):
        v, desc = oracle_sample(wl, cat, gal_fraction=0.002, max_bin_pairs=600, workers=cores)
        if k >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": value, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "box_L": wl.box_L, "mesh_n": wl.mesh_n,
                   "n_gal": int(cat.n)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------- ranks
def mock_seed(seed, rank):
    """Each rank draws its own mock: the path shards by mock (weak scaling)."""
    return seed + rank


def max_over_ranks(x, dist, torch, device):
    """The slowest rank's value (the job's step time); x itself without ranks."""
    if not dist:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_mock(ms_per_step, world):
    """Whole-job ms per mock: every rank finishes one mock per step."""
    return ms_per_step / world


# ---------------------------------------------------------- many mocks
def _draw_mock(k):
    from paper_1705_03464_gb300 import synth
    w, hod = synth.many_mocks(1, seed0=k)[0]
    return w, synth.make_catalogue(w, k, hod).pos


def many_mocks_line(args, pg, np, torch):
    """The uneven many-mock batch: mocks/s and per-mock latency of the batch
    driver (autotuned pair meshes per batch, shared scratch, plans built
    ahead), against the plain per-mock loop (a fresh plan per mock, built
    and freed in turn, same FP32 form) and, on a few mocks, the plain
    per-bin FP64 form."""
    import multiprocessing as mp
    import tempfile
    K = args.many_mocks
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        drawn = pool.map(_draw_mock, range(K))
    t_draw = time.perf_counter() - t0
    ws = [w for w, _ in drawn]
    cats = [(pos,) for _, pos in drawn]
    stream = torch.cuda.Stream()
    # batch size per mesh size, tuned on the largest catalogue of that size
    tune = {}
    cache = os.path.join(tempfile.gettempdir(), "pairgal_tune.json")
    for N in sorted({w.mesh_n for w in ws}):
        k = max((i for i in range(K) if ws[i].mesh_n == N), key=lambda i: cats[i][0].shape[0])
        best, ms = pg.autotune_cached(pg.Problem.of(ws[k]), cats[k][0], cache_path=cache,
                                      candidates=(8, 16, 32), stream=stream)
        tune[N] = {"bins_per_batch": best, "ms": ms}
    probs = [pg.Problem.of(w, bins_per_batch=tune[w.mesh_n]["bins_per_batch"]) for w in ws]
    pg.pg_run_batch(probs[:2], cats[:2], stream=stream)   # warm-up (module load, first plans)
    torch.cuda.synchronize()
    outs, lat, st = pg.pg_run_batch(probs, cats, stream=stream)
    torch.cuda.synchronize()
    # the work-queue driver: two runners on their own streams, plans and
    # scratch; each runner holds its own scratch per mesh size, so its pair
    # meshes per batch are half the tuned count (at least 8) to fit twice
    probs2 = [pg.Problem.of(w, bins_per_batch=max(8, tune[w.mesh_n]["bins_per_batch"] // 2)) for w in ws]
    try:
        outs2, lat2, st2 = pg.pg_run_batch(probs2, cats, stream=stream, n_streams=2)
        torch.cuda.synchronize()
        same2 = all(np.array_equal(np.asarray(a["b_pg"]), np.asarray(b["b_pg"]), equal_nan=True)
                    for a, b in zip(outs, outs2))
        del outs2
        two = {"mocks_per_s": st2["mocks_per_s"], "p50_ms": st2["p50_ms"], "p99_ms": st2["p99_ms"],
               "wall_s": st2["wall_ms"] / 1e3, "shared_scratch": st2["n_workspaces"],
               "bins_per_batch": {str(N): max(8, tune[N]["bins_per_batch"] // 2) for N in tune},
               "outputs_equal_one_stream": bool(same2),
               "form": "pg_run_batch_streams: two runners claim mocks from one work queue"}
    except pg.PairgalError as e:
        two = {"mocks_per_s": None, "error": str(e)}
    # the plain per-mock loop
    loop_ms = []
    t1 = time.perf_counter()
    for w, c in zip(ws, cats):
        a = time.perf_counter()
        plan = pg.Plan.of(w)
        pg.pg_forward_host(plan, c[0], stream=stream)
        plan.close()
        loop_ms.append(1e3 * (time.perf_counter() - a))
    loop_wall = time.perf_counter() - t1
    # the plain per-bin FP64 form on the first few mocks
    n64 = min(args.many_mocks_fp64, K)
    fp64_ms, diff = [], 0.0
    for i in range(n64):
        a = time.perf_counter()
        plan = pg.Plan.of(ws[i], precision=1, bins_per_batch=1)
        r64 = pg.pg_forward_host(plan, cats[i][0], stream=stream)
        plan.close()
        fp64_ms.append(1e3 * (time.perf_counter() - a))
        b, c = np.asarray(outs[i]["b_pg"]), np.asarray(r64["b_pg"])
        ok = np.isfinite(b) & np.isfinite(c)
        if ok.any():
            diff = max(diff, float(np.max(np.abs(b[ok] - c[ok]) / np.maximum(np.abs(c[ok]), 1e-300))))
    Ns = [w.mesh_n for w in ws]
    return {
        "mocks": K, "meshes": {str(N): Ns.count(N) for N in sorted(set(Ns))},
        "n_gal_range": [int(min(c[0].shape[0] for c in cats)), int(max(c[0].shape[0] for c in cats))],
        "mocks_per_s": st["mocks_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
        "wall_s": st["wall_ms"] / 1e3, "plans": st["n_plans"], "shared_scratch": st["n_workspaces"],
        "gpu_launches": st["gpu_launches"], "bins_per_batch": tune,
        "two_streams": two,
        "plain_loop": {"mocks_per_s": K / loop_wall, "p50_ms": float(np.percentile(loop_ms, 50)),
                       "p99_ms": float(np.percentile(loop_ms, 99)),
                       "form": "a fresh FP32 plan per mock, built, run and freed in turn"},
        "plain_fp64": {"mocks": n64, "ms": fp64_ms,
                       "batched_ms_same_mocks": [float(x) for x in lat[:n64]],
                       "max_rel_diff_b_pg": diff},
        "draw_s": t_draw, "latency": "a mock's turn (its plan wait included) to its results on the host",
    }


def summary(value, fwd_adj, plain, smooth, many, cpu, roofline, breakdown, peak, hod=None):
    """Compact figures of every leg: forward and forward+adjoint ms per
    mock, the FP64 plain form, the smooth-W estimator, the many-mock batch,
    the oracle on one and all cores, and each kernel family's fraction of
    the HBM peak (algorithmic bytes over CUDA-event time)."""
    r = lambda x, d=1: None if x is None else round(float(x), d)
    out = {"fwd_ms": r(value), "fwd_adj_ms": None, "fwd_adj_over_fwd": None}
    if fwd_adj:
        out["fwd_adj_ms"] = r(fwd_adj["ms_per_mock"])
        out["fwd_adj_over_fwd"] = r(fwd_adj["ratio_to_fwd"], 3)
    if plain:
        out["plain_fp64_ms"] = r(plain["ms_per_mock"])
        out["fp32_batched_speedup"] = r(plain["speedup_of_fp32_batched"], 2)
    if smooth:
        out["smooth_w_ms"] = r(smooth["ms_per_mock"])
        out["smooth_w_fwd_adj_ms"] = r(smooth["fwd_adj_ms_per_mock"])
        if "rsd_dp30_grid" in smooth:
            out["smooth_w_rsd_dp30_ms"] = r(smooth["rsd_dp30_grid"]["ms_per_mock"])
    if many:
        out["many_mocks_per_s"] = r(many["mocks_per_s"], 2)
        out["many_mocks_per_s_two_streams"] = r(many["two_streams"]["mocks_per_s"], 2)
        out["many_p50_p99_ms"] = [r(many["p50_ms"]), r(many["p99_ms"])]
        out["plain_loop_mocks_per_s"] = r(many["plain_loop"]["mocks_per_s"], 2)
    if hod:
        out["hod_emulator_ms"] = r(hod["emulator_ms"], 2)
        out["hod_14_evaluations_ms"] = r(hod["fourteen_evaluations_ms"], 2)
        out["hod_delta_q_eff_ms"] = r(hod["delta_q_eff_ms"])
    if cpu:
        out["oracle_ms"] = {f"{cpu['cores']}_cores": r(cpu["value"], 0),
                            "1_core": r(cpu["one_core"]["value"], 0)}
    out["top_kernel_frac"] = r(roofline.get("frac"), 3)
    out["hbm_frac"] = {k: r(v["GBps"] / peak, 2) for k, v in breakdown.items()
                       if v.get("GBps") and v["ms_per_step"] >= 0.5}
    return out


def hod_study_line(wl, pg, np, torch, share_with):
    """Sec. 5 at the paper-scale box (L = 1100 Mpc/h, 1024^3): soft HOD
    candidates around the Z09 design; the emulator of w(d_perp) on a
    20 x 5 (d_perp, d_par) grid to 30 Mpc/h with exact first and second
    derivatives in (log10 M_cut, log10 M_1, sigma, alpha), against the 14
    separate evaluations the paper uses (timed here as 14 evaluations of the
    same statistic); the alpha = 1.05 and 0.95 fits with the paper's error
    model; delta Q_eff and delta xi from three redshift-space smooth-W
    forwards (d_p,max = 30 weighting, TSC) on the same grid."""
    from paper_1705_03464_gb300 import hod_study as hs, synth
    th0 = np.array(synth.HOD_Z09, dtype=np.float64)
    cand = synth.make_candidates(wl.box_L, wl.n_gal, seed=0)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    P, V, M, K, H = dev(cand.pos), dev(cand.vel), dev(cand.mass), dev(cand.kind), dev(cand.kh)
    perp = tuple(np.linspace(0.0, 30.0, 21))
    par = tuple(np.linspace(0.0, 30.0, 6))
    gp = pg.Plan(wl.box_L, wl.mesh_n, 1, perp, len(par) - 1, wl.r_edges, wl.n_mur, par_edges=par,
                 share_with=share_with)
    hs.emulator(gp, P, None, M, K, H, th0)   # warm-up
    em = hs.emulator(gp, P, None, M, K, H, th0)
    # the paper's route: 14 evaluations of the statistic at distinct HODs,
    # each its least work on this path (soft weights and weighted pair
    # counts, from which xi and w(d_perp) follow)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(14):
        th = th0.copy()
        th[k % 4] += 0.01 * (1 + k // 4)
        w, _ = pg.pg_hod_weights(M, K, H, th, with_grad=False)
        pg.pg_find_pairs(gp, P, w, with_list=False)
    torch.cuda.synchronize()
    ms14 = 1e3 * (time.perf_counter() - t0)
    t1 = time.perf_counter()
    fits = {a: hs.fit_at_alpha(em, a, perp, 30.0) for a in (1.05, 0.95)}
    fit_s = time.perf_counter() - t1
    sp = pg.Plan(wl.box_L, wl.mesh_n, 2, perp, len(par) - 1, wl.r_edges, wl.n_mur,
                 rsd_factor=synth.RSD_FACTOR_Z05, par_edges=par, share_with=share_with)
    hs.delta_q_eff(sp, pg.W_DP30, P, V, M, K, H, fits[1.05][0], fits[0.95][0], th0)   # warm-up
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    dq, dx, _ = hs.delta_q_eff(sp, pg.W_DP30, P, V, M, K, H, fits[1.05][0], fits[0.95][0], th0)
    torch.cuda.synchronize()
    dq_ms = 1e3 * (time.perf_counter() - t2)
    sp.close()
    gp.close()
    fin = lambda a: np.asarray(a)[np.isfinite(a)]
    return {"candidates": int(cand.pos.shape[0]), "grid": "d_perp 0-30 (20) x |d_par| 0-30 (5)",
            "emulator_ms": em["ms"], "fourteen_evaluations_ms": ms14,
            "fit_s": fit_s, "fits": {str(a): {"theta": [round(float(t), 4) for t in f[0]], "chi2": f[1]}
                                     for a, f in fits.items()},
            "delta_q_eff_ms": dq_ms, "max_abs_delta_q_eff": float(np.max(np.abs(fin(dq)))),
            "max_abs_delta_xi": float(np.max(np.abs(fin(dx))))}


# ---------------------------------------------------------------- our path
def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1705_03464_gb300 import build_lib
    if rank == 0:
        build_lib.build(verbose=False)
    if dist:
        dist.barrier()
    from paper_1705_03464_gb300 import pairgal as pg, synth

    wl = synth.WORKLOADS[args.workload]
    cat = synth.make_catalogue(wl, mock_seed(args.seed, rank))
    pos = torch.from_numpy(cat.pos).cuda()
    vel = torch.from_numpy(np.ascontiguousarray(cat.vel)).cuda() if wl.rsd else None
    plan = pg.Plan.of(wl, **({"bins_per_batch": args.bins_per_batch} if args.bins_per_batch else {}))
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        out = pg.pg_forward(plan, pos, vel, stream=stream)
    n_pairs = int(out["dd"].sum())

    plan.set_profiling(True)
    fam_ms, fam_bytes, fam_launch = {}, {}, {}
    launches = 0
    sampler = ClockSampler(device_smi_index(torch, local))
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        out = pg.pg_forward(plan, pos, vel, stream=stream)
        fams, nl = plan.last_stats()
        launches += nl
        for k, v in fams.items():
            fam_ms[k] = fam_ms.get(k, 0.0) + v["ms"]
            fam_bytes[k] = fam_bytes.get(k, 0.0) + v["bytes"]
            fam_launch[k] = fam_launch.get(k, 0) + v["launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    t_ms = max_over_ranks(e0.elapsed_time(e1), dist, torch, "cuda")
    plan.set_profiling(False)
    ms_per_step = t_ms / args.steps
    value = per_mock(ms_per_step, world)

    # end to end through the host-buffer entry point: pinned inputs in,
    # result arrays out, both copies inside the timed region
    e2e = None
    if not args.no_e2e:
        pos_h = torch.from_numpy(cat.pos).pin_memory()
        vel_h = torch.from_numpy(np.ascontiguousarray(cat.vel)).pin_memory() if wl.rsd else None
        ph, vh = pos_h.numpy(), (vel_h.numpy() if vel_h is not None else None)
        h2d = ph.nbytes + (vh.nbytes if vh is not None else 0)
        res, arrs = plan.new_result()
        d2h = sum(a.nbytes for a in arrs.values())
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(args.steps):
            pg.pg_forward_host(plan, ph, vh, None, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        te = max_over_ranks(a0.elapsed_time(a1), dist, torch, "cuda")
        e2e = {"value": per_mock(te / args.steps, world), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "wall_s": time.perf_counter() - t0}

    # forward + adjoint: dL/dw of every galaxy weight for L = sum(b_pg) +
    # sum(Q_eff), the spectra recomputed in the backward pass
    fwd_adj = None
    if args.adjoint_steps > 0:
        grads = {k: np.ones(np.asarray(out[k]).shape) for k in ("b_pg", "q_eff")}
        pg.pg_forward(plan, pos, vel, stream=stream)
        pg.pg_backward(plan, grads, int(cat.n), stream=stream)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(args.adjoint_steps):
            pg.pg_forward(plan, pos, vel, stream=stream)
            wbar = pg.pg_backward(plan, grads, int(cat.n), stream=stream)
        b1.record(stream)
        torch.cuda.synchronize()
        tb = max_over_ranks(b0.elapsed_time(b1), dist, torch, "cuda")
        # one more forward + backward (outside the timed steps), the backward
        # with per-family event timing: the same sequence as a timed step
        pg.pg_forward(plan, pos, vel, stream=stream)
        plan.set_profiling(True)
        pg.pg_backward(plan, grads, int(cat.n), stream=stream)
        bfams, bl = plan.last_stats()
        plan.set_profiling(False)
        fwd_adj = {"ms_per_mock": per_mock(tb / args.adjoint_steps, world), "steps": args.adjoint_steps,
                   "ratio_to_fwd": per_mock(tb / args.adjoint_steps, world) / value,
                   "loss": "sum(b_pg) + sum(q_eff)",
                   "grad_finite": bool(torch.isfinite(wbar).all().item()),
                   "backward_launches": bl,
                   "backward_kernels": {k: {"ms": v["ms"],
                                            "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                                        for k, v in bfams.items() if v["launches"] > 0}}

    # the plain form: FP64 FFT passes, one pair mesh per batch, same inputs;
    # reported as the speedup of the batched FP32 form and the largest
    # relative differences between the two forms' outputs
    plain = None
    if args.plain_steps > 0:
        plan64 = pg.Plan.of(wl, precision=1, bins_per_batch=1)
        ref64 = pg.pg_forward(plan64, pos, vel, stream=stream)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.plain_steps):
            ref64 = pg.pg_forward(plan64, pos, vel, stream=stream)
        c1.record(stream)
        torch.cuda.synchronize()
        tp = max_over_ranks(c0.elapsed_time(c1), dist, torch, "cuda")
        del plan64
        torch.cuda.empty_cache()

        def rel(k):
            a, b = np.asarray(out[k], np.float64), np.asarray(ref64[k], np.float64)
            ok = np.isfinite(a) & np.isfinite(b)
            return float(np.max(np.abs(a[ok] - b[ok]) / np.maximum(np.abs(b[ok]), 1e-300))) if ok.any() else None

        plain_ms = per_mock(tp / args.plain_steps, world)
        plain = {"ms_per_mock": plain_ms, "steps": args.plain_steps,
                 "form": "FP64 FFT passes, one pair mesh per batch",
                 "speedup_of_fp32_batched": plain_ms / value,
                 "fp32_vs_fp64_max_rel": {k: rel(k) for k in ("xi_gg", "xi_pg", "b_pg", "q_eff", "b_pg_agg")}}

    # the paper's own estimator (eq. bpg_final with the Gauss-sigmoid W of
    # Table tab:weightings, d_p,max = 10 Mpc/h) with TSC assignment, on the same
    # catalogue: all pair bins from one convolution
    smooth = None
    if args.smooth_steps > 0:
        sp = pg.Plan.of(wl, assign=2, share_with=plan)
        r = pg.pg_forward_smooth(sp, pg.W_DP10, pos, vel, stream=stream)   # warm-up, W's spectrum
        pg.pg_forward_smooth(sp, pg.W_DP10, pos, vel, stream=stream)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for _ in range(args.smooth_steps):
            r = pg.pg_forward_smooth(sp, pg.W_DP10, pos, vel, stream=stream)
        d1.record(stream)
        torch.cuda.synchronize()
        ts = max_over_ranks(d0.elapsed_time(d1), dist, torch, "cuda")
        sp.set_profiling(True)
        pg.pg_forward_smooth(sp, pg.W_DP10, pos, vel, stream=stream)
        sfams, sl = sp.last_stats()
        sp.set_profiling(False)
        # the adjoint (dL/dw for every galaxy, L = sum b_pg + sum q_eff): forward
        # + backward per step, timed the same way
        sg = {"b_pg": np.ones(sp.P), "q_eff": np.ones(sp.P)}
        pg.pg_backward_smooth(sp, sg, int(cat.n), stream=stream)   # warm-up (adjoint scratch)
        torch.cuda.synchronize()
        d0.record(stream)
        for _ in range(args.smooth_steps):
            pg.pg_forward_smooth(sp, pg.W_DP10, pos, vel, stream=stream)
            gw = pg.pg_backward_smooth(sp, sg, int(cat.n), stream=stream)
        d1.record(stream)
        torch.cuda.synchronize()
        tsa = max_over_ranks(d0.elapsed_time(d1), dist, torch, "cuda")
        b = np.asarray(r["b_pg"])
        smooth = {"ms_per_mock": per_mock(ts / args.smooth_steps, world), "steps": args.smooth_steps,
                  "fwd_adj_ms_per_mock": per_mock(tsa / args.smooth_steps, world),
                  "fwd_adj_ratio": tsa / ts, "grad_finite": bool(torch.isfinite(gw).all().item()),
                  "assign": "tsc", "w": {"sigma": 30.0, "r_s": 20.0, "s0": 0.8, "r_cut": 10.0},
                  "xi_dw": r["xi_dw"], "b_pg_range": [float(np.nanmin(b)), float(np.nanmax(b))],
                  "launches": sl,
                  "kernels": {k: {"ms": v["ms"],
                                  "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                              for k, v in sfams.items() if v["launches"] > 0}}
        sp.close()
        del sp
        # the paper's redshift-space configuration (d_p,max = 30 Mpc/h, W of
        # Table tab:weightings row 2) on the (d_perp, d_par) grid of its
        # redshift-space b_pg / Q_eff maps, positions displaced along z
        vz = torch.from_numpy(np.ascontiguousarray(cat.vel)).cuda()
        perp = tuple(np.linspace(0.0, 30.0, 21))
        par = tuple(np.linspace(0.0, 30.0, 6))
        sg30 = pg.Plan(wl.box_L, wl.mesh_n, 2, perp, len(par) - 1, wl.r_edges, wl.n_mur,
                       rsd_factor=synth.RSD_FACTOR_Z05, par_edges=par, share_with=plan)
        r30 = pg.pg_forward_smooth(sg30, pg.W_DP30, pos, vz, stream=stream)   # warm-up, W's spectrum
        torch.cuda.synchronize()
        d0.record(stream)
        for _ in range(args.smooth_steps):
            r30 = pg.pg_forward_smooth(sg30, pg.W_DP30, pos, vz, stream=stream)
        d1.record(stream)
        torch.cuda.synchronize()
        t30 = max_over_ranks(d0.elapsed_time(d1), dist, torch, "cuda")
        b30 = np.asarray(r30["b_pg"])
        smooth["rsd_dp30_grid"] = {
            "ms_per_mock": per_mock(t30 / args.smooth_steps, world), "assign": "tsc",
            "w": {"sigma": 50.0, "r_s": 35.0, "s0": 0.5, "r_cut": 20.0},
            "pair_grid": "d_perp 0-30 (20) x |d_par| 0-30 (5)", "n_pairs": int(np.sum(r30["dd"])),
            "xi_dw": r30["xi_dw"], "b_pg_range": [float(np.nanmin(b30)), float(np.nanmax(b30))]}
        sg30.close()
        del sg30, vz

    hod = None
    if args.hod_study > 0:
        hod = hod_study_line(wl, pg, np, torch, plan)

    many = None
    if args.many_mocks > 0 and rank == 0 and world == 1:
        del plan
        torch.cuda.empty_cache()
        many = many_mocks_line(args, pg, np, torch)

    peak, peak_src = peaks()
    top = max(fam_ms, key=lambda k: fam_ms[k])
    achieved = fam_bytes[top] / (fam_ms[top] * 1e-3) / 1e9 if fam_ms[top] > 0 else None
    traffic = ncu_traffic(top, wl.name, fam_bytes[top] / max(1, fam_launch[top]))
    roofline = {"bound": "hbm", "kernel": top, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": traffic, "peak_source": peak_src,
                "bytes_per_launch": fam_bytes[top] / max(1, fam_launch[top]),
                "ms_per_launch": fam_ms[top] / max(1, fam_launch[top])}
    breakdown = {k: {"ms_per_step": fam_ms[k] / args.steps,
                     "GBps": (fam_bytes[k] / (fam_ms[k] * 1e-3) / 1e9) if fam_ms[k] > 0 else None,
                     "launches_per_step": fam_launch[k] / args.steps}
                 for k in fam_ms}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc = oracle_sample(wl, cat, gal_fraction=0.005)
        cores = host_cores()
        vall, dall = oracle_sample(wl, cat, gal_fraction=0.005, workers=cores)
        cpu = {"value": vall, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": dall,
               "one_core": {"value": v, "cores": 1, "sample": desc}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "box_L": wl.box_L, "mesh_n": wl.mesh_n,
                       "assign": "cic" if wl.assign else "ngp", "n_gal": int(cat.n),
                       "n_pairs": n_pairs, "pair_bins": f"{len(wl.s_edges) - 1}x{wl.n_mu}",
                       "corr_bins": f"{len(wl.r_edges) - 1}x{wl.n_mur}",
                       "precision": "fp32 FFT passes, fp64 positions/pairs/reductions/ratios",
                       "l2": "no flush: each step streams ~70 GB of spectra, far above the 129 MB L2",
                       "mocks_per_step": world},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches), "clocks": clocks, "kernels": breakdown,
            "hod_study": hod, "many_mocks": many, "smooth_w": smooth, "plain_fp64": plain,
            "fwd_adj": fwd_adj,
        }
        # the line ends with a short summary of every leg, so that a reader
        # who keeps only its last characters still sees the whole metric
        line["summary"] = summary(value, fwd_adj, plain, smooth, many, cpu, roofline, breakdown, peak, hod)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
