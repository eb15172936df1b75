"""Benchmark: candidates evaluated per second and time-to-optimal reduction of the
exhaustive Kron-based search (Algorithm 1) on the 1,000-bus synthetic feeder.

One step = one full reduction through the C ABI: load flow of both scenarios,
renumbering/LCA/path impedances, the search to 50 % reduction (or until no
candidate is feasible), and the result export, on inputs already resident in
HBM (``okr_reduce_device``).  ``e2e`` repeats the measurement through
``okr_reduce`` from pinned host buffers, with the result read back.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank reduces its own replica of the workload (the search of
one feeder is one sequential chain of merges; replicas scale weakly).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidates evaluated/s & time-to-optimal reduction, 1000-node feeder vs FP64"
WORKLOAD = "feeder1000"
# FP32 ALU peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flop per FMA x 2.07 GHz
# (the search's counted arithmetic is its FP32 candidate terms)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# algorithmic FP operations per (candidate, kept phase-node, scenario) item: the
# 3-term complex product of the voltage change, the magnitude change, the error
# against the cluster extremes, a max and a sum
FLOPS_PER_ITEM = 40
# DRAM bytes of one search launch on this workload from the ncu capture in
# profiles/, valid only for the kernel source it was taken on (None otherwise)
NCU_TRAFFIC = {"bytes": 1166336 + 768, "source": "paper_2510_19608_gb300/csrc/okr_incr.cu",
               "sha256_prefix": "56d4cc024db929ed", "summary": "profiles/k_search_inc_feeder1000.md"}
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2

# Latency floor of one merge of the incremental search.  One merge is a chain
# of phases, each of which needs the previous one's result: selection, the
# merge's own FP64 evaluation (beside the changed-set scan), the rebuilt
# candidates, the terms that change.  The floor takes, per phase, its longest
# chain of dependent steps at the latencies measured on a GB300 (one-off
# clock64 probes, one CTA of 512 threads), with unlimited parallelism inside a
# phase.  Cycles:
PRIM_CYCLES = {"l2": 290,        # dependent L2 load (ld.global.cg, 8 MB footprint)
               "l1": 47,         # dependent load through L1 / shared memory, data the CTA wrote
               "bar": 48,        # __syncthreads of 512 threads arriving together
               "dfma": 64,       # dependent DFMA
               "dsqrt_add": 675,  # dependent FP64 square root + add
               "ffma": 4}        # dependent FFMA (nominal)
MERGE_CHAIN = {
    # two block reductions over the selection records, then the winner's candidate
    "select": lambda c: 2 * (c["l1"] + c["bar"]) + c["l2"],
    # position -> lca -> path impedance -> 3-term complex product (6 dependent
    # DFMAs) -> magnitude -> barrier
    "merge_eval": lambda c: c["l1"] + 2 * c["l2"] + 6 * c["dfma"] + c["dsqrt_add"] + c["bar"],
    # a rebuilt pair: label -> parent's cluster -> lca -> child offsets -> child
    # search -> subtree size (six dependent L2 loads), then a barrier
    "rebuild": lambda c: 6 * c["l2"] + c["bar"],
    # offsets scan (two barriers), entry lookup (four shared loads), state, lca
    # and path-impedance loads, one FP32 term (about 40 dependent operations),
    # the sums' shared update, a barrier, the carried sum's load, a barrier
    "terms": lambda c: 2 * c["bar"] + 4 * c["l1"] + 3 * c["l2"] + 40 * c["ffma"] + c["bar"] + c["l2"] + c["bar"],
}
SM_CLOCK_HZ = 2.07e9


def merge_floor_us(clock_hz: float = SM_CLOCK_HZ) -> tuple[float, dict]:
    """Latency floor of one merge (µs) and its per-phase cycles."""
    cyc = {k: f(PRIM_CYCLES) for k, f in MERGE_CHAIN.items()}
    return sum(cyc.values()) / clock_hz * 1e6, cyc


def _ncu_traffic():
    """Per-launch DRAM bytes from the committed ncu capture, or None when the
    kernel source has changed since it was taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, NCU_TRAFFIC["source"]), "rb") as fh:
            h = hashlib.sha256(fh.read()).hexdigest()
    except OSError:
        return None
    if not NCU_TRAFFIC["sha256_prefix"] or NCU_TRAFFIC["bytes"] is None:
        return None
    return NCU_TRAFFIC["bytes"] if h.startswith(NCU_TRAFFIC["sha256_prefix"]) else None


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-feeder batch measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-scorer training and evaluation")
    ap.add_argument("--no-large", action="store_true", help="skip the 2,200- and 3,100-bus rows and their CPU baseline")
    ap.add_argument("--cpu-repeats", type=int, default=3, help="oracle runs per CPU baseline (median)")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (the job's time is its slowest
    replica's); the identity on a single process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_step: float, steps: int, world: int, slowest_ms: float) -> float:
    """Whole-job throughput of `world` replicas that each processed
    units_per_step units per step for `steps` steps, timed by the slowest."""
    return world * units_per_step * steps / (slowest_ms / 1e3)


def _workload_config(f, run):
    return {"workload": f"{WORKLOAD}: {f.n_bus} buses ({f.n_phase_nodes} phase nodes), 12.47 kV, "
                        f"{f.n_scen} loading scenarios, target {int(run['target'] * 100)}% reduction, "
                        f"margin {run['margin']} p.u.",
            "n_bus": f.n_bus, "n_phase_nodes": f.n_phase_nodes, "scenarios": f.n_scen,
            "target_reduction": run["target"], "margin_pu": run["margin"], "seed": f.meta["seed"]}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = open(os.devnull, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                data, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                data, _ = self.proc.communicate()
            self.lines = [l for l in data.splitlines() if l.strip()]

    def summary(self):
        if not self.lines:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            c = [x.strip() for x in line.split(",")]
            try:
                sm.append(float(c[1]))
                smax.append(float(c[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(f, run, repeats=3):
    """The CPU oracle (delta mode, FP64, OpenMP over candidates) on the same
    feeder: the full reduction, median of `repeats` runs."""
    from oracle import oracle as O
    vhat, ihat = O.operating_points(f)
    merges = O.max_merges_for(f.n_bus, run["target"])
    times = []
    for _ in range(max(1, repeats)):
        t0 = time.perf_counter()
        res = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=merges)
        times.append(time.perf_counter() - t0)
    dt = statistics.median(times)
    cores = O.num_threads()
    # the same oracle on one thread (first 50 merges), and its literal mode
    # (a full network solve per candidate) on the 40-bus case
    O.set_threads(1)
    try:
        t1 = time.perf_counter()
        r1 = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=min(merges, 50))
        d1 = time.perf_counter() - t1
        import feedergen as fg
        f40, run40 = fg.preset("feeder40")
        v40, i40 = O.operating_points(f40)
        t2 = time.perf_counter()
        r40 = O.reduce(f40, v40, i40, margin=run40["margin"], max_merges=f40.n_bus - 1, mode="literal")
        d2 = time.perf_counter() - t2
    finally:
        O.set_threads(cores)
    return {"value": res["candidates"] / dt, "unit": "candidates/s", "cores": cores, "kind": "oracle",
            "sample": f"full {WORKLOAD} reduction ({res['n_iter']} merges, {res['candidates']} candidates) "
                      f"in {dt:.2f} s, delta mode, median of {len(times)}", "seconds": dt, "merges": int(res["n_iter"]),
            "one_thread": {"value": r1["candidates"] / d1, "unit": "candidates/s", "cores": 1,
                           "sample": f"first {r1['n_iter']} merges of {WORKLOAD}, delta mode", "seconds": d1},
            "literal_feeder40": {"value": r40["candidates"] / d2, "unit": "candidates/s", "cores": 1,
                                 "sample": f"feeder40 until infeasible ({r40['n_iter']} merges), literal mode",
                                 "seconds": d2}}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle (the paper ships no code; the oracle is
    the plain FP64 statement of Algorithm 1) timed on the host cores on the
    same workload as our arm, one full reduction per step."""
    import feedergen as fg
    from oracle import oracle as O
    if rank != 0:
        return
    f, run = fg.preset(WORKLOAD)
    vhat, ihat = O.operating_points(f)
    merges = O.max_merges_for(f.n_bus, run["target"])
    for _ in range(args.warmup):
        O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=merges)
    times, cands = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=merges)
        times.append(time.perf_counter() - t0)
        cands += r["candidates"]
    total = sum(times)
    value = cands / total
    line = {"metric": METRIC, "value": value, "unit": "candidates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _workload_config(f, run),
            "step": f"one full reduction ({r['n_iter']} merges) by the CPU oracle, delta mode",
            "cpu_baseline": {"value": value, "unit": "candidates/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"full {WORKLOAD} reduction per step ({r['n_iter']} merges), delta mode"},
            "e2e": {"value": value, "unit": "candidates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_line(K, ctx, reps=3):
    """Many-feeder workload: 256 seeded feeders, n ~ U[200, 2000], targets in
    {50, 70, 90} %, margin 0.005, reduced by okr_reduce_batch: the incremental
    engine (one CTA per feeder) and the sweep engine (one persistent launch,
    autotuned teams), each with FP32 terms (FP64 rescoring and merges) and in
    plain FP64.  Inputs (about 1 GB of device buffers) exceed L2, so no flush
    is needed between repetitions."""
    import feedergen as fg
    batch = fg.batch_presets(256)
    feeders = [f for f, _ in batch]
    out = {"workload": "256 feeders, n ~ U[200, 2000] buses (sum %d), targets {50, 70, 90} %%, margin 0.005 p.u., "
                       "2 scenarios" % sum(f.n_bus for f in feeders)}
    rows = (("incremental_mixed", 2, 1), ("incremental_fp64", 2, 0), ("sweep_mixed", 1, 1), ("sweep_fp64", 1, 0))
    for key, engine, prec in rows:
        plist = [K.default_params(margin=r["margin"], target_reduction=r["target"], precision=prec, engine=engine)
                 for _, r in batch]
        if key == "sweep_mixed":
            cfg, ms = ctx.batch_autotune(feeders, plist)
            out["autotune"] = {"config": cfg, "search_ms_by_config": [round(x, 3) for x in ms],
                               "configs": ["1 CTA per feeder", "2 CTAs", "4 CTAs", "8 CTAs"]}
        ctx.reduce_batch(feeders, plist, want_assignment=False)          # warm-up
        walls, dev_ms, st = [], [], None
        for _ in range(reps):
            t0 = time.perf_counter()
            items, _, st = ctx.reduce_batch(feeders, plist, want_assignment=True)
            walls.append(time.perf_counter() - t0)
            dev_ms.append(st["setup_ms"] + st["search_ms"])
        bad = sum(1 for it in items if it["status"] != 0)
        wall = statistics.median(walls)
        dms = statistics.median(dev_ms)
        out[key] = {"feeders_per_s": len(feeders) / (dms / 1e3), "candidates_per_s": st["candidates"] / (dms / 1e3),
                    "device_ms": dms, "setup_ms": st["setup_ms"], "search_ms": st["search_ms"],
                    "e2e_feeders_per_s": len(feeders) / wall, "e2e_ms": 1e3 * wall,
                    "candidates": st["candidates"], "ctas": st["ctas"], "fallbacks": st["fallbacks"],
                    "failed_feeders": bad}
        if key == "incremental_mixed":
            # the same batch captured once as a CUDA graph and replayed
            plan = ctx.batch_plan(feeders, plist)
            try:
                plan.run()                                                # warm-up
                walls, dev_ms = [], []
                for _ in range(reps):
                    t0 = time.perf_counter()
                    items, _, st = plan.run()
                    walls.append(time.perf_counter() - t0)
                    dev_ms.append(st["setup_ms"] + st["search_ms"])
            finally:
                plan.close()
            wall = statistics.median(walls)
            dms = statistics.median(dev_ms)
            out["incremental_mixed_graph"] = {
                "feeders_per_s": len(feeders) / (dms / 1e3), "device_ms": dms, "e2e_feeders_per_s": len(feeders) / wall,
                "e2e_ms": 1e3 * wall, "failed_feeders": sum(1 for it in items if it["status"] != 0),
                "note": "okr_batch_plan_run: input copy, setup, search and result copies replayed as one CUDA graph"}
    return out


def learned_line(K, ctx, n_train=64, record=64):
    """Learned scorer: trained on the GPU on the exhaustive-search scores of the
    first `record` iterations of 64 seeded feeders (500-2,000 buses, the
    45/15/40 % phase mix, lognormal loads), then ranked against the exhaustive
    search on the first iterations of the 3,100-bus stand-in: how often the
    committed candidate falls outside the top-k predictions."""
    import numpy as np
    import feedergen as fg
    from paper_2510_19608_gb300 import scorer
    runs = []
    for k in range(n_train):
        n = int(np.random.default_rng(10000 + k).integers(500, 2001))
        f = fg.make_feeder(n, 10000 + k, phase_mode=(0.45, 0.15, 0.4), load=("lognormal", 15.0, 1.0),
                           pf_range=(0.85, 0.99))
        runs.append((f, K.default_params(margin=0.005, target_reduction=0.8, max_merges=record)))
    t0 = time.perf_counter()
    X, T, _ = scorer.collect(ctx, runs, record)
    t_collect = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = scorer.train(ctx, X, T, epochs=8, batch=8192, lr=1e-3, seed=0)
    t_train = time.perf_counter() - t0
    trained = ctx.scorer_params().copy()
    f3, run3 = fg.preset("feeder3100")
    Xt, Tt, groups = scorer.collect(ctx, [(f3, K.default_params(margin=run3["margin"], target_reduction=run3["target"],
                                                                max_merges=record))], record)
    t0 = time.perf_counter()
    q = scorer.miss_rate(ctx, Xt, groups, ks=(16, 64, 256), T=Tt, margin=run3["margin"])
    t_eval = time.perf_counter() - t0
    # the search with learned pruning against the exhaustive search, full runs
    pruned = {}
    for name in ("feeder3100", "feeder2200", WORKLOAD):
        fx, rx = fg.preset(name)
        rows = {}
        # (name, top-k, engine, precision, certified pruning, trained weights)
        for key, k, engine, prec, exact, tw in (("exhaustive_incremental", 0, 2, 1, 0, 1),
                                                ("exhaustive_sweep", 0, 1, 1, 0, 1),
                                                ("top64", 64, 1, 1, 0, 1), ("top16", 16, 1, 1, 0, 1),
                                                ("exhaustive_sweep_fp64", 0, 1, 0, 0, 1),
                                                ("certified_top64_fp64", 64, 1, 0, 1, 1),
                                                ("certified_top64_fp64_untrained", 64, 1, 0, 1, 0)):
            ctx.scorer_init(X.shape[1], trained if tw else scorer.init_params(X.shape[1], 5))
            px = K.default_params(margin=rx["margin"], target_reduction=rx["target"], precision=prec, scorer_topk=k,
                                  engine=engine, prune_exact=exact)
            ctx.reduce(fx, px)                                        # warm-up
            times = []
            for _ in range(3):
                t0 = time.perf_counter()
                ctx.reduce(fx, px)
                times.append(time.perf_counter() - t0)
            sm = ctx.summary()
            rows[key] = {
                "ms": 1e3 * statistics.median(times), "search_ms": sm["search_ms"], "merges": sm["n_iter"],
                "stop_reason": sm["stop_reason"], "smice": sm["smice"], "max_error": sm["max_error"],
                "fallbacks": sm["scorer_fallbacks"]}
            if exact:
                rows[key]["pruned_fraction"] = sm["pruned"] / max(1, sm["candidates"])
                rows[key]["candidates_scored"] = sm["candidates"] - sm["pruned"]
                rows[key]["same_decisions_as_exhaustive_fp64"] = (
                    sm["smice"] == rows["exhaustive_sweep_fp64"]["smice"]
                    and sm["n_iter"] == rows["exhaustive_sweep_fp64"]["merges"])
        pruned[name] = rows
    inference = scorer.inference_timing(ctx, 1 << 20)       # replaces the trained network: last
    return {"train_feeders": n_train, "iterations_per_feeder": record, "samples": int(X.shape[0]),
            "epochs": len(loss), "loss_first_last": [float(loss[0]), float(loss[-1])],
            "collect_s": t_collect, "train_s": t_train, "train_samples_per_s": len(loss) * X.shape[0] / t_train,
            "eval": {"workload": "feeder3100, first %d iterations" % record, "candidates": int(Xt.shape[0]),
                     "predict_and_rank_s": t_eval,
                     "top_k": {str(k): v for k, v in q.items() if isinstance(k, int)},
                     "winner_rank_percentile": q["winner_rank_percentile"],
                     "tie_band_median": q.get("tie_band_median"), "tie_band_max": q.get("tie_band_max"),
                     "note": "miss_rate: the committed candidate (the smallest (r, s) of the candidates tied with the "
                             "optimum) outside the top-k; optimum_missed: no optimal candidate in the top-k"},
            "pruned_search": pruned, "inference": inference}


def sweeps_line(K, ctx):
    """Margin sweep (eight margins of the 1,000-bus stand-in in one batched
    launch, run until infeasible, with radialization) and the robustness of its
    0.005 p.u. reduction over 24 synthetic hours (library: heaviest and lightest
    hour)."""
    import feedergen as fg
    from paper_2510_19608_gb300 import sweeps
    f, run = fg.preset(WORKLOAD)
    margins = [0.0005, 0.001, 0.002, 0.003, 0.005, 0.0075, 0.01, 0.015]
    t0 = time.perf_counter()
    rows, st = sweeps.margin_sweep(ctx, f, margins)
    t_sweep = time.perf_counter() - t0
    hours = fg.daily_profiles(f, hours=24, seed=0)
    t0 = time.perf_counter()
    rob = sweeps.profile_robustness(ctx, f, hours, margin=run["margin"], target=1.0)
    t_rob = time.perf_counter() - t0
    return {"margin_sweep": {"rows": [{k: (round(v, 6) if isinstance(v, float) else v) for k, v in r.items()}
                                      for r in rows],
                             "wall_s": t_sweep, "search_ms": st["search_ms"], "setup_ms": st["setup_ms"]},
            "robustness": {"hours": 24, "wall_s": t_rob, **{k: v for k, v in rob.items() if k != "max_error_by_hour"},
                           "max_error_by_hour": [round(e, 6) for e in rob["max_error_by_hour"]]}}


def search_roofline(K, ctx, dfeed, run, search_ms: float, merges: int) -> dict:
    """Roofline block of the incremental search kernel (one CTA runs a
    feeder's whole search, a chain of dependent merges): its per-merge time
    against the latency floor of a merge, and, beside it, its counted FP32
    arithmetic against the FP32 ALU peak.  search_ms: the kernel's CUDA-event
    time per launch; items are counted by the kernel in one profiled run."""
    pp = K.default_params(margin=run["margin"], target_reduction=run["target"], precision=1, engine=2, profile=1)
    ctx.reduce_device(dfeed, pp)
    ps = ctx.summary()
    items = ps["terms"]
    floor_us, cyc = merge_floor_us()
    per_merge_us = 1e3 * search_ms / max(merges, 1)
    achieved_flops = items * FLOPS_PER_ITEM / (search_ms / 1e3) / 1e12 if search_ms > 0 else 0.0
    return {"bound": "latency", "achieved": 1e6 / per_merge_us, "peak": 1e6 / floor_us, "unit": "merges/s",
            "frac": floor_us / per_merge_us, "kernel": "k_search_inc",
            "measured_us_per_merge": per_merge_us, "floor_us_per_merge": floor_us,
            "floor_cycles_per_phase": cyc, "floor_clock_hz": SM_CLOCK_HZ,
            "peak_source": "latency floor of one merge: per phase, the longest chain of dependent steps at latencies "
                           "measured on a GB300 (L2 290, L1 47, barrier 48, DFMA 64, DP sqrt+add 675 cycles; FFMA 4 "
                           "nominal), unlimited parallelism inside a phase",
            "avg_launch_us": 1e3 * search_ms, "launches_per_step": 1, "merges": merges,
            "items_per_launch": items, "flops_per_item": FLOPS_PER_ITEM, "flops_per_launch": items * FLOPS_PER_ITEM,
            "alu": {"bound": "alu", "achieved": achieved_flops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved_flops / FP32_PEAK_TFLOPS,
                    "peak_source": "derived FP32 ALU rate: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"},
            # incremental engine's phase timer (CTA 0): selection = block summaries and pass A (11) + pass B (0);
            # changed set = the winner's record (12) + the scan beside the merge's evaluation (1)
            "phase_us_per_merge": {k: round(1e3 * v / max(merges, 1), 3) for k, v in (
                ("select", ps["phase_ms"][11] + ps["phase_ms"][0]), ("changed_set", ps["phase_ms"][12] + ps["phase_ms"][1]),
                ("merge_and_rebuild", ps["phase_ms"][2]), ("terms", ps["phase_ms"][3]))},
            "rechecks": ps["rechecks"], "recheck_candidates": ps["recheck_cands"],
            "shape": {k: ps[k] for k in ("inc_threads", "inc_eval_warps", "inc_shared_entries", "inc_records")}}


def large_feeder_rows(K, ctx, stream, steps: int, flush) -> dict:
    """The 2,200- and 3,100-bus stand-ins of the paper's 5,991- and 8,381-node
    feeders (Table 2) at their targets (90 %, 80 %): time to optimal reduction
    with inputs resident in HBM (CUDA events around okr_reduce_device on the
    library's stream, L2 flushed between steps), candidates/s, the (candidate,
    phase-node, scenario) items evaluated per second, the FP64 sweep beside
    it, and the search kernel's roofline block."""
    import numpy as np
    import torch
    import feedergen as fg
    out = {}
    for name in ("feeder2200", "feeder3100"):
        f, run = fg.preset(name)
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f.parent, f.phases, f.z_line, f.s_load)]
        dfeed = K.device_feeder(f.n_bus, f.n_scen, *[t.data_ptr() for t in dev], f.v_slack)
        row = {"workload": f"{name}: {f.n_bus} buses ({f.n_phase_nodes} phase nodes), 12.47 kV, {f.n_scen} "
                           f"scenarios, 45/15/40 % phase mix, lognormal loads, target {int(run['target'] * 100)}%, "
                           f"margin {run['margin']} p.u."}
        for key, prec, engine in (("incremental_mixed", 1, 2), ("sweep_fp64", 0, 1)):
            p = K.default_params(margin=run["margin"], target_reduction=run["target"], precision=prec, engine=engine)
            for _ in range(3):
                ctx.reduce_device(dfeed, p)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            kern = []
            for a, b in ev:
                flush.fill_(1.0)
                a.record(stream)
                ctx.reduce_device(dfeed, p)
                b.record(stream)
                kern.append(ctx.summary()["search_ms"])
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / steps
            sm = ctx.summary()
            row[key] = {"time_to_optimal_ms": ms, "candidates_per_s": sm["candidates"] / (ms / 1e3),
                        "candidates": sm["candidates"], "merges": sm["n_iter"], "stop_reason": sm["stop_reason"],
                        "search_kernel_ms": statistics.median(kern), "smice": sm["smice"]}
            if key == "incremental_mixed":
                rl = search_roofline(K, ctx, dfeed, run, statistics.median(kern), sm["n_iter"])
                row[key]["items_per_s"] = rl["items_per_launch"] / (ms / 1e3)
                row[key]["roofline"] = rl
        row["fp64_over_incremental"] = row["sweep_fp64"]["time_to_optimal_ms"] / row["incremental_mixed"]["time_to_optimal_ms"]
        out[name] = row
    return out


def cpu_baseline_large(name: str = "feeder2200", repeats: int = 3) -> dict:
    """The oracle's full reduction of a large stand-in on every host core
    (median of `repeats`)."""
    import feedergen as fg
    from oracle import oracle as O
    f, run = fg.preset(name)
    vhat, ihat = O.operating_points(f)
    merges = O.max_merges_for(f.n_bus, run["target"])
    times, res = [], None
    for _ in range(repeats):
        t0 = time.perf_counter()
        res = O.reduce(f, vhat, ihat, margin=run["margin"], max_merges=merges)
        times.append(time.perf_counter() - t0)
    dt = statistics.median(times)
    return {"value": res["candidates"] / dt, "unit": "candidates/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"full {name} reduction ({res['n_iter']} merges, {res['candidates']} candidates), delta mode, "
                      f"median of {repeats}", "seconds": dt, "seconds_all": times}


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import feedergen as fg
    import paper_2510_19608_gb300 as K
    from paper_2510_19608_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    f, run = fg.preset(WORKLOAD)
    stream = torch.cuda.current_stream()
    ctx = K.Context(local, stream.cuda_stream)
    # every engine and precision selects the same candidates.  Headline: the
    # incremental engine with FP32 terms (carried bounds, FP64 rescoring where
    # the bound cannot decide, FP64 merges).  "vs FP64": the plain FP64 search
    # that scores every candidate afresh each iteration (the sweep engine).
    p = K.default_params(margin=run["margin"], target_reduction=run["target"], precision=1, engine=2)
    p64 = K.default_params(margin=run["margin"], target_reduction=run["target"], precision=0, engine=1)
    others = {"sweep_mixed": K.default_params(margin=run["margin"], target_reduction=run["target"], precision=1,
                                              engine=1),
              "incremental_fp64": K.default_params(margin=run["margin"], target_reduction=run["target"], precision=0,
                                                   engine=2)}

    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f.parent, f.phases, f.z_line, f.s_load)]
    dfeed = K.device_feeder(f.n_bus, f.n_scen, *[t.data_ptr() for t in dev], f.v_slack)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(max(args.warmup, 3)):
        ctx.reduce_device(dfeed, p)
    summ = ctx.summary()
    cand_per_step = summ["candidates"]
    launches_per_step = summ["launches"]

    # ---- device-resident timed region
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))                      # evict L2 between steps (outside the events)
            starts[i].record(stream)
            ctx.reduce_device(dfeed, p)
            ends[i].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if dist:
        dist.barrier()
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    summ_last = ctx.summary()                          # the last timed step
    ms = max_over_ranks(ms, dist, "cuda")
    value = replica_value(cand_per_step, args.steps, world, ms)

    # ---- the same workload with the other engines / precisions (comparison rows)
    def timed_row(params):
        for _ in range(3):
            ctx.reduce_device(dfeed, params)
        steps = max(1, min(args.steps, 50))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush.fill_(0.0)
            a.record(stream)
            ctx.reduce_device(dfeed, params)
            b.record(stream)
        torch.cuda.synchronize()
        msr = sum(a.elapsed_time(b) for a, b in ev) / steps
        sr = ctx.summary()
        return {"ms_per_step": msr, "value": sr["candidates"] / (msr / 1e3), "unit": "candidates/s",
                "search_kernel_ms": sr["search_ms"], "merges": sr["n_iter"], "smice": sr["smice"]}

    fp64_row = timed_row(p64)
    fp64_row["engine"] = "sweep: every candidate scored afresh in FP64 each iteration (one persistent launch)"
    other_rows = {k: timed_row(v) for k, v in others.items()}
    other_rows["sweep_mixed"]["engine"] = "sweep: FP32 screen with bounds, FP64 recheck, FP64 merges"
    other_rows["incremental_fp64"]["engine"] = "incremental: FP64 terms carried across merges"

    # ---- end to end: pinned host inputs through okr_reduce, result read back
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (f.parent, f.phases, f.z_line, f.s_load)]

    import types
    host_feeder = types.SimpleNamespace(parent=pinned[0].numpy(), phases=pinned[1].numpy(), z_line=pinned[2].numpy(),
                                        s_load=pinned[3].numpy(), v_slack=f.v_slack)

    h2d = sum(t.numel() * t.element_size() for t in pinned)
    e2e_steps = max(1, min(args.steps, 50))
    for _ in range(max(3, args.warmup)):                  # warm-up: the host-input path's first calls
        ctx.reduce(host_feeder, p)
        ctx.assignment()
        ctx.decisions()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.reduce(host_feeder, p)
        sup = ctx.assignment()
        dec = ctx.decisions()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    d2h = sup.nbytes + sum(v.nbytes for v in dec.values())
    e2e = {"value": cand_per_step / e2e_s, "unit": "candidates/s", "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "time_to_optimal_s": e2e_s}

    # ---- roofline of the dominant kernel: the search kernel (one CTA runs the
    # whole search), timed with CUDA events around its launch on the library
    # stream; its (candidate, phase-node, scenario) items are counted by the
    # kernel in one profiled step
    search_ms = summ_last["search_ms"]
    roofline = search_roofline(K, ctx, dfeed, run, search_ms, summ["n_iter"])
    roofline["traffic"] = _ncu_traffic()
    roofline["share_of_step"] = search_ms / (ms / args.steps)
    roofline["note"] = ("one CTA runs the whole search, a chain of dependent merges: its time is latency, not "
                        "arithmetic or memory traffic; frac = latency floor / measured time per merge")
    # output Y_Kron of the chosen network (Sec. II-B), formed once per feeder
    yk, _ = ctx.kron()
    kron = {"ms": ctx.summary()["kron_ms"], "k_phi": int(yk.shape[0]),
            "note": "device time of okr_kron on the chosen network (outside the step)"}
    large = large_feeder_rows(K, ctx, stream, max(1, min(args.steps, 10)), flush) if not args.no_large else None
    batch = batch_line(K, ctx) if not args.no_batch else None
    learned = learned_line(K, ctx) if not args.no_learned else None
    studies = sweeps_line(K, ctx) if not args.no_batch else None
    if rank == 0:
        cb = cpu_baseline(f, run, repeats=args.cpu_repeats) if world == 1 else None
        if cb is not None and not args.no_large:
            cb["feeder2200"] = cpu_baseline_large("feeder2200", repeats=args.cpu_repeats)
        line = {"metric": METRIC, "value": value, "unit": "candidates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "fp64_search": {"ms_per_step": fp64_row["ms_per_step"], "value": fp64_row["value"],
                                "unit": "candidates/s", "headline_speedup": fp64_row["ms_per_step"] / (ms / args.steps),
                                "engine": "sweep, plain FP64: every candidate scored afresh each iteration"},
                "large_feeders": large,
                "config": _workload_config(f, run) | {
                    "engine": "incremental: every candidate's score carried across merges as an exact fixed-point "
                              "sum of its terms; only the terms whose inputs the last merge changed are evaluated "
                              "again; one CTA",
                    "precision": "FP32 terms with carried rigorous bounds, FP64 rescoring of the candidates the bound "
                                 "cannot separate, FP64 merges",
                    "value_counts": "every candidate of every iteration gets its exact score and feasibility; the "
                                    "incremental engine carries most scores from the last merge and recomputes only "
                                    "the terms whose inputs changed (roofline.items_per_launch); fp64_search scores "
                                    "every candidate afresh",
                    "fp64_search": fp64_row, "other_engines": other_rows, "rechecks": summ_last["rechecks"],
                    "recheck_candidates": summ_last["recheck_cands"],
                    "l2": "flushed between steps (256 MB write outside the timed events)",
                    "parallelism": f"replicas x{world}", "time_to_optimal_ms": ms / args.steps,
                    "candidates_per_step": cand_per_step, "merges": summ["n_iter"],
                    "stop_reason": summ["stop_reason"], "wall_s": t_wall, "y_kron": kron,
                    "batch": batch, "learned_scorer": learned, "studies": studies},
                "clocks": clk.summary(), "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "roofline": roofline}
        if cb:
            line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = _args()
    rank, world, local = _dist()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
