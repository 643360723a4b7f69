#!/usr/bin/env python
"""Benchmark of the PT hot path: branch-optimised topologies/s.

Default workload (pt128, the configuration the metric is quoted on): 128
taxa x 10000 sites, GTR+Gamma4 (exchangeabilities ~ Dirichlet(1^6),
frequencies ~ Dirichlet(5^4), alpha 0.5), simulated on a random tree with
Exp(mean 0.02) branches; 32 hill-climbs (on the GPU) give the starts, PT with
threshold 15 and a 2^24-slot visited table grows the frontier during set-up.
One step = one PT round on that fixed frontier: every NNI neighbour is keyed,
deduplicated against the device visited table (reset at the start of the
step), proposal-optimised by Newton on its five NNI branches, thresholded at
lmax - 15, and the kept ones are fully optimised.  Unit: unique neighbours
scored to convergence per second, whole job.  --workload pt27: the 27-taxon x
2000-site configuration (8 hill-climbs from random trees, threshold 10).

value: device-resident inputs, learned warm start + mixed precision, the round
       replayed as one CUDA graph (pt_graph_run; frontier in the graph's buffers).
e2e:   the same graph round through the host-buffer entry points: frontier
       copied in from pinned host memory (pt_graph_set_frontier), next
       frontier copied out (pt_graph_get_next), inside every step.
direct_launch: the same round issued kernel by kernel (pt_expand_frontier_dev);
       its per-stage CUDA events give the kernel times of the rooflines.
fp64_gpu: the plain FP64 GPU path on the same frontier (plain Newton start).
error: the timed round against the plain FP64 GPU round (every proposal and
       visit, visited-set agreement) and, from the oracle leg, sampled
       proposals and visits against the FP64 oracle.
--workload batch16: 16 alignments (taxa ~ U[20,100], sites ~ U[300,5000]),
       256 frontier trees each (random topologies with optimised lengths),
       one graph round over all of them per step.
--workload warm64: the warm-start network trained on about 1 M logged pairs,
       then 4-round searches on fresh 64-taxon x 1500-site alignments from
       hill-climbed starts, plain against learned start (Newton evaluations
       saved, identical decisions).
--impl reference: the FP64 CPU oracle, timed on this host's cores on a
bounded sample of the same step.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Workloads: the configuration the metric is quoted on (pt128) and the 27-taxon one.
#   starts: hill-climbs (GPU) from `starts` trees: uniform random topologies, or
#   (perturb > 0) the generating topology with `perturb` random leaves
#   reinserted -- climbs from uniform random 128-taxon topologies take ~700
#   moves each (590 s for 32 on the GPU) and all reach the topology these reach.
WORKLOADS = {
    "pt128": dict(taxa=128, sites=10000, mean_branch=0.02, thresh=15.0, starts=32, perturb=3, table_log2=24,
                  seed_off=5, frontier=256, steps=5),
    "pt27": dict(taxa=27, sites=2000, mean_branch=0.05, thresh=10.0, starts=8, perturb=0, table_log2=22,
                 seed_off=2, frontier=256, steps=50),
}
# DRAM bytes per launch of the two persistent kernels, from one ncu capture of each on the
# workload's shapes (dram__bytes_read.sum + dram__bytes_write.sum of the captured launch divided
# by its units: neighbours, or full-optimisation sweeps of kept trees); None until captured
# (profiles/ holds the captures)
DRAM = {"pt128": {"per_neighbour": (1.492012e9 + 0.312236e9) / 1961,      # profiles/k_propose_128taxa_5908patterns.md
                  "per_full_sweep": (145.843998e9 + 84.912576e9) / 692},   # profiles/k_fullopt_128taxa_5908patterns.md
        "pt27": {"per_neighbour": None, "per_full_sweep": None}}
FP32_LANES_PER_SM = 128
# warm-start training runs (log_training_runs): 27-taxon x 2000-site searches from 8 hill-climbs
# (threshold 10, up to 8 rounds) and 7-taxon JC69 exhaustive searches; TRAIN_RUNS runs log about
# 0.2 M pairs (--workload warm64 logs about 1 M)
TRAIN_TAXA, TRAIN_SITES, TRAIN_THRESH, TRAIN_STARTS, TRAIN_ROUNDS = 27, 2000, 10.0, 8, 8
TRAIN_RUNS, TRAIN_STEPS, TRAIN_LOG_CAP = 30, 4000, 1 << 21
BATCH_THRESH = 10.0  # --workload batch16


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default: 5 for pt128, 50 for pt27, 5 for batch16; 3 for the oracle)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--frontier", type=int, default=0, help="frontier cap (0: the workload's)")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-mlp", action="store_true", help="plain Newton start (no learned warm start)")
    p.add_argument("--no-autotune", action="store_true", help="no tuning trials: default CTA sizes, or those of --tune-cache")
    p.add_argument("--tune-cache", default=None, help="JSON cache of tuned launch shapes: read, and written when tuning")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=0, help="frontier trees in the CPU baseline sample (0: one per thread)")
    p.add_argument("--cpu-threads", type=int, default=0, help="threads of the CPU baseline (0: all cores)")
    p.add_argument("--workload", default="pt128", choices=["pt128", "pt27", "batch16", "warm64"])
    args = p.parse_args()
    if args.steps is None:  # a few seconds of timed GPU work; the oracle's steps take a few seconds each
        args.steps = 3 if args.impl == "reference" else (5 if args.workload == "batch16" else
                                                          3 if args.workload == "warm64" else
                                                          WORKLOADS[args.workload]["steps"])
    return args


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev, self.rows, self.proc = dev, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the sampler is live before the timed work starts: wait for its first
            # line (at most 5 s) and keep only the samples taken after it
            t0 = time.time()
            while not self.rows and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.rows.clear()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.lower() in ("active", "1", "yes"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def workload(W, rank: int):
    """The alignment and the hill-climb starting trees of a workload."""
    from paper_1811_11007_gb300 import synth
    seed = synth.SEED_BASE + W["seed_off"] + 1000 * rank
    n = W["taxa"]
    a = synth.simulate(n, W["sites"], seed, model="gtr", alpha=0.5, mean_branch=W["mean_branch"])
    if W["perturb"]:
        rng = np.random.default_rng(seed + 1)
        e = np.stack([synth.reinsert_leaves(a.tree_edges, n, W["perturb"], rng) for _ in range(W["starts"])])
        starts = (np.ascontiguousarray(e, np.int32), np.full((W["starts"], 2 * n - 3), 0.1))
    else:
        starts = synth.random_trees(n, W["starts"], seed + 1)
    return a, starts


def build_frontier(ctx, aid, edges, lengths, F, thresh):
    """PT search (threshold thresh) from the given trees until the frontier holds
    >= F trees or empties; returns the largest frontier seen (first F), the
    lmax before it and the rounds run."""
    lmax, front = ctx.begin(aid, edges, lengths, thresh)
    best = (lmax, front)
    rounds = 0
    for _ in range(200):
        if len(front["edges"]) >= F or len(front["edges"]) == 0:
            break
        lm, nx = ctx.expand(aid, front["edges"], front["lengths"], thresh, lmax)
        rounds += 1
        if len(nx["edges"]) > len(best[1]["edges"]):
            best = (lm, nx)
        lmax, front = lm, nx
    lmax, front = best if len(front["edges"]) < F else (lmax, front)
    k = min(F, len(front["edges"]))
    return lmax, {key: v[:k] for key, v in front.items()}, rounds


def reduce_over_ranks(ms: float, units: float, world: int, device="cuda"):
    """Whole-job timing: the slowest rank's time and the units of all ranks
    (each rank runs its own independent alignment; no data-path collective)."""
    if world <= 1:
        return ms, units
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    u = torch.tensor([units], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(u)
    return float(t.item()), float(u.item())


def log_training_runs(ctx, rank, n_runs, seed0=5000):
    """Logs (features, optimised lengths) pairs of the plain start's proposals
    from PT runs on fresh seeded alignments shaped like the two small
    workloads: every 5th run a 7-taxon x 500-site JC69 search with an infinite
    threshold (all 945 topologies), the others 27-taxon x 2000-site GTR+G4
    searches from 8 hill-climbs (threshold 10, frontier capped at 256 trees, up
    to 8 rounds).  The climbs are not logged.  Returns the runs' shapes."""
    from paper_1811_11007_gb300 import synth
    ctx.mlp_enable(False)
    runs = {"jc7_exhaustive": 0, "gtr27_climbed": 0}
    for j in range(n_runs):
        seed = synth.SEED_BASE + seed0 + j + 100000 * rank
        if j % 5 == 4:
            a = synth.simulate(7, 500, seed, model="jc", alpha=None, mean_branch=0.1)
            aid = ctx.load_alignment(a.codes)
            ctx.set_model(aid, a.exch, a.freqs, 1.0, 1)
            e, l = synth.random_trees(7, 1, seed + 1)
            thr, cap, rounds = math.inf, 1024, 16
            runs["jc7_exhaustive"] += 1
        else:
            a = synth.simulate(TRAIN_TAXA, TRAIN_SITES, seed, model="gtr", alpha=0.5, mean_branch=0.05)
            aid = ctx.load_alignment(a.codes)
            ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
            hc = ctx.hill_climb(aid, *synth.random_trees(TRAIN_TAXA, TRAIN_STARTS, seed + 1))
            e, l = hc["edges"], hc["lengths"]
            thr, cap, rounds = TRAIN_THRESH, 256, TRAIN_ROUNDS
            runs["gtr27_climbed"] += 1
        ctx.training_log(True, TRAIN_LOG_CAP)
        lmax, front = ctx.begin(aid, e, l, thr)
        for _ in range(rounds):
            if not len(front["edges"]):
                break
            lmax, front = ctx.expand(aid, front["edges"][:cap], front["lengths"][:cap], thr, lmax)
        ctx.training_log(False)
    return runs


def mlp_init_weights():
    """He-normal hidden layers, a small output layer; padding rows and columns zero."""
    from paper_1811_11007_gb300 import synth
    rng = np.random.default_rng(synth.SEED_BASE + 99)
    w = np.zeros(27912, np.float32)
    w[0:69 * 128] = rng.normal(0, np.sqrt(2 / 69), 69 * 128)
    w[80 * 128 + 128:80 * 128 + 128 + 128 * 128] = rng.normal(0, np.sqrt(2 / 128), 128 * 128)
    w3 = rng.normal(0, 0.1 * np.sqrt(1 / 128), (128, 8))
    w3[:, 5:] = 0
    o3 = 80 * 128 + 128 + 128 * 128 + 128
    w[o3:o3 + 1024] = w3.ravel()
    return w


def warm_start_weights(rank, n_runs=None):
    """The warm-start network's weights, trained (untimed set-up) on pairs
    logged from other alignments' PT runs (log_training_runs, in a context of
    its own with small visited tables) by the library's own kernels."""
    from paper_1811_11007_gb300 import pt, synth
    t0 = time.time()
    with pt.Context(precision="mixed", table_log2=18) as tc:
        runs = log_training_runs(tc, rank, TRAIN_RUNS if n_runs is None else n_runs)
        x, t = tc.training_pairs()
        t_log = time.time() - t0
        tc.mlp_set_weights(mlp_init_weights())
        loss = tc.mlp_train(TRAIN_STEPS, batch=2048, lr=2e-3, seed=synth.SEED_BASE + 7)
        w = tc.mlp_get_weights()
    return w, {"train_pairs": int(len(x)), "runs": runs, "steps": TRAIN_STEPS, "batch": 2048,
               "final_batch_loss": loss,
               "zero_prediction_loss": float(np.mean(np.asarray(t, np.float64) ** 2)) if len(t) else None,
               "log_s": t_log, "train_s": time.time() - t0 - t_log}


def train_warm_start(ctx, rank, n_runs=None):
    """Trains the warm-start network (warm_start_weights), loads it into ctx
    and enables it there."""
    w, info = warm_start_weights(rank, n_runs)
    ctx.mlp_set_weights(w)
    ctx.mlp_enable(True)
    return info


def _keys(k):
    return [(int(lo), int(hi)) for lo, hi in np.asarray(k, np.uint64).reshape(-1, 2)]


def _start_diff(pl, pp, vl, vp, nl, np_):
    """The timed (learned-start) round against the plain-start round on the same
    frontier: decisions must agree; a proposal still moving at the sweep cap
    ends where its start led it, so proposal scores can differ."""
    a = dict(zip(_keys(pl["keys"]), pl["lnl"]))
    b = dict(zip(_keys(pp["keys"]), pp["lnl"]))
    d = np.array([abs(a[k] - b[k]) for k in set(a) & set(b)] or [0.0])
    va, vb = dict(zip(_keys(vl["keys"]), vl["status"])), dict(zip(_keys(vp["keys"]), vp["status"]))
    fa, fb = dict(zip(_keys(nl["keys"]), nl["lnl"])), dict(zip(_keys(np_["keys"]), np_["lnl"]))
    return {"statuses_equal": va == vb, "next_frontier_equal": set(fa) == set(fb),
            "max_abs_dlnl_next_frontier": float(max((abs(fa[k] - fb[k]) for k in set(fa) & set(fb)), default=0.0)),
            "proposals_differing_gt_1e-3": int(np.sum(d > 1e-3)), "proposals_compared": int(len(d)),
            "max_abs_dlnl_proposals": float(d.max())}


def run_ours(args, W, rank, world, dev):
    import torch
    from paper_1811_11007_gb300 import pt
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    a, starts = workload(W, rank)
    n, T = W["taxa"], W["thresh"]
    E, m = 2 * n - 3, 2 * (n - 3)
    setup = {}

    def make(prec):
        ctx = pt.Context(precision=prec, table_log2=W["table_log2"], stream=stream)
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        return ctx, aid

    ctx, aid = make("mixed")
    learned = None
    t0 = time.time()
    if not args.no_mlp:
        learned = train_warm_start(ctx, rank)
        ctx.mlp_enable(False)  # set-up searches from the plain start; the timed rounds use the network
    setup["train_s"] = time.time() - t0
    # the starts: hill-climbs on the GPU (best-improving NNI moves until none gains > 1e-6)
    t0 = time.time()
    hc = ctx.hill_climb(aid, starts[0], starts[1])
    setup["climb_s"] = time.time() - t0
    setup["climb_moves"] = [int(x) for x in hc["moves"]]
    setup["climb_distinct_topologies"] = len(set(_keys(hc["keys"])))
    setup["climb_best_lnl"] = float(np.max(hc["lnl"]))
    # PT from the climbed starts until the frontier is large: the timed rounds' frontier
    t0 = time.time()
    F_cap = args.frontier or W["frontier"]
    lmax0, front, setup_rounds = build_frontier(ctx, aid, hc["edges"], hc["lengths"], F_cap, T)
    setup["frontier_rounds"] = setup_rounds
    setup["frontier_s"] = time.time() - t0
    if learned is not None:
        ctx.mlp_enable(True)
    # CTA sizes tuned on this workload's own rounds: the first untimed warm-up step runs the trials
    ctx.autotune(not args.no_autotune, args.tune_cache)
    # launches of the two persistent kernels before the first timed step, for profilers
    print(f"propose_launches_before_timed={setup_rounds + args.warmup}", file=sys.stderr)
    F = len(front["edges"])
    _, P = ctx.alignment_info(aid)
    d_e = torch.from_numpy(np.ascontiguousarray(front["edges"])).to(dev)
    d_l = torch.from_numpy(np.ascontiguousarray(front["lengths"])).to(dev)
    cap = F * m
    o_e = torch.empty((cap, E, 2), dtype=torch.int32, device=dev)
    o_l = torch.empty((cap, E), dtype=torch.float64, device=dev)
    o_n = torch.empty(cap, dtype=torch.float64, device=dev)
    o_k = torch.empty((cap, 2), dtype=torch.int64, device=dev)

    def step_dev(c, i):
        c.reset_visited(i)
        lm, cnt = c.expand_dev(i, F, d_e.data_ptr(), d_l.data_ptr(), T, lmax0, cap, o_e.data_ptr(),
                               o_l.data_ptr(), o_n.data_ptr(), o_k.data_ptr())
        st = c.stats()
        times = c.stage_times()
        return st["scored"], st["launches"] + 1, times, st, cnt

    def timed(c, i, step, steps, warmup, label):
        for _ in range(warmup):
            step(c, i)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        # an NVTX range around the timed steps, so a profiler can select them (ncu --nvtx --nvtx-include)
        torch.cuda.nvtx.range_push(label)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        acc = {"units": 0, "launches": 0, "prop_ms": 0.0, "part_ms": 0.0, "full_ms": 0.0, "flops": 0.0,
               "full_flops": 0.0, "prop_launches": 0, "full_launches": 0, "full_sweeps": 0, "kept": 0}
        stats, times = None, {}
        e0.record(stream)
        for _ in range(steps):
            w, l, times, st, _ = step(c, i)
            acc["units"] += w
            acc["launches"] += l
            acc["prop_ms"] += times["propose"]
            acc["part_ms"] += times["partials"]
            acc["full_ms"] += times["fullopt_kernel"]
            acc["full_sweeps"] += st["full_sweeps"]
            acc["kept"] += st["kept"]
            stats = st
            nb = 5 if c.cfg.propose_mode == 0 else 1
            acc["flops"] += P * (st["prop_sweeps"] * nb * 2 * 272 + st["prop_evals"] * 100)
            # full optimisation: per sweep (2n-3) edge visits (two sides + sum-table, 2 x 272
            # flops per site) and n-2 refreshes of a vector below a node (272), 100 per evaluation
            acc["full_flops"] += P * (st["full_sweeps"] * ((2 * n - 3) * 544 + (n - 2) * 272) + st["full_evals"] * 100)
        e1.record(stream)
        torch.cuda.nvtx.range_pop()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ms, units = reduce_over_ranks(ms, acc["units"], world, device=f"cuda:{dev}")
        acc.update({"ms": ms, "units": units, "stats": stats, "times": times, "steps": steps})
        return acc

    # kernel by kernel: its per-stage CUDA events give the kernel times of the rooflines
    n_direct = max(1, min(args.steps, 3))
    res = timed(ctx, aid, step_dev, n_direct, args.warmup, "direct")
    props_mixed = ctx.last_proposals()
    vis_mixed = ctx.visited(aid)
    ng = res["stats"]["good"]
    nxt_mixed = {"keys": o_k[:ng].cpu().numpy(), "lnl": o_n[:ng].cpu().numpy(), "edges": o_e[:ng].cpu().numpy(),
                 "lengths": o_l[:ng].cpu().numpy()}

    # the round as one CUDA graph, recorded once and replayed every step (the headline)
    g = ctx.graph([aid], [F], [T])
    g.set_frontier(0, front["edges"], front["lengths"])

    def step_graph(c, i):
        c.reset_visited(i)
        _, nn = g.run([F], [lmax0])
        st = c.stats()
        return st["scored"], st["launches"] + 1, c.stage_times(), st, nn[0]

    # the graph round must reproduce the kernel-by-kernel round exactly
    _, _, _, _, cnt_d = step_dev(ctx, aid)
    keys_d = o_k[:cnt_d].cpu().numpy().astype(np.uint64)
    lnl_d = o_n[:cnt_d].cpu().numpy()
    step_graph(ctx, aid)
    nxt = g.next(0)
    graph_check = {"next_frontier": int(cnt_d),
                   "identical": bool(len(nxt["keys"]) == cnt_d and np.array_equal(nxt["keys"], keys_d)
                                     and np.array_equal(nxt["lnl"], lnl_d))}

    with ClockSampler(dev) as clk:
        resg = timed(ctx, aid, step_graph, args.steps, args.warmup, "graph")
    clocks = clk.summary()

    # end to end: host buffers (pinned), copies inside every step
    h_e = torch.from_numpy(np.ascontiguousarray(front["edges"])).pin_memory()
    h_l = torch.from_numpy(np.ascontiguousarray(front["lengths"])).pin_memory()
    ho_e = torch.empty((cap, E, 2), dtype=torch.int32).pin_memory()
    ho_l = torch.empty((cap, E), dtype=torch.float64).pin_memory()
    ho_n = torch.empty(cap, dtype=torch.float64).pin_memory()
    ho_k = torch.empty((cap, 2), dtype=torch.int64).pin_memory()
    bytes_io = {"h2d": 0, "d2h": 0}

    def step_host(c, i):
        c.reset_visited(i)
        L = pt.lib()
        c._ck(L.pt_graph_set_frontier(c._h, g._g, 0, F, C.c_void_p(h_e.data_ptr()), C.c_void_p(h_l.data_ptr())))
        nf, lm, nn = (C.c_int * 1)(F), (C.c_double * 1)(lmax0), (C.c_int * 1)()
        c._ck(L.pt_graph_run(c._h, g._g, nf, lm, nn))
        st = c.stats()
        cnt = C.c_int()
        c._ck(L.pt_graph_get_next(c._h, g._g, 0, cap, C.c_void_p(ho_e.data_ptr()), C.c_void_p(ho_l.data_ptr()),
                                  C.c_void_p(ho_n.data_ptr()), C.c_void_p(ho_k.data_ptr()), C.byref(cnt)))
        bytes_io["h2d"] = F * E * 2 * 4 + F * E * 8
        bytes_io["d2h"] = cnt.value * (E * 2 * 4 + E * 8 + 8 + 16)
        return st["scored"], st["launches"] + 1, c.stage_times(), st, cnt.value

    n_e2e = max(1, min(args.steps, 5))
    e2e = timed(ctx, aid, step_host, n_e2e, 1, "e2e")
    g.close()

    plain = judge = None
    props_plain, vis_plain = props_mixed, vis_mixed
    nxt_plain = nxt_mixed
    if learned is not None:
        judge = ctx.mlp_judge(aid)  # the plain start's judgement of the network on this alignment
        ctx.mlp_enable(False)
        plain = timed(ctx, aid, step_dev, 1, 1, "plain")
        props_plain, vis_plain = ctx.last_proposals(), ctx.visited(aid)
        ngp = plain["stats"]["good"]
        nxt_plain = {"keys": o_k[:ngp].cpu().numpy(), "lnl": o_n[:ngp].cpu().numpy()}
        ctx.mlp_enable(True)
    fp64 = err64 = None
    if not args.no_fp64:
        ctx64, aid64 = make("fp64")
        fp64 = timed(ctx64, aid64, step_dev, 1, 1, "fp64")
        # the timed (mixed) round against the plain FP64 GPU round on the same frontier
        p64 = ctx64.last_proposals()
        v64 = ctx64.visited(aid64)
        n64 = {"keys": o_k[:fp64["stats"]["good"]].cpu().numpy(), "lnl": o_n[:fp64["stats"]["good"]].cpu().numpy()}
        ctx64.close()
        # precision: the mixed round from the same (plain) start as the FP64 round
        sm_, sd_ = dict(zip(_keys(props_plain["keys"]), props_plain["lnl"])), dict(zip(_keys(p64["keys"]), p64["lnl"]))
        vm_ = dict(zip(_keys(vis_plain["keys"]), vis_plain["status"]))
        vd_ = dict(zip(_keys(v64["keys"]), v64["status"]))
        fm_, fd_ = dict(zip(_keys(nxt_plain["keys"]), nxt_plain["lnl"])), dict(zip(_keys(n64["keys"]), n64["lnl"]))
        common = set(sm_) & set(sd_)
        err64 = {"rounds": "mixed precision (plain start) vs FP64, same frontier",
                 "proposals_compared": len(common),
                 "scored_sets_equal": set(sm_) == set(sd_),
                 "visited_sets_equal": set(vm_) == set(vd_),
                 "statuses_equal": all(vm_[k] == vd_.get(k) for k in vm_),
                 "max_abs_dlnl_proposals": float(max((abs(sm_[k] - sd_[k]) for k in common), default=0.0)),
                 "next_frontier_equal": set(fm_) == set(fd_),
                 "max_abs_dlnl_visits": float(max((abs(fm_[k] - fd_[k]) for k in set(fm_) & set(fd_)), default=0.0))}

    out = None
    if rank == 0:
        pk = peaks()
        value = resg["units"] / (resg["ms"] / 1e3)
        sm_max = pk.get("sm_max_mhz", 2070.0)
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        hbm_peak = pk.get("hbm_gbs")
        peak_note = "of measured (MEASURED_PEAKS.json hbm_gbs)" if hbm_peak else "of fallback (6800 GB/s)"
        hbm_peak = hbm_peak or 6800.0
        st = res["stats"]
        nd = res["steps"]
        # algorithmic bytes: per neighbour the path's 320*P (its four member
        # vectors, shared by the two swaps of an edge, 128*P, and the amortised production of the
        # parent's partials, 192*P), over the proposal kernel's time; a visit writes and reads each
        # of its 2n-5 stored vectors once per sweep, 128*P*(2n-5) per sweep, plus the first
        # bottom-up pass 128*P*(n-2) and the pair pass (h and l) 256*P*(n-2) per kept tree
        prop_bytes = 320.0 * P * res["units"] / max(world, 1)
        full_bytes = 128.0 * P * ((2 * n - 5) * res["full_sweeps"] + 3 * (n - 2) * res["kept"])
        prop_s, full_s = res["prop_ms"] / 1e3, res["full_ms"] / 1e3
        dram = DRAM.get(args.workload, {})
        prop_roof = {"bound": "hbm", "kernel": "k_propose (proposal Newton, five branches)",
                     "achieved": prop_bytes / prop_s / 1e9 if prop_s > 0 else None, "peak": hbm_peak, "unit": "GB/s",
                     "traffic": (dram["per_neighbour"] * res["units"] / nd) if dram.get("per_neighbour") else None,
                     "ms_per_step": res["prop_ms"] / nd, "peak_note": peak_note,
                     "alu": {"achieved": res["flops"] / prop_s / 1e12 if prop_s > 0 else None, "peak": alu_peak,
                             "unit": "TFLOP/s"}}
        full_roof = {"bound": "hbm", "kernel": "k_fullopt (visit: full optimisation)",
                     "achieved": full_bytes / full_s / 1e9 if full_s > 0 else None, "peak": hbm_peak, "unit": "GB/s",
                     "traffic": (dram["per_full_sweep"] * res["full_sweeps"] / nd) if dram.get("per_full_sweep") else None,
                     "ms_per_step": res["full_ms"] / nd, "peak_note": peak_note,
                     "alu": {"achieved": res["full_flops"] / full_s / 1e12 if full_s > 0 else None, "peak": alu_peak,
                             "unit": "TFLOP/s"}}
        for r_ in (prop_roof, full_roof):
            r_["frac"] = (r_["achieved"] / r_["peak"]) if r_["achieved"] else None
            r_["alu"]["frac"] = (r_["alu"]["achieved"] / alu_peak) if r_["alu"]["achieved"] else None
        dominant = dict(full_roof if res["full_ms"] > res["prop_ms"] else prop_roof)
        ws = f"{n} taxa x {W['sites']} sites ({P} patterns)"
        out = {
            "metric": "branch-optimised topologies/sec (unique NNI neighbours scored per PT round)",
            "value": value,
            "path": ("learned warm start + " if learned is not None else "") +
                    "batched persistent launches replayed as one CUDA graph + FP32 partials / FP64 reductions "
                    "(scores from compensated FP32 pairs)",
            "unit": "topologies/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": resg["ms"] / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 partials + f64 reductions",
            "data": "synthetic (seeded simulation; the paper's datasets are not available)",
            "config": {"workload": f"PT round on a {F}-tree frontier, {ws}, GTR+G4, threshold {T}, "
                                   f"2^{W['table_log2']}-slot visited table; frontier grown by PT from "
                                   f"{W['starts']} GPU hill-climbs",
                       "taxa": n, "sites": W["sites"], "patterns": P, "frontier": F,
                       "neighbours_per_step": st["scored"], "kept_per_step": st["kept"],
                       "threshold": T, "parallelism": f"replicas x{world} (independent alignments)",
                       "l2": "inputs larger than L2 (frontier partials and residuals ~%.1f GB per step)" % (
                           F * (2 * n - 5) * P * 132 / 1e9)},
            "setup": setup,
            "e2e": {"value": e2e["units"] / (e2e["ms"] / 1e3), "unit": "topologies/s", "steps": n_e2e,
                    "h2d_bytes_per_step": bytes_io["h2d"], "d2h_bytes_per_step": bytes_io["d2h"]},
            "direct_launch": {"value": res["units"] / (res["ms"] / 1e3), "unit": "topologies/s",
                              "ms_per_step": res["ms"] / nd, "gpu_launches": res["launches"], "steps": nd,
                              "note": "the same round issued kernel by kernel with host reads of the counts"},
            "graph_check": graph_check,
            "fp64_gpu": ({"value": fp64["units"] / (fp64["ms"] / 1e3), "unit": "topologies/s",
                          "ms_per_step": fp64["ms"], "speedup_of_value": value / (fp64["units"] / (fp64["ms"] / 1e3)),
                          "note": "plain FP64 GPU path, plain Newton start, same frontier"} if fp64 else None),
            "error_vs_fp64_gpu": err64,
            "learned_vs_plain_start": _start_diff(props_mixed, props_plain, vis_mixed, vis_plain, nxt_mixed, nxt_plain),
            "mixed_plain_start": ({"value": plain["units"] / (plain["ms"] / 1e3), "unit": "topologies/s",
                                   "prop_evals_per_neighbour": plain["stats"]["prop_evals"] /
                                   max(plain["stats"]["scored"], 1)} if plain else None),
            "learned_warm_start": (dict(learned, judge=judge) if learned else None),
            "roofline": dominant,
            "rooflines": {"k_propose": prop_roof, "k_fullopt": full_roof},
            "stage_ms_per_step": {k: v / 1 for k, v in res.get("times", {}).items()},
            "newton": {"prop_evals_per_neighbour": st["prop_evals"] / max(st["scored"], 1),
                       "prop_sweeps_per_neighbour": st["prop_sweeps"] / max(st["scored"], 1),
                       "full_evals_per_kept_tree": st["full_evals"] / max(st["kept"], 1),
                       "full_sweeps_per_kept_tree": st["full_sweeps"] / max(st["kept"], 1),
                       "nonconverged": st["nonconverged"]},
            "autotune": ctx.autotune_report(),
            "gpu_launches": resg["launches"],
            "clocks": clocks,
        }
    # for the oracle leg: the frontier, lmax, one timed round's proposals and next frontier
    round_info = {"props": props_mixed, "next": nxt_mixed, "scored": res["stats"]["scored"],
                  "kept": res["stats"]["kept"], "full_sweeps": res["stats"]["full_sweeps"]}
    return out, (a, front, lmax0, round_info)


def batch16_alignments(rank: int):
    """16 GTR+G4 alignments of uneven shape: taxa ~ U[20, 100], sites ~ U[300, 5000]."""
    from paper_1811_11007_gb300 import synth
    rng = np.random.default_rng(synth.SEED_BASE + 3 + 1000 * rank)
    out = []
    for i in range(16):
        n = int(rng.integers(20, 101))
        sites = int(rng.integers(300, 5001))
        out.append(synth.simulate(n, sites, synth.SEED_BASE + 300 + 1000 * rank + i, model="gtr", alpha=0.5,
                                  mean_branch=0.05))
    return out


def run_batch16(args, rank, world, dev):
    """One graph round over 16 uneven alignments per step, 256 frontier trees
    each (random topologies with fully optimised lengths; lmax = the best)."""
    import torch
    from paper_1811_11007_gb300 import pt, synth
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    alns = batch16_alignments(rank)
    F = args.frontier or 256
    ctx = pt.Context(precision="mixed", table_log2=22, stream=stream)
    ctx.autotune(not args.no_autotune)
    ids, fronts, lmax0 = [], [], []
    for i, a in enumerate(alns):
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        e, l = synth.random_trees(a.codes.shape[0], F, synth.SEED_BASE + 400 + 1000 * rank + i)
        lnl, lens, _ = ctx.score(aid, e, l, mode="full")
        ids.append(aid)
        fronts.append((e, lens))
        lmax0.append(float(np.max(lnl)))
    parts = [{"aln": aid, "edges": e, "lengths": l, "threshold": BATCH_THRESH, "lmax": lm}
             for aid, (e, l), lm in zip(ids, fronts, lmax0)]

    def run_steps(step, steps, warmup):
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        units, launches, times = 0, 0, {}
        e0.record(stream)
        for _ in range(steps):
            for aid in ids:
                ctx.reset_visited(aid)
            step()
            st = ctx.stats()
            units += st["scored"]
            launches += st["launches"] + len(ids)
            times = ctx.stage_times()
        e1.record(stream)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms, units = reduce_over_ranks(e0.elapsed_time(e1), units, world, device=f"cuda:{dev}")
        return {"ms": ms, "units": units, "launches": launches, "times": times, "stats": ctx.stats()}

    def direct():
        for aid in ids:
            ctx.reset_visited(aid)
        return ctx.expand_batch(parts)

    res_d = run_steps(direct, max(1, min(args.steps, 2)), 1)  # kernel by kernel (also tunes CTA sizes)
    g = ctx.graph(ids, [F] * len(ids), [BATCH_THRESH] * len(ids))
    for k, (e, l) in enumerate(fronts):
        g.set_frontier(k, e, l)
    ref = direct()
    for aid in ids:
        ctx.reset_visited(aid)
    g.run([F] * len(ids), lmax0)
    same = all(np.array_equal(g.next(k)["keys"], ref[k][1]["keys"]) for k in range(len(ids)))
    with ClockSampler(dev) as clk:
        res = run_steps(lambda: g.run([F] * len(ids), lmax0), args.steps, args.warmup)
    g.close()
    if rank != 0:
        return None
    st = res["stats"]
    shapes = [(a.codes.shape[0], ctx.alignment_info(aid)[1]) for a, aid in zip(alns, ids)]
    return {
        "metric": "branch-optimised topologies/sec (unique NNI neighbours scored per PT round)",
        "value": res["units"] / (res["ms"] / 1e3), "unit": "topologies/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["ms"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 partials + f64 reductions",
        "data": "synthetic (seeded simulation; the paper's datasets are not available)",
        "config": {"workload": f"batched graph round: 16 alignments (taxa 20-100, sites 300-5000), {F} frontier "
                               f"trees each (random topologies, optimised lengths), GTR+G4, threshold {BATCH_THRESH}",
                   "alignments": [{"taxa": n, "patterns": P} for n, P in shapes],
                   "neighbours_per_step": st["scored"], "kept_per_step": st["kept"],
                   "parallelism": f"replicas x{world}", "l2": "inputs larger than L2"},
        "direct_launch": {"value": res_d["units"] / (res_d["ms"] / 1e3), "unit": "topologies/s",
                          "ms_per_step": res_d["ms"] / max(1, min(args.steps, 2))},
        "graph_check": {"identical_next_frontiers": bool(same)},
        "stage_ms_per_step": res_d["times"],
        "autotune": ctx.autotune_report(),
        "gpu_launches": res["launches"],
        "clocks": clk.summary(),
    }


WARM64_RUNS = 150  # --workload warm64: about 1 M logged pairs


def run_warm64(args, rank, world, dev):
    """The learned warm start at its stated scale: the network trained on about
    1 M pairs (WARM64_RUNS runs of log_training_runs), then PT on fresh
    64-taxon x 1500-site GTR+G4 alignments (Exp(0.05) branches) from 8
    hill-climbs, threshold 10, 4 rounds with the frontier capped at 256 trees,
    once from the plain start (untimed; the comparison) and once from the
    learned start (one timed step per alignment, its visited table reset).
    Decisions must be identical; the Newton evaluations saved are reported."""
    import torch
    from paper_1811_11007_gb300 import pt, synth
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    w, info = warm_start_weights(rank, WARM64_RUNS)
    setup_s = time.time() - t0
    n, sites, T, R = 64, 1500, 10.0, 4
    ctx = pt.Context(precision="mixed", table_log2=20, stream=stream)
    ctx.mlp_set_weights(w)
    res = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def search(aid, lmax, front, on):
        ctx.mlp_enable(on)
        ctx.reset_visited(aid)
        lm, f = lmax, front
        ev, sc, nl, fronts = 0, 0, 0, []
        e0.record(stream)
        for _ in range(R):
            if not len(f["edges"]):
                break
            lm, f = ctx.expand(aid, f["edges"][:256], f["lengths"][:256], T, lm)
            st = ctx.stats()
            ev += st["prop_evals"]
            sc += st["scored"]
            nl += st["launches"]
            fronts.append((lm, _keys(f["keys"])))
        e1.record(stream)
        torch.cuda.synchronize()
        v = ctx.visited(aid)
        return {"ms": e0.elapsed_time(e1), "evals": ev, "scored": sc, "launches": nl, "fronts": fronts,
                "visited": dict(zip(_keys(v["keys"]), v["status"]))}

    steps = args.steps
    with ClockSampler(dev) as clk:
        for k in range(steps):
            seed = synth.SEED_BASE + 640 + k + 1000 * rank
            a = synth.simulate(n, sites, seed, model="gtr", alpha=0.5, mean_branch=0.05)
            aid = ctx.load_alignment(a.codes)
            ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
            ctx.mlp_enable(False)
            hc = ctx.hill_climb(aid, *synth.random_trees(n, 8, seed + 1))
            lmax, front = ctx.begin(aid, hc["edges"], hc["lengths"], T)
            p = search(aid, lmax, front, False)
            q = search(aid, lmax, front, True)
            same = (p["visited"] == q["visited"] and [x[1] for x in p["fronts"]] == [x[1] for x in q["fronts"]]
                    and all(abs(x[0] - y[0]) <= 1e-3 for x, y in zip(p["fronts"], q["fronts"])))
            res.append({"seed": seed, "patterns": ctx.alignment_info(aid)[1], "scored": q["scored"],
                        "visited": len(q["visited"]), "plain_evals": p["evals"], "learned_evals": q["evals"],
                        "plain_ms": p["ms"], "learned_ms": q["ms"], "launches": q["launches"],
                        "identical_decisions": bool(same),
                        "judge": ctx.mlp_judge(aid)})
    ms = sum(r["learned_ms"] for r in res)
    units = sum(r["scored"] for r in res)
    ms, units = reduce_over_ranks(ms, units, world, device=f"cuda:{dev}")
    if rank != 0:
        return None
    pe, le = sum(r["plain_evals"] for r in res), sum(r["learned_evals"] for r in res)
    return {
        "metric": "branch-optimised topologies/sec (unique NNI neighbours scored per PT round)",
        "value": units / (ms / 1e3), "unit": "topologies/s", "n_gpus": world, "steps": steps, "warmup": 0,
        "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 partials + f64 reductions", "data": "synthetic (seeded simulation)",
        "config": {"workload": f"learned warm start: fresh {n}-taxon x {sites}-site GTR+G4 alignments, 8 hill-climbs, "
                               f"threshold {T}, {R} rounds (frontier <= 256); one step = the learned-start search "
                               f"on one alignment (the plain-start search on it untimed)",
                   "parallelism": f"replicas x{world}", "l2": "per-step working set below L2 (searches, not repeats)"},
        "plain_start_value": sum(r["scored"] for r in res) / (sum(r["plain_ms"] for r in res) / 1e3),
        "newton_evals_saved": 1 - le / pe, "prop_evals_per_neighbour": {"plain": pe / units, "learned": le / units},
        "identical_decisions": all(r["identical_decisions"] for r in res),
        "alignments": res, "learned_warm_start": info, "setup_s": setup_s, "clocks": clk.summary(),
        "gpu_launches": sum(r["launches"] for r in res),
    }


def _oracle_problem(a):
    import oracle
    from paper_1811_11007_gb300 import synth
    tips, w = synth.compress_patterns(a.codes)
    return lambda: oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)


def _time_proposals(problem, edges, lengths, ks, threads):
    """The oracle's proposal optimisation of neighbours ks of one tree, spread
    over a thread pool (each thread its own problem; the C calls release the
    GIL): (wall seconds, lnL per neighbour)."""
    import concurrent.futures
    local = threading.local()

    def one(k):
        if not hasattr(local, "pb"):
            local.pb = problem()
        return local.pb.propose(edges, lengths, int(k))[0]

    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda _: problem(), range(threads)))  # warm the library
        t0 = time.perf_counter()
        out = list(ex.map(one, ks))
        return time.perf_counter() - t0, out


def cpu_baseline(W, a, front, lmax0, info, sample, threads):
    """The oracle as it stands on the host cores (the one leg of the bench that
    runs it), on a bounded sample of the timed round: the proposal optimisation
    of frontier tree 0's first neighbours on a thread pool (measured), one
    pruning per thread (measured), and from those the oracle's time for the
    whole round (the round's own counts of proposals, kept trees and
    full-optimisation sweeps; an oracle sweep is 2n-3 prunings, each followed
    by Newton on one branch).  Also the round's error against the oracle on
    samples: proposals of frontier tree 0 that tree 0 won, and visited trees
    of the next frontier (lnL at the GPU's lengths)."""
    import concurrent.futures
    from paper_1811_11007_gb300 import pt
    n = W["taxa"]
    problem = _oracle_problem(a)
    threads = max(1, threads or (os.cpu_count() or 1))
    k = max(threads, sample or 2 * threads)
    e0, l0 = front["edges"][0], front["lengths"][0]
    dt, lps = _time_proposals(problem, e0, l0, range(min(k, 2 * (n - 3))), threads)
    nprop = len(lps)
    # one pruning per thread, twice
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        pbs = list(ex.map(lambda _: problem(), range(threads)))
        t0 = time.perf_counter()
        for _ in range(2):
            list(ex.map(lambda pb: pb.loglik(e0, l0), pbs))
        t_prune = (time.perf_counter() - t0) / 2  # wall time of `threads` prunings in parallel
    t_prop = dt / nprop * threads  # one proposal on one thread
    t1 = time.perf_counter()
    pbs[0].propose(e0, l0, 0)
    d1 = time.perf_counter() - t1
    S, K, sw = info["scored"], info["kept"], info["full_sweeps"]
    round_s = (S * t_prop + sw * (2 * n - 3) * t_prune) / threads
    # error against the oracle on samples of the timed round
    props = info["props"]
    gk = pt.keys_to_int(props["keys"])
    _, _, nk = __import__("oracle").nni_neighbours(n, e0, l0)
    ok = pt.keys_to_int(nk)
    mine = {kk: x for kk, x, par in zip(gk, props["lnl"], props["parent"]) if par == 0}
    dprop = [abs(mine[ok[j]] - lps[j]) for j in range(nprop) if ok[j] in mine]
    nxt = info["next"]
    nv = min(len(nxt["lnl"]), threads)
    with concurrent.futures.ThreadPoolExecutor(threads) as ex:
        want = list(ex.map(lambda i: pbs[i].loglik(nxt["edges"][i], nxt["lengths"][i]), range(nv)))
    dvis = [abs(want[i] - nxt["lnl"][i]) for i in range(nv)]
    return {"value": S / round_s, "unit": "topologies/s", "cores": threads, "kind": "oracle",
            "sample": f"{nprop} proposal optimisations of frontier tree 0's neighbours in {dt:.1f} s and "
                      f"{threads} prunings in {t_prune:.2f} s on {threads} threads; the round's time modelled from "
                      f"them with its own counts ({S} proposals, {K} kept trees, {sw} full-optimisation sweeps "
                      f"of 2n-3 prunings each): {round_s:.0f} s",
            "proposals_only": {"value": nprop / dt, "unit": "topologies/s", "cores": threads},
            "single_thread": {"value": 1.0 / d1, "unit": "proposals/s", "cores": 1,
                              "sample": f"one proposal optimisation in {d1:.2f} s"},
            "error_vs_oracle": {"proposals_compared": len(dprop),
                                "max_abs_dlnl_proposals": float(max(dprop, default=0.0)),
                                "visits_compared": nv, "max_abs_dlnl_visits": float(max(dvis, default=0.0)),
                                "note": "proposals of frontier tree 0 (oracle propose vs the GPU's score of the same "
                                        "key); visits: oracle lnL at the GPU's optimised lengths"}}


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, same metric and config.  The
    oracle cannot climb or search this workload in the step budget, so its
    frontier tree is the generating topology at its generating lengths; each
    step is the proposal optimisation of `threads` of its neighbours on a
    thread pool.  The visits of kept neighbours are not in the step (one takes
    minutes here), so the value is an upper bound on the oracle's round rate."""
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": f"no reference arm for workload {args.workload}"}))
        return
    W = WORKLOADS[args.workload]
    a, _ = workload(W, 0)
    n = W["taxa"]
    problem = _oracle_problem(a)
    threads = max(1, args.cpu_threads or (os.cpu_count() or 1))
    e0, l0 = a.tree_edges, a.tree_lengths
    m = 2 * (n - 3)
    vals = []
    for it in range(args.warmup + args.steps):
        ks = [(it * threads + j) % m for j in range(threads)]
        dt, _ = _time_proposals(problem, e0, l0, ks, threads)
        if it >= args.warmup:
            vals.append((len(ks), dt))
    units = sum(v[0] for v in vals)
    secs = sum(v[1] for v in vals)
    v = units / secs
    line = {"impl": "reference", "metric": "branch-optimised topologies/sec (unique NNI neighbours scored per PT round)",
            "value": v, "unit": "topologies/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / len(vals), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"proposal optimisations of NNI neighbours of the generating topology, {n} taxa x "
                                   f"{W['sites']} sites, GTR+G4, threshold {W['thresh']} (bounded CPU sample; "
                                   "visits excluded: an upper bound on the oracle's round rate)"},
            "cpu_baseline": {"value": v, "unit": "topologies/s", "cores": threads, "kind": "oracle",
                             "sample": f"{threads} proposal optimisations per step on {threads} threads"},
            "e2e": {"value": v, "unit": "topologies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1811_11007_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    if args.workload in ("batch16", "warm64"):
        out = (run_batch16 if args.workload == "batch16" else run_warm64)(args, rank, world, local)
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    W = WORKLOADS[args.workload]
    out, (a, front, lmax0, info) = run_ours(args, W, rank, world, local)
    if rank == 0:
        if world == 1 and not args.no_cpu:
            out["cpu_baseline"] = cpu_baseline(W, a, front, lmax0, info, args.cpu_sample, args.cpu_threads)
            out["error_vs_oracle"] = out["cpu_baseline"].pop("error_vs_oracle")
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
