#!/usr/bin/env python
"""Benchmark of the PT hot path: branch-optimised topologies/s.

One step = one PT round on a fixed frontier of F topologies of a 27-taxon,
2000-site GTR+Gamma4 alignment (exchangeabilities ~ Dirichlet(1^6),
frequencies ~ Dirichlet(5^4), alpha 0.5, simulated on a random tree with
Exp(mean 0.05) branches): every NNI neighbour of the frontier is keyed,
deduplicated against the device visited table (reset at the start of the
step), proposal-optimised by Newton on its five NNI branches, thresholded at
lmax - 10, and the kept ones are fully optimised.  The frontier is the one a
PT search (threshold 10, 8 random starts) reaches on the GPU during set-up.
Unit: unique neighbours scored to convergence per second, whole job.

value: device-resident inputs, mixed precision, the round replayed as one
       CUDA graph (pt_graph_run; frontier resident in the graph's buffers).
e2e:   the same graph round through the host-buffer entry points: frontier
       copied in from pinned host memory (pt_graph_set_frontier), next
       frontier copied out (pt_graph_get_next), inside every step.
direct_launch: the same round issued kernel by kernel (pt_expand_frontier_dev);
       its per-stage CUDA events give the kernel times of the rooflines.
fp64:  the plain FP64 GPU path on the same frontier.
--workload batch16: 16 alignments (taxa ~ U[20,100], sites ~ U[300,5000]),
       256 frontier trees each (random topologies with optimised lengths),
       one graph round over all of them per step.
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

N_TAXA, N_SITES, THRESH, N_STARTS = 27, 2000, 10.0, 8
# DRAM bytes per unit of the two persistent kernels on this workload, from one ncu capture of each
# (dram__bytes_read.sum + dram__bytes_write.sum of a 2055-neighbour / 375-tree launch, divided by
# its units; profiles/k_propose_27taxa_925patterns.md, profiles/k_fullopt_27taxa_925patterns.md)
DRAM_PER_NEIGHBOUR = 126.28e6 / 2055
DRAM_PER_KEPT_TREE = 12.488e9 / 375
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default: 50 for round27, ~1 s of timed work; 5 for batch16; 3 for the oracle)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--frontier", type=int, default=256)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-mlp", action="store_true", help="plain Newton start (no learned warm start)")
    p.add_argument("--no-autotune", action="store_true", help="default CTA sizes (for profiling runs)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--cpu-sample", type=int, default=0, help="frontier trees in the CPU baseline sample (0: one per thread)")
    p.add_argument("--cpu-threads", type=int, default=0, help="threads of the CPU baseline (0: all cores)")
    p.add_argument("--workload", default="round27", choices=["round27", "batch16"])
    args = p.parse_args()
    if args.steps is None:  # about a second of timed GPU work; the oracle's steps take ~10 s each
        args.steps = 3 if args.impl == "reference" else (5 if args.workload == "batch16" else 50)
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


def workload(rank: int):
    from paper_1811_11007_gb300 import synth
    seed = synth.SEED_BASE + 2 + 1000 * rank
    a = synth.simulate(N_TAXA, N_SITES, seed, model="gtr", alpha=0.5, mean_branch=0.05)
    starts = synth.random_trees(N_TAXA, N_STARTS, seed + 1)
    return a, starts


def build_frontier(ctx, aid, starts, F):
    """Runs the PT search (threshold 10) until the frontier holds >= F trees;
    returns the largest frontier seen (first F) and the lmax before it."""
    lmax, front = ctx.begin(aid, starts[0], starts[1], THRESH)
    best = (lmax, front)
    rounds = 0
    for _ in range(200):
        if len(front["edges"]) >= F or len(front["edges"]) == 0:
            break
        lmax, front = ctx.expand(aid, front["edges"], front["lengths"], THRESH, lmax)
        rounds += 1
        if len(front["edges"]) > len(best[1]["edges"]):
            best = (lmax, front)
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


def train_warm_start(ctx, rank):
    """Trains the warm-start network on proposals logged from PT searches on
    other alignments of the same shape (untimed set-up), then enables it."""
    from paper_1811_11007_gb300 import synth
    for j in range(3):
        seed = synth.SEED_BASE + 40 + j + 1000 * rank
        a = synth.simulate(N_TAXA, N_SITES, seed, model="gtr", alpha=0.5, mean_branch=0.05)
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        # the same regime as the benchmark frontier: search (threshold 10) until
        # the frontier is large, then log the proposals of the next rounds
        lmax, front, _ = build_frontier(ctx, aid, synth.random_trees(N_TAXA, N_STARTS, seed + 1), 256)
        ctx.reset_visited(aid)  # score the saved frontier's neighbours afresh, as a benchmark step does
        ctx.training_log(True, 1 << 20)
        for _ in range(3):
            if not len(front["edges"]):
                break
            lmax, front = ctx.expand(aid, front["edges"][:256], front["lengths"][:256], THRESH, lmax)
        ctx.training_log(False)
    x, t = ctx.training_pairs()
    rng = np.random.default_rng(synth.SEED_BASE + 99)
    w = np.zeros(27912, np.float32)
    # He-normal hidden layers, small output layer; padding rows/columns zero
    w[0:69 * 128] = rng.normal(0, np.sqrt(2 / 69), 69 * 128)
    w[80 * 128 + 128:80 * 128 + 128 + 128 * 128] = rng.normal(0, np.sqrt(2 / 128), 128 * 128)
    w3 = rng.normal(0, 0.1 * np.sqrt(1 / 128), (128, 8))
    w3[:, 5:] = 0
    o3 = 80 * 128 + 128 + 128 * 128 + 128
    w[o3:o3 + 1024] = w3.ravel()
    ctx.mlp_set_weights(w)
    loss = ctx.mlp_train(2000, batch=1024, lr=2e-3, seed=synth.SEED_BASE + 7)
    ctx.mlp_enable(True)
    return {"train_pairs": int(len(x)), "final_batch_loss": loss,
            "zero_prediction_loss": float(np.mean(np.asarray(t, np.float64) ** 2)) if len(t) else None}


def run_ours(args, rank, world, dev):
    import torch
    from paper_1811_11007_gb300 import pt
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    a, starts = workload(rank)
    n, E = N_TAXA, 2 * N_TAXA - 3
    m = 2 * (n - 3)

    def make(prec):
        ctx = pt.Context(precision=prec, table_log2=22, stream=stream)
        aid = ctx.load_alignment(a.codes)
        ctx.set_model(aid, a.exch, a.freqs, 0.5, 4)
        return ctx, aid

    ctx, aid = make("mixed")
    learned = None
    if not args.no_mlp:
        learned = train_warm_start(ctx, rank)
    lmax0, front, setup_rounds = build_frontier(ctx, aid, starts, args.frontier)
    # CTA sizes tuned on this workload's own rounds: the first untimed warm-up step runs the trials
    ctx.autotune(not args.no_autotune)
    # launches of the two persistent kernels before the first timed step, for profilers
    # (one proposal and one full-optimisation launch per round; begin adds one of the latter)
    print(f"propose_launches_before_timed={setup_rounds + args.warmup}", file=sys.stderr)
    print(f"fullopt_launches_before_timed={setup_rounds + args.warmup + 1}", file=sys.stderr)
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
        lm, cnt = c.expand_dev(i, F, d_e.data_ptr(), d_l.data_ptr(), THRESH, lmax0, cap, o_e.data_ptr(),
                               o_l.data_ptr(), o_n.data_ptr(), o_k.data_ptr())
        st = c.stats()
        times = c.stage_times()
        return st["scored"], st["launches"] + 1, times, st, cnt

    def timed(c, i, step, steps, warmup):
        for _ in range(warmup):
            step(c, i)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        units, launches, prop_ms, part_ms, stats, flops, times = 0, 0, 0.0, 0.0, None, 0.0, {}
        full_ms, full_flops = 0.0, 0.0
        e0.record(stream)
        for _ in range(steps):
            w, l, times, st, _ = step(c, i)
            units += w
            launches += l
            prop_ms += times["propose"]
            part_ms += times["partials"]
            full_ms += times["fullopt_kernel"]
            stats = st
            nb = 5 if c.cfg.propose_mode == 0 else 1
            flops += P * (st["prop_sweeps"] * nb * 2 * 272 + st["prop_evals"] * 100)
            # full optimisation: per sweep (2n-3) edge visits (two sides + sum-table, 2 x 272
            # flops per site) and n-2 refreshes of a vector below a node (272), 100 per evaluation
            full_flops += P * (st["full_sweeps"] * ((2 * n - 3) * 544 + (n - 2) * 272) + st["full_evals"] * 100)
        e1.record(stream)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        ms, units = reduce_over_ranks(ms, units, world, device=f"cuda:{dev}")
        return {"ms": ms, "units": units, "launches": launches, "prop_ms": prop_ms, "part_ms": part_ms,
                "stats": stats, "flops": flops, "times": times, "full_ms": full_ms, "full_flops": full_flops}

    # kernel by kernel: its per-stage CUDA events give the kernel times of the rooflines
    res = timed(ctx, aid, step_dev, args.steps, args.warmup)

    # the round as one CUDA graph, recorded once and replayed every step (the headline)
    g = ctx.graph([aid], [F], [THRESH])
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
        resg = timed(ctx, aid, step_graph, args.steps, args.warmup)
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

    e2e = timed(ctx, aid, step_host, args.steps, 1)
    g.close()

    plain = None
    if learned is not None:
        judge = ctx.mlp_judge(aid)  # the plain start's judgement of the network on this alignment
        ctx.mlp_enable(False)
        plain = timed(ctx, aid, step_dev, max(1, min(args.steps, 3)), 1)
        ctx.mlp_enable(True)
    fp64 = None
    if not args.no_fp64:
        ctx64, aid64 = make("fp64")
        fp64 = timed(ctx64, aid64, step_dev, max(1, min(args.steps, 2)), 1)
        ctx64.close()

    out = None
    if rank == 0:
        pk = peaks()
        value = resg["units"] / (resg["ms"] / 1e3)
        sm_max = pk.get("sm_max_mhz", 2070.0)
        nsm = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        prop_s = res["prop_ms"] / 1e3
        achieved_tf = res["flops"] / prop_s / 1e12 if prop_s > 0 else None
        hbm_peak = pk.get("hbm_gbs", 6800.0)
        alg_bytes = 320.0 * P * res["units"] / max(world, 1)
        ph_s = (res["prop_ms"] + res["part_ms"]) / 1e3
        achieved_gb = alg_bytes / ph_s / 1e9 if ph_s > 0 else None
        st = res["stats"]
        peak_note = f"FP32 FMA: {nsm} SMs x 128 lanes x 2 flop x {sm_max:.0f} MHz (recipe unit counts)"
        prop_roof = {"bound": "alu", "kernel": "k_propose (proposal Newton, five branches)", "achieved": achieved_tf,
                     "peak": alu_peak, "unit": "TFLOP/s", "frac": (achieved_tf / alu_peak) if achieved_tf else None,
                     "traffic": DRAM_PER_NEIGHBOUR * res["stats"]["scored"],
                     "traffic_note": "bytes per launch: ncu DRAM bytes per neighbour x neighbours of this launch",
                     "ms_per_step": res["prop_ms"] / args.steps, "peak_note": peak_note}
        full_tf = res["full_flops"] / (res["full_ms"] / 1e3) / 1e12 if res["full_ms"] > 0 else None
        full_roof = {"bound": "alu", "kernel": "k_fullopt (visit: full optimisation)", "achieved": full_tf,
                     "peak": alu_peak, "unit": "TFLOP/s", "frac": (full_tf / alu_peak) if full_tf else None,
                     "traffic": DRAM_PER_KEPT_TREE * res["stats"]["kept"],
                     "traffic_note": "bytes per launch: ncu DRAM bytes per kept tree x kept trees of this launch",
                     "ms_per_step": res["full_ms"] / args.steps, "peak_note": peak_note}
        dominant = full_roof if res["full_ms"] > res["prop_ms"] else prop_roof
        out = {
            "metric": "branch-optimised topologies/sec (unique NNI neighbours scored per PT round)",
            "value": value,
            "path": ("learned warm start + " if learned is not None else "") +
                    "batched persistent launches replayed as one CUDA graph + FP32 partials / FP64 reductions",
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
            "config": {"workload": f"PT round on a {F}-tree frontier, {N_TAXA} taxa x {N_SITES} sites ({P} patterns), "
                                   f"GTR+G4, threshold {THRESH}",
                       "taxa": N_TAXA, "sites": N_SITES, "patterns": P, "frontier": F,
                       "neighbours_per_step": st["scored"], "kept_per_step": st["kept"],
                       "threshold": THRESH, "parallelism": f"replicas x{world} (independent alignments)",
                       "l2": "inputs larger than L2 (frontier partials ~%.2f GB per step)" % (
                           F * (2 * N_TAXA - 5) * P * 68 / 1e9)},
            "e2e": {"value": e2e["units"] / (e2e["ms"] / 1e3), "unit": "topologies/s",
                    "h2d_bytes_per_step": bytes_io["h2d"], "d2h_bytes_per_step": bytes_io["d2h"]},
            "direct_launch": {"value": res["units"] / (res["ms"] / 1e3), "unit": "topologies/s",
                              "ms_per_step": res["ms"] / args.steps, "gpu_launches": res["launches"],
                              "note": "the same round issued kernel by kernel with host reads of the counts"},
            "graph_check": graph_check,
            "fp64_gpu": ({"value": fp64["units"] / (fp64["ms"] / 1e3), "unit": "topologies/s",
                          "ms_per_step": fp64["ms"] / max(1, min(args.steps, 2)),
                          "note": "plain FP64 GPU path, plain Newton start, same frontier"} if fp64 else None),
            "mixed_plain_start": ({"value": plain["units"] / (plain["ms"] / 1e3), "unit": "topologies/s",
                                   "prop_evals_per_neighbour": plain["stats"]["prop_evals"] /
                                   max(plain["stats"]["scored"], 1)} if plain else None),
            "learned_warm_start": (dict(learned, judge=judge) if learned else None),
            "roofline": dominant,
            "rooflines": {"k_propose": prop_roof, "k_fullopt": full_roof},
            "roofline_hbm": {"bound": "hbm", "achieved": achieved_gb, "peak": hbm_peak, "unit": "GB/s",
                             "frac": (achieved_gb / hbm_peak) if achieved_gb else None,
                             "note": "algorithmic 320*P bytes per neighbour over partials + proposal kernel time; "
                                     "peak = measured copy bandwidth"},
            "stage_ms_per_step": {k: v for k, v in res.get("times", {}).items()},
            "newton": {"prop_evals_per_neighbour": st["prop_evals"] / max(st["scored"], 1),
                       "prop_sweeps_per_neighbour": st["prop_sweeps"] / max(st["scored"], 1),
                       "full_evals_per_kept_tree": st["full_evals"] / max(st["kept"], 1),
                       "full_sweeps_per_kept_tree": st["full_sweeps"] / max(st["kept"], 1),
                       "nonconverged": st["nonconverged"]},
            "autotune": ctx.autotune_report(),
            "gpu_launches": resg["launches"],
            "clocks": clocks,
        }
    return out, (a, front, lmax0)


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
    F = args.frontier
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
    parts = [{"aln": aid, "edges": e, "lengths": l, "threshold": THRESH, "lmax": lm}
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
    g = ctx.graph(ids, [F] * len(ids), [THRESH] * len(ids))
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
                               f"trees each (random topologies, optimised lengths), GTR+G4, threshold {THRESH}",
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


def cpu_baseline(a, front, lmax0, sample, threads):
    """The oracle as it stands on the host cores: one PT round per frontier tree
    of the sample, the trees spread over a thread pool (the oracle's C calls
    release the GIL; each thread has its own problem and search objects)."""
    import concurrent.futures
    import oracle
    from paper_1811_11007_gb300 import synth
    tips, w = synth.compress_patterns(a.codes)
    threads = max(1, threads or (os.cpu_count() or 1))
    k = max(1, min(sample or threads, len(front["edges"])))

    def one(i):
        pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
        s = oracle.Search(pb, front["edges"][i:i + 1], front["lengths"][i:i + 1], THRESH, frontier_lmax=lmax0)
        s.round()
        st = s.stats()
        return st["scored"], st["kept"]

    t0 = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(min(threads, k)) as ex:
        res = list(ex.map(one, range(k)))
    dt = time.perf_counter() - t0
    scored, kept = sum(r[0] for r in res), sum(r[1] for r in res)
    # the same oracle on one core: the round of the first sample tree alone
    t1 = time.perf_counter()
    s1, k1 = one(0)
    d1 = time.perf_counter() - t1
    return {"value": scored / dt, "unit": "topologies/s", "cores": min(threads, k), "kind": "oracle",
            "sample": f"one PT round on each of {k} frontier trees ({scored} neighbours scored, {kept} fully "
                      f"optimised) in {dt:.1f} s on {min(threads, k)} threads",
            "single_thread": {"value": s1 / d1, "unit": "topologies/s", "cores": 1,
                              "sample": f"one PT round on frontier tree 0 ({s1} neighbours scored, {k1} fully "
                                        f"optimised) in {d1:.1f} s on 1 thread"}}


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, same metric and config: each
    step is one PT round on each frontier tree (the oracle's own fully
    optimised random starts), the trees spread over a thread pool."""
    if rank != 0:
        return
    import concurrent.futures
    import oracle
    from paper_1811_11007_gb300 import synth
    a, starts = workload(0)
    tips, w = synth.compress_patterns(a.codes)
    threads = max(1, args.cpu_threads or (os.cpu_count() or 1))
    k = len(starts[0])

    def start(i):
        pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
        lnl, le = pb.full_optimise(starts[0][i], starts[1][i])[:2]
        return lnl, le

    with concurrent.futures.ThreadPoolExecutor(min(threads, k)) as ex:
        opt = list(ex.map(start, range(k)))
    lmax = max(o[0] for o in opt)
    edges = np.ascontiguousarray(starts[0])
    lens = np.stack([o[1] for o in opt])

    def one(i):
        pb = oracle.Problem(tips, w, a.exch, a.freqs, 0.5, 4)
        s = oracle.Search(pb, edges[i:i + 1], lens[i:i + 1], THRESH, frontier_lmax=lmax)
        s.round()
        return s.stats()["scored"]

    vals = []
    with concurrent.futures.ThreadPoolExecutor(min(threads, k)) as ex:
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            scored = sum(ex.map(one, range(k)))
            dt = time.perf_counter() - t0
            if it >= args.warmup:
                vals.append((scored, dt))
    units = sum(v[0] for v in vals)
    secs = sum(v[1] for v in vals)
    v = units / secs
    cores = min(threads, k)
    line = {"impl": "reference", "metric": "branch-optimised topologies/sec (unique NNI neighbours scored per PT round)",
            "value": v, "unit": "topologies/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / len(vals), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"PT round on {k} frontier trees (the fully optimised random starts), {N_TAXA} taxa "
                                   f"x {N_SITES} sites, GTR+G4, threshold {THRESH} (bounded CPU sample)"},
            "cpu_baseline": {"value": v, "unit": "topologies/s", "cores": cores, "kind": "oracle",
                             "sample": f"one PT round on each of {k} start trees per step, {cores} threads"},
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
    if args.workload == "batch16":
        out = run_batch16(args, rank, world, local)
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    out, (a, front, lmax0) = run_ours(args, rank, world, local)
    if rank == 0:
        if world == 1 and not args.no_cpu:
            out["cpu_baseline"] = cpu_baseline(a, front, lmax0, args.cpu_sample, args.cpu_threads)
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
