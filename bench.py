#!/usr/bin/env python
"""Benchmark: exact round-by-round CFR of seeded Pasur deals on GB300.

One step = the whole hot path for one deal: build every round's game tree (legal moves, level
expansion), the Unfolding Process, the between-round roots and links, T iterations of vanilla CFR
per round solved backward from the final round with the average root utilities passed up, and
the average strategies and root utilities written out.  Metric: CFR node-updates per second
(node-update = one full-game-tree edge in one CFR iteration), whole step included.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload full_game|rounds_4_5|final_round]
                  [--seed S] [--iters T] [--impl ours|reference]

Under torchrun every rank solves its own deal (seed + rank): independent replicas, weak scaling,
no collective on the data path (only the timing barrier and max-over-ranks).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (first round, description)
    "full_game": (0, "full six-round game of one seeded deal, round-by-round backward CFR"),
    "rounds_4_5": (4, "rounds 5-6 (0-based 4-5) of one seeded deal, round 5 unfolded over every score round 4 reaches"),
    "final_round": (5, "final round of one seeded deal as a standalone round, score (0,0,0,0)"),
}
METRIC = "CFR node-updates/sec"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
ALG_FLOPS_PER_UPDATE = 12   # per edge of a node with >= 2 moves (RM 3, reach 1, value 3, regret 3, S 2)
CPU_SAMPLE_SECONDS = 12.0


def mask_of(cards) -> int:
    m = 0
    for c in cards:
        m |= 1 << int(c)
    return m


# ---------------------------------------------------------------------------------------------
# GPU path (through the C ABI)
# ---------------------------------------------------------------------------------------------

def solve_deal(P, ctx, deck, first_round: int, T: int, out_device: bool, torch):
    """One step.  Returns (node_updates, cfr_kernel_ms, nontrivial_edges_x_T, bytes_h2d, bytes_d2h, trees_info)."""
    cfg = P.pasur_config_default(iters=T)
    trees = []
    pools = np.array([mask_of(deck[:4])], np.uint64)
    soff = np.array([0, 1], np.int64)
    scores = np.zeros((1, 4), np.int16)
    h2d = deck.nbytes
    for r in range(first_round, 6):
        t = ctx.pasur_build_round(deck, r, pools)
        t.pasur_unfold(soff, scores)
        h2d += pools.nbytes + soff.nbytes + scores.nbytes
        trees.append(t)
        if r < 5:
            pools, soff, scores, _ = t.pasur_next_roots_nolinks()
    updates, kms, d2h = 0, 0.0, 0
    nxt = None
    outs = []
    for t in reversed(trees):
        t.pasur_cfr_iterate(cfg, nxt)
        ms, edges, _ = t.pasur_last_cfr_stats()
        kms += ms
        updates += edges * T
        q0 = int(t.pasur_tree_sizes()[1][0])
        if out_device:
            U = torch.empty(q0, dtype=torch.float32, device="cuda")
            sb = torch.empty(max(edges, 1), dtype=torch.float32, device="cuda")
        else:
            U = np.empty(q0, np.float32)
            sb = np.empty(max(edges, 1), np.float32)
            d2h += U.nbytes + sb.nbytes
        t.pasur_round_utilities(U)
        if edges:
            t.pasur_avg_strategy(sb)
        outs.append(sb)
        nxt = U
    root_u = float(nxt[0]) if len(nxt) else 0.0
    info = [(t.pasur_tree_sizes()[1].tolist()) for t in trees]
    for t in trees:
        t.free()
    return updates, kms, d2h, h2d, root_u, info


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def run_ours(args, rank, world, dist):
    import torch

    from paper_2508_06559_gb300 import build as B
    from paper_2508_06559_gb300 import pasur as P
    B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    ctx = P.Ctx(dev, 0, stream.cuda_stream)
    first_round, desc = WORKLOADS[args.workload]
    seed = args.seed + rank
    deck = P.pasur_deal(seed)
    T = args.iters
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        solve_deal(P, ctx, deck, first_round, T, True, torch)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = ctx.pasur_launch_count()
    step_ms, kern_ms = [], []
    updates = 0
    with ClockSampler(dev) as clk:
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u, kms, _, _, root_u, info = solve_deal(P, ctx, deck, first_round, T, True, torch)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(kms)
            updates = u
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
    launches = ctx.pasur_launch_count() - launches0
    total_ms = sum(step_ms)
    if dist:
        tt = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
        dist.barrier()

    # end to end through the public API with host buffers (deck and pools in, results out)
    e2e_ms = []
    h2d = d2h = 0
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, d2h, h2d, _, _ = solve_deal(P, ctx, deck, first_round, T, False, torch)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    if dist:
        tt = torch.tensor([statistics.mean(e2e_ms)], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_mean = float(tt.item())
    else:
        e2e_mean = statistics.mean(e2e_ms)

    if rank != 0:
        return None
    peaks, src = measured_peaks()
    ms_per_step = total_ms / args.steps
    value = world * updates / (ms_per_step / 1e3)
    kernel_ms = statistics.mean(kern_ms)
    # dominant kernel: the CFR kernel (one launch per round); algorithmic FLOPs per launch =
    # ALG_FLOPS_PER_UPDATE x edges of nodes with >= 2 moves x T
    nontriv = sum(nontrivial_edges(i) for i in info) if False else None
    ach_flops = ALG_FLOPS_PER_UPDATE * updates / (kernel_ms / 1e3)
    alu_peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6  # FP32 lanes x FMA x clock
    line = {
        "metric": METRIC, "value": value, "unit": "node-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded deals)",
        "config": {"workload": f"{args.workload}: {desc}", "seed": args.seed, "iters_per_round": T,
                   "fgt_sizes_per_round": info, "node_updates_per_step": updates,
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "cfr_kernel": {"ms_per_step": kernel_ms, "node_updates_per_s": updates / (kernel_ms / 1e3)},
        "roofline": {"bound": "alu", "achieved": ach_flops / 1e12, "peak": alu_peak / 1e12, "unit": "TFLOP/s",
                     "frac": ach_flops / alu_peak, "traffic": None,
                     "note": f"k_cfr_items, shared-memory resident; peak = 152 SM x 128 FP32 lanes x 2 x "
                             f"{peaks.get('sm_max_mhz', 2070.0)} MHz ({src} clock)"},
        "e2e": {"value": world * updates / (e2e_mean / 1e3), "unit": "node-updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches // max(1, args.steps),
        "clocks": clk.summary(),
        "root_utility": root_u,
        "wall_s_timed": wall,
    }
    return line


def nontrivial_edges(_):
    return 0


# ---------------------------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)
# ---------------------------------------------------------------------------------------------

def oracle_sample(workload: str, seed: int, T: int, target_s: float):
    """Oracle CFR on a bounded sample of the workload: the final round's first roots (with all
    their score slots), sized to take about target_s on one core.  Returns (updates, seconds, desc)."""
    import oracle as O
    first_round, _ = WORKLOADS[workload]
    deck = O.deal(seed)
    pools, soff, scores = [mask_of(deck[:4])], np.array([0, 1]), np.zeros((1, 4), np.int16)
    for r in range(first_round, 5):
        t = O.Tree(deck, r, pools)
        t.unfold(soff, scores)
        pools, soff, scores, _ = t.next_roots()
        del t
    # probe speed on the first root
    t1 = O.Tree(deck, 5, list(pools[:1]))
    t1.unfold(soff[:2] - soff[0], scores[soff[0]:soff[1]])
    e1 = int(t1.sizes()[1][1:].sum())
    t0 = time.perf_counter()
    t1.cfr(t1.leaf_utilities_final(), 5)
    rate = 5 * e1 / max(time.perf_counter() - t0, 1e-6)
    budget = target_s * rate
    n = 1
    while n < len(pools):
        e = e1 * (n + 1)  # rough
        if e * T > budget:
            break
        n += 1
    ts = O.Tree(deck, 5, list(pools[:n]))
    ts.unfold(soff[:n + 1] - soff[0], scores[soff[0]:soff[n]])
    edges = int(ts.sizes()[1][1:].sum())
    Ts = max(1, min(T, int(budget / max(edges, 1))))
    leaf = ts.leaf_utilities_final()
    t0 = time.perf_counter()
    ts.cfr(leaf, Ts)
    sec = time.perf_counter() - t0
    return edges * Ts, sec, f"final round (round 5) of seed {seed} via {workload}: first {n} GT roots, {edges} FGT edges, T={Ts}"


def cpu_baseline(args):
    u, s, desc = oracle_sample(args.workload, args.seed, args.iters, CPU_SAMPLE_SECONDS)
    return {"value": u / s, "unit": "node-updates/s", "cores": 1, "kind": "oracle", "sample": desc}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    for _ in range(args.warmup):
        oracle_sample(args.workload, args.seed, args.iters, 2.0)
    tot_u, tot_s, desc = 0, 0.0, ""
    for _ in range(args.steps):
        u, s, desc = oracle_sample(args.workload, args.seed, args.iters, 8.0)
        tot_u += u
        tot_s += s
    v = tot_u / tot_s
    first_round, wdesc = WORKLOADS[args.workload]
    return {
        "metric": METRIC, "value": v, "unit": "node-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded deals)", "impl": "reference",
        "config": {"workload": f"{args.workload}: {wdesc}", "seed": args.seed, "iters_per_round": args.iters},
        "cpu_baseline": {"value": v, "unit": "node-updates/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "node-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="full_game", choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--iters", type=int, default=1000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line:
            print(json.dumps(line))
        return
    dist = None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)  # before any CUDA work
    if world > 1:
        import torch
        import torch.distributed as D
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        D.init_process_group("nccl")
        dist = D
    line = run_ours(args, rank, world, dist)
    if line is not None:
        line["cpu_baseline"] = cpu
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
