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
    "batch64": (3, "64 seeded deals (seeds S..S+63), rounds 4-6 (0-based 3-5) of each from the standalone root, "
                   "solved together: one merged persistent launch per round and size class under a CUDA graph"),
    "surrogate64": (0, "64 seeded deals (seeds S..S+63): rounds 1-3 (0-based 0-2) solved in one batch with the "
                       "leaves of round 3 valued by the trained surrogate at the round-4 roots; 10 % of every "
                       "deal's round-4 pools solved exactly (rounds 4-6 from those roots only), a copy of the "
                       "surrogate tuned on their exact utilities, the other roots valued by the tuned copy, the "
                       "sampled ones by their exact utilities, and rounds 1-3 solved again; against the exact "
                       "batched solve of all six rounds"),
}
SUR_DEALS = 64
# the timed form: the surrogate tuned on an exact 10 % sample of the deals' round-4 pools
HYBRID_TIMED = dict(eps=None, tune_frac=0.1, tune_scope="batch")
# frontier forms: (eps, select, tune_frac, tune_scope); eps None = no fallback passes, eps and
# select = the exact fallback for the roots the average strategies ("reach") or best responses
# too ("response") reach with probability above eps
HYBRID_FORMS = ([(None, "reach", 0.0, "batch")] + [(e, "reach", 0.0, "batch") for e in (1e-2, 1e-3, 1e-4, 0.0)]
                + [(e, "response", 0.0, "batch") for e in (1e-2, 1e-3, 1e-4)]
                + [(None, "reach", 0.1, "batch"), (None, "reach", 0.1, "deal"), (None, "reach", 0.2, "batch"),
                   (1e-3, "response", 0.1, "batch"), (1e-3, "response", 0.2, "batch")])
SUR_TRAIN_DEALS = 4096   # training deals (seeds 10000..)
SUR_TRAIN_FRAC = 0.1     # share of each training deal's round-4 pools solved for labels
SUR_LABEL_ITERS = 300
BATCH_DEALS = 64
METRIC = "CFR node-updates/sec"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
ALG_BYTES_PER_UPDATE = 16   # regret and strategy sum, f32, read + write, per node-update
# shared-memory bytes the CFR kernel moves per iteration, counted from its node code (one slot):
# per swept edge the child's regret (read twice, written once), value and strategy sum (read,
# written) and reach (written), 7 words = 28 B; per (active node, slot) pair its two packed entry
# words in each pass, its parent's reach in each pass, its own reach and value, 8 words = 32 B
SMEM_BYTES_PER_EDGE, SMEM_BYTES_PER_PAIR = 28, 32
SMEM_BYTES_PER_CLK_PER_SM = 128  # 32 banks of 4 bytes
CPU_SAMPLE_SECONDS = 12.0
# the first seed (counting from 0) whose complete six-round full game tree has over 1e9 nodes, the
# paper's average deal size: 3.38e9 FGT nodes (seed 0 has 3.4e7)
FULL_GAME_SEED = 47


def mask_of(cards) -> int:
    m = 0
    for c in cards:
        m |= 1 << int(c)
    return m


# ---------------------------------------------------------------------------------------------
# GPU path (through the C ABI)
# ---------------------------------------------------------------------------------------------

SELFPLAY_GAMES = 10000  # self-play games per deal and step
_PINNED: dict = {}


def host_out(torch, key, n: int, dtype):
    """A page-locked host array of n elements (reused across steps, grown when too small): the
    end-to-end leg reads results into pinned memory."""
    buf = _PINNED.get(key)
    itemsize = np.dtype(dtype).itemsize
    if buf is None or buf.numel() < n * itemsize:
        buf = torch.empty(max(n * itemsize, 16), dtype=torch.uint8, pin_memory=True)
        _PINNED[key] = buf
    return buf.numpy()[:n * itemsize].view(dtype)
_DECK_SEEDS: dict = {}


def deck_seed(deck) -> int:
    """Philox key of a deal's self-play: the seed the deal was drawn from."""
    return _DECK_SEEDS[bytes(np.asarray(deck, np.uint8))]


def selfplay_summary(ctx, games):
    ms, n = ctx.pasur_last_selfplay_stats()
    g = games.cpu().numpy() if hasattr(games, "cpu") else games
    return {"games": int(n), "kernel_ms": ms, "alex_win_frac": float((g > 0).mean()), "tie_frac": float((g == 0).mean()),
            "mean_final_diff": float(g.astype(np.float64).mean())}


def solve_deal(P, ctx, deck, first_round: int, T: int, out_device: bool, torch):
    """One step.  Returns (node_updates, cfr_kernel_ms, nontrivial_edges_x_T, bytes_h2d, bytes_d2h, trees_info)."""
    cfg = P.pasur_config_default(iters=T, **SOLVER)
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
    _WORK.clear()
    for t in reversed(trees):
        t.pasur_cfr_iterate(cfg, nxt)
        ms, edges, _ = t.pasur_last_cfr_stats()
        kms += ms
        updates += edges * T
        solved, swept = t.pasur_solved_sizes()
        _WORK["solved"] = _WORK.get("solved", 0) + int(solved[1:].sum()) * T
        _WORK["swept"] = _WORK.get("swept", 0) + swept * T
        _WORK["pairs"] = _WORK.get("pairs", 0) + t.pasur_swept_pairs() * T
        q0 = int(t.pasur_tree_sizes()[1][0])
        if out_device:
            U = torch.empty(q0, dtype=torch.float32, device="cuda")
            sb = torch.empty(max(edges, 1), dtype=torch.float32, device="cuda")
        else:
            U = host_out(torch, ("U", len(outs)), q0, np.float32)
            sb = host_out(torch, ("sb", len(outs)), max(edges, 1), np.float32)
            d2h += U.nbytes + sb.nbytes
        t.pasur_round_utilities(U)
        if edges:
            # the strategies travel to the host while the next round solves (pasur_sync below)
            t.pasur_avg_strategy_async(sb)
        outs.append(sb)
        nxt = U
    root_u = float(nxt[0]) if len(nxt) else 0.0
    # self-play of the solved profile through the rounds (fair value = P(Alex wins))
    if out_device:
        games = torch.empty(SELFPLAY_GAMES, dtype=torch.int16, device="cuda")
    else:
        games = host_out(torch, "games", SELFPLAY_GAMES, np.int16)
        d2h += games.nbytes
    ctx.pasur_selfplay(trees, SELFPLAY_GAMES, int(deck_seed(deck)), sigmas=None, out=games)
    ctx.pasur_sync()
    sp = selfplay_summary(ctx, games)
    info = [(t.pasur_tree_sizes()[1].tolist()) for t in trees]
    for t in trees:
        t.free()
    return updates, kms, d2h, h2d, root_u, info, sp


def solve_batch(P, ctx, decks, first_round: int, T: int, out_device: bool, torch):
    """One step of the batched workload: build every deal's rounds, solve them in the batch,
    write out every tree's average strategies and root utilities, free."""
    cfg = P.pasur_config_default(iters=T, **SOLVER)
    b = P.Batch(ctx, decks, first_round, cfg)
    u = b.pasur_batch_solve()
    ms, edges, launches = b.pasur_batch_stats()
    solved, swept = b.pasur_batch_work()
    _WORK.update(solved=solved * T, swept=swept * T, pairs=b.pasur_batch_pairs() * T)
    d2h = 0
    info = []
    _BATCH_SIZES[:] = [0] * len(decks)
    for d in range(len(decks)):
        for r in range(first_round, 6):
            t = b.pasur_batch_tree(d, r)
            q = t.pasur_tree_sizes()[1]
            _BATCH_SIZES[d] += int(q.sum())
            ne = int(q[1:].sum())
            if out_device:
                U = torch.empty(int(q[0]), dtype=torch.float32, device="cuda")
                sb = torch.empty(max(ne, 1), dtype=torch.float32, device="cuda")
            else:
                U = host_out(torch, ("U", d, r), int(q[0]), np.float32)
                sb = host_out(torch, ("sb", d, r), max(ne, 1), np.float32)
                d2h += U.nbytes + sb.nbytes
            t.pasur_round_utilities(U)
            if ne:
                t.pasur_avg_strategy(sb)
            if d == 0:
                info.append(q.tolist())
    seeds = np.array([deck_seed(dk) for dk in decks], np.uint64)
    if out_device:
        games = torch.empty((len(decks), SELFPLAY_GAMES), dtype=torch.int16, device="cuda")
    else:
        games = host_out(torch, "games", len(decks) * SELFPLAY_GAMES, np.int16).reshape(len(decks), SELFPLAY_GAMES)
        d2h += games.nbytes
    b.pasur_batch_selfplay(SELFPLAY_GAMES, seeds, out=games)
    sp = selfplay_summary(ctx, games)
    b.free()
    return edges * T, ms, d2h, decks.nbytes + seeds.nbytes, float(u[0]), info, sp


_SUR: dict = {}
_BATCH_SIZES: list = []  # FGT nodes of every deal of the last batched step (all solved rounds)
# node-updates of the last step over the solved slots (slots differing only in the inherited
# difference share one solve) and over the swept edges (those with CFR state, i.e. not on a
# forced-move chain): the work the kernels actually do
_WORK: dict = {}
SOLVER: dict = {}  # solver settings from the command line (pasur_config fields)


def size_histogram(sizes):
    """Spread of the deals' FGT sizes: min / median / max and a count per decade."""
    a = np.asarray(sizes, np.float64)
    dec = np.floor(np.log10(np.maximum(a, 1))).astype(int)
    hist = {f"1e{k}-1e{k + 1}": int((dec == k).sum()) for k in range(int(dec.min()), int(dec.max()) + 1)}
    return {"deals": len(a), "min": int(a.min()), "median": float(np.median(a)), "max": int(a.max()),
            "per_decade": hist}


def no_learning_params(P):
    """A network whose output is the estimate without learning: +7 / -7 when the 7-clubs bonus is
    already Alex's / Bob's, else 0."""
    p = np.zeros(P.N_MLP_PARAMS, np.float32)
    per = 256 * 256 + 256
    p[0:65536].reshape(256, 256)[0, 212] = 10
    p[0:65536].reshape(256, 256)[1, 213] = 10
    for l in (1, 2):
        W = p[l * per:l * per + 65536].reshape(256, 256)
        W[0, 0], W[1, 1] = 1, 1
    p[3 * per], p[3 * per + 1] = 0.7, -0.7
    return p


def surrogate_setup(P, ctx, decks, T, torch):
    """Untimed: train the surrogate on exact solves of other deals, solve the bench deals exactly
    (batched, all six rounds, timed for the speedups), then the surrogate's cut in every form of the
    frontier (create + solve + tuning and exact passes, timed), each measured by the exploitability of
    its whole-game profile (rounds 1-3 from the solve under test, rounds 4-6 exact; fp64
    best-response chain over the six exact rounds)."""
    from paper_2508_06559_gb300 import hybrid as H
    t0 = time.perf_counter()
    none = P.Mlp(ctx)
    none.set_params(no_learning_params(P))
    mlp = P.Mlp(ctx, dataset_capacity=2_000_000, seed=7)
    cfg_l = P.pasur_config_default(iters=SUR_LABEL_ITERS)
    # labels on the roots the surrogate is asked about: round-4 roots that play reaches from the
    # deal's start (rounds 1-3 built, not solved), a seeded sample of each deal's pools solved exactly
    for i in range(0, SUR_TRAIN_DEALS, 64):
        dk = np.stack([P.pasur_deal(10000 + i + j) for j in range(64)])
        cut = P.Batch(ctx, dk, 0, cfg_l, last_round=2, mlp=none)
        roots = []
        for d in range(64):
            pools, soff, scores, _ = cut.pasur_batch_tree(d, 2).pasur_next_roots()
            pools, soff, scores = np.asarray(pools, np.uint64), np.asarray(soff, np.int64), np.asarray(scores, np.int16)
            sel = H.sample_pools(pools, soff, SUR_TRAIN_FRAC, np.random.default_rng([1, i + d]))
            roots.append(H.roots_subset(pools, soff, scores, sel))
        cut.free()
        b = P.Batch(ctx, dk, 3, cfg_l, roots=roots)
        b.pasur_batch_solve()
        for d in range(64):
            mlp.dataset_add_tree(b.pasur_batch_tree(d, 3))
        b.free()
    gen_s = time.perf_counter() - t0
    losses = mlp.train(5, 1024, 1e-3, shuffle_seed=1)
    train_ms, steps = mlp.stats()
    cfg = P.pasur_config_default(iters=T, **SOLVER)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    be = P.Batch(ctx, decks, 0, cfg)
    be.pasur_batch_solve()
    torch.cuda.synchronize()
    exact_s = time.perf_counter() - t1
    _, exact_edges, _ = be.pasur_batch_stats()
    te = [[be.pasur_batch_tree(d, r) for r in range(6)] for d in range(len(decks))]
    br = [(P.chain_values(te[d], 1)[0], P.chain_values(te[d], 2)[0]) for d in range(len(decks))]
    expl_exact = [(a - b) / 2 for a, b in br]

    def exploitability_of(bs):
        ex = []
        for d in range(len(decks)):
            sig = [bs.pasur_batch_tree(d, r).pasur_avg_strategy() for r in range(3)] + [None] * 3
            ex.append((P.chain_values(te[d], 1, sig)[0] - P.chain_values(te[d], 2, sig)[0]) / 2)
        return ex

    frontier = []
    for eps, select, frac, scope in HYBRID_FORMS:
        for key, net in (("surrogate", mlp), ("no_learning", none)):
            if key == "no_learning" and (eps is not None or select != "reach" or frac > 0):
                continue
            torch.cuda.synchronize()
            if eps is None and frac == 0:
                t2 = time.perf_counter()
                bs = P.Batch(ctx, decks, 0, cfg, last_round=2, mlp=net)
                bs.pasur_batch_solve()
                torch.cuda.synchronize()
                st = dict(passes=0, exact_roots=0, wall_s=time.perf_counter() - t2)
            else:
                bs, st = H.solve_hybrid(P, ctx, decks, cfg, net, 0, 2, eps=eps, torch=torch, select=select,
                                        tune_frac=frac, tune_scope=scope)
            ex = exploitability_of(bs)
            bs.free()
            gap = float(np.mean(ex)) - float(np.mean(expl_exact))
            frontier.append({"net": key, "eps": eps, "select": select, "tune_frac": frac,
                             "tune_scope": scope if frac > 0 else None, "create_solve_s": st["wall_s"],
                             "tune_s": st.get("tune_s", 0.0),
                             "speedup_vs_exact": exact_s / st["wall_s"], "exploitability_mean": float(np.mean(ex)),
                             "gap_vs_exact": gap, "max_deal_gap": float(np.max(np.array(ex) - np.array(expl_exact))),
                             "passes": st["passes"], "exact_round4_roots": st["exact_roots"],
                             "round4_roots": st.get("roots_after_cut")})
    be.free()
    none.free()
    _SUR.update(mlp=mlp, info={
        "deals": len(decks), "train_deals": SUR_TRAIN_DEALS, "train_pool_frac": SUR_TRAIN_FRAC,
        "train_rows": mlp.dataset_size(),
        "label_iters": SUR_LABEL_ITERS, "data_gen_s": gen_s, "train_ms": train_ms, "adam_steps": steps,
        "train_loss_first_last": [float(losses[0]), float(losses[-1])],
        "exact_batch_s": exact_s, "exact_node_updates": exact_edges * T,
        "exploitability_mean_exact": float(np.mean(expl_exact)),
        "frontier": frontier, "timed_form": HYBRID_TIMED, "target_gap": 1e-3})


def solve_surrogate(P, ctx, decks, first_round: int, T: int, out_device: bool, torch):
    """One step of the surrogate workload: rounds 1-3 of every deal batched with the surrogate at
    the round-4 roots, tuned on an exact sample of them (HYBRID_TIMED); then every tree's average
    strategies and root utilities written out."""
    from paper_2508_06559_gb300 import hybrid as H
    cfg = P.pasur_config_default(iters=T, **SOLVER)
    b, st = H.solve_hybrid(P, ctx, decks, cfg, _SUR["mlp"], 0, 2, torch=torch, **HYBRID_TIMED)
    ms, edges, _ = b.pasur_batch_stats()
    solved, swept = b.pasur_batch_work()
    _WORK.update(solved=solved * T, swept=swept * T, pairs=b.pasur_batch_pairs() * T)
    d2h = 0
    info = []
    for d in range(len(decks)):
        for r in range(0, 3):
            t = b.pasur_batch_tree(d, r)
            q = t.pasur_tree_sizes()[1]
            ne = int(q[1:].sum())
            if out_device:
                U = torch.empty(int(q[0]), dtype=torch.float32, device="cuda")
                sb = torch.empty(max(ne, 1), dtype=torch.float32, device="cuda")
            else:
                U = host_out(torch, ("U", d, r), int(q[0]), np.float32)
                sb = host_out(torch, ("sb", d, r), max(ne, 1), np.float32)
                d2h += U.nbytes + sb.nbytes
            t.pasur_round_utilities(U)
            if ne:
                t.pasur_avg_strategy(sb)
            if d == 0:
                info.append(q.tolist())
    u0 = float(b.pasur_batch_tree(0, 0).pasur_round_utilities()[0])
    b.free()
    return st["node_updates"], ms, d2h, decks.nbytes, u0, info, None


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


def rank_deal_seeds(workload: str, seed: int, rank: int):
    """Seeds of the deals one rank solves: independent replicas, each rank its own deals (weak
    scaling, no collective on the data path)."""
    if workload == "batch64":
        return [seed + rank * BATCH_DEALS + i for i in range(BATCH_DEALS)]
    if workload == "surrogate64":
        return [seed + rank * SUR_DEALS + i for i in range(SUR_DEALS)]
    return [seed + rank]


def reduce_over_ranks(dist, x: float, op: str, device) -> float:
    """max or sum of a per-rank number over all ranks (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(total_updates: float, slowest_seconds: float) -> float:
    """Whole-job throughput: every rank's node-updates over the slowest rank's time."""
    return total_updates / slowest_seconds


def _record(name: str):
    """A committed ncu summary under profiles/ (JSON), or None when it is missing or the kernel
    sources it names have changed since the capture (their sha256 differs)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    h = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return rec if h.hexdigest() == rec["source_sha256"] else None


def recorded_traffic(workload: str, seed: int):
    """DRAM bytes of the CFR kernels (every k_cfr_items and k_cfr_cluster launch of one solve) per
    step from the committed ncu record of this workload, while the kernel source is unchanged
    since the capture; else None."""
    rec = _record(f"cfr_{workload}_seed{seed}.traffic.json")
    if rec is None:
        return None
    return rec["dram_bytes_read_per_solve"] + rec["dram_bytes_write_per_solve"]


def onchip_roofline(swept: int, pairs: int, kernel_ms: float, sm_mhz: float, n_sms: int):
    """The CFR kernel against its on-chip bound: the shared-memory bytes its node code moves (counted
    per swept edge and per (active node, slot) pair) per second of CFR-kernel time, against the
    shared-memory bandwidth of every SM at the SM clock measured during the run (32 banks x 4 B per
    clock), plus the issue and shared-memory counters of the committed ncu record while the source
    is unchanged."""
    if not pairs or not kernel_ms:
        return None
    moved = SMEM_BYTES_PER_EDGE * swept + SMEM_BYTES_PER_PAIR * pairs
    ach = moved / (kernel_ms / 1e3) / 1e9
    peak = SMEM_BYTES_PER_CLK_PER_SM * n_sms * sm_mhz * 1e6 / 1e9
    out = {"bound": "smem", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "bytes_per_step": moved,
           "note": (f"{SMEM_BYTES_PER_EDGE} B per swept edge + {SMEM_BYTES_PER_PAIR} B per (active node, slot) "
                    f"pair per iteration, from the node code; peak = {SMEM_BYTES_PER_CLK_PER_SM} B/clk x {n_sms} SMs "
                    "x median SM clock of the timed region (derived, not measured)")}
    rec = _record("cfr_onchip_full_game_seed47.json")  # the headline deal's final round (one-pass counters)
    if rec is not None:
        out["ncu"] = {k: rec[k] for k in ("workload", "issue_active_pct", "warps_active_pct") if k in rec}
    rec = _record("cfr_onchip_batch64.json")  # shared-memory counters need several passes: a smaller case
    if rec is not None:
        out["ncu_smem"] = {k: rec[k] for k in ("workload", "smem_wavefront_pct_of_peak", "bank_conflict_share") if k in rec}
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def seed0_secondary(P, ctx, T, torch, stream, flush, steps: int = 5, warmup: int = 2):
    """The seed-0 full game (3.4e7 FGT nodes), timed like the main workload: a secondary figure
    beside a paper-scale headline deal."""
    deck = P.pasur_deal(0)
    _DECK_SEEDS[bytes(deck)] = 0
    for _ in range(warmup):
        solve_deal(P, ctx, deck, 0, T, True, torch)
    ms, kms, upd = [], [], 0
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        upd, k, _, _, _, _, _ = solve_deal(P, ctx, deck, 0, T, True, torch)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        kms.append(k)
    m, km = statistics.mean(ms), statistics.mean(kms)
    return {"seed": 0, "steps": steps, "warmup": warmup, "ms_per_step": m, "node_updates_per_step": upd,
            "value": upd / (m / 1e3), "cfr_kernel_ms_per_step": km, "cfr_kernel_node_updates_per_s": upd / (km / 1e3),
            "swept_node_updates_per_step": _WORK.get("swept"), "solved_node_updates_per_step": _WORK.get("solved")}


def run_ours(args, rank, world, dist):
    import torch

    from paper_2508_06559_gb300 import build as B
    from paper_2508_06559_gb300 import pasur as P
    B.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    ctx = P.Ctx(dev, 0, stream.cuda_stream)
    ctx_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    first_round, desc = WORKLOADS[args.workload]
    seeds = rank_deal_seeds(args.workload, args.seed, rank)
    T = args.iters
    decks = np.stack([P.pasur_deal(s) for s in seeds])
    for s, dk in zip(seeds, decks):
        _DECK_SEEDS[bytes(dk)] = s
    if args.workload == "surrogate64":
        deck = decks
        solve = solve_surrogate
        surrogate_setup(P, ctx, deck, T, torch)
    elif args.workload == "batch64":
        deck = decks
        solve = solve_batch
    else:
        deck = decks[0]
        solve = solve_deal
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        solve(P, ctx, deck, first_round, T, True, torch)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = ctx.pasur_launch_count()
    step_ms, kern_ms, work = [], [], []
    updates = 0
    with ClockSampler(dev) as clk:
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1.0)  # L2 flush between timed steps (outside the events)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            u, kms, _, _, root_u, info, sp = solve(P, ctx, deck, first_round, T, True, torch)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            kern_ms.append(kms)
            work.append(dict(_WORK))
            updates = u
        torch.cuda.synchronize()
        wall = time.perf_counter() - t_wall
    launches = ctx.pasur_launch_count() - launches0
    total_ms = reduce_over_ranks(dist, sum(step_ms), "max", "cuda")
    job_updates = reduce_over_ranks(dist, float(updates), "sum", "cuda")
    if dist:
        dist.barrier()

    # end to end through the public API with host buffers (deck and pools in, results out)
    e2e_ms = []
    h2d = d2h = 0
    solve(P, ctx, deck, first_round, T, False, torch)  # untimed: allocates the pinned host buffers
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, d2h, h2d, _, _, _ = solve(P, ctx, deck, first_round, T, False, torch)
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_mean = reduce_over_ranks(dist, statistics.mean(e2e_ms), "max", "cuda")
    secondary = None
    if args.workload == "full_game" and args.seed != 0 and world == 1:
        secondary = seed0_secondary(P, ctx, T, torch, stream, flush)

    if rank != 0:
        return None
    peaks, src = measured_peaks()
    ms_per_step = total_ms / args.steps
    value = job_rate(job_updates, ms_per_step / 1e3)
    kernel_ms = statistics.mean(kern_ms)
    solved = work[-1].get("solved", updates)
    swept = work[-1].get("swept", updates)
    # dominant kernel: the CFR kernel (k_cfr_items, one launch per size class and round); the
    # algorithmic traffic of CFR is the regret and strategy-sum read + write of every edge that
    # carries CFR state, per iteration (the swept node-updates)
    ach_gbs = ALG_BYTES_PER_UPDATE * swept / (kernel_ms / 1e3) / 1e9
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    clocks = clk.summary()
    onchip = onchip_roofline(swept, work[-1].get("pairs", 0), kernel_ms,
                             float(clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)), ctx_sms)
    line = {
        "metric": METRIC, "value": value, "unit": "node-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded deals)",
        "config": {"workload": f"{args.workload}: {desc}", "seed": args.seed, "iters_per_round": T, "solver": dict(SOLVER),
                   "fgt_sizes_per_round": info, "node_updates_per_step": updates,
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{world}"},
        "cfr_kernel": {"ms_per_step": kernel_ms, "node_updates_per_s": updates / (kernel_ms / 1e3),
                       "solved_node_updates_per_s": solved / (kernel_ms / 1e3),
                       "swept_node_updates_per_s": swept / (kernel_ms / 1e3)},
        "work": {"fgt_node_updates_per_step": updates, "solved_node_updates_per_step": solved,
                 "swept_node_updates_per_step": swept,
                 "solved_node_updates_per_s": job_rate(solved, ms_per_step / 1e3),
                 "note": ("value counts every full-game-tree edge per iteration (the paper's FGT); the CFR solves "
                          "one score slot per group of slots of a root that differ only in the inherited point "
                          "difference (identical leaf values, so identical runs; results shared), and keeps "
                          "state only for edges below nodes with more than one path (swept); forced-move chains "
                          "are resolved once")},
        "roofline": {"bound": "hbm", "achieved": ach_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": ach_gbs / hbm_peak,
                     "traffic": recorded_traffic(args.workload, args.seed),
                     "traffic_unit": "bytes per step (every k_cfr_items and k_cfr_cluster launch of one solve; ncu "
                                     "record in profiles/)",
                     "note": (f"k_cfr_items; achieved = {ALG_BYTES_PER_UPDATE} B per swept node-update (R and S "
                              f"read + write) x swept node-updates / CFR kernel time, peak = {src} HBM copy "
                              "bandwidth; the kernel keeps each root's state in shared memory for all T "
                              "iterations, so its DRAM traffic is far below the algorithmic bytes (ncu counters "
                              "in profiles/): the fraction is an HBM-equivalent rate, the kernel is bound on chip "
                              "(shared memory, issue, block barriers): see onchip")},
        "onchip": onchip,
        "e2e": {"value": job_rate(job_updates, e2e_mean / 1e3), "unit": "node-updates/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches // max(1, args.steps),
        "clocks": clocks,
        "root_utility": root_u,
        "selfplay": None if sp is None else dict(
            sp, note="games per deal through every solved round, moves drawn from the average "
                     "strategy with Philox4x64-10 (key = deal seed); inside each timed step"),
        "wall_s_timed": wall,
        "device_memory_peak_bytes": int(ctx.memory()[1]),
    }
    if secondary:
        line["seed0_full_game"] = secondary
    if args.workload == "batch64" and _BATCH_SIZES:
        line["config"]["fgt_nodes_per_deal"] = size_histogram(_BATCH_SIZES)
    if args.workload == "surrogate64":
        si = dict(_SUR["info"])
        si["hybrid_step_s"] = ms_per_step / 1e3
        si["speedup_vs_exact_timed"] = si["exact_batch_s"] / (ms_per_step / 1e3)
        si["note"] = ("exploitability = (BR_Alex - BR_Bob) / 2 of the whole-game profile (rounds 1-3 from the solve "
                      "under test, rounds 4-6 exact), fp64 best-response chain over all six exact rounds; speedups "
                      "compare whole create+solve wall times of the batched forms; eps None = no fallback passes; "
                      "tune_frac = the share of every deal's round-4 pools solved exactly to tune a copy of the "
                      "surrogate (tune_scope deal: one copy per deal, batch: one for all deals)")
        line["surrogate"] = si
    return line


# ---------------------------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)
# ---------------------------------------------------------------------------------------------

ORACLE_KEEP_ROOTS = 4  # GT roots (with all their score slots) kept per round on the way to the final round


def _oracle_round5(workload: str, seed: int):
    """Final-round roots of the workload's deal reached by the oracle's own chain of rounds, each
    earlier round built from its first ORACLE_KEEP_ROOTS GT roots only (a paper-scale deal's full
    round 5 takes the oracle minutes and gigabytes to build; the sample stays genuine end states
    of that deal).  Returns (deck, pools, score offsets, scores)."""
    import oracle as O
    first_round, _ = WORKLOADS[workload]
    deck = O.deal(seed)
    pools, soff, scores = [mask_of(deck[:4])], np.array([0, 1]), np.zeros((1, 4), np.int16)
    for r in range(first_round, 5):
        keep = min(len(pools), ORACLE_KEEP_ROOTS)
        t = O.Tree(deck, r, pools[:keep])
        t.unfold(np.asarray(soff[:keep + 1]), np.asarray(scores[:soff[keep]]))
        pools, soff, scores, _ = t.next_roots()
        del t
    return deck, np.asarray(pools, np.uint64), np.asarray(soff), np.asarray(scores)


def _oracle_job(args):
    """One core: oracle CFR on FGT roots [first, first+count) of the final round, sized to about
    target_s seconds (iterations from a 2-iteration probe of the same roots, at most T).
    Returns (node-updates, CFR seconds, FGT edges, iterations)."""
    workload, seed, first, count, T, target_s = args
    import oracle as O
    deck, pools, soff, scores = _oracle_round5(workload, seed)
    root_of_slot = np.repeat(np.arange(len(pools)), np.diff(soff))
    sel = [(int(root_of_slot[f]), int(f - soff[root_of_slot[f]])) for f in range(first, first + count)]
    roots = sorted({g for g, _ in sel})
    so, sc = [0], []
    for g in roots:
        for _, s_ in [x for x in sel if x[0] == g]:
            sc.append(scores[soff[g] + s_])
        so.append(len(sc))
    t = O.Tree(deck, 5, [int(pools[g]) for g in roots])
    t.unfold(np.array(so), np.array(sc, np.int16))
    edges = int(t.sizes()[1][1:].sum())
    leaf = t.leaf_utilities_final()
    t0 = time.perf_counter()
    t.cfr(leaf, 2)
    probe = (time.perf_counter() - t0) / 2
    Ts = max(1, min(T, int(target_s / max(probe, 1e-9))))
    t0 = time.perf_counter()
    t.cfr(leaf, Ts)
    return edges * Ts, time.perf_counter() - t0, edges, Ts


def oracle_sample(workload: str, seed: int, T: int, target_s: float, cores: int):
    """The fp64 oracle as it stands, on `cores` host cores (one process each, disjoint FGT roots
    of the workload's final round), each sized to about target_s of CPU work.  Returns
    (node-updates, seconds, description): the node-updates of all processes over the longest
    process's CFR time (they run at the same time; process start-up and tree builds excluded)."""
    import multiprocessing as mp
    _, pools, soff, _ = _oracle_round5(workload, seed)
    n_roots = int(soff[-1])
    per_core = max(1, min(n_roots // max(cores, 1), 64))
    jobs = [(workload, seed, (i * per_core) % max(n_roots - per_core + 1, 1), per_core, T, target_s)
            for i in range(cores)]
    if cores == 1:
        res = [_oracle_job(jobs[0])]
    else:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_job, jobs)
    upd = sum(r[0] for r in res)
    secs = max(r[1] for r in res)
    return upd, secs, (f"final round of seed {seed} ({workload}), roots reached through the first "
                       f"{ORACLE_KEEP_ROOTS} GT roots of every earlier round: {cores} processes x {per_core} FGT roots, "
                       f"T={min(r[3] for r in res)}..{max(r[3] for r in res)}, {sum(r[2] for r in res)} FGT edges in all")


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(args):
    """The oracle on all host cores (one process per core, disjoint roots) and on one core."""
    cores = host_cores()
    u, s, desc = oracle_sample(args.workload, args.seed, args.iters, CPU_SAMPLE_SECONDS, cores)
    u1, s1, desc1 = oracle_sample(args.workload, args.seed, args.iters, CPU_SAMPLE_SECONDS / 2, 1)
    return {"value": u / s, "unit": "node-updates/s", "cores": cores, "kind": "oracle", "sample": desc,
            "single_core": {"value": u1 / s1, "unit": "node-updates/s", "cores": 1, "sample": desc1}}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample(args.workload, args.seed, args.iters, 1.0, cores)
    tot_u, tot_s, desc = 0, 0.0, ""
    for _ in range(args.steps):
        u, s, desc = oracle_sample(args.workload, args.seed, args.iters, 6.0, cores)
        tot_u += u
        tot_s += s
    v = tot_u / tot_s
    first_round, wdesc = WORKLOADS[args.workload]
    return {
        "metric": METRIC, "value": v, "unit": "node-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded deals)", "impl": "reference",
        "config": {"workload": f"{args.workload}: {wdesc}", "seed": args.seed, "iters_per_round": args.iters},
        "cpu_baseline": {"value": v, "unit": "node-updates/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "node-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="full_game", choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=None,
                    help=f"deal seed (default: {FULL_GAME_SEED} for full_game, the first seed whose full game tree "
                         "exceeds 1e9 nodes; 0 otherwise)")
    ap.add_argument("--iters", type=int, default=1000)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--slots-per-item", type=int, default=0, help="pasur_config.slots_per_item (0 = automatic)")
    ap.add_argument("--threads", type=int, default=0, help="pasur_config.threads (0 = per class)")
    ap.add_argument("--no-merge", action="store_true", help="solve every score slot (pasur_config.merge_delta = 0)")
    ap.add_argument("--stream-bytes", type=int, default=0,
                    help="pasur_config.stream_bytes: roots needing more state stream over every SM (0 = default rule)")
    ap.add_argument("--split-bytes", type=int, default=0,
                    help="pasur_config.split_bytes: roots needing more state split over a cluster (0 = default rule)")
    args = ap.parse_args()
    if args.seed is None:
        args.seed = FULL_GAME_SEED if args.workload == "full_game" else 0
    SOLVER.update(slots_per_item=args.slots_per_item, threads=args.threads, merge_delta=0 if args.no_merge else 1,
                  stream_bytes=args.stream_bytes, split_bytes=args.split_bytes)
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
