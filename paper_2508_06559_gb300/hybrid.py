"""The surrogate with the exact solve as its fallback: host logic around the C ABI.

The early rounds of every deal are solved batched with the surrogate's predicted round-start
utilities at the roots after the cut (pasur_batch_create_cut).  Then, pass after pass, the roots
after the cut that the current average strategies reach with probability above eps
(pasur_round_reach chained over the solved rounds) and that are not exact yet are solved exactly
(the later rounds built from just those roots, all deals in one batch: pasur_batch_create_roots);
their exact utilities replace the predictions (pasur_batch_set_cut_values) and the early rounds
are solved again.  It stops when a pass adds no root, or after max_passes.  With eps = 0 every
root the play can reach is exact when it stops; larger eps trade exactness off the likely lines
of play for time.  With select="response" a root is also chosen when a best response of either
player to the other's current average strategies (pasur_response_reach, the best responses taken
on the current after-cut values) reaches it with probability above eps: exploitability is what
best responses gain, and they go where the average strategies rarely do.
"""
from __future__ import annotations

import time

import numpy as np


def root_reach_after_cut(batch, deal: int, first_round: int, last_round: int):
    """Probability of every root after the cut for one deal under the batch's average strategies."""
    r = None
    for rnd in range(first_round, last_round + 1):
        r = batch.pasur_batch_tree(deal, rnd).pasur_round_reach(root_reach=r)
    return r


def response_reach_after_cut(batch, deal: int, first_round: int, last_round: int, cut_values, mode: int):
    """Probability of every root after the cut when one player best-responds (mode 1 Alex, 2 Bob)
    to the other's average strategies, the after-cut roots valued at cut_values: best-response
    values chained backward over the cut rounds, then the reach forward."""
    trees = [batch.pasur_batch_tree(deal, r) for r in range(first_round, last_round + 1)]
    nxt_of = [None] * len(trees)
    nxt = np.asarray(cut_values, np.float64)
    for i in range(len(trees) - 1, -1, -1):
        nxt_of[i] = nxt
        nxt = trees[i].pasur_root_values(mode, next_values=nxt)
    r = None
    for i, t in enumerate(trees):
        r = t.pasur_response_reach(mode, nxt_of[i], root_reach=r)
    return r


def solve_hybrid(P, ctx, decks, cfg, mlp, first_round: int = 0, last_round: int = 2, eps: float = 1e-3,
                 max_passes: int = 4, torch=None, select: str = "reach"):
    """Returns (cut batch, stats).  stats: passes, exact roots per pass, wall seconds, and the
    FGT node-updates of every solve (the cut batch's and the exact sub-batches')."""
    def sync():
        if torch is not None:
            torch.cuda.synchronize()

    t0 = time.perf_counter()
    b = P.Batch(ctx, decks, first_round, cfg, last_round=last_round, mlp=mlp)
    n = len(decks)
    pred, nxt, exact = [], [], []
    for d in range(n):
        t = b.pasur_batch_tree(d, last_round)
        pred.append(np.asarray(mlp.predict_next(t), np.float32).copy())
        pools, soff, scores, _ = t.pasur_next_roots()
        nxt.append((np.asarray(pools, np.uint64), np.asarray(soff, np.int64), np.asarray(scores, np.int16)))
        exact.append(np.zeros(len(scores), bool))
    b.pasur_batch_solve()
    cut_edges = b.pasur_batch_stats()[1]
    updates = cut_edges * cfg.iters
    added = []
    for _ in range(max_passes):
        picks = []
        for d in range(n):
            r = root_reach_after_cut(b, d, first_round, last_round)
            hit = r > eps
            if select == "response":
                for mode in (1, 2):
                    hit |= response_reach_after_cut(b, d, first_round, last_round, pred[d], mode) > eps
            new = hit & ~exact[d]
            picks.append(np.nonzero(new)[0])
        total = int(sum(len(x) for x in picks))
        added.append(total)
        if total == 0:
            break
        roots = []
        for d in range(n):
            pools, soff, scores = nxt[d]
            sel = picks[d]
            root_of = np.repeat(np.arange(len(pools)), np.diff(soff))
            g = root_of[sel]
            up = np.unique(g)
            so = [0]
            for p in up:
                so.append(so[-1] + int((g == p).sum()))
            roots.append((pools[up], np.array(so, np.int64), scores[sel]))
        e = P.Batch(ctx, decks, last_round + 1, cfg, roots=roots)
        e.pasur_batch_solve()
        updates += e.pasur_batch_stats()[1] * cfg.iters
        for d in range(n):
            if len(picks[d]) == 0:
                continue
            u = np.asarray(e.pasur_batch_tree(d, last_round + 1).pasur_round_utilities())
            pred[d][picks[d]] = u  # the sub-batch's roots are the picks in ascending order
            exact[d][picks[d]] = True
            b.pasur_batch_set_cut_values(d, pred[d])
        e.free()
        b.pasur_batch_solve()
        updates += cut_edges * cfg.iters
    sync()
    wall = time.perf_counter() - t0
    n_exact = int(sum(int(x.sum()) for x in exact))
    n_roots = int(sum(len(x) for x in exact))
    return b, dict(passes=len(added), exact_roots_added=added, exact_roots=n_exact, roots_after_cut=n_roots,
                   wall_s=wall, eps=eps, node_updates=updates)
