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

Tuning on the deals at hand (tune_frac > 0) comes first: a seeded sample of each deal's pools
after the cut (every score slot of a sampled pool) is solved exactly in one batch; a copy of the
network, started from the trained weights with fresh Adam state, is trained on those exact
utilities (pasur_mlp_dataset_add_tree, pasur_mlp_train) and predicts the other roots; the sampled
roots keep their exact values.  tune_scope "deal" trains one copy per deal on that deal's sample
alone, "batch" one copy on the samples of all the deals together.  The network's error across
deals, not within one deal, is what the sample corrects: a deal's roots share its cards.
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


def roots_subset(pools, soff, scores, sel):
    """The roots sel (ascending indices into the score slots of pasur_next_roots' pools, soff,
    scores) as (pools, score offsets, scores) for pasur_batch_create_roots."""
    root_of = np.repeat(np.arange(len(pools)), np.diff(soff))
    up, cnt = np.unique(root_of[sel], return_counts=True)
    return pools[up], np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64), scores[sel]


def sample_pools(pools, soff, frac: float, rng):
    """Every score slot of a uniform sample of round(frac x pools) pools (at least one pool when
    there is any), as ascending slot indices."""
    n = len(pools)
    if n == 0 or frac <= 0:
        return np.zeros(0, np.int64)
    k = min(n, max(1, int(round(frac * n))))
    up = np.sort(rng.choice(n, k, replace=False))
    return np.concatenate([np.arange(soff[p], soff[p + 1]) for p in up]).astype(np.int64)


def tune_copy(mlp, tuner, exact_trees, epochs: int, lr: float, seed: int, batch: int = 1024):
    """Copy mlp's weights into tuner (fresh Adam state) and train it on every root of exact_trees
    (solved trees of the first round after the cut) in batches of at most `batch` rows.  Returns
    the epoch losses."""
    tuner.set_params(mlp.get_params())
    tuner.dataset_clear()
    for t in exact_trees:
        tuner.dataset_add_tree(t)
    rows = tuner.dataset_size()
    if rows == 0 or epochs <= 0:
        return np.zeros(0, np.float32)
    return tuner.train(epochs, min(batch, -(-rows // 128) * 128), lr, shuffle_seed=seed)


def solve_hybrid(P, ctx, decks, cfg, mlp, first_round: int = 0, last_round: int = 2, eps=1e-3,
                 max_passes: int = 4, torch=None, select: str = "reach", tune_frac: float = 0.0,
                 tune_scope: str = "batch", tune_epochs: int = 40, tune_lr: float = 1e-3, tune_seed: int = 0):
    """Returns (cut batch, stats).  eps None: no fallback passes (the surrogate, tuned when
    tune_frac > 0, alone).  stats: passes, exact roots per pass, the tuning sample's roots and
    time, wall seconds, and the FGT node-updates of every solve (the cut batch's and the exact
    sub-batches')."""
    def sync():
        if torch is not None:
            torch.cuda.synchronize()

    if tune_scope not in ("deal", "batch") or select not in ("reach", "response"):
        raise ValueError("tune_scope is 'deal' or 'batch', select 'reach' or 'response'")
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
    updates = 0
    tune_roots, tune_s, tune_loss = 0, 0.0, []
    if tune_frac > 0:
        t1 = time.perf_counter()
        picks = [sample_pools(nxt[d][0], nxt[d][1], tune_frac, np.random.default_rng([tune_seed, d]))
                 for d in range(n)]
        e = P.Batch(ctx, decks, last_round + 1, cfg, roots=[roots_subset(*nxt[d], picks[d]) for d in range(n)])
        e.pasur_batch_solve()
        updates += e.pasur_batch_stats()[1] * cfg.iters
        per_deal = tune_scope == "deal"
        cap = max(len(x) for x in picks) if per_deal else sum(len(x) for x in picks)
        tuner = P.Mlp(ctx, dataset_capacity=max(int(cap), 1), seed=tune_seed)
        if not per_deal:
            losses = tune_copy(mlp, tuner, [e.pasur_batch_tree(d, last_round + 1) for d in range(n) if len(picks[d])],
                               tune_epochs, tune_lr, tune_seed)
            tune_loss.append((float(losses[0]), float(losses[-1])) if len(losses) else None)
        for d in range(n):
            if len(picks[d]) == 0:
                continue
            et = e.pasur_batch_tree(d, last_round + 1)
            if per_deal:
                losses = tune_copy(mlp, tuner, [et], tune_epochs, tune_lr, tune_seed + d)
                tune_loss.append((float(losses[0]), float(losses[-1])) if len(losses) else None)
            pred[d] = np.asarray(tuner.predict_next(b.pasur_batch_tree(d, last_round)), np.float32).copy()
            pred[d][picks[d]] = np.asarray(et.pasur_round_utilities())
            exact[d][picks[d]] = True
            b.pasur_batch_set_cut_values(d, pred[d])
        tuner.free()
        e.free()
        tune_roots = int(sum(len(x) for x in picks))
        sync()
        tune_s = time.perf_counter() - t1
    b.pasur_batch_solve()
    cut_edges = b.pasur_batch_stats()[1]
    updates += cut_edges * cfg.iters
    added = []
    for _ in range(max_passes if eps is not None else 0):
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
        e = P.Batch(ctx, decks, last_round + 1, cfg, roots=[roots_subset(*nxt[d], picks[d]) for d in range(n)])
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
                   wall_s=wall, eps=eps, node_updates=updates, tune_roots=tune_roots, tune_s=tune_s,
                   tune_loss_first_last=tune_loss)
