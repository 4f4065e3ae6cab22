"""Batched solve of several deals (one merged persistent launch per round and size class, under a
captured CUDA graph) against the per-tree path and the oracle.

Every work item's arithmetic depends only on its own subtree, so the batch must reproduce the
per-tree solves bit for bit whatever block sizes the autotuner picks and whichever deals share a
launch; replaying the graph must reproduce the first solve bit for bit; and the deals' root values
must match the oracle's chained solve of the same rounds.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

SEEDS = [0, 1, 2, 5, 9]
FIRST, T = 4, 300


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_06559_gb300 import build as B
    from paper_2508_06559_gb300 import pasur as P
    B.build()
    c = P.Ctx(0)
    yield c
    c.close()


def P():
    from paper_2508_06559_gb300 import pasur
    return pasur


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


def per_tree_solve(ctx, deck, first, cfg):
    """The same rounds through the single-tree entry points."""
    pools, soff, scores = [mask_ids(deck[:4])], [0, 1], [[0, 0, 0, 0]]
    trees = []
    for r in range(first, 6):
        t = ctx.pasur_build_round(deck, r, pools)
        t.pasur_unfold(soff, scores)
        trees.append(t)
        if r < 5:
            pools, soff, scores, _ = t.pasur_next_roots()
    nxt, out = None, {}
    for i in range(len(trees) - 1, -1, -1):
        trees[i].pasur_cfr_iterate(cfg, nxt)
        out[first + i] = (trees[i].pasur_round_utilities(), trees[i].pasur_avg_strategy())
        nxt = out[first + i][0]
    for t in trees:
        t.free()
    return out


def test_batch_equals_per_tree_and_replays(ctx):
    decks = np.stack([O.deal(s) for s in SEEDS])
    cfg = P().pasur_config_default(iters=T)
    b = P().Batch(ctx, decks, FIRST, cfg)
    u1 = b.pasur_batch_solve()
    got = {(d, r): (b.pasur_batch_tree(d, r).pasur_round_utilities(), b.pasur_batch_tree(d, r).pasur_avg_strategy())
           for d in range(len(SEEDS)) for r in range(FIRST, 6)}
    u2 = b.pasur_batch_solve()  # graph replay
    assert (u1 == u2).all()
    ms, edges, launches = b.pasur_batch_stats()
    assert ms > 0 and edges > 0 and launches > 0
    for d, s in enumerate(SEEDS):
        ref = per_tree_solve(ctx, decks[d], FIRST, cfg)
        for r in range(FIRST, 6):
            assert (got[(d, r)][0] == ref[r][0]).all(), (s, r)
            assert (got[(d, r)][1] == ref[r][1]).all(), (s, r)
        assert u1[d] == ref[FIRST][0][0]
    b.free()


CHAIN_SEEDS, CHAIN_FIRST = [0, 2, 5, 9, 11, 13], 3


def chain_bound(rounds_above: int, umax: float) -> float:
    """Largest |U_gpu - U_oracle| allowed for a root `rounds_above` rounds above the final one,
    each side chaining its own utilities (eq. passuputil).  The final round's utilities agree
    within U_TOL = 1e-5 (the single-round parity bound).  A round's average root utility is a
    mean over iterations of convex combinations of its leaf values, so a leaf perturbation of at
    most e moves it by at most e when the strategies coincide; every round passes its utilities
    up as float32 (a rounding of at most 2^-24 |U|) and its leaves d + u are float32 sums (another
    2^-24 |leaf|), and adds its own f32 CFR error (U_TOL).  Hence e_r <= e_{r+1} + U_TOL +
    2 * 2^-24 * umax, i.e. (rounds_above + 1) * U_TOL + rounds_above * 2^-23 * umax."""
    return (rounds_above + 1) * 1e-5 + rounds_above * 2.0 ** -23 * umax


def test_chain_matches_oracle_chain(ctx):
    """Rounds 4-6 (0-based 3-5) of several deals: the GPU batch chains its own round utilities
    backward (as the full-game solve does) and so does the oracle; every FGT root of every round
    is compared at the bound derived in chain_bound."""
    from tests import oracle_jobs as J
    decks = np.stack([O.deal(s) for s in CHAIN_SEEDS])
    cfg = P().pasur_config_default(iters=T)
    b = P().Batch(ctx, decks, CHAIN_FIRST, cfg)
    b.pasur_batch_solve()
    got = {(d, r): np.array(b.pasur_batch_tree(d, r).pasur_round_utilities()) for d in range(len(decks))
           for r in range(CHAIN_FIRST, 6)}
    b.free()
    with J.pool(len(decks)) as p:
        want = p.map(J.chain_utilities, [dict(deck=dk, first=CHAIN_FIRST, T=T) for dk in decks])
    worst = {}
    for d in range(len(decks)):
        umax = max(float(np.abs(want[d][r]).max(initial=0)) for r in range(CHAIN_FIRST, 6))
        for r in range(CHAIN_FIRST, 6):
            err = float(np.abs(got[(d, r)] - want[d][r]).max(initial=0))
            worst[r] = max(worst.get(r, 0.0), err)
            assert err <= chain_bound(5 - r, umax), (CHAIN_SEEDS[d], r, err, chain_bound(5 - r, umax))
    print("largest |U_gpu - U_oracle| per round:", {r: f"{e:.2e}" for r, e in sorted(worst.items())})


def test_batch_with_subtrees_at_the_shared_memory_limit(ctx):
    """Seeds 1000..1063 (rounds 4-6) include a root whose subtree needs nearly the whole opt-in
    shared memory of a block; the class budget must leave room for the kernel's static shared
    memory.  The batch runs, and one deal equals its per-tree solve."""
    decks = np.stack([O.deal(s) for s in range(1000, 1064)])
    cfg = P().pasur_config_default(iters=5)
    b = P().Batch(ctx, decks, 3, cfg)
    u = b.pasur_batch_solve()
    assert np.isfinite(u).all()
    got = b.pasur_batch_tree(0, 3).pasur_round_utilities()
    b.free()
    ref = per_tree_solve(ctx, decks[0], 3, cfg)
    assert (got == ref[3][0]).all()
