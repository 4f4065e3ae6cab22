"""The CFR's work counts against the game tree they come from.

For a round of one root and one score slot, the (active node, slot) pairs the CFR updates per
iteration (pasur_swept_pairs) are the GT nodes that are local (the root, or a child of an active
node) and not the head of a forced-move chain (a subtree that is one path of single moves), and the
swept edges (pasur_solved_sizes) are the local nodes below the root, both counted here from the
exported level structure.  With several slots per root, merging slots that differ only in the
inherited difference never adds work, and a batch's pairs are the sum of its trees'.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_06559_gb300 import build as B
    from paper_2508_06559_gb300 import pasur
    B.build()
    return pasur


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Ctx(0)
    yield c
    c.close()


def local_active(t):
    """Per level, which GT nodes are local and which are active (numpy, from the exported levels)."""
    M = t.pasur_tree_sizes()[0]
    lv = [t.pasur_export_level(k) for k in range(9)]
    chain = [None] * 9
    chain[8] = np.ones(int(M[8]), bool)
    for k in range(7, -1, -1):
        nc = lv[k]["nchild"].astype(np.int64)
        first = np.concatenate([[0], np.cumsum(nc)])[:-1]
        one = nc == 1
        ch = np.zeros(int(M[k]), bool)
        ch[one] = chain[k + 1][first[one]]
        chain[k] = (nc == 0) | ch
    local, active = [None] * 9, [None] * 9
    local[0] = np.ones(int(M[0]), bool)
    for k in range(9):
        active[k] = local[k] & ~chain[k]
        if k < 8:
            local[k + 1] = active[k][lv[k + 1]["parent"]]
    return local, active


@pytest.mark.parametrize("seed", [0, 2, 5, 11])
def test_single_root_counts(P, ctx, seed):
    deck = P.pasur_deal(seed)
    pools = np.array([sum(1 << int(c) for c in deck[:4])], np.uint64)
    t = ctx.pasur_build_round(deck, 5, pools)
    t.unfold_single()
    t.pasur_cfr_iterate(P.pasur_config_default(iters=3))
    local, active = local_active(t)
    pairs = sum(int(a.sum()) for a in active)
    swept = sum(int(x.sum()) for x in local[1:]) if pairs else 0
    assert t.pasur_swept_pairs() == pairs
    assert t.pasur_solved_sizes()[1] == swept
    t.free()


def test_merged_pairs_and_batch_sum(P, ctx):
    decks = np.stack([P.pasur_deal(s) for s in (1, 4, 7)])
    got = {}
    for merge in (1, 0):
        b = P.Batch(ctx, decks, 3, P.pasur_config_default(iters=4, threads=128, merge_delta=merge))
        b.pasur_batch_solve()
        trees = [b.pasur_batch_tree(d, r) for d in range(3) for r in (3, 4, 5)]
        per_tree = [t.pasur_swept_pairs() for t in trees]
        swept = [t.pasur_solved_sizes()[1] for t in trees]
        assert b.pasur_batch_pairs() == sum(per_tree)
        assert all(0 < p <= e for p, e in zip(per_tree, swept))
        got[merge] = per_tree
        b.free()
    assert all(a <= b for a, b in zip(got[1], got[0])) and sum(got[1]) < sum(got[0])
