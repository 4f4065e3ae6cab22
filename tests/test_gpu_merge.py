"""Merged score slots (cfg.merge_delta) against solving every slot.

No utility contains the inherited point difference (eq. final_util: the round difference after
CleanUp plus the 7-clubs bonus; eq. passuputil: the round difference plus the next round's
utility, itself free of it), so the slots of a root that differ only in delta have identical
leaf values and identical CFR runs.  Solving one of them and sharing its results must reproduce
the per-slot solve bit for bit: average strategies of every FGT edge, root utilities and leaf
values, in final and non-final rounds, per tree and in the batch.  A non-final round given
next-round utilities that do depend on delta must not merge.  Agreement with the oracle (which
solves every slot) is checked by the parity tests, which run with merging on (the default).
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


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


def chain(P, ctx, seed, first, last):
    """Trees of rounds first..last of a deal from the standalone root, each unfolded over the
    roots the previous one reaches."""
    deck = P.pasur_deal(seed)
    pools = np.array([mask_ids(deck[:4])], np.uint64)
    soff = np.array([0, 1], np.int64)
    sc = np.zeros((1, 4), np.int16)
    trees = []
    for r in range(first, last + 1):
        t = ctx.pasur_build_round(deck, r, pools)
        t.pasur_unfold(soff, sc)
        trees.append(t)
        if r < 5:
            pools, soff, sc, _ = t.pasur_next_roots()
    return trees


def solve_chain(P, trees, T, merge):
    """Solve the chain backward; per round (sigma-bar, U, leaf values, solved sizes)."""
    cfg = P.pasur_config_default(iters=T, merge_delta=merge)
    out = []
    nxt = None
    for t in reversed(trees):
        t.pasur_cfr_iterate(cfg, nxt)
        U = np.array(t.pasur_round_utilities())
        out.append((np.array(t.pasur_avg_strategy()), U, np.array(t.pasur_leaf_values()), t.pasur_solved_sizes()))
        nxt = U
    return out[::-1]


@pytest.mark.parametrize("seed", [0, 3, 9])
def test_merged_chain_is_bit_identical(P, ctx, seed):
    a = chain(P, ctx, seed, 3, 5)
    b = chain(P, ctx, seed, 3, 5)
    ra = solve_chain(P, a, 60, 1)
    rb = solve_chain(P, b, 60, 0)
    merged_any = False
    for t, (sa, ua, la, (ca, ea)), (sb, ub, lb, (cb, eb)) in zip(a, ra, rb):
        q = t.pasur_tree_sizes()[1]
        assert np.array_equal(sa, sb) and np.array_equal(ua, ub) and np.array_equal(la, lb)
        assert (cb == q).all()          # unmerged: every slot solved
        assert (ca <= q).all() and ea <= eb
        merged_any |= bool((ca < q).any())
    assert merged_any  # rounds 5-6 of these deals carry roots with many slots differing in delta
    for t in a + b:
        t.free()


def test_merge_follows_the_given_utilities(P, ctx):
    """Round 5 (0-based 4) unfolded over the end states of rounds 3-4 (roots with several slots),
    given next-round utilities from the caller: utilities that depend on delta forbid merging
    (every slot solved, the result equal to the unmerged solve); utilities that do not allow it."""
    for dep, expect_merge in ((True, False), (False, True)):
        outs = []
        for merge in (1, 0):
            t2, t3, t4 = chain(P, ctx, 3, 2, 4)
            _, _, sc, _ = t4.pasur_next_roots()
            u = (0.5 * sc[:, 0] - 0.25 * sc[:, 1] + (0.125 * sc[:, 2] if dep else 0.0)).astype(np.float32)
            t4.pasur_cfr_iterate(P.pasur_config_default(iters=40, merge_delta=merge), u)
            c, _ = t4.pasur_solved_sizes()
            q = t4.pasur_tree_sizes()[1]
            if merge:
                assert bool((c < q).any()) == expect_merge
            outs.append((np.array(t4.pasur_avg_strategy()), np.array(t4.pasur_round_utilities())))
            for t in (t2, t3, t4):
                t.free()
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("extra", [{}, {"stream_bytes": 1}, {"split_bytes": 4096}])
def test_merged_batch_is_bit_identical(P, ctx, extra):
    decks = np.stack([P.pasur_deal(s) for s in (1, 4, 7)])
    res = []
    for merge in (1, 0):
        b = P.Batch(ctx, decks, 3, P.pasur_config_default(iters=30, threads=128, merge_delta=merge, **extra))
        u = np.array(b.pasur_batch_solve())
        sig = [np.array(b.pasur_batch_tree(d, r).pasur_avg_strategy()) for d in range(3) for r in (3, 4, 5)]
        ut = [np.array(b.pasur_batch_tree(d, r).pasur_round_utilities()) for d in range(3) for r in (3, 4, 5)]
        work = b.pasur_batch_work()
        edges = b.pasur_batch_stats()[1]
        b.free()
        res.append((u, sig, ut, work, edges))
    (u0, s0, t0, w0, e0), (u1, s1, t1, w1, e1) = res
    assert np.array_equal(u0, u1)
    for x, y in zip(s0, s1):
        assert np.array_equal(x, y)
    for x, y in zip(t0, t1):
        assert np.array_equal(x, y)
    assert e0 == e1 and w1[0] == e1 and w0[0] < w1[0] and w0[1] < w1[1]
