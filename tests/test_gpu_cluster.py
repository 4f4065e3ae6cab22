"""Root subtrees split over thread-block clusters (distributed shared memory) against the same
solve in single blocks.  Splitting moves reaches and values between the CTAs of a cluster but
changes no arithmetic, so with any split (forced here through cfg.split_bytes) the average
strategies and root utilities must be bit-identical to the unsplit solve, which the parity tests
pin to the oracle.  Also run: the DCFR variant, continuation over several calls, the batched form,
and the self-play and exploitability passes that read the split trees' strategies.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


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


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


def chain(ctx, deck, first):
    trees = []
    pools, soff, scores = [mask_ids(deck[:4])], [0, 1], [[0, 0, 0, 0]]
    for r in range(first, 6):
        t = ctx.pasur_build_round(deck, r, pools)
        t.pasur_unfold(soff, scores)
        trees.append(t)
        if r < 5:
            pools, soff, scores, _ = t.pasur_next_roots()
    return trees


def solve(ctx, deck, first, cfg, calls=1):
    trees = chain(ctx, deck, first)
    nxt, out = None, []
    for t in reversed(trees):
        for _ in range(calls):
            t.pasur_cfr_iterate(cfg, nxt)
        nxt = t.pasur_round_utilities()
        out.append((nxt.copy(), t.pasur_avg_strategy()))
    return trees, out


@pytest.mark.parametrize("seed,first,split", [(0, 4, 4096), (2, 4, 2048), (5, 3, 8192), (9, 4, 1)])
def test_split_equals_unsplit(ctx, seed, first, split, capfd, monkeypatch):
    from paper_2508_06559_gb300 import pasur as P
    deck = O.deal(seed)
    base = P.pasur_config_default(iters=200)
    t0, ref = solve(ctx, deck, first, base)
    cut = P.pasur_config_default(iters=200, split_bytes=split)
    capfd.readouterr()
    monkeypatch.setenv("PASUR_VERBOSE", "1")
    t1, got = solve(ctx, deck, first, cut)
    monkeypatch.delenv("PASUR_VERBOSE")
    assert "cluster items:" in capfd.readouterr().err  # the forced split did happen
    for (u0, s0), (u1, s1) in zip(ref, got):
        assert (u0 == u1).all()
        assert (s0 == s1).all()
    for t in t0 + t1:
        t.free()


def test_split_dcfr_and_continuation(ctx):
    from paper_2508_06559_gb300 import pasur as P
    deck = O.deal(2)
    base = P.pasur_config_default(iters=50, variant=1)
    cut = P.pasur_config_default(iters=50, variant=1, split_bytes=3000)
    t0, ref = solve(ctx, deck, 4, base, calls=3)
    t1, got = solve(ctx, deck, 4, cut, calls=3)
    for (u0, s0), (u1, s1) in zip(ref, got):
        assert (u0 == u1).all() and (s0 == s1).all()
    # the split trees' strategies drive self-play and the exploitability passes unchanged
    assert (ctx.pasur_selfplay(t0, 2000, 3) == ctx.pasur_selfplay(t1, 2000, 3)).all()
    assert (P.chain_values(t0, 1) == P.chain_values(t1, 1)).all()
    for t in t0 + t1:
        t.free()


def test_split_in_batch(ctx):
    from paper_2508_06559_gb300 import pasur as P
    decks = np.stack([O.deal(s) for s in (0, 2, 5, 9)])
    base = P.pasur_config_default(iters=100)
    cut = P.pasur_config_default(iters=100, split_bytes=6000)
    b0 = P.Batch(ctx, decks, 3, base)
    b1 = P.Batch(ctx, decks, 3, cut)
    u0, u1 = b0.pasur_batch_solve(), b1.pasur_batch_solve()
    assert (u0 == u1).all()
    for d in range(len(decks)):
        for r in (3, 4, 5):
            assert (b0.pasur_batch_tree(d, r).pasur_avg_strategy() == b1.pasur_batch_tree(d, r).pasur_avg_strategy()).all()
    b0.free()
    b1.free()
