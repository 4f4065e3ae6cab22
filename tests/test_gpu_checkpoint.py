"""Checkpoint and resume of a round's CFR (pasur_save_round / pasur_load_round).

A run of T1 iterations, saved, loaded into a tree built and set up the same way and continued for
T2 iterations, gives the average strategies and root utilities of the uninterrupted T1 + T2 run
bit for bit: vanilla and DCFR, a final round and a round fed next-round utilities, with resident
items and with clusters.  A checkpoint is refused by a tree of another deal, by a tree given other
next-round utilities, and when truncated.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

T1, T2 = 30, 45


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


def round_tree(P, ctx, seed, rnd):
    """Round rnd of seed's deal unfolded over the end states of the round before (one root and
    slot when rnd is the first), with next-round utilities for a non-final round."""
    deck = P.pasur_deal(seed)
    pools = np.array([sum(1 << int(c) for c in deck[:4])], np.uint64)
    soff, sc = np.array([0, 1], np.int64), np.zeros((1, 4), np.int16)
    prev = None
    for r in range(rnd - 1, rnd + 1):
        t = ctx.pasur_build_round(deck, r, pools)
        t.pasur_unfold(soff, sc)
        if r < 5:
            pools, soff, sc, _ = t.pasur_next_roots()
        if prev is not None:
            prev.free()
        prev = t
    nxt = None
    if rnd < 5:
        nxt = (np.sin(np.arange(len(sc))) * 3).astype(np.float32)
    return prev, nxt


@pytest.mark.parametrize("seed,rnd,variant,extra", [(9, 5, 0, {}), (5, 5, 1, {}), (3, 4, 0, {}),
                                                    (9, 5, 0, {"split_bytes": 4096})])
def test_resume_is_bit_identical(P, ctx, seed, rnd, variant, extra):
    cfg = lambda it: P.pasur_config_default(iters=it, variant=variant, **extra)  # noqa: E731
    a, nxt = round_tree(P, ctx, seed, rnd)
    a.pasur_cfr_iterate(cfg(T1), nxt)
    a.pasur_cfr_iterate(cfg(T2), nxt)
    want_s, want_u = np.array(a.pasur_avg_strategy()), np.array(a.pasur_round_utilities())
    b, _ = round_tree(P, ctx, seed, rnd)
    b.pasur_cfr_iterate(cfg(T1), nxt)
    ck = b.pasur_save_round()
    b.free()
    c, _ = round_tree(P, ctx, seed, rnd)
    c.pasur_cfr_iterate(cfg(0), nxt)
    c.pasur_load_round(ck)
    c.pasur_cfr_iterate(cfg(T2), nxt)
    assert np.array_equal(np.array(c.pasur_avg_strategy()), want_s)
    assert np.array_equal(np.array(c.pasur_round_utilities()), want_u)
    for t in (a, c):
        t.free()


def test_foreign_checkpoints_are_refused(P, ctx):
    cfg = P.pasur_config_default(iters=10)
    a, nxt = round_tree(P, ctx, 3, 4)
    a.pasur_cfr_iterate(cfg, nxt)
    ck = a.pasur_save_round()
    other, nxt2 = round_tree(P, ctx, 5, 4)
    other.pasur_cfr_iterate(P.pasur_config_default(iters=0), nxt2)
    with pytest.raises(P.PasurError):
        other.pasur_load_round(ck)
    shifted, _ = round_tree(P, ctx, 3, 4)
    shifted.pasur_cfr_iterate(P.pasur_config_default(iters=0), nxt + 1.0)  # other next-round utilities
    with pytest.raises(P.PasurError):
        shifted.pasur_load_round(ck)
    same, _ = round_tree(P, ctx, 3, 4)
    same.pasur_cfr_iterate(P.pasur_config_default(iters=0), nxt)
    with pytest.raises(P.PasurError):
        same.pasur_load_round(ck[:-4])
    same.pasur_load_round(ck)
    for t in (a, other, shifted, same):
        t.free()
