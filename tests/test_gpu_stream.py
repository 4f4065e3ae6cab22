"""The level-streaming sweep of class 5 (roots whose state lives in device memory, one launch per
level step over all SMs) against the block sweep.

A (node, slot) pair runs the same node code in both, so forcing every root onto the streaming
path (cfg.stream_bytes = 1) must reproduce the default solve bit for bit: average strategies and
root utilities, for single-slot and multi-slot roots, vanilla CFR and DCFR, over several
pasur_cfr_iterate calls, and inside the batched solve.  Agreement with the oracle then follows
from the block path's parity tests.
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


def final_round(P, ctx, seed):
    deck = P.pasur_deal(seed)
    t = ctx.pasur_build_round(deck, 5, [mask_ids(deck[:4])])
    t.unfold_single()
    return t


def multi_slot_round(P, ctx, seed):
    """Round 6 (0-based 5) rooted at every end state of round 5: roots with many score slots."""
    deck = P.pasur_deal(seed)
    t4 = ctx.pasur_build_round(deck, 4, [mask_ids(deck[:4])])
    t4.unfold_single()
    pools, soff, scores, _ = t4.pasur_next_roots()
    t4.free()
    t5 = ctx.pasur_build_round(deck, 5, pools)
    t5.pasur_unfold(soff, scores)
    assert int(np.diff(soff).max()) > 1
    return t5


def solve(P, t, calls, **cfg):
    for T in calls:
        t.pasur_cfr_iterate(P.pasur_config_default(iters=T, **cfg))
    return np.array(t.pasur_avg_strategy()), np.array(t.pasur_round_utilities())


@pytest.mark.parametrize("seed", [2, 5])
@pytest.mark.parametrize("variant", [0, 1])
def test_streamed_final_round_is_bit_identical(P, ctx, seed, variant):
    a = final_round(P, ctx, seed)
    b = final_round(P, ctx, seed)
    sa, ua = solve(P, a, [40], variant=variant)
    sb, ub = solve(P, b, [40], variant=variant, stream_bytes=1)
    assert np.array_equal(sa, sb) and np.array_equal(ua, ub)
    a.free()
    b.free()


@pytest.mark.parametrize("seed", [0, 9])
def test_streamed_multi_slot_roots_over_several_calls(P, ctx, seed):
    a = multi_slot_round(P, ctx, seed)
    b = multi_slot_round(P, ctx, seed)
    sa, ua = solve(P, a, [15, 10])
    sb, ub = solve(P, b, [15, 10], stream_bytes=1)
    assert np.array_equal(sa, sb) and np.array_equal(ua, ub)
    assert np.isfinite(ua).all()
    a.free()
    b.free()


def test_streamed_batch_is_bit_identical(P, ctx):
    decks = np.stack([P.pasur_deal(s) for s in (1, 4, 7)])
    out = []
    for extra in ({}, {"stream_bytes": 1}):
        b = P.Batch(ctx, decks, 4, P.pasur_config_default(iters=30, threads=128, **extra))
        u = np.array(b.pasur_batch_solve())
        sig = [np.array(b.pasur_batch_tree(d, 5).pasur_avg_strategy()) for d in range(3)]
        b.free()
        out.append((u, sig))
    (u0, s0), (u1, s1) = out
    assert np.array_equal(u0, u1)
    for x, y in zip(s0, s1):
        assert np.array_equal(x, y)


def test_stream_bytes_must_be_non_negative(P, ctx):
    t = final_round(P, ctx, 2)
    with pytest.raises(P.PasurError) as e:
        t.pasur_cfr_iterate(P.pasur_config_default(iters=5, stream_bytes=-1))
    assert e.value.code == P.PASUR_EINVAL
    t.free()
