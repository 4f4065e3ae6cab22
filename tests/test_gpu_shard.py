"""Root ranges on the GPU (pasur_cfr_iterate_roots): solving a round's GT roots in ranges and
adding the ranges' root utilities must reproduce the whole-round solve bit for bit, and the
backward chain of paper_2508_06559_gb300/shard.py run with the GPU as the range solver (the
ranks' all-reduce replaced by a sum over ranges solved one after the other on this one GPU) must
equal the unsharded GPU chain bit for bit.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

T = 80


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


def build_chain(ctx, deck, first):
    pools = np.array([sum(1 << int(c) for c in deck[:4])], np.uint64)
    soff, sc = np.array([0, 1], np.int64), np.zeros((1, 4), np.int16)
    out = []
    for r in range(first, 6):
        t = ctx.pasur_build_round(deck, r, pools)
        t.pasur_unfold(soff, sc)
        out.append(t)
        if r < 5:
            pools, soff, sc, _ = t.pasur_next_roots()
    return out


@pytest.mark.parametrize("seed", [3, 9])
def test_ranges_add_up_to_the_round(P, ctx, seed):
    from paper_2508_06559_gb300.shard import partition_roots
    from tests import oracle_jobs as J
    deck = P.pasur_deal(seed)
    cfg = P.pasur_config_default(iters=T)
    full = build_chain(ctx, deck, 4)[-1]
    full.pasur_cfr_iterate(cfg)
    u_full, s_full = full.pasur_round_utilities(), full.pasur_avg_strategy()
    n = int(full.pasur_tree_sizes()[0][0])
    assert n >= 3
    _, gs, _, _ = build_chain(ctx, deck, 4)[0].pasur_next_roots()  # score offsets of the final round
    root_of = J.gpu_root_of(full)
    acc = np.zeros_like(u_full)
    for first, count in partition_roots(full.pasur_root_sizes(), 3):
        t = build_chain(ctx, deck, 4)[-1]
        t.pasur_cfr_iterate_roots(cfg, None, first, count)
        u, s = t.pasur_round_utilities(), t.pasur_avg_strategy()
        lo, hi = int(gs[first]), int(gs[first + count])
        assert not u[:lo].any() and not u[hi:].any()
        roots = list(range(first, first + count))
        idx = J.edge_index(root_of, gs, roots, {g: list(range(int(gs[g + 1] - gs[g]))) for g in roots})
        assert np.array_equal(s[idx], s_full[idx])
        acc += u
        t.free()
    assert np.array_equal(acc, u_full)
    bad = build_chain(ctx, deck, 4)[-1]
    with pytest.raises(P.PasurError):
        bad.pasur_cfr_iterate_roots(cfg, None, 0, n + 1)
    bad.free()
    full.free()


def test_sharded_chain_on_one_gpu(P, ctx):
    """sharded_backward for two ranks, each a host thread with its own context (stream); their
    all-reduce is a sum over the two threads' vectors behind a barrier."""
    import threading

    from paper_2508_06559_gb300.shard import sharded_backward
    deck = P.pasur_deal(9)
    cfg = P.pasur_config_default(iters=T)
    ref = build_chain(ctx, deck, 3)
    nxt, want = None, []
    for t in reversed(ref):
        t.pasur_cfr_iterate(cfg, nxt)
        nxt = t.pasur_round_utilities()
        want.append(nxt)
    want = want[::-1]
    world = 2
    slots, result, errors = [None] * world, {}, []
    bar = threading.Barrier(world)

    def rank_main(rank):
        try:
            c = P.Ctx(0)
            rounds = build_chain(c, deck, 3)

            def solve_range(t, u_next, first, count):
                t.pasur_cfr_iterate_roots(cfg, u_next, first, count)
                return t.pasur_round_utilities()

            def sum_over_ranks(u):
                slots[rank] = u
                bar.wait()
                total = np.sum(slots, axis=0, dtype=np.float32)
                bar.wait()
                return total

            result[rank] = sharded_backward(rounds, lambda t: t.pasur_root_sizes(), solve_range, sum_over_ranks, rank,
                                            world)
            for t in rounds:
                t.free()
            c.close()
        except Exception as e:  # noqa: BLE001 -- reported below
            errors.append(e)
            bar.abort()

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(world)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors
    for rank in range(world):
        for got, w in zip(result[rank], want):
            assert np.array_equal(got, w)
    for t in ref:
        t.free()
