"""Self-play on the GPU against the oracle.

With the same float strategies on both sides (the oracle's average strategy rounded to float32,
passed to both), every game is decided by the same float comparisons on the same Philox draws,
so the GPU's final game differences must equal the oracle sampler's game by game.  With the
GPU's own solved strategies the games are compared in distribution: the sample mean against the
oracle's exact on-policy value (forward distribution pass), within 4 standard errors plus the
value tolerance of two independent CFR solves.  The batched form runs at the size the benchmark
uses (64 deals, rounds 4-6, 10,000 games per deal) and is checked per deal on sampled deals.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

XS = np.arange(-128, 129)


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


def oracle_chain(deck, first, T):
    """Oracle trees, links and fp64 strategies of rounds first..5 from the standalone root."""
    trees, lnks = [], []
    pools, soff, scores = [mask_ids(deck[:4])], np.array([0, 1], np.int64), np.zeros((1, 4), np.int16)
    for r in range(first, 6):
        t = O.Tree(deck, r, pools)
        t.unfold(soff, scores)
        trees.append(t)
        if r < 5:
            pools, soff, scores, lnk = t.next_roots()
            lnks.append(lnk)
    sig = [None] * len(trees)
    u_next = None
    for i in range(len(trees) - 1, -1, -1):
        t = trees[i]
        leaf = t.leaf_utilities_final() if i == len(trees) - 1 else t.leaf_utilities_linked(lnks[i], u_next)
        sig[i], u_next = t.cfr(leaf, T)
    return trees, lnks, sig


def gpu_chain(ctx, deck, first):
    trees = []
    pools, soff, scores = [mask_ids(deck[:4])], [0, 1], [[0, 0, 0, 0]]
    for r in range(first, 6):
        t = ctx.pasur_build_round(deck, r, pools)
        t.pasur_unfold(soff, scores)
        trees.append(t)
        if r < 5:
            pools, soff, scores, _ = t.pasur_next_roots()
    return trees


@pytest.mark.parametrize("seed,first", [(2, 5), (0, 4), (5, 4), (9, 4)])
def test_games_equal_oracle_with_shared_strategy(ctx, seed, first):
    deck = O.deal(seed)
    ot, ol, osig = oracle_chain(deck, first, 150)
    s32 = [s.astype(np.float32) for s in osig]
    gt = gpu_chain(ctx, deck, first)
    N = 20000
    want = O.selfplay(ot, s32, ol, 0, N, 1000 + seed)
    got = ctx.pasur_selfplay(gt, N, 1000 + seed, sigmas=s32)
    assert (got == want).all(), np.flatnonzero(got != want)[:10]
    ms, games = ctx.pasur_last_selfplay_stats()
    assert games == N and ms > 0
    # a prefix of the games does not depend on how many are played
    assert (ctx.pasur_selfplay(gt, 100, 1000 + seed, sigmas=s32) == want[:100]).all()
    for t in gt:
        t.free()


def test_games_from_inner_roots_and_device_buffers(ctx):
    """Games started at several FGT roots of a many-root final round; strategy and results in
    device memory."""
    import torch
    deck = O.deal(0)
    o4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
    o4.unfold_single()
    pools, soff, scores, _ = o4.next_roots()
    o5 = O.Tree(deck, 5, pools)
    o5.unfold(soff, scores)
    s5, _ = o5.cfr(o5.leaf_utilities_final(), 100)
    s32 = s5.astype(np.float32)
    g5 = ctx.pasur_build_round(deck, 5, pools)
    g5.pasur_unfold(soff, scores)
    q0 = int(o5.sizes()[1][0])
    sd = torch.from_numpy(s32).cuda()
    for root_q in [0, 1, q0 // 2, q0 - 1]:
        want = O.selfplay([o5], [s32], [], root_q, 3000, 77)
        out = torch.zeros(3000, dtype=torch.int16, device="cuda")
        ctx.pasur_selfplay([g5], 3000, 77, root_q=root_q, sigmas=[sd], out=out)
        torch.cuda.synchronize()
        assert (out.cpu().numpy() == want).all(), root_q
    g5.free()


def test_games_with_solved_strategy_match_exact_value(ctx):
    from paper_2508_06559_gb300 import pasur as P
    deck = O.deal(0)
    T = 300
    ot, ol, osig = oracle_chain(deck, 4, T)
    gt = gpu_chain(ctx, deck, 4)
    cfg = P.pasur_config_default(iters=T)
    nxt = None
    for t in reversed(gt):
        t.pasur_cfr_iterate(cfg, nxt)
        nxt = t.pasur_round_utilities()
    N = 200000
    got = ctx.pasur_selfplay(gt, N, 4242)
    p = O.outcome_distribution(ot, osig, ol, 0)
    mean, var = (XS * p).sum(), (XS * XS * p).sum() - (XS * p).sum() ** 2
    assert abs(got.mean() - mean) <= 4 * np.sqrt(var / N) + 1e-2, (got.mean(), mean)
    assert set(np.unique(got)) <= set(XS[p > 0]), "a final difference the exact distribution excludes"
    for t in gt:
        t.free()


def test_invalid_arguments(ctx):
    from paper_2508_06559_gb300 import pasur as P
    deck = O.deal(2)
    gt = gpu_chain(ctx, deck, 4)
    q = [t.pasur_tree_sizes()[1] for t in gt]
    sig = [np.full(int(x[1:].sum()), 0.5, np.float32) for x in q]
    assert (ctx.pasur_selfplay(gt, 0, 1, sigmas=sig) == np.zeros(0, np.int16)).all()
    cases = [
        dict(trees=gt, sigmas=None),                 # no CFR run and no strategy
        dict(trees=gt[:1], sigmas=sig[:1]),          # last tree not the final round
        dict(trees=[gt[1], gt[0]], sigmas=sig[::-1]),  # not consecutive
        dict(trees=gt, sigmas=sig, root_q=int(q[0][0])),  # root out of range
    ]
    for c in cases:
        with pytest.raises(P.PasurError) as e:
            ctx.pasur_selfplay(c["trees"], 10, 1, root_q=c.get("root_q", 0), sigmas=c["sigmas"])
        assert e.value.code == P.PASUR_EINVAL
    for t in gt:
        t.free()


def test_batch_selfplay_full_size(ctx):
    """The benchmark's self-play configuration: 64 deals, rounds 4-6 from the standalone root,
    T = 1000, 10,000 games per deal, one launch.  Every deal's games equal the single-chain call
    on the batch's trees (same seeds); sampled deals' outcome means match the oracle's exact
    on-policy value of its own solve."""
    from paper_2508_06559_gb300 import pasur as P
    n_deals, first, T, N = 64, 3, 1000, 10000
    decks = np.stack([O.deal(s) for s in range(n_deals)])
    b = P.Batch(ctx, decks, first, P.pasur_config_default(iters=T))
    b.pasur_batch_solve()
    seeds = np.arange(n_deals, dtype=np.uint64)
    games = b.pasur_batch_selfplay(N, seeds)
    assert games.shape == (n_deals, N)
    assert (np.abs(games.astype(np.int64)) <= 128).all()
    assert (b.pasur_batch_selfplay(N, seeds) == games).all()
    for d in [0, 37, 63]:
        trees = [b.pasur_batch_tree(d, r) for r in range(first, 6)]
        assert (ctx.pasur_selfplay(trees, N, int(seeds[d])) == games[d]).all(), d
    for d in [0, 37]:
        ot, ol, osig = oracle_chain(decks[d], first, T)
        p = O.outcome_distribution(ot, osig, ol, 0)
        mean, var = (XS * p).sum(), (XS * XS * p).sum() - (XS * p).sum() ** 2
        assert abs(games[d].mean() - mean) <= 4 * np.sqrt(var / N) + 1e-2, (d, games[d].mean(), mean)
    b.free()
