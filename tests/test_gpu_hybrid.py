"""The pieces of the surrogate's exact fallback (paper_2508_06559_gb300/hybrid.py).

- pasur_round_reach: the probability of every next-round root under the average strategies
  conserves probability (each round's roots pass on exactly their own reach) and equals the same
  product of strategies along every path computed from the oracle's tree structure;
- pasur_response_reach: the same with one player best-responding, against the oracle's values;
- pasur_batch_create_roots: a batch started from a subset of a round's roots gives those roots
  the utilities of the batch over all roots, bit for bit (roots are independent);
- pasur_batch_set_cut_values: a cut batch given the exact next-round utilities reproduces the
  exact batch's early rounds bit for bit;
- the fallback loop runs and, solving every reached root exactly, ends with an exploitability no
  worse than the surrogate alone;
- tuning a copy of the surrogate on an exact sample of the roots after the cut: with every pool
  sampled the early rounds are the exact batch's bit for bit; with a partial sample the copy fits
  its sample better than the network it started from, which stays unchanged.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

SEEDS = [1, 4, 7]
T = 60


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


def test_round_reach(P, ctx):
    deck = P.pasur_deal(9)
    pools = np.array([sum(1 << int(c) for c in deck[:4])], np.uint64)
    t3 = ctx.pasur_build_round(deck, 3, pools)
    t3.unfold_single()
    p4, s4, c4, _ = t3.pasur_next_roots()
    t4 = ctx.pasur_build_round(deck, 4, p4)
    t4.pasur_unfold(s4, c4)
    t4.pasur_next_roots()
    t3.pasur_cfr_iterate(P.pasur_config_default(iters=T), np.zeros(len(c4), np.float32))
    t4.pasur_cfr_iterate(P.pasur_config_default(iters=T), np.zeros(t4.n_next_roots(), np.float32))
    r4 = t3.pasur_round_reach()
    r5 = t4.pasur_round_reach(root_reach=r4)
    # probability is conserved up to the float32 normalisation of the average strategies (each
    # parent's strategies sum to 1 within a few float32 ulps, over 8 levels per round)
    assert abs(r4.sum() - 1.0) < 1e-6 and abs(r5.sum() - 1.0) < 2e-6 and (r5 >= 0).all()
    # the same product along every path, from the oracle's structure and the GPU's strategies
    ot = O.Tree(deck, 3, pools)
    ot.unfold_single()
    sb = np.asarray(t3.pasur_avg_strategy(), np.float64)
    q = ot.sizes()[1]
    reach, base = np.ones(int(q[0])), 0
    for k in range(1, 9):
        reach = reach[ot.fgt_parents(k)] * sb[base:base + q[k]]
        base += int(q[k])
    _, _, _, lnk = ot.next_roots()
    want = np.bincount(lnk, weights=reach, minlength=len(c4))
    assert np.allclose(r4, want, rtol=1e-12, atol=1e-15)
    for t in (t3, t4):
        t.free()


def test_response_reach(P, ctx):
    """pasur_response_reach: mode 3 is pasur_round_reach (to rounding); with a best responder the
    probability is still conserved, and it equals the reach computed on the host from the
    oracle's node values (its best responses: the first best child) and the GPU's strategies."""
    deck = P.pasur_deal(9)
    pools = np.array([sum(1 << int(c) for c in deck[:4])], np.uint64)
    t3 = ctx.pasur_build_round(deck, 3, pools)
    t3.unfold_single()
    _, _, c4, _ = t3.pasur_next_roots()
    rng = np.random.default_rng(11)
    nxt = rng.normal(0.0, 4.0, len(c4)).astype(np.float32)
    t3.pasur_cfr_iterate(P.pasur_config_default(iters=T), nxt)
    nv = nxt.astype(np.float64)
    # the leaves' reaches are added into their next-round roots in no fixed order: equal to
    # rounding
    assert np.allclose(t3.pasur_response_reach(3, nv), t3.pasur_round_reach(), rtol=1e-12, atol=1e-15)
    ot = O.Tree(deck, 3, pools)
    ot.unfold_single()
    _, _, _, lnk = ot.next_roots()
    leaf = ot.leaf_utilities_linked(lnk, nv)
    sb = np.asarray(t3.pasur_avg_strategy(), np.float64)
    q = ot.sizes()[1]
    for mode in (1, 2):
        got = t3.pasur_response_reach(mode, nv)
        assert abs(got.sum() - 1.0) < 1e-5 and (got >= 0).all()
        vals = ot.node_values(leaf, mode, sb)
        reach, base = np.ones(int(q[0])), 0
        for k in range(8):
            par = ot.fgt_parents(k + 1)
            sig = sb[base:base + q[k + 1]]
            base += int(q[k + 1])
            responder = (mode == 1) == (k % 2 == 0)
            if responder:
                v = vals[k + 1]
                best = {}
                for i in range(len(par)):  # one slot per root: children of a parent are consecutive
                    p = int(par[i])
                    if p not in best or ((v[i] > v[best[p]]) if k % 2 == 0 else (v[i] < v[best[p]])):
                        best[p] = i
                chosen = np.zeros(len(par), bool)
                chosen[list(best.values())] = True
                reach = np.where(chosen, reach[par], 0.0)
            else:
                reach = reach[par] * sig
        want = np.bincount(lnk, weights=reach, minlength=len(c4))
        assert np.allclose(got, want, rtol=1e-12, atol=1e-15), (mode, np.abs(got - want).max())
        print("response reach mode", mode, "roots reached", int((got > 0).sum()), "of", len(got))
    t3.free()


def test_batch_from_roots_and_cut_values(P, ctx):
    decks = np.stack([P.pasur_deal(s) for s in SEEDS])
    cfg = P.pasur_config_default(iters=T, threads=128)
    full = P.Batch(ctx, decks, 0, cfg)
    full.pasur_batch_solve()
    # a batch of rounds 4-6 from every other root of round 4 of each deal
    roots, picked = [], []
    for d in range(len(SEEDS)):
        pools, soff, scores, _ = full.pasur_batch_tree(d, 2).pasur_next_roots()
        sel = np.arange(0, len(scores), 2)
        root_of = np.repeat(np.arange(len(pools)), np.diff(soff))
        g = root_of[sel]
        up = np.unique(g)
        so = np.concatenate([[0], np.cumsum([(g == p).sum() for p in up])]).astype(np.int64)
        roots.append((pools[up], so, scores[sel]))
        picked.append(sel)
    sub = P.Batch(ctx, decks, 3, cfg, roots=roots)
    sub.pasur_batch_solve()
    for d in range(len(SEEDS)):
        u_full = np.asarray(full.pasur_batch_tree(d, 3).pasur_round_utilities())
        u_sub = np.asarray(sub.pasur_batch_tree(d, 3).pasur_round_utilities())
        assert np.array_equal(u_sub, u_full[picked[d]])
    sub.free()
    # a cut batch (rounds 1-3) given the exact round-4 utilities: the exact early rounds
    net = P.Mlp(ctx, seed=3)
    cut = P.Batch(ctx, decks, 0, cfg, last_round=2, mlp=net)
    for d in range(len(SEEDS)):
        cut.pasur_batch_set_cut_values(d, full.pasur_batch_tree(d, 3).pasur_round_utilities())
    with pytest.raises(P.PasurError):
        cut.pasur_batch_set_cut_values(0, np.zeros(3, np.float32))
    cut.pasur_batch_solve()
    for d in range(len(SEEDS)):
        for r in range(3):
            a, b = cut.pasur_batch_tree(d, r), full.pasur_batch_tree(d, r)
            assert np.array_equal(a.pasur_round_utilities(), b.pasur_round_utilities())
            assert np.array_equal(a.pasur_avg_strategy(), b.pasur_avg_strategy())
    cut.free()
    net.free()
    full.free()


def test_fallback_loop(P, ctx):
    import torch

    from paper_2508_06559_gb300 import hybrid as H
    decks = np.stack([P.pasur_deal(s) for s in SEEDS])
    cfg = P.pasur_config_default(iters=T, threads=128)
    full = P.Batch(ctx, decks, 0, cfg)
    full.pasur_batch_solve()
    te = [[full.pasur_batch_tree(d, r) for r in range(6)] for d in range(len(SEEDS))]
    net = P.Mlp(ctx, seed=3)

    def expl(b):
        out = []
        for d in range(len(SEEDS)):
            sig = [b.pasur_batch_tree(d, r).pasur_avg_strategy() for r in range(3)] + [None] * 3
            out.append((P.chain_values(te[d], 1, sig)[0] - P.chain_values(te[d], 2, sig)[0]) / 2)
        return np.array(out)

    alone = P.Batch(ctx, decks, 0, cfg, last_round=2, mlp=net)
    alone.pasur_batch_solve()
    e_alone = expl(alone)
    alone.free()
    b, st = H.solve_hybrid(P, ctx, decks, cfg, net, 0, 2, eps=0.0, max_passes=8, torch=torch)
    e_hyb = expl(b)
    print("exploitability: surrogate alone", e_alone, "with every reached root exact", e_hyb, st)
    assert st["exact_roots"] > 0 and st["exact_roots_added"][-1] == 0
    assert e_hyb.mean() <= e_alone.mean() + 1e-9
    b.free()
    net.free()
    full.free()


@pytest.mark.parametrize("scope", ["batch", "deal"])
def test_tuned_cut(P, ctx, scope):
    """Tuning a copy of the surrogate on an exact sample of the round-4 pools: with every pool
    sampled every root after the cut is exact and the cut batch's rounds 1-3 are the exact batch's
    bit for bit; with a partial sample the sampled roots are counted as exact, the same seeded
    sample is drawn again, the tuning loss falls, the tuned copy fits the exact sample better than
    the network it starts from, and the network itself is left as it was."""
    import torch

    from paper_2508_06559_gb300 import hybrid as H
    decks = np.stack([P.pasur_deal(s) for s in SEEDS])
    cfg = P.pasur_config_default(iters=T, threads=128)
    full = P.Batch(ctx, decks, 0, cfg)
    full.pasur_batch_solve()
    net = P.Mlp(ctx, seed=3)
    params0 = net.get_params()
    b, st = H.solve_hybrid(P, ctx, decks, cfg, net, 0, 2, eps=None, torch=torch, tune_frac=1.0, tune_scope=scope,
                           tune_epochs=3)
    assert st["passes"] == 0 and st["exact_roots"] == st["roots_after_cut"] == st["tune_roots"] > 0
    for d in range(len(SEEDS)):
        for r in range(3):
            x, y = b.pasur_batch_tree(d, r), full.pasur_batch_tree(d, r)
            assert np.array_equal(x.pasur_round_utilities(), y.pasur_round_utilities())
            assert np.array_equal(x.pasur_avg_strategy(), y.pasur_avg_strategy())
    b.free()
    sampled = []
    for _ in range(2):
        b, st = H.solve_hybrid(P, ctx, decks, cfg, net, 0, 2, eps=None, torch=torch, tune_frac=0.3, tune_scope=scope,
                               tune_epochs=20, tune_seed=4)
        assert 0 < st["tune_roots"] == st["exact_roots"] < st["roots_after_cut"]
        assert len(st["tune_loss_first_last"]) == (len(SEEDS) if scope == "deal" else 1)
        for first, last in st["tune_loss_first_last"]:
            assert np.isfinite(first) and last < first
        sampled.append(st["tune_roots"])
        b.free()
    assert sampled[0] == sampled[1]  # the sample is seeded
    # the tuned copy fits its exact sample better than the network it starts from.  Two tunings
    # are not bit-identical: training sums the weight gradients with atomics (split K), and Adam's
    # first steps move every weight by about lr whatever its gradient's size, so a gradient near
    # zero whose sign the summation order flips moves that weight the other way
    cut = full.pasur_batch_tree(0, 2)
    pools, soff, scores, _ = cut.pasur_next_roots()
    sel = H.sample_pools(np.asarray(pools), np.asarray(soff), 0.3, np.random.default_rng(0))
    roots = [H.roots_subset(np.asarray(pools), np.asarray(soff), np.asarray(scores), sel)]
    e = P.Batch(ctx, decks[:1], 3, cfg, roots=roots)
    e.pasur_batch_solve()
    et = e.pasur_batch_tree(0, 3)
    u = np.asarray(et.pasur_round_utilities(), np.float64)
    base = np.asarray(net.predict_next(cut), np.float64)[sel]
    tuner = P.Mlp(ctx, dataset_capacity=len(sel))
    preds = []
    for _ in range(2):
        losses = H.tune_copy(net, tuner, [et], 30, 1e-3, seed=2)
        assert len(losses) == 30 and losses[-1] < losses[0]
        preds.append(np.asarray(tuner.predict_next(cut), np.float64))
    fits = [float(np.mean((p[sel] - u) ** 2)) for p in preds]
    assert max(fits) < np.mean((base - u) ** 2)
    assert abs(fits[0] - fits[1]) <= 0.1 * max(fits)
    assert np.max(np.abs(preds[0] - preds[1])) <= 0.1
    assert np.array_equal(net.get_params(), params0)
    tuner.free()
    e.free()
    with pytest.raises(ValueError):
        H.solve_hybrid(P, ctx, decks, cfg, net, 0, 2, eps=None, tune_frac=0.3, tune_scope="everything")
    net.free()
    full.free()
