"""Parity of the CUDA path (through the C ABI) with the fp64 oracle on the same seeded inputs.

Integer work (tree structure, states, running scores, unfolding, next roots, links, leaf values)
must be bit-exact.  Floating point, after the same number of iterations:
  - root utilities agree within U_TOL = 1e-5 absolute, no exception;
  - average strategies agree within 1e-4 absolute on every edge whose parent has own-reach mass
    sum_t pi_p^t(h) >= 1e-3 * T and is well conditioned: the oracle's own recursion carried out
    in float32, and oracle runs whose leaf values carry f32-sized noise (relative and absolute
    1e-6, seeded), each move that edge's average strategy by at most 1e-5.
  - at an ill-conditioned parent (a near-indifferent node, where regret matching flips on noise
    of that size even in fp64, so the split between its moves is not fixed by the arithmetic)
    an edge beyond 1e-4 needs value parity instead: swapping the oracle's average strategy at
    that one node for the GPU's moves the round root's value under the oracle's average
    strategies (the node's reach probability times the change of its own value, with the
    oracle's on-policy values of its children) by at most VALUE_TOL = 1e-5 plus what the
    oracle's own float32 recursion and noisy-leaf runs move it by at that node (the arithmetic's
    own limit: the fp64 oracle carried out in float32 lands there too), and never by more than
    VALUE_CAP = 1e-3.  The count of such edges and parents, the largest strategy difference
    there and the value changes are printed;
  - at rarely reached parents the strategy must be a valid distribution.
"""
import numpy as np
import pytest

import oracle as O
from tests.oracle_jobs import check_sigma, check_utilities, oracle_sensitivity, own_mass

pytestmark = pytest.mark.gpu


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


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


def compare_tree(gt, ot):
    gs, gq = gt.pasur_tree_sizes()
    os_, oq = ot.sizes()
    assert gs.tolist() == os_.tolist()
    for k in range(9):
        g = gt.pasur_export_level(k)
        o = ot.level(k)
        assert (g["parent"] == o.parent).all(), k
        assert (g["nchild"] == o.nchild).all(), k
        assert (g["lay"] == o.lay).all(), k
        assert (g["pick"] == o.pick).all(), k
        assert (g["state"] == o.state).all(), k
        assert (g["rus"] == o.rus).all(), k


def unfold_both(gt, ot, score_off, scores):
    q1 = gt.pasur_unfold(score_off, scores)
    q2 = ot.unfold(score_off, scores)
    assert q1.tolist() == q2.tolist()
    return q1


def compare_cfr(gt, ot, leaf_o, T, variant=0, next_util=None, tau=1e-6):
    cfg = P().pasur_config_default(iters=T, variant=variant, rm_deadzone=tau)
    gt.pasur_cfr_iterate(cfg, next_util)
    sb_o, U_o, R_o, S_o = ot.cfr(leaf_o, T, tau=tau, variant=variant, want_rs=True)
    leaf_g = gt.pasur_leaf_values()
    assert np.allclose(leaf_g, leaf_o, atol=1e-5, rtol=0)
    U_g = gt.pasur_round_utilities()
    sb_g = gt.pasur_avg_strategy()
    pert = []
    dp, _ = oracle_sensitivity(ot, leaf_o, sb_o, U_o, T, variant, tau, keep=pert)
    du = check_utilities(U_g, U_o)
    check_sigma(ot, leaf_o, sb_g, sb_o, own_mass(ot, S_o), dp, T, f" T={T} variant={variant} max|dU| {du:.2e}",
                perturbed=pert)
    return U_g, U_o, sb_g, sb_o


# ---- structure --------------------------------------------------------------------------------

@pytest.mark.parametrize("seed,rnd", [(0, 5), (2, 5), (0, 4), (7, 2), (11, 0)])
def test_round_tree_bit_exact_single_root(ctx, seed, rnd):
    deck = O.deal(seed)
    pools = [mask_ids(deck[:4])]
    compare_tree(ctx.pasur_build_round(deck, rnd, pools), O.Tree(deck, rnd, pools))


def test_round_tree_bit_exact_many_roots(ctx):
    # next roots of round 4 of seed 0 (the config of rounds 5-6) as round-5 roots, plus edge cases:
    # an empty pool, a pool of Kings/Queens/Jacks, a pool full of small numerics
    deck = O.deal(0)
    t4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
    t4.unfold_single()
    pools, soff, scores, lnk = t4.next_roots()
    hands = mask_ids(deck[44:52])
    extra = [0]
    free = [c for c in range(52) if not hands >> c & 1]
    extra.append(mask_ids([c for c in free if c >= 40][:6]))
    extra.append(mask_ids([c for c in free if c < 20][:10]))
    allp = sorted(set(int(p) for p in pools) | set(extra))
    compare_tree(ctx.pasur_build_round(deck, 5, allp), O.Tree(deck, 5, allp))


def test_empty_root_list(ctx):
    deck = O.deal(1)
    t = ctx.pasur_build_round(deck, 5, np.zeros(0, np.uint64))
    assert t.pasur_tree_sizes()[0].tolist() == [0] * 9
    q = t.pasur_unfold(np.zeros(1, np.int64), np.zeros((0, 4), np.int16))
    assert q.tolist() == [0] * 9
    t.pasur_cfr_iterate(P().pasur_config_default(iters=10))
    assert t.pasur_round_utilities().shape == (0,)


def test_invalid_arguments(ctx):
    deck = O.deal(3)
    pool = mask_ids(deck[:4])
    with pytest.raises(P().PasurError) as e:
        ctx.pasur_build_round(deck, 6, [pool])
    assert e.value.code == P().PASUR_EINVAL
    with pytest.raises(P().PasurError):
        ctx.pasur_build_round(deck, 5, [pool, pool])  # not strictly ascending
    with pytest.raises(P().PasurError):
        ctx.pasur_build_round(deck, 5, [pool | (1 << int(deck[44]))])  # overlaps Alex's hand
    t = ctx.pasur_build_round(deck, 4, [pool])
    with pytest.raises(P().PasurError):
        t.pasur_cfr_iterate(P().pasur_config_default(iters=1))  # not unfolded
    t.unfold_single()
    with pytest.raises(P().PasurError):
        t.pasur_cfr_iterate(P().pasur_config_default(iters=1))  # non-final round without next roots
    with pytest.raises(P().PasurError):
        t.pasur_unfold([0, 2], [[0, 0, 1, 0], [0, 0, 0, 0]])  # already unfolded / unsorted


# ---- unfolding, next roots, leaves --------------------------------------------------------------

def test_next_roots_and_links_bit_exact(ctx):
    deck = O.deal(0)
    pool = mask_ids(deck[:4])
    g4 = ctx.pasur_build_round(deck, 4, [pool])
    o4 = O.Tree(deck, 4, [pool])
    unfold_both(g4, o4, [0, 2], [[0, 0, -3, 0], [2, 5, 1, 0]])
    gp, gs, gsc, gl = g4.pasur_next_roots()
    op, os_, osc, ol = o4.next_roots()
    assert gp.tolist() == op.tolist() and gs.tolist() == os_.tolist()
    assert (gsc == osc).all() and (gl == ol).all()


def test_final_leaf_values_bit_exact(ctx):
    deck = O.deal(5)
    pools = [0, mask_ids(deck[:4])]
    gt = ctx.pasur_build_round(deck, 5, pools)
    ot = O.Tree(deck, 5, pools)
    so = [0, 3, 5]
    sc = [[0, 0, 0, 0], [3, 4, 2, 0], [6, 0, -7, 0], [0, 0, 4, 1], [0, 0, 9, 2]]
    unfold_both(gt, ot, so, sc)
    gt.pasur_cfr_iterate(P().pasur_config_default(iters=0))
    assert (gt.pasur_leaf_values() == ot.leaf_utilities_final()).all()


# ---- CFR ----------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 2, 5, 9])
def test_cfr_final_round_single_root(ctx, seed):
    """Final round of a seeded deal standalone (seed 0 is the paper-config round; 2, 5, 9 are
    non-degenerate), T = 1000."""
    deck = O.deal(seed)
    pools = [mask_ids(deck[:4])]
    gt, ot = ctx.pasur_build_round(deck, 5, pools), O.Tree(deck, 5, pools)
    gt.unfold_single()
    ot.unfold_single()
    compare_cfr(gt, ot, ot.leaf_utilities_final(), 1000)


def test_cfr_many_roots_and_slots(ctx):
    """Round 5 over the 37 next pools of seed 0's round 4, each with several score slots
    (clubs near the bonus threshold so that the bonus differs between slots)."""
    deck = O.deal(0)
    t4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
    t4.unfold_single()
    pools, _, _, _ = t4.next_roots()
    rng = np.random.default_rng(4)
    soff, scores = [0], []
    for _ in pools:
        k = int(rng.integers(1, 6))
        rows = {(int(rng.integers(0, 7)), int(rng.integers(0, 7)), int(rng.integers(-9, 10)), 0) for _ in range(k)}
        rows = sorted(rows)
        scores += rows
        soff.append(len(scores))
    gt, ot = ctx.pasur_build_round(deck, 5, pools), O.Tree(deck, 5, pools)
    unfold_both(gt, ot, soff, scores)
    compare_cfr(gt, ot, ot.leaf_utilities_final(), 500)


def test_cfr_split_calls_equal_one_call(ctx):
    deck = O.deal(2)
    pools = [mask_ids(deck[:4])]
    a, b = ctx.pasur_build_round(deck, 5, pools), ctx.pasur_build_round(deck, 5, pools)
    a.unfold_single()
    b.unfold_single()
    a.pasur_cfr_iterate(P().pasur_config_default(iters=300))
    a.pasur_cfr_iterate(P().pasur_config_default(iters=700))
    b.pasur_cfr_iterate(P().pasur_config_default(iters=1000))
    assert (a.pasur_avg_strategy() == b.pasur_avg_strategy()).all()
    assert np.abs(a.pasur_round_utilities() - b.pasur_round_utilities()).max() < 1e-6


def test_cfr_dcfr_variant(ctx):
    deck = O.deal(5)
    pools = [mask_ids(deck[:4])]
    gt, ot = ctx.pasur_build_round(deck, 5, pools), O.Tree(deck, 5, pools)
    gt.unfold_single()
    ot.unfold_single()
    compare_cfr(gt, ot, ot.leaf_utilities_final(), 300, variant=1)


def test_two_round_chain_rounds_4_5(ctx):
    """Rounds 5-6 of the seed-0 deal (0-based rounds 4 and 5): round 5 over every root round 4
    reaches, 2000 iterations per round, round-5 utilities passed back into round 4.  Round 4 gets
    the same next-round utilities on both sides (the oracle's, rounded to float32), so that its
    comparison isolates the CFR arithmetic; round 5's utilities were compared just before."""
    T = 2000
    deck = O.deal(0)
    pool = mask_ids(deck[:4])
    g4, o4 = ctx.pasur_build_round(deck, 4, [pool]), O.Tree(deck, 4, [pool])
    g4.unfold_single()
    o4.unfold_single()
    gp, gs, gsc, gl = g4.pasur_next_roots()
    op, os_, osc, ol = o4.next_roots()
    assert gp.tolist() == op.tolist() and (gl == ol).all()
    g5, o5 = ctx.pasur_build_round(deck, 5, gp), O.Tree(deck, 5, op)
    unfold_both(g5, o5, gs, gsc)
    U5g, U5o, _, _ = compare_cfr(g5, o5, o5.leaf_utilities_final(), T)
    u5 = U5o.astype(np.float32)
    leaf4 = o4.leaf_utilities_linked(ol, u5.astype(np.float64))
    compare_cfr(g4, o4, leaf4, T, next_util=u5)
