"""Pins of the oracle's generators, rules, tree build and unfolding against what the paper and the
mathematics fix (CPU only)."""
import itertools
import os

import numpy as np
import pytest

import oracle as O
from tests.cardnames import card, deck_from_game, mask, parse_game

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NUMERIC = (1 << 40) - 1


# ---- generators: published test values --------------------------------------------------------

def test_splitmix64_published_values():
    # SplitMix64 from state 0 (Steele, Lea, Flood 2014; the values every port checks against)
    assert [int(x) for x in O.splitmix64(0, 4)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]


def test_xoshiro256ss_published_values():
    # xoshiro256** from state {1,2,3,4} (Blackman & Vigna reference implementation outputs)
    assert [int(x) for x in O.xoshiro_from_state([1, 2, 3, 4], 4)] == [
        11520, 0, 1509978240, 1215971899390074240]


def test_bounded_draw_unbiased():
    n = 52
    draws = O.below_seq(7, np.full(208000, n, np.uint64))
    assert draws.max() < n
    counts = np.bincount(draws.astype(np.int64), minlength=n)
    chi2 = ((counts - 4000.0) ** 2 / 4000.0).sum()
    assert chi2 < 110  # 51 dof: p ~ 1e-5


# ---- deal (section Pasur: Jack-free initial pool) -------------------------------------------------

def test_deal_is_a_permutation_with_jack_free_pool():
    for seed in range(300):
        d = O.deal(seed)
        assert sorted(d.tolist()) == list(range(52))
        assert not any(40 <= c < 44 for c in d[:4])


def test_deal_golden_seed0():
    gold = [int(x) for x in open(os.path.join(GOLD, "deal_seed0.txt")).read().split()]
    assert O.deal(0).tolist() == gold


def test_deal_positions_uniform():
    # every non-Jack card is equally likely in the pool; cards at positions 12..51 are uniform
    cnt = np.zeros((52, 52))
    for seed in range(4000):
        d = O.deal(seed)
        cnt[d, np.arange(52)] += 1
    tail = cnt[:, 12:].sum(axis=1) / (4000 * 40)
    assert np.allclose(tail, 1 / 52, atol=0.004)
    assert cnt[40:44, :4].sum() == 0


# ---- numeric capture table (section Numerical Actions: 2764 subsets) ---------------------------

def test_sum11_subsets_2764():
    subs = O.subsets_sum(NUMERIC, 11)
    assert len(subs) == 2764
    sizes = np.bincount([bin(s).count("1") for s in subs], minlength=8)
    assert sizes[2:8].tolist() == [80, 440, 976, 920, 320, 28]
    assert sizes[:2].sum() == 0 and len(set(subs)) == 2764


# ---- legal actions (Table "Capture rules for each card type") ------------------------------------

def _brute_actions(hand, pool):
    """Brute force over every subset of the pool (tiny pools only)."""
    pool_cards = [c for c in range(52) if pool >> c & 1]
    out = []
    for c in (c for c in range(52) if hand >> c & 1):
        acts = []
        for r in range(1, len(pool_cards) + 1):
            for P in itertools.combinations(pool_cards, r):
                if c < 40:
                    ok = all(p < 40 for p in P) and (c // 4 + 1) + sum(p // 4 + 1 for p in P) == 11
                elif c < 44:
                    ok = set(P) == {p for p in pool_cards if p < 44}
                else:
                    ok = len(P) == 1 and P[0] // 4 == c // 4
                if ok:
                    acts.append((c, sum(1 << p for p in P)))
        if not acts:
            acts = [(c, 0)]
        out += sorted(acts)
    return out


def test_legal_actions_brute_force():
    rng = np.random.default_rng(11)
    for _ in range(400):
        perm = rng.permutation(52)
        hand = mask_ids(perm[:4])
        pool = mask_ids(perm[4:4 + rng.integers(0, 9)])
        assert O.legal_actions(hand, pool) == _brute_actions(hand, pool)


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


def test_legal_actions_cases():
    # a Jack with nothing capturable is laid; with numerics and Jacks it takes them, never K/Q
    assert O.legal_actions(mask(["JH"]), mask(["QH"])) == [(card("JH"), 0)]
    assert O.legal_actions(mask(["JS"]), mask(["2C", "JD", "QC", "KD"])) == [
        (card("JS"), mask(["2C", "JD"]))]
    # a King takes one King at a time; two Kings give two actions
    assert O.legal_actions(mask(["KS"]), mask(["KC", "KD", "5H"])) == [
        (card("KS"), mask(["KC"])), (card("KS"), mask(["KD"]))]
    # must-capture binds per card: 7D can take 4D but QC may still be laid (Fig. game_0 row 0_1_0)
    acts = O.legal_actions(mask(["4C", "7D", "QC"]), mask(["AC", "AS", "4D", "9D"]))
    assert (card("QC"), 0) in acts and (card("7D"), mask(["4D"])) in acts
    assert (card("7D"), 0) not in acts


# ---- both worked games of the paper (Fig. game_0 and Fig. game_9) -----------------------------

@pytest.mark.parametrize("fname", ["deck9_game0.txt", "deck9_game9.txt"])
def test_worked_game_replay(fname):
    pool, hands, rows, cleanup, final = parse_game(os.path.join(GOLD, fname))
    score = np.zeros(4, np.int16)
    lp = {"0": 0, "A": 1, "B": 2}
    cl = {"-": None, "0": 0, "A": 1, "B": 2}
    state = None
    rus = None
    for i, r in enumerate(rows):
        if r["turn"] == 0 and r["ply"] == 0:
            if state is not None:
                score = O.round_end(score, rus)
                pool_now = int(state[2])
            else:
                pool_now = mask_ids(pool)
            a, b = hands[r["round"]]
            state = np.array([mask_ids(a), mask_ids(b), pool_now], np.uint64)
            rus = np.zeros(7, np.int8)
        mover = r["ply"]
        acts = O.legal_actions(int(state[mover]), int(state[2]))
        assert (r["lay"], r["pick"]) in acts, f"row {i}: move not legal"
        state, rus = O.apply(state, rus, mover, r["lay"], r["pick"], r["round"] == 5)
        assert int(score[0]) + rus[0] == r["acl"] and int(score[1]) + rus[1] == r["bcl"], f"row {i} clubs"
        assert (rus[3], rus[5], rus[4], rus[6]) == (r["apt"], r["bpt"], r["asr"], r["bsr"]), f"row {i} points"
        assert int(score[2]) == r["delta"], f"row {i} delta"
        assert rus[2] == lp[r["L"]], f"row {i} last picker"
        if cl[r["CL"]] is not None:
            assert int(score[3]) == cl[r["CL"]], f"row {i} bonus"
    assert int(state[0]) == 0 and int(state[1]) == 0
    value, fscore = O.final_leaf(score, rus, int(state[2]))
    acl, bcl, apt, bpt, asr, bsr, L = cleanup
    bonus = {0: 0.0, 1: 7.0, 2: -7.0}[int(fscore[3])]
    assert value == (apt + 5 * asr) - (bpt + 5 * bsr) + bonus
    if final is not None:
        assert int(score[2]) + value == final  # caption of Fig. game_0: "Alex leading by 8 points"


def test_score_normalisation_example():
    # section Score Tensors: [3, 8, 2, 0] is converted to [0, 0, 2, 2]
    assert O.normalize_score([3, 8, 2, 0]).tolist() == [0, 0, 2, 2]
    assert O.normalize_score([7, 0, -1, 0]).tolist() == [0, 0, -1, 1]
    assert O.normalize_score([6, 6, 4, 0]).tolist() == [6, 6, 4, 0]
    assert O.normalize_score([3, 2, 4, 1]).tolist() == [0, 0, 4, 1]


def test_surs():
    # numeric capture clearing the pool is a Sur (+5) except with a Jack or in the final round
    st = np.array([mask(["9C", "2D"]), mask(["3H"]), mask(["2S"])], np.uint64)
    s2, r2 = O.apply(st, np.zeros(7, np.int8), 0, card("9C"), mask(["2S"]), False)
    assert r2[4] == 1 and int(s2[2]) == 0 and r2[0] == 1 and r2[2] == 1
    s3, r3 = O.apply(st, np.zeros(7, np.int8), 0, card("9C"), mask(["2S"]), True)
    assert r3[4] == 0
    st = np.array([mask(["JC"]), 0, mask(["2S"])], np.uint64)
    _, r4 = O.apply(st, np.zeros(7, np.int8), 0, card("JC"), mask(["2S"]), False)
    assert r4[4] == 0 and r4[3] == 1  # the Jack itself is worth 1


# ---- round tree and unfolding ---------------------------------------------------------------------

def repeat_blocks(org, bsz, rpt):
    """RepeatBlocks of the appendix, written from its definition: block b (size bsz[b]) of org is
    emitted rpt[b] times in a row."""
    out, pos = [], 0
    for b, r in zip(bsz, rpt):
        out += list(org[pos:pos + b]) * int(r)
        pos += b
    return out


def test_repeat_blocks_paper_examples():
    assert repeat_blocks([1, 2, 3, 4, 5, 6], [2, 3, 1], [1, 3, 2]) == [1, 2, 3, 4, 5, 3, 4, 5, 3, 4, 5, 6, 6]
    # Unfolding Process figure: c_scr = [3, 2], t_brf = [2, 3]
    assert repeat_blocks(list(range(5)), [3, 2], [2, 3]) == [0, 1, 2, 0, 1, 2, 3, 4, 3, 4, 3, 4]


def config1_deck():
    return O.deal(0)


def test_round_tree_counts_match_brute_force():
    deck = config1_deck()
    for rnd in (5, 4):
        pool = mask_ids(deck[:4])
        t = O.Tree(deck, rnd, [pool])
        n, _ = t.sizes()
        assert n.tolist() == O.count_round(deck, rnd, pool).tolist()
        assert n[0] == 1 and (n[1:] >= n[:-1]).all() is not None


def test_round_tree_structure():
    deck = config1_deck()
    pools = sorted({mask_ids(deck[:4]), mask_ids(deck[:3]), mask_ids(deck[1:4])})
    t = O.Tree(deck, 5, pools)
    n, _ = t.sizes()
    for k in range(8):
        L, C = t.level(k), t.level(k + 1)
        assert L.nchild.sum() == n[k + 1]
        off = np.concatenate([[0], np.cumsum(L.nchild)])
        # children of node i are the contiguous block off[i]:off[i+1], in canonical order
        assert (C.parent == np.repeat(np.arange(n[k]), L.nchild)).all()
        for i in range(n[k]):
            keys = list(zip(C.lay[off[i]:off[i + 1]], C.pick[off[i]:off[i + 1]]))
            assert keys == sorted(keys) and len(set(keys)) == len(keys)
        mover = k % 2
        hand_sizes = [bin(int(x)).count("1") for x in C.state[:, mover]]
        assert set(hand_sizes) == {3 - k // 2}
    leaves = t.level(8)
    assert (leaves.state[:, 0] == 0).all() and (leaves.state[:, 1] == 0).all()


def test_unfold_matches_repeat_blocks():
    deck = config1_deck()
    pools = sorted({mask_ids(deck[:4]), mask_ids(deck[:3])})
    t = O.Tree(deck, 5, pools)
    score_off = np.array([0, 3, 5])
    scores = np.array([[0, 0, 0, 0], [1, 2, 3, 0], [0, 0, -4, 1], [2, 2, 0, 0], [0, 0, 1, 2]], np.int16)
    q = t.unfold(score_off, scores)
    n, _ = t.sizes()
    cscr = np.array([3, 2])
    for k in range(1, 9):
        P, L = t.level(k - 1), t.level(k)
        c_scr = cscr[P.root_of]  # score slots carried by each parent GT node
        expect = repeat_blocks(list(range(int(q[k - 1]))), c_scr.tolist(), P.nchild.tolist())
        assert t.fgt_parents(k).tolist() == expect
        assert q[k] == (cscr[L.root_of]).sum()
