"""Pins of the oracle's self-play: the counter-based generator against numpy's Philox bit
generator, the exact outcome distribution against the on-policy value of the round-by-round
chain, and the sampled games against both (sample mean within 4 standard errors, outcome
frequencies within 5 binomial standard errors)."""
import numpy as np
import pytest

import oracle as O


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


def _inc(c):
    c = list(c)
    for i in range(4):
        c[i] = (c[i] + 1) % 2**64
        if c[i]:
            break
    return c


@pytest.mark.parametrize("key,ctr", [((0, 0), (0, 0, 0, 0)), ((123456789, 987654321), (5, 6, 7, 8)),
                                     ((2**64 - 1, 2**64 - 1), (2**64 - 1,) * 4), ((7, 0), (41, 2**63, 0, 9))])
def test_philox_matches_numpy(key, ctr):
    # numpy's Philox (4x64, 10 rounds) advances its 256-bit counter before every block
    raw = np.random.Philox(key=list(key), counter=list(ctr)).random_raw(12)
    c, mine = list(ctr), []
    for _ in range(3):
        c = _inc(c)
        mine.append(O.philox4x64(c, key))
    assert (np.concatenate(mine) == raw).all()


def test_philox_published_zero_vector():
    # Philox4x64-10 of counter 0 under key 0 (the known-answer vector of the generator's authors)
    got = O.philox4x64((0, 0, 0, 0), (0, 0))
    assert [int(x) for x in got] == [0x16554D9ECA36314C, 0xDB20FE9D672D0FDC, 0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]


def chain_4_5(seed, T=200):
    deck = O.deal(seed)
    t4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
    t4.unfold_single()
    pools, soff, scores, lnk = t4.next_roots()
    t5 = O.Tree(deck, 5, pools)
    t5.unfold(soff, scores)
    leaf5 = t5.leaf_utilities_final()
    s5, U5 = t5.cfr(leaf5, T)
    leaf4 = t4.leaf_utilities_linked(lnk, U5)
    s4, _ = t4.cfr(leaf4, T)
    return t4, t5, lnk, s4, s5, leaf5


def on_policy_chain(t4, t5, lnk, s4, s5, leaf5):
    v5 = t5.root_values(leaf5, O.ON_POLICY, s5)
    return t4.root_values(t4.leaf_utilities_linked(lnk, v5), O.ON_POLICY, s4)


@pytest.mark.parametrize("seed", [0, 2])
def test_distribution_mean_is_on_policy_value(seed):
    t4, t5, lnk, s4, s5, leaf5 = chain_4_5(seed)
    p = O.outcome_distribution([t4, t5], [s4, s5], [lnk], 0)
    xs = np.arange(-128, 129)
    assert abs(p.sum() - 1.0) < 1e-12
    assert abs((xs * p).sum() - on_policy_chain(t4, t5, lnk, s4, s5, leaf5)[0]) < 1e-9


@pytest.mark.parametrize("seed", [0, 2])
def test_selfplay_matches_exact_distribution(seed):
    t4, t5, lnk, s4, s5, leaf5 = chain_4_5(seed)
    N = 40000
    out = O.selfplay([t4, t5], [s4.astype(np.float32), s5.astype(np.float32)], [lnk], 0, N, seed)
    p = O.outcome_distribution([t4, t5], [s4, s5], [lnk], 0)
    xs = np.arange(-128, 129)
    mean, var = (xs * p).sum(), (xs * xs * p).sum() - (xs * p).sum() ** 2
    assert abs(out.mean() - mean) <= 4 * np.sqrt(var / N) + 1e-9
    freq = np.bincount(out.astype(np.int64) + 128, minlength=257) / N
    assert (freq[p == 0] == 0).all()
    se = np.sqrt(p * (1 - p) / N)
    assert (np.abs(freq - p) <= 5 * se + 1e-12).all()
    # the games of a prefix do not depend on how many games are played (counter-based draws)
    assert (O.selfplay([t4, t5], [s4.astype(np.float32), s5.astype(np.float32)], [lnk], 0, 100, seed) == out[:100]).all()


def first_child_sigma(t):
    """Pure strategy: all weight on every parent's first child."""
    n, q = t.sizes()
    parts = []
    for k in range(1, 9):
        par = t.fgt_parents(k)
        first = np.zeros(len(par), np.float64)
        # children of FGT parent (g, s) are (c, s) for the GT children c: slot-interleaved, so the
        # first child is the first occurrence of the parent index
        first[np.unique(par, return_index=True)[1]] = 1.0
        parts.append(first)
    return np.concatenate(parts)


def test_pure_and_zero_strategies_give_one_game():
    t4, t5, lnk, _, _, leaf5 = chain_4_5(0, T=1)
    f4, f5 = first_child_sigma(t4), first_child_sigma(t5)
    p = O.outcome_distribution([t4, t5], [f4, f5], [lnk], 0)
    assert np.isclose(p.max(), 1.0)
    val = int(np.argmax(p)) - 128
    out = O.selfplay([t4, t5], [f4.astype(np.float32), f5.astype(np.float32)], [lnk], 0, 50, 11)
    assert (out == val).all()
    # all-zero strategies fall back to the first move everywhere: the same game
    z4, z5 = np.zeros_like(f4, np.float32), np.zeros_like(f5, np.float32)
    assert (O.selfplay([t4, t5], [z4, z5], [lnk], 0, 20, 3) == val).all()
    # and that game's value is the on-policy value of the pure profile
    assert abs(on_policy_chain(t4, t5, lnk, f4, f5, leaf5)[0] - val) < 1e-12


def test_inherited_difference_shifts_every_game():
    """A root with inherited difference D yields every game's difference shifted by D."""
    deck = O.deal(2)
    pool = mask_ids(deck[:4])
    ta = O.Tree(deck, 5, [pool])
    ta.unfold(np.array([0, 2], np.int64), np.array([[0, 0, 0, 0], [0, 0, 9, 0]], np.int16))
    sa, _ = ta.cfr(ta.leaf_utilities_final(), 100)
    s32 = sa.astype(np.float32)
    g0 = O.selfplay([ta], [s32], [], 0, 300, 5)
    g1 = O.selfplay([ta], [s32], [], 1, 300, 5)
    # slot 1 plays the same strategy values only if CFR gave both slots the same sigma (it does:
    # utilities do not depend on the inherited difference), so the games coincide up to the shift
    assert (g1 - g0 == 9).all()
