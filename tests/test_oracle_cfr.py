"""Pins of the oracle's CFR, minimax, best response and round linking (CPU only).

What fixes the values: the sequence-form LP value of the round (an independent method for the
game value), the T=1 closed form (uniform play), the regret identity sum_a sigma(a) r(a) = 0,
the O(1/sqrt(T)) convergence of CFR's average root utility to the game value and of the
average strategy's exploitability to zero (Thms. avst / rm), BR_Bob <= value <= BR_Alex, and a
direct backward induction across two rounds for the between-round links.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.optimize import linprog

import oracle as O


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


@pytest.fixture(scope="module", params=[2, 5])
def cfg1(request):
    """Final round of a seeded deal as a standalone round: pool = deck[0:4], score (0,0,0,0).
    (Seed 0's final round holds no point card, so all its leaves are 0; seeds 2 and 5 are not
    degenerate.)"""
    deck = O.deal(request.param)
    t = O.Tree(deck, 5, [mask_ids(deck[:4])])
    t.unfold_single()
    return deck, t, t.leaf_utilities_final()


def sequence_form_value(t: O.Tree, leaf) -> float:
    """Game value of a single-root round by the sequence-form LP (Koller-Megiddo-von Stengel),
    solved by HiGHS: max_{x,v} f.v s.t. F^T v <= A^T x, E x = e, x >= 0."""
    n, _ = t.sizes()
    levels = [t.level(k) for k in range(9)]
    seqA = [np.zeros(n[k], np.int64) for k in range(9)]
    seqB = [np.zeros(n[k], np.int64) for k in range(9)]
    nA, nB = 1, 1
    E_rows, F_rows = [], []  # (row, col, val)
    eA, eB = 1, 1  # constraint row counters (row 0: empty sequence = 1)
    E_rows.append((0, 0, 1.0))
    F_rows.append((0, 0, 1.0))
    for k in range(8):
        L = levels[k]
        off = np.concatenate([[0], np.cumsum(L.nchild)])
        for i in range(n[k]):
            kids = range(off[i], off[i + 1])
            if k % 2 == 0:
                E_rows.append((eA, seqA[k][i], -1.0))
                for c in kids:
                    seqA[k + 1][c] = nA
                    seqB[k + 1][c] = seqB[k][i]
                    E_rows.append((eA, nA, 1.0))
                    nA += 1
                eA += 1
            else:
                F_rows.append((eB, seqB[k][i], -1.0))
                for c in kids:
                    seqB[k + 1][c] = nB
                    seqA[k + 1][c] = seqA[k][i]
                    F_rows.append((eB, nB, 1.0))
                    nB += 1
                eB += 1
    r, c, v = zip(*E_rows)
    E = sp.csr_matrix((v, (r, c)), shape=(eA, nA))
    r, c, v = zip(*F_rows)
    F = sp.csr_matrix((v, (r, c)), shape=(eB, nB))
    A = sp.csr_matrix((leaf, (seqA[8], seqB[8])), shape=(nA, nB))
    # variables z = [x (nA), v (eB)]; maximise v_0  ->  minimise -v_0
    cost = np.zeros(nA + eB)
    cost[nA] = -1.0
    A_ub = sp.hstack([-A.T, F.T]).tocsr()
    A_eq = sp.hstack([E, sp.csr_matrix((eA, eB))]).tocsr()
    b_eq = np.zeros(eA)
    b_eq[0] = 1.0
    bounds = [(0, None)] * nA + [(None, None)] * eB
    res = linprog(cost, A_ub=A_ub, b_ub=np.zeros(nB), A_eq=A_eq, b_eq=b_eq, bounds=bounds, method="highs")
    assert res.status == 0
    return -res.fun


def test_seed0_final_round_is_degenerate():
    deck = O.deal(0)
    t = O.Tree(deck, 5, [mask_ids(deck[:4])])
    t.unfold_single()
    assert (t.leaf_utilities_final() == 0).all()


def test_minimax_equals_sequence_form_lp(cfg1):
    deck, t, leaf = cfg1
    mm = t.root_values(leaf, O.MINIMAX)[0]
    assert abs(sequence_form_value(t, leaf) - mm) < 1e-7
    # and equals direct backward induction over the same round
    assert mm == O.minimax_rounds(deck, 5, mask_ids(deck[:4]))


def test_cfr_t1_is_uniform_play(cfg1):
    _, t, leaf = cfg1
    sb, U, R, S = t.cfr(leaf, 1, want_rs=True)
    assert abs(U[0] - t.root_values(leaf, O.UNIFORM)[0]) < 1e-12
    # regret identity: with uniform sigma the instant regrets of every node sum to zero
    q = t.sizes()[1]
    base = 0
    for k in range(1, 9):
        par = t.fgt_parents(k)
        sums = np.bincount(par, weights=R[base:base + q[k]], minlength=int(q[k - 1]))
        scale = np.bincount(par, weights=np.abs(R[base:base + q[k]]), minlength=int(q[k - 1])) + 1.0
        assert (np.abs(sums) <= 1e-12 * scale).all()
        base += q[k]


def test_cfr_converges_to_game_value(cfg1):
    _, t, leaf = cfg1
    mm = t.root_values(leaf, O.MINIMAX)[0]
    gaps, expl = [], []
    for T in (10, 100, 1000):
        sb, U = t.cfr(leaf, T)
        br_a = t.root_values(leaf, O.BR_ALEX, sb)[0]
        br_b = t.root_values(leaf, O.BR_BOB, sb)[0]
        assert br_b - 1e-9 <= mm <= br_a + 1e-9
        gaps.append(abs(U[0] - mm))
        expl.append((br_a - br_b) / 2)
        bound = 2.0 * np.abs(leaf).max() * np.sqrt(40.0) / np.sqrt(T)  # O(1/sqrt T) with a loose constant
        assert gaps[-1] <= bound
    assert expl[0] > 0 and expl[2] < expl[0] and expl[2] < 0.05
    assert gaps[0] > 0 and gaps[2] < 0.05


def test_sigma_bar_normalised_and_single_action_nodes(cfg1):
    _, t, leaf = cfg1
    sb, U, R, S = t.cfr(leaf, 50, want_rs=True)
    q = t.sizes()[1]
    base = 0
    for k in range(1, 9):
        par = t.fgt_parents(k)
        sums = np.bincount(par, weights=sb[base:base + q[k]], minlength=int(q[k - 1]))
        assert np.allclose(sums, 1.0, atol=1e-12)
        deg = np.bincount(par, minlength=int(q[k - 1]))[par]
        single = deg == 1
        assert (R[base:base + q[k]][single] == 0).all()
        assert (sb[base:base + q[k]][single] == 1.0).all()
        base += q[k]


def test_delta_does_not_enter_utilities():
    # eq. final_util: only the bonus column enters; roots differing only in Delta get equal values
    deck = O.deal(3)
    t = O.Tree(deck, 5, [mask_ids(deck[:4])])
    t.unfold(np.array([0, 3]), np.array([[1, 2, 0, 0], [1, 2, 9, 0], [1, 2, -4, 0]], np.int16))
    leaf = t.leaf_utilities_final()
    sb, U = t.cfr(leaf, 30)
    assert U[0] == U[1] == U[2]
    q = t.sizes()[1]
    base = 0
    for k in range(1, 9):
        x = sb[base:base + q[k]].reshape(-1, 3)
        assert (x[:, 0] == x[:, 1]).all() and (x[:, 0] == x[:, 2]).all()
        base += q[k]


def test_two_round_chain_matches_direct_backward_induction():
    """Round 4 -> 5 of the seed-0 deal: minimax of round 5 at every linked root, passed up through
    the links (eq. passuputil), equals direct backward induction over both rounds."""
    deck = O.deal(0)
    pool = mask_ids(deck[:4])
    t4 = O.Tree(deck, 4, [pool])
    t4.unfold_single()
    pools, soff, scores, lnk = t4.next_roots()
    # roots sorted by (pool, score), unique
    keys = [(int(pools[g]),) + tuple(int(x) for x in scores[s]) for g in range(len(pools))
            for s in range(soff[g], soff[g + 1])]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # every normalised score: clubs are reset once a bonus is held, and stay below 7 otherwise
    assert all((s[3] != 0 and s[0] == 0 and s[1] == 0) or (s[3] == 0 and s[0] < 7 and s[1] < 7) for s in scores)
    t5 = O.Tree(deck, 5, pools)
    t5.unfold(soff, scores)
    mm5 = t5.root_values(t5.leaf_utilities_final(), O.MINIMAX)
    leaf4 = t4.leaf_utilities_linked(lnk, mm5)
    mm4 = t4.root_values(leaf4, O.MINIMAX)[0]
    assert mm4 == O.minimax_rounds(deck, 4, pool)
    # the leaf's linked root holds the leaf's pool
    leaves = t4.level(8)
    root_pool = np.repeat(pools, np.diff(soff))
    assert (root_pool[lnk] == leaves.state[:, 2]).all()


def test_dcfr_variant_converges(cfg1):
    _, t, leaf = cfg1
    mm = t.root_values(leaf, O.MINIMAX)[0]
    sb, U = t.cfr(leaf, 200, variant=1)
    br_a = t.root_values(leaf, O.BR_ALEX, sb)[0]
    br_b = t.root_values(leaf, O.BR_BOB, sb)[0]
    assert br_b - 1e-9 <= mm <= br_a + 1e-9
    assert (br_a - br_b) / 2 < 0.05


def test_node_values_agree_with_root_values(cfg1):
    """or_node_values keeps the value of every FGT node of the same recursion as or_root_values:
    its level 0 is the root values (pinned above by the LP for mode 0), a leaf is its utility,
    and each internal node is the max (Alex) / min (Bob) or sigma-mean of its children."""
    _, t, leaf = cfg1
    sb, _ = t.cfr(leaf, 50)
    q = t.sizes()[1]
    for mode in (O.MINIMAX, O.BR_ALEX, O.BR_BOB, O.ON_POLICY):
        nv = t.node_values(leaf, mode, sb)
        assert np.array_equal(nv[0], t.root_values(leaf, mode, sb))
        assert np.array_equal(nv[8], leaf)
        base = 0
        for k in range(1, 9):
            par = t.fgt_parents(k)
            sig = sb[base:base + q[k]]
            ev = np.bincount(par, weights=sig * nv[k], minlength=int(q[k - 1]))
            mx = np.full(int(q[k - 1]), -np.inf)
            mn = np.full(int(q[k - 1]), np.inf)
            np.maximum.at(mx, par, nv[k])
            np.minimum.at(mn, par, nv[k])
            alex = (k - 1) % 2 == 0
            want = {O.MINIMAX: mx if alex else mn, O.BR_ALEX: mx if alex else ev, O.BR_BOB: ev if alex else mn,
                    O.ON_POLICY: ev}[mode]
            assert np.allclose(nv[k - 1], want, rtol=0, atol=1e-12)
            base += q[k]
