"""Closed-form pins of the oracle's CFR updates after T = 1, 2 and 3 iterations (CPU only).

The convergence pins of the oracle (minimax, best response, exploitability -> 0) would still pass
with a wrongly weighted average strategy or a wrongly indexed DCFR discount, since those still
converge.  Here the regrets R and strategy sums S of every edge are fixed by hand.

The game.  A real round tree (the standalone final round of a seeded deal, one root, one score
slot) with leaf values chosen so that only the first two plies matter: every leaf below the
first child (b = 0) of Bob's node under Alex's first root move (a = 0) is worth V, every other
leaf 0.  Let n = the root's number of moves and m = the number of moves of Bob's node under
a = 0 (both >= 2).  Every node from level 2 down has children of equal value, so its value is
exactly that of its first child (the pivoted value of the section "CFR Algorithm"), its instant
regrets are exactly 0 for ever and it plays uniformly.  The dead zone is tau = 0.

Vanilla CFR (eq. RM, eq. avsigma; R(h,a) += s_p pi_{-p}(h) (v(h.a) - v(h)),
S(h,a) += pi_p(h) sigma(h,a)):

  t = 1, sigma uniform.  Bob's node a=0 sees (V, 0, ..., 0): v = V/m; Bob's other nodes: 0;
    the root sees (V/m, 0, ...): v = V/(mn).
    root:      r = V(n-1)/(mn) (a=0), -V/(mn) (a>=1);      S += 1 * 1/n
    Bob a=0:   pi_Alex = 1/n, s = -1:  r = -(1/n)(V - V/m) = -V(m-1)/(mn) (b=0),
               +(1/n)(V/m) = V/(mn) (b>=1);                 S += pi_Bob = 1 times 1/m
    Bob a>=1:  r = 0;                                       S += 1/d
  t = 2 and 3.  Regret matching: the root plays a = 0 (its only positive regret), Bob's node
    a=0 plays b >= 1 uniformly (1/(m-1) each), other nodes uniform.  Then Bob's node a=0 is
    worth V - (m-1) V/(m-1) = 0 and so is the root.
    root:      r = 0;                                        S += (1, 0, ..., 0)
    Bob a=0:   pi_Alex = 1: r = -V (b=0), 0 (b>=1);         S += (0, 1/(m-1), ...)
    Bob a>=1:  pi_Alex = 0: r = 0;                          S += 1/d
    (the signs of the regrets do not change, so t = 3 repeats t = 2)
  U(root) = (V/(mn) + 0 + ...)/T.
  Deeper node h (level k >= 2) with ancestors a, b: sigma is uniform below level 1, so
    pi_p^t(h) = u_p(h) * (sigma_root^t(a) if p = Alex else sigma_Bob^t(b|a)), where u_p(h) is the
    product of 1/d over the uniform moves of player p on the path from level 2; R(h,.) = 0 and
    S(h,.) = u_p(h) * sum_t (that sigma) / d(h).

DCFR with alpha = 1.5, beta = 0, gamma = 2 (eqs. DFCR_REG / DFCR_AVG: R^t = R^{t-1} d^{t-1} +
r^t with d^{t'} = t'^a/(t'^a+1) where R^{t-1} > 0, t'^b/(t'^b+1) otherwise, t' = t-1;
S^t = (1-1/t)^g S^{t-1} + pi sigma).  The instant regrets and sigma^t are those above (the signs
never change).  With p = 1/2 (t'=1, either sign; beta = 0 gives 1/2 at every t') and
q = 2^1.5/(2^1.5+1) (t'=2, positive):
  t = 1: as vanilla (R^0 = 0, S factor (1-1)^2 = 0).
  t = 2: root R = (V(n-1)/(2mn), -V/(2mn));  S = (1/(4n) + 1, 1/(4n)).
         Bob a=0: R = (-V(m-1)/(2mn) - V, V/(2mn));  S = (1/(4m), 1/(4m) + 1/(m-1)).
         Bob a>=1: S = 1/(4d) + 1/d.
  t = 3: root R = (V(n-1) q/(2mn), -V/(4mn));  S = ((1/(4n) + 1) 4/9 + 1, 1/(9n)).
         Bob a=0: R = ((-V(m-1)/(2mn) - V)/2 - V, V q/(2mn));
                  S = (1/(9m), (1/(4m) + 1/(m-1)) 4/9 + 1/(m-1)).
         Bob a>=1: S = (1/(4d) + 1/d) 4/9 + 1/d.
  Deeper nodes: S(h,.) = u_p(h)/d(h) * (discounted sum of that sigma): T=2: s1/4 + s2;
  T=3: s1/9 + 4 s2/9 + s3.
"""
import math

import numpy as np
import pytest

import oracle as O

V = 4.0


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


@pytest.fixture(scope="module", params=[5, 2])
def game(request):
    """(tree, leaf values, structure) of the two-ply game embedded in a final round: seed 5 has
    n = m = 4 (exact binary fractions), seed 2 has n = 5, m = 4."""
    deck = O.deal(request.param)
    t = O.Tree(deck, 5, [mask_ids(deck[:4])])
    t.unfold_single()
    n_gt, q = t.sizes()
    assert (n_gt == q).all()  # one root, one slot: FGT index = GT index
    lv = [t.level(k) for k in range(9)]
    # ancestors at levels 1 and 2 of every node, and the child index of each node in its parent
    anc1 = [None, np.arange(n_gt[1])]
    anc2 = [None, None, np.arange(n_gt[2])]
    for k in range(2, 9):
        anc1.append(anc1[k - 1][lv[k].parent])
        if k >= 3:
            anc2.append(anc2[k - 1][lv[k].parent])
    first_child = [np.concatenate([[0], np.cumsum(lv[k].nchild)])[:-1] for k in range(8)]
    rank = [None] + [np.arange(n_gt[k]) - first_child[k - 1][lv[k].parent] for k in range(1, 9)]
    b_of2 = rank[2]                   # index b of a level-2 node among its parent's moves
    a_of2 = lv[2].parent              # its level-1 parent a
    n = int(lv[0].nchild[0])
    m = int(lv[1].nchild[0])
    assert n >= 2 and m >= 2
    leaf = np.where((anc1[8] == 0) & (b_of2[anc2[8]] == 0), V, 0.0)
    base = np.concatenate([[0], np.cumsum(q[1:])])  # edge offset of level k at base[k - 1]
    return dict(t=t, leaf=leaf, lv=lv, n=n, m=m, q=q, base=base, anc1=anc1, anc2=anc2, a_of2=a_of2, b_of2=b_of2)


def edges(g, k):
    """Slice of the concatenated edge arrays holding level k (k = 1..8)."""
    return slice(int(g["base"][k - 1]), int(g["base"][k]))


def top_sums(g, T, variant):
    """Per-iteration sigma of the two decisive nodes, folded with the discount weights of the
    strategy sum: returns (root weight per a, Bob weight per (a, b) at level 2)."""
    n, m = g["n"], g["m"]
    w = [1.0] * T if variant == 0 else {1: [1.0], 2: [0.25, 1.0], 3: [1 / 9, 4 / 9, 1.0]}[T]
    a1 = np.arange(n)
    root = sum(wt * np.where(a1 == 0, 1.0 / n if t == 0 else 1.0, 1.0 / n if t == 0 else 0.0)
               for t, wt in enumerate(w))
    a2, b2 = g["a_of2"], g["b_of2"]
    d1 = g["lv"][1].nchild[a2].astype(np.float64)
    bob = np.zeros(len(a2))
    for t, wt in enumerate(w):
        if t == 0:
            s = 1.0 / d1
        else:
            s = np.where(a2 == 0, np.where(b2 == 0, 0.0, 1.0 / (m - 1)), 1.0 / d1)
        bob += wt * s
    return root, bob


def expected(g, T, variant):
    """Hand-derived R and S of every edge after T iterations (see the module docstring)."""
    n, m, lv = g["n"], g["m"], g["lv"]
    ne = int(g["q"][1:].sum())
    R = np.zeros(ne)
    S = np.zeros(ne)
    a = np.arange(n)
    a2, b2 = g["a_of2"], g["b_of2"]
    if variant == 0:
        ra = (V * (n - 1) / (m * n), -V / (m * n))
        rb = (-V * (m - 1) / (m * n) - (T - 1) * V, V / (m * n))
    else:
        qf = 2 ** 1.5 / (2 ** 1.5 + 1)
        if T == 1:
            ra = (V * (n - 1) / (m * n), -V / (m * n))
            rb = (-V * (m - 1) / (m * n), V / (m * n))
        elif T == 2:
            ra = (V * (n - 1) / (2 * m * n), -V / (2 * m * n))
            rb = (-V * (m - 1) / (2 * m * n) - V, V / (2 * m * n))
        else:
            ra = (V * (n - 1) * qf / (2 * m * n), -V / (4 * m * n))
            rb = ((-V * (m - 1) / (2 * m * n) - V) / 2 - V, V * qf / (2 * m * n))
    R[edges(g, 1)] = np.where(a == 0, ra[0], ra[1])
    R[edges(g, 2)] = np.where(a2 == 0, np.where(b2 == 0, rb[0], rb[1]), 0.0)
    root_w, bob_w = top_sums(g, T, variant)
    S[edges(g, 1)] = root_w
    S[edges(g, 2)] = bob_w
    # deeper edges, out of a level-(k-1) node h: R = 0 and S = u_p(h) * (the weighted sigma of
    # the decisive node of h's mover above h) / d(h)
    u = own_reach_products(g)
    for k in range(3, 9):
        par = lv[k].parent
        d = lv[k - 1].nchild[par].astype(np.float64)
        alex = (k - 1) % 2 == 0
        top = root_w[g["anc1"][k - 1][par]] if alex else bob_w[g["anc2"][k - 1][par]]
        S[edges(g, k)] = u[k - 1][par] * top / d
    return R, S


def own_reach_products(g):
    """u_p(h) for every node h of levels 2..7: the product of 1/d over the moves of h's mover
    on the path from level 2 (the moves below the decisive plies are uniform)."""
    lv = g["lv"]
    out = {2: np.ones(len(lv[2].parent)), 3: np.ones(len(lv[3].parent))}
    for k in range(4, 8):
        gp = lv[k - 1].parent[lv[k].parent]  # the level k-2 ancestor, moved by the same player
        out[k] = out[k - 2][gp] / lv[k - 2].nchild[gp].astype(np.float64)
    return out


@pytest.mark.parametrize("T", [1, 2, 3])
@pytest.mark.parametrize("tau", [0.0, 1e-6])
def test_vanilla_regrets_and_strategy_sums(game, T, tau):
    g = game
    sb, U, R, S = g["t"].cfr(g["leaf"], T, tau=tau, want_rs=True)
    R_x, S_x = expected(g, T, 0)
    assert np.abs(R - R_x).max() <= 1e-12
    assert np.abs(S - S_x).max() <= 1e-12
    assert abs(U[0] - V / (g["m"] * g["n"]) / T) <= 1e-13
    # the average strategy of the root's moves is the normalised strategy sum
    n = g["n"]
    sroot = np.where(np.arange(n) == 0, 1.0 / n + (T - 1), 1.0 / n) / T
    assert np.abs(sb[edges(g, 1)] - sroot).max() <= 1e-12


@pytest.mark.parametrize("T", [1, 2, 3])
def test_dcfr_regrets_and_strategy_sums(game, T):
    g = game
    sb, U, R, S = g["t"].cfr(g["leaf"], T, tau=0.0, variant=1, alpha=1.5, beta=0.0, gamma=2.0, want_rs=True)
    R_x, S_x = expected(g, T, 1)
    assert np.abs(R - R_x).max() <= 1e-12
    assert np.abs(S - S_x).max() <= 1e-12
    # the root utility is the plain mean of v(root) over the iterations in both variants
    assert abs(U[0] - V / (g["m"] * g["n"]) / T) <= 1e-13


def test_dcfr_discount_values():
    """The two discounts the DCFR pins rely on, from eq. DFCR_REG / DFCR_AVG directly."""
    assert math.isclose(2 ** 1.5 / (2 ** 1.5 + 1), 2 * math.sqrt(2) / (2 * math.sqrt(2) + 1))
    assert (1 - 1 / 2) ** 2 == 0.25 and math.isclose((1 - 1 / 3) ** 2, 4 / 9)


@pytest.mark.parametrize("seed", [2, 5])
def test_dead_zone_effect_on_final_rounds(seed):
    """The regret-matching dead zone (tau = 1e-6 of t * Umax) against the exact positive part
    (tau = 0) on standalone final rounds at T = 1000: the root utility and the exploitability of
    the average strategy are unchanged; only edges at exact ties move (seed 2: one node's
    sigma-bar by 1.2e-2, both sides optimal)."""
    deck = O.deal(seed)
    t = O.Tree(deck, 5, [mask_ids(deck[:4])])
    t.unfold_single()
    leaf = t.leaf_utilities_final()
    s1, u1 = t.cfr(leaf, 1000, tau=1e-6)
    s0, u0 = t.cfr(leaf, 1000, tau=0.0)

    def expl(s):
        return (t.root_values(leaf, O.BR_ALEX, s)[0] - t.root_values(leaf, O.BR_BOB, s)[0]) / 2

    print(f"seed {seed}: |dU| {abs(u1 - u0).max():.3e}, max |d sigma-bar| {abs(s1 - s0).max():.3e}, "
          f"exploitability {expl(s1):.6f} (tau 1e-6) vs {expl(s0):.6f} (tau 0)")
    assert abs(u1 - u0).max() <= 1e-12
    assert abs(expl(s1) - expl(s0)) <= 1e-12
    assert abs(s1 - s0).max() <= 0.02
