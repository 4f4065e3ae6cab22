"""Full six-round game of the seed-0 deal at full size, in the launch configuration bench.py times
(T = 1000 per round, default solver settings), checked against the fp64 oracle:

  - every round's GT and FGT level sizes, next roots and links: bit-exact (the oracle builds the
    whole game itself);
  - the final round's CFR on a seeded sample of FGT roots (the oracle solves only those roots,
    with its own leaf values): U within 1e-5, average strategies per the parity policy;
  - every earlier round's CFR on a seeded sample of FGT roots with a seeded synthetic
    next-round utility vector fed to both sides (no oracle input comes from the GPU).
"""
import numpy as np
import pytest

import oracle as O
from tests.test_gpu_parity import check_sigma, check_utilities, mask_ids, oracle_sensitivity, own_mass

pytestmark = pytest.mark.gpu

SEED, T, SAMPLE = 0, 1000, 12


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


def fgt_index(ot, soff):
    """per level: root_of and FGT offset of every GT node of the oracle tree."""
    n, _ = ot.sizes()
    out = []
    for k in range(9):
        lv = ot.level(k)
        slots = (soff[lv.root_of + 1] - soff[lv.root_of]).astype(np.int64)
        off = np.concatenate([[0], np.cumsum(slots)])
        out.append((lv.root_of, off))
    return out


def sampled_edges(idx, picks):
    """GPU FGT indices (levels 1..8 concatenated) of the sub-round made of the picked
    (root, slot) pairs, in the order of an oracle tree built from just those pairs."""
    by_root = {}
    for g, s in picks:
        by_root.setdefault(g, []).append(s)
    roots = sorted(by_root)
    parts = []
    base = 0
    sizes = [len(idx[k][0]) for k in range(9)]
    for k in range(1, 9):
        root_of, off = idx[k]
        lvl = []
        for g in roots:
            js = np.nonzero(root_of == g)[0]
            ss = np.array(sorted(by_root[g]), np.int64)
            lvl.append((off[js][:, None] + ss[None, :]).reshape(-1))
        parts.append(base + np.concatenate(lvl))
        base += int(off[-1])
    return roots, {g: sorted(v) for g, v in by_root.items()}, np.concatenate(parts)


def sub_tree(deck, rnd, pools, soff, scores, roots, slots):
    sp = [int(pools[g]) for g in roots]
    so, sc = [0], []
    for g in roots:
        for s in slots[g]:
            sc.append(scores[soff[g] + s])
        so.append(len(sc))
    t = O.Tree(deck, rnd, sp)
    t.unfold(np.array(so), np.array(sc, np.int16))
    return t


def test_full_game_seed0(ctx):
    deck = O.deal(SEED)
    rng = np.random.default_rng(7)
    cfg = P().pasur_config_default(iters=T)
    pools, soff, scores = np.array([mask_ids(deck[:4])], np.uint64), np.array([0, 1]), np.zeros((1, 4), np.int16)
    rounds = []
    for r in range(6):
        gt = ctx.pasur_build_round(deck, r, pools)
        gq = gt.pasur_unfold(soff, scores)
        ot = O.Tree(deck, r, pools)
        oq = ot.unfold(soff, scores)
        assert gt.pasur_tree_sizes()[0].tolist() == ot.sizes()[0].tolist()
        assert gq.tolist() == oq.tolist()
        rounds.append(dict(gt=gt, ot=ot, pools=pools, soff=np.asarray(soff), scores=np.asarray(scores)))
        if r < 5:
            gp, gs, gsc, gl = gt.pasur_next_roots()
            op, os_, osc, ol = ot.next_roots()
            assert gp.tolist() == op.tolist() and gs.tolist() == os_.tolist()
            assert (gsc == osc).all() and (gl == ol).all()
            rounds[-1]["next"] = (op, os_, osc, ol)
            pools, soff, scores = op, os_, osc
    # the whole backward solve on the GPU, as the benchmark runs it
    nxt = None
    for r in range(5, -1, -1):
        g = rounds[r]["gt"]
        g.pasur_cfr_iterate(cfg, nxt)
        rounds[r]["U"] = g.pasur_round_utilities()
        rounds[r]["sb"] = g.pasur_avg_strategy()
        nxt = rounds[r]["U"]
        assert np.isfinite(rounds[r]["U"]).all()
    # sampled checks, round by round
    for r in range(6):
        R = rounds[r]
        ot, pools, soff, scores = R["ot"], R["pools"], R["soff"], R["scores"]
        n_fgt_roots = int(soff[-1])
        flat = rng.choice(n_fgt_roots, size=min(SAMPLE, n_fgt_roots), replace=False)
        root_of_slot = np.repeat(np.arange(len(pools)), np.diff(soff))
        picks = [(int(root_of_slot[f]), int(f - soff[root_of_slot[f]])) for f in flat]
        idx = fgt_index(ot, soff)
        roots, slots, edges = sampled_edges(idx, picks)
        sub = sub_tree(deck, r, pools, soff, scores, roots, slots)
        if r == 5:
            leaf = sub.leaf_utilities_final()
            U_g, sb_g = R["U"], R["sb"]
        else:
            # seeded synthetic next-round utilities, exactly representable in float32
            op, os_, osc, ol = R["next"]
            n_next = len(osc)
            u_syn = (np.round(rng.normal(0.0, 6.0, n_next) * 256) / 256).astype(np.float32)
            g2 = ctx.pasur_build_round(deck, r, pools)
            g2.pasur_unfold(soff, scores)
            g2.pasur_next_roots()
            g2.pasur_cfr_iterate(cfg, u_syn)
            U_g, sb_g = g2.pasur_round_utilities(), g2.pasur_avg_strategy()
            # leaf values of the whole round (eq. passuputil): exact, since d + u is a float32
            leaf_full = ot.leaf_utilities_linked(ol, u_syn.astype(np.float64))
            assert (g2.pasur_leaf_values() == leaf_full).all()
            g2.free()
            key = {}
            root_pool = np.repeat(op, np.diff(os_))
            for i in range(n_next):
                key[(int(root_pool[i]),) + tuple(int(x) for x in osc[i])] = i
            sp, sso, ssc, sl = sub.next_roots()
            sroot_pool = np.repeat(sp, np.diff(sso))
            u_sub = np.array([u_syn[key[(int(sroot_pool[i]),) + tuple(int(x) for x in ssc[i])]]
                              for i in range(len(ssc))], np.float64)
            leaf = sub.leaf_utilities_linked(sl, u_sub)
        sb_o, U_o, R_o, S_o = sub.cfr(leaf, T, want_rs=True)
        gpu_roots = np.array([soff[g] + s for g in roots for s in slots[g]])
        dp, du = oracle_sensitivity(sub, leaf, sb_o, U_o, T)
        check_utilities(U_g[gpu_roots], U_o, du)
        well, ill = check_sigma(sb_g[edges], sb_o, own_mass(sub, S_o), dp, T)
        assert well > 0
    for R in rounds:
        R["gt"].free()
