"""Full six-round game of the seed-0 deal at full size, solved as bench.py's secondary full-game
line runs it (T = 1000 per round, default solver settings), checked against the fp64 oracle:

  - every round's GT and FGT level sizes, next roots and links: bit-exact (the oracle builds the
    whole game itself);
  - the final round's CFR on 256 seeded FGT roots (the oracle solves only those roots, with its
    own leaf values): root utilities within 1e-5, average strategies per the parity policy of
    tests/test_gpu_parity.py;
  - every earlier round's CFR on 256 seeded FGT roots with a seeded synthetic next-round utility
    vector fed to both sides (no oracle input comes from the GPU).
The oracle's sampled solves run in a pool of spawned processes.
"""
import numpy as np
import pytest

import oracle as O
from tests import oracle_jobs as J

pytestmark = pytest.mark.gpu

SEED, T, SAMPLE = 0, 1000, 256


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


def split(picks, n):
    return [picks[i::n] for i in range(n) if picks[i::n]]


def test_full_game_seed0(ctx):
    deck = O.deal(SEED)
    rng = np.random.default_rng(7)
    cfg = P().pasur_config_default(iters=T)
    chain = J.oracle_chain(deck, 0, 5)
    gts = []
    for R in chain:
        gt = ctx.pasur_build_round(deck, R["round"], R["pools"])
        gq = gt.pasur_unfold(R["soff"], R["scores"])
        assert gt.pasur_tree_sizes()[0].tolist() == R["tree"].sizes()[0].tolist()
        assert gq.tolist() == R["tree"].sizes()[1].tolist()
        if R["round"] < 5:
            gp, gs, gsc, gl = gt.pasur_next_roots()
            op, os_, osc, ol = R["next"]
            assert gp.tolist() == op.tolist() and gs.tolist() == os_.tolist()
            assert (gsc == osc).all() and (gl == ol).all()
        gts.append(gt)
    # the whole backward solve on the GPU, as the benchmark runs it
    nxt = None
    res = {}
    for r in range(5, -1, -1):
        g = gts[r]
        g.pasur_cfr_iterate(cfg, nxt)
        res[r] = (g.pasur_round_utilities(), g.pasur_avg_strategy())
        nxt = res[r][0]
        assert np.isfinite(nxt).all()
    # sampled checks, round by round
    jobs = []
    for R in chain:
        r, pools, soff, scores, ot = R["round"], R["pools"], R["soff"], R["scores"], R["tree"]
        n_fgt_roots = int(soff[-1])
        flat = rng.choice(n_fgt_roots, size=min(SAMPLE, n_fgt_roots), replace=False)
        root_of_slot = np.repeat(np.arange(len(pools)), np.diff(soff))
        picks = [(int(root_of_slot[f]), int(f - soff[root_of_slot[f]])) for f in flat]
        if r == 5:
            U_g, sb_g, nx = res[5][0], res[5][1], None
        else:
            # seeded synthetic next-round utilities, exactly representable in float32
            op, os_, osc, ol = R["next"]
            u_syn = (np.round(rng.normal(0.0, 6.0, len(osc)) * 256) / 256).astype(np.float32)
            g2 = ctx.pasur_build_round(deck, r, pools)
            g2.pasur_unfold(soff, scores)
            g2.pasur_next_roots()
            g2.pasur_cfr_iterate(cfg, u_syn)
            U_g, sb_g = g2.pasur_round_utilities(), g2.pasur_avg_strategy()
            # leaf values of the whole round (eq. passuputil): exact, since d + u is a float32
            assert (g2.pasur_leaf_values() == ot.leaf_utilities_linked(ol, u_syn.astype(np.float64))).all()
            g2.free()
            nx = (op, os_, osc, u_syn.astype(np.float64))
        for part in split(picks, 16):
            roots, slots, fl = J.pick_layout(soff, part)
            idx = J.full_edge_index(ot, soff, roots, slots)
            jobs.append(dict(deck=deck, rnd=r, pools=pools, soff=soff, scores=scores, picks=part, T=T, variant=0,
                             U_g=U_g[fl], sb_g=sb_g[idx], nxt=nx, label=f"seed {SEED} round {r}"))
    with J.pool() as p:
        out = p.map(J.check_sampled, jobs)
    for r in range(6):
        o = [x for x in out if x["label"] == f"seed {SEED} round {r}"]
        print(f"round {r}: {sum(x['fgt_roots'] for x in o)} FGT roots, {sum(x['edges'] for x in o)} edges, "
              f"max |dU| {max(x['du'] for x in o):.2e}, well-conditioned edges {sum(x['well'] for x in o)}, "
              f"ill-conditioned parents {sum(x['ill_parents'] for x in o)} (max |d sigma| "
              f"{max(x['ill_dsigma'] for x in o):.2e}, max value change {max(x['ill_dvalue'] for x in o):.2e})")
        assert sum(x["well"] for x in o) > 0
    for g in gts:
        g.free()
