"""Deals of the paper's size (over 1e9 full-game-tree nodes; section "Introduction") against the
fp64 oracle on sampled roots.

Seed 47 is the first seed whose complete six-round game exceeds 1e9 FGT nodes (3.4e9) and the
benchmark's headline deal: the GPU solves the whole game exactly as bench.py times it (T = 1000
per round, default settings); seed 93 (1.9e9) has root subtrees large enough for the
level-streaming path, solved here at T = 20.  The oracle builds its own chain of rounds up to the
final one (every root of every round), checks the final round's roots against the GPU's, then
solves sampled FGT roots of the final round with its own leaves: random ones plus the largest
roots of every solve path (one block, thread-block cluster, level-streaming sweep) at their
natural sizes.  Root utilities within 1e-5; average strategies per the parity policy of
tests/test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle as O
from tests import oracle_jobs as J

pytestmark = pytest.mark.gpu

CASES = {47: dict(T=1000, random=48, per_path=2), 93: dict(T=20, random=16, per_path=1)}


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


@pytest.mark.parametrize("seed", sorted(CASES))
def test_paper_scale_final_round(ctx, seed):
    case = CASES[seed]
    T = case["T"]
    deck = O.deal(seed)
    rng = np.random.default_rng(seed)
    # the GPU: the whole game, built forward and solved backward
    cfg = P().pasur_config_default(iters=T)
    pools = np.array([sum(1 << int(c) for c in deck[:4])], np.uint64)
    soff, sc = np.array([0, 1], np.int64), np.zeros((1, 4), np.int16)
    gts = []
    for r in range(6):
        t = ctx.pasur_build_round(deck, r, pools)
        t.pasur_unfold(soff, sc)
        gts.append((t, pools, soff, sc))
        if r < 5:
            pools, soff, sc, _ = t.pasur_next_roots_nolinks()
    total = sum(int(t.pasur_tree_sizes()[1].sum()) for t, _, _, _ in gts)
    assert total > 1e9
    nxt = None
    for t, _, _, _ in reversed(gts):
        t.pasur_cfr_iterate(cfg, nxt)
        nxt = t.pasur_round_utilities()
    g5, gp, gs, gsc = gts[5]
    U_g, sb_g, paths = g5.pasur_round_utilities(), g5.pasur_avg_strategy(), g5.pasur_root_paths()
    # the oracle's own chain: its final-round roots must be the GPU's
    chain = J.oracle_chain(deck, 0, 4)
    op, os_, osc, _ = chain[-1]["next"]
    assert np.array_equal(op, gp) and np.array_equal(os_, gs) and np.array_equal(osc, gsc)
    del chain  # the sampled solves below take their roots from the oracle's own op, os_, osc
    # picks: random FGT roots, plus the largest roots of every path taken
    root_of = J.gpu_root_of(g5)
    gt_size = sum(np.bincount(ro, minlength=len(gp)) for ro in root_of)
    n_fgt = int(gs[-1])
    root_of_slot = np.repeat(np.arange(len(gp)), np.diff(gs))
    flat = rng.choice(n_fgt, size=min(case["random"], n_fgt), replace=False)
    picks = {(int(root_of_slot[f]), int(f - gs[root_of_slot[f]])) for f in flat}
    covered = {}
    for path in sorted(set(paths.tolist()) - {-1}):
        gs_ = np.nonzero(paths == path)[0]
        for g in gs_[np.argsort(-gt_size[gs_])][:case["per_path"]]:
            picks.add((int(g), 0))
            covered[path] = covered.get(path, 0) + 1
    print(f"seed {seed}: {total} FGT nodes; final-round paths taken {sorted(covered)}; picks {len(picks)}")
    assert 6 in covered or seed != 47  # the headline deal has cluster roots
    if seed == 93:
        assert 5 in covered  # and this one level-streamed roots
    # one worker job per large root, the random picks in chunks
    picks = sorted(picks)
    big = {(g, s) for g, s in picks if paths[g] >= 4}
    chunks = [[x] for x in sorted(big)] + [c for c in (sorted(set(picks) - big)[i::8] for i in range(8)) if c]
    jobs = []
    for part in chunks:
        roots, slots, fl = J.pick_layout(os_, part)
        idx = J.edge_index(root_of, gs, roots, slots)
        label = f"seed {seed} final round, paths {sorted({int(paths[g]) for g in roots})}"
        jobs.append(dict(deck=deck, rnd=5, pools=op, soff=os_, scores=osc, picks=part, T=T, variant=0,
                         U_g=U_g[fl], sb_g=sb_g[idx], nxt=None, label=label))
    with J.pool() as p:
        out = p.map(J.check_sampled, jobs)
    for o in out:
        print(f"{o['label']}: {o['fgt_roots']} FGT roots, {o['edges']} edges, max |dU| {o['du']:.2e}, "
              f"well-conditioned edges {o['well']}, ill-conditioned parents {o['ill_parents']} "
              f"(max |d sigma| {o['ill_dsigma']:.2e}, max value change {o['ill_dvalue']:.2e})")
    assert sum(o["well"] for o in out) > 0
    for t, _, _, _ in gts:
        t.free()
