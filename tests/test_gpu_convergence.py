"""The convergence diagnostic (pasur_cfr_convergence) against the fp64 oracle.

The paper measures CFR convergence per round as the mean squared error of each intermediate
average strategy to the final one (section "Experimental Evaluation", figure "Convergence of
CFR").  The oracle computes the same curve from independent runs: CFR is deterministic, so the
average strategy after t iterations of one run is that of a fresh run of t iterations.  The
GPU's curve must match it; merged score slots must give the curve of solving every slot.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

CHECKPOINTS = [10, 40, 100, 250, 500]


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


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


def final_round_multi(seed):
    """Round 6 (0-based 5) over every end state of round 5: (deck, pools, score offsets, scores)."""
    deck = O.deal(seed)
    t4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
    t4.unfold_single()
    pools, soff, sc, _ = t4.next_roots()
    return deck, pools, soff, sc


def oracle_curve(ot, leaf, variant):
    sig = [ot.cfr(leaf, T, variant=variant)[0] for T in CHECKPOINTS]
    return np.array([np.mean((s - sig[-1]) ** 2) for s in sig])


@pytest.mark.parametrize("seed", [5, 9])
@pytest.mark.parametrize("variant", [0, 1])
def test_convergence_curve_matches_oracle(P, ctx, seed, variant):
    """Seeds whose final round (over round 5's end states) has slots that differ only in delta."""
    deck, pools, soff, sc = final_round_multi(seed)
    ot = O.Tree(deck, 5, pools)
    ot.unfold(soff, sc)
    want = oracle_curve(ot, ot.leaf_utilities_final(), variant)
    got = {}
    for merge in (1, 0):
        gt = ctx.pasur_build_round(deck, 5, pools)
        gt.pasur_unfold(soff, sc)
        got[merge] = gt.pasur_cfr_convergence(P.pasur_config_default(variant=variant, merge_delta=merge), CHECKPOINTS)
        merged = (gt.pasur_solved_sizes()[0] < gt.pasur_tree_sizes()[1]).any()
        assert merged == bool(merge)
        gt.free()
    print(f"seed {seed} variant {variant}: oracle {want}, gpu {got[1]}")
    assert got[1][-1] == 0.0 and got[0][-1] == 0.0
    assert np.allclose(got[1], got[0], rtol=1e-9, atol=1e-15)
    # f32 CFR against fp64: the curves agree to 2 % of each point (or 1e-7 absolute, the size of
    # f32 strategy noise squared); the first checkpoint is further from the end than the last
    assert np.all(np.abs(got[1] - want) <= 0.02 * want + 1e-7), (got[1], want)
    assert want[0] > want[-2] > 0


def test_convergence_continues_a_run(P, ctx):
    """Checkpoints count iterations from the start of the run: 100 iterations, then checkpoints
    [200, 300] give the oracle's sigma-bar distance between 200 and 300 iterations."""
    deck = O.deal(5)
    pools = [mask_ids(deck[:4])]
    ot = O.Tree(deck, 5, pools)
    ot.unfold_single()
    leaf = ot.leaf_utilities_final()
    s2, s3 = ot.cfr(leaf, 200)[0], ot.cfr(leaf, 300)[0]
    gt = ctx.pasur_build_round(deck, 5, pools)
    gt.unfold_single()
    gt.pasur_cfr_iterate(P.pasur_config_default(iters=100))
    mse = gt.pasur_cfr_convergence(P.pasur_config_default(), [200, 300])
    want = np.mean((s2 - s3) ** 2)
    assert abs(mse[0] - want) <= 0.02 * want + 1e-7 and mse[1] == 0.0
    with pytest.raises(P.PasurError):
        gt.pasur_cfr_convergence(P.pasur_config_default(), [300])  # not past the iterations done
    gt.free()
