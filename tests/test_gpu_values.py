"""fp64 game values on the GPU (minimax, best responses, on-policy) against the oracle's recursion,
chained over rounds 5 and 6 with the oracle's own strategy (rounded to float32) given to both
sides.  Both sum child by child in canonical order without fused multiply-add, so the values
agree to rounding (1e-12 relative); the best-response values bracket the on-policy and minimax
values."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


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


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


@pytest.mark.parametrize("seed", [0, 2, 5, 9])
def test_chained_values_match_oracle(ctx, seed):
    from paper_2508_06559_gb300 import pasur as P
    deck = O.deal(seed)
    o4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
    o4.unfold_single()
    pools, soff, scores, lnk = o4.next_roots()
    o5 = O.Tree(deck, 5, pools)
    o5.unfold(soff, scores)
    leaf5 = o5.leaf_utilities_final()
    s5, U5 = o5.cfr(leaf5, 100)
    s4, _ = o4.cfr(o4.leaf_utilities_linked(lnk, U5), 100)
    s4f, s5f = s4.astype(np.float32), s5.astype(np.float32)
    g4 = ctx.pasur_build_round(deck, 4, [mask_ids(deck[:4])])
    g4.unfold_single()
    g4.pasur_next_roots()
    g5 = ctx.pasur_build_round(deck, 5, pools)
    g5.pasur_unfold(soff, scores)
    vals = {}
    for mode in (O.MINIMAX, O.BR_ALEX, O.BR_BOB, O.ON_POLICY):
        o_v5 = o5.root_values(leaf5, mode, s5f.astype(np.float64))
        o_v4 = o4.root_values(o4.leaf_utilities_linked(lnk, o_v5), mode, s4f.astype(np.float64))
        got = P.chain_values([g4, g5], mode, [s4f, s5f])
        got5 = g5.pasur_root_values(mode, s5f)
        assert np.allclose(got5, o_v5, rtol=1e-12, atol=1e-12)
        assert np.allclose(got, o_v4, rtol=1e-12, atol=1e-12), (mode, got, o_v4)
        vals[mode] = got[0]
    assert vals[O.BR_BOB] <= vals[O.ON_POLICY] + 1e-12 <= vals[O.BR_ALEX] + 2e-12
    assert vals[O.BR_BOB] <= vals[O.MINIMAX] + 1e-12 <= vals[O.BR_ALEX] + 2e-12
    assert abs(vals[O.MINIMAX] - O.minimax_rounds(deck, 4, mask_ids(deck[:4]))) < 1e-9
    for t in (g4, g5):
        t.free()


def test_solved_strategy_exploitability_is_small(ctx):
    """After CFR on the GPU the chained best-response gap of the solved profile is small and
    shrinks with more iterations."""
    from paper_2508_06559_gb300 import pasur as P
    deck = O.deal(2)
    gaps = []
    for T in (50, 800):
        g4 = ctx.pasur_build_round(deck, 4, [mask_ids(deck[:4])])
        g4.unfold_single()
        pools, soff, scores, _ = g4.pasur_next_roots()
        g5 = ctx.pasur_build_round(deck, 5, pools)
        g5.pasur_unfold(soff, scores)
        cfg = P.pasur_config_default(iters=T)
        g5.pasur_cfr_iterate(cfg)
        g4.pasur_cfr_iterate(cfg, g5.pasur_round_utilities())
        a = P.chain_values([g4, g5], 1)[0]
        b = P.chain_values([g4, g5], 2)[0]
        gaps.append((a - b) / 2)
        for t in (g4, g5):
            t.free()
    assert gaps[0] >= 0 and gaps[1] >= 0
    assert gaps[1] < gaps[0]
