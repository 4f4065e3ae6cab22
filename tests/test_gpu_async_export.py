"""pasur_avg_strategy_async: the strategies written to page-locked host memory while the next
round's CFR runs, complete after pasur_sync, equal pasur_avg_strategy bit for bit; a device buffer
gets the same values in stream order."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_06559_gb300 import build as B
    from paper_2508_06559_gb300 import pasur
    B.build()
    return pasur


def test_async_export_equals_sync(P):
    import torch
    ctx = P.Ctx(0)
    deck = P.pasur_deal(9)
    pools = np.array([sum(1 << int(c) for c in deck[:4])], np.uint64)
    soff, sc = np.array([0, 1], np.int64), np.zeros((1, 4), np.int16)
    trees = []
    for r in (3, 4, 5):
        t = ctx.pasur_build_round(deck, r, pools)
        t.pasur_unfold(soff, sc)
        trees.append(t)
        if r < 5:
            pools, soff, sc, _ = t.pasur_next_roots()
    cfg = P.pasur_config_default(iters=50)
    nxt, got, dev = None, [], []
    for t in reversed(trees):
        t.pasur_cfr_iterate(cfg, nxt)
        nxt = t.pasur_round_utilities()
        h = torch.empty(t.n_edges(), dtype=torch.float32, pin_memory=True)
        h.fill_(-1.0)
        t.pasur_avg_strategy_async(h)  # completes after pasur_sync, while the next round solves
        d = torch.empty(t.n_edges(), dtype=torch.float32, device="cuda")
        t.pasur_avg_strategy_async(d)
        got.append(h)
        dev.append(d)
    ctx.pasur_sync()
    for t, h, d in zip(reversed(trees), got, dev):
        want = np.asarray(t.pasur_avg_strategy())
        assert np.array_equal(h.numpy(), want)
        assert np.array_equal(d.cpu().numpy(), want)
    with pytest.raises(P.PasurError):
        trees[0].pasur_avg_strategy_async(np.zeros(3, np.float32))
    for t in trees:
        t.free()
    ctx.close()
