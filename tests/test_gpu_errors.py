"""Argument checks of the newer entry points: each invalid call returns its documented status
(raised as PasurError by the binding) and leaves the context usable."""
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


def raises(code, fn, *a, **k):
    from paper_2508_06559_gb300 import pasur as P
    with pytest.raises(P.PasurError) as e:
        fn(*a, **k)
    assert e.value.code == code, (e.value.code, str(e.value))


def test_surrogate_arguments(ctx):
    from paper_2508_06559_gb300 import pasur as P
    m = P.Mlp(ctx, dataset_capacity=10)
    raises(P.PASUR_EINVAL, m.set_params, np.zeros(10, np.float32))               # wrong length
    raises(P.PASUR_EINVAL, m.train, 1, 100, 1e-3)                                # batch not a multiple of 128
    raises(P.PASUR_EINVAL, m.train, 1, 128, 1e-3)                                # empty training set
    raises(P.PASUR_EOVERFLOW, m.dataset_add_rows, np.zeros((11, 256), np.uint16), np.zeros(11, np.float32))
    m.dataset_add_rows(np.zeros((3, 256), np.uint16), np.ones(3, np.float32))
    assert m.dataset_size() == 3
    m.dataset_clear()
    assert m.dataset_size() == 0
    deck = O.deal(2)
    t5 = ctx.pasur_build_round(deck, 5, [mask_ids(deck[:4])])
    t5.unfold_single()
    raises(P.PASUR_EINVAL, m.dataset_add_tree, t5)                               # not solved yet
    raises(P.PASUR_EINVAL, m.predict_next, t5)                                   # final round has no next roots
    assert m.forward(np.zeros((0, 256), np.uint16)).shape == (0,)
    t5.free()
    m.free()


def test_value_pass_and_cut_batch_arguments(ctx):
    from paper_2508_06559_gb300 import pasur as P
    deck = O.deal(2)
    t4 = ctx.pasur_build_round(deck, 4, [mask_ids(deck[:4])])
    t4.unfold_single()
    raises(P.PASUR_EINVAL, t4.pasur_root_values, 5)                              # bad mode
    raises(P.PASUR_EINVAL, t4.pasur_root_values, 0)                              # non-final round without links
    t4.free()
    cfg = P.pasur_config_default(iters=10)
    raises(P.PASUR_EINVAL, P.Batch, ctx, deck[None], 3, cfg, 2)                  # last round before first
    raises(P.PASUR_EINVAL, P.Batch, ctx, deck[None], 3, cfg, 4)                  # a cut needs the surrogate
    raises(P.PASUR_EINVAL, P.Batch, ctx, deck[None], 0, P.pasur_config_default(iters=10, split_bytes=-1))
    m = P.Mlp(ctx)
    b = P.Batch(ctx, deck[None], 3, cfg, last_round=4, mlp=m)
    raises(P.PASUR_EINVAL, b.pasur_batch_selfplay, 10, np.zeros(1, np.uint64))   # before solving
    b.pasur_batch_solve()
    raises(P.PASUR_EINVAL, b.pasur_batch_selfplay, 10, np.zeros(1, np.uint64))   # cut before the final round
    b.free()
    m.free()
    # the context still works
    t = ctx.pasur_build_round(deck, 5, [mask_ids(deck[:4])])
    t.unfold_single()
    t.pasur_cfr_iterate(cfg)
    assert np.isfinite(t.pasur_round_utilities()).all()
    t.free()
