"""Batch creation on several host threads (one worker context per thread, each with its own
stream and error word, allocations charged to the parent context).

What a deal's build produces depends only on the deal, so the thread count may change neither the
results nor the number of kernels launched; the memory the workers allocate is accounted to the
parent and returns to it when the batch is freed; and a device-memory budget that the batch
exceeds fails the creation with PASUR_ENOMEM, leaks nothing and leaves the context usable.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEEDS = list(range(20, 32))
FIRST, T = 4, 60


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2508_06559_gb300 import build as B
    from paper_2508_06559_gb300 import pasur
    B.build()
    return pasur


def decks(P):
    return np.stack([P.pasur_deal(s) for s in SEEDS])


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


def warm(P, ctx):
    """One small build so that the context's capture table is in place before a baseline."""
    d = P.pasur_deal(1)
    t = ctx.pasur_build_round(d, 5, [mask_ids(d[:4])])
    t.free()


def solve(P, ctx, n_workers, monkeypatch):
    monkeypatch.setenv("PASUR_BUILD_WORKERS", str(n_workers))
    l0 = ctx.pasur_launch_count()
    b = P.Batch(ctx, decks(P), FIRST, P.pasur_config_default(iters=T, threads=128))
    launches_create = ctx.pasur_launch_count() - l0
    u = np.array(b.pasur_batch_solve())
    sig = []
    for d in (0, 5, 11):
        t = b.pasur_batch_tree(d, 5)
        sig.append(np.array(t.pasur_avg_strategy()))
    b.free()
    return u, sig, launches_create


def test_worker_count_does_not_change_results(P, monkeypatch):
    ctx = P.Ctx(0)
    u1, s1, l1 = solve(P, ctx, 1, monkeypatch)
    u8, s8, l8 = solve(P, ctx, 8, monkeypatch)
    u3, s3, l3 = solve(P, ctx, 3, monkeypatch)
    assert np.array_equal(u1, u8) and np.array_equal(u1, u3)
    for a, b, c in zip(s1, s8, s3):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    assert l1 == l8 == l3 > 0          # every worker's launches are counted on the parent
    ctx.close()


def test_worker_memory_returns_to_parent(P, monkeypatch):
    ctx = P.Ctx(0)
    warm(P, ctx)
    base = ctx.memory()[0]
    monkeypatch.setenv("PASUR_BUILD_WORKERS", "8")
    b = P.Batch(ctx, decks(P), FIRST, P.pasur_config_default(iters=T, threads=128))
    held = ctx.memory()[0]
    assert held > base
    b.pasur_batch_solve()
    b.free()
    assert ctx.memory()[0] == base
    ctx.close()


def test_budget_exceeded_by_workers_fails_cleanly(P, monkeypatch):
    monkeypatch.setenv("PASUR_BUILD_WORKERS", "8")
    probe = P.Ctx(0)
    warm(P, probe)
    base, _ = probe.memory()
    b = P.Batch(probe, decks(P), FIRST, P.pasur_config_default(iters=T, threads=128))
    need = probe.memory()[1] - base
    b.free()
    probe.close()
    assert need > 0
    ctx = P.Ctx(0, base + need // 2)
    warm(P, ctx)
    base2 = ctx.memory()[0]
    with pytest.raises(P.PasurError) as e:
        P.Batch(ctx, decks(P), FIRST, P.pasur_config_default(iters=T, threads=128))
    assert e.value.code == P.PASUR_ENOMEM
    assert "budget" in str(e.value)
    assert ctx.memory()[0] == base2        # nothing the workers allocated is left behind
    # the context still builds and solves within its budget
    d = P.pasur_deal(3)
    t = ctx.pasur_build_round(d, 5, [mask_ids(d[:4])])
    t.unfold_single()
    t.pasur_cfr_iterate(P.pasur_config_default(iters=10))
    assert np.isfinite(t.pasur_round_utilities()).all()
    t.free()
    ctx.close()
