"""Host logic of the surrogate's exact fallback and tuning (paper_2508_06559_gb300/hybrid.py) on
CPU: the root subsets handed to pasur_batch_create_roots and the seeded pool sample."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2508_06559_gb300 import hybrid as H  # noqa: E402


def random_roots(rng):
    n = int(rng.integers(0, 30))
    soff = np.concatenate([[0], np.cumsum(rng.integers(1, 5, n))]).astype(np.int64)
    pools = np.sort(rng.choice(1 << 40, n, replace=False)).astype(np.uint64)
    scores = rng.integers(0, 50, (int(soff[-1]), 4)).astype(np.int16)
    return pools, soff, scores


def test_roots_subset():
    rng = np.random.default_rng(0)
    for _ in range(300):
        pools, soff, scores = random_roots(rng)
        m = int(soff[-1])
        sel = np.sort(rng.choice(m, int(rng.integers(0, m + 1)), replace=False)) if m else np.zeros(0, np.int64)
        p, so, sc = H.roots_subset(pools, soff, scores, sel)
        # rebuilt slot by slot: every selected slot under its own pool, pools ascending and distinct
        want_p, want_so = [], [0]
        for i in sel:
            g = int(np.searchsorted(soff, i, side="right") - 1)
            if not want_p or want_p[-1] != pools[g]:
                want_p.append(pools[g])
                want_so.append(want_so[-1])
            want_so[-1] += 1
        assert np.array_equal(p, np.array(want_p, np.uint64)) and np.array_equal(so, np.array(want_so, np.int64))
        assert np.array_equal(sc, scores[sel]) and so.dtype == np.int64


def test_sample_pools():
    rng = np.random.default_rng(1)
    for trial in range(300):
        pools, soff, _ = random_roots(rng)
        frac = float(rng.choice([0.0, 0.05, 0.3, 1.0]))
        s = H.sample_pools(pools, soff, frac, np.random.default_rng([7, trial]))
        assert np.array_equal(s, H.sample_pools(pools, soff, frac, np.random.default_rng([7, trial])))
        if len(pools) == 0 or frac == 0:
            assert len(s) == 0
            continue
        assert np.all(np.diff(s) > 0)
        g = np.searchsorted(soff, s, side="right") - 1
        picked = np.unique(g)
        assert len(picked) == min(len(pools), max(1, round(frac * len(pools))))
        assert np.array_equal(s, np.concatenate([np.arange(soff[p], soff[p + 1]) for p in picked]))
