"""Pins of the oracle surrogate network (oracle/mlp.py): backpropagation against central finite
differences, GELU against the normal CDF's identities and a tabulated value, Adam's first step
against its closed form, and the feature encoding against what the deal fixes."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M


def mask_ids(ids):
    m = 0
    for c in ids:
        m |= 1 << int(c)
    return m


def small_problem(seed=0, n=7):
    rng = np.random.default_rng(seed)
    p = M.unflatten(M.init_params(seed))
    for k in ("b0", "b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.1, p[k].shape)
    X = rng.normal(0, 1, (n, M.IN))
    y = rng.normal(0, 2, n)
    return p, X, y


def test_gelu_identities_and_value():
    z = np.linspace(-6, 6, 101)
    assert np.allclose(M.gelu(-z), M.gelu(z) - z, atol=1e-14)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert abs(M.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15   # Phi(1)
    assert abs(M.gelu(np.array([8.0]))[0] - 8.0) < 1e-12
    h = 1e-6
    fd = (M.gelu(z + h) - M.gelu(z - h)) / (2 * h)
    assert np.allclose(M.gelu_grad(z), fd, atol=1e-8)


def test_backprop_matches_finite_differences():
    p, X, y = small_problem()
    loss, g, _ = M.loss_and_grads(p, X, y)
    flat, gflat = M.flatten(p), M.flatten(g)
    rng = np.random.default_rng(1)
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in M.SHAPES])
    # every bias and output weight, plus 300 random matrix entries
    idx = np.concatenate([np.arange(offs[1], offs[2]), np.arange(offs[3], offs[4]), np.arange(offs[5], offs[8]),
                          rng.integers(0, offs[1], 100), rng.integers(offs[2], offs[3], 100),
                          rng.integers(offs[4], offs[5], 100)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        lp = M.loss_and_grads(M.unflatten(flat + e), X, y)[0]
        lm = M.loss_and_grads(M.unflatten(flat - e), X, y)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, gflat[i])


def test_forward_is_the_composition():
    """Forward on one row equals the layer formulas written out with plain loops."""
    p, X, _ = small_problem(n=1)
    x = X[0]
    h = x
    for l in range(3):
        W, b = p[f"W{l}"], p[f"b{l}"]
        z = [sum(W[o, i] * h[i] for i in range(len(h))) + b[o] for o in range(M.HID)]
        h = np.array([zz * 0.5 * (1 + math.erf(zz / math.sqrt(2))) for zz in z])
    want = float(h @ p["w3"] + p["b3"][0])
    assert abs(M.forward(p, X)[0][0] - want) < 1e-10


def test_adam_first_step_is_signed_lr():
    rng = np.random.default_rng(2)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    new, m, v = M.adam_step(w, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(new, w - 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.005859375, 3.0e38, -2.5, 1 + 2 ** -8, 1 + 3 * 2 ** -9])
    r = M.to_bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[5] == 1.0   # 1 + 2^-8 is a tie -> even (1.0)
    assert r[2] == 1.0078125 and r[4] == -2.5
    assert r[6] == 1 + 2 ** -7                  # above the tie
    assert (M.to_bf16(r) == r).all()


@pytest.mark.parametrize("seed", [0, 3])
def test_features_of_real_roots(seed):
    deck = O.deal(seed)
    t4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
    t4.unfold_single()
    pools, soff, scores, _ = t4.next_roots()
    for rnd, plist, sof, sc in [(4, [mask_ids(deck[:4])], [0, 1], [[0, 0, 0, 0]]), (5, pools, soff, scores)]:
        for g, pool in enumerate(plist):
            for s in range(sof[g], sof[g + 1]):
                x = M.features(deck, rnd, int(pool), sc[s])
                assert (M.to_bf16(x) == x).all()
                onehot = x[:208].reshape(4, 52)
                assert (onehot.sum(axis=0) == 1).all()                 # every card in one place
                assert onehot[0].sum() == 4 * (6 - rnd) and onehot[1].sum() == 4 * (6 - rnd)
                assert onehot[2].sum() == bin(int(pool)).count("1")
                assert (onehot[2] == [(int(pool) >> c) & 1 for c in range(52)]).all()
                hands_a = [int(c) for i in range(rnd, 6) for c in deck[4 + 8 * i: 8 + 8 * i]]
                assert sorted(np.flatnonzero(onehot[0])) == sorted(hands_a)
                assert x[208] * 8 == sc[s][0] and x[209] * 8 == sc[s][1] and x[210] * 32 == sc[s][2]
                assert x[211:214].sum() == 1 and x[211 + sc[s][3]] == 1
                assert x[214 + rnd] == 1 and x[214:220].sum() == 1 and not x[232:].any()
                for L in range(3):
                    ids = np.flatnonzero(onehot[L])
                    assert x[223 + 4 * L] * 32 == len(ids)
                    assert x[220 + 4 * L] * 8 == sum(1 for c in ids if c % 4 == 0)        # clubs
                    assert x[222 + 4 * L] * 4 == sum(1 for c in ids if c // 4 == 10)      # Jacks
                    pts = {0: 1, 1: 1, 2: 1, 3: 1, 40: 1, 41: 1, 42: 1, 43: 1, 4: 2, 37: 3}
                    assert x[221 + 4 * L] * 8 == sum(pts.get(int(c), 0) for c in ids)
