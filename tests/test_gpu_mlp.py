"""The surrogate network's tensor-core kernels against the oracle network (oracle/mlp.py).

Forward values and gradients are compared with the oracle evaluated in fp64 on the same
bf16-rounded weights and inputs, with the oracle rounding to bf16 exactly the values the GPU
feeds to its tensor cores in bf16 (round_act=True); the remaining differences are f32
accumulation order and f32 GELU, so the bounds are tight (forward 1e-3, gradients 1e-2
relative per tensor as the surrogate's parity bound).  Against the plain fp64 network (no
rounding) the bound is the bf16 one (3e-2).  Rows come from real round-start roots, in counts
that leave a ragged last tile.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M

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


def bf16_bits(a):
    return (np.asarray(M.to_bf16(a), np.float32).view(np.uint32) >> 16).astype(np.uint16)


def real_rows(seeds):
    """Oracle features of the round-5 roots reached from round 4 of each deal (and the round-4
    root), plus a target: each deal's oracle-solved round-5 root utility."""
    X, Y = [], []
    for sd in seeds:
        deck = O.deal(sd)
        t4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
        t4.unfold_single()
        pools, soff, scores, _ = t4.next_roots()
        X.append(M.features(deck, 4, mask_ids(deck[:4]), (0, 0, 0, 0)))
        Y.append(0.0)
        t5 = O.Tree(deck, 5, pools)
        t5.unfold(soff, scores)
        _, U5 = t5.cfr(t5.leaf_utilities_final(), 50)
        for g, pool in enumerate(pools):
            for s in range(soff[g], soff[g + 1]):
                X.append(M.features(deck, 5, int(pool), scores[s]))
                Y.append(U5[s])
    return np.array(X), np.array(Y)


def params(seed):
    """f32 parameters with nonzero biases; the oracle's view: weights rounded to bf16."""
    rng = np.random.default_rng(seed)
    p = M.unflatten(M.init_params(seed))
    for k in ("b0", "b1", "b2", "b3"):
        p[k] = rng.normal(0, 0.2, p[k].shape)
    flat32 = M.flatten(p).astype(np.float32)
    return flat32, oracle_view(flat32)


def oracle_view(flat32):
    p = M.unflatten(flat32.astype(np.float64))
    for k in ("W0", "W1", "W2"):
        p[k] = M.to_bf16(p[k])
    return p


def test_features_bit_exact(ctx):
    from paper_2508_06559_gb300 import pasur as P
    for sd in (0, 5):
        deck = O.deal(sd)
        t4 = O.Tree(deck, 4, [mask_ids(deck[:4])])
        t4.unfold_single()
        pools, soff, scores, _ = t4.next_roots()
        got = P.pasur_mlp_root_features(ctx, deck, 5, pools, soff, scores)
        want = np.array([M.features(deck, 5, int(pools[g]), scores[s])
                         for g in range(len(pools)) for s in range(soff[g], soff[g + 1])])
        assert (got == bf16_bits(want)).all()


@pytest.mark.parametrize("seed", [0, 1])
def test_forward_matches_oracle(ctx, seed):
    from paper_2508_06559_gb300 import pasur as P
    X, _ = real_rows([0, 2, 5, 9])
    assert len(X) % 128 != 0
    flat32, po = params(seed)
    mlp = P.Mlp(ctx)
    mlp.set_params(flat32)
    got = mlp.forward(bf16_bits(X))
    want, _ = M.forward(po, X, round_act=True)
    exact, _ = M.forward(M.unflatten(flat32.astype(np.float64)), X)
    assert np.abs(got - want).max() <= 1e-3 * (1 + np.abs(want).max()), np.abs(got - want).max()
    assert np.abs(got - exact).max() <= 3e-2 * (1 + np.abs(exact).max())
    # random dense rows too (every input column in use), several tiles
    rng = np.random.default_rng(seed)
    Xr = M.to_bf16(rng.normal(0, 1, (517, 256)))
    got = mlp.forward(bf16_bits(Xr))
    want, _ = M.forward(po, Xr, round_act=True)
    assert np.abs(got - want).max() <= 1e-3 * (1 + np.abs(want).max()), np.abs(got - want).max()
    mlp.free()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


BF16_ELEM_TOL = 2.0 ** -6


def grad_scale(po, X, target):
    """Per gradient element, the sum of the absolute values of the products that form it: the
    backward pass of the oracle network carried out on absolute values (|dz|, |h|, |W|,
    |gelu'|), the scale of a rounding-error bound for that element."""
    y, c = M.forward(po, X, round_act=True)
    n = len(y)
    gy = np.abs(2.0 * (y - target) / n)
    out = {"w3": c["h3"].T.__abs__() @ gy, "b3": np.array([gy.sum()])}
    adh = np.outer(gy, np.abs(po["w3"]))
    for l in (2, 1, 0):
        adz = adh * np.abs(M.gelu_grad(c[f"z{l}"]))
        out[f"b{l}"] = adz.sum(axis=0)
        out[f"W{l}"] = adz.T @ np.abs(c[f"h{l}"])
        if l:
            adh = adz @ np.abs(po[f"W{l}"])
    return out


@pytest.mark.parametrize("n", [300, 1000])
def test_gradients_match_oracle(ctx, n):
    from paper_2508_06559_gb300 import pasur as P
    X, Y = real_rows([0, 2, 5, 9, 11, 13])
    rng = np.random.default_rng(n)
    idx = rng.integers(0, len(X), n)
    X, Y = X[idx], Y[idx] + rng.normal(0, 0.5, n)
    flat32, po = params(3)
    mlp = P.Mlp(ctx)
    mlp.set_params(flat32)
    loss, g = mlp.gradients(bf16_bits(X), Y.astype(np.float32))
    lo, go, _ = M.loss_and_grads(po, X, Y.astype(np.float32).astype(np.float64), round_act=True)
    le, ge, _ = M.loss_and_grads(M.unflatten(flat32.astype(np.float64)), X, Y.astype(np.float32).astype(np.float64))
    assert abs(loss - lo) <= 1e-3 * lo
    gg = M.unflatten(g.astype(np.float64))
    scale = grad_scale(po, X, Y.astype(np.float32).astype(np.float64))
    for name, _ in M.SHAPES:
        # element by element: every product that enters a gradient element may be off by one
        # bf16 rounding of each operand (2^-8 relative) plus what earlier layers carried in; the
        # bound is BF16_ELEM_TOL times the sum of the absolute values of those products
        ratio = np.abs(gg[name] - go[name]) / (scale[name] + 1e-30)
        print(f"{name}: max |g_gpu - g_oracle| / scale {ratio.max():.3e}, norm-relative {rel(gg[name], go[name]):.2e}")
        assert (np.abs(gg[name] - go[name]) <= BF16_ELEM_TOL * scale[name] + 1e-12).all(), (name, float(ratio.max()))
        assert rel(gg[name], ge[name]) <= 3e-2, (name, rel(gg[name], ge[name]))
    mlp.free()


def test_adam_steps_match_oracle(ctx):
    """Three full-batch Adam steps on 256 rows: GPU parameters against the oracle's."""
    from paper_2508_06559_gb300 import pasur as P
    X, Y = real_rows([0, 2, 5, 9, 11, 13, 17])
    X, Y = X[:256], Y[:256].astype(np.float32)
    flat32, _ = params(4)
    lr = 1e-3
    mlp = P.Mlp(ctx, dataset_capacity=256)
    mlp.set_params(flat32)
    mlp.dataset_add_rows(bf16_bits(X), Y)
    xs, ys = mlp.dataset_export()
    assert (xs == bf16_bits(X)).all() and (ys == Y).all()
    mlp.train(3, 256, lr, shuffle_seed=9)
    got = mlp.get_params()
    flat = flat32.astype(np.float64)
    m = np.zeros_like(flat)
    v = np.zeros_like(flat)
    for t in (1, 2, 3):
        _, g, _ = M.loss_and_grads(oracle_view(flat.astype(np.float32)), X, Y.astype(np.float64), round_act=True)
        flat, m, v = M.adam_step(flat, M.flatten(g), m, v, t, lr)
    d = np.abs(got - flat)
    # an update is lr * m_hat / sqrt(v_hat): elements whose gradient is at rounding level may move
    # differently, by at most 2 lr per step; all others agree closely
    assert d.max() <= 6 * lr + 1e-6
    assert (d > 0.1 * lr).mean() < 0.01, (d > 0.1 * lr).mean()
    assert np.median(d) < 1e-5
    mlp.free()


def test_dataset_from_tree_and_prediction_order(ctx):
    from paper_2508_06559_gb300 import pasur as P
    deck = O.deal(5)
    t4 = ctx.pasur_build_round(deck, 4, [mask_ids(deck[:4])])
    t4.unfold_single()
    pools, soff, scores, _ = t4.pasur_next_roots()
    t5 = ctx.pasur_build_round(deck, 5, pools)
    t5.pasur_unfold(soff, scores)
    t5.pasur_cfr_iterate(P.pasur_config_default(iters=100))
    mlp = P.Mlp(ctx, dataset_capacity=10000, seed=1)
    mlp.dataset_add_tree(t5)
    x, y = mlp.dataset_export()
    want = np.array([M.features(deck, 5, int(pools[g]), scores[s]) for g in range(len(pools))
                     for s in range(soff[g], soff[g + 1])])
    assert (x == bf16_bits(want)).all()
    assert (y == t5.pasur_round_utilities()).all()
    # predictions for round 4's next roots = forward of the same rows
    pred = mlp.predict_next(t4)
    assert (pred == mlp.forward(x)).all()
    for t in (t4, t5):
        t.free()
    mlp.free()


def no_learning_params():
    """A network that outputs exactly the estimate without learning: +7 when Alex holds the
    7-clubs bonus, -7 when Bob does, else 0 (two units passed through GELU at scale 10, where
    gelu(10) = 10 to float precision)."""
    from paper_2508_06559_gb300 import pasur as P
    p = np.zeros(P.N_MLP_PARAMS, np.float32)
    per = 256 * 256 + 256
    W0 = p[0:65536].reshape(256, 256)
    W0[0, 212], W0[1, 213] = 10, 10
    for l in (1, 2):
        W = p[l * per:l * per + 65536].reshape(256, 256)
        W[0, 0], W[1, 1] = 1, 1
    p[3 * per], p[3 * per + 1] = 0.7, -0.7
    return p


def test_surrogate_gain_over_no_learning(ctx):
    """What the trained network gains: trained on exact round-start utilities of 4096 seeded deals
    (rounds 4-6 of each, batched exact solves), it replaces the unfolding of rounds 4-6 when rounds
    1-3 of 8 held-out deals are solved.  Against the estimate without learning it must lower the
    squared error of the round-4 root values by at least 30 %.  The exploitability of the composed
    whole-game profile (rounds 1-3 from the surrogate solve, 4-6 exact; fp64 best-response chain
    over all six exact rounds) is measured for both and must be a valid gap (>= 0); it is not
    asserted to improve: over deals 0-7 the two estimates give mean gaps of 2.5 and 2.2 points
    (against 0.02 for the exact solve), so the network's error still decides some early moves."""
    from paper_2508_06559_gb300 import pasur as P
    m0 = P.Mlp(ctx)
    m0.set_params(no_learning_params())
    xf = np.zeros((3, 256), np.float64)
    xf[1, 212] = 1
    xf[2, 213] = 1
    assert np.allclose(m0.forward(bf16_bits(xf)), [0, 7, -7], atol=1e-4)
    mlp = P.Mlp(ctx, dataset_capacity=2_000_000, seed=7)
    cfg_l = P.pasur_config_default(iters=300)
    for i in range(0, 4096, 64):
        b = P.Batch(ctx, np.stack([O.deal(10000 + i + j) for j in range(64)]), 3, cfg_l)
        b.pasur_batch_solve()
        for d in range(64):
            for r in (3, 4, 5):
                mlp.dataset_add_tree(b.pasur_batch_tree(d, r))
        b.free()
    losses = mlp.train(5, 1024, 1e-3, shuffle_seed=1)
    assert losses[-1] < losses[0]
    cfg = P.pasur_config_default(iters=1000)
    res = {"mlp": [], "none": []}
    for s in range(8):
        deck = O.deal(s)[None]
        be = P.Batch(ctx, deck, 0, cfg)
        be.pasur_batch_solve()
        te = [be.pasur_batch_tree(0, r) for r in range(6)]
        u3 = te[3].pasur_round_utilities()
        for key, net in (("mlp", mlp), ("none", m0)):
            bs = P.Batch(ctx, deck, 0, cfg, last_round=2, mlp=net)
            bs.pasur_batch_solve()
            ts = [bs.pasur_batch_tree(0, r) for r in range(3)]
            sig = [t.pasur_avg_strategy() for t in ts] + [None] * 3
            mse = float(((net.predict_next(ts[2]) - u3) ** 2).mean())
            expl = (P.chain_values(te, 1, sig)[0] - P.chain_values(te, 2, sig)[0]) / 2
            res[key].append((mse, expl))
            bs.free()
        be.free()
    a, z = np.array(res["mlp"]), np.array(res["none"])
    assert a[:, 0].mean() < 0.7 * z[:, 0].mean(), (a[:, 0].mean(), z[:, 0].mean())
    assert (a[:, 1] >= -1e-9).all() and (z[:, 1] >= -1e-9).all() and np.isfinite(a).all()
    mlp.free()
    m0.free()
