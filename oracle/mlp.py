"""FP64 reference of the round-start utility surrogate -- TEST INFRASTRUCTURE ONLY.

A small MLP predicts the average utility U of a round-start FGT root (the value the exact solver
propagates back between rounds, eq. passuputil) from the root's card state and score, so that an
earlier round can be solved without building and solving every later one.  This file restates,
in plain numpy fp64, what the surrogate computes:

  features(deck, round, pool, score) -> x in R^256   (layout below; every value exact in bf16)
  h1 = gelu(x W0^T + b0), h2 = gelu(h1 W1^T + b1), h3 = gelu(h2 W2^T + b2), y = h3 . w3 + b3
  loss = mean over rows of (y - target)^2
  Adam (Kingma and Ba, 2015) with bias correction.

gelu(z) = z * Phi(z) with Phi the standard normal CDF (Hendrycks and Gimpel, 2016).

``round_act=True`` rounds to bfloat16 exactly the values the GPU feeds to its tensor cores in
bfloat16 (h1, h2 and the pre-activation gradients dz; the callers pass inputs and weights
already rounded), so that the GPU's f32 accumulation can be compared closely;
``round_act=False`` is the plain fp64 network.
Pinned by tests/test_oracle_mlp.py (central finite differences, GELU identities, Adam's first
step, feature invariants).
"""
from __future__ import annotations

import math

import numpy as np

IN, HID = 256, 256
N_FEATURES_USED = 232

# flat parameter layout (shared with the C ABI's documented layout)
SHAPES = [("W0", (HID, IN)), ("b0", (HID,)), ("W1", (HID, HID)), ("b1", (HID,)), ("W2", (HID, HID)),
          ("b2", (HID,)), ("w3", (HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], np.float64).reshape(shp)
        o += n
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in SHAPES])


def to_bf16(a):
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def features(deck, rnd: int, pool: int, score) -> np.ndarray:
    """Input vector of a round-start root of round `rnd` (0..5) of deal `deck`.

    [0, 208): card locations, one-hot per card, location-major: Alex (holds now or is dealt
    later: deck[4+8i : 8+8i] for rounds i >= rnd), Bob (deck[8+8i : 12+8i], i >= rnd), pool
    (the root's pool set), out (every other card: captured in earlier rounds); feature index
    = 52 * location + card id.
    208, 209: Alex's and Bob's carried club counts / 8;  210: inherited difference / 32;
    211..213: 7-clubs bonus one-hot (none, Alex, Bob);  214..219: round one-hot;
    220 + 4 * loc + (0, 1, 2, 3) for loc = Alex, Bob, pool: that location's clubs / 8, points / 8
    (Aces and Jacks 1, two of clubs 2, ten of diamonds 3; Table "Pasur Scoring System"),
    Jacks / 4 and cards / 32;  232..255: 0.
    """
    x = np.zeros(IN, np.float64)
    deck = [int(c) for c in deck]
    loc = [3] * 52
    for i in range(rnd, 6):
        for c in deck[4 + 8 * i: 8 + 8 * i]:
            loc[c] = 0
        for c in deck[8 + 8 * i: 12 + 8 * i]:
            loc[c] = 1
    for c in range(52):
        if (int(pool) >> c) & 1:
            loc[c] = 2
    for c in range(52):
        x[52 * loc[c] + c] = 1.0
    ac, bc, delta, bonus = (int(v) for v in score)
    x[208] = ac / 8.0
    x[209] = bc / 8.0
    x[210] = delta / 32.0
    x[211 + bonus] = 1.0
    x[214 + rnd] = 1.0
    for L in range(3):
        cards = [c for c in range(52) if loc[c] == L]
        clubs = sum(1 for c in cards if c % 4 == 0)
        points = sum(1 for c in cards if c < 4 or 40 <= c < 44) + 2 * (4 in cards) + 3 * (37 in cards)
        jacks = sum(1 for c in cards if 40 <= c < 44)
        x[220 + 4 * L] = clubs / 8.0
        x[221 + 4 * L] = points / 8.0
        x[222 + 4 * L] = jacks / 4.0
        x[223 + 4 * L] = len(cards) / 32.0
    return x


_SQRT2 = math.sqrt(2.0)
_INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)
_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    return z * 0.5 * (1.0 + _erf(z / _SQRT2))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / _SQRT2)) + z * _INV_SQRT_2PI * np.exp(-0.5 * z * z)


def forward(p, X, round_act: bool = False):
    """Returns (y, cache) for rows X [n, 256]."""
    X = np.asarray(X, np.float64)
    cache = {"h0": X}
    h = X
    for l in range(3):
        z = h @ p[f"W{l}"].T + p[f"b{l}"]
        a = gelu(z)
        if round_act and l < 2:  # h1, h2 are tensor-core operands; h3 feeds the f32 output dot
            a = to_bf16(a)
        cache[f"z{l}"] = z
        cache[f"h{l + 1}"] = a
        h = a
    y = h @ p["w3"] + p["b3"][0]
    return y, cache


def loss_and_grads(p, X, target, round_act: bool = False):
    """Mean squared error and its gradient with respect to every parameter (backpropagation)."""
    y, c = forward(p, X, round_act)
    n = len(y)
    r = y - np.asarray(target, np.float64)
    loss = float((r * r).mean())
    g_y = 2.0 * r / n
    grads = {"w3": c["h3"].T @ g_y, "b3": np.array([g_y.sum()])}
    dh = np.outer(g_y, p["w3"])
    for l in (2, 1, 0):
        dz = dh * gelu_grad(c[f"z{l}"])
        grads[f"b{l}"] = dz.sum(axis=0)
        if round_act:  # dz is a tensor-core operand of the weight and input gradients
            dz = to_bf16(dz)
        grads[f"W{l}"] = dz.T @ c[f"h{l}"]
        if l:
            dh = dz @ p[f"W{l}"]
    return loss, grads, y


def adam_step(flat, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) of flat parameters; returns (flat, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (numpy generator)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in SHAPES:
        if name.startswith("b"):
            p[name] = np.zeros(shp)
        else:
            fan_in = shp[-1] if len(shp) == 2 else shp[0]
            p[name] = rng.uniform(-1.0, 1.0, shp) / math.sqrt(fan_in)
    return flatten(p)
