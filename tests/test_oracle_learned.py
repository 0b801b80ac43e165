"""Pins of the oracle's learned-warm-start parts (no counterpart in the paper):
features on a hand-worked graph, GELU values, MLP gradients against central
finite differences, Adam's first step, the softmax start."""
import math

import numpy as np


def test_features_hand_worked(orc, gg):
    # edges 0->2, 1->2, 2->0 ; in-degrees (1, 0, 2), out-degrees (1, 1, 1)
    g = gg.from_edges(3, [0, 1, 2], [2, 2, 0])
    f = orc.features(g, 0.85)
    l2 = math.log(2.0)
    expect = np.array([
        [l2, l2, l2, l2, 0.85],              # vertex 0: in-neighbour 2 (out-degree 1)
        [0.0, l2, 0.0, 0.0, 0.85],           # vertex 1: no in-neighbours
        [math.log(3.0), l2, l2, l2, 0.85],   # vertex 2: in-neighbours 0, 1
    ])
    assert np.abs(f - expect).max() < 1e-15


def test_gelu_values(orc):
    # GELU(x) = x Phi(x): Phi(0) = 1/2, Phi(1) = 0.8413447460685429 (normal CDF table)
    assert orc.gelu(np.array([0.0]))[0] == 0.0
    assert abs(orc.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(orc.gelu(np.array([-1.0]))[0] + (1 - 0.8413447460685429)) < 1e-15
    x = np.linspace(-3, 3, 13)
    h = 1e-6
    fd = (orc.gelu(x + h) - orc.gelu(x - h)) / (2 * h)
    assert np.abs(fd - orc.gelu_grad(x)).max() < 1e-8


def _params(seed=3):
    rng = np.random.default_rng(seed)
    return {k: rng.normal(0, 0.5, s) for k, s in {"W1": (64, 5), "b1": (64,), "W2": (64, 64), "b2": (64,),
                                                  "W3": (1, 64), "b3": (1,)}.items()}


def test_mlp_gradient_matches_finite_differences(orc):
    rng = np.random.default_rng(0)
    F = rng.normal(0, 1, (40, 5))
    t = rng.normal(0, 1, 40)
    p = _params()
    y, cache = orc.mlp_forward(F, p)
    g = orc.mlp_backward(p, cache, y, t)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = orc.mse_loss(orc.mlp_forward(F, p)[0], t)
            flat[idx] = old - h
            lm = orc.mse_loss(orc.mlp_forward(F, p)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_adam_first_step_moves_by_lr(orc):
    # with zero moments and bias correction, the first step is lr * g / (|g| + eps)
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-3])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    orc.adam_update(p, g, m, v, 1, lr=0.01)
    expect = np.array([1.0, -2.0, 0.5]) - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8)
    assert np.abs(p["w"] - expect).max() < 1e-12


def test_softmax_start(orc):
    y = np.array([0.0, 1.0, -2.0, 700.0, 699.0])
    r = orc.warm_start_from_logits(y)
    assert abs(r.sum() - 1.0) < 1e-15 and np.all(r >= 0)
    assert np.allclose(orc.warm_start_from_logits(y + 5.0), r)
    assert abs(r[3] / r[4] - math.e) < 1e-12


def test_bf16_rounding(orc):
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.140625, 1e-3], np.float32)
    r = orc.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                                          # 1 + 2^-8 is the tie: even -> 1.0
    assert r[2] == 1.0 + 2 ** -7                                # above the tie rounds up
    assert r[3] == -3.140625
    assert abs(r[4] - 1e-3) / 1e-3 < 2 ** -8
