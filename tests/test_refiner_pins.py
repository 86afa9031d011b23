"""Pins of the oracle's learned-refiner definition (oracle/refiner.py): a
hand-built patch, the rounding of the patch precisions, closed forms of the
loss and of Adam's first step, a hand-evaluated network, positive
homogeneity, the backward pass against finite differences of the loss, and
the threshold rule of the decision."""
import math

import numpy as np

import oracle.refiner as orf
import synth

T_TRIG = 1 << 20
T0 = T_TRIG + 3000


def _snake():
    """16 pixels on x 100..103 x y 49..52 in snake order, ToT 100, the k-th
    30 ticks after the first; two extra packets on occupied pixels."""
    xs, ys = [], []
    for r, y in enumerate(range(49, 53)):
        row = list(range(100, 104)) if r % 2 == 0 else list(range(103, 99, -1))
        xs += row
        ys += [y] * 4
    t = [T0 + 30 * k for k in range(16)]
    tot = [100] * 16
    # (101, 50): equal ToT, later packet -> wins the cell; (103, 52): dimmer -> loses
    xs += [101, 103]
    ys += [50, 52]
    tot += [100, 50]
    t += [T0 + 190, T0 + 370]
    return np.array(xs), np.array(ys), np.array(tot), np.array(t)


def test_hand_built_patch():
    x, y, tot, t = _snake()
    pk = np.concatenate([synth.encode_tdcs([T_TRIG]), synth.encode_pixels(x, y, tot, t)])
    p, sel, centre, r = orf.patches(pk, min_pixels=12)
    assert sel.size == 1 and r["clusters"][0]["n"] == 18
    # s_tot 1750, s_x 177650, s_y 88400: centroid (101.514, 50.514) -> (102, 51)
    assert tuple(centre[0]) == (102, 51)
    want = np.zeros(162, np.float32)
    v_tot = np.float32(0.09765625)          # 100 / 1023 = 0.097752... in bf16
    for k in range(16):
        cell = (y[k] - 47) * 9 + (x[k] - 98)
        want[cell] = v_tot
        want[81 + cell] = min(8.0, 30 * k / 32)
    want[(50 - 47) * 9 + (101 - 98) + 81] = 190 / 32
    assert np.array_equal(p[0], want)


def test_bf16_rounding():
    assert orf.bf16(1.0) == 1.0
    assert orf.bf16(1.0 + 2.0 ** -8) == 1.0                     # tie -> even
    assert orf.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6     # tie -> even (up)
    assert orf.bf16(1.0 + 1.5 * 2.0 ** -8) == 1.0 + 2.0 ** -7
    assert orf.bf16(-0.75) == -0.75
    assert orf.bf16(100 / 1023) == 0.09765625


def _const_net(h, b3):
    p = np.zeros(orf.layout(h)["total"])
    p[orf.layout(h)["b3"][0]:] = b3
    return p


def test_loss_closed_forms():
    x = np.random.default_rng(0).random((3, 162))
    p = _const_net(4, [0, 0, 0, 0, 0, 0])
    y = np.array([[1, 1.0, 2.0, 7.0, 7.0]] * 3)            # single: second offsets ignored
    assert abs(orf.loss(p, 4, x, y, 0.5) - (math.log(2) + 0.5 * 0.5 * 5.0)) < 1e-12
    p = _const_net(4, [0, math.log(3), 0, 0, 0, 0])
    y = np.array([[2, 0, 0, 1.0, -1.0]] * 3)               # pair: all four offsets count
    assert abs(orf.loss(p, 4, x, y, 2.0) - (math.log(4 / 3) + 0.5 * 2.0 * 2.0)) < 1e-12


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p0 = np.array([1.0, 1.0, 1.0, 1.0])
    p1, m, v = orf.adam(p0, np.zeros(4), np.zeros(4), g, 1, 0.01)
    assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_hand_evaluated_network():
    h = 1
    L = orf.layout(h)
    p = np.zeros(L["total"])
    p[L["w1"][0] + 0] = 1.0                 # W1[cell 0, 0]
    p[L["w2"][0]] = 2.0
    p[L["b2"][0]] = -1.0
    p[L["w3"][0]: L["w3"][0] + 6] = [1, -1, 0.5, 0, 0, 0]
    p[L["b3"][0]: L["b3"][0] + 6] = [0, 0, 1, 0, 0, 0]
    x = np.zeros((2, 162))
    x[0, 0], x[1, 0] = 0.75, 0.25
    x[:, 1:] = 5.0                           # no weight on other inputs
    out = orf.forward(p, h, x)
    assert np.allclose(out[0], [0.5, -0.5, 1.25, 0, 0, 0], atol=1e-15)
    assert np.allclose(out[1], [0, 0, 1, 0, 0, 0], atol=1e-15)


def test_bias_free_network_is_positively_homogeneous():
    rng = np.random.default_rng(1)
    h = 6
    L = orf.layout(h)
    p = rng.normal(size=L["total"])
    for k in ("b1", "b2", "b3"):
        p[L[k][0]: L[k][0] + L[k][1]] = 0.0
    x = rng.random((5, 162))
    assert np.allclose(orf.forward(p, h, 2.5 * x), 2.5 * orf.forward(p, h, x), rtol=1e-12, atol=1e-12)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    h, n, w = 5, 7, 0.7
    p = rng.normal(scale=0.3, size=orf.layout(h)["total"])
    x = rng.random((n, 162))
    y = np.zeros((n, 5))
    y[:, 0] = rng.integers(1, 3, n)
    y[:, 1:] = rng.normal(size=(n, 4))
    g = orf.grad(p, h, x, y, w)
    eps = 1e-6
    num = np.empty_like(p)
    for i in range(p.size):
        d = np.zeros_like(p)
        d[i] = eps
        num[i] = (orf.loss(p + d, h, x, y, w) - orf.loss(p - d, h, x, y, w)) / (2 * eps)
    assert np.max(np.abs(num - g)) < 1e-7 * max(1.0, np.max(np.abs(g)))


def test_decide_threshold_rule():
    out = np.array([[0, 0, .5, .5, 1, 1],        # margin 0: p = 1/2
                    [1, 0, .25, -.25, 0, 0],     # margin -1: p(one) = 0.731
                    [0, 3, 1, 2, 3, 4],          # margin 3: p(two) = 0.953
                    [0, 1, 0, 0, 0, 0]], np.float32)
    centre = np.array([[10, 20]] * 4)
    cxy = np.array([[10.3, 19.6]] * 4)
    r = orf.decide(out, centre, cxy, 0.5)
    assert list(r[:, 0]) == [2, 1, 2, 2]
    r = orf.decide(out, centre, cxy, 0.9)
    assert list(r[:, 0]) == [0, 0, 2, 0]
    assert np.allclose(r[0, 1:3], [10.3, 19.6]) and np.allclose(r[2], [2, 11, 22, 13, 24])
    r = orf.decide(out, centre, cxy, 0.7)
    assert list(r[:, 0]) == [0, 1, 2, 2] and np.allclose(r[1], [1, 10.3, 19.6, 0, 0])


def test_oracle_training_reduces_the_loss():
    """The pieces compose: Adam on the analytic gradient lowers the loss of a
    toy task (the count is whether cell 40's ToT exceeds 0.5)."""
    rng = np.random.default_rng(3)
    h, n = 8, 64
    x = rng.random((n, 162)) * 0.2
    x[:, 40] = rng.random(n)
    y = np.zeros((n, 5))
    y[:, 0] = np.where(x[:, 40] > 0.5, 2, 1)
    p = rng.normal(scale=0.1, size=orf.layout(h)["total"])
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = orf.loss(p, h, x, y, 1.0)
    for step in range(1, 301):
        p, m, v = orf.adam(p, m, v, orf.grad(p, h, x, y, 1.0), step, 0.01)
    assert orf.loss(p, h, x, y, 1.0) < 0.3 * l0


def test_bf16_inference_precision():
    """On inputs, weights and activations that bf16 holds exactly, the
    inference precision is the plain network; a hidden activation of
    1 + 2^-8 (a bf16 tie) becomes 1, and 1 + 3 * 2^-8 becomes 1 + 2^-6."""
    rng = np.random.default_rng(4)
    h = 4
    L = orf.layout(h)
    p = np.zeros(L["total"])
    # W1, b1, W3, b3: multiples of 1/8 in [-1/2, 1/2]; W2: half a cyclic shift
    for k in ("w1", "b1", "w3", "b3"):
        o, n = L[k]
        p[o: o + n] = rng.integers(-4, 5, n) / 8.0
    w2 = np.zeros((h, h))
    w2[np.arange(h), (np.arange(h) + 1) % h] = 0.5
    p[L["w2"][0]: L["w2"][0] + h * h] = w2.ravel()
    p[L["b2"][0]: L["b2"][0] + h] = rng.integers(0, 5, h) / 8.0
    # two inputs of 1/8 .. 1 per row: a1 < 2 in steps of 1/64, a2 < 1.5 in
    # steps of 1/128 -- at most 8 significant bits, exact in bf16
    x = np.zeros((6, 162))
    for r in range(6):
        x[r, rng.choice(162, 2, replace=False)] = rng.integers(1, 9, 2) / 8.0
    assert np.array_equal(orf.forward_bf16(p, h, x), orf.forward(p, h, x))
    assert np.array_equal(orf.bf16_array(np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8], np.float32)),
                          np.array([1.0, 1 + 2 ** -6], np.float32))
    h = 1
    L = orf.layout(h)
    p = np.zeros(L["total"])
    p[L["w1"][0]] = 1.0
    p[L["b1"][0]] = 2.0 ** -8                # a1 = 1 + 2^-8 -> 1 in bf16
    p[L["w2"][0]] = 1.0
    p[L["w3"][0]: L["w3"][0] + 6] = [1, 0, 0, 0, 0, 0]
    x = np.zeros((1, 162))
    x[0, 0] = 1.0
    assert orf.forward_bf16(p, h, x)[0, 0] == 1.0
    assert orf.forward(p, h, x)[0, 0] == 1.0 + 2.0 ** -8
