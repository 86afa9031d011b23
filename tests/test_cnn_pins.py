"""Pins of the oracle's convolutional refiner (oracle/refiner.py, CNN part):
the convolution against a hand-evaluated case and against scipy's 2-D
correlation, its translation equivariance, the layer shapes and parameter
count, the backward pass against central finite differences of the loss, and
the inference precision equal to the plain network on bf16-exact values."""
import numpy as np
import pytest

import oracle.refiner as orf


def test_hand_evaluated_convolution():
    # one channel 4 x 4, v[y][x] = 10 y + x; kernel w[ky][kx] = 3 ky + kx + 1; bias 0.5
    x = (10 * np.arange(4)[:, None] + np.arange(4)[None, :]).astype(float).reshape(1, 1, 4, 4)
    w = (3 * np.arange(3)[:, None] + np.arange(3)[None, :] + 1).astype(float).reshape(1, 1, 3, 3)
    out = orf.conv2d(x, w, np.array([0.5]))
    # by hand: sum_{ky,kx} (3ky + kx + 1)(10(y + ky) + x + kx) + 0.5
    assert out.shape == (1, 1, 2, 2)
    assert out[0, 0, 0, 0] == 681.5        # 8 + 167 + 506
    assert out[0, 0, 0, 1] == 726.5        # 14 + 182 + 530
    assert out[0, 0, 1, 0] == 1131.5       # + 10 * 45
    assert out[0, 0, 1, 1] == 1176.5


def test_convolution_equals_scipy_correlate2d():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 5, 9, 9))
    w = rng.normal(size=(4, 5, 3, 3))
    b = rng.normal(size=4)
    out = orf.conv2d(x, w, b)
    for n in range(3):
        for co in range(4):
            want = b[co] + sum(signal.correlate2d(x[n, ci], w[co, ci], mode="valid") for ci in range(5))
            assert np.allclose(out[n, co], want, rtol=0, atol=1e-12)


def test_convolution_is_translation_equivariant():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 2, 9, 9))
    w = rng.normal(size=(3, 2, 3, 3))
    b = rng.normal(size=3)
    shifted = np.zeros_like(x)
    shifted[:, :, 1:, 2:] = x[:, :, :-1, :-2]
    a, s = orf.conv2d(x, w, b), orf.conv2d(shifted, w, b)
    assert np.allclose(s[:, :, 1:, 2:], a[:, :, :-1, :-2], atol=1e-12)


def test_layer_shapes_and_parameter_count():
    L = orf.cnn_layout()
    assert L["total"] == 49_750
    p = np.random.default_rng(3).normal(size=L["total"]) * 0.1
    out, (a0, a1, a2, a3, a4) = orf.cnn_forward(p, np.zeros((2, 162)), keep=True)
    assert (a0.shape, a1.shape, a2.shape, a3.shape, a4.shape, out.shape) == (
        (2, 2, 9, 9), (2, 16, 7, 7), (2, 16, 5, 5), (2, 32, 3, 3), (2, 144), (2, 6))
    # zero input: every layer passes its bias through
    P = orf.cnn_unpack(p)
    assert np.allclose(a1[0, :, 3, 3], np.maximum(P["b1"], 0))


def test_fc1_reads_conv3_in_channel_row_column_order():
    L = orf.cnn_layout()
    p = np.zeros(L["total"])
    P = orf.cnn_unpack(p)
    # a3 channel 5 at (row 2, column 1) only, unit chain up to there: W4 column 5*9 + 2*3 + 1
    x = np.zeros((1, 162))
    # ToT channel, input pixel (row 5, column 4): each centre tap moves it one
    # row and column up, to a1 (4, 3), a2 (3, 2), a3 (2, 1)
    x[0, 5 * 9 + 4] = 1.0
    P["w1"][0, 0, 1, 1] = 1.0
    P["w2"][0, 0, 1, 1] = 1.0
    P["w3"][5, 0, 1, 1] = 1.0
    P["w4"][7, 5 * 9 + 2 * 3 + 1] = 2.0
    P["w5"][0, 7] = 3.0
    out = orf.cnn_forward(p, x)
    assert out[0, 0] == 6.0 and np.count_nonzero(out) == 1


def test_cnn_backward_matches_finite_differences():
    rng = np.random.default_rng(4)
    L = orf.cnn_layout()
    p = rng.normal(size=L["total"]) * 0.2
    x = rng.normal(size=(4, 162))
    y = np.c_[rng.integers(1, 3, 4), rng.normal(size=(4, 4))]
    g = orf.cnn_grad(p, x, y, 0.7)
    idx = np.r_[rng.choice(L["total"], 30, replace=False), L["b1"][0], L["b5"][0] + 5, L["w1"][0]]
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (orf.cnn_loss(p + e, x, y, 0.7) - orf.cnn_loss(p - e, x, y, 0.7)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_cnn_inference_precision_on_bf16_exact_values():
    rng = np.random.default_rng(5)
    L = orf.cnn_layout()
    # weights and inputs on a coarse dyadic grid: exact in bf16; ReLU outputs
    # stay exact as long as sums stay on the grid (small integers / 8)
    p = rng.integers(-2, 3, size=L["total"]).astype(np.float64) / 8
    x = rng.integers(0, 3, size=(3, 162)).astype(np.float64) / 4
    P = orf.cnn_unpack(p)
    for k in ("w2", "w3", "w4", "w5"):
        P[k][...] = 0.0
    for k in ("w2", "w3"):
        P[k][:, :, 1, 1] = np.eye(P[k].shape[0], P[k].shape[1]) if P[k].shape[0] == P[k].shape[1] else np.eye(*P[k].shape[:2])
    P["w4"][:, :8] = 0.125
    P["w5"][:, :4] = 0.25
    assert np.array_equal(orf.cnn_forward_bf16(p, x), orf.cnn_forward(p, x))
