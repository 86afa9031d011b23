"""The learned overlap refiner, oracle side (test infrastructure: only tests/,
the smoke check and the CPU baseline of bench.py use it).

The paper has no learned stage; its multi-hit discussion (Sec. VII.B) and the
local-maximum count of Sec. V.B motivate one: a cluster may hold two
particles, and a small network looking at the cluster's pixels can say how
many and where. This file is the plain definition the CUDA path is checked
against, in float64 (the patch values in float32, the precision the CUDA
path feeds the network):

  patch   : for a CC-mode cluster with more than `min_pixels` pixels, a
            9 x 9 window centred on the centroid rounded half up (the earliest
            pixel when the cluster has no charge). Channel 0 holds ToT / 1023
            rounded to bfloat16, channel 1 the pixel time minus the earliest
            pixel's time, in units of 32 ticks, clamped to [-8, 8], rounded to
            float16 (the patch precisions); empty cells hold 0. When two
            packets fall on one cell, the larger ToT wins, then the later
            packet.
  network : 162 inputs -> H -> H -> 6, ReLU after the two hidden layers;
            outputs two logits (one, two particles) and (dx, dy) of the first
            and of the second particle in pixels from the patch centre.
  loss    : mean over the minibatch of the softmax cross-entropy of the count
            plus w * 1/2 * sum of squared errors of the offsets of the
            particles that exist (the first always, the second in pairs).
  Adam    : Kingma and Ba (2015), beta1 0.9, beta2 0.999, eps 1e-8.
  infer   : the same network at the inference precision: inputs and
            weights rounded to bfloat16, each hidden activation rounded to
            bfloat16 after its ReLU, sums and biases wider.
  decide  : two particles at the network's positions when that count's
            probability reaches the threshold; else the plain centroid
            (Sec. V.C), flagged 1 when the probability of one particle
            reaches the threshold and 0 when neither does.

Parity pins (tests/test_refiner_pins.py): a hand-built patch, the closed
forms of the cross-entropy and of Adam's first step, a hand-evaluated
one-unit network, positive homogeneity of the bias-free ReLU network, the
backward pass against central finite differences of the loss, and the
inference precision equal to the plain network on bf16-exact values and
rounding a hand-made activation tie to even.
"""
from __future__ import annotations

import numpy as np

from . import run as _run, Config as _Config, MODE_CC

PS = 9
PC = PS * PS
NIN = 2 * PC
NOUT = 6


# ---------------------------------------------------------------- patches
def bf16(v) -> np.float32:
    """A float32 rounded to bfloat16 (its upper 16 bits), to nearest, ties
    to even; returned widened to float32. (Finite inputs only.)"""
    u = int(np.float32(v).view(np.uint32))
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return np.uint32(u).view(np.float32)


def patches(packets: np.ndarray, min_pixels: int = 12, cfg: _Config | None = None, idx_base: int = 0):
    """(patches float32 [n x 162], record index [n], centre int32 [n x 2],
    oracle result) for the clusters with more than `min_pixels` pixels."""
    cfg = cfg or _Config()
    assert cfg.mode == MODE_CC
    r = _run(packets, cfg, idx_base=idx_base, want_info=True)
    cl, labels, info = r["clusters"], r["labels"], r["info"]
    sel = np.nonzero(cl["n"] > min_pixels)[0]
    out = np.zeros((sel.size, NIN), np.float32)
    centre = np.zeros((sel.size, 2), np.int32)
    members = {}
    for q in np.nonzero(labels >= 0)[0]:
        members.setdefault(int(labels[q]), []).append(int(q))
    for s, i in enumerate(sel):
        c = cl[i]
        root = int(c["label"]) - idx_base
        if c["s_tot"] > 0:
            cx = (2 * int(c["s_x"]) + int(c["s_tot"])) // (2 * int(c["s_tot"]))
            cy = (2 * int(c["s_y"]) + int(c["s_tot"])) // (2 * int(c["s_tot"]))
        else:
            cx, cy = int(info["x"][root]), int(info["y"][root])
        centre[s] = (cx, cy)
        best = {}
        for q in members.get(int(c["label"]), []):
            dx, dy = int(info["x"][q]) - cx + PS // 2, int(info["y"][q]) - cy + PS // 2
            if not (0 <= dx < PS and 0 <= dy < PS):
                continue
            key = (int(info["tot"][q]), q)
            if (dy, dx) not in best or key > best[(dy, dx)]:
                best[(dy, dx)] = key
        for (dy, dx), (tot, q) in best.items():
            cell = dy * PS + dx
            d = int(info["t"][q]) - int(info["t"][root])
            out[s, cell] = bf16(np.float32(tot) / np.float32(1023))
            out[s, PC + cell] = np.float16(min(8.0, max(-8.0, float(np.float32(d) / np.float32(32)))))
    return out, sel, centre, r


# ---------------------------------------------------------------- network
def layout(h: int) -> dict:
    """Offsets of W1 [162 x h], b1, W2 [h x h], b2, W3 [h x 6], b3 in the
    flat parameter vector, and its length."""
    o, d = 0, {}
    for name, size in (("w1", NIN * h), ("b1", h), ("w2", h * h), ("b2", h), ("w3", h * NOUT), ("b3", NOUT)):
        d[name] = (o, size)
        o += size
    d["total"] = o
    return d


def unpack(p: np.ndarray, h: int):
    L = layout(h)
    g = lambda k, shape: p[L[k][0]: L[k][0] + L[k][1]].reshape(shape)   # noqa: E731
    return g("w1", (NIN, h)), g("b1", (h,)), g("w2", (h, h)), g("b2", (h,)), g("w3", (h, NOUT)), g("b3", (NOUT,))


def forward(p: np.ndarray, h: int, x: np.ndarray, keep: bool = False):
    w1, b1, w2, b2, w3, b3 = unpack(np.asarray(p, np.float64), h)
    x = np.asarray(x, np.float64)
    a1 = np.maximum(x @ w1 + b1, 0.0)
    a2 = np.maximum(a1 @ w2 + b2, 0.0)
    out = a2 @ w3 + b3
    return (out, a1, a2) if keep else out


def bf16_array(a) -> np.ndarray:
    """Elementwise bf16 rounding (as `bf16`) of a float32 array."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def forward_bf16(p: np.ndarray, h: int, x: np.ndarray) -> np.ndarray:
    """The inference precision: inputs and weights rounded to bf16, sums
    exact (float64 here), biases in float32, each hidden activation rounded
    to bf16 after its ReLU."""
    w1, b1, w2, b2, w3, b3 = unpack(np.asarray(p, np.float32), h)
    r = lambda a: bf16_array(a).astype(np.float64)              # noqa: E731
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)  # noqa: E731
    a1 = r(np.maximum(r(x) @ r(w1) + f(b1), 0.0).astype(np.float32))
    a2 = r(np.maximum(a1 @ r(w2) + f(b2), 0.0).astype(np.float32))
    return a2 @ r(w3) + f(b3)


def loss(p: np.ndarray, h: int, x: np.ndarray, y: np.ndarray, w_off: float) -> float:
    """The minibatch loss of the module docstring (y rows: count, dx1, dy1,
    dx2, dy2)."""
    out = forward(p, h, x)
    y = np.asarray(y, np.float64)
    two = y[:, 0] > 1.5
    z = np.logaddexp(out[:, 0], out[:, 1])
    ce = z - np.where(two, out[:, 1], out[:, 0])
    used = np.stack([np.ones_like(two), np.ones_like(two), two, two], axis=1)
    se = (((out[:, 2:] - y[:, 1:]) ** 2) * used).sum(axis=1)
    return float(np.mean(ce + 0.5 * w_off * se))


def grad(p: np.ndarray, h: int, x: np.ndarray, y: np.ndarray, w_off: float) -> np.ndarray:
    """d loss / d p by the chain rule, layer by layer."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = x.shape[0]
    w1, b1, w2, b2, w3, b3 = unpack(np.asarray(p, np.float64), h)
    out, a1, a2 = forward(p, h, x, keep=True)
    two = y[:, 0] > 1.5
    p2 = 1.0 / (1.0 + np.exp(out[:, 0] - out[:, 1]))
    dout = np.zeros_like(out)
    dout[:, 0] = (1.0 - p2) - (~two)
    dout[:, 1] = p2 - two
    used = np.stack([np.ones_like(two), np.ones_like(two), two, two], axis=1)
    dout[:, 2:] = w_off * (out[:, 2:] - y[:, 1:]) * used
    dout /= n
    g3, gb3 = a2.T @ dout, dout.sum(0)
    d2 = (dout @ w3.T) * (a2 > 0)
    g2, gb2 = a1.T @ d2, d2.sum(0)
    d1 = (d2 @ w2.T) * (a1 > 0)
    g1, gb1 = x.T @ d1, d1.sum(0)
    return np.concatenate([g1.ravel(), gb1, g2.ravel(), gb2, g3.ravel(), gb3])


def adam(p, m, v, g, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update; returns new (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def decide(out: np.ndarray, centre: np.ndarray, centroid_xy: np.ndarray, threshold: float) -> np.ndarray:
    """Rows (k, x1, y1, x2, y2) as the module docstring states. The count
    is decided in float32 on the logit margin: p(two) >= thr exactly when
    o1 - o0 >= log(thr / (1 - thr)); positions are float32 sums."""
    o = np.asarray(out, np.float32)
    margin = o[:, 1] - o[:, 0]
    thr = float(np.float32(threshold))          # the threshold is a float32 argument
    lt = np.float32(np.log(thr / (1.0 - thr)))
    res = np.zeros((o.shape[0], 5), np.float32)
    for s in range(o.shape[0]):
        cx, cy = np.float32(centre[s][0]), np.float32(centre[s][1])
        if margin[s] >= lt:
            res[s] = (2, cx + o[s, 2], cy + o[s, 3], cx + o[s, 4], cy + o[s, 5])
        else:
            res[s] = (1 if -margin[s] >= lt else 0, np.float32(centroid_xy[s][0]), np.float32(centroid_xy[s][1]), 0, 0)
    return res


# ---------------------------------------------------------------- CNN
# The convolutional refiner: the same patch, count and offsets, through three
# 3 x 3 convolutions without padding and two dense layers:
#   input  2 x 9 x 9 (ToT, ToA)
#   conv1  2 -> 16 channels, 7 x 7, ReLU
#   conv2 16 -> 16 channels, 5 x 5, ReLU
#   conv3 16 -> 32 channels, 3 x 3, ReLU
#   fc1   288 (conv3 flattened channel, row, column) -> 144, ReLU
#   fc2   144 -> 6
# A convolution here is the plain cross-correlation
#   out[co, y, x] = b[co] + sum_{ci, ky, kx} W[co, ci, ky, kx] in[ci, y + ky, x + kx].
# Parameters, flat: W1 [16, 2, 3, 3], b1, W2 [16, 16, 3, 3], b2, W3 [32, 16, 3, 3],
# b3, W4 [144, 288], b4, W5 [6, 144], b5 (49,750 floats).
CNN_SHAPES = (("w1", (16, 2, 3, 3)), ("b1", (16,)), ("w2", (16, 16, 3, 3)), ("b2", (16,)),
              ("w3", (32, 16, 3, 3)), ("b3", (32,)), ("w4", (144, 288)), ("b4", (144,)),
              ("w5", (NOUT, 144)), ("b5", (NOUT,)))


def cnn_layout() -> dict:
    o, d = 0, {}
    for name, shape in CNN_SHAPES:
        size = int(np.prod(shape))
        d[name] = (o, size, shape)
        o += size
    d["total"] = o
    return d


def cnn_unpack(p: np.ndarray) -> dict:
    L = cnn_layout()
    return {k: p[L[k][0]: L[k][0] + L[k][1]].reshape(L[k][2]) for k, _ in CNN_SHAPES}


def conv2d(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [n, ci, h, w], w [co, ci, 3, 3] -> [n, co, h - 2, w - 2], the sum
    written out over the nine kernel taps."""
    n, ci, h, wd = x.shape
    co = w.shape[0]
    out = np.zeros((n, co, h - 2, wd - 2), np.float64) + b.reshape(1, co, 1, 1)
    for ky in range(3):
        for kx in range(3):
            patch = x[:, :, ky: ky + h - 2, kx: kx + wd - 2]          # [n, ci, h-2, w-2]
            out += np.einsum("nchw,oc->nohw", patch, w[:, :, ky, kx])
    return out


def conv2d_back(x: np.ndarray, w: np.ndarray, d: np.ndarray):
    """Gradients of conv2d given d = d loss / d out: (d x, d w, d b)."""
    n, ci, h, wd = x.shape
    dx = np.zeros_like(x, dtype=np.float64)
    dw = np.zeros_like(w, dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            patch = x[:, :, ky: ky + h - 2, kx: kx + wd - 2]
            dw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", d, patch)
            dx[:, :, ky: ky + h - 2, kx: kx + wd - 2] += np.einsum("nohw,oc->nchw", d, w[:, :, ky, kx])
    return dx, dw, d.sum(axis=(0, 2, 3))


def cnn_forward(p: np.ndarray, x: np.ndarray, keep: bool = False, act=None):
    """The CNN in float64; `act` (optional) maps every hidden activation after
    its ReLU (the inference precision passes bf16 rounding)."""
    P = cnn_unpack(np.asarray(p, np.float64))
    a0 = np.asarray(x, np.float64).reshape(-1, 2, PS, PS)
    f = act or (lambda a: a)
    a1 = f(np.maximum(conv2d(a0, P["w1"], P["b1"]), 0.0))
    a2 = f(np.maximum(conv2d(a1, P["w2"], P["b2"]), 0.0))
    a3 = f(np.maximum(conv2d(a2, P["w3"], P["b3"]), 0.0))
    h3 = a3.reshape(a3.shape[0], -1)                                  # (channel, row, column)
    a4 = f(np.maximum(h3 @ P["w4"].T + P["b4"], 0.0))
    out = a4 @ P["w5"].T + P["b5"]
    return (out, (a0, a1, a2, a3, a4)) if keep else out


def cnn_forward_bf16(p: np.ndarray, x: np.ndarray) -> np.ndarray:
    """The inference precision: inputs and weights rounded to bf16 (biases
    float32), sums exact, every hidden activation rounded to bf16 after its
    ReLU; the outputs unrounded."""
    p32 = np.asarray(p, np.float32)
    L = cnn_layout()
    q = p32.copy()
    for k, _ in CNN_SHAPES:
        if k.startswith("w"):
            o, size, _ = L[k]
            q[o: o + size] = bf16_array(p32[o: o + size])
    r = lambda a: bf16_array(np.asarray(a, np.float32)).astype(np.float64)   # noqa: E731
    return cnn_forward(q.astype(np.float64), r(x), act=r)


def cnn_loss(p: np.ndarray, x: np.ndarray, y: np.ndarray, w_off: float) -> float:
    out = cnn_forward(p, x)
    y = np.asarray(y, np.float64)
    two = y[:, 0] > 1.5
    z = np.logaddexp(out[:, 0], out[:, 1])
    ce = z - np.where(two, out[:, 1], out[:, 0])
    used = np.stack([np.ones_like(two), np.ones_like(two), two, two], axis=1)
    se = (((out[:, 2:] - y[:, 1:]) ** 2) * used).sum(axis=1)
    return float(np.mean(ce + 0.5 * w_off * se))


def cnn_grad(p: np.ndarray, x: np.ndarray, y: np.ndarray, w_off: float) -> np.ndarray:
    """d loss / d p by the chain rule through the five layers."""
    y = np.asarray(y, np.float64)
    P = cnn_unpack(np.asarray(p, np.float64))
    out, (a0, a1, a2, a3, a4) = cnn_forward(p, x, keep=True)
    n = out.shape[0]
    two = y[:, 0] > 1.5
    p2 = 1.0 / (1.0 + np.exp(out[:, 0] - out[:, 1]))
    dout = np.zeros_like(out)
    dout[:, 0] = (1.0 - p2) - (~two)
    dout[:, 1] = p2 - two
    used = np.stack([np.ones_like(two), np.ones_like(two), two, two], axis=1)
    dout[:, 2:] = w_off * (out[:, 2:] - y[:, 1:]) * used
    dout /= n
    g = {}
    g["w5"], g["b5"] = dout.T @ a4, dout.sum(0)
    d4 = (dout @ P["w5"]) * (a4 > 0)
    h3 = a3.reshape(n, -1)
    g["w4"], g["b4"] = d4.T @ h3, d4.sum(0)
    d3 = ((d4 @ P["w4"]).reshape(a3.shape)) * (a3 > 0)
    dx2, g["w3"], g["b3"] = conv2d_back(a2, P["w3"], d3)
    d2 = dx2 * (a2 > 0)
    dx1, g["w2"], g["b2"] = conv2d_back(a1, P["w2"], d2)
    d1 = dx1 * (a1 > 0)
    _, g["w1"], g["b1"] = conv2d_back(a0, P["w1"], d1)
    return np.concatenate([g[k].ravel() for k, _ in CNN_SHAPES])
