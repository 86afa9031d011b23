"""Timewalk calibration, the oracle side (test infrastructure: only tests/,
the smoke check and the CPU baseline of bench.py use it).

Plain, slow and independent of the CUDA path and of its host fitting code,
following Sec. IV.C in its order:
  1. the ToT-ToF joint histogram of the kept pixels inside a narrow ToF
     slice around one ion peak (np.add.at over the oracle's own decode);
  2. per ToT value, the centre of the ToF distribution: a Gaussian is a
     parabola in log(counts), so the centre is the vertex of a weighted
     quadratic fit to the logarithm of the bins around the maximum;
  3. Eq. 1,  dToF(ToT) = a / (ToT + b)^d + c,  fitted to the centres: for
     fixed (b, d) the model is linear in (a, c), solved by weighted linear
     least squares; (b, d) by a coarse grid search refined twice around the
     best point.
"""
from __future__ import annotations

import numpy as np

from . import run as _run, Config as _Config

N_TOT = 1024


def histogram(packets: np.ndarray, tof_lo: int, tof_bin: int, n_bins: int, cfg: _Config | None = None) -> np.ndarray:
    """Step 1: counts of kept pixels by (ToT, ToF bin) inside the slice
    [tof_lo, tof_lo + n_bins * tof_bin) ticks (no timewalk table)."""
    r = _run(packets, cfg or _Config(), want_info=True)
    info = r["info"]
    kept = r["labels"] >= 0
    tof = info["tof"][kept].astype(np.int64)
    tot = info["tot"][kept].astype(np.int64)
    d = tof - tof_lo
    ok = (d >= 0) & (d < n_bins * tof_bin)
    h = np.zeros((N_TOT, n_bins), dtype=np.int64)
    np.add.at(h, (tot[ok], d[ok] // tof_bin), 1)
    return h


def centre(counts: np.ndarray, x: np.ndarray, half_width: int = 3):
    """Step 2 for one ToT row: vertex of the weighted quadratic fit to
    log(counts) over the bins within `half_width` of the maximum (weights =
    counts, the inverse variance of log counts). None if it cannot be
    formed (fewer than 3 non-empty bins, or no maximum)."""
    k = int(np.argmax(counts))
    lo, hi = max(0, k - half_width), min(counts.size, k + half_width + 1)
    y, xx = counts[lo:hi].astype(float), x[lo:hi].astype(float)
    m = y > 0
    if m.sum() < 3:
        return None
    A = np.stack([xx[m] ** 2, xx[m], np.ones(m.sum())], axis=1)
    w = np.sqrt(y[m])
    coef, *_ = np.linalg.lstsq(A * w[:, None], np.log(y[m]) * w, rcond=None)
    if coef[0] >= 0:
        return None
    return -coef[1] / (2.0 * coef[0])


def centres(hist: np.ndarray, tof_lo: int, tof_bin: int, min_counts: int = 40):
    """Step 2 for every ToT row with enough counts: (tots, centres, weights)
    with weights = counts (the centre's variance falls like 1/counts)."""
    nb = hist.shape[1]
    x = tof_lo + (np.arange(nb) + 0.5) * tof_bin
    t, c, w = [], [], []
    for tot in range(hist.shape[0]):
        n = hist[tot].sum()
        if n < min_counts:
            continue
        v = centre(hist[tot], x)
        if v is None:
            continue
        t.append(tot)
        c.append(v)
        w.append(float(n))
    return np.array(t, dtype=float), np.array(c), np.array(w)


def _linear(tots, cen, w, b, d):
    """Best (a, c) and the weighted squared residual for fixed (b, d)."""
    g = 1.0 / np.power(tots + b, d)
    A = np.stack([g, np.ones_like(g)], axis=1)
    sw = np.sqrt(w)
    (a, c), *_ = np.linalg.lstsq(A * sw[:, None], cen * sw, rcond=None)
    r = cen - (a * g + c)
    return a, c, float((w * r * r).sum())


def fit_eq1(tots, cen, w, fix_d: bool = False):
    """Step 3: (a, b, c, d) minimising the weighted squared residual."""
    tots = np.asarray(tots, dtype=float)
    b_lo = -tots.min() + 1e-3
    bs = np.linspace(b_lo, b_lo + 200.0, 201)
    ds = np.array([1.0]) if fix_d else np.linspace(0.3, 3.0, 55)
    best = None
    for _ in range(3):
        for b in bs:
            for d in ds:
                a, c, e = _linear(tots, cen, w, b, d)
                if best is None or e < best[4]:
                    best = (a, b, c, d, e)
        _, b0, _, d0, _ = best
        sb = (bs[1] - bs[0]) if bs.size > 1 else 1.0
        bs = np.linspace(max(b_lo, b0 - 2 * sb), b0 + 2 * sb, 41)
        if not fix_d:
            sd = ds[1] - ds[0]
            ds = np.linspace(max(0.05, d0 - 2 * sd), d0 + 2 * sd, 41)
    a, b, c, d, _ = best
    return float(a), float(b), float(c), float(d)
