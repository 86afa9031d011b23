"""Timewalk calibration (Sec. IV.C, Eq. 1).

Dim pixels cross threshold late, so a pixel's measured ToF depends on its
ToT. The calibration takes a narrow ToF slice around one ion peak, finds per
ToT value the centre of the ToF distribution by a Gaussian fit, and fits
Eq. 1,  dToF(ToT) = a / (ToT + b)^d + c,  to those centres. The correction
subtracts a / (ToT + b)^d -- the shift of each ToT slice relative to the
bright-pixel asymptote c -- so every slice lines up with the brightest ones.

The data-parallel part, the ToT-ToF joint histogram of all hits in the
slice, runs on the GPU (`tpx_tot_tof_histogram`); the fits work on the
1024 x (bins) histogram on the host. The result is the int16 table of
`tpx_config.d_timewalk_lut` (ticks, indexed by ToT, rounded half away from
zero), which the fused and general paths subtract after the background cut.
"""
from __future__ import annotations

import dataclasses

import numpy as np

N_TOT = 1024


def _gauss(x, amp, mu, sigma):
    return amp * np.exp(-0.5 * ((x - mu) / sigma) ** 2)


def model(tot, a, b, c, d):
    """Eq. 1: the ToF centre of pixels with time over threshold `tot`."""
    return a / np.power(np.asarray(tot, dtype=float) + b, d) + c


@dataclasses.dataclass
class Fit:
    a: float
    b: float
    c: float
    d: float
    tots: np.ndarray        # ToT values whose centre entered the fit
    centres: np.ndarray     # their ToF centres (ticks)
    errors: np.ndarray      # standard errors of the centres (ticks)
    rms: float              # weighted rms residual of Eq. 1 (ticks)

    def shift(self, tot) -> np.ndarray:
        """a / (ToT + b)^d in ticks: what the table subtracts."""
        t = np.asarray(tot, dtype=float) + self.b
        return self.a / np.power(np.maximum(t, 1e-9), self.d)

    def lut(self) -> np.ndarray:
        """The int16 timewalk table (ticks; ToT values below the fitted range
        take the value of the smallest fitted ToT)."""
        tot = np.arange(N_TOT, dtype=float)
        tot = np.maximum(tot, float(self.tots.min()))
        v = self.shift(tot)
        r = np.sign(v) * np.floor(np.abs(v) + 0.5)
        return np.clip(r, -32768, 32767).astype(np.int16)


def gaussian_centres(hist: np.ndarray, tof_lo: int, bin_ticks: int, min_counts: int = 40):
    """Per ToT row with at least `min_counts` counts: the centre of a
    least-squares Gaussian fit to the row's ToF distribution (Poisson
    weights), and its standard error. Returns (tots, centres, errors)."""
    from scipy.optimize import curve_fit
    hist = np.asarray(hist, dtype=float).reshape(N_TOT, -1)
    nb = hist.shape[1]
    x = tof_lo + (np.arange(nb) + 0.5) * bin_ticks
    tots, mus, errs = [], [], []
    for tot in range(N_TOT):
        y = hist[tot]
        n = y.sum()
        if n < min_counts:
            continue
        m0 = float((x * y).sum() / n)
        s0 = float(np.sqrt(((x - m0) ** 2 * y).sum() / n)) or float(bin_ticks)
        try:
            p, cov = curve_fit(_gauss, x, y, p0=[y.max(), m0, max(s0, 0.5 * bin_ticks)],
                               sigma=np.sqrt(np.maximum(y, 1.0)), maxfev=4000)
        except (RuntimeError, ValueError):
            continue
        if not np.all(np.isfinite(cov)) or not (x[0] <= p[1] <= x[-1]):
            continue
        tots.append(tot)
        mus.append(p[1])
        errs.append(max(float(np.sqrt(cov[1, 1])), 1e-3))
    return np.array(tots, dtype=float), np.array(mus), np.array(errs)


def fit_eq1(tots: np.ndarray, centres: np.ndarray, errors: np.ndarray, fix_d: bool = False) -> Fit:
    """Weighted least-squares fit of Eq. 1 to the ToT centres (d fixed to 1
    when `fix_d`, as the paper allows when d comes out close to 1)."""
    from scipy.optimize import curve_fit
    tots = np.asarray(tots, dtype=float)
    c0 = float(np.median(centres[tots >= np.percentile(tots, 75)]))
    a0 = max(float((centres[0] - c0) * (tots[0] + 1.0)), 1e-3)
    lo_b = -float(tots.min()) + 1e-3
    if fix_d:
        f = lambda t, a, b, c: model(t, a, b, c, 1.0)   # noqa: E731
        p, _ = curve_fit(f, tots, centres, p0=[a0, 1.0, c0], sigma=errors,
                         bounds=([0.0, lo_b, -np.inf], [np.inf, 1e4, np.inf]), maxfev=20000)
        a, b, c, d = p[0], p[1], p[2], 1.0
    else:
        p, _ = curve_fit(model, tots, centres, p0=[a0, 1.0, c0, 1.0], sigma=errors,
                         bounds=([0.0, lo_b, -np.inf, 0.2], [np.inf, 1e4, np.inf, 5.0]), maxfev=20000)
        a, b, c, d = p
    res = (centres - model(tots, a, b, c, d)) / errors
    return Fit(float(a), float(b), float(c), float(d), tots, np.asarray(centres), np.asarray(errors),
               float(np.sqrt(np.mean(res ** 2))))


def calibrate(ctx, hits: dict, n_hits: int, tof_lo: int, tof_bin: int, n_bins: int,
              min_counts: int = 40, fix_d: bool = False) -> tuple[Fit, np.ndarray]:
    """The whole calibration on decoded hits (a context without a timewalk
    table): the GPU histogram of the ToF slice, then the two fits. Returns
    the fit and the histogram (1024 x n_bins, host)."""
    import torch
    d_hist = ctx.tpx_tot_tof_histogram(hits, n_hits, tof_lo, tof_bin, n_bins)
    torch.cuda.synchronize()
    hist = d_hist.cpu().numpy().view(np.uint32).reshape(N_TOT, n_bins)
    tots, mus, errs = gaussian_centres(hist, tof_lo, tof_bin, min_counts)
    if tots.size < 4:
        raise ValueError("too few ToT values with enough counts in the ToF slice")
    return fit_eq1(tots, mus, errs, fix_d), hist
