"""Pins of the oracle's timewalk calibration (Sec. IV.C, Eq. 1): exact
recovery from noise-free model data, the vertex of a sampled Gaussian, the
generator's known delay model recovered from a simulated calibration run,
and the host fitting code of the library agreeing with the oracle."""
import numpy as np
import pytest

import oracle.timewalk as otw
import synth
from paper_2603_04942_gb300 import timewalk as tw

TICK = 1.5625


def test_eq1_fit_recovers_noise_free_parameters():
    tots = np.arange(12, 700, 3, dtype=float)
    a, b, c, d = 120.0, 4.0, 3300.0, 1.15
    cen = a / (tots + b) ** d + c
    fa, fb, fc, fd = otw.fit_eq1(tots, cen, np.ones_like(tots))
    assert abs(fb - b) < 0.02 and abs(fd - d) < 0.002
    assert abs(fa - a) / a < 0.01 and abs(fc - c) < 0.02
    ga, gb, gc, gd = otw.fit_eq1(tots, a / (tots + b) + c, np.ones_like(tots), fix_d=True)
    assert gd == 1.0 and abs(gb - b) < 0.02 and abs(ga - a) / a < 0.005


def test_centre_of_a_sampled_gaussian_is_its_mean():
    x = np.arange(64) + 0.5 + 3000
    for mu in (3020.0, 3031.37, 3044.9):
        counts = 1000.0 * np.exp(-0.5 * ((x - mu) / 2.3) ** 2)
        assert abs(otw.centre(counts, x) - mu) < 1e-6


def test_library_fits_agree_with_the_oracle_on_model_histograms():
    """A noise-free histogram whose rows are Gaussians centred on Eq. 1: the
    library's Gaussian least-squares centres and Eq. 1 fit, and the oracle's
    log-parabola centres and grid fit, both land on the model."""
    lo, nb = 3190, 160
    x = lo + np.arange(nb) + 0.5
    a, b, c = 960.0, 5.0, 3206.4
    h = np.zeros((1024, nb))
    for tot in range(10, 1024, 2):
        h[tot] = 500.0 * np.exp(-0.5 * ((x - (a / (tot + b) + c)) / 2.0) ** 2)
    t1, c1, e1 = tw.gaussian_centres(h, lo, 1)
    f = tw.fit_eq1(t1, c1, e1, fix_d=True)
    t2, c2, w2 = otw.centres(h, lo, 1)
    oa, ob, oc, _ = otw.fit_eq1(t2, c2, w2, fix_d=True)
    for got in ((f.a, f.b, f.c), (oa, ob, oc)):
        assert abs(got[0] - a) / a < 0.02 and abs(got[1] - b) < 0.3 and abs(got[2] - c) < 0.1
    lut = f.lut()
    assert lut.dtype == np.int16 and lut[1023] == round(a / (1023 + b))


@pytest.fixture(scope="module")
def calib():
    p = synth.calibration(n_shots=500)
    pk = synth.generate(p)[0]
    return p, pk


def test_oracle_recovers_the_generators_timewalk(calib):
    p, pk = calib
    lo, nb = synth.CALIBRATION_TOF_TICKS - 10, 128
    h = otw.histogram(pk, lo, 1, nb)
    assert h.sum() > 100_000
    t, cen, w = otw.centres(h, lo, 1)
    a, b, c, d = otw.fit_eq1(t, cen, w, fix_d=True)
    a_true, c_true = p.timewalk_a / TICK, synth.CALIBRATION_TOF_TICKS + p.timewalk_c / TICK
    assert abs(a - a_true) / a_true < 0.1
    assert abs(b - p.timewalk_b) < 2.0
    assert abs(c - c_true) < 1.0
