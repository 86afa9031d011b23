"""Timewalk calibration on the GPU (Sec. IV.C, Eq. 1): the ToT-ToF histogram
kernel bit-exact against the oracle's histogram, the whole calibration
recovering the generator's delay model and agreeing with the oracle's fit,
and the resulting table flattening the ToT-ToF correlation when the fused
path applies it."""
import numpy as np
import pytest

import oracle.timewalk as otw
import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import to_device
from paper_2603_04942_gb300 import timewalk as tw

pytestmark = pytest.mark.gpu

TICK = 1.5625
LO, NB = synth.CALIBRATION_TOF_TICKS - 10, 128


@pytest.fixture(scope="module")
def calib():
    p = synth.calibration(n_shots=800)
    return p, synth.generate(p)[0]


def _decode(ctx, pk):
    dec = ctx.tpx_decode(to_device(pk))
    rc, _ = ctx.tpx_sync(check=False)
    assert rc == 0
    return dec["hits"], int(dec["n_hits"].item())


def test_histogram_kernel_matches_the_oracle(calib):
    _, pk = calib
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        hits, nh = _decode(ctx, pk)
        h = ctx.tpx_tot_tof_histogram(hits, nh, LO, 1, NB)
        h = ctx.tpx_tot_tof_histogram(hits, nh, LO, 1, NB, hist=h)   # calls accumulate
        g = h.cpu().numpy().view(np.uint32).reshape(1024, NB).astype(np.int64)
        o = otw.histogram(pk, LO, 1, NB)
        assert np.array_equal(g, 2 * o)
        # wider bins and an offset window
        h2 = ctx.tpx_tot_tof_histogram(hits, nh, LO + 7, 3, 20)
        g2 = h2.cpu().numpy().view(np.uint32).reshape(1024, 20).astype(np.int64)
        assert np.array_equal(g2, otw.histogram(pk, LO + 7, 3, 20))
    finally:
        ctx.close()


def test_calibration_recovers_the_delay_model_and_flattens_the_correlation(calib):
    import torch
    p, pk = calib
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        hits, nh = _decode(ctx, pk)
        fit, hist = tw.calibrate(ctx, hits, nh, LO, 1, NB, fix_d=True)
    finally:
        ctx.close()
    a_true, c_true = p.timewalk_a / TICK, synth.CALIBRATION_TOF_TICKS + p.timewalk_c / TICK
    assert abs(fit.a - a_true) / a_true < 0.1 and abs(fit.b - p.timewalk_b) < 2.0 and abs(fit.c - c_true) < 1.0
    oa, ob, oc, _ = otw.fit_eq1(*otw.centres(otw.histogram(pk, LO, 1, NB), LO, 1), fix_d=True)
    assert abs(fit.a - oa) / oa < 0.05 and abs(fit.c - oc) < 0.5
    before = np.ptp(fit.centres)
    # apply the table and look again: every ToT slice lines up
    lut = torch.from_numpy(fit.lut()).cuda()
    ctx2 = tpx.Context(tpx.Config(timewalk_lut=lut), max_packets=pk.size)
    try:
        hits2, nh2 = _decode(ctx2, pk)
        h2 = ctx2.tpx_tot_tof_histogram(hits2, nh2, LO - 40, 1, NB).cpu().numpy().view(np.uint32).reshape(1024, NB)
        t2, c2, _ = tw.gaussian_centres(h2, LO - 40, 1)
        # the fused path with the table: records' ToF near the true peak
        out = ctx2.process(to_device(pk), cluster_capacity=pk.size, trig_capacity=pk.size)
    finally:
        ctx2.close()
    # before: the slices spread over > 40 ticks; after: only the rounding of
    # the generator's delay and of the table (half a tick each) and fit noise
    assert before > 40.0
    assert np.std(c2) < 0.7 and np.ptp(c2) < 4.0
    assert abs(np.median(c2) - (synth.CALIBRATION_TOF_TICKS + p.timewalk_c / TICK)) < 1.0
    tof = out["clusters"]["tof"]
    assert np.abs(np.median(tof) - (synth.CALIBRATION_TOF_TICKS + p.timewalk_c / TICK)) < 1.0
