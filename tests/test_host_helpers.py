"""Host-side helpers on the CPU: shard cut planning (edge cases) and the
timewalk table's rounding and clamping (Sec. IV.C, Eq. 1)."""
import numpy as np

from paper_2603_04942_gb300 import shard
from paper_2603_04942_gb300 import timewalk as tw


def test_plan_cuts_edge_cases():
    is_tdc = np.zeros(100, bool)
    is_tdc[[0, 10, 50, 90]] = True
    cuts = shard.plan_cuts(is_tdc, 4)
    assert cuts[0] == 0 and cuts[-1] == 100 and cuts == sorted(cuts)
    assert all(is_tdc[c] for c in cuts[1:-1] if c < 100)        # every inner cut is a trigger packet
    assert shard.plan_cuts(is_tdc, 1) == [0, 100]
    # more ranks than triggers: later ranges are empty, never negative
    many = shard.plan_cuts(is_tdc, 16)
    assert len(many) == 17 and many == sorted(many) and many[-1] == 100
    # no trigger at all: everything in the first range
    assert shard.plan_cuts(np.zeros(10, bool), 3) == [0, 10, 10, 10]


def _fit(a, b, d, tots):
    t = np.asarray(tots, float)
    return tw.Fit(a, b, 0.0, d, t, np.zeros_like(t), np.ones_like(t), 0.0)


def test_timewalk_table_rounds_half_away_and_clamps():
    f = _fit(a=10.0, b=0.0, d=1.0, tots=[4, 5, 20])
    lut = f.lut()
    assert lut.dtype == np.int16 and lut.size == 1024
    # 10 / ToT: 2.5 -> 3 (half away from zero), 2.0 -> 2, 0.5 -> 1, ToT below the fitted range
    # takes the smallest fitted ToT's value
    assert lut[4] == 3 and lut[5] == 2 and lut[20] == 1 and lut[0] == lut[4] == 3
    assert lut[21] == 0                                            # 10/21 = 0.476 -> 0
    neg = _fit(a=-10.0, b=0.0, d=1.0, tots=[4, 20]).lut()
    assert neg[4] == -3 and neg[20] == -1                          # -2.5 -> -3, -0.5 -> -1
    big = _fit(a=1e9, b=0.0, d=1.0, tots=[1, 2]).lut()
    assert big[1] == 32767                                         # clamped to int16
    assert np.allclose(f.shift([5, 10]), [2.0, 1.0])
