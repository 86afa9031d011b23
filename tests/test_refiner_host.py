"""Host-side parts of the learned refiner on the CPU: the matching of the
generator's particles to clusters (on the oracle's clusters of a refiner
recipe), the error summary against hand-made hits, and the pairwise-distance
histogram of the hits of each shot."""
import numpy as np

import oracle.refiner as orf
import synth
from paper_2603_04942_gb300 import refiner as R


def test_truth_matching_on_oracle_clusters():
    p = synth.refiner(n_shots=120)
    pk, truth, _ = synth.generate(p)
    _, sel, centre, r = orf.patches(pk)
    cl = r["clusters"]
    count, pos, sep, ok = R._truth_match(cl, truth, sel, centre, p.t_start_ticks, p.shot_begin, p.trig_period_ticks)
    assert ok.mean() > 0.98
    # every particle belongs to exactly one cluster: the counts add up
    assert count.sum() <= truth["shot"].size
    # merged pairs: two particles, the brighter first, separation from the truth
    two = ok & (count == 2)
    assert two.sum() > 0.2 * ok.sum()
    assert np.allclose(sep[two], np.hypot(pos[two, 0] - pos[two, 2], pos[two, 1] - pos[two, 3]))
    # single particles: the plain centroid sits on the particle (Sec. V.C)
    one = ok & (count == 1)
    c = cl[sel[one]]
    assert np.median(np.hypot(c["x"] - pos[one, 0], c["y"] - pos[one, 1])) < 0.05


class _DS:
    """A minimal stand-in for a Dataset: two single particles, two pairs."""
    count = np.array([1, 1, 2, 2])
    pos = np.array([[10.0, 10.0, 0, 0], [20.0, 20.0, 0, 0], [30.0, 30.0, 32.0, 30.0], [40.0, 40.0, 40.5, 40.0]])
    centroid = np.array([[10.1, 10.0], [20.0, 20.2], [31.0, 30.0], [40.25, 40.0]])
    sep = np.array([0.0, 0.0, 2.0, 0.5])


def test_evaluate_against_hand_made_hits():
    hits = np.array([[1, 10.1, 10.0, 0, 0],            # single kept as one
                     [2, 20.0, 20.5, 20.0, 19.5],       # single split in two
                     [2, 30.1, 30.0, 31.9, 30.0],       # pair resolved
                     [0, 40.25, 40.0, 0, 0]], float)    # pair left to the centroid
    ev = R.evaluate(_DS(), hits)
    assert ev["singles"] == 2 and ev["pairs"] == 2
    assert ev["pair_recall"] == 0.5 and ev["single_split"] == 0.5 and ev["fallback"] == 0.25
    assert abs(ev["single_err_centroid"] - 0.15) < 1e-12
    assert abs(ev["single_err_refined"] - (0.1 + 0.5) / 2) < 1e-12
    assert abs(ev["pair_err_refined"] - (0.1 + 0.1 + 0.25 + 0.25) / 4) < 1e-12
    assert abs(ev["pair_err_centroid"] - (1.0 + 1.0 + 0.25 + 0.25) / 4) < 1e-12
    rs = {tuple(b["sep"]): b for b in ev["resolving"]}
    assert rs[(2, 3)]["pairs"] == 1 and rs[(2, 3)]["resolved_refined"] == 1.0
    assert rs[(0, 1)]["pairs"] == 1 and rs[(0, 1)]["resolved_refined"] == 0.0


def test_pair_distance_histogram_by_brute_force():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0, 20, 60), rng.uniform(0, 20, 60)
    shot = rng.integers(0, 3, 60)
    h = R.pair_distance_histogram(x, y, shot, 4.0, 0.5)
    want = np.zeros(8, int)
    for i in range(60):
        for j in range(i + 1, 60):
            d = np.hypot(x[i] - x[j], y[i] - y[j])
            if shot[i] == shot[j] and d <= 4.0:
                want[min(int(d // 0.5), 7)] += 1
    assert np.array_equal(h, want)
