"""Generator properties the parity tests rely on (determinism, independent
shot ranges, the planted pixel-wrap straddle, cloud sizes)."""
import numpy as np

import oracle
import synth


def test_deterministic_and_shot_ranges_regenerate():
    p = synth.small(n_shots=60, dark_per_shot=5.0, pair_frac=0.1)
    a = synth.generate(p)[0]
    assert np.array_equal(a, synth.generate(p.replace(n_threads=3))[0])
    b1 = synth.generate(p.replace(n_shots=25))[0]
    b2 = synth.generate(p.replace(shot_begin=25, n_shots=35))[0]
    assert np.array_equal(a, np.concatenate([b1, b2]))


def test_small_config_straddles_a_pixel_wrap():
    p = synth.small(shot_begin=495, n_shots=10)
    pk = synth.generate(p)[0]
    pix = pk[(pk >> np.uint64(60)) == 0xB]
    raw_coarse = ((pix & np.uint64(0xFFFF)) << np.uint64(14)) | ((pix >> np.uint64(30)) & np.uint64(0x3FFF))
    hi = raw_coarse > (1 << 29) + (1 << 28)
    lo = raw_coarse < (1 << 28)
    # both sides of the wrap are present and interleave in stream order
    assert hi.any() and lo.any()
    first_lo = np.argmax(lo)
    assert hi[first_lo:].any()
    r = oracle.run(pk, want_info=True)
    t = r["info"]["t"][r["info"]["type"] == 1]
    assert t.max() - t.min() < 11 * 640_000


def test_cloud_sizes():
    s = synth.Stream(synth.small(n_shots=100))
    assert 23 < s.n_packets / s.n_particles < 27
    s2 = synth.Stream(synth.stated_size(synth.small(n_shots=100)))
    assert 9 < s2.n_packets / s2.n_particles < 13
