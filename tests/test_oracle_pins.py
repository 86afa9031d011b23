"""Pins for the CPU oracle: each checks it against something other than
itself -- the paper's printed worked example, closed forms, hand-composed
packets, brute force on tiny inputs, invariants and planted ground truth."""
import os

import numpy as np
import pytest

import oracle
import synth
from streams import StreamBuilder, brute_force, random_dense_stream

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sections(path):
    sec, cur = {}, None
    for line in open(path):
        line = line.split("#")[0].rstrip()
        if not line.strip():
            continue
        if line.startswith("["):
            cur = line[1:line.index("]")]
            sec[cur] = []
        else:
            sec[cur].append([float(v) for v in line.split()])
    return sec


# ---------------------------------------------------------------- Sec. IV.A
def test_wrap_periods_closed_form():
    # 1.5625 ns ticks: 2^34 ticks == 2^42 units of 25/4096 ns == 26.8435456 s
    assert (1 << 34) * 1.5625e-9 == pytest.approx(26.8435456, abs=1e-12)
    assert (1 << 42) * 25 / 4096 * 1e-9 == pytest.approx(26.8435456, abs=1e-12)
    assert (1 << 36) * 1.5625e-9 == pytest.approx(107.3741824, abs=1e-12)
    assert oracle.WRAP_THR_TICKS * 1.5625e-9 == pytest.approx(20.0)
    assert oracle.TOF_MAX_TICKS * 1.5625e-9 == pytest.approx(100e-6)


def _golden_packets():
    rows = []
    for line in open(os.path.join(GOLDEN, "packet_layout.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        lhs, rhs = line.split("|")
        f = lhs.split()
        exp = [int(v) for v in rhs.split()]
        if f[0] == "pixel":
            dcol, spix, pix, toa, tot, ftoa, spidr = (int(v) for v in f[1:])
            w = (0xB << 60) | (dcol << 53) | (spix << 47) | (pix << 44) | (toa << 30) | (tot << 20) | (ftoa << 16) | spidr
            rows.append(("pix", w, tot, exp))
        else:
            counter, coarse = int(f[1]), int(f[2])
            w = (0x6 << 60) | (0xF << 56) | (counter << 44) | (coarse << 9)
            rows.append(("tdc", w, None, exp))
    return rows


def test_packet_layout_golden():
    rows = _golden_packets()
    for kind, w, tot, exp in rows:
        info = oracle.run(np.array([w], np.uint64), want_info=True)["info"][0]
        if kind == "pix":
            assert (info["type"], info["x"], info["y"], info["tot"], info["t"]) == (1, exp[0], exp[1], tot, exp[2])
        else:
            assert (info["type"], info["t"]) == (2, exp[0])


def test_generator_encoder_matches_layout():
    # the generator's encoder is pinned by the same hand-composed table
    for kind, w, tot, exp in _golden_packets():
        if kind == "pix":
            got = synth.encode_pixels([exp[0]], [exp[1]], [tot], [exp[2]])[0]
            info = oracle.run(np.array([got], np.uint64), want_info=True)["info"][0]
            assert (info["x"], info["y"], info["tot"], info["t"]) == (exp[0], exp[1], tot, exp[2])
        else:
            got = synth.encode_tdcs([exp[0]], [0])[0]
            assert oracle.run(np.array([got], np.uint64), want_info=True)["info"][0]["t"] == exp[0]


def test_unknown_headers_are_counted_and_skipped():
    pk = np.array([0x0 << 60, 0x7 << 60 | 5, 0xF << 60], np.uint64)
    r = oracle.run(pk)
    assert r["status"] == 0 and r["counters"]["corrupt"] == 3 and r["clusters"].size == 0
    assert oracle.run(pk, oracle.Config(strict=True))["status"] == -4


def test_unwrap_stragglers_across_pixel_wrap():
    """Sec. IV.A: a pixel reported after a wrap but whose ToA precedes it must
    not take the wrap; the next post-wrap pixel re-advances."""
    P = 1 << 34
    b = StreamBuilder()
    b.tdc(P - 10_000)
    # real steps stay below 20 s and a packet falls in the last 6.8 s before
    # each wrap, as in any dense stream
    true = [P - 5000, P - 4000, P + 100, P - 3000, P + 200, P - 10, P + 300,
            P + 8_000_000_000, P + 16_000_000_000, 2 * P + 5, 2 * P - 7, 2 * P + 9]
    for t in true:
        b.pix(5, 5, 10, t)
    info = oracle.run(b.packets(), want_info=True)["info"]
    assert list(info["t"][1:]) == true


def test_unwrap_tdc_wrap_and_stragglers():
    P = 1 << 36
    b = StreamBuilder()
    step = 12_000_000_000           # below the 20 s threshold
    tt = [P - 4, P + 2, P - 2, P + 6] + [P + 6 + k * step for k in range(1, 6)] + [2 * P + 4]
    for t in tt:
        b.tdc(t)
    r = oracle.run(b.packets(), want_info=True)
    assert list(r["info"]["t"]) == tt
    assert r["status"] == -4   # the straggler makes the trigger list decrease: flagged


def test_unwrap_long_stream_many_wraps():
    """Monotone pixel stream over many wraps; steps below 1.5 s, so a packet
    always falls in the last 6.8 s before each wrap."""
    P = 1 << 34
    rng = np.random.default_rng(7)
    t = np.cumsum(rng.integers(1, 1_000_000_000, size=1000)).astype(np.int64)
    b = StreamBuilder()
    b.tdc(0)
    for v in t:
        b.pix(1, 1, 1, int(v))
    info = oracle.run(b.packets(), oracle.Config(tof_max_ticks=1 << 62), want_info=True)["info"]
    assert np.array_equal(info["t"][1:], t)
    assert t[-1] > 20 * P


# ---------------------------------------------------------------- Sec. IV.B
def test_background_cut_and_pre_trigger_drop():
    b = StreamBuilder()
    b.pix(1, 1, 5, 900)                 # before any trigger: dropped
    b.tdc(1000)
    b.pix(2, 2, 5, 1000 + 64_000)       # ToF == 100 us: kept
    b.pix(3, 3, 5, 1000 + 64_001)       # ToF > 100 us: dropped
    b.pix(4, 4, 5, 1000)                # ToF == 0: kept
    r = oracle.run(b.packets())
    c = r["counters"]
    assert (c["dropped_pre_trigger"], c["dropped_background"], c["kept"]) == (1, 1, 2)
    assert list(r["labels"]) == [-1, -1, 2, -1, 4]


def test_shot_is_most_recent_trigger_in_time():
    """A pixel read out after the next TDC packet but timed before it belongs
    to the earlier trigger (Sec. IV.B: the most recent laser trigger)."""
    b = StreamBuilder()
    b.tdc(1000)
    b.pix(1, 1, 5, 1500)
    b.tdc(2000)
    b.pix(1, 2, 5, 1900)                # late report, earlier time: shot 0, joins (1,1)
    b.pix(9, 9, 5, 2100)
    r = oracle.run(b.packets(), oracle.Config(tof_max_ticks=10_000, dt_ticks=500), want_info=True)
    assert list(r["info"]["shot"]) == [-1, 0, -1, 0, 1]
    assert list(r["labels"]) == [-1, 1, -1, 1, 4]


def test_timewalk_correction_after_cut():
    """Sec. IV.C: the ToT-dependent shift is applied after the background cut
    and moves the time used for clustering and the ToF centroid."""
    lut = np.zeros(1024, np.int16)
    lut[10] = 40                        # ToT 10 arrives 40 ticks late
    b = StreamBuilder()
    b.tdc(0)
    b.pix(5, 5, 100, 1000)
    b.pix(5, 6, 10, 1050)               # 50 ticks later raw, 10 corrected -> adjacent (dt 32)
    b.pix(50, 50, 10, 64_010)           # raw ToF 64010 > cut -> dropped despite correction
    r0 = oracle.run(b.packets())
    r1 = oracle.run(b.packets(), oracle.Config(timewalk_lut=lut))
    assert r0["clusters"].size == 2 and r1["clusters"].size == 1
    c = r1["clusters"][0]
    assert c["t0"] == 1000 and c["s_t"] == 10 * 10 and c["s_tot"] == 110
    assert r1["counters"]["dropped_background"] == 1


# ---------------------------------------------------------- Sec. V.A - V.C
def _worked_example_stream(sec, y=100, t=5000):
    b = StreamBuilder()
    b.tdc(0)
    for X, T in zip(sec["X"][0], sec["ToT"][0]):
        b.pix(int(X), y, int(T), t)
    return b


def test_worked_example_golden_is_consistent():
    sec = _sections(os.path.join(GOLDEN, "worked_example_sec5.txt"))
    X = np.array(sec["X"][0]); T = np.array(sec["ToT"][0]); r = sec["radius"][0][0]
    D = np.array(sec["D_X"]); A = np.array(sec["A_X"])
    assert np.array_equal(D, X[None, :] - X[:, None])
    assert np.array_equal(A, (np.abs(D) <= r).astype(float))
    M = T[None, :] * A
    assert np.array_equal(np.array(sec["ToT_A_diff"]), M - M.T)


def test_worked_example_local_maxima_and_centroids():
    sec = _sections(os.path.join(GOLDEN, "worked_example_sec5.txt"))
    b = _worked_example_stream(sec)
    rx = int(sec["radius"][0][0])
    rp = oracle.run(b.packets(), oracle.Config(rx=rx, ry=0, dt_ticks=0, mode=oracle.MODE_PAPER))
    peaks_1based = [i for i in range(1, 6) if rp["is_peak"][i]]    # packet 0 is the trigger
    assert peaks_1based == [int(v) for v in sec["local_maxima_1based"][0]]
    assert list(rp["clusters"]["x"]) == pytest.approx(sec["centroid_X"][0], abs=1e-12)
    A = np.array(sec["A_X"])
    assert list(rp["clusters"]["n"]) == [int(A[i - 1].sum()) for i in peaks_1based]
    assert np.all(rp["clusters"]["y"] == 100)
    # CC mode: components of the same adjacency; one peak each here
    rc = oracle.run(b.packets(), oracle.Config(rx=rx, ry=0, dt_ticks=0))
    assert rc["clusters"].size == 2
    assert list(rc["clusters"]["x"]) == pytest.approx(sec["centroid_X"][0], abs=1e-12)
    assert list(rc["clusters"]["n_peaks"]) == [1, 1]
    assert list(rc["labels"][1:]) == [1, 1, 3, 3, 1]


def test_equal_tot_tie_goes_to_later_pixel():
    """Sec. V.B: equal ToT neighbours -- the later one in the stream is the
    single local maximum."""
    b = StreamBuilder()
    b.tdc(0)
    b.pix(10, 10, 77, 100)
    b.pix(11, 10, 77, 101)
    b.pix(12, 10, 30, 102)
    r = oracle.run(b.packets())
    assert list(r["is_peak"]) == [0, 0, 1, 0]
    assert r["clusters"]["n_peaks"][0] == 1


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("mode", [oracle.MODE_CC, oracle.MODE_PAPER])
def test_bruteforce_tiny_dense(seed, mode):
    rng = np.random.default_rng(1000 + seed)
    rx, ry, dt = [(1, 1, 32), (0, 2, 10), (2, 1, 0), (3, 3, 100)][seed % 4]
    lut = None
    if seed % 3 == 2:
        lut = rng.integers(-20, 20, size=1024).astype(np.int16)
    b = random_dense_stream(rng, n_shots=3, per_shot=50 + 10 * (seed % 3))
    exp = brute_force(b, rx=rx, ry=ry, dt=dt, lut=lut, mode=mode, idx_base=17)
    got = oracle.run(b.packets(), oracle.Config(rx=rx, ry=ry, dt_ticks=dt, mode=mode, timewalk_lut=lut), idx_base=17)
    assert got["status"] == 0
    assert np.array_equal(got["labels"], exp["labels"])
    assert np.array_equal(got["is_peak"], exp["is_peak"])
    assert np.array_equal(got["triggers"], exp["triggers"])
    cl = got["clusters"]
    assert cl.size == len(exp["clusters"])
    for g, e in zip(cl, exp["clusters"]):
        for f in ("label", "shot", "t0", "s_tot", "s_x", "s_y", "s_t", "n", "n_peaks"):
            assert int(g[f]) == e[f], f
        for f in ("x", "y", "tof"):
            assert (np.isnan(g[f]) and np.isnan(e[f])) or g[f] == e[f], f


# ----------------------------------------------------- invariants, planted truth
@pytest.fixture(scope="module")
def small_run():
    p = synth.small(n_shots=200, pair_frac=0.05, dark_per_shot=3.0)
    pk, truth, trig = synth.generate(p)
    return pk, truth, trig, oracle.run(pk, want_info=True)


def test_invariants_small(small_run):
    pk, truth, trig, r = small_run
    labels, cl, info = r["labels"], r["clusters"], r["info"]
    kept = labels >= 0
    assert np.array_equal(r["triggers"], trig)
    # every kept pixel is in exactly one cluster, whose label is a member
    assert set(np.unique(labels[kept])) == set(cl["label"])
    assert np.all(labels[cl["label"]] == cl["label"])
    assert np.all(np.diff(cl["label"]) > 0)
    # ToT conservation, counts
    assert cl["s_tot"].sum() == info["tot"][kept].sum()
    assert cl["n"].sum() == kept.sum() == r["counters"]["kept"]
    assert cl.size <= kept.sum()
    # the label is the earliest member by (time, stream index)
    order = np.lexsort((np.arange(len(labels))[kept], info["t"][kept], labels[kept]))
    first = np.arange(len(labels))[kept][order]
    lab_sorted = labels[kept][order]
    starts = np.r_[True, lab_sorted[1:] != lab_sorted[:-1]]
    assert np.array_equal(first[starts], lab_sorted[starts])
    # dark counts far after the trigger are cut
    assert r["counters"]["dropped_background"] > 0


def test_planted_isolated_particles_recovered(small_run):
    pk, truth, trig, r = small_run
    cl = r["clusters"]
    tick = 1.5625
    matched = 0
    for s in range(len(trig)):
        sel = np.flatnonzero(truth["shot"] == s)
        cs = cl[cl["shot"] == s]
        for i in sel:
            if truth["kind"][i] != 0:
                continue
            d = np.hypot(truth["cx"][sel] - truth["cx"][i], truth["cy"][sel] - truth["cy"][i])
            dtt = np.abs(truth["t"][sel] - truth["t"][i])
            # isolated: no other particle nearby while its pixels could be
            # busy (a pixel stays over threshold for up to 16*1023 ticks)
            others = (d < 8) & (dtt < 16 * 1024 + 200) & (sel != i)
            if others.any() or not (3 < truth["cx"][i] < 252 and 3 < truth["cy"][i] < 252):
                continue
            dist = np.hypot(cs["x"] - truth["cx"][i], cs["y"] - truth["cy"][i])
            j = np.argmin(dist)
            assert dist[j] < 0.5
            assert abs(cs["tof"][j] - (truth["t"][i] - trig[s])) < 3.0 / tick * 3
            near_t = np.abs(cs["tof"] - (truth["t"][i] - trig[s])) < 100
            assert np.sum((dist < 4) & near_t) == 1
            matched += 1
    assert matched > 1000


@pytest.mark.parametrize("cx,cy", [(100.0, 50.0), (100.5, 50.0), (31.5, 200.5), (7.0, 7.5)])
def test_symmetric_cloud_centroid_closed_form(cx, cy):
    """A cloud centred on a pixel centre or half-integer has a mirror-symmetric
    ToT pattern, so its centre of mass (Sec. V.C) is exactly the centre."""
    b = StreamBuilder()
    b.tdc(0)
    cells = []
    for x in range(int(cx) - 4, int(cx) + 6):
        for y in range(int(cy) - 4, int(cy) + 6):
            v = int(np.floor(800 * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / 2.0)))
            if v >= 10:
                cells.append((x, y, v))
    rng = np.random.default_rng(3)
    for i in rng.permutation(len(cells)):
        x, y, v = cells[i]
        b.pix(x, y, v, 3000 + int(rng.integers(0, 5)))
    r = oracle.run(b.packets())
    assert r["clusters"].size == 1
    c = r["clusters"][0]
    assert c["x"] == cx and c["y"] == cy
    assert c["n"] == len(cells)


def test_empty_and_degenerate_inputs():
    r = oracle.run(np.zeros(0, np.uint64))
    assert r["status"] == 0 and r["clusters"].size == 0 and r["triggers"].size == 0
    b = StreamBuilder()
    b.tdc(0)
    b.pix(0, 0, 0, 10)            # zero ToT: a cluster with no weight -> NaN centroid
    r = oracle.run(b.packets())
    assert r["clusters"].size == 1 and np.isnan(r["clusters"]["x"][0])
    b = StreamBuilder()
    for _ in range(3):
        b.pix(1, 1, 1, 1)         # no trigger at all
    r = oracle.run(b.packets())
    assert r["counters"]["dropped_pre_trigger"] == 3 and r["clusters"].size == 0


def test_slice_with_initial_epochs_matches_full_stream():
    """A slice cut from the middle of a stream, given the number of wraps
    before it, reproduces the full stream's times and clusters for its shots."""
    p = synth.small(n_shots=40, shot_begin=480)
    full, _, trig = synth.generate(p)
    rf = oracle.run(full, want_info=True)
    tdc_pos = np.flatnonzero((full >> np.uint64(60)) == 6)
    k = 25
    sl = full[tdc_pos[k]:tdc_pos[k + 1]]
    tk = int(trig[k])
    P, PT = 1 << 34, 1 << 36
    # first pixel: the epoch whose time lies within half a period of the trigger
    w = int(sl[1])
    raw = ((((w & 0xFFFF) << 14) | ((w >> 30) & 0x3FFF)) * 16 - ((w >> 16) & 0xF)) % P
    e_pix = round((tk - raw) / P)
    cfg = oracle.Config(epoch0_pix=e_pix, epoch0_tdc=tk // PT)
    rs = oracle.run(sl, cfg, idx_base=int(tdc_pos[k]), want_info=True)
    assert rs["triggers"][0] == tk
    assert np.array_equal(rs["info"]["t"], rf["info"]["t"][tdc_pos[k]:tdc_pos[k + 1]])
    cf = rf["clusters"][rf["clusters"]["shot"] == k]
    cs = rs["clusters"].copy()
    cs["shot"] += k
    assert np.array_equal(cf, cs)
    assert np.array_equal(rs["labels"], rf["labels"][tdc_pos[k]:tdc_pos[k + 1]])


def test_slice_continuing_a_stream_across_a_wrap():
    """A slice given the previous raw values and wrap counts applies the step
    rule of Sec. IV.A to its first packet too, so a cut placed right after a
    wrap still reproduces the full stream's times."""
    P = 1 << 34
    b = StreamBuilder()
    b.tdc(P - 100_000)
    true = [P - 9000, P - 5000, P + 300, P - 100, P + 900, P + 5000]
    for t in true:
        b.pix(3, 3, 10, t)
    pk = b.packets()
    full = oracle.run(pk, want_info=True)["info"]["t"]
    # cut after the first post-wrap pixel: the slice starts with a straggler
    cfg = oracle.Config(epoch0_pix=1, epoch0_tdc=0, prev_pix_raw=(P + 300) % P, prev_tdc_raw=P - 100_000)
    part = oracle.run(pk[4:], cfg, want_info=True)["info"]["t"]
    assert list(part) == list(full[4:]) == true[3:]


def test_literal_tie_break_diverges_only_past_position_1000():
    """Sec. V.B's +0.001 * position tie-break, literally, against the exact
    (ToT, position) reading: equal on ties and below position 1000; past it
    the literal key lets a dimmer, later pixel beat a brighter neighbour."""
    import oracle.tiebreak as tb
    adj = np.array([[0, 1], [1, 0]], bool)
    # a tie: the later pixel wins under both readings
    assert list(tb.maxima_literal([50, 50], [3, 7], adj)) == list(tb.maxima_exact([50, 50], [3, 7], adj)) == [False, True]
    # brighter earlier pixel, positions below 1000: the readings agree
    assert list(tb.maxima_literal([101, 100], [0, 999], adj)) == list(tb.maxima_exact([101, 100], [0, 999], adj)) == [True, False]
    # past position 1000 the literal key flips the order of two ToT values
    assert list(tb.maxima_exact([101, 100], [0, 1500], adj)) == [True, False]
    assert list(tb.maxima_literal([101, 100], [0, 1500], adj)) == [False, True]
    # the oracle follows the exact reading on such a pair (a shot of 1,501 pixels)
    b = StreamBuilder()
    b.tdc(1000)
    for k in range(1499):                     # far-away filler pixels, one per position
        b.pix(200 + (k % 40), 200 + (k // 40) % 40, 20, 2000 + 40 * k)
    b.pix(10, 10, 101, 3000)                  # the brighter pixel, stream position 1500
    b.pix(10, 11, 100, 3001)                  # its dimmer neighbour, stream position 1501
    pk = b.packets()
    r = oracle.run(pk)
    assert r["labels"][1500] >= 0 and r["labels"][1501] == r["labels"][1500]
    assert r["is_peak"][1500] == 1 and r["is_peak"][1501] == 0


@pytest.mark.parametrize("rx,ry,dt", [(1, 1, 32), (2, 1, 8)])
def test_bruteforce_large_dense_shot(rx, ry, dt):
    """One shot of 4,000 pixels crowded into 40 x 40 pixels and 3,000 ticks
    (long adjacency chains, crowded time windows: the regime of a shot longer
    than a tile's range). The oracle's components, canonical labels (the
    stream index of each component's earliest pixel in (time, index) order)
    and per-cluster counts and sums equal the connected components of the
    dense pairwise adjacency matrix (Sec. V.A box rule), found by scipy."""
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    sparse = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(77 + rx)
    n, t0 = 4000, 1_000_000
    xs = rng.integers(100, 140, n)
    ys = rng.integers(100, 140, n)
    tots = rng.integers(1, 200, n)
    ts = t0 + 700 + rng.integers(0, 3000, n)
    b = StreamBuilder()
    b.tdc(t0)
    for i in range(n):
        b.pix(int(xs[i]), int(ys[i]), int(tots[i]), int(ts[i]))
    b.tdc(t0 + 640_000)
    got = oracle.run(b.packets(), oracle.Config(rx=rx, ry=ry, dt_ticks=dt))
    assert got["status"] == 0
    adj = ((np.abs(xs[:, None] - xs[None, :]) <= rx) & (np.abs(ys[:, None] - ys[None, :]) <= ry)
           & (np.abs(ts[:, None] - ts[None, :]) <= dt))
    ncomp, comp = csgraph.connected_components(sparse.csr_matrix(adj), directed=False)
    pos = np.arange(n) + 1                      # stream index of pixel i (after the first trigger)
    first = np.lexsort((pos, ts))               # (time, index) order
    label = np.full(ncomp, -1, np.int64)
    for i in first:
        if label[comp[i]] < 0:
            label[comp[i]] = pos[i]
    assert np.array_equal(got["labels"][1:n + 1], label[comp])
    cl = got["clusters"]
    assert cl.size == ncomp
    order = np.argsort(label)
    assert np.array_equal(cl["label"], label[order])
    w = tots.astype(np.int64)
    for f, vals in (("n", np.ones(n, np.int64)), ("s_tot", w), ("s_x", w * xs), ("s_y", w * ys)):
        assert np.array_equal(cl[f], np.bincount(comp, weights=vals, minlength=ncomp).astype(np.int64)[order]), f
