"""Hand-built packet streams for tests, plus an O(n^2) brute-force model.

The builders place pixels and triggers at chosen true times and encode them
with the generator's encoder; the brute force works from those chosen values
(never from the oracle's or the GPU's decoding), applies the box adjacency of
Sec. V.A pairwise, closes it with a naive union-find, and forms the Sec. V.B
local maxima and Sec. V.C sums directly from their definitions.
"""
from __future__ import annotations

import numpy as np

import synth


class StreamBuilder:
    """Collects events in stream order; `packets()` encodes them."""

    def __init__(self):
        self.kind = []      # "pix" | "tdc" | "bad"
        self.vals = []

    def tdc(self, t):
        self.kind.append("tdc"); self.vals.append((int(t),))

    def pix(self, x, y, tot, t):
        self.kind.append("pix"); self.vals.append((int(x), int(y), int(tot), int(t)))

    def bad(self, word):
        self.kind.append("bad"); self.vals.append((int(word),))

    def packets(self) -> np.ndarray:
        out = np.empty(len(self.kind), np.uint64)
        for i, (k, v) in enumerate(zip(self.kind, self.vals)):
            if k == "pix":
                out[i] = synth.encode_pixels([v[0]], [v[1]], [v[2]], [v[3]])[0]
            elif k == "tdc":
                out[i] = synth.encode_tdcs([v[0]], [i & 0xFFF])[0]
            else:
                out[i] = np.uint64(v[0])
        return out


def brute_force(b: StreamBuilder, rx=1, ry=1, dt=32, tof_max=64_000, lut=None, mode=0, idx_base=0):
    """Expected oracle outputs for a stream built from known true times."""
    trig = [v[0] for k, v in zip(b.kind, b.vals) if k == "tdc"]
    kept = []   # (idx, shot, tc, x, y, tot)
    for i, (k, v) in enumerate(zip(b.kind, b.vals)):
        if k != "pix":
            continue
        x, y, tot, t = v
        shot = -1
        for s, tt in enumerate(trig):     # most recent trigger in time
            if tt <= t:
                shot = s
        if shot < 0 or t - trig[shot] > tof_max:
            continue
        tc = t - (int(lut[tot]) if lut is not None else 0)
        kept.append((i, shot, tc, x, y, tot))
    n = len(kept)
    A = np.zeros((n, n), bool)
    for a in range(n):
        for c in range(n):
            ia, sa, ta, xa, ya, _ = kept[a]
            ic, sc, tcc, xc, yc, _ = kept[c]
            A[a, c] = sa == sc and abs(xa - xc) <= rx and abs(ya - yc) <= ry and abs(ta - tcc) <= dt
    parent = list(range(n))

    def find(u):
        while parent[u] != u:
            u = parent[u]
        return u
    for a in range(n):
        for c in range(a + 1, n):
            if A[a, c]:
                ra, rc = find(a), find(c)
                if ra != rc:
                    parent[rc] = ra
    peak = []
    for a in range(n):
        p = True
        for c in range(n):
            if c != a and A[a, c]:
                if kept[c][5] > kept[a][5] or (kept[c][5] == kept[a][5] and kept[c][0] > kept[a][0]):
                    p = False
        peak.append(p)
    n_pk = len(b.kind)
    labels = np.full(n_pk, -1, np.int64)
    is_peak = np.zeros(n_pk, np.uint8)
    for a in range(n):
        is_peak[kept[a][0]] = int(peak[a])
    recs = []
    if mode == 0:
        comps = {}
        for a in range(n):
            comps.setdefault(find(a), []).append(a)
        for members in comps.values():
            first = min(members, key=lambda m: (kept[m][1], kept[m][2], kept[m][0]))
            lab = idx_base + kept[first][0]
            for m in members:
                labels[kept[m][0]] = lab
            recs.append(_sums(lab, kept, members, kept[first][2], trig, sum(peak[m] for m in members)))
    else:
        for a in range(n):
            labels[kept[a][0]] = idx_base + kept[a][0]
            if not peak[a]:
                continue
            members = [c for c in range(n) if A[a, c]]
            t0 = min(kept[c][2] for c in members)
            recs.append(_sums(idx_base + kept[a][0], kept, members, t0, trig, 1))
    recs.sort(key=lambda r: r["label"])
    return dict(labels=labels, is_peak=is_peak, clusters=recs, triggers=np.array(trig, np.int64),
                n_kept=n)


def _sums(label, kept, members, t0, trig, n_peaks):
    shot = kept[members[0]][1]
    s_tot = sum(kept[m][5] for m in members)
    s_x = sum(kept[m][3] * kept[m][5] for m in members)
    s_y = sum(kept[m][4] * kept[m][5] for m in members)
    s_t = sum((kept[m][2] - t0) * kept[m][5] for m in members)
    with np.errstate(all="ignore"):
        x = np.float64(s_x) / np.float64(s_tot)
        y = np.float64(s_y) / np.float64(s_tot)
        tof = np.float64(t0 - trig[shot]) + np.float64(s_t) / np.float64(s_tot)
    return dict(label=label, shot=shot, t0=t0, s_tot=s_tot, s_x=s_x, s_y=s_y, s_t=s_t,
                n=len(members), n_peaks=int(n_peaks), x=float(x), y=float(y), tof=float(tof))


def random_dense_stream(rng: np.random.Generator, n_shots=3, per_shot=60, area=8, t_spread=80,
                        tot_hi=20, period=640_000, t0=1_000_000, extras=True) -> StreamBuilder:
    """Dense tiny shots: pixels crowd a small area and time window so that
    adjacency, merging, equal-ToT ties and same-cell repeats are frequent."""
    b = StreamBuilder()
    if extras:   # pixels before the first trigger are dropped
        for _ in range(3):
            b.pix(rng.integers(0, 256), rng.integers(0, 256), rng.integers(0, tot_hi), t0 - rng.integers(1, 5000))
    for s in range(n_shots):
        tt = t0 + s * period
        b.tdc(tt)
        ev = []
        x0, y0 = rng.integers(0, 256 - area), rng.integers(0, 256 - area)
        base = tt + int(rng.integers(640, 6400))
        for _ in range(per_shot):
            ev.append((x0 + rng.integers(0, area), y0 + rng.integers(0, area),
                       rng.integers(0, tot_hi), base + rng.integers(0, t_spread)))
        if extras:
            ev.append((rng.integers(0, 256), rng.integers(0, 256), 5, tt + 64_000))      # ToF == cut: kept
            ev.append((rng.integers(0, 256), rng.integers(0, 256), 5, tt + 64_001))      # beyond: dropped
            ev.append((x0, y0, 7, base))                                                # same cell, same time
        order = rng.permutation(len(ev))
        for i in order:
            b.pix(*ev[i])
        if extras and s == 1:
            b.bad(0x1234_5678_9ABC_DEF0)
    return b
