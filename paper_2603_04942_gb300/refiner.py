"""The learned overlap refiner: data, training and inference on the GPU.

The paper stops at one ToT-weighted centroid per cluster (Sec. V.C); its
multi-hit discussion (Sec. VII.B) and the local-maximum count (Sec. V.B) note
that two particles landing close in space and time merge into one cluster.
This module trains a small network on clusters that the project's generator
and its own clustering produce, to say whether a cluster holds one or two
particles and where they are; below a confidence threshold the plain
centroid stands.

  data     : generator packets with planted pairs -> tpx_process (CC mode) ->
             tpx_refine_patches for clusters with more than 12 pixels. The
             generator's particles are matched to clusters on the host
             (nearest cluster in x, y and ToF/8 within a shot); clusters that
             hold one or two particles inside their patch become training
             rows (count, offsets of the brighter particle, then of the
             other, in pixels from the patch centre).
  training : tpx_refiner_train_step per minibatch (fp32 GEMMs, Adam).
  inference: tpx_refiner_infer (all layers in one tensor-core kernel, bf16
             operands) or tpx_refiner_forward (fp32), then
             tpx_refine_decide.

Every arithmetic step runs in the library's kernels; this module only
prepares targets on the host and moves buffers.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import CLUSTER_DTYPE, Context

NIN = 162
HIDDEN = 160          # 162 -> 160 -> 160 -> 6: 52,806 parameters
MIN_PIXELS = 12
TOF_SCALE = 8.0       # ticks per pixel-equivalent when matching particles to clusters
TRIG_PERIOD_TICKS = 640_000


@dataclasses.dataclass
class Dataset:
    """Patches (device) and targets for the clusters whose truth is one or
    two particles inside the patch."""
    x: object              # torch float32 [n x 162] (device)
    xb: object             # the same rows as bf16 bits (torch int16 [n x 162], device)
    y: object              # torch float32 [n x 5] (device): count, dx1, dy1, dx2, dy2
    count: np.ndarray      # [n] truth count (1 or 2)
    pos: np.ndarray        # [n x 4] truth positions (x1, y1, x2, y2), pixels
    centroid: np.ndarray   # [n x 2] the plain centroid of the cluster
    sep: np.ndarray        # [n] pair separation (0 for singles), pixels
    rows: np.ndarray       # [n] row in the patch arrays of the call
    patches: dict          # the tpx_refine_patches outputs (device)
    patches16: dict        # the tpx_refine_patches_bf16 outputs (device)
    clusters: np.ndarray   # host copy of all records of the call
    clusters_dev: object   # the records on the device (uint8 tensor)
    n_selected: int        # clusters with more than MIN_PIXELS pixels
    sel: np.ndarray        # [n_selected] record index of each patch (host)
    truth: dict            # the generator's particles (shot relative to the stream, cx, cy)


def _truth_match(cl: np.ndarray, truth: dict, sel: np.ndarray, centre: np.ndarray, t_start: int,
                 shot_begin: int = 0, period: int = TRIG_PERIOD_TICKS):
    """Per selected cluster: the particles whose nearest cluster (same shot,
    distance in x, y, ToF / TOF_SCALE) it is. Shot k of the generator has
    its trigger at t_start + k * period and is trigger k - shot_begin of the
    stream."""
    from scipy.spatial import cKDTree
    big = 1e6
    cpts = np.stack([cl["x"], cl["y"], cl["tof"] / TOF_SCALE, cl["shot"] * big], axis=1)
    tof = truth["t"] - (t_start + truth["shot"] * period)
    ppts = np.stack([truth["cx"], truth["cy"], tof / TOF_SCALE, (truth["shot"] - shot_begin) * big], axis=1)
    _, owner = cKDTree(cpts).query(ppts)
    slot = np.full(cl.size, -1, np.int64)
    slot[sel] = np.arange(sel.size)
    s_of_p = slot[owner]
    order = np.argsort(s_of_p, kind="stable")
    s_sorted = s_of_p[order]
    starts = np.searchsorted(s_sorted, np.arange(sel.size))
    ends = np.searchsorted(s_sorted, np.arange(sel.size), side="right")
    n = sel.size
    count = (ends - starts).astype(np.int64)
    pos = np.zeros((n, 4))
    sep = np.zeros(n)
    ok = (count == 1) | (count == 2)
    for s in np.nonzero(ok)[0]:
        ps = order[starts[s]: ends[s]]
        if ps.size == 2 and truth["peak"][ps[1]] > truth["peak"][ps[0]]:
            ps = ps[::-1]                       # the brighter particle first
        for k, p in enumerate(ps):
            pos[s, 2 * k] = truth["cx"][p]
            pos[s, 2 * k + 1] = truth["cy"][p]
        if ps.size == 2:
            sep[s] = math.hypot(pos[s, 0] - pos[s, 2], pos[s, 1] - pos[s, 3])
    # every particle inside the patch (|offset| <= 4.5 px)
    off = pos - np.repeat(centre, 2, axis=0).reshape(n, 4) * 1.0
    inside = np.abs(off[:, :2]).max(axis=1) <= 4.5
    inside &= (count == 1) | (np.abs(off[:, 2:]).max(axis=1) <= 4.5)
    return count, pos, sep, ok & inside


def make_dataset(ctx: Context, p, min_pixels: int = MIN_PIXELS, shuffle_seed: int | None = 0) -> Dataset:
    """Generate the recipe `p` (synth.Params), cluster it with tpx_process,
    extract patches and match the generator's particles."""
    import torch
    import synth
    s = synth.Stream(p)
    try:
        host = s.packets()
        truth = s.truth()
    finally:
        s.close()
    d_pk = torch.from_numpy(host.view(np.int64)).cuda()
    n = d_pk.numel()
    ctx.reserve(n)
    out = ctx.alloc_outputs(n, labels=True)
    ctx.tpx_process(d_pk, out)
    ctx.tpx_sync()
    n_cl = int(out["n_clusters"].item())
    pt = ctx.tpx_refine_patches(d_pk, out["labels"], out["clusters"], n_cl, min_pixels)
    pt16 = ctx.tpx_refine_patches_bf16(d_pk, out["labels"], out["clusters"], n_cl, min_pixels)
    torch.cuda.synchronize()
    n_sel = int(pt["n"].item())
    cl = np.frombuffer(out["clusters"][: n_cl * CLUSTER_DTYPE.itemsize].cpu().numpy().tobytes(), CLUSTER_DTYPE)
    sel = pt["sel"][:n_sel].cpu().numpy()
    centre = pt["centre"][:n_sel].cpu().numpy()
    count, pos, sep, ok = _truth_match(cl, truth, sel, centre, p.t_start_ticks, p.shot_begin, p.trig_period_ticks)
    rows = np.nonzero(ok)[0]
    if shuffle_seed is not None:
        rows = rows[np.random.default_rng(shuffle_seed).permutation(rows.size)]
    y = np.zeros((rows.size, 5), np.float32)
    y[:, 0] = count[rows]
    c2 = np.repeat(centre[rows], 2, axis=0).reshape(rows.size, 4)
    y[:, 1:] = (pos[rows] - c2) * (np.repeat(count[rows], 4).reshape(-1, 4) >= np.array([1, 1, 2, 2]))
    d_rows = torch.from_numpy(rows).cuda()
    x = pt["patches"][:n_sel].index_select(0, d_rows).contiguous()
    xb = pt16["patches"][:n_sel].index_select(0, d_rows).contiguous()
    c = cl[sel[rows]]
    return Dataset(x=x, xb=xb, y=torch.from_numpy(y).cuda(), count=count[rows], pos=pos[rows],
                   centroid=np.stack([c["x"], c["y"]], axis=1), sep=sep[rows], rows=rows, patches=pt, patches16=pt16,
                   clusters=cl, clusters_dev=out["clusters"], n_selected=n_sel, sel=sel,
                   truth=dict(shot=truth["shot"] - p.shot_begin, cx=truth["cx"], cy=truth["cy"]))


class Refiner:
    """The network's parameters and Adam state, on the device."""

    def __init__(self, ctx: Context, hidden: int = HIDDEN, seed: int = 0):
        import torch
        self.ctx, self.h = ctx, int(hidden)
        self.n_params = Context.tpx_refiner_params(self.h)
        rng = np.random.default_rng(seed)
        p = np.zeros(self.n_params, np.float32)
        o = 0
        for fan_in, fan_out in ((NIN, self.h), (self.h, self.h), (self.h, 6)):
            lim = math.sqrt(6.0 / fan_in)                        # He-uniform for ReLU layers
            p[o: o + fan_in * fan_out] = rng.uniform(-lim, lim, fan_in * fan_out)
            o += fan_in * fan_out + fan_out                      # biases start at 0
        assert o == self.n_params
        self.params = torch.from_numpy(p).cuda()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0

    def train(self, ds: Dataset, epochs: int = 1, batch: int = 4096, lr: float = 2e-3, offset_weight: float = 1.0,
              seed: int = 0, lr_final: float | None = None) -> np.ndarray:
        """Minibatch Adam over the (pre-shuffled) rows; minibatch order is
        permuted each epoch. Returns the per-step losses (host). With
        `lr_final`, the rate decays geometrically to it over the run."""
        import torch
        n = ds.x.shape[0]
        nb = max(1, n // batch)
        work = torch.empty((batch * (4 * self.h + 12),), dtype=torch.float32, device=ds.x.device)
        losses = torch.zeros(epochs * nb, dtype=torch.float32, device=ds.x.device)
        rng = np.random.default_rng(seed)
        total = epochs * nb
        k = 0
        for _ in range(epochs):
            for b in rng.permutation(nb):
                self.step += 1
                rate = lr if lr_final is None else lr * (lr_final / lr) ** (k / max(1, total - 1))
                r0 = int(b) * batch
                self.ctx.tpx_refiner_train_step(self.params, self.m, self.v, self.grad, self.h, self.step,
                                                ds.x[r0: r0 + batch], ds.y[r0: r0 + batch], rate, offset_weight,
                                                work, losses[k:], n=batch)
                k += 1
        torch.cuda.synchronize()
        return losses.cpu().numpy()

    def forward(self, x, n: int | None = None):
        """The fp32 network (the training precision)."""
        return self.ctx.tpx_refiner_forward(self.params, self.h, x, n)

    def infer(self, x, n: int | None = None, out=None):
        """The network on the tensor cores (bf16 operands, fp32 sums); the
        bf16 copy of the parameters is refreshed after training steps."""
        if getattr(self, "_packed_step", None) != self.step:
            self.packed = self.ctx.tpx_refiner_pack(self.params, self.h, getattr(self, "packed", None))
            self._packed_step = self.step
        return self.ctx.tpx_refiner_infer(self.packed, self.h, x, n, out)

    def refine(self, patches: dict, clusters_dev, n: int, threshold: float = 0.8, fp32: bool = False):
        """Refined hits (device [n x 5]) of the first n patches of a
        tpx_refine_patches call."""
        out = self.forward(patches["patches"], n) if fp32 else self.infer(patches["patches"], n)
        return self.ctx.tpx_refine_decide(out, clusters_dev, patches["sel"], patches["centre"], n, threshold)

    def refine_rows(self, ds: Dataset, threshold: float = 0.8, fp32: bool = False) -> np.ndarray:
        """Refined hits (host [n x 5]) of the dataset's rows."""
        import torch
        rows = torch.from_numpy(ds.rows).cuda()
        sel = ds.patches["sel"][: ds.n_selected].index_select(0, rows).contiguous()
        centre = ds.patches["centre"][: ds.n_selected].index_select(0, rows).contiguous()
        out = self.forward(ds.x) if fp32 else self.infer(ds.x)
        n = ds.x.shape[0]
        return self.ctx.tpx_refine_decide(out, ds.clusters_dev, sel, centre, n, threshold)[:n].cpu().numpy()

    def state(self) -> dict:
        return dict(hidden=self.h, params=self.params.cpu().numpy(), step=self.step)


class CnnRefiner:
    """The convolutional refiner (conv 2->16->16->32 channels of 3 x 3, fc
    288->144->6; 49,750 parameters) and its Adam state, on the device;
    trained in fp32, inferred on the tensor cores with bf16 operands."""

    def __init__(self, ctx: Context, seed: int = 0):
        import torch
        self.ctx = ctx
        self.n_params = Context.tpx_cnn_params()
        rng = np.random.default_rng(seed)
        p = np.zeros(self.n_params, np.float32)
        o = 0
        for fan_in, size, bias in ((2 * 9, 16 * 2 * 9, 16), (16 * 9, 16 * 16 * 9, 16), (16 * 9, 32 * 16 * 9, 32),
                                   (288, 144 * 288, 144), (144, 6 * 144, 6)):
            lim = math.sqrt(6.0 / fan_in)                        # He-uniform for ReLU layers
            p[o: o + size] = rng.uniform(-lim, lim, size)
            o += size + bias                                     # biases start at 0
        assert o == self.n_params
        self.params = torch.from_numpy(p).cuda()
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.step = 0

    def train(self, ds: Dataset, epochs: int = 1, batch: int = 4096, lr: float = 2e-3, offset_weight: float = 1.0,
              seed: int = 0, lr_final: float | None = None) -> np.ndarray:
        import torch
        from . import lib
        n = ds.x.shape[0]
        nb = max(1, n // batch)
        work = torch.empty(int(lib().tpx_cnn_work_floats(batch)), dtype=torch.float32, device=ds.x.device)
        losses = torch.zeros(epochs * nb, dtype=torch.float32, device=ds.x.device)
        rng = np.random.default_rng(seed)
        total = epochs * nb
        k = 0
        for _ in range(epochs):
            for b in rng.permutation(nb):
                self.step += 1
                rate = lr if lr_final is None else lr * (lr_final / lr) ** (k / max(1, total - 1))
                r0 = int(b) * batch
                self.ctx.tpx_cnn_train_step(self.params, self.m, self.v, self.grad, self.step, ds.x[r0: r0 + batch],
                                            ds.y[r0: r0 + batch], rate, offset_weight, work, losses[k:], n=batch)
                k += 1
        torch.cuda.synchronize()
        return losses.cpu().numpy()

    def forward(self, x, n: int | None = None):
        """The fp32 network (the training precision)."""
        return self.ctx.tpx_cnn_forward(self.params, x, n)

    def infer(self, xb, n: int | None = None, out=None):
        """The network on the tensor cores; xb: bf16 patches."""
        if getattr(self, "_packed_step", None) != self.step:
            self.packed = self.ctx.tpx_cnn_pack(self.params, getattr(self, "packed", None))
            self._packed_step = self.step
        return self.ctx.tpx_cnn_infer(self.packed, xb, n, out=out)

    def refine(self, patches16: dict, clusters_dev, n: int, threshold: float = 0.8):
        """Refined hits (device [n x 5]) of the first n patches of a
        tpx_refine_patches_bf16 call."""
        out = self.infer(patches16["patches"], n)
        return self.ctx.tpx_refine_decide(out, clusters_dev, patches16["sel"], patches16["centre"], n, threshold)

    def refine_rows(self, ds: Dataset, threshold: float = 0.8, fp32: bool = False) -> np.ndarray:
        import torch
        rows = torch.from_numpy(ds.rows).cuda()
        sel = ds.patches["sel"][: ds.n_selected].index_select(0, rows).contiguous()
        centre = ds.patches["centre"][: ds.n_selected].index_select(0, rows).contiguous()
        out = self.forward(ds.x) if fp32 else self.infer(ds.xb)
        n = ds.x.shape[0]
        return self.ctx.tpx_refine_decide(out, ds.clusters_dev, sel, centre, n, threshold)[:n].cpu().numpy()


def evaluate(ds: Dataset, hits: np.ndarray) -> dict:
    """Errors against the generator's truth on the dataset's rows, for the
    refined hits (rows k, x1, y1, x2, y2 from tpx_refine_decide, k = 0 the
    centroid) and for the plain centroid.

    Per particle the error is the distance to the nearest reported hit of
    its cluster; merged pairs are the rows whose truth count is 2."""
    k = hits[:, 0].astype(int)
    n = k.size
    h1 = hits[:, 1:3]
    h2 = np.where((k == 2)[:, None], hits[:, 3:5], h1)
    p1, p2 = ds.pos[:, :2], ds.pos[:, 2:]
    d = lambda a, b: np.hypot(a[:, 0] - b[:, 0], a[:, 1] - b[:, 1])   # noqa: E731
    e1 = np.minimum(d(p1, h1), d(p1, h2))
    e2 = np.minimum(d(p2, h1), d(p2, h2))
    c = ds.centroid
    c1, c2 = d(p1, c), d(p2, c)
    pair = ds.count == 2
    single = ~pair
    res = dict(rows=int(n), singles=int(single.sum()), pairs=int(pair.sum()),
               fallback=float(np.mean(k == 0)) if n else 0.0,
               count_accuracy=float(np.mean(np.where(k == 0, 1, k) == ds.count)) if n else 0.0,
               pair_recall=float(np.mean(k[pair] == 2)) if pair.any() else 0.0,
               single_split=float(np.mean(k[single] == 2)) if single.any() else 0.0,
               single_err_refined=float(np.mean(e1[single])) if single.any() else 0.0,
               single_err_centroid=float(np.mean(c1[single])) if single.any() else 0.0,
               pair_err_refined=float(np.mean(np.r_[e1[pair], e2[pair]])) if pair.any() else 0.0,
               pair_err_centroid=float(np.mean(np.r_[c1[pair], c2[pair]])) if pair.any() else 0.0)
    # resolving power: pairs whose two particles each got their own hit within 1 px
    bins = [0, 1, 2, 3, 4.01]
    rp = []
    for lo, hi in zip(bins[:-1], bins[1:]):
        m = pair & (ds.sep >= lo) & (ds.sep < hi)
        if not m.any():
            rp.append(dict(sep=[lo, min(hi, 4)], pairs=0, resolved_refined=0.0))
            continue
        own = (k[m] == 2) & (np.maximum(np.minimum(d(p1[m], h1[m]), d(p1[m], h2[m])),
                                        np.minimum(d(p2[m], h1[m]), d(p2[m], h2[m]))) < 1.0)
        # the two particles must not share the nearest hit
        a1 = d(p1[m], h1[m]) <= d(p1[m], h2[m])
        a2 = d(p2[m], h1[m]) <= d(p2[m], h2[m])
        own &= a1 != a2
        rp.append(dict(sep=[lo, min(hi, 4)], pairs=int(m.sum()), resolved_refined=float(np.mean(own))))
    res["resolving"] = rp
    return res


def hit_list(ds: Dataset, hits_selected: np.ndarray):
    """All hits of the dataset's stream (x, y, shot): every cluster's plain
    centroid, except that a selected cluster reported as two particles
    (rows of a refine() call over all selected patches) gives its two
    positions."""
    cl = ds.clusters
    two = np.zeros(cl.size, bool)
    k = hits_selected[:, 0].astype(int)
    two[ds.sel[k == 2]] = True
    h2 = hits_selected[k == 2]
    x = np.concatenate([cl["x"][~two], h2[:, 1], h2[:, 3]])
    y = np.concatenate([cl["y"][~two], h2[:, 2], h2[:, 4]])
    s2 = cl["shot"][ds.sel[k == 2]]
    shot = np.concatenate([cl["shot"][~two], s2, s2])
    return x, y, shot


def pair_distance_histogram(x, y, shot, r_max: float = 4.0, bin_px: float = 0.25) -> np.ndarray:
    """Counts of hit pairs of the same shot by distance, in bins of `bin_px`
    up to `r_max` (the multi-hit measure of the paper's Fig. 6)."""
    from scipy.spatial import cKDTree
    pts = np.stack([np.asarray(x, float), np.asarray(y, float), np.asarray(shot, float) * 1e4], axis=1)
    pairs = cKDTree(pts).query_pairs(r_max, output_type="ndarray")
    d = np.hypot(pts[pairs[:, 0], 0] - pts[pairs[:, 1], 0], pts[pairs[:, 0], 1] - pts[pairs[:, 1], 1])
    return np.histogram(d, bins=np.arange(0.0, r_max + 1e-9, bin_px))[0]
