"""The learned overlap refiner on the GPU against the oracle's definition
(oracle/refiner.py): patches bit-exact, the network's forward pass, loss,
gradients and Adam step within fp32 tolerance of the float64 oracle, the
decision exact, and training on generator data splitting merged pairs
better than the plain centroid (Sec. V.C) locates them."""
import numpy as np
import pytest

import oracle
import oracle.refiner as orf
import paper_2603_04942_gb300 as tpx
import synth
from gpu_common import to_device
from paper_2603_04942_gb300 import refiner as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def data():
    p = synth.refiner(n_shots=300)
    pk = synth.generate(p)[0]
    return pk, orf.patches(pk)


def _gpu_patches(ctx, pk, min_pixels=12, capacity=None, index_base=0):
    d = to_device(pk)
    out = ctx.alloc_outputs(pk.size, labels=True, cluster_capacity=max(16, pk.size // 4))
    ctx.tpx_process(d, out, index_base)
    rc, _ = ctx.tpx_sync(check=False)
    assert rc == 0
    n_cl = int(out["n_clusters"].item())
    pt = ctx.tpx_refine_patches(d, out["labels"], out["clusters"], n_cl, min_pixels, capacity, index_base)
    import torch
    torch.cuda.synchronize()
    return out, n_cl, pt


def test_patches_bit_exact(data):
    pk, (op, osel, ocentre, _) = data
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        out, n_cl, pt = _gpu_patches(ctx, pk)
        n = int(pt["n"].item())
        assert pt["status"] == 0 and n == osel.size > 5000
        assert np.array_equal(pt["sel"][:n].cpu().numpy(), osel)
        assert np.array_equal(pt["centre"][:n].cpu().numpy(), ocentre)
        assert np.array_equal(pt["patches"][:n].cpu().numpy(), op)
    finally:
        ctx.close()


@pytest.mark.parametrize("min_pixels,base", [(0, 0), (30, 1 << 33), (10 ** 6, 0)])
def test_patches_other_thresholds_and_base(data, min_pixels, base):
    pk = data[0][: 60_000]
    op, osel, ocentre, _ = orf.patches(pk, min_pixels=min_pixels, idx_base=base)
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        _, _, pt = _gpu_patches(ctx, pk, min_pixels=min_pixels, index_base=base)
        n = int(pt["n"].item())
        assert n == osel.size
        assert np.array_equal(pt["sel"][:n].cpu().numpy(), osel)
        assert np.array_equal(pt["centre"][:n].cpu().numpy(), ocentre)
        assert np.array_equal(pt["patches"][:n].cpu().numpy(), op)
    finally:
        ctx.close()


def test_patches_capacity_overflow_writes_the_first(data):
    pk = data[0][: 60_000]
    op, osel, _, _ = orf.patches(pk)
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        _, _, pt = _gpu_patches(ctx, pk, capacity=100)
        assert pt["status"] == tpx.EOVERFLOW and int(pt["n"].item()) == osel.size
        assert np.array_equal(pt["sel"][:100].cpu().numpy(), osel[:100])
        assert np.array_equal(pt["patches"][:100].cpu().numpy(), op[:100])
    finally:
        ctx.close()


def test_patches_of_an_empty_call():
    import torch
    ctx = tpx.Context(tpx.Config(), max_packets=16)
    try:
        d = torch.zeros(2, dtype=torch.int64, device="cuda")
        lab = torch.zeros(2, dtype=torch.int64, device="cuda")
        cl = torch.zeros(88, dtype=torch.uint8, device="cuda")
        pt = ctx.tpx_refine_patches(d, lab, cl, 0)
        torch.cuda.synchronize()
        assert pt["status"] == 0 and int(pt["n"].item()) == 0
    finally:
        ctx.close()


def _params(h, seed, scale=0.15):
    return np.random.default_rng(seed).normal(scale=scale, size=orf.layout(h)["total"]).astype(np.float32)


@pytest.mark.parametrize("h,n", [(160, 4099), (37, 1), (64, 640), (5, 77)])
def test_forward_matches_oracle(data, h, n):
    import torch
    op = data[1][0]
    x = np.concatenate([op, np.random.default_rng(h).random((max(0, n - op.shape[0]), 162), np.float32)])[:n]
    p = _params(h, n)
    ctx = tpx.Context(tpx.Config(), max_packets=16)
    try:
        out = ctx.tpx_refiner_forward(torch.from_numpy(p).cuda(), h, torch.from_numpy(x).cuda())
        g = out[:n].cpu().numpy().astype(np.float64)
    finally:
        ctx.close()
    o = orf.forward(p.astype(np.float64), h, x.astype(np.float64))
    # fp32 products summed over K <= 162 terms: relative error a few 1e-6
    # of the summed magnitudes; 1e-4 of the output scale bounds it
    assert np.abs(g - o).max() <= 1e-4 * max(1.0, np.abs(o).max())


@pytest.mark.parametrize("h,n", [(160, 4099), (128, 129), (64, 1), (160, 20_000)])
def test_bf16_inference_matches_oracle(data, h, n):
    """The tensor-core kernel against the oracle's inference precision.
    Sums are fp32 on the GPU and exact in the oracle, so a hidden activation
    can round to the neighbouring bf16 value (2^-8 relative) in a few rows:
    nearly all rows agree to 1e-4 of the output scale, every row to 3e-2."""
    import torch
    op = data[1][0]
    x = np.concatenate([op, np.random.default_rng(h).random((max(0, n - op.shape[0]), 162), np.float32)])[:n]
    p = _params(h, n + 1)
    ctx = tpx.Context(tpx.Config(), max_packets=16)
    try:
        packed = ctx.tpx_refiner_pack(torch.from_numpy(p).cuda(), h)
        g = ctx.tpx_refiner_infer(packed, h, torch.from_numpy(x).cuda())[:n].cpu().numpy().astype(np.float64)
        with pytest.raises(tpx.TpxError):
            ctx.tpx_refiner_pack(torch.from_numpy(p).cuda(), 100)
    finally:
        ctx.close()
    o = orf.forward_bf16(p, h, x)
    scale = max(1.0, np.abs(o).max())
    row_err = np.abs(g - o).max(axis=1)
    assert np.mean(row_err <= 1e-4 * scale) >= 0.95
    assert row_err.max() <= 3e-2 * scale


def _targets(n, seed):
    rng = np.random.default_rng(seed)
    y = np.zeros((n, 5), np.float32)
    y[:, 0] = rng.integers(1, 3, n)
    y[:, 1:] = rng.normal(size=(n, 4))
    return y


@pytest.mark.parametrize("h,n", [(160, 1000), (37, 333)])
def test_train_step_matches_oracle(data, h, n):
    import torch
    x = data[1][0][:n]
    y = _targets(n, 5)
    p0 = _params(h, 7, 0.1)
    w, lr = 0.8, 1e-3
    ctx = tpx.Context(tpx.Config(), max_packets=16)
    try:
        P = torch.from_numpy(p0.copy()).cuda()
        m, v, gr = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
        work = torch.empty(n * (4 * h + 12), dtype=torch.float32, device="cuda")
        loss = torch.zeros(2, dtype=torch.float32, device="cuda")
        X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ctx.tpx_refiner_train_step(P, m, v, gr, h, 1, X, Y, lr, w, work, loss[0:])
        torch.cuda.synchronize()
        g1, p1, m1, v1 = gr.cpu().numpy(), P.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy()
        ctx.tpx_refiner_train_step(P, m, v, gr, h, 2, X, Y, lr, w, work, loss[1:])
        torch.cuda.synchronize()
        l = loss.cpu().numpy()
        p2 = P.cpu().numpy()
    finally:
        ctx.close()
    pd = p0.astype(np.float64)
    og = orf.grad(pd, h, x, y, w)
    assert abs(l[0] - orf.loss(pd, h, x, y, w)) <= 1e-5 * abs(l[0]) + 1e-6
    gs = np.abs(og).max()
    assert np.abs(g1 - og).max() <= 1e-4 * gs
    assert np.allclose(m1, 0.1 * og, rtol=0, atol=1e-5 * gs)
    assert np.allclose(v1, 0.001 * og * og, rtol=0, atol=1e-5 * gs * gs)
    op1, om, ov = orf.adam(pd, 0, 0, og, 1, lr)
    big = np.abs(og) > 1e-2 * gs     # where the sign of g is beyond doubt
    assert np.abs(p1 - op1)[big].max() <= 1e-6 + 1e-3 * lr
    # second step from the GPU's first-step parameters
    og2 = orf.grad(p1.astype(np.float64), h, x, y, w)
    assert abs(l[1] - orf.loss(p1.astype(np.float64), h, x, y, w)) <= 1e-5 * abs(l[1]) + 1e-6
    op2, _, _ = orf.adam(p1.astype(np.float64), m1.astype(np.float64), v1.astype(np.float64), og2, 2, lr)
    big2 = big & (np.abs(og2) > 1e-2 * np.abs(og2).max())
    assert np.abs(p2 - op2)[big2].max() <= 1e-6 + 2e-3 * lr


def test_decide_matches_oracle(data):
    import torch
    pk = data[0][: 60_000]
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        out, n_cl, pt = _gpu_patches(ctx, pk)
        n = int(pt["n"].item())
        o = np.random.default_rng(9).normal(scale=2.0, size=(n, 6)).astype(np.float32)
        o[:50, 1] = o[:50, 0] + np.float32(np.log(0.8 / 0.2))   # on the threshold
        for thr in (0.5, 0.8, 0.97):
            hits = ctx.tpx_refine_decide(torch.from_numpy(o).cuda(), out["clusters"], pt["sel"], pt["centre"], n, thr)
            g = hits[:n].cpu().numpy()
            cl = ctx.collect(out, 0, {})["clusters"]
            sel = pt["sel"][:n].cpu().numpy()
            want = orf.decide(o, pt["centre"][:n].cpu().numpy(), np.stack([cl["x"][sel], cl["y"][sel]], 1), thr)
            assert np.array_equal(g, want), thr
        with pytest.raises(tpx.TpxError):
            ctx.tpx_refine_decide(torch.from_numpy(o).cuda(), out["clusters"], pt["sel"], pt["centre"], n, 1.0)
    finally:
        ctx.close()


def test_training_splits_merged_pairs():
    """Trained on about 60k generator clusters, the network reports most
    merged pairs as two hits, rarely splits single particles, and its
    per-particle error on merged pairs is below the plain centroid's."""
    ctx = tpx.Context(tpx.Config(), max_packets=1 << 20)
    try:
        train = R.make_dataset(ctx, synth.refiner(n_shots=3000, seed=6))
        test = R.make_dataset(ctx, synth.refiner(n_shots=500, seed=7), shuffle_seed=None)
        net = R.Refiner(ctx, hidden=64, seed=0)
        losses = net.train(train, epochs=4, batch=1024, lr=2e-3, lr_final=2e-4)
        assert losses[-20:].mean() < 0.5 * losses[:5].mean()
        hits = net.refine_rows(test, 0.8)
        # the fp32 network decides nearly every cluster the same way
        h32 = net.refine_rows(test, 0.8, fp32=True)
        assert np.mean(h32[:, 0] == hits[:, 0]) > 0.99
        ev = R.evaluate(test, hits)
        assert ev["pairs"] > 2000 and ev["singles"] > 4000
        assert ev["pair_recall"] > 0.6 and ev["single_split"] < 0.05
        assert ev["pair_err_refined"] < 0.7 * ev["pair_err_centroid"]
        assert ev["single_err_refined"] <= ev["single_err_centroid"] + 0.05
        # the whole inference path on every selected patch
        n = test.n_selected
        h = net.refine(test.patches, test.clusters_dev, n, 0.8)[:n].cpu().numpy()
        assert np.array_equal(h[test.rows], hits)
        # Fig. 6 measure: below 2 px the refined hits recover pairs the
        # centroids merge (the truth has them)
        tr = test.truth
        ht = R.pair_distance_histogram(tr["cx"], tr["cy"], tr["shot"], 2.0, 0.5)
        hc = R.pair_distance_histogram(test.clusters["x"], test.clusters["y"], test.clusters["shot"], 2.0, 0.5)
        hr = R.pair_distance_histogram(*R.hit_list(test, h), 2.0, 0.5)
        assert hc[1:].sum() < 0.2 * ht[1:].sum() and hr[1:].sum() > 0.6 * ht[1:].sum()
    finally:
        ctx.close()
