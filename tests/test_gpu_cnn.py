"""The convolutional refiner on the GPU against the oracle's definition
(oracle/refiner.py, CNN part): bf16 patches equal to the fp32 patches
rounded, the fp32 forward pass, the loss, gradients and Adam steps within fp32
tolerance of the float64 oracle, the tensor-core (tcgen05) inference against
the oracle's inference precision, and training on generator data splitting
merged pairs better than the plain centroid (Sec. V.C) locates them."""
import numpy as np
import pytest

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


def _bf16_bits(a):
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return u.astype(np.uint16)


def _params(seed, scale=0.15):
    return np.random.default_rng(seed).normal(scale=scale, size=orf.cnn_layout()["total"]).astype(np.float32)


def test_bf16_patches_are_the_fp32_patches_rounded(data):
    import torch
    pk, (op, osel, _, _) = data
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    try:
        d = to_device(pk)
        out = ctx.alloc_outputs(pk.size, labels=True, cluster_capacity=max(16, pk.size // 4))
        ctx.tpx_process(d, out)
        assert ctx.tpx_sync(check=False)[0] == 0
        n_cl = int(out["n_clusters"].item())
        p16 = ctx.tpx_refine_patches_bf16(d, out["labels"], out["clusters"], n_cl, 12)
        torch.cuda.synchronize()
        n = int(p16["n"].item())
        assert n == osel.size > 5000
        g = p16["patches"][:n].cpu().numpy().view(np.uint16)
        assert np.array_equal(g, _bf16_bits(op))
        # the patch values are exact in bf16
        back = (g.astype(np.uint32) << 16).view(np.float32)
        assert np.array_equal(back, op)
    finally:
        ctx.close()


@pytest.mark.parametrize("n", [1, 77, 3001])
def test_fp32_forward_matches_oracle(data, n):
    import torch
    op = data[1][0]
    x = np.concatenate([op, np.random.default_rng(n).random((max(0, n - op.shape[0]), 162), np.float32)])[:n]
    p = _params(n)
    ctx = tpx.Context(tpx.Config(), max_packets=16)
    try:
        g = ctx.tpx_cnn_forward(torch.from_numpy(p).cuda(), torch.from_numpy(x).cuda())[:n].cpu().numpy()
    finally:
        ctx.close()
    o = orf.cnn_forward(p.astype(np.float64), x.astype(np.float64))
    assert np.abs(g - o).max() <= 1e-4 * max(1.0, np.abs(o).max())


def _targets(n, seed):
    rng = np.random.default_rng(seed)
    y = np.zeros((n, 5), np.float32)
    y[:, 0] = rng.integers(1, 3, n)
    y[:, 1:] = rng.normal(size=(n, 4))
    return y


@pytest.mark.parametrize("n", [512, 37])
def test_train_steps_match_oracle(data, n):
    import torch
    x = data[1][0][:n]
    y = _targets(n, 5)
    p0 = _params(7, 0.1)
    w, lr = 0.8, 1e-3
    ctx = tpx.Context(tpx.Config(), max_packets=16)
    try:
        P = torch.from_numpy(p0.copy()).cuda()
        m, v, gr = torch.zeros_like(P), torch.zeros_like(P), torch.zeros_like(P)
        work = torch.empty(int(tpx.lib().tpx_cnn_work_floats(n)), dtype=torch.float32, device="cuda")
        loss = torch.zeros(2, dtype=torch.float32, device="cuda")
        X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ctx.tpx_cnn_train_step(P, m, v, gr, 1, X, Y, lr, w, work, loss[0:])
        torch.cuda.synchronize()
        g1, p1, m1, v1 = gr.cpu().numpy(), P.cpu().numpy(), m.cpu().numpy(), v.cpu().numpy()
        ctx.tpx_cnn_train_step(P, m, v, gr, 2, X, Y, lr, w, work, loss[1:])
        torch.cuda.synchronize()
        l = loss.cpu().numpy()
        p2 = P.cpu().numpy()
    finally:
        ctx.close()
    pd = p0.astype(np.float64)
    og = orf.cnn_grad(pd, x, y, w)
    assert abs(l[0] - orf.cnn_loss(pd, x, y, w)) <= 1e-5 * abs(l[0]) + 1e-6
    gs = np.abs(og).max()
    # split-K sums in fp32 over up to 25,000 rows (atomic order): 2e-4 of the scale
    assert np.abs(g1 - og).max() <= 2e-4 * gs
    assert np.allclose(m1, 0.1 * og, rtol=0, atol=2e-5 * gs)
    op1, _, _ = orf.adam(pd, 0, 0, og, 1, lr)
    big = np.abs(og) > 1e-2 * gs
    assert np.abs(p1 - op1)[big].max() <= 1e-6 + 1e-3 * lr
    og2 = orf.cnn_grad(p1.astype(np.float64), x, y, w)
    assert abs(l[1] - orf.cnn_loss(p1.astype(np.float64), x, y, w)) <= 1e-5 * abs(l[1]) + 1e-6
    op2, _, _ = orf.adam(p1.astype(np.float64), m1.astype(np.float64), v1.astype(np.float64), og2, 2, lr)
    big2 = big & (np.abs(og2) > 1e-2 * np.abs(og2).max())
    assert np.abs(p2 - op2)[big2].max() <= 1e-6 + 2e-3 * lr


@pytest.mark.parametrize("n", [4099, 128, 1, 20_000])
def test_tensor_core_inference_matches_oracle(data, n):
    """tcgen05 implicit GEMMs against the oracle's inference precision. The
    GPU sums in fp32 in tensor memory, the oracle exactly, so a hidden
    activation can round to the neighbouring bf16 value in a few rows: nearly
    all rows agree to 1e-3 of the output scale, every row to 5e-2."""
    import torch
    op = data[1][0]
    x = np.concatenate([op, np.random.default_rng(n).random((max(0, n - op.shape[0]), 162), np.float32)])[:n]
    xb = _bf16_bits(x)
    p = _params(n + 1)
    ctx = tpx.Context(tpx.Config(), max_packets=16)
    try:
        packed = ctx.tpx_cnn_pack(torch.from_numpy(p).cuda())
        XB = torch.from_numpy(xb.view(np.int16)).cuda()
        g = ctx.tpx_cnn_infer(packed, XB)[:n].cpu().numpy().astype(np.float64)
        assert ctx.tpx_sync(check=False)[0] == 0
    finally:
        ctx.close()
    o = orf.cnn_forward_bf16(p, (xb.astype(np.uint32) << 16).view(np.float32))
    scale = max(1.0, np.abs(o).max())
    row_err = np.abs(g - o).max(axis=1)
    assert np.mean(row_err <= 1e-3 * scale) >= 0.95, np.sort(row_err)[-10:]
    assert row_err.max() <= 5e-2 * scale


def test_cnn_training_splits_merged_pairs():
    ctx = tpx.Context(tpx.Config(), max_packets=1 << 20)
    try:
        train = R.make_dataset(ctx, synth.refiner(n_shots=3000, seed=6))
        test = R.make_dataset(ctx, synth.refiner(n_shots=500, seed=7), shuffle_seed=None)
        net = R.CnnRefiner(ctx, seed=0)
        losses = net.train(train, epochs=4, batch=1024, lr=2e-3, lr_final=2e-4)
        assert losses[-20:].mean() < 0.5 * losses[:5].mean()
        hits = net.refine_rows(test, 0.8)
        h32 = net.refine_rows(test, 0.8, fp32=True)
        assert np.mean(h32[:, 0] == hits[:, 0]) > 0.99
        ev = R.evaluate(test, hits)
        assert ev["pair_recall"] > 0.6 and ev["single_split"] < 0.05
        assert ev["pair_err_refined"] < 0.7 * ev["pair_err_centroid"]
        n = test.n_selected
        h = net.refine(test.patches16, test.clusters_dev, n, 0.8)[:n].cpu().numpy()
        assert np.array_equal(h[test.rows], hits)
    finally:
        ctx.close()
