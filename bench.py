#!/usr/bin/env python
"""Benchmark: pixel hits/s clustered and centroided, as a fraction of HBM peak.

Workload (one GPU): the large batch -- 10^6 laser shots at 1 kHz, Poisson(50)
particles per shot, 5% planted as overlapping pairs, Gaussian charge clouds of
sigma 1 px with ToT >= 10 (about 1.27e9 packets, 10 GB, read from HBM once per
step). A step is one pass of the whole path (decode, unwrap, shot binning and
cut, clustering, local maxima, centroids, per-pixel labels) over the batch.

Prints one JSON line. `--impl reference` times the CPU oracle instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pixel hits/s clustered+centroided"
UNIT = "hits/s"
CLUSTER_BYTES = 88        # tpx_record as written
ALG_CLUSTER_BYTES = 56    # the per-cluster sums the method must write: label, t0, shot, n, 4 sums, n_peaks
KERNEL_SRC = [os.path.join(ROOT, "paper_2603_04942_gb300", "csrc", f) for f in ("tpx_fused.cu", "tpx_fused_body.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fused_kernel_large_batch.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--shots", type=int, default=1_000_000)
    ap.add_argument("--variant", choices=["literal", "stated"], default="literal")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--parity-shots", type=int, default=10_000,
                    help="shots per range of the sampled oracle check of the timed call")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-shots", type=int, default=50_000)
    ap.add_argument("--cpu-shots-per-core", type=int, default=10_000)
    ap.add_argument("--ref-shots", type=int, default=10_000)
    ap.add_argument("--tile", choices=["default", "4096", "2048"], default="default",
                    help="fused-kernel tile geometry (speed only; results are identical)")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-timewalk", action="store_true")
    ap.add_argument("--no-refiner", action="store_true")
    ap.add_argument("--refiner-only", action="store_true")
    ap.add_argument("--refiner-shots", type=int, default=500_000, help="training shots (about 20 clusters each)")
    ap.add_argument("--refiner-epochs", type=int, default=1)
    ap.add_argument("--phase-shares", type=int, default=0, metavar="SHOTS",
                    help="per-phase cycle shares of the fused kernel (instrumented build) on SHOTS shots of the "
                         "large recipe, --tile geometry (2048 when default)")
    ap.add_argument("--cnn-phase-shares", type=int, default=0, metavar="N",
                    help="per-phase cycle shares of the CNN inference kernel (instrumented build) on N patches")
    ap.add_argument("--cnn-infer-only", type=int, default=0, metavar="N",
                    help="time only the CNN refiner's tcgen05 inference on N random bf16 patches (random weights)")
    ap.add_argument("--batch-runs", type=int, default=4096)
    ap.add_argument("--batch-only", action="store_true")
    ap.add_argument("--big-shot-batch", type=int, default=0, metavar="RUNS",
                    help="time one batch of RUNS ion runs whose shots all take the big-range path")
    ap.add_argument("--batch-phase-shares", type=int, default=0, metavar="RUNS",
                    help="per-phase cycle shares of the batch kernel on the first RUNS runs (instrumented build)")
    ap.add_argument("--batch-steps", type=int, default=3, help="timed whole calls of the batch (each ~5 s)")
    ap.add_argument("--stream-only", action="store_true")
    ap.add_argument("--stream-chunks", type=int, default=150)
    ap.add_argument("--stream-rates", type=str, default="10,40,80")
    return ap.parse_args()


def workload(args, rank=0):
    """One acquisition (seed 1) of args.shots shots per GPU: rank r takes shots
    [r * shots, (r + 1) * shots), the packets from its first trigger packet to
    the next rank's (weak scaling: the work per GPU is fixed)."""
    import synth
    p = synth.large(n_shots=args.shots, seed=1, shot_begin=rank * args.shots)
    if args.variant == "stated":
        p = synth.stated_size(p)
    desc = (f"large batch: {args.shots:,} shots at 1 kHz x Poisson(50) particles, 5% overlapping pairs "
            f"(sep 0-4 px, dToA 0-20 ns, amp 0.3-1), sigma 1 px, peak ToT 200-1023, "
            f"ToT >= {int(p.tot_min)} ({args.variant} parameters), ToF 1-10 us, seed {p.seed}")
    return p, desc


def shard_start(ctx, d_pk, n: int, world: int):
    """A rank's starting unwrap state and stream index base: one all_gather of
    every rank's unwrap summary of its range (8 int64) and packet count, then
    the in-order combination of its predecessors' (no packets cross ranks).
    Rank 0 starts the stream (no state)."""
    if world == 1:
        return None, 0
    import torch
    import torch.distributed as dist

    from paper_2603_04942_gb300 import shard
    state, _ = shard.exchange_states(ctx.tpx_summarize(d_pk, n))
    sizes = [torch.zeros(1, dtype=torch.int64, device=d_pk.device) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([n], dtype=torch.int64, device=d_pk.device))
    rank = dist.get_rank()
    base = int(sum(int(x.item()) for x in sizes[:rank]))
    return (state if rank > 0 else None), base


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def profile_per_packet(key: str = "dram_bytes_per_packet"):
    """A per-packet figure of the fused kernel (DRAM bytes, warp
    instructions) from the committed ncu summary, if it was taken on the
    current kernel source."""
    try:
        txt = open(TRAFFIC_FILE).read()
        sha = hashlib.sha256(b"".join(open(f, "rb").read() for f in KERNEL_SRC)).hexdigest()[:16]
        m_sha = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
        m_b = re.search(key + r":\s*([0-9.]+)", txt)
        if m_sha and m_b and m_sha.group(1) == sha:
            return float(m_b.group(1))
    except Exception:
        pass
    return None


def oracle_timed(p, shot_begin: int, n_shots: int) -> tuple[float, int, int]:
    """Generate shots [shot_begin, shot_begin + n_shots) of workload `p` and
    time the oracle on them (generation untimed). A slice that starts after
    wraps is given its wrap counts, so it computes the same as the full run."""
    import oracle
    import synth
    st = synth.Stream(p.replace(shot_begin=shot_begin, n_shots=n_shots))
    pk = st.packets()
    e_pix, e_tdc = st.wrap_counts()
    st.close()
    hits = int(((pk >> np.uint64(60)) == 0xB).sum())
    cfg = oracle.Config(epoch0_pix=e_pix, epoch0_tdc=e_tdc)
    t0 = time.perf_counter()
    r = oracle.run(pk, cfg)
    dt = time.perf_counter() - t0
    assert r["status"] == 0, r["status"]
    return dt, hits, pk.size


FIRST_TDC_WRAP_SHOT = 81_031   # first trigger at or after 2^36 ticks on the recipe's time line


def sample_ranges(n_shots: int, k: int) -> list[tuple[int, int]]:
    """Shot ranges of k shots checked against the oracle: the start of the
    stream (the first pixel wrap, shot 500), the first TDC wrap (also a pixel
    wrap), and the end of the stream (the last tiles)."""
    k = min(k, n_shots)
    want = [0, FIRST_TDC_WRAP_SHOT - k // 2, n_shots - k]
    out = []
    for s0 in want:
        s0 = max(0, min(s0, n_shots - k))
        if (s0, s0 + k) not in out:
            out.append((s0, s0 + k))
    return out


def parity_sampled(p, h_pk, d_pk, out, n_cl: int, n_shots: int, k: int) -> dict:
    """The timed call's outputs against the oracle on sampled shot ranges.
    A range [s0, s1) is the packets from trigger s0's TDC packet to trigger
    s1's; it is regenerated independently (and must equal that part of the
    stream), and the oracle runs on it from the wrap counts at its start. The
    triggers of the range, the records of its shots (all but the last, whose
    late pixels may follow the range) and the labels of their pixels must
    equal the oracle's: integers bit for bit, centroids within 1e-6."""
    import torch

    import oracle
    import paper_2603_04942_gb300 as tpx
    import synth
    oracle.build()
    tdc_pos = torch.nonzero((d_pk >> 60) == 6).flatten().cpu().numpy()
    assert tdc_pos.size == n_shots, (tdc_pos.size, n_shots)
    rec_i64 = out["clusters"][: n_cl * CLUSTER_BYTES].view(torch.int64).view(n_cl, CLUSTER_BYTES // 8)
    rec_label = rec_i64[:, 0].contiguous()
    a_pk = h_pk.numpy().view(np.uint64)
    n = a_pk.size
    res = {"ranges": [], "ok": True, "records": 0, "labels": 0, "triggers": 0}
    for s0, s1 in sample_ranges(n_shots, k):
        a = 0 if s0 == 0 else int(tdc_pos[s0])
        b = n if s1 >= n_shots else int(tdc_pos[s1])
        st = synth.Stream(p.replace(shot_begin=s0, n_shots=s1 - s0))
        pk = st.packets()
        e_pix, e_tdc = st.wrap_counts()
        st.close()
        ok = pk.size == b - a and np.array_equal(pk, a_pk[a:b])
        o = oracle.run(pk, oracle.Config(epoch0_pix=e_pix, epoch0_tdc=e_tdc), idx_base=a)
        ok = ok and o["status"] == 0
        last = s1 - 1 if s1 >= n_shots else s1 - 2      # the last shot compared
        # triggers
        g_tr = out["trig"][s0:s1].cpu().numpy()
        ok = ok and np.array_equal(g_tr, o["triggers"])
        # records of shots [s0, last]: their labels lie in [a, b)
        i0, i1 = (int(v) for v in torch.searchsorted(rec_label, torch.tensor([a, b], device=rec_label.device)))
        g_cl = np.frombuffer(out["clusters"][i0 * CLUSTER_BYTES: i1 * CLUSTER_BYTES].cpu().numpy().tobytes(),
                             tpx.CLUSTER_DTYPE)
        g_cl = g_cl[(g_cl["shot"] >= s0) & (g_cl["shot"] <= last)]
        o_cl = o["clusters"].copy()
        o_cl["shot"] += s0
        o_cl = o_cl[o_cl["shot"] <= last]
        ok = ok and g_cl.size == o_cl.size and g_cl.size > 0
        if ok:
            for f in ("label", "shot", "t0", "s_tot", "s_x", "s_y", "s_t", "n", "n_peaks"):
                ok = ok and np.array_equal(g_cl[f], o_cl[f])
            for f in ("x", "y", "tof"):
                ok = ok and bool(np.all(np.abs(g_cl[f] - o_cl[f]) <= 1e-6))
        # labels of the pixels of those records
        g_lab = out["labels"][a:b].cpu().numpy()
        o_lab = o["labels"]
        sel = o_lab >= 0
        pos = np.searchsorted(o_cl["label"], o_lab[sel])
        inside = (pos < o_cl.size) & (o_cl["label"][np.minimum(pos, max(o_cl.size - 1, 0))] == o_lab[sel])
        m = np.zeros(o_lab.size, bool)
        m[np.flatnonzero(sel)[inside]] = True
        ok = ok and bool(np.array_equal(g_lab[m], o_lab[m])) and int(m.sum()) > 0
        res["ranges"].append({"shots": [s0, s1], "packets": [a, b], "records": int(o_cl.size),
                              "labels": int(m.sum()), "wraps_at_start": [int(e_pix), int(e_tdc)], "ok": bool(ok)})
        res["records"] += int(o_cl.size)
        res["labels"] += int(m.sum())
        res["triggers"] += int(g_tr.size)
        res["ok"] = res["ok"] and bool(ok)
    return res


def cpu_baseline(args, sample_shots: int) -> dict:
    """The oracle as it stands, single-threaded, on the first shots of the
    same workload, in chunks of 25,000 shots."""
    import oracle
    oracle.build()
    p, _ = workload(args)
    tot_t, tot_h, tot_p = 0.0, 0, 0
    for b in range(0, sample_shots, 25_000):
        dt, h, n = oracle_timed(p, b, min(25_000, sample_shots - b))
        tot_t += dt
        tot_h += h
        tot_p += n
    return {"value": tot_h / tot_t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {sample_shots:,} shots of the workload ({tot_h:,} pixel hits, {tot_p:,} packets) "
                      f"in 25,000-shot calls, {tot_t:.1f} s single-threaded"}


def _oracle_worker(p, shot_begin, n_shots, barrier, out_q):
    """One process of the parallel CPU baseline: generate its shot range
    (untimed), wait for the others, time the oracle on it."""
    import oracle
    import synth
    st = synth.Stream(p.replace(shot_begin=shot_begin, n_shots=n_shots, n_threads=1))
    pk = st.packets()
    e_pix, e_tdc = st.wrap_counts()
    st.close()
    hits = int(((pk >> np.uint64(60)) == 0xB).sum())
    cfg = oracle.Config(epoch0_pix=e_pix, epoch0_tdc=e_tdc)
    barrier.wait()
    t0 = time.perf_counter()
    r = oracle.run(pk, cfg)
    out_q.put((time.perf_counter() - t0, hits, int(r["status"])))


def cpu_baseline_parallel(args, shots_per_core: int) -> dict:
    """The same oracle on every host core at once: one process per core,
    each on its own range of shots (shots are independent; each range gets
    its wrap counts), started together; throughput = all hits / the slowest
    process's time."""
    import multiprocessing as mp

    import oracle
    oracle.build()
    p, _ = workload(args)
    n = min(64, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(n)
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(p, k * shots_per_core, shots_per_core, barrier, q))
             for k in range(n)]
    for pr in procs:
        pr.start()
    res = [q.get() for _ in procs]
    for pr in procs:
        pr.join()
    assert all(r[2] == 0 for r in res)
    wall = max(r[0] for r in res)
    hits = sum(r[1] for r in res)
    return {"value": hits / wall, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{n} processes x {shots_per_core:,} shots of the workload ({hits:,} pixel hits), one "
                      f"single-threaded oracle per core started together, slowest {wall:.1f} s"}


def stream_bench(args) -> dict:
    """Streaming: a continuous ion-like stream (ToF over the whole 1 ms
    period) at each rate, cut into chunks of U[1,100] ms of acquisition time
    at arbitrary packets; each chunk is submitted from pinned host memory and
    polled at once (service latency = submit entry to records on the host)."""
    import torch

    import paper_2603_04942_gb300 as tpx
    import synth
    out = {"workload": "continuous ion-like stream, 1 kHz triggers, sigma 1.2 px, ToF uniform over the 1 ms "
                       "period (cut at the full period), chunks of U[1,100] ms of acquisition time cut at "
                       "arbitrary packets, hold 2 shots open, general path", "rates": {}}
    rng = np.random.default_rng(3)
    for rate_m in [float(r) for r in args.stream_rates.split(",") if r]:
        durs = rng.uniform(1.0, 100.0, size=args.stream_chunks)
        n_shots = int(np.ceil(durs.sum())) + 3
        st = synth.Stream(synth.streaming(rate_m * 1e6, n_shots))
        n = st.n_packets
        h = torch.empty(n, dtype=torch.int64, pin_memory=True)
        pk = st.packets_into(h.numpy().view(np.uint64))
        st.close()
        tdc = np.flatnonzero((pk >> np.uint64(60)) == 6)
        # chunk ends at arbitrary packets: interpolate between trigger packets
        ends_ms = np.cumsum(durs)
        k = np.floor(ends_ms).astype(np.int64)
        frac = ends_ms - k
        cut = tdc[np.minimum(k, tdc.size - 2)] + (frac * (tdc[np.minimum(k + 1, tdc.size - 1)]
                                                           - tdc[np.minimum(k, tdc.size - 2)])).astype(np.int64)
        cut = np.minimum(np.maximum.accumulate(cut), n)
        cut[-1] = n
        sizes = np.diff(np.r_[0, cut])
        cfg = tpx.Config(tof_max_ticks=synth.STREAM_TOF_MAX_TICKS)
        s = tpx.Stream(cfg, max_chunk_packets=int(sizes.max()), max_hold_packets=int(4 * n / n_shots) + 65536,
                       hold_triggers=2, slots=2)
        # warm-up on a copy of the first chunks in a separate stream object
        w = tpx.Stream(cfg, max_chunk_packets=int(sizes.max()), max_hold_packets=int(4 * n / n_shots) + 65536,
                       hold_triggers=2, slots=2)
        pos = 0
        for c in sizes[:3]:
            w.poll(w.submit(pk[pos:pos + c]))
            pos += c
        w.close()
        lat, hits_done, clusters = [], 0, 0
        pos = 0
        t_all0 = time.perf_counter()
        for c in sizes:
            r = s.poll(s.submit(pk[pos:pos + c]))
            lat.append(r["latency_us"])
            clusters += r["clusters"].size
            pos += c
        r = s.poll(s.finish())
        clusters += r["clusters"].size
        wall = time.perf_counter() - t_all0
        s.close()
        hits = int(((pk >> np.uint64(60)) == 0xB).sum())
        lat = np.array(lat)
        acq_s = float(durs.sum()) / 1e3
        out["rates"][f"{rate_m:g} Mhit/s"] = {
            "chunks": int(sizes.size), "packets": int(n), "pixel_hits": hits, "clusters": int(clusters),
            "latency_us": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "p99.9": float(np.percentile(lat, 99.9)), "max": float(lat.max())},
            "sustained_hits_per_s": hits / wall, "acquisition_s": acq_s, "processing_s": wall,
            "realtime_factor": acq_s / wall}
    return out


def batch_bench(args) -> dict:
    """Uneven batch: independent runs (log-uniform shots and particles per
    shot, electron- or ion-like) concatenated on the device and processed by
    one tpx_process_batch launch per step; device-resident, CUDA events."""
    import torch

    import paper_2603_04942_gb300 as tpx
    import synth
    runs = synth.batched(n_runs=args.batch_runs)
    t0 = time.perf_counter()
    parts, sizes, staging = [], [], None
    for p in runs:
        st = synth.Stream(p)
        n = st.n_packets
        if staging is None or staging.numel() < n:
            staging = torch.empty(max(n, 1 << 24), dtype=torch.int64, pin_memory=True)
        st.packets_into(staging.numpy().view(np.uint64))
        st.close()
        parts.append(staging[:n].to("cuda", non_blocking=False))
        sizes.append(n)
    del staging
    d_pk = torch.cat(parts) if parts else torch.zeros(2, dtype=torch.int64, device="cuda")
    del parts
    torch.cuda.empty_cache()
    gen_s = time.perf_counter() - t0
    offs = np.zeros(len(runs) + 1, np.int64)
    offs[1:] = np.cumsum(sizes)
    n = int(offs[-1])
    shots = sum(p.n_shots for p in runs)
    expect = sum(p.n_shots * p.particles_per_shot for p in runs)
    s = torch.cuda.Stream()   # a stream of its own: the call is also captured into a CUDA graph below
    ctx = tpx.Context(tpx.Config(), max_packets=max(1, n), stream=s)
    out = ctx.alloc_batch_outputs(n, len(runs), labels=False, is_peak=False,
                                  cluster_capacity=int(1.3 * expect) + (1 << 20), trig_capacity=shots + 16)
    torch.cuda.synchronize()
    for _ in range(max(3, min(args.warmup, 3))):
        ctx.tpx_process_batch(d_pk, offs, out)
        rc, counters = ctx.tpx_sync(check=False)
        if rc != 0:
            raise SystemExit(f"tpx_process_batch failed in warm-up: {rc} {counters}")
    # a step is the whole call: the launch and the tpx_sync that redoes the
    # runs the tiles could not hold (host wall clock, device synchronised)
    steps = args.batch_steps
    step_ms = []
    torch.cuda.synchronize()
    for k in range(steps):
        t0 = time.perf_counter()
        ctx.tpx_process_batch(d_pk, offs, out)
        rc, counters = ctx.tpx_sync(check=False)
        torch.cuda.synchronize()
        step_ms.append(1e3 * (time.perf_counter() - t0))
        assert rc == 0, rc
    total_ms = sum(step_ms)
    # the tiles' pass alone (one launch, CUDA events), for the split
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(s)
    ctx.tpx_process_batch(d_pk, offs, out)
    ev1.record(s)
    torch.cuda.synchronize()
    tiles_ms = ev0.elapsed_time(ev1)
    rc2, _ = ctx.tpx_sync(check=False)
    assert rc2 == 0, rc2
    # the same call captured once into a CUDA graph, then replayed (the run
    # tables' upload and the persistent kernel), each replay with its tpx_sync
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
        ctx.tpx_process_batch(d_pk, offs, out)
    graph_ms = []
    for k in range(steps):
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            g.replay()
        rc3, c3 = ctx.tpx_sync(check=False)
        torch.cuda.synchronize()
        graph_ms.append(1e3 * (time.perf_counter() - t0))
        assert rc3 == 0 and c3["redone"] == counters["redone"], (rc3, c3)
    assert int(out["n_clusters"].item()) > 0
    del g
    tune = ctx.tpx_tuning()
    n_cl = int(out["n_clusters"].item())
    res = {"workload": f"{len(runs)} independent runs, one launch per step: shots log-uniform 10-10^4, Poisson "
                       "particles per shot with a mean log-uniform 1-500, electron-like (sigma 0.6 px, ToF 0-50 ns) "
                       "or ion-like (sigma 1.2 px, ToF 1-20 us), seed 2",
           "metric": "pixel hits/s clustered+centroided", "unit": "hits/s",
           "value": counters["pixels"] * steps / (total_ms / 1e3), "ms_per_step": total_ms / steps,
           "timing": "wall clock per whole call (launch + tpx_sync, redone runs included), device synchronised",
           "tiles_pass_ms": tiles_ms,
           "graph": {"ms_per_step": sum(graph_ms) / steps,
                     "value": counters["pixels"] * steps / (sum(graph_ms) / 1e3),
                     "timing": "the call captured once into a CUDA graph; per step one replay + tpx_sync"},
           "runs": len(runs), "shots": shots, "packets": n, "pixel_hits": counters["pixels"], "clusters": n_cl,
           "redone_runs": counters["redone"], "steps": steps, "warmup": 3,
           "tile_geometry": {1: "4096-packet tiles", 2: "2048-packet tiles"}.get(tune["tile_geometry"], "sampling"),
           "generation_s": round(gen_s, 1)}
    ctx.close()
    del d_pk, out
    torch.cuda.empty_cache()
    return res


def timewalk_bench(args) -> dict:
    """Timewalk calibration (Sec. IV.C): the GPU ToT-ToF histogram of a
    calibration run (one ion peak, a known delay model) timed with CUDA
    events, then the host fits of Eq. 1."""
    import torch

    import paper_2603_04942_gb300 as tpx
    import synth
    from paper_2603_04942_gb300 import timewalk as tw
    p = synth.calibration(n_shots=20_000)
    pk = synth.generate(p)[0]
    d = torch.from_numpy(pk.view(np.int64)).cuda()
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    dec = ctx.tpx_decode(d)
    ctx.tpx_sync()
    nh = int(dec["n_hits"].item())
    lo, nb = synth.CALIBRATION_TOF_TICKS - 10, 128
    hist = ctx.tpx_tot_tof_histogram(dec["hits"], nh, lo, 1, nb)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(ctx.stream)
    for _ in range(reps):
        ctx.tpx_tot_tof_histogram(dec["hits"], nh, lo, 1, nb, hist=hist)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    t0 = time.perf_counter()
    fit, _ = tw.calibrate(ctx, dec["hits"], nh, lo, 1, nb, fix_d=True)
    fit_s = time.perf_counter() - t0
    ctx.close()
    return {"workload": "calibration run: 20,000 shots x 20 particles at one ToF (5 us), ToA delay "
                        "1500 / (ToT + 5) + 10 ns per pixel, seed 4",
            "hits": nh, "histogram_ms": ms, "histogram_hits_per_s": nh / (ms / 1e3), "calibration_s": fit_s,
            "fit_ticks": {"a": fit.a, "b": fit.b, "c": fit.c, "d": fit.d, "rms": fit.rms},
            "truth_ticks": {"a": p.timewalk_a / 1.5625, "b": p.timewalk_b,
                            "c": synth.CALIBRATION_TOF_TICKS + p.timewalk_c / 1.5625, "d": 1.0}}


def phase_bench(shots: int, tile: str) -> dict:
    """Per-phase cycle shares of the fused kernel on `shots` shots of the
    large recipe (the instrumented library must be loaded): two untimed calls,
    then one call whose counters are read."""
    import torch

    import paper_2603_04942_gb300 as tpx
    import synth
    geo = tpx.TILE_4096 if tile == "4096" else tpx.TILE_2048
    pk = synth.generate(synth.large(n_shots=shots))[0]
    d = torch.from_numpy(pk.view(np.int64)).cuda()
    ctx = tpx.Context(tpx.Config(tile_geometry=geo), max_packets=pk.size)
    out = ctx.alloc_outputs(pk.size, True, False, pk.size // 8, shots + 16)
    for _ in range(2):
        ctx.tpx_process(d, out)
    ctx.tpx_sync()
    tpx.phase_times(geo, clear=True)
    ctx.tpx_process(d, out)
    ctx.tpx_sync()
    cyc = tpx.phase_times(geo, clear=True).astype(np.float64)
    ctx.close()
    return {"metric": "fused-kernel phase shares (warp cycles, barrier waits included)", "packets": int(pk.size),
            "tile_geometry": tile if tile != "default" else "2048",
            "shares": {nm: round(float(c / cyc.sum()), 4) for nm, c in zip(tpx.PHASE_NAMES, cyc)}}


def big_shot_batch(n_runs: int) -> dict:
    """A batch of ion-like runs whose shots all hold 14k-19k pixels (60 shots
    per run, 400-520 Poisson particles per shot): every range goes through
    the big-range path. One untimed call, then one timed call (wall clock,
    device synchronised)."""
    import torch

    import paper_2603_04942_gb300 as tpx
    import synth
    rng = np.random.default_rng(3)
    pks = []
    for r in range(n_runs):
        p = synth.Params(n_shots=60, seed=77 + r, poisson=True, particles_per_shot=float(400 + 40 * (r % 4)),
                         t_start_ticks=int(rng.integers(0, synth.PIX_PERIOD_TICKS)), **synth.ION)
        pks.append(synth.generate(p)[0])
    offs = np.zeros(len(pks) + 1, np.int64)
    offs[1:] = np.cumsum([x.size for x in pks])
    pk = np.concatenate(pks)
    d = torch.from_numpy(pk.view(np.int64)).cuda()
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    out = ctx.alloc_batch_outputs(pk.size, n_runs, labels=False, is_peak=False, cluster_capacity=pk.size // 4,
                                  trig_capacity=1 << 16)
    ctx.tpx_process_batch(d, offs, out)
    rc, cnt = ctx.tpx_sync(check=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.tpx_process_batch(d, offs, out)
    rc, cnt = ctx.tpx_sync(check=False)
    dt = time.perf_counter() - t0
    ctx.close()
    return {"metric": "pixel hits/s, big-shot batch", "runs": n_runs, "packets": int(pk.size), "status": rc,
            "redone": cnt["redone"], "clusters": cnt["clusters"], "ms": round(dt * 1e3, 3),
            "hits_per_s": cnt["pixels"] / dt}


def batch_phase_bench(n_runs: int) -> dict:
    """Per-phase cycle shares of the batch kernel on the first `n_runs` runs
    of the uneven batch (the instrumented library must be loaded): one
    untimed call, then one call whose counters are read."""
    import torch

    import paper_2603_04942_gb300 as tpx
    import synth
    runs = synth.batched(n_runs=n_runs)
    pks = [synth.generate(p)[0] for p in runs]
    offs = np.zeros(len(pks) + 1, np.int64)
    offs[1:] = np.cumsum([x.size for x in pks])
    pk = np.concatenate(pks)
    del pks
    d = torch.from_numpy(pk.view(np.int64)).cuda()
    ctx = tpx.Context(tpx.Config(), max_packets=pk.size)
    shots = sum(p.n_shots for p in runs)
    expect = sum(p.n_shots * p.particles_per_shot for p in runs)
    out = ctx.alloc_batch_outputs(pk.size, len(runs), labels=False, is_peak=False,
                                  cluster_capacity=int(1.3 * expect) + (1 << 20), trig_capacity=shots + 16)
    ctx.tpx_process_batch(d, offs, out)
    rc, cnt = ctx.tpx_sync(check=False)
    tpx.phase_times(tpx.TILE_4096, clear=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.tpx_process_batch(d, offs, out)
    rc, cnt = ctx.tpx_sync(check=False)
    wall = time.perf_counter() - t0
    cyc = tpx.phase_times(tpx.TILE_4096, clear=True).astype(np.float64)
    ctx.close()
    main, sub = cyc[:20], cyc[20:len(tpx.PHASE_NAMES)]   # the big-range steps lie inside phase 17
    return {"metric": "batch-kernel phase shares (warp cycles, barrier waits included)", "runs": n_runs,
            "packets": int(pk.size), "status": rc, "redone": cnt["redone"], "wall_s_instrumented": round(wall, 3),
            "shares": {nm: round(float(c / main.sum()), 4) for nm, c in zip(tpx.PHASE_NAMES[:20], main)},
            "big_range_steps": {nm: round(float(c / max(main[17], 1.0)), 4)
                                for nm, c in zip(tpx.PHASE_NAMES[20:], sub)}}


CNN_FLOPS_PER_PATCH = 2 * (49 * 18 * 16 + 25 * 144 * 16 + 9 * 144 * 32 + 288 * 144 + 144 * 6)


def cnn_infer_bench(n: int, steps: int, warmup: int, phases: bool = False) -> dict:
    """The CNN refiner's inference alone: n patches of bf16 values in [0, 2),
    weights N(0, 0.1), both seeded; `steps` timed calls after `warmup`."""
    import numpy as np
    import torch

    import paper_2603_04942_gb300 as tpx
    ctx = tpx.Context(tpx.Config(), max_packets=16)
    w = np.random.default_rng(0).normal(scale=0.1, size=tpx.Context.tpx_cnn_params()).astype(np.float32)
    x32 = np.random.default_rng(1).random((n, 162), np.float32) * 2
    x16 = (x32.view(np.uint32) >> np.uint32(16)).astype(np.uint16).view(np.int16)
    packed = ctx.tpx_cnn_pack(torch.from_numpy(w).cuda())
    x = torch.from_numpy(x16).cuda()
    out = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    work = torch.empty(int(tpx.lib().tpx_cnn_infer_work_bytes(n)), dtype=torch.uint8, device="cuda")
    for _ in range(max(1, warmup)):
        ctx.tpx_cnn_infer(packed, x, n, work=work, out=out)
    torch.cuda.synchronize()
    if phases:
        tpx.cnn_phase_times(clear=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(steps):
        ctx.tpx_cnn_infer(packed, x, n, work=work, out=out)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rc, _ = ctx.tpx_sync(check=False)
    ctx.close()
    if phases:
        cyc = tpx.cnn_phase_times(clear=True).astype(np.float64)
        return {"metric": "CNN inference phase shares (thread 0 cycles per CTA)", "patches": n,
                "shares": {nm: round(float(c / cyc.sum()), 4) for nm, c in zip(tpx.CNN_PHASE_NAMES, cyc)},
                "cycles_per_group": float(cyc.sum() / ((n + 47) // 48) / steps), "status": rc}
    return {"metric": "CNN refiner inference", "patches": n, "ms_per_call": ms, "patches_per_s": n / (ms / 1e3),
            "tflops": CNN_FLOPS_PER_PATCH * n / (ms / 1e3) / 1e12, "status": rc, "steps": steps, "warmup": warmup}


def refiner_bench(args) -> dict:
    """The learned overlap refiner: a training set of generator clusters
    with planted pairs (seed 6), one pass of minibatch Adam, then the errors
    on a held-out set (seed 7) against the generator's truth next to the
    plain centroid's, and the inference throughput (patch extraction,
    network, decision) timed with CUDA events."""
    import torch

    import paper_2603_04942_gb300 as tpx
    import synth
    from paper_2603_04942_gb300 import refiner as R
    ctx = tpx.Context(tpx.Config(), max_packets=1 << 20)
    t0 = time.perf_counter()
    train = R.make_dataset(ctx, synth.refiner(n_shots=args.refiner_shots, seed=6))
    test = R.make_dataset(ctx, synth.refiner(n_shots=max(2000, args.refiner_shots // 25), seed=7), shuffle_seed=None)
    data_s = time.perf_counter() - t0
    net = R.Refiner(ctx, hidden=R.HIDDEN, seed=0)
    t0 = time.perf_counter()
    losses = net.train(train, epochs=args.refiner_epochs, batch=4096, lr=2e-3, lr_final=1e-4)
    train_s = time.perf_counter() - t0
    thr = 0.8
    ev = R.evaluate(test, net.refine_rows(test, thr))
    ev32 = R.evaluate(test, net.refine_rows(test, thr, fp32=True))
    # resolving power as the paper's Fig. 6 measures it: pairwise distances of
    # the hits of each shot, for the generator's particles, the plain
    # centroids and the refined hits
    h_all = net.refine(test.patches, test.clusters_dev, test.n_selected, thr)[: test.n_selected].cpu().numpy()
    tr = test.truth
    bins = 0.25
    hist = {"bin_px": bins,
            "truth": R.pair_distance_histogram(tr["cx"], tr["cy"], tr["shot"], 4.0, bins).tolist(),
            "centroid": R.pair_distance_histogram(test.clusters["x"], test.clusters["y"], test.clusters["shot"],
                                                  4.0, bins).tolist(),
            "refined": R.pair_distance_histogram(*R.hit_list(test, h_all), 4.0, bins).tolist()}
    # inference on every selected cluster of the training stream: patches from
    # the fused path's outputs, the network, the decision
    pk = synth.Stream(synth.refiner(n_shots=args.refiner_shots, seed=6))
    host = pk.packets()
    pk.close()
    d = torch.from_numpy(host.view(np.int64)).cuda()
    del host
    n = d.numel()
    out = ctx.alloc_outputs(n, labels=True)
    ctx.tpx_process(d, out)
    ctx.tpx_sync()
    n_cl = int(out["n_clusters"].item())
    pt = ctx.tpx_refine_patches(d, out["labels"], out["clusters"], n_cl, R.MIN_PIXELS)
    ns = int(pt["n"].item())
    o6 = torch.empty((ns, 6), dtype=torch.float32, device="cuda")
    hits = torch.empty((ns, 5), dtype=torch.float32, device="cuda")
    net.infer(pt["patches"], ns, o6)          # packs the bf16 weights
    for _ in range(2):
        ctx.tpx_refiner_infer(net.packed, net.h, pt["patches"], ns, o6)
        ctx.tpx_refine_decide(o6, out["clusters"], pt["sel"], pt["centre"], ns, thr, hits)
    torch.cuda.synchronize()
    reps = 5
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    tot = [0.0, 0.0, 0.0]
    for _ in range(reps):
        e[0].record(ctx.stream)
        pt2 = ctx.tpx_refine_patches(d, out["labels"], out["clusters"], n_cl, R.MIN_PIXELS)   # synchronises (count)
        e[1].record(ctx.stream)
        ctx.tpx_refiner_infer(net.packed, net.h, pt2["patches"], ns, o6)
        e[2].record(ctx.stream)
        ctx.tpx_refine_decide(o6, out["clusters"], pt2["sel"], pt2["centre"], ns, thr, hits)
        e[3].record(ctx.stream)
        torch.cuda.synchronize()
        for k in range(3):
            tot[k] += e[k].elapsed_time(e[k + 1]) / reps
        del pt2
    # the fp32 network on the same patches, for comparison
    work = torch.empty(2 * ns * R.HIDDEN, dtype=torch.float32, device="cuda")
    ctx.tpx_refiner_forward(net.params, net.h, pt["patches"], ns, work, o6)
    e[0].record(ctx.stream)
    for _ in range(reps):
        ctx.tpx_refiner_forward(net.params, net.h, pt["patches"], ns, work, o6)
    e[1].record(ctx.stream)
    torch.cuda.synchronize()
    fp32_ms = e[0].elapsed_time(e[1]) / reps
    del work
    # the convolutional refiner: trained on the same rows, inferred with
    # tcgen05 implicit GEMMs on bf16 patches
    cnn = R.CnnRefiner(ctx, seed=0)
    t0 = time.perf_counter()
    closses = cnn.train(train, epochs=args.refiner_epochs, batch=4096, lr=2e-3, lr_final=1e-4)
    ctrain_s = time.perf_counter() - t0
    cev = R.evaluate(test, cnn.refine_rows(test, thr))
    cev32 = R.evaluate(test, cnn.refine_rows(test, thr, fp32=True))
    ch_all = cnn.refine(test.patches16, test.clusters_dev, test.n_selected, thr)[: test.n_selected].cpu().numpy()
    hist["refined_cnn"] = R.pair_distance_histogram(*R.hit_list(test, ch_all), 4.0, bins).tolist()
    pt16 = ctx.tpx_refine_patches_bf16(d, out["labels"], out["clusters"], n_cl, R.MIN_PIXELS)
    cnn.infer(pt16["patches"], ns, o6)
    cwork = torch.empty(int(tpx.lib().tpx_cnn_infer_work_bytes(ns)), dtype=torch.uint8, device="cuda")
    for _ in range(2):
        ctx.tpx_cnn_infer(cnn.packed, pt16["patches"], ns, work=cwork, out=o6)
    torch.cuda.synchronize()
    ctot = [0.0, 0.0, 0.0]
    for _ in range(reps):
        e[0].record(ctx.stream)
        p16 = ctx.tpx_refine_patches_bf16(d, out["labels"], out["clusters"], n_cl, R.MIN_PIXELS)   # synchronises (count)
        e[1].record(ctx.stream)
        ctx.tpx_cnn_infer(cnn.packed, p16["patches"], ns, work=cwork, out=o6)
        e[2].record(ctx.stream)
        ctx.tpx_refine_decide(o6, out["clusters"], p16["sel"], p16["centre"], ns, thr, hits)
        e[3].record(ctx.stream)
        torch.cuda.synchronize()
        for k in range(3):
            ctot[k] += e[k].elapsed_time(e[k + 1]) / reps
        del p16
    rc_c, _ = ctx.tpx_sync(check=False)
    ctx.close()
    cflops = CNN_FLOPS_PER_PATCH * ns
    cms = sum(ctot)
    cnn_res = {"network": f"CNN: conv 3x3 2->16->16->32 channels (9x9 -> 3x3), fc 288->144->6, {cnn.n_params:,} "
                          "parameters; trained in fp32, inferred with tcgen05 (bf16 operands, fp32 accumulators in "
                          "tensor memory)",
               "train_s": round(ctrain_s, 2), "train_clusters_per_s": args.refiner_epochs * train.x.shape[0] / ctrain_s,
               "loss_first": float(closses[:10].mean()), "loss_last": float(closses[-10:].mean()), "eval": cev,
               "eval_fp32": {k: cev32[k] for k in ("pair_recall", "single_split", "pair_err_refined", "fallback")},
               "infer": {"clusters": ns, "patches_ms": ctot[0], "network_ms": ctot[1], "decide_ms": ctot[2],
                         "clusters_per_s": ns / (cms / 1e3), "network_tflops": cflops / (ctot[1] / 1e3) / 1e12,
                         "status": rc_c}}
    ms = sum(tot)
    flops = 2 * ns * (162 * net.h + net.h * net.h + net.h * 6)
    return {"workload": f"{args.refiner_shots:,} shots x Poisson(20) ion-like particles, 30% with a planted "
                        "partner (separation 0-4 px, ToA gap 0-20 ns, amplitude ratio 0.3-1), seed 6; "
                        "held-out set seed 7",
            "network": f"162-{net.h}-{net.h}-6 perceptron, {net.n_params:,} parameters; trained in fp32, "
                       "inferred with bf16 operands",
            "train_clusters": int(train.x.shape[0]), "epochs": args.refiner_epochs, "data_s": round(data_s, 1),
            "train_s": round(train_s, 2), "train_clusters_per_s": args.refiner_epochs * train.x.shape[0] / train_s,
            "loss_first": float(losses[:10].mean()), "loss_last": float(losses[-10:].mean()),
            "threshold": thr, "eval": ev,
            "pair_distance_histogram": hist,
            "eval_fp32": {k: ev32[k] for k in ("pair_recall", "single_split", "pair_err_refined", "fallback")},
            "infer": {"clusters": ns, "patches_ms": tot[0], "network_ms": tot[1], "decide_ms": tot[2],
                      "clusters_per_s": ns / (ms / 1e3), "network": "bf16 tensor cores (mma.sync), fp32 sums",
                      "network_tflops": flops / (tot[1] / 1e3) / 1e12,
                      "fp32_network_ms": fp32_ms, "fp32_network_tflops": flops / (fp32_ms / 1e3) / 1e12},
            "cnn": cnn_res}


def run_reference(args):
    """The reference arm: the CPU oracle as it stands, one bounded sample of
    the workload per step (a different shot range each step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    p, desc = workload(args)
    sample = args.ref_shots
    times, hits_tot = [], 0
    for k in range(args.warmup + args.steps):
        dt, hits, _ = oracle_timed(p, (k * sample) % max(1, args.shots - sample), sample)
        if k >= args.warmup:
            times.append(dt)
            hits_tot += hits
    v = hits_tot / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": desc, "sample_shots_per_step": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{sample:,} shots per step, single-threaded CPU oracle"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _section(fn, *a):
    """A secondary part of the line: a failure there is reported in the line
    (and on stderr) instead of losing the main measurement."""
    try:
        return fn(*a)
    except (Exception, SystemExit) as e:   # noqa: BLE001
        import traceback
        traceback.print_exc(file=sys.stderr)
        return {"error": f"{type(e).__name__}: {e}"[:500]}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.phase_shares:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2603_04942_gb300 import build as tbuild
        import paper_2603_04942_gb300 as tpx
        tpx.load(tbuild.build(phases=True))
        print(json.dumps(phase_bench(args.phase_shares, args.tile)), flush=True)
        return 0
    if args.big_shot_batch:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        print(json.dumps(big_shot_batch(args.big_shot_batch)), flush=True)
        return 0
    if args.batch_phase_shares:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2603_04942_gb300 import build as tbuild
        import paper_2603_04942_gb300 as tpx
        tpx.load(tbuild.build(phases=True))
        print(json.dumps(batch_phase_bench(args.batch_phase_shares)), flush=True)
        return 0
    if args.cnn_phase_shares:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2603_04942_gb300 import build as tbuild
        import paper_2603_04942_gb300 as tpx
        tpx.load(tbuild.build(phases=True))
        res = cnn_infer_bench(args.cnn_phase_shares, 1, max(1, args.warmup), phases=True)
        print(json.dumps(res), flush=True)
        return 0
    if args.cnn_infer_only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2603_04942_gb300 import build as tbuild
        tbuild.build()
        print(json.dumps(cnn_infer_bench(args.cnn_infer_only, args.steps, args.warmup)), flush=True)
        return 0
    if args.stream_only or args.batch_only or args.refiner_only:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2603_04942_gb300 import build as tbuild
        tbuild.build()
        f = stream_bench if args.stream_only else batch_bench if args.batch_only else refiner_bench
        print(json.dumps(f(args)), flush=True)
        return 0
    import torch
    import torch.distributed as dist

    import paper_2603_04942_gb300 as tpx
    import synth
    from paper_2603_04942_gb300 import build as tbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    tbuild.build()
    tpx.load()

    p, desc = workload(args, rank)
    t_gen = time.perf_counter()
    st = synth.Stream(p)
    n = st.n_packets
    h_pk = torch.empty(n, dtype=torch.int64, pin_memory=True)
    st.packets_into(h_pk.numpy().view(np.uint64))
    st.close()
    t_gen = time.perf_counter() - t_gen
    hits = int(((h_pk.numpy().view(np.uint64) >> np.uint64(60)) == 0xB).sum())
    d_pk = h_pk.to("cuda", non_blocking=False)

    tile = {"default": tpx.TILE_DEFAULT, "4096": tpx.TILE_4096, "2048": tpx.TILE_2048}[args.tile]
    ctx = tpx.Context(tpx.Config(tile_geometry=tile), max_packets=n)
    cl_cap = max(1024, n // 16)
    out = ctx.alloc_outputs(n, labels=True, is_peak=False, cluster_capacity=cl_cap,
                            trig_capacity=args.shots + 16)
    s = ctx.stream
    state, idx_base = shard_start(ctx, d_pk, n, world)

    def step():
        if state is not None:
            ctx.tpx_set_state(state)
        ctx.tpx_process(d_pk, out, idx_base)

    for _ in range(args.warmup):
        step()
    rc, counters = ctx.tpx_sync(check=False)
    if rc != 0:
        raise SystemExit(f"tpx_process failed in warm-up: {rc} {counters}")
    n_cl = int(out["n_clusters"].item())
    n_tr = int(out["n_trig"].item())
    tuning = ctx.tpx_tuning()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ctx.tpx_kernel_timing(True)   # events on the launching stream around the pre-pass and the fused kernel
    ev[0].record(s)
    for k in range(args.steps):
        step()
        ev[k + 1].record(s)
    torch.cuda.synchronize()
    ktimes = ctx.tpx_kernel_times()
    ctx.tpx_kernel_timing(False)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    rc, counters = ctx.tpx_sync(check=False)
    assert rc == 0, rc
    t_max = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
    h_all = torch.tensor([hits * args.steps], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
        dist.all_reduce(h_all, op=dist.ReduceOp.SUM)
    value = float(h_all.item()) / (float(t_max.item()) / 1e3)

    # sampled oracle parity of the timed call's outputs
    parity = None
    if not args.no_parity and rank == 0:
        parity = _section(parity_sampled, p, h_pk, d_pk, out, n_cl, n_tr, args.parity_shots)

    # roofline of the fused kernel (95% of a step's kernel time; the unwrap pre-pass is the rest)
    pk_info, peak_kind = peaks()
    alg_bytes = 8 * n + 8 * n + ALG_CLUSTER_BYTES * n_cl + 8 * n_tr
    avg_ms = ktimes["fused_ms"] / max(1, ktimes["launches"])
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    peak = float(pk_info.get("hbm_gbs", 6800.0))
    tpp = profile_per_packet("dram_bytes_per_packet")
    wpp = profile_per_packet("warp_instructions_per_packet")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None if tpp is None else tpp * n,
            "algorithmic_bytes": alg_bytes, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
            "kernel": {1: "geo_t4096::fused_kernel<CC, staged>", 2: "geo_t2048::fused_kernel<CC, staged>"}.get(
                tuning["tile_geometry"], "fused_kernel"), "avg_launch_ms": avg_ms,
            "prepass_avg_ms": ktimes["prepass_ms"] / max(1, ktimes["launches"]),
            "launches_timed": ktimes["launches"],
            "bytes_per_unit": {"packet": 16, "cluster": ALG_CLUSTER_BYTES, "trigger": 8}}
    if wpp is not None:
        # the bound that holds: warp-instruction issue, 4 schedulers per SM at the sampled clock
        mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
        ipk = wpp * n / (avg_ms / 1e3)
        ipeak = 4.0 * torch.cuda.get_device_properties(local).multi_processor_count * mhz * 1e6
        roof["issue"] = {"warp_instructions_per_packet": wpp, "achieved_per_s": ipk, "peak_per_s": ipeak,
                         "frac": ipk / ipeak, "clock_mhz": mhz}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        del out
        torch.cuda.empty_cache()
        h_lab = torch.empty(n, dtype=torch.int64, pin_memory=True)
        h_cl = torch.empty(cl_cap * CLUSTER_BYTES, dtype=torch.uint8, pin_memory=True)
        h_tr = torch.empty(args.shots + 16, dtype=torch.int64, pin_memory=True)
        a_pk = h_pk.numpy().view(np.uint64)
        a_tr = h_tr.numpy()
        a_cl = h_cl.numpy().view(tpx.CLUSTER_DTYPE)
        # the modes of the host call: staged through device memory with
        # pipelined copies, or TPX_FLAG_HOST_DIRECT (the kernels read the
        # pinned packets and write the pinned outputs in place over the host
        # link); labels as int64 stream indices or int32 (TPX_FLAG_LABELS32)
        modes = [("staged through device memory, pipelined copies", False, False, False),
                 ("staged through device memory, pipelined copies, int32 labels (TPX_FLAG_LABELS32)", False, True, False),
                 ("staged, pipelined, int32 labels, 64-byte records (TPX_FLAG_RECORDS64)", False, True, True),
                 ("TPX_FLAG_HOST_DIRECT: kernels on the pinned host buffers in place, no copies", True, False, False),
                 ("TPX_FLAG_HOST_DIRECT + TPX_FLAG_LABELS32: in place, int32 labels", True, True, False),
                 ("TPX_FLAG_HOST_DIRECT + TPX_FLAG_LABELS32 + TPX_FLAG_RECORDS64: in place, compact outputs", True, True,
                  True)]
        results = []
        for mode, direct, l32, r64 in modes:
            a_lab = h_lab.numpy().view(np.int32)[:n] if l32 else h_lab.numpy()
            rdt = tpx.CLUSTER64_DTYPE if r64 else tpx.CLUSTER_DTYPE
            a_cl = h_cl.numpy()[: cl_cap * rdt.itemsize].view(rdt)
            hctx = tpx.Context(tpx.Config(tile_geometry=tuning["tile_geometry"] or tpx.TILE_2048, host_direct=direct,
                                          labels32=l32, records64=r64), max_packets=n)
            try:
                def host_step():
                    if state is not None:
                        hctx.tpx_set_state(state)
                    return hctx.tpx_process_host(a_pk, a_lab, None, a_cl, a_tr, idx_base)

                rc, ncl_h, ntr_h = host_step()   # untimed: staging, autotuning
                assert rc == 0, rc
                if world > 1:
                    dist.barrier()
                tim = []
                for _ in range(args.steps):
                    t0 = time.perf_counter()
                    rc, ncl_m, ntr_m = host_step()
                    tim.append(time.perf_counter() - t0)
                    assert rc == 0 and ncl_m == ncl_h, (rc, ncl_m, ncl_h)
            finally:
                hctx.close()
            e_t = torch.tensor([sum(tim)], dtype=torch.float64, device="cuda")
            if world > 1:
                dist.all_reduce(e_t, op=dist.ReduceOp.MAX)
            lab_b = (4 if l32 else 8) * n
            results.append({"value": float(h_all.item()) / float(e_t.item()), "unit": UNIT,
                            # in place, the pre-pass and the fused kernel each read the packets
                            "h2d_bytes_per_step": 8 * n * (2 if direct else 1),
                            "d2h_bytes_per_step": lab_b + (64 if r64 else CLUSTER_BYTES) * ncl_h + 8 * ntr_h + 16,
                            "ms_per_step": 1e3 * statistics.mean(tim), "mode": mode,
                            "step_ms": {"min": 1e3 * min(tim), "median": 1e3 * statistics.median(tim),
                                        "max": 1e3 * max(tim)}})
        best = max(range(len(results)), key=lambda k: results[k]["value"])
        e2e = dict(results[best])
        e2e["other_modes"] = [{k: r[k] for k in ("value", "ms_per_step", "mode")}
                              for k2, r in enumerate(results) if k2 != best]

    cpu = cpu_par = None
    if rank == 0 and not args.no_cpu:
        cpu = _section(cpu_baseline, args, args.cpu_shots)
        cpu_par = _section(cpu_baseline_parallel, args, args.cpu_shots_per_core)
    del d_pk
    ctx.close()
    torch.cuda.empty_cache()
    stream = None
    if rank == 0 and not args.no_stream:
        stream = _section(stream_bench, args)
    batch = None
    if rank == 0 and not args.no_batch:
        batch = _section(batch_bench, args)
    timewalk = None
    if rank == 0 and not args.no_timewalk:
        timewalk = _section(timewalk_bench, args)
    refiner = None
    if rank == 0 and not args.no_refiner:
        torch.cuda.empty_cache()
        refiner = _section(refiner_bench, args)
        if "error" not in refiner:
            # the main path's cluster rate: the budget the refiner's inference is held to
            refiner["main_path_clusters_per_s"] = value * n_cl / max(1, hits) / world
            refiner["infer"]["vs_main_path"] = refiner["infer"]["clusters_per_s"] / refiner["main_path_clusters_per_s"]
            refiner["cnn"]["infer"]["vs_main_path"] = (refiner["cnn"]["infer"]["clusters_per_s"] /
                                                       refiner["main_path_clusters_per_s"])

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": float(t_max.item()) / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                "data": "synthetic",
                "config": {"workload": desc, "packets_per_gpu": n, "pixel_hits_per_gpu": hits,
                           "clusters_per_gpu": n_cl, "shots_per_gpu": n_tr,
                           "l2": "inputs larger than L2 (10 GB packet stream per step)",
                           "parallelism": (f"{world} shot ranges of one acquisition, one all_gather of unwrap "
                                           "summaries before the timed region" if world > 1 else "1 GPU"),
                           "tile_geometry": {1: "4096-packet tiles, 1024-thread CTAs",
                                             2: "2048-packet tiles, 2 x 512-thread CTAs per SM"}.get(
                               tuning["tile_geometry"], "sampling"),
                           "tile_choice": "autotuned in warm-up" if args.tile == "default" else "fixed by --tile",
                           "generation_s": round(t_gen, 1)},
                "parity_sampled": None if parity is None else (parity.get("ok") is True),
                "parity": parity,
                "roofline": roof, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_par, "e2e": e2e, "stream": stream, "batch": batch, "timewalk": timewalk,
                "refiner": refiner, "clocks": clk,
                "gpu_launches": 6 * args.steps - 1,   # 4 pre-pass kernels + the fused kernel per call, and the status carries between unsynchronised calls
                "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)},
                "counters": counters}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    if parity is not None and parity.get("ok") is not True:
        print(f"sampled oracle parity failed: {json.dumps(parity)[:2000]}", file=sys.stderr)
        return 1
    return 0


if __name__ == "__main__":
    sys.exit(main())
