"""Multi-GPU sharding by shot ranges, one process per GPU.

Shots are independent, so each rank takes a contiguous range of the packet
stream cut at trigger (TDC) packets and runs the fused path on it. The only
thing a range needs from the ranges before it is the ToA unwrap state at its
start (Sec. IV.A: the wrap count of each stream and the last raw value) and
the number of triggers before it. That state is an associative combination of
per-range summaries, so ranks exchange one small summary each (one
all_gather of 8 int64 values) and combine their predecessors' summaries in
stream order. No packets cross ranks and nothing touches the data path.

Exact as long as no kept pixel is reported after the next range's first
trigger packet while belonging to an earlier trigger (true whenever tof_max
plus the pixel readout delay is shorter than the trigger spacing at the cut).
"""
from __future__ import annotations

import numpy as np

SUMMARY_FIELDS = ("pixels", "pix_first_raw", "pix_last_raw", "pix_wraps",
                  "triggers", "tdc_first_raw", "tdc_last_raw", "tdc_wraps")
STATE_FIELDS = ("pixels", "pix_last_raw", "pix_wraps", "triggers", "tdc_last_raw", "tdc_wraps")
WRAP_THR_TICKS = 12_800_000_000   # 20 s


def _step(d: int, thr: int) -> int:
    return 1 if d < -thr else (-1 if d > thr else 0)


def identity() -> dict:
    return {f: 0 for f in SUMMARY_FIELDS}


def _chain(na, fa, la, wa, nb, fb, lb, wb, thr):
    n = na + nb
    first = fa if na else fb
    last = lb if nb else la
    wraps = wa + wb + (_step(fb - la, thr) if na and nb else 0)
    return n, first, last, wraps


def combine(a: dict, b: dict, thr_pix: int = WRAP_THR_TICKS, thr_tdc: int = WRAP_THR_TICKS) -> dict:
    """Summary of stretch a followed by stretch b."""
    p = _chain(a["pixels"], a["pix_first_raw"], a["pix_last_raw"], a["pix_wraps"],
               b["pixels"], b["pix_first_raw"], b["pix_last_raw"], b["pix_wraps"], thr_pix)
    t = _chain(a["triggers"], a["tdc_first_raw"], a["tdc_last_raw"], a["tdc_wraps"],
               b["triggers"], b["tdc_first_raw"], b["tdc_last_raw"], b["tdc_wraps"], thr_tdc)
    return dict(zip(SUMMARY_FIELDS, p + t))


def state_of(summary: dict) -> dict:
    """Starting state (tpx_set_state) of a range whose predecessors sum to `summary`."""
    return {"pixels": summary["pixels"], "pix_last_raw": summary["pix_last_raw"],
            "pix_wraps": summary["pix_wraps"], "triggers": summary["triggers"],
            "tdc_last_raw": summary["tdc_last_raw"], "tdc_wraps": summary["tdc_wraps"]}


def plan_cuts(is_tdc: np.ndarray, world: int) -> list[int]:
    """Cut points [0, c1, ..., n]: c_r is the first trigger packet at or after
    r*n/world (ranges may be empty if triggers are sparse)."""
    n = int(is_tdc.size)
    pos = np.flatnonzero(is_tdc)
    cuts = [0]
    for r in range(1, world):
        target = (n * r) // world
        k = int(np.searchsorted(pos, target))
        c = int(pos[k]) if k < pos.size else n
        cuts.append(max(c, cuts[-1]))
    cuts.append(n)
    return cuts


def states_from_summaries(summaries: list[dict]) -> list[dict]:
    """Exclusive in-order combination: the starting state of every range."""
    acc = identity()
    out = []
    for s in summaries:
        out.append(state_of(acc))
        acc = combine(acc, s)
    return out


def exchange_states(summary: dict, group=None) -> tuple[dict, list[dict]]:
    """all_gather every rank's summary; return this rank's starting state and
    all summaries (rank order = stream order)."""
    import torch
    import torch.distributed as dist
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    mine = torch.tensor([summary[f] for f in SUMMARY_FIELDS], dtype=torch.int64, device=dev)
    world = dist.get_world_size(group)
    bufs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(bufs, mine, group=group)
    summaries = [dict(zip(SUMMARY_FIELDS, (int(v) for v in b.cpu().tolist()))) for b in bufs]
    rank = dist.get_rank(group)
    return states_from_summaries(summaries)[rank], summaries


def process_shard(ctx, d_packets, cut_start: int, state: dict, out: dict):
    """Run the fused path on this rank's range from its starting state."""
    ctx.tpx_set_state(state)
    ctx.tpx_process(d_packets, out, index_base=cut_start)
