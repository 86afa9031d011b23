// tpx_prepass.cu -- the unwrap state before every tile of the fused kernel.
//
// ToA unwrapping (Sec. IV.A) is a chain along each of the two streams (pixels,
// TDCs): a step down by more than the threshold adds a wrap, a step up by more
// removes one. The fused kernel needs, for each tile of packets it claims, the
// chain state where the tile starts: the wraps counted so far, the raw value
// of the last pixel and TDC packet before it, and the number of triggers
// before it (the shot index base). This pass computes those states ahead of
// the fused kernel, so that a tile never waits for its predecessors:
//   1. k_tile_aggs: one warp per tile reads the tile once (coalesced 16-byte
//      loads) and forms the tile's chain aggregate (count, first and last raw
//      value, wraps inside) of each stream. Wraps are rare, so the steps are
//      found lane by lane with ballots instead of a scan per load;
//   2. k_block_scan: an exclusive scan of the tile aggregates inside blocks of
//      1024 tiles, and each block's total;
//   3. k_top_scan: one block scans the block totals, starting from the state
//      before the call;
//   4. k_apply: the state before each tile, and after the last one.
// In a batch of independent runs every run is a stream of its own: the scan is
// segmented, restarting at each run's first tile.
#include <cuda_runtime.h>

#include <cstdint>

#include "tpx_common.cuh"
#include "tpx_fused.cuh"

namespace tpxk {
namespace {

constexpr int SB = 1024;       // tiles per block of the scan
constexpr int AW = 8;          // warps per block of k_tile_aggs

// the packets of a tile: [base, base + cnt), and whether a run starts there
struct TileSpan { long long base; int cnt; bool run_first; };
__device__ __forceinline__ TileSpan tile_span(const Params &p, long long tile, int T) {
    TileSpan s;
    long long rend = p.n;
    if (p.bt.tile_run) {
        const int run = p.bt.tile_run[tile];
        const long long t0 = p.bt.run_tile0[run];
        s.base = p.bt.run_off[run] + (tile - t0) * T;
        rend = p.bt.run_off[run + 1];
        s.run_first = tile == t0;
    } else {
        s.base = tile * T;
        s.run_first = tile == 0;
    }
    s.cnt = (int)max(0LL, min((long long)T, rend - s.base));
    return s;
}

// Stream-order accumulation of one chain by a warp, 64 packets per step (two
// per lane). Per lane: its pair's first / last raw value and the wrap steps
// inside the pair; across lanes: the last value of the nearest lower lane
// that has one (ballot), and the last value of the previous step.
struct WarpChain {
    long long first, last, sum;   // sum: per lane, of the steps it detected
    long long n;
    bool any;
};
__device__ __forceinline__ void warp_chain_step(WarpChain &c, bool h0, long long r0, bool h1, long long r1,
                                                long long thr, int lane) {
    const bool has = h0 || h1;
    const unsigned m = __ballot_sync(0xffffffffu, has);
    if (!m) return;
    const long long pf = h0 ? r0 : r1;       // first of the pair
    const long long pl = h1 ? r1 : r0;       // last of the pair
    long long s = (h0 && h1) ? jump(r1 - r0, thr) : 0;
    // the value before this pair: the last one of the nearest lower lane with
    // a value, else the chain's last value before this step
    const unsigned lower = m & ((1u << lane) - 1u);
    const int src = lower ? 31 - __clz(lower) : 0;
    const long long prev_lane = __shfl_sync(0xffffffffu, pl, src);
    if (has) {
        if (lower) s += jump(pf - prev_lane, thr);
        else if (c.any) s += jump(pf - c.last, thr);
    }
    c.sum += s;
    const int lo = __ffs(m) - 1, hi = 31 - __clz(m);
    const long long step_first = __shfl_sync(0xffffffffu, pf, lo);
    const long long step_last = __shfl_sync(0xffffffffu, pl, hi);
    if (!c.any) c.first = step_first;
    c.last = step_last;
    c.any = true;
    c.n += __popc(m) + __popc(__ballot_sync(0xffffffffu, h0 && h1));
}

__global__ void __launch_bounds__(AW * 32) k_tile_aggs(const Params p, int T) {
    const int lane = threadIdx.x & 31;
    const long long warp = (long long)blockIdx.x * AW + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * AW;
    const long long tp = p.thr_pix, tt = p.thr_tdc;
    unsigned long long c_pix = 0, c_tdc = 0, c_bad = 0;
    for (long long tile = warp; tile < p.n_tiles; tile += nw) {
        const TileSpan sp = tile_span(p, tile, T);
        WarpChain cp{0, 0, 0, 0, false}, ct{0, 0, 0, 0, false};
        const uint64_t *src = p.pk + sp.base;
        const bool vec = (sp.base & 1) == 0;
        // the lane's two packets of step q0 (zero past the tile)
        auto load2 = [&](int q0, uint64_t &a, uint64_t &b) {
            const int q = q0 + 2 * lane;
            a = 0;
            b = 0;
            if (vec && q + 1 < sp.cnt) {
                const ulonglong2 v = __ldcs(reinterpret_cast<const ulonglong2 *>(src + q));
                a = v.x;
                b = v.y;
            } else {
                if (q < sp.cnt) a = __ldcs(src + q);
                if (q + 1 < sp.cnt) b = __ldcs(src + q + 1);
            }
        };
        // one step ahead: the next 64 packets are in flight while these are combined
        uint64_t nx0, nx1;
        load2(0, nx0, nx1);
        for (int q0 = 0; q0 < sp.cnt; q0 += 64) {
            const int q = q0 + 2 * lane;
            const uint64_t w0 = nx0, w1 = nx1;
            if (q0 + 64 < sp.cnt) load2(q0 + 64, nx0, nx1);
            const bool in0 = q < sp.cnt, in1 = q + 1 < sp.cnt;
            const unsigned h0 = (unsigned)(w0 >> 60), h1 = (unsigned)(w1 >> 60);
            const bool p0 = in0 && h0 == 0xBu, p1 = in1 && h1 == 0xBu;
            const bool t0 = in0 && h0 == 0x6u, t1 = in1 && h1 == 0x6u;
            c_pix += (unsigned)p0 + (unsigned)p1;
            c_tdc += (unsigned)t0 + (unsigned)t1;
            c_bad += (unsigned)(in0 && !p0 && !t0) + (unsigned)(in1 && !p1 && !t1);
            warp_chain_step(cp, p0, p0 ? pix_raw(w0) : 0, p1, p1 ? pix_raw(w1) : 0, tp, lane);
            if (__any_sync(0xffffffffu, t0 || t1))
                warp_chain_step(ct, t0, t0 ? tdc_raw(w0) : 0, t1, t1 ? tdc_raw(w1) : 0, tt, lane);
        }
        long long sp_ = cp.sum, st_ = ct.sum;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sp_ += __shfl_xor_sync(0xffffffffu, sp_, o);
            st_ += __shfl_xor_sync(0xffffffffu, st_, o);
        }
        if (lane == 0) {
            GAgg a;
            a.pix.n = cp.n; a.pix.first = cp.first; a.pix.last = cp.last; a.pix.sum = sp_;
            a.tdc.n = ct.n; a.tdc.first = ct.first; a.tdc.last = ct.last; a.tdc.sum = st_;
            if (!cp.any) a.pix = chain_id();
            if (!ct.any) a.tdc = chain_id();
            p.ts.agg[tile] = a;
        }
    }
    // packet-class counters of the call (Ctl is cleared before the launch)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c_pix += __shfl_xor_sync(0xffffffffu, c_pix, o);
        c_tdc += __shfl_xor_sync(0xffffffffu, c_tdc, o);
        c_bad += __shfl_xor_sync(0xffffffffu, c_bad, o);
    }
    if (lane == 0) {
        if (c_pix) atomicAdd(&p.ctl->counters[C_PIXELS], c_pix);
        if (c_tdc) atomicAdd(&p.ctl->counters[C_TDCS], c_tdc);
        if (c_bad) atomicAdd(&p.ctl->counters[C_CORRUPT], c_bad);
    }
}

// segmented combine: a run start (flag) discards what came before it
struct SAgg { GAgg a; bool f; };
__device__ __forceinline__ SAgg scomb(const SAgg &x, const SAgg &y, long long tp, long long tt) {
    SAgg r;
    r.f = x.f || y.f;
    r.a = y.f ? y.a : acomb(x.a, y.a, tp, tt);
    return r;
}
__device__ __forceinline__ SAgg shfl_up_sagg(const SAgg &v, int o) {
    SAgg u;
    u.a = shfl_up_agg(v.a, o);
    u.f = __shfl_up_sync(0xffffffffu, (int)v.f, o) != 0;
    return u;
}
__device__ __forceinline__ SAgg sid() { SAgg s; s.a = agg_id(); s.f = false; return s; }

// block-wide exclusive segmented scan (SB threads); total in *tot
__device__ SAgg block_excl_sagg(const SAgg &v, SAgg *s_w, SAgg *tot, long long tp, long long tt) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    SAgg incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const SAgg u = shfl_up_sagg(incl, o);
        if (lane >= o) incl = scomb(u, incl, tp, tt);
    }
    SAgg ex = shfl_up_sagg(incl, 1);
    if (lane == 0) ex = sid();
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        SAgg x = s_w[lane];
        SAgg xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const SAgg u = shfl_up_sagg(xi, o);
            if (lane >= o) xi = scomb(u, xi, tp, tt);
        }
        SAgg xe = shfl_up_sagg(xi, 1);
        if (lane == 0) xe = sid();
        s_w[lane] = xe;
        if (lane == 31) *tot = xi;
    }
    __syncthreads();
    const SAgg r = scomb(s_w[w], ex, tp, tt);
    __syncthreads();
    return r;
}

// a run's first tile restarts the chains (batches only: one stream otherwise)
__device__ __forceinline__ bool run_starts_at(const Params &p, long long tile) {
    return p.bt.tile_run && p.bt.run_tile0[p.bt.tile_run[tile]] == tile;
}

// per block of SB tiles: the exclusive scan inside the block (into pre[]) and
// the block's total (into bagg[], its flag into bflag[])
__global__ void __launch_bounds__(SB) k_block_scan(const Params p, GAgg *bagg, int *bflag) {
    __shared__ SAgg s_w[32];
    __shared__ SAgg s_tot;
    const long long t = (long long)blockIdx.x * SB + threadIdx.x;
    SAgg v = sid();
    if (t < p.n_tiles) {
        v.a = p.ts.agg[t];
        v.f = run_starts_at(p, t);
    }
    const SAgg ex = block_excl_sagg(v, s_w, &s_tot, p.thr_pix, p.thr_tdc);
    if (t < p.n_tiles) p.ts.pre[t] = v.f ? agg_id() : ex.a;   // a run starts from nothing
    if (threadIdx.x == 0) {
        bagg[blockIdx.x] = s_tot.a;
        bflag[blockIdx.x] = s_tot.f ? 1 : 0;
    }
}

// one block: exclusive segmented scan of the block totals, from the state
// before the call (E0; a batch starts every run from nothing)
__global__ void __launch_bounds__(SB) k_top_scan(const Params p, GAgg *bagg, const int *bflag, long long nb) {
    __shared__ SAgg s_w[32];
    __shared__ SAgg s_tot;
    __shared__ SAgg s_carry;
    const long long tp = p.thr_pix, tt = p.thr_tdc;
    if (threadIdx.x == 0) {
        s_carry.a = (!p.bt.tile_run && p.E0) ? *p.E0 : agg_id();
        s_carry.f = false;
    }
    __syncthreads();
    for (long long b0 = 0; b0 < nb; b0 += SB) {
        const long long b = b0 + threadIdx.x;
        SAgg v = sid();
        if (b < nb) {
            v.a = bagg[b];
            v.f = bflag[b] != 0;
        }
        const SAgg ex = block_excl_sagg(v, s_w, &s_tot, tp, tt);
        const SAgg carry = s_carry;
        const SAgg r = scomb(carry, ex, tp, tt);
        __syncthreads();
        if (b < nb) bagg[b] = r.a;      // now: the state before block b
        if (threadIdx.x == 0) s_carry = scomb(carry, s_tot, tp, tt);
        __syncthreads();
    }
}

// the state before each tile: within its block's scan, after the state before
// the block unless its run started inside the block; the last tile also gives
// the state after the call
__global__ void __launch_bounds__(256) k_apply(const Params p, const GAgg *bpre) {
    const long long t = (long long)blockIdx.x * 256 + threadIdx.x;
    if (t >= p.n_tiles) return;
    const long long b = t / SB, bstart = b * SB;
    const long long tp = p.thr_pix, tt = p.thr_tdc;
    bool fresh;   // the run of tile t starts inside block b (at or before t)
    if (p.bt.tile_run) fresh = p.bt.run_tile0[p.bt.tile_run[t]] >= bstart;
    else fresh = false;
    const GAgg loc = p.ts.pre[t];
    const GAgg e = fresh ? loc : acomb(bpre[b], loc, tp, tt);
    p.ts.pre[t] = e;
    if (t == p.n_tiles - 1 && !p.bt.tile_run && p.state_out) *p.state_out = acomb(e, p.ts.agg[t], tp, tt);
}

}  // namespace

size_t unwrap_prepass_scratch_bytes(long long n_tiles) {
    const long long nb = (n_tiles + SB - 1) / SB + 1;
    return (size_t)nb * (sizeof(GAgg) + sizeof(int)) + 256;
}

cudaError_t launch_unwrap_prepass(const Params &p, int T, int grid, cudaStream_t s) {
    if (p.n_tiles <= 0) return cudaSuccess;
    const long long nb = (p.n_tiles + SB - 1) / SB;
    GAgg *bagg = p.ts.blk;
    int *bflag = reinterpret_cast<int *>(bagg + nb + 1);
    long long g = (p.n_tiles + AW - 1) / AW;
    if (g > (long long)grid * 8) g = (long long)grid * 8;
    k_tile_aggs<<<(unsigned)g, AW * 32, 0, s>>>(p, T);
    k_block_scan<<<(unsigned)nb, SB, 0, s>>>(p, bagg, bflag);
    k_top_scan<<<1, SB, 0, s>>>(p, bagg, bflag, nb);
    k_apply<<<(unsigned)((p.n_tiles + 255) / 256), 256, 0, s>>>(p, bagg);
    return cudaGetLastError();
}

}  // namespace tpxk
