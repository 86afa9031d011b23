// tpx_general.cu -- the general (global-memory) path: tpx_decode,
// tpx_cluster, tpx_centroid, the exact redo of a tpx_process call whose
// input the fused kernel cannot hold on chip, and the streaming calls.
//
// decode  : tile aggregates of the two unwrap chains (Sec. IV.A) -> prefix
//           over tiles -> per-packet unwrapped times and the trigger list ->
//           each pixel binned to the most recent trigger in time by binary
//           search, cut at tof_max (Sec. IV.B), timewalk table subtracted
//           (Sec. IV.C) -> kept pixels compacted in stream order.
// cluster : stable LSD radix sort of the hits on (shot, corrected ToF) --
//           ties keep stream order. In that order a gap larger than dt ends
//           every cluster, so the sorted hits split into independent
//           segments. One warp clusters a segment of up to 64 hits in
//           registers: ballots give each hit's adjacency row (Sec. V.A box
//           rule) and local-maximum flag (Sec. V.B); components are closures
//           over the rows seeded at the earliest hit; the root's int64
//           moments are warp sums. Longer segments (shots whose particles
//           arrive within dt of each other) find their pairs through a hash
//           of (shot, x, y) cells and join them in a global lock-free
//           union-find whose root is the smallest position.
// centroid: cluster ids in ascending label order (a scan over root flags in
//           stream order), f64 final division (Sec. V.C); PAPER mode sums the
//           box neighbourhood of each local maximum.
// No capacity limit besides 2^31 - 1 kept pixels per call.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

#include "tpx.h"
#include "tpx_common.cuh"
#include "tpx_ctx.h"
#include "tpx_fused.cuh"

namespace tpxg {

using namespace tpxk;

constexpr int GT = 256;             // threads per block
constexpr int GW = GT / 32;
constexpr int GK = 16;              // packets (or keys) per thread
constexpr int GTILE = GT * GK;      // 4096
constexpr int kBias = 32768;        // corrected ToF + bias >= 0 for int16 timewalk shifts

// ------------------------------------------------------------ block scans
__device__ GAgg block_scan_agg_g(const GAgg &v, GAgg *s_w, GAgg *total, long long tp, long long tt) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    GAgg incl = warp_incl_scan(v, lane, tp, tt);
    GAgg wex = shfl_up_agg(incl, 1);
    if (lane == 0) wex = agg_id();
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        GAgg x = lane < GW ? s_w[lane] : agg_id();
        GAgg xi = warp_incl_scan(x, lane, tp, tt);
        GAgg xe = shfl_up_agg(xi, 1);
        if (lane == 0) xe = agg_id();
        if (lane < GW) s_w[lane] = xe;
        if (lane == GW - 1) *total = xi;
    }
    __syncthreads();
    GAgg r = acomb(s_w[w], wex, tp, tt);
    __syncthreads();
    return r;
}

__device__ long long block_scan_ll(long long v, long long *s_w, long long *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        long long x = lane < GW ? s_w[lane] : 0;
        long long xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long u = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += u;
        }
        if (lane < GW) s_w[lane] = xi - x;
        if (lane == GW - 1) *total = xi;
    }
    __syncthreads();
    long long r = s_w[w] + incl - v;
    __syncthreads();
    return r;
}

// single-block scans (PT threads, each over a contiguous strip of items)
constexpr int PT = 1024;
__device__ long long block_excl_ll_pt(long long v, long long *s32, long long *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) s32[w] = incl;
    __syncthreads();
    if (w == 0) {
        const long long x = s32[lane];
        long long xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += u;
        }
        s32[lane] = xi - x;
        if (lane == 31) *total = xi;
    }
    __syncthreads();
    const long long r = s32[w] + incl - v;
    __syncthreads();
    return r;
}
__device__ GAgg block_excl_agg_pt(const GAgg &v, GAgg *s32, long long tp, long long tt) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const GAgg incl = warp_incl_scan(v, lane, tp, tt);
    GAgg lex = shfl_up_agg(incl, 1);
    if (lane == 0) lex = agg_id();
    if (lane == 31) s32[w] = incl;
    __syncthreads();
    if (w == 0) {
        const GAgg xi = warp_incl_scan(s32[lane], lane, tp, tt);
        GAgg xe = shfl_up_agg(xi, 1);
        if (lane == 0) xe = agg_id();
        s32[lane] = xe;
    }
    __syncthreads();
    const GAgg r = acomb(s32[w], lex, tp, tt);
    __syncthreads();
    return r;
}
__device__ __forceinline__ void strip_of(long long items, long long *b, long long *e) {
    const long long per = (items + PT - 1) / PT;
    *b = min(items, (long long)threadIdx.x * per);
    *e = min(items, *b + per);
}

// ------------------------------------------------------------ decode kernels
__global__ void __launch_bounds__(GT) k_tile_agg(const uint64_t *pk, long long n, long long tp, long long tt,
                                                 GAgg *tagg, long long *tcnt) {
    __shared__ GAgg s_w[GW];
    __shared__ GAgg s_tot;
    const long long tile = blockIdx.x, base = tile * GTILE;
    GAgg a = agg_id();
    long long ntdc = 0;
    for (int j = 0; j < GK; ++j) {
        const long long q = base + threadIdx.x * GK + j;
        if (q >= n) break;
        const uint64_t w = pk[q];
        const unsigned h = (unsigned)(w >> 60);
        if (h == 0xBu) chain_push(a.pix, pix_raw(w), tp);
        else if (h == 0x6u) { chain_push(a.tdc, tdc_raw(w), tt); ++ntdc; }
    }
    (void)block_scan_agg_g(a, s_w, &s_tot, tp, tt);
    if (threadIdx.x == 0) {
        tagg[tile] = s_tot;
        tcnt[tile] = s_tot.tdc.n;
    }
}

// exclusive prefix over tiles, starting from the state before the call (one
// block: strips of tiles, a block scan of the strip aggregates, then strips)
__global__ void __launch_bounds__(PT) k_tile_prefix(const GAgg *tagg, GAgg *tpre, const long long *tcnt, long long *toff,
                                                    long long tiles, long long tp, long long tt, long long *n_trig_out,
                                                    const GAgg *E0, GAgg *state_out) {
    __shared__ GAgg s_a[32];
    __shared__ long long s_c[32];
    __shared__ long long s_tot;
    long long b, e;
    strip_of(tiles, &b, &e);
    GAgg a = agg_id();
    long long cn = 0;
    for (long long t = b; t < e; ++t) {
        a = acomb(a, tagg[t], tp, tt);
        cn += tcnt[t];
    }
    const GAgg ex = block_excl_agg_pt(a, s_a, tp, tt);
    long long off = block_excl_ll_pt(cn, s_c, &s_tot);
    GAgg acc = acomb(E0 ? *E0 : agg_id(), ex, tp, tt);
    for (long long t = b; t < e; ++t) {
        tpre[t] = acc;
        toff[t] = off;
        acc = acomb(acc, tagg[t], tp, tt);
        off += tcnt[t];
    }
    if (threadIdx.x == PT - 1) {   // its strip is the last (possibly empty) one
        toff[tiles] = off;
        *n_trig_out = off;
        if (state_out) *state_out = acc;
    }
}

__global__ void __launch_bounds__(GT) k_unwrap(const uint64_t *pk, long long n, const GAgg *tpre, const long long *toff,
                                               long long tp, long long tt, long long *t_all, long long *trig,
                                               long long trig_cap, unsigned *status, long long *trig_pos) {
    __shared__ GAgg s_w[GW];
    __shared__ GAgg s_tot;
    const long long tile = blockIdx.x, base = tile * GTILE;
    const long long q0 = base + threadIdx.x * GK;
    GAgg a = agg_id();
    for (int j = 0; j < GK; ++j) {
        const long long q = q0 + j;
        if (q >= n) break;
        const uint64_t w = pk[q];
        const unsigned h = (unsigned)(w >> 60);
        if (h == 0xBu) chain_push(a.pix, pix_raw(w), tp);
        else if (h == 0x6u) chain_push(a.tdc, tdc_raw(w), tt);
    }
    const GAgg ex = block_scan_agg_g(a, s_w, &s_tot, tp, tt);
    const GAgg st = acomb(tpre[tile], ex, tp, tt);
    bool hp = st.pix.n > 0, ht = st.tdc.n > 0;
    long long lp = st.pix.last, ep = st.pix.sum, lt = st.tdc.last, et = st.tdc.sum;
    long long ti = toff[tile] + ex.tdc.n;
    for (int j = 0; j < GK; ++j) {
        const long long q = q0 + j;
        if (q >= n) break;
        const uint64_t w = pk[q];
        const unsigned h = (unsigned)(w >> 60);
        long long t = 0;
        if (h == 0xBu) {
            const long long r = pix_raw(w);
            if (hp) ep += jump(r - lp, tp);
            hp = true;
            lp = r;
            t = r + ep * kPixPeriod;
        } else if (h == 0x6u) {
            const long long r = tdc_raw(w);
            if (ht) et += jump(r - lt, tt);
            ht = true;
            lt = r;
            t = r + et * kTdcPeriod;
            if (ti < trig_cap) {
                trig[ti] = t;
                if (trig_pos) trig_pos[ti] = q;
            } else {
                atomicOr(status, ST_TRIG_CAP);
            }
            ++ti;
        }
        t_all[q] = t;
    }
}

// the trigger count of the call, or -1 when it exceeded the trigger capacity
// (the status is latched and nothing is binned)
__device__ __forceinline__ long long usable_triggers(const long long *n_trig, long long trig_cap) {
    const long long v = *n_trig;
    return v > trig_cap ? -1 : v;
}

__global__ void k_check_trig(const long long *trig, const long long *n_trig, long long trig_cap, unsigned *status) {
    const long long ntr = usable_triggers(n_trig, trig_cap);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i + 1 < ntr; i += (long long)gridDim.x * blockDim.x)
        if (trig[i + 1] < trig[i]) atomicOr(status, ST_TRIG_ORDER);
}

// most recent trigger in time: last index with trig <= t, or -1
__device__ __forceinline__ long long shot_of(const long long *trig, long long ntr, long long t) {
    long long lo = 0, hi = ntr;
    while (lo < hi) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (trig[mid] <= t) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

// 0 keep, 1 background, 2 before any trigger, 3 not a pixel
__device__ __forceinline__ int bin_pixel(uint64_t w, long long t, const long long *trig, long long ntr,
                                         long long tof_max, long long *shot, long long *tof) {
    if ((w >> 60) != 0xBu) return 3;
    const long long s = shot_of(trig, ntr, t);
    if (s < 0) return 2;
    const long long f = t - trig[s];
    if (f > tof_max) return 1;
    *shot = s;
    *tof = f;
    return 0;
}

// per tile: kept pixels and the drop counters (packets read warp-strided)
__global__ void __launch_bounds__(GT) k_bin(const uint64_t *pk, long long n, const long long *t_all, const long long *trig,
                                            const long long *n_trig, long long trig_cap, long long tof_max,
                                            long long *tile_kept, unsigned long long *counters) {
    __shared__ long long s_w[GW];
    __shared__ long long s_tot;
    const long long tile = blockIdx.x, base = tile * GTILE;
    const long long ntr = usable_triggers(n_trig, trig_cap);
    long long keep = 0, bg = 0, pre = 0, pix = 0, tdc = 0, bad = 0;
    for (int j = 0; j < GK && ntr >= 0; ++j) {
        const long long q = base + j * GT + threadIdx.x;
        if (q >= n) break;
        const uint64_t w = pk[q];
        const unsigned h = (unsigned)(w >> 60);
        if (h == 0x6u) { ++tdc; continue; }
        if (h != 0xBu) { ++bad; continue; }
        ++pix;
        long long s, f;
        const int v = bin_pixel(w, t_all[q], trig, ntr, tof_max, &s, &f);
        keep += v == 0;
        bg += v == 1;
        pre += v == 2;
    }
    const long long vals[6] = {keep, bg, pre, pix, tdc, bad};
    const int idx[6] = {C_KEPT, C_DROP_BG, C_DROP_PRE, C_PIXELS, C_TDCS, C_CORRUPT};
    for (int k = 0; k < 6; ++k) {
        unsigned long long v = (unsigned long long)vals[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&counters[idx[k]], v);
    }
    (void)block_scan_ll(keep, s_w, &s_tot);
    if (threadIdx.x == 0) tile_kept[tile] = s_tot;
}

// exclusive prefix of per-tile counts (one block)
__global__ void __launch_bounds__(PT) k_count_prefix(const long long *cnt, long long *off, long long tiles,
                                                     long long *total_out) {
    __shared__ long long s_c[32];
    __shared__ long long s_tot;
    long long b, e;
    strip_of(tiles, &b, &e);
    long long v = 0;
    for (long long t = b; t < e; ++t) v += cnt[t];
    long long o = block_excl_ll_pt(v, s_c, &s_tot);
    for (long long t = b; t < e; ++t) {
        off[t] = o;
        o += cnt[t];
    }
    if (threadIdx.x == PT - 1) {
        off[tiles] = o;
        if (total_out) *total_out = o;
    }
}

// kept pixels in stream order: per round of GT consecutive packets, a ballot
// and the warp counts give every kept pixel its slot (coalesced writes)
__global__ void __launch_bounds__(GT) k_compact(const uint64_t *pk, long long n, long long idx_base, const long long *t_all,
                                                const long long *trig, const long long *n_trig, long long trig_cap,
                                                long long tof_max, const int16_t *lut, const long long *tile_off,
                                                tpx_hits hits, long long cap, unsigned *status, const GAgg *E0) {
    __shared__ unsigned s_wc[GW];
    const long long trig_base = E0 ? E0->tdc.n : 0;
    const long long ntr = usable_triggers(n_trig, trig_cap);
    if (ntr < 0) return;
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const long long tile = blockIdx.x, base = tile * GTILE;
    long long o = tile_off[tile];
    for (int j = 0; j < GK; ++j) {
        if (base + j * GT >= n) break;                  // uniform over the block
        const long long q = base + j * GT + threadIdx.x;
        uint64_t w = 0;
        long long s = 0, f = 0;
        bool keep = false;
        if (q < n) {
            w = pk[q];
            keep = bin_pixel(w, t_all[q], trig, ntr, tof_max, &s, &f) == 0;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_wc[wi] = __popc(bal);
        __syncthreads();
        unsigned before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < GW; ++k) {
            const unsigned c = s_wc[k];
            before += k < wi ? c : 0u;
            total += c;
        }
        if (keep) {
            const long long slot = o + before + __popc(bal & ((1u << lane) - 1u));
            if (slot < cap) {
                const int tot = pix_tot(w);
                const long long corr = lut ? (long long)lut[tot] : 0LL;
                hits.index[slot] = idx_base + q;
                hits.shot[slot] = s + trig_base;
                hits.t[slot] = t_all[q] - corr;
                hits.tof[slot] = (int32_t)(f - corr);
                hits.x[slot] = (uint8_t)pix_x(w);
                hits.y[slot] = (uint8_t)pix_y(w);
                hits.tot[slot] = (uint16_t)tot;
            } else {
                atomicOr(status, ST_CLUSTER_CAP);
            }
        }
        o += total;
        __syncthreads();
    }
}

// ------------------------------------------------------------ radix sort
// stable LSD sort of (key, value) pairs on 8-bit digits
__global__ void __launch_bounds__(GT) k_sort_hist(const unsigned long long *keys, long long n, int shift, unsigned *hist,
                                                  long long tiles) {
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = blockIdx.x * (long long)GTILE;
    for (int j = 0; j < GK; ++j) {
        const long long i = base + j * GT + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(GT) k_sort_scatter(const unsigned long long *kin, const unsigned *vin, long long n,
                                                     int shift, const unsigned *offs, long long tiles,
                                                     unsigned long long *kout, unsigned *vout) {
    __shared__ unsigned run[256];       // running count per digit in this tile
    __shared__ unsigned wcnt[GW][256];  // per-warp counts of the current round
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    run[threadIdx.x] = offs[(long long)threadIdx.x * tiles + blockIdx.x];
    const long long base = blockIdx.x * (long long)GTILE;
    for (int j = 0; j < GK; ++j) {
        for (int k = 0; k < GW; ++k) wcnt[k][threadIdx.x] = 0;
        __syncthreads();
        const long long i = base + j * GT + threadIdx.x;
        const bool ok = i < n;
        const unsigned long long key = ok ? kin[i] : 0ull;
        const unsigned d = ok ? (unsigned)((key >> shift) & 255) : 256u + lane;   // unique dummy for idle lanes
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned before = __popc(peers & ((1u << lane) - 1u));
        if (ok && before == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        unsigned pos = 0;
        if (ok) {
            unsigned acc = 0;
            for (int k = 0; k < w; ++k) acc += wcnt[k][d];
            pos = run[d] + acc + before;
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
        // advance the running counts by this round's totals
        unsigned tot = 0;
        for (int k = 0; k < GW; ++k) tot += wcnt[k][threadIdx.x];
        run[threadIdx.x] += tot;
        __syncthreads();
    }
}

// exclusive scan of unsigned counts (serial over block sums; general path only)
__global__ void __launch_bounds__(GT) k_scan_blocks(const unsigned *in, unsigned *out, long long n, unsigned *bsum) {
    __shared__ long long s_w[GW];
    __shared__ long long s_tot;
    const long long base = blockIdx.x * (long long)GTILE + threadIdx.x * GK;
    long long mine = 0;
    for (int j = 0; j < GK; ++j)
        if (base + j < n) mine += in[base + j];
    long long o = block_scan_ll(mine, s_w, &s_tot);
    for (int j = 0; j < GK; ++j)
        if (base + j < n) { out[base + j] = (unsigned)o; o += in[base + j]; }
    if (threadIdx.x == 0) bsum[blockIdx.x] = (unsigned)s_tot;
}
__global__ void __launch_bounds__(PT) k_scan_bsum(unsigned *bsum, long long nb) {
    __shared__ long long s_c[32];
    __shared__ long long s_tot;
    long long b, e;
    strip_of(nb, &b, &e);
    long long v = 0;
    for (long long t = b; t < e; ++t) v += bsum[t];
    long long o = block_excl_ll_pt(v, s_c, &s_tot);
    for (long long t = b; t < e; ++t) {
        const unsigned x = bsum[t];
        bsum[t] = (unsigned)o;
        o += x;
    }
}
__global__ void k_scan_add(unsigned *out, long long n, const unsigned *bsum) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] += bsum[i / GTILE];
}

// ------------------------------------------------------------ cluster kernels
// sort key: (shot relative to the call's first shot) << 24 | corrected ToF + bias
__global__ void k_make_keys(tpx_hits h, long long n, const unsigned long long *shot_min, unsigned long long *keys,
                            unsigned *vals) {
    const unsigned long long m = *shot_min;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        keys[i] = (((unsigned long long)h.shot[i] - m) << 24) | (unsigned long long)(h.tof[i] + kBias);
        vals[i] = (unsigned)i;
    }
}
__global__ void k_shot_range(tpx_hits h, long long n, unsigned long long *mn, unsigned long long *mx) {
    unsigned long long lo = ~0ull, hi = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long v = (unsigned long long)h.shot[i];
        lo = min(lo, v);
        hi = max(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_down_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_down_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mn, lo);
        atomicMax(mx, hi);
    }
}

struct Sorted {                     // hits in sorted order
    unsigned *hit;                  // sorted position -> hit index
    long long *shot;
    int *tofb;                      // corrected ToF + bias
    unsigned char *x, *y;
    unsigned short *tot;
    long long *index;
};

__global__ void k_gather(tpx_hits h, const unsigned *vals, long long n, Sorted s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned k = vals[i];
        s.hit[i] = k;
        s.shot[i] = h.shot[k];
        s.tofb[i] = h.tof[k] + kBias;
        s.x[i] = h.x[k];
        s.y[i] = h.y[k];
        s.tot[i] = h.tot[k];
        s.index[i] = h.index[k];
    }
}

// Segments: in sorted order a gap larger than dt (or a new shot) separates
// everything before it from everything after it -- no adjacent pair spans
// it -- so each run between such gaps clusters on its own.
__global__ void k_seg_flags(Sorted s, long long n, int dt, unsigned *f) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        f[i] = (i == 0 || s.shot[i] != s.shot[i - 1] || s.tofb[i] - s.tofb[i - 1] > dt) ? 1u : 0u;
}
__global__ void k_seg_starts(const unsigned *f, const unsigned *off, long long n, long long *start, long long *nseg) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (f[i]) start[off[i]] = i;
        if (i == n - 1) {
            const long long m = (long long)off[i] + f[i];
            start[m] = n;
            *nseg = m;
        }
    }
}

// per-root moments, indexed by the hit position of the root
struct AccH { long long s_tot, s_x, s_y, s_t; unsigned n, npk; };

constexpr int WREG = 64;            // hits of a segment held in registers (two per lane)
constexpr int WCAP = 256;           // hits of a segment held by one warp in shared memory
constexpr int ECAP = 1024;          // adjacent pairs of a segment kept for the hooking rounds
constexpr int HBW = 512;            // cell-hash buckets of a warp's segment
constexpr int SEGW = 4;             // warps per block
struct SegSm {
    int tofb[WCAP];
    int parent[WCAP];
    unsigned edge[ECAP];            // (k << 16) | j, k < j
    unsigned hhead[HBW];            // cell hash: first position, 0xFFFF = none
    unsigned ecnt;
    unsigned short hnext[WCAP];
    unsigned short tot[WCAP];
    unsigned char x[WCAP], y[WCAP], np[WCAP];
};
__device__ __forceinline__ unsigned wcell(int x, int y) { return (unsigned)(x * 67 + y * 131) & (HBW - 1); }

__device__ __forceinline__ int s_find(volatile int *par, int x) {
    for (;;) {
        const int p = par[x];
        if (p == x) return x;
        const int g = par[p];
        if (g == p) return p;
        par[x] = g;
        x = g;
    }
}
// lock-free union in shared memory; the smaller position becomes the root
__device__ __forceinline__ void s_unite(int *par, int a, int b) {
    for (;;) {
        a = s_find(par, a);
        b = s_find(par, b);
        if (a == b) return;
        if (a > b) { const int t = a; a = b; b = t; }
        const int old = atomicCAS(&par[b], b, a);
        if (old == b) return;
        b = old;
    }
}

// Sec. V.B tie rule: equal ToT goes to the hit later in the stream
__device__ __forceinline__ bool j_brighter(int tj, int ti, const long long *index, long long j, long long i) {
    return tj > ti || (tj == ti && index[j] > index[i]);
}

// Segments of at most 64 hits, in registers: lane l holds hits l and l + 32.
// For every hit k (warp-uniform loop) the ballots of "adjacent to k" give
// its adjacency row as a 64-bit mask and "brighter than k" its local-maximum
// flag; components are breadth-first closures over the rows, seeded at the
// lowest unvisited position, so the seed is the component's earliest hit.
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ void seg_small(const Sorted &s, long long s0, int L, int rx, int ry, int dt, int cc, bool emit,
                          long long *labels, unsigned char *is_peak, unsigned *rflag, AccH *acc, int lane,
                          SegSm &W) {
    constexpr unsigned FULL = 0xffffffffu;
    const int a = lane, b = lane + 32;
    const bool va = a < L, vb = b < L;
    int ta = 0, tb = 0;
    unsigned pa = 0, pb = 0, oa = 0, ob = 0, ha = 0, hb = 0;
    long long ia = 0, ib = 0;
    if (va) {
        ta = s.tofb[s0 + a]; pa = s.x[s0 + a] | ((unsigned)s.y[s0 + a] << 8); oa = s.tot[s0 + a];
        ia = s.index[s0 + a]; ha = s.hit[s0 + a];
    }
    if (vb) {
        tb = s.tofb[s0 + b]; pb = s.x[s0 + b] | ((unsigned)s.y[s0 + b] << 8); ob = s.tot[s0 + b];
        ib = s.index[s0 + b]; hb = s.hit[s0 + b];
    }
    unsigned long long rowA = 0, rowB = 0;
    bool npA = false, npB = false;
    // A compact segment (one particle, or a few close ones) with the 8-neighbour
    // box: its hits go into a 16 x 16 occupancy grid of their bounding box and
    // every lane reads its hits' 8 neighbour cells -- a few dozen instructions
    // per hit instead of one warp-wide step per hit of the segment. Two hits on
    // one pixel, a larger box or other radii take the all-pairs steps below.
    bool grid = false;
    if (rx == 1 && ry == 1) {
        const unsigned xa = pa & 255u, ya = pa >> 8, xb = pb & 255u, yb = pb >> 8;
        const unsigned x0 = __reduce_min_sync(FULL, min(va ? xa : 255u, vb ? xb : 255u));
        const unsigned x1 = __reduce_max_sync(FULL, max(va ? xa : 0u, vb ? xb : 0u));
        const unsigned y0 = __reduce_min_sync(FULL, min(va ? ya : 255u, vb ? yb : 255u));
        const unsigned y1 = __reduce_max_sync(FULL, max(va ? ya : 0u, vb ? yb : 0u));
        if (x1 - x0 <= 13u && y1 - y0 <= 13u) {
            unsigned *cell = W.edge;   // 256 cells: hit + 1, 0 = empty (the edge list is not in use)
            __syncwarp();              // the warp's previous segment is done with W
            for (int i = lane; i < 256; i += 32) cell[i] = 0u;
            if (va) { W.tofb[a] = ta; W.tot[a] = (unsigned short)oa; }
            if (vb) { W.tofb[b] = tb; W.tot[b] = (unsigned short)ob; }
            __syncwarp();
            const int ca = (int)(xa - x0 + 1) + 16 * (int)(ya - y0 + 1), cb = (int)(xb - x0 + 1) + 16 * (int)(yb - y0 + 1);
            bool twice = false;
            if (va && atomicCAS(&cell[ca], 0u, (unsigned)a + 1u) != 0u) twice = true;
            if (vb && atomicCAS(&cell[cb], 0u, (unsigned)b + 1u) != 0u) twice = true;
            __syncwarp();
            grid = !__any_sync(FULL, twice);
            if (grid) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const bool v = h ? vb : va;
                    if (!v) continue;
                    const int c = h ? cb : ca, t = h ? tb : ta;
                    const unsigned o = h ? ob : oa;
                    const long long ix = h ? ib : ia;
                    unsigned long long row = 0;
                    bool np = false;
#pragma unroll
                    for (int d = 0; d < 9; ++d) {
                        if (d == 4) continue;
                        const unsigned j1 = cell[c + (d % 3 - 1) + 16 * (d / 3 - 1)];
                        if (!j1) continue;
                        const int j = (int)j1 - 1;
                        if (abs(W.tofb[j] - t) > dt) continue;
                        row |= 1ull << j;
                        const unsigned oj = W.tot[j];
                        if (oj > o || (oj == o && s.index[s0 + j] > ix)) np = true;
                    }
                    if (h) { rowB = row; npB = np; } else { rowA = row; npA = np; }
                }
            }
            __syncwarp();
        }
    }
    const unsigned rxy = (unsigned)rx | ((unsigned)ry << 8);   // per-byte box radii
    for (int k = 0; k < (grid ? 0 : L); ++k) {
        const bool kb = k >= 32;
        const int src = k & 31;
        const int kt = __shfl_sync(FULL, kb ? tb : ta, src);
        const unsigned kp = __shfl_sync(FULL, kb ? pb : pa, src);
        const unsigned ko = __shfl_sync(FULL, kb ? ob : oa, src);
        const bool adjA = va && a != k && abs(ta - kt) <= dt && __vcmpleu4(__vabsdiffu4(pa, kp), rxy) == FULL;
        const bool adjB = vb && b != k && abs(tb - kt) <= dt && __vcmpleu4(__vabsdiffu4(pb, kp), rxy) == FULL;
        const unsigned lo = __ballot_sync(FULL, adjA), hi = __ballot_sync(FULL, adjB);
        bool brA = adjA && oa > ko, brB = adjB && ob > ko;
        const bool tA = adjA && oa == ko, tB = adjB && ob == ko;
        if (__any_sync(FULL, tA || tB)) {   // Sec. V.B ties: the later hit in the stream wins
            const long long ki = __shfl_sync(FULL, kb ? ib : ia, src);
            brA = brA || (tA && ia > ki);
            brB = brB || (tB && ib > ki);
        }
        const bool knp = __any_sync(FULL, brA || brB);
        if (lane == src) {
            const unsigned long long row = ((unsigned long long)hi << 32) | lo;
            if (kb) { rowB = row; npB = knp; } else { rowA = row; npA = knp; }
        }
    }
    const bool pkA = va && !npA, pkB = vb && !npB;
    if (!cc) {   // PAPER mode: every hit is its own label; local maxima carry the records
        if (va) {
            if (labels) labels[ha] = ia;
            if (is_peak) is_peak[ha] = pkA;
            if (rflag) rflag[ha] = emit && pkA;
        }
        if (vb) {
            if (labels) labels[hb] = ib;
            if (is_peak) is_peak[hb] = pkB;
            if (rflag) rflag[hb] = emit && pkB;
        }
        return;
    }
    const unsigned long long peaks = ((unsigned long long)__ballot_sync(FULL, pkB) << 32) | __ballot_sync(FULL, pkA);
    unsigned long long todo = L == 64 ? ~0ull : ((1ull << L) - 1ull);
    long long rootA = 0, rootB = 0;
    int rposA = -1, rposB = -1;
    while (todo) {
        const int seed = __ffsll((long long)todo) - 1;
        unsigned long long comp = 1ull << seed, front = comp;
        while (front) {
            unsigned long long c = 0;
            if ((front >> a) & 1ull) c |= rowA;
            if ((front >> b) & 1ull) c |= rowB;
            const unsigned lo = __reduce_or_sync(FULL, (unsigned)c);
            const unsigned hi = __reduce_or_sync(FULL, (unsigned)(c >> 32));
            const unsigned long long nb = ((unsigned long long)hi << 32) | lo;
            front = nb & ~comp;
            comp |= nb;
        }
        const long long sidx = __shfl_sync(FULL, seed >= 32 ? ib : ia, seed & 31);
        const bool inA = (comp >> a) & 1ull, inB = (comp >> b) & 1ull;
        if (inA) { rootA = sidx; rposA = seed; }
        if (inB) { rootB = sidx; rposB = seed; }
        if (acc && emit) {
            const int st = __shfl_sync(FULL, seed >= 32 ? tb : ta, seed & 31);
            unsigned long long v_tot = 0, v_x = 0, v_y = 0, v_t = 0;
            if (inA) { v_tot += oa; v_x += (unsigned long long)oa * (pa & 255u); v_y += (unsigned long long)oa * (pa >> 8);
                       v_t += (unsigned long long)(ta - st) * oa; }
            if (inB) { v_tot += ob; v_x += (unsigned long long)ob * (pb & 255u); v_y += (unsigned long long)ob * (pb >> 8);
                       v_t += (unsigned long long)(tb - st) * ob; }
            v_tot = warp_sum_u64(v_tot);
            v_x = warp_sum_u64(v_x);
            v_y = warp_sum_u64(v_y);
            v_t = warp_sum_u64(v_t);
            if (lane == (seed & 31)) {
                AccH r;
                r.s_tot = (long long)v_tot; r.s_x = (long long)v_x; r.s_y = (long long)v_y; r.s_t = (long long)v_t;
                r.n = (unsigned)__popcll(comp); r.npk = (unsigned)__popcll(comp & peaks);
                acc[seed >= 32 ? hb : ha] = r;
            }
        }
        todo &= ~comp;
    }
    if (va) {
        if (labels) labels[ha] = rootA;
        if (is_peak) is_peak[ha] = pkA;
        if (rflag) rflag[ha] = emit && rposA == a;
    }
    if (vb) {
        if (labels) labels[hb] = rootB;
        if (is_peak) is_peak[hb] = pkB;
        if (rflag) rflag[hb] = emit && rposB == b;
    }
}

// One warp per segment. Up to 64 hits: in registers (seg_small). Up to
// WCAP: in shared memory, where a cell hash of the segment gives every hit
// the candidates of the forward half of its box (same cell: later positions
// only), so that each adjacent pair is met once even when the whole segment
// lies within dt; pairs set the local-maximum flags and are joined by
// hooking rounds; then labels, peaks, root flags (emitted shots only) and
// the root's int64 moments. Longer segments are marked for the cell-hash
// kernels in global memory below.
__global__ void __launch_bounds__(SEGW * 32) k_segments(Sorted s, const long long *seg_start, const long long *nseg_p,
                                                        int rx, int ry, int dt, int cc, long long shot_limit,
                                                        long long *labels, unsigned char *is_peak, unsigned *rflag,
                                                        AccH *acc, unsigned char *mark) {
    __shared__ SegSm sm[SEGW];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    SegSm &W = sm[wi];
    const long long nseg = *nseg_p;
    for (long long seg = blockIdx.x * (long long)SEGW + wi; seg < nseg; seg += (long long)gridDim.x * SEGW) {
        const long long s0 = seg_start[seg], len = seg_start[seg + 1] - s0;
        if (len > WCAP) {
            for (long long k = lane; k < len; k += 32) mark[s0 + k] = 1;
            continue;
        }
        const int L = (int)len;
        const bool emit = s.shot[s0] < shot_limit;
        const bool sums = cc && acc && emit;
        if (L > 1 && L <= WREG) {
            seg_small(s, s0, L, rx, ry, dt, cc, emit, labels, is_peak, rflag, sums ? acc : nullptr, lane, W);
            continue;
        }
        if (L == 1) {
            if (lane == 0) {
                const unsigned hh = s.hit[s0];
                if (labels) labels[hh] = s.index[s0];
                if (is_peak) is_peak[hh] = 1;
                if (rflag) rflag[hh] = emit;
                if (sums) {
                    const long long t = s.tot[s0];
                    AccH a;
                    a.s_tot = t; a.s_x = t * s.x[s0]; a.s_y = t * s.y[s0]; a.s_t = 0; a.n = 1; a.npk = 1;
                    acc[hh] = a;
                }
            }
            continue;
        }
        for (int k = lane; k < L; k += 32) {
            W.tofb[k] = s.tofb[s0 + k];
            W.x[k] = s.x[s0 + k];
            W.y[k] = s.y[s0 + k];
            W.tot[k] = s.tot[s0 + k];
            W.parent[k] = k;
            W.np[k] = 0;
        }
        for (int b = lane; b < HBW; b += 32) W.hhead[b] = 0xFFFFu;
        if (lane == 0) W.ecnt = 0;
        __syncwarp();
        for (int k = lane; k < L; k += 32) W.hnext[k] = (unsigned short)atomicExch(&W.hhead[wcell(W.x[k], W.y[k])], (unsigned)k);
        __syncwarp();
        for (int k = lane; k < L; k += 32) {
            const int tb = W.tofb[k], xk = W.x[k], yk = W.y[k], tk = W.tot[k];
            for (int dx = 0; dx <= rx; ++dx) {
                const int cx = xk + dx;
                if (cx > 255) break;
                for (int dy = (dx == 0 ? 0 : -ry); dy <= ry; ++dy) {
                    const int cy = yk + dy;
                    if (cy < 0 || cy > 255) continue;
                    for (unsigned j = W.hhead[wcell(cx, cy)]; j != 0xFFFFu; j = W.hnext[j]) {
                        if (dx == 0 && dy == 0 && (int)j <= k) continue;
                        if (W.x[j] != cx || W.y[j] != cy) continue;
                        const int d = W.tofb[j] - tb;
                        if (d < -dt || d > dt) continue;
                        // the pair (lo, hi) in position order
                        const int lo = min(k, (int)j), hi = max(k, (int)j);
                        if (j_brighter(W.tot[j], tk, s.index, s0 + j, s0 + k)) W.np[k] = 1; else W.np[j] = 1;
                        if (cc) {   // record the pair (warp-aggregated slot); beyond the buffer, join it now
                            const unsigned am = __activemask();
                            const int leader = __ffs(am) - 1;
                            unsigned slot = 0;
                            if (lane == leader) slot = atomicAdd(&W.ecnt, (unsigned)__popc(am));
                            slot = __shfl_sync(am, slot, leader) + __popc(am & ((1u << lane) - 1u));
                            if (slot < (unsigned)ECAP) W.edge[slot] = ((unsigned)lo << 16) | (unsigned)hi;
                            else s_unite(W.parent, lo, hi);
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (cc) {
            // rounds of: pointer jumping until every hit points at its root,
            // then every recorded pair whose roots differ hooks the larger
            // root onto the smaller one (CAS on a root only, so no link is
            // ever overwritten); until no pair has two roots. Pointers only
            // go to smaller positions, so the root is the earliest hit.
            const int m = min((int)W.ecnt, ECAP);
            for (;;) {
                for (;;) {
                    bool moved = false;
                    for (int k = lane; k < L; k += 32) {
                        const int p = W.parent[k], pp = W.parent[p];
                        if (pp != p) { W.parent[k] = pp; moved = true; }
                    }
                    __syncwarp();
                    if (!__any_sync(0xffffffffu, moved)) break;
                }
                bool hooked = false;
                for (int e = lane; e < m; e += 32) {
                    const unsigned ed = W.edge[e];
                    const int a = W.parent[ed >> 16], b = W.parent[ed & 0xFFFFu];
                    if (a != b) {
                        atomicCAS(&W.parent[max(a, b)], max(a, b), min(a, b));
                        hooked = true;
                    }
                }
                __syncwarp();
                if (!__any_sync(0xffffffffu, hooked)) break;
            }
        }
        __syncwarp();
        // roots of every hit (full compression; only reads after the barrier)
        int rk[WCAP / 32];
#pragma unroll
        for (int u = 0; u < WCAP / 32; ++u) {
            const int k = u * 32 + lane;
            rk[u] = (k < L && cc) ? s_find(W.parent, k) : k;
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < WCAP / 32; ++u) {
            const int k = u * 32 + lane;
            if (k < L) W.parent[k] = rk[u];
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < WCAP / 32; ++u) {
            const int k = u * 32 + lane;
            if (k >= L) break;
            const int r = rk[u];
            const unsigned hh = s.hit[s0 + k];
            const bool peak = W.np[k] == 0;
            if (labels) labels[hh] = s.index[s0 + r];
            if (is_peak) is_peak[hh] = peak;
            if (rflag) rflag[hh] = emit && (cc ? r == k : peak);
        }
        if (sums) {
            // each root's lane sweeps the segment once (broadcast reads, no
            // atomics): exact 64-bit moments in registers
            for (int base = 0; base < L; base += 32) {
                const int k = base + lane;
                const bool own = k < L && W.parent[k] == k;
                if (__ballot_sync(0xffffffffu, own) == 0) continue;
                unsigned long long st = 0, sx = 0, sy = 0, stt = 0;
                unsigned cnt = 0, npk = 0;
                const int tk = own ? W.tofb[k] : 0;
                for (int j = own ? k : L; j < L; ++j) {   // members sit at or after their root
                    if (W.parent[j] != k) continue;
                    const unsigned long long t = W.tot[j];
                    st += t;
                    sx += t * W.x[j];
                    sy += t * W.y[j];
                    stt += (unsigned long long)(W.tofb[j] - tk) * t;
                    cnt += 1;
                    npk += W.np[j] == 0;
                }
                if (own) {
                    AccH a;
                    a.s_tot = (long long)st; a.s_x = (long long)sx; a.s_y = (long long)sy; a.s_t = (long long)stt;
                    a.n = cnt; a.npk = npk;
                    acc[s.hit[s0 + k]] = a;
                }
            }
        }
        __syncwarp();
    }
}

// ---- segments longer than WCAP: the same rules through global memory ----
__device__ __forceinline__ int g_find(int *parent, int x) {
    for (;;) {
        const int p = ((volatile int *)parent)[x];
        if (p == x) return x;
        const int g = ((volatile int *)parent)[p];
        if (g == p) return p;
        ((volatile int *)parent)[x] = g;
        x = g;
    }
}
__device__ void g_unite(int *parent, int a, int b) {
    for (;;) {
        a = g_find(parent, a);
        b = g_find(parent, b);
        if (a == b) return;
        if (a > b) { const int t = a; a = b; b = t; }
        const int old = atomicCAS(&parent[b], b, a);
        if (old == b) return;
        b = old;
    }
}
__global__ void k_long_init(Sorted s, long long n, const unsigned char *mark, int *parent, unsigned char *notpeak,
                            AccH *acc) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!mark[i]) continue;
        parent[i] = (int)i;
        notpeak[i] = 0;
        if (acc) {
            AccH z;
            z.s_tot = 0; z.s_x = 0; z.s_y = 0; z.s_t = 0; z.n = 0; z.npk = 0;
            acc[s.hit[i]] = z;
        }
    }
}
// Long segments can hold thousands of hits within dt of each other (a shot
// of many particles arriving together), so their pairs come from a hash of
// (shot, x, y) cells: every hit looks up the cells of the forward half of its
// box (same cell: later positions only), which meets each adjacent pair once.
__device__ __forceinline__ unsigned long long cell_hash(long long shot, int x, int y, unsigned long long mask) {
    unsigned long long k = ((unsigned long long)shot << 16) ^ ((unsigned long long)x << 8) ^ (unsigned long long)y;
    k *= 0x9E3779B97F4A7C15ull;   // Fibonacci hashing
    return (k >> 20) & mask;
}
// a marked hit's cell and time in one word for the pair search: x, y, the
// shot's low 16 bits, ToF + bias (the full shot is compared on a match)
__device__ __forceinline__ unsigned cell_key(long long shot, int x, int y) {
    return (unsigned)x | ((unsigned)y << 8) | ((unsigned)(shot & 0xFFFF) << 16);
}
__global__ void k_long_insert(Sorted s, long long n, const unsigned char *mark, unsigned *head, unsigned *next,
                              unsigned long long *word, unsigned long long mask) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!mark[i]) continue;
        const long long sh = s.shot[i];
        const int x = s.x[i], y = s.y[i];
        word[i] = (unsigned long long)cell_key(sh, x, y) | ((unsigned long long)(unsigned)s.tofb[i] << 32);
        next[i] = atomicExch(&head[cell_hash(sh, x, y, mask)], (unsigned)i);
    }
}
__global__ void k_long_pairs(Sorted s, long long n, const unsigned char *mark, const unsigned *head,
                             const unsigned *next, const unsigned long long *word, unsigned long long mask, int rx,
                             int ry, int dt, int cc, int *parent, unsigned char *notpeak) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!mark[i]) continue;
        const unsigned long long wi = word[i];
        const long long sh = s.shot[i];
        const int tb = (int)(unsigned)(wi >> 32), xi = (int)(wi & 255), yi = (int)((wi >> 8) & 255), ti = s.tot[i];
        for (int dx = 0; dx <= rx; ++dx) {
            const int cx = xi + dx;
            if (cx > 255) break;
            for (int dy = (dx == 0 ? 0 : -ry); dy <= ry; ++dy) {
                const int cy = yi + dy;
                if (cy < 0 || cy > 255) continue;
                const unsigned key = cell_key(sh, cx, cy);
                for (unsigned j = head[cell_hash(sh, cx, cy, mask)]; j != 0xFFFFFFFFu; j = next[j]) {
                    if (dx == 0 && dy == 0 && (long long)j <= i) continue;
                    const unsigned long long wj = word[j];
                    if ((unsigned)wj != key || s.shot[j] != sh) continue;
                    const int d = (int)(unsigned)(wj >> 32) - tb;
                    if (d < -dt || d > dt) continue;
                    if (j_brighter(s.tot[j], ti, s.index, j, i)) notpeak[i] = 1; else notpeak[j] = 1;
                    if (cc) g_unite(parent, (int)i, (int)j);
                }
            }
        }
    }
}
__global__ void k_long_finish(Sorted s, long long n, const unsigned char *mark, int cc, long long shot_limit,
                              int *parent, const unsigned char *notpeak, long long *labels, unsigned char *is_peak,
                              unsigned *rflag, AccH *acc) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!mark[i]) continue;
        const long long r = cc ? g_find(parent, (int)i) : i;
        const unsigned hh = s.hit[i];
        const bool peak = notpeak[i] == 0, emit = s.shot[i] < shot_limit;
        if (labels) labels[hh] = s.index[r];
        if (is_peak) is_peak[hh] = peak;
        if (rflag) rflag[hh] = emit && (cc ? r == i : peak);
        if (cc && acc && emit) {
            AccH &a = acc[s.hit[r]];
            const unsigned long long t = s.tot[i];
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.s_tot), t);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.s_x), t * s.x[i]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.s_y), t * s.y[i]);
            atomicAdd(reinterpret_cast<unsigned long long *>(&a.s_t), (unsigned long long)(s.tofb[i] - s.tofb[r]) * t);
            atomicAdd(&a.n, 1u);
            if (peak) atomicAdd(&a.npk, 1u);
        }
    }
}

// ------------------------------------------------------------ centroid kernels
__global__ void k_root_flags(tpx_hits h, const long long *labels, const unsigned char *is_peak, long long n, int cc,
                             unsigned *flags) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        flags[i] = cc ? (labels[i] == h.index[i]) : (unsigned)is_peak[i];
}

__device__ __forceinline__ long long find_index(const long long *index, long long n, long long v) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (index[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

struct Acc { unsigned long long n, s_tot, s_x, s_y, s_t, npk; };

__global__ void k_accum(tpx_hits h, const long long *labels, const unsigned char *is_peak, long long n,
                        const unsigned *cid, Acc *acc) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long rp = find_index(reinterpret_cast<const long long *>(h.index), n, labels[i]);
        const unsigned c = cid[rp];
        const unsigned long long tot = h.tot[i];
        atomicAdd(&acc[c].n, 1ull);
        atomicAdd(&acc[c].s_tot, tot);
        atomicAdd(&acc[c].s_x, tot * h.x[i]);
        atomicAdd(&acc[c].s_y, tot * h.y[i]);
        atomicAdd(&acc[c].s_t, tot * (unsigned long long)(h.t[i] - h.t[rp]));
        if (is_peak && is_peak[i]) atomicAdd(&acc[c].npk, 1ull);
    }
}

__global__ void k_final(tpx_hits h, long long n, const unsigned *flags, const unsigned *cid, const Acc *acc,
                        tpx_record *out, long long cap) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!flags[i]) continue;
        const long long c = cid[i];
        if (c >= cap) continue;
        const Acc a = acc[c];
        tpx_record o;
        o.label = h.index[i];
        o.shot = h.shot[i];
        o.t0 = h.t[i];
        o.s_tot = (long long)a.s_tot; o.s_x = (long long)a.s_x; o.s_y = (long long)a.s_y; o.s_t = (long long)a.s_t;
        o.n = (int)a.n; o.n_peaks = (int)a.npk;
        com_from_moments(o.s_x, o.s_y, o.s_t, o.s_tot, h.tof[i], &o.x, &o.y, &o.tof);
        out[c] = o;
    }
}

// PAPER mode: each local maximum sums its box neighbourhood (both directions
// in sorted order, within dt)
__global__ void k_paper(Sorted s, long long n, int rx, int ry, int dt, const unsigned *flag_hit,
                        const unsigned *cid_hit, tpx_hits h, tpx_record *out, long long cap) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned hi = s.hit[i];
        if (!flag_hit[hi]) continue;
        const long long c = cid_hit[hi];
        if (c >= cap) continue;
        const long long sh = s.shot[i];
        const int tb = s.tofb[i], xi = s.x[i], yi = s.y[i];
        long long m = 0, st = 0, sx = 0, sy = 0, a2 = 0;
        int tmin = tb;
        for (int dir = -1; dir <= 1; dir += 2) {
            for (long long j = (dir < 0 ? i : i + 1); j >= 0 && j < n; j += dir) {
                if (s.shot[j] != sh) break;
                const int d = s.tofb[j] - tb;
                if (d > dt || d < -dt) break;
                const int dx = (int)s.x[j] - xi, dy = (int)s.y[j] - yi;
                if (dx < -rx || dx > rx || dy < -ry || dy > ry) continue;
                const long long tj = s.tot[j];
                m += 1; st += tj; sx += tj * s.x[j]; sy += tj * s.y[j]; a2 += tj * s.tofb[j];
                tmin = min(tmin, s.tofb[j]);
            }
        }
        tpx_record o;
        o.label = s.index[i];
        o.shot = sh;
        const long long tofc0 = (long long)tmin - kBias;
        o.t0 = h.t[hi] - h.tof[hi] + tofc0;
        o.s_tot = st; o.s_x = sx; o.s_y = sy; o.s_t = a2 - (long long)tmin * st;
        o.n = (int)m; o.n_peaks = 1;
        com_from_moments(sx, sy, o.s_t, st, tofc0, &o.x, &o.y, &o.tof);
        out[c] = o;
    }
}

// number of records; latches the capacity status and the clusters counter
__global__ void k_count_from_scan(const unsigned *flags, const unsigned *cid, long long n, long long *out,
                                  long long cap, unsigned *status, unsigned long long *counter) {
    const long long m = n ? (long long)cid[n - 1] + flags[n - 1] : 0;
    *out = m;
    if (m > cap) atomicOr(status, ST_CLUSTER_CAP);
    if (counter) *counter = (unsigned long long)m;
}

// position of every record's root hit, in record (label) order
__global__ void k_root_list(const unsigned *rflag, const unsigned *cid, long long n, long long cap, unsigned *rootpos) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (rflag[i] && cid[i] < cap) rootpos[cid[i]] = (unsigned)i;
}
// CC records from the per-root moments, one thread per record
__global__ void k_records(tpx_hits h, const long long *n_rec, long long cap, const unsigned *rootpos, const AccH *acc,
                          tpx_record *out) {
    const long long m = min(*n_rec, cap);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < m; c += (long long)gridDim.x * blockDim.x) {
        const long long i = rootpos[c];
        const AccH a = acc[i];
        tpx_record o;
        o.label = h.index[i];
        o.shot = h.shot[i];
        o.t0 = h.t[i];
        o.s_tot = a.s_tot; o.s_x = a.s_x; o.s_y = a.s_y; o.s_t = a.s_t;
        o.n = (int)a.n; o.n_peaks = (int)a.npk;
        com_from_moments(o.s_x, o.s_y, o.s_t, o.s_tot, h.tof[i], &o.x, &o.y, &o.tof);
        out[c] = o;
    }
}

// ------------------------------------------------------------ host helpers
// a failed CUDA call becomes TPX_ECUDA; with TPX_DEBUG set in the
// environment its error is also printed to stderr
inline int ck(cudaError_t e, int line = __builtin_LINE()) {
    if (e == cudaSuccess) return TPX_OK;
    if (std::getenv("TPX_DEBUG")) std::fprintf(stderr, "tpx_general.cu:%d: %s\n", line, cudaGetErrorString(e));
    return TPX_ECUDA;
}
inline unsigned grid_for(long long n) {
    long long g = (n + GT - 1) / GT;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (unsigned)g;
}

struct Arena {
    char *p;
    size_t used, cap;
    template <class T>
    T *take(long long count) {
        const size_t b = ((size_t)(count > 0 ? count : 1) * sizeof(T) + 255) & ~size_t(255);
        T *r = reinterpret_cast<T *>(p + used);
        used += b;
        return r;
    }
};
inline size_t sz(long long count, size_t elem) { return ((size_t)(count > 0 ? count : 1) * elem + 255) & ~size_t(255); }

int reserve(tpx_ctx *c, size_t bytes) {
    if (c->g_mem && c->g_bytes >= bytes) return TPX_OK;
    if (ck(cudaStreamSynchronize(c->stream))) return TPX_ECUDA;
    if (c->g_mem) cudaFree(c->g_mem);
    c->g_mem = nullptr;
    c->g_bytes = 0;
    if (cudaMalloc(&c->g_mem, bytes) != cudaSuccess) { cudaGetLastError(); return TPX_ENOMEM; }
    c->g_bytes = bytes;
    return TPX_OK;
}

// exclusive scan of n unsigned counts into out (a.used advanced for temporaries)
int scan_u32(Arena &a, const unsigned *in, unsigned *out, long long n, cudaStream_t s) {
    const long long nb = (n + GTILE - 1) / GTILE;
    unsigned *bsum = a.take<unsigned>(nb);
    k_scan_blocks<<<(unsigned)(nb > 0 ? nb : 1), GT, 0, s>>>(in, out, n, bsum);
    k_scan_bsum<<<1, PT, 0, s>>>(bsum, nb);
    k_scan_add<<<grid_for(n), GT, 0, s>>>(out, n, bsum);
    return ck(cudaGetLastError());
}

size_t sort_bytes(long long n) {
    const long long tiles = (n + GTILE - 1) / GTILE;
    return 2 * sz(n, 8) + 2 * sz(n, 4) + 2 * sz(256 * tiles, 4) + sz((256 * tiles + GTILE - 1) / GTILE + 1, 4) +
           sz(2, 8) + 4096;
}

// sort the hits by (shot, corrected ToF); returns the sorted values buffer.
// shot_span >= 0 bounds max shot - min shot (no host round trip); < 0 reads it.
int sort_hits(tpx_ctx *c, Arena &a, const tpx_hits &h, long long n, long long shot_span, unsigned **vals_out) {
    cudaStream_t s = c->stream;
    const long long tiles = (n + GTILE - 1) / GTILE;
    unsigned long long *k0 = a.take<unsigned long long>(n), *k1 = a.take<unsigned long long>(n);
    unsigned *v0 = a.take<unsigned>(n), *v1 = a.take<unsigned>(n);
    unsigned *hist = a.take<unsigned>(256 * tiles), *offs = a.take<unsigned>(256 * tiles);
    unsigned long long *mm = a.take<unsigned long long>(2);   // min, max shot
    const unsigned long long init[2] = {~0ull, 0ull};
    if (ck(cudaMemcpyAsync(mm, init, sizeof init, cudaMemcpyHostToDevice, s))) return TPX_ECUDA;
    k_shot_range<<<grid_for(n), GT, 0, s>>>(h, n, mm, mm + 1);
    k_make_keys<<<grid_for(n), GT, 0, s>>>(h, n, mm, k0, v0);
    unsigned long long span = (unsigned long long)shot_span;
    if (shot_span < 0) {
        unsigned long long hm[2] = {0, 0};
        if (ck(cudaMemcpyAsync(hm, mm, sizeof hm, cudaMemcpyDeviceToHost, s))) return TPX_ECUDA;
        if (ck(cudaStreamSynchronize(s))) return TPX_ECUDA;
        span = hm[1] - hm[0];
    }
    int bits = 24;
    while (bits < 64 && (span >> (bits - 24)) != 0) ++bits;
    const size_t mark = a.used;
    for (int shift = 0; shift < bits; shift += 8) {
        a.used = mark;
        k_sort_hist<<<(unsigned)tiles, GT, 0, s>>>(k0, n, shift, hist, tiles);
        int rc = scan_u32(a, hist, offs, 256 * tiles, s);
        if (rc) return rc;
        k_sort_scatter<<<(unsigned)tiles, GT, 0, s>>>(k0, v0, n, shift, offs, tiles, k1, v1);
        unsigned long long *tk = k0; k0 = k1; k1 = tk;
        unsigned *tv = v0; v0 = v1; v1 = tv;
    }
    a.used = mark;
    *vals_out = v0;
    return ck(cudaGetLastError());
}

size_t decode_bytes(long long n) {
    const long long tiles = (n + GTILE - 1) / GTILE;
    return sz(tiles, sizeof(GAgg)) * 2 + sz(tiles + 1, 8) * 4 + sz(n, 8) + 4096;
}

int decode_impl(tpx_ctx *c, const uint64_t *pk, int64_t n, int64_t base, const tpx_hits &h, int64_t cap,
                int64_t *d_n_hits, int64_t *trig, int64_t trig_cap, int64_t *d_n_trig, bool clear_ctl,
                const GAgg *E0, GAgg *state_out, long long *trig_pos, long long **t_all_out) {
    cudaStream_t s = c->stream;
    const long long tiles = (n + GTILE - 1) / GTILE;
    int rc = reserve(c, decode_bytes(n));
    if (rc) return rc;
    Arena a{static_cast<char *>(c->g_mem), 0, c->g_bytes};
    GAgg *tagg = a.take<GAgg>(tiles), *tpre = a.take<GAgg>(tiles);
    long long *tcnt = a.take<long long>(tiles + 1), *toff = a.take<long long>(tiles + 1);
    long long *tkept = a.take<long long>(tiles + 1), *tkoff = a.take<long long>(tiles + 1);
    long long *t_all = a.take<long long>(n);
    if (t_all_out) *t_all_out = t_all;
    if (clear_ctl && cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), s) != cudaSuccess) return TPX_ECUDA;
    if (cudaMemsetAsync(d_n_hits, 0, 8, s) != cudaSuccess || cudaMemsetAsync(d_n_trig, 0, 8, s) != cudaSuccess)
        return TPX_ECUDA;
    if (n == 0) {   // the state passes through unchanged
        if (!state_out) return TPX_OK;
        if (E0) return ck(cudaMemcpyAsync(state_out, E0, sizeof(GAgg), cudaMemcpyDeviceToDevice, s));
        return ck(cudaMemsetAsync(state_out, 0, sizeof(GAgg), s));
    }
    const long long tp = c->cfg.wrap_thr_pix_ticks, tt = c->cfg.wrap_thr_tdc_ticks;
    long long *ntr = reinterpret_cast<long long *>(d_n_trig);
    long long *tr = reinterpret_cast<long long *>(trig);
    k_tile_agg<<<(unsigned)tiles, GT, 0, s>>>(pk, n, tp, tt, tagg, tcnt);
    k_tile_prefix<<<1, PT, 0, s>>>(tagg, tpre, tcnt, toff, tiles, tp, tt, ntr, E0, state_out);
    k_unwrap<<<(unsigned)tiles, GT, 0, s>>>(pk, n, tpre, toff, tp, tt, t_all, tr, trig_cap, &c->ctl->status, trig_pos);
    k_check_trig<<<152, GT, 0, s>>>(tr, ntr, trig_cap, &c->ctl->status);
    k_bin<<<(unsigned)tiles, GT, 0, s>>>(pk, n, t_all, tr, ntr, trig_cap, c->cfg.tof_max_ticks, tkept,
                                         c->ctl->counters);
    k_count_prefix<<<1, PT, 0, s>>>(tkept, tkoff, tiles, reinterpret_cast<long long *>(d_n_hits));
    k_compact<<<(unsigned)tiles, GT, 0, s>>>(pk, n, base, t_all, tr, ntr, trig_cap, c->cfg.tof_max_ticks,
                                             c->cfg.d_timewalk_lut, tkoff, h, cap, &c->ctl->status, E0);
    const unsigned long long np = (unsigned long long)n;
    if (cudaMemcpyAsync(&c->ctl->counters[C_PACKETS], &np, 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TPX_ECUDA;
    return ck(cudaGetLastError());
}

size_t cluster_bytes(long long n) {
    return sort_bytes(n) + sz(n, 4) + sz(n, 8) * 2 + sz(n, 4) + sz(n, 2) + 2 * sz(n, 1)   // sorted hits
           + 2 * sz(n, 4) + sz(n + 1, 8) + sz(1, 8)                                     // segments
           + 2 * sz(n, 1) + sz(n, 4)                                                    // long segments
           + 2 * sz(n, 4) + sz(n, sizeof(AccH)) + sz((n + GTILE - 1) / GTILE + 1, 4)    // records
           + sz(4 * n + 2, 4) + sz(n, 4) + sz(n, 8)                                    // long-segment hash
           + 8192;
}

// The whole clustering stage: sort, segments, labels, local maxima and, when
// `out` is given, the records of the hits whose shot is below shot_limit.
// labels / is_peak (per hit) may be NULL. No host round trip when
// shot_span >= 0.
int cluster_all(tpx_ctx *c, const tpx_hits &h, int64_t n, int64_t *labels, uint8_t *is_peak, long long shot_limit,
                long long shot_span, tpx_record *out, int64_t cap, int64_t *d_n_clusters) {
    cudaStream_t s = c->stream;
    const int cc = c->cfg.mode == TPX_MODE_CC;
    if (out && cudaMemsetAsync(d_n_clusters, 0, 8, s) != cudaSuccess) return TPX_ECUDA;
    if (n <= 0) return TPX_OK;
    int rc = reserve(c, cluster_bytes(n));
    if (rc) return rc;
    Arena a{static_cast<char *>(c->g_mem), 0, c->g_bytes};
    Sorted so;
    so.hit = a.take<unsigned>(n);
    so.shot = a.take<long long>(n);
    so.index = a.take<long long>(n);
    so.tofb = a.take<int>(n);
    so.tot = a.take<unsigned short>(n);
    so.x = a.take<unsigned char>(n);
    so.y = a.take<unsigned char>(n);
    unsigned *segf = a.take<unsigned>(n), *sego = a.take<unsigned>(n);
    long long *seg_start = a.take<long long>(n + 1), *nseg = a.take<long long>(1);
    unsigned char *mark = a.take<unsigned char>(n), *notpeak = a.take<unsigned char>(n);
    int *parent = a.take<int>(n);
    unsigned *rflag = a.take<unsigned>(n), *cid = a.take<unsigned>(n);
    AccH *acc = a.take<AccH>(n);
    unsigned long long lmask = 1;   // the long segments' cell hash: >= 2n buckets
    while (lmask + 1 < 2ull * (unsigned long long)n) lmask = 2 * lmask + 1;
    unsigned *lhead = a.take<unsigned>((long long)lmask + 1), *lnext = a.take<unsigned>(n);
    unsigned long long *lword = a.take<unsigned long long>(n);
    const size_t mark_used = a.used;
    unsigned *vals = nullptr;
    rc = sort_hits(c, a, h, n, shot_span, &vals);
    if (rc) return rc;
    k_gather<<<grid_for(n), GT, 0, s>>>(h, vals, n, so);
    a.used = mark_used;   // the sort's scratch is free again
    const int dt = c->cfg.dt_ticks;
    k_seg_flags<<<grid_for(n), GT, 0, s>>>(so, n, dt, segf);
    rc = scan_u32(a, segf, sego, n, s);
    if (rc) return rc;
    k_seg_starts<<<grid_for(n), GT, 0, s>>>(segf, sego, n, seg_start, nseg);
    if (ck(cudaMemsetAsync(mark, 0, (size_t)n, s))) return TPX_ECUDA;
    long long *lab = reinterpret_cast<long long *>(labels);
    unsigned *rf = out ? rflag : nullptr;
    AccH *ac = (out && cc) ? acc : nullptr;
    int seg_blocks = c->num_sms * 8;
    if ((long long)seg_blocks * SEGW > n) seg_blocks = (int)((n + SEGW - 1) / SEGW);
    k_segments<<<seg_blocks, SEGW * 32, 0, s>>>(so, seg_start, nseg, c->cfg.rx, c->cfg.ry, dt, cc, shot_limit, lab,
                                                is_peak, rf, ac, mark);
    k_long_init<<<grid_for(n), GT, 0, s>>>(so, n, mark, parent, notpeak, ac);
    if (ck(cudaMemsetAsync(lhead, 0xFF, sizeof(unsigned) * (size_t)(lmask + 1), s))) return TPX_ECUDA;
    k_long_insert<<<grid_for(n), GT, 0, s>>>(so, n, mark, lhead, lnext, lword, lmask);
    k_long_pairs<<<grid_for(n), GT, 0, s>>>(so, n, mark, lhead, lnext, lword, lmask, c->cfg.rx, c->cfg.ry, dt, cc,
                                            parent, notpeak);
    k_long_finish<<<grid_for(n), GT, 0, s>>>(so, n, mark, cc, shot_limit, parent, notpeak, lab, is_peak, rf, ac);
    if (!out) return ck(cudaGetLastError());
    rc = scan_u32(a, rflag, cid, n, s);
    if (rc) return rc;
    k_count_from_scan<<<1, 1, 0, s>>>(rflag, cid, n, reinterpret_cast<long long *>(d_n_clusters), cap,
                                      &c->ctl->status, &c->ctl->counters[C_CLUSTERS]);
    if (cc) {
        unsigned *rootpos = segf;   // free again: the segments are done
        k_root_list<<<grid_for(n), GT, 0, s>>>(rflag, cid, n, cap, rootpos);
        k_records<<<grid_for(n / 16 + 1), GT, 0, s>>>(h, reinterpret_cast<const long long *>(d_n_clusters), cap, rootpos,
                                                     acc, out);
    } else
        k_paper<<<grid_for(n), GT, 0, s>>>(so, n, c->cfg.rx, c->cfg.ry, dt, rflag, cid, h, out, cap);
    return ck(cudaGetLastError());
}

int cluster_impl(tpx_ctx *c, const tpx_hits &h, int64_t n, int64_t *labels, uint8_t *is_peak) {
    return cluster_all(c, h, n, labels, is_peak, LLONG_MAX, -1, nullptr, 0, nullptr);
}

int centroid_impl(tpx_ctx *c, const tpx_hits &h, const int64_t *labels, const uint8_t *is_peak, int64_t n,
                  tpx_record *out, int64_t cap, int64_t *d_n_clusters) {
    cudaStream_t s = c->stream;
    if (ck(cudaMemsetAsync(d_n_clusters, 0, 8, s))) return TPX_ECUDA;
    if (n <= 0) return TPX_OK;
    const int cc = c->cfg.mode == TPX_MODE_CC;
    if (!cc && !is_peak) return TPX_EINVAL;
    const size_t need = 2 * sz(n, 4) + sz(n, sizeof(Acc)) + sort_bytes(n) + sz(n, 4) + sz(n, 8) * 2 + sz(n, 4) +
                        sz(n, 2) + 3 * sz(n, 1) + 4096;
    int rc = reserve(c, need);
    if (rc) return rc;
    Arena a{static_cast<char *>(c->g_mem), 0, c->g_bytes};
    unsigned *flags = a.take<unsigned>(n), *cid = a.take<unsigned>(n);
    Acc *acc = a.take<Acc>(n);
    const long long *lab = reinterpret_cast<const long long *>(labels);
    k_root_flags<<<grid_for(n), GT, 0, s>>>(h, lab, is_peak, n, cc, flags);
    rc = scan_u32(a, flags, cid, n, s);
    if (rc) return rc;
    k_count_from_scan<<<1, 1, 0, s>>>(flags, cid, n, reinterpret_cast<long long *>(d_n_clusters), cap,
                                      &c->ctl->status, &c->ctl->counters[C_CLUSTERS]);
    if (cc) {
        if (ck(cudaMemsetAsync(acc, 0, sizeof(Acc) * (size_t)n, s))) return TPX_ECUDA;
        k_accum<<<grid_for(n), GT, 0, s>>>(h, lab, is_peak, n, cid, acc);
        k_final<<<grid_for(n), GT, 0, s>>>(h, n, flags, cid, acc, out, cap);
    } else {
        Sorted so;
        so.hit = a.take<unsigned>(n);
        so.shot = a.take<long long>(n);
        so.index = a.take<long long>(n);
        so.tofb = a.take<int>(n);
        so.tot = a.take<unsigned short>(n);
        so.x = a.take<unsigned char>(n);
        so.y = a.take<unsigned char>(n);
        unsigned *vals = nullptr;
        rc = sort_hits(c, a, h, n, -1, &vals);
        if (rc) return rc;
        k_gather<<<grid_for(n), GT, 0, s>>>(h, vals, n, so);
        k_paper<<<grid_for(n), GT, 0, s>>>(so, n, c->cfg.rx, c->cfg.ry, c->cfg.dt_ticks, flags, cid, h, out, cap);
    }
    return ck(cudaGetLastError());
}

__global__ void k_packet_outputs(tpx_hits h, const long long *hl, const unsigned char *hp, long long nh, long long base,
                                 long long *labels, unsigned char *is_peak) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nh; i += (long long)gridDim.x * blockDim.x) {
        const long long q = h.index[i] - base;
        if (labels) labels[q] = hl[i];
        if (is_peak) is_peak[q] = hp[i];
    }
}
__global__ void k_packet_labels32(tpx_hits h, const long long *hl, long long nh, long long base, long long lbase,
                                  int *labels) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nh; i += (long long)gridDim.x * blockDim.x)
        labels[h.index[i] - base] = (int)(hl[i] - lbase);
}
__global__ void k_fill_i32(int *p, long long n, int v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_records64(const tpx_record *src, const long long *n, long long cap, tpx_record64 *dst) {
    const long long m = min(*n, cap);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        dst[i] = *reinterpret_cast<const tpx_record64 *>(src + i);
}
__global__ void k_fill_ll(long long *p, long long n, long long v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_count_peaks(const unsigned char *hp, long long n, unsigned long long *cnt) {
    unsigned long long m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) m += hp[i];
    for (int o = 16; o > 0; o >>= 1) m += __shfl_down_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(cnt, m);
}

int redo_last(tpx_ctx *c) {
    if (!c->last.valid) return TPX_EINVAL;
    const auto L = c->last;
    const long long n = L.n;
    if (n >= (1LL << 31)) return TPX_EUNSUPPORTED;
    cudaStream_t s = c->stream;
    // hits and per-hit outputs live in a separate allocation from the arena
    // used by the stages (each stage reuses the arena from its start)
    const size_t hb = sz(n, 8) * 4 + sz(n, 4) + 3 * sz(n, 2) + sz(n, 1) * 3 + 4096;
    void *hm = nullptr;
    if (cudaMalloc(&hm, hb) != cudaSuccess) { cudaGetLastError(); return TPX_ENOMEM; }
    Arena a{static_cast<char *>(hm), 0, hb};
    tpx_hits h;
    h.index = reinterpret_cast<int64_t *>(a.take<long long>(n));
    h.shot = reinterpret_cast<int64_t *>(a.take<long long>(n));
    h.t = reinterpret_cast<int64_t *>(a.take<long long>(n));
    h.tof = a.take<int32_t>(n);
    h.x = a.take<uint8_t>(n);
    h.y = a.take<uint8_t>(n);
    h.tot = a.take<uint16_t>(n);
    long long *hl = a.take<long long>(n);
    unsigned char *hp = a.take<unsigned char>(n);
    long long *nh_d = a.take<long long>(1);
    int rc = decode_impl(c, L.pk, n, L.base, h, n, reinterpret_cast<int64_t *>(nh_d), L.trig, L.trig_cap, L.n_trig, true,
                         L.E0, L.state_out, nullptr, nullptr);
    long long nh = 0;
    if (!rc) rc = ck(cudaMemcpyAsync(&nh, nh_d, 8, cudaMemcpyDeviceToHost, s));
    if (!rc) rc = ck(cudaStreamSynchronize(s));
    unsigned status = 0;
    if (!rc) rc = ck(cudaMemcpy(&status, &c->ctl->status, 4, cudaMemcpyDeviceToHost));
    if (!rc && !(status & (ST_TRIG_ORDER | ST_TRIG_CAP))) {
        // TPX_FLAG_RECORDS64: the full records go to a scratch array first,
        // then their first 64 bytes to the caller's buffer
        const bool r64 = (c->cfg.flags & TPX_FLAG_RECORDS64) != 0 && L.cl_cap > 0;
        const int64_t cap64 = r64 ? std::min<int64_t>(L.cl_cap, std::max<long long>(nh, 1)) : 0;
        tpx_record *out = L.cl;
        void *tmp = nullptr;
        if (r64) {
            if (cudaMalloc(&tmp, sizeof(tpx_record) * (size_t)cap64) != cudaSuccess) { cudaGetLastError(); rc = TPX_ENOMEM; }
            out = static_cast<tpx_record *>(tmp);
        }
        if (!rc) rc = cluster_all(c, h, nh, reinterpret_cast<int64_t *>(hl), hp, LLONG_MAX, -1, out, r64 ? cap64 : L.cl_cap,
                                  L.n_cl);
        if (!rc && r64) {
            k_records64<<<grid_for(cap64), GT, 0, s>>>(static_cast<const tpx_record *>(tmp), reinterpret_cast<const long long *>(L.n_cl),
                                                     cap64, reinterpret_cast<tpx_record64 *>(L.cl));
            rc = ck(cudaStreamSynchronize(s));
        }
        if (tmp) cudaFree(tmp);
        if (!rc && (L.labels || L.is_peak)) {
            long long *l64 = L.lab32 ? nullptr : reinterpret_cast<long long *>(L.labels);
            int *l32 = L.lab32 ? reinterpret_cast<int *>(L.labels) : nullptr;
            if (l64) k_fill_ll<<<grid_for(n), GT, 0, s>>>(l64, n, -1);
            if (l32) k_fill_i32<<<grid_for(n), GT, 0, s>>>(l32, n, -1);
            if (L.is_peak && cudaMemsetAsync(L.is_peak, 0, (size_t)n, s) != cudaSuccess) rc = TPX_ECUDA;
            k_packet_outputs<<<grid_for(nh), GT, 0, s>>>(h, hl, hp, nh, L.base, l64, L.is_peak);
            if (l32) k_packet_labels32<<<grid_for(nh), GT, 0, s>>>(h, hl, nh, L.base, L.lab32_base, l32);
        }
        if (!rc && nh > 0) {
            unsigned long long z = 0;
            rc = ck(cudaMemcpyAsync(&c->ctl->counters[C_PEAKS], &z, 8, cudaMemcpyHostToDevice, s));
            k_count_peaks<<<grid_for(nh), GT, 0, s>>>(hp, nh, &c->ctl->counters[C_PEAKS]);
        }
    }
    if (!rc) {
        // the counters now describe the redone call
        unsigned long long np = (unsigned long long)n;
        rc = ck(cudaMemcpyAsync(&c->ctl->counters[C_PACKETS], &np, 8, cudaMemcpyHostToDevice, s));
    }
    if (!rc) rc = ck(cudaStreamSynchronize(s));
    cudaFree(hm);
    return rc;
}

// ---- redo of a batch's failed runs ----
__global__ void k_add_ll(long long *v, long long n, long long d) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] += d;
}
// first record of each run of a group: records are in label order and the
// runs' labels are the runs' packet ranges
__global__ void k_rec_bounds(const tpx_record *rec, long long ncl, const long long *run_start, long long nr,
                             long long *bound) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k <= nr; k += (long long)gridDim.x * blockDim.x) {
        if (k == nr) { bound[k] = ncl; continue; }
        long long lo = 0, hi = ncl;
        while (lo < hi) {
            const long long mid = lo + ((hi - lo) >> 1);
            if (rec[mid].label < run_start[k]) lo = mid + 1; else hi = mid;
        }
        bound[k] = lo;
    }
}
// records of group run k count their shots from the run's first trigger
__global__ void k_rec_shots(tpx_record *rec, long long ncl, const long long *bound, const long long *shot_base,
                            long long nr) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncl; i += (long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = nr;   // the run k with bound[k] <= i < bound[k + 1]
        while (hi - lo > 1) {
            const long long mid = (lo + hi) >> 1;
            if (bound[mid] <= i) lo = mid; else hi = mid;
        }
        rec[i].shot -= shot_base[lo];
    }
}
// segmented copy of 8-byte words: segment i moves len[i] words src[i] -> dst[i]
__global__ void k_seg_copy(const unsigned long long *const *src, unsigned long long *const *dst, const long long *len,
                           long long nseg) {
    for (long long i = blockIdx.x; i < nseg; i += gridDim.x) {
        const unsigned long long *a = src[i];
        unsigned long long *b = dst[i];
        for (long long w = threadIdx.x; w < len[i]; w += blockDim.x) b[w] = a[w];
    }
}

namespace {
// a device buffer that keeps its contents when it grows
struct Grow {
    char *p = nullptr;
    size_t used = 0, cap = 0;
    int ensure(size_t want, cudaStream_t s) {
        if (want <= cap) return TPX_OK;
        size_t nc = cap ? cap : (size_t)1 << 24;
        while (nc < want) nc *= 2;
        char *q = nullptr;
        if (cudaMalloc(&q, nc) != cudaSuccess) { cudaGetLastError(); return TPX_ENOMEM; }
        if (used && ck(cudaMemcpyAsync(q, p, used, cudaMemcpyDeviceToDevice, s))) { cudaFree(q); return TPX_ECUDA; }
        if (ck(cudaStreamSynchronize(s))) { cudaFree(q); return TPX_ECUDA; }
        if (p) cudaFree(p);
        p = q;
        cap = nc;
        return TPX_OK;
    }
    ~Grow() { if (p) cudaFree(p); }
};
}  // namespace

int redo_batch(tpx_ctx *c, int64_t *n_redone) {
    auto &B = c->batch;
    cudaStream_t s = c->stream;
    const int64_t R = B.n_runs;
    const int64_t *off = B.h_off;   // the run offsets of the call (host)
    *n_redone = 0;
    std::vector<unsigned> failed((size_t)R);
    std::vector<int64_t> roff((size_t)R + 1), toff((size_t)R + 1);
    Ctl snap;
    if (ck(cudaMemcpyAsync(failed.data(), B.bt.run_failed, 4 * (size_t)R, cudaMemcpyDeviceToHost, s)) ||
        ck(cudaMemcpyAsync(roff.data(), B.bt.run_rec_off, 8 * (size_t)(R + 1), cudaMemcpyDeviceToHost, s)) ||
        ck(cudaMemcpyAsync(toff.data(), B.bt.run_trig_off, 8 * (size_t)(R + 1), cudaMemcpyDeviceToHost, s)) ||
        ck(cudaMemcpyAsync(&snap, c->ctl, sizeof snap, cudaMemcpyDeviceToHost, s)))
        return TPX_ECUDA;
    if (ck(cudaStreamSynchronize(s))) return TPX_ECUDA;
    // the tiles' pass wrote records and triggers only below the capacities
    for (int64_t r = 0; r <= R; ++r) {
        roff[(size_t)r] = std::min<int64_t>(roff[(size_t)r], B.cl_cap);
        toff[(size_t)r] = std::min<int64_t>(toff[(size_t)r], B.trig_cap);
    }
    std::vector<int64_t> F;
    int64_t max_len = 0;
    for (int64_t r = 0; r < R; ++r)
        if (failed[(size_t)r]) {
            F.push_back(r);
            max_len = std::max<int64_t>(max_len, off[r + 1] - off[r]);
        }
    *n_redone = (int64_t)F.size();
    if (F.empty()) return TPX_OK;
    // failed runs are redone in groups of consecutive failed runs holding at
    // most G packets (or one larger run): each run decodes on its own (a
    // stream of its own), its shots offset to keep the group's shots apart,
    // and one clustering pass serves the whole group
    const int64_t G = std::max<int64_t>(max_len, 1LL << 26);
    if (G >= (1LL << 31)) return TPX_EUNSUPPORTED;
    const bool per_packet = B.labels || B.is_peak;
    const size_t hb = sz(G, 8) * 3 + sz(G, 4) + sz(G, 2) + 2 * sz(G, 1) + (per_packet ? sz(G, 8) + sz(G, 1) : 0) +
                      sz(G, 8) + sz(G, sizeof(tpx_record)) + 3 * sz((int64_t)F.size() + 1, 8) + sz(4, 8) + 4096;
    void *hm = nullptr;
    if (cudaMalloc(&hm, hb) != cudaSuccess) { cudaGetLastError(); return TPX_ENOMEM; }
    Arena a{static_cast<char *>(hm), 0, hb};
    tpx_hits h;
    h.index = reinterpret_cast<int64_t *>(a.take<long long>(G));
    h.shot = reinterpret_cast<int64_t *>(a.take<long long>(G));
    h.t = reinterpret_cast<int64_t *>(a.take<long long>(G));
    h.tof = a.take<int32_t>(G);
    h.tot = a.take<uint16_t>(G);
    h.x = a.take<uint8_t>(G);
    h.y = a.take<uint8_t>(G);
    long long *hl = per_packet ? a.take<long long>(G) : nullptr;
    unsigned char *hp = per_packet ? a.take<unsigned char>(G) : nullptr;
    long long *tr = a.take<long long>(G);
    tpx_record *grec = a.take<tpx_record>(G);
    long long *d_start = a.take<long long>((int64_t)F.size() + 1), *d_base = a.take<long long>((int64_t)F.size() + 1);
    long long *d_bound = a.take<long long>((int64_t)F.size() + 1);
    long long *cnt = a.take<long long>(4);
    Grow acc_rec, acc_trig;   // the redone runs' records and triggers, run after run
    std::vector<int64_t> nrec((size_t)R), ntrg((size_t)R), rstart((size_t)R), tstart((size_t)R);
    int rc = TPX_OK;
    for (size_t i = 0; i < F.size() && !rc;) {
        size_t j = i;
        int64_t pk_sum = 0;
        while (j < F.size() && (j == i || pk_sum + (off[F[j] + 1] - off[F[j]]) <= G)) {
            pk_sum += off[F[j] + 1] - off[F[j]];
            ++j;
        }
        const int64_t nr = (int64_t)(j - i);
        std::vector<long long> start((size_t)nr), base((size_t)nr);
        int64_t hoff = 0, tcount = 0;
        for (int64_t k = 0; k < nr && !rc; ++k) {
            const int64_t r = F[i + (size_t)k], len = off[r + 1] - off[r];
            tpx_hits hk = h;
            hk.index += hoff; hk.shot += hoff; hk.t += hoff; hk.tof += hoff; hk.tot += hoff; hk.x += hoff; hk.y += hoff;
            rc = decode_impl(c, B.pk + off[r], len, off[r], hk, len, reinterpret_cast<int64_t *>(cnt),
                             reinterpret_cast<int64_t *>(tr + tcount), len, reinterpret_cast<int64_t *>(cnt + 1), false,
                             nullptr, nullptr, nullptr, nullptr);
            long long hc[2] = {0, 0};
            if (!rc) rc = ck(cudaMemcpyAsync(hc, cnt, 16, cudaMemcpyDeviceToHost, s));
            if (!rc) rc = ck(cudaStreamSynchronize(s));
            if (rc) break;
            if (hc[0] > 0 && tcount > 0) k_add_ll<<<grid_for(hc[0]), GT, 0, s>>>(reinterpret_cast<long long *>(hk.shot), hc[0], tcount);
            start[(size_t)k] = off[r];
            base[(size_t)k] = tcount;
            ntrg[(size_t)r] = hc[1];
            hoff += hc[0];
            tcount += hc[1];
        }
        if (rc) break;
        // one clustering pass for the group; records in label order = run order
        rc = cluster_all(c, h, hoff, reinterpret_cast<int64_t *>(hl), hp, LLONG_MAX, tcount, grec, hoff,
                         reinterpret_cast<int64_t *>(cnt + 2));
        if (!rc && per_packet && hoff > 0) {
            for (int64_t k = 0; k < nr; ++k) {
                const int64_t r = F[i + (size_t)k], len = off[r + 1] - off[r];
                if (B.labels) k_fill_ll<<<grid_for(len), GT, 0, s>>>(reinterpret_cast<long long *>(B.labels) + off[r], len, -1);
                if (B.is_peak && ck(cudaMemsetAsync(B.is_peak + off[r], 0, (size_t)len, s))) rc = TPX_ECUDA;
            }
            k_packet_outputs<<<grid_for(hoff), GT, 0, s>>>(h, hl, hp, hoff, 0, reinterpret_cast<long long *>(B.labels),
                                                           B.is_peak);
        }
        long long ncl = 0;
        if (!rc) rc = ck(cudaMemcpyAsync(&ncl, cnt + 2, 8, cudaMemcpyDeviceToHost, s));
        if (!rc) rc = ck(cudaMemcpyAsync(d_start, start.data(), 8 * (size_t)nr, cudaMemcpyHostToDevice, s));
        if (!rc) rc = ck(cudaMemcpyAsync(d_base, base.data(), 8 * (size_t)nr, cudaMemcpyHostToDevice, s));
        if (!rc) rc = ck(cudaStreamSynchronize(s));
        if (rc) break;
        if (hoff == 0) ncl = 0;
        std::vector<long long> bound((size_t)nr + 1, 0);
        if (ncl > 0) {
            k_rec_bounds<<<grid_for(nr + 1), GT, 0, s>>>(grec, ncl, d_start, nr, d_bound);
            k_rec_shots<<<grid_for(ncl), GT, 0, s>>>(grec, ncl, d_bound, d_base, nr);
            rc = ck(cudaMemcpyAsync(bound.data(), d_bound, 8 * (size_t)(nr + 1), cudaMemcpyDeviceToHost, s));
        }
        // append the group's records and triggers
        if (!rc) rc = acc_rec.ensure(acc_rec.used + sizeof(tpx_record) * (size_t)ncl, s);
        if (!rc) rc = acc_trig.ensure(acc_trig.used + 8 * (size_t)tcount, s);
        if (!rc && ncl > 0)
            rc = ck(cudaMemcpyAsync(acc_rec.p + acc_rec.used, grec, sizeof(tpx_record) * (size_t)ncl,
                                    cudaMemcpyDeviceToDevice, s));
        if (!rc && tcount > 0)
            rc = ck(cudaMemcpyAsync(acc_trig.p + acc_trig.used, tr, 8 * (size_t)tcount, cudaMemcpyDeviceToDevice, s));
        if (!rc) rc = ck(cudaStreamSynchronize(s));
        if (rc) break;
        for (int64_t k = 0; k < nr; ++k) {
            const int64_t r = F[i + (size_t)k];
            nrec[(size_t)r] = bound[(size_t)k + 1] - bound[(size_t)k];
            rstart[(size_t)r] = (int64_t)(acc_rec.used / sizeof(tpx_record)) + bound[(size_t)k];
            tstart[(size_t)r] = (int64_t)(acc_trig.used / 8) + base[(size_t)k];
        }
        acc_rec.used += sizeof(tpx_record) * (size_t)ncl;
        acc_trig.used += 8 * (size_t)tcount;
        i = j;
    }
    // the runs' final offsets; every run from the first redone one on moves
    // (the tiles' outputs of the others are kept aside first)
    const int64_t first = F.front();
    std::vector<long long> NO((size_t)R + 1), NTo((size_t)R + 1);
    NO[0] = 0;
    NTo[0] = 0;
    for (int64_t r = 0; r < R; ++r) {
        NO[(size_t)r + 1] = NO[(size_t)r] + (failed[(size_t)r] ? nrec[(size_t)r] : roff[(size_t)r + 1] - roff[(size_t)r]);
        NTo[(size_t)r + 1] = NTo[(size_t)r] + (failed[(size_t)r] ? ntrg[(size_t)r] : toff[(size_t)r + 1] - toff[(size_t)r]);
    }
    const int64_t old_rec = roff[(size_t)R] - roff[(size_t)first], old_trig = toff[(size_t)R] - toff[(size_t)first];
    Grow keep;
    if (!rc) rc = keep.ensure(sizeof(tpx_record) * (size_t)old_rec + 8 * (size_t)old_trig + 512, s);
    tpx_record *old_rec_copy = reinterpret_cast<tpx_record *>(keep.p);
    long long *old_trig_copy = reinterpret_cast<long long *>(keep.p + ((sizeof(tpx_record) * (size_t)old_rec + 255) & ~size_t(255)));
    if (!rc && old_rec > 0)
        rc = ck(cudaMemcpyAsync(old_rec_copy, B.cl + roff[(size_t)first], sizeof(tpx_record) * (size_t)old_rec,
                                cudaMemcpyDeviceToDevice, s));
    if (!rc && old_trig > 0)
        rc = ck(cudaMemcpyAsync(old_trig_copy, B.trig + toff[(size_t)first], 8 * (size_t)old_trig, cudaMemcpyDeviceToDevice, s));
    // one segmented copy for all moved runs (records, then triggers)
    std::vector<const unsigned long long *> src;
    std::vector<unsigned long long *> dst;
    std::vector<long long> len;
    constexpr int WPR = (int)(sizeof(tpx_record) / 8);
    for (int64_t r = first; r < R && !rc; ++r) {
        const int64_t nr = NO[(size_t)r + 1] - NO[(size_t)r], nt = NTo[(size_t)r + 1] - NTo[(size_t)r];
        const int64_t kr = std::max<int64_t>(0, std::min<int64_t>(nr, B.cl_cap - NO[(size_t)r]));
        const int64_t kt = std::max<int64_t>(0, std::min<int64_t>(nt, B.trig_cap - NTo[(size_t)r]));
        const tpx_record *sr = failed[(size_t)r] ? reinterpret_cast<const tpx_record *>(acc_rec.p) + rstart[(size_t)r]
                                                 : old_rec_copy + (roff[(size_t)r] - roff[(size_t)first]);
        const long long *st = failed[(size_t)r] ? reinterpret_cast<const long long *>(acc_trig.p) + tstart[(size_t)r]
                                                : old_trig_copy + (toff[(size_t)r] - toff[(size_t)first]);
        if (kr > 0) {
            src.push_back(reinterpret_cast<const unsigned long long *>(sr));
            dst.push_back(reinterpret_cast<unsigned long long *>(B.cl + NO[(size_t)r]));
            len.push_back(kr * WPR);
        }
        if (kt > 0) {
            src.push_back(reinterpret_cast<const unsigned long long *>(st));
            dst.push_back(reinterpret_cast<unsigned long long *>(B.trig + NTo[(size_t)r]));
            len.push_back(kt);
        }
    }
    if (!rc && !len.empty()) {
        {   // pieces of at most 2^16 words, so that large runs spread over blocks
            std::vector<const unsigned long long *> s2;
            std::vector<unsigned long long *> d2;
            std::vector<long long> l2;
            for (size_t k = 0; k < len.size(); ++k)
                for (long long o = 0; o < len[k]; o += 1 << 16) {
                    s2.push_back(src[k] + o);
                    d2.push_back(dst[k] + o);
                    l2.push_back(std::min<long long>(1 << 16, len[k] - o));
                }
            src.swap(s2);
            dst.swap(d2);
            len.swap(l2);
        }
        const size_t ns = len.size();
        Grow desc;
        rc = desc.ensure(3 * 8 * ns + 512, s);
        void **d_src = reinterpret_cast<void **>(desc.p);
        void **d_dst = d_src + ns;
        long long *d_len = reinterpret_cast<long long *>(d_dst + ns);
        if (!rc) rc = ck(cudaMemcpyAsync(d_src, src.data(), 8 * ns, cudaMemcpyHostToDevice, s));
        if (!rc) rc = ck(cudaMemcpyAsync(d_dst, dst.data(), 8 * ns, cudaMemcpyHostToDevice, s));
        if (!rc) rc = ck(cudaMemcpyAsync(d_len, len.data(), 8 * ns, cudaMemcpyHostToDevice, s));
        if (!rc)
            k_seg_copy<<<(unsigned)std::min<size_t>(ns, 152 * 8), 256, 0, s>>>(
                reinterpret_cast<const unsigned long long *const *>(d_src), reinterpret_cast<unsigned long long *const *>(d_dst),
                d_len, (long long)ns);
        if (!rc) rc = ck(cudaStreamSynchronize(s));   // the descriptors are freed on return
    }
    if (!rc) {
        // offsets, totals; the counters keep describing the tiles' pass
        snap.counters[C_CLUSTERS] = (unsigned long long)NO[(size_t)R];
        if (NO[(size_t)R] > B.cl_cap) snap.status |= ST_CLUSTER_CAP;
        if (NTo[(size_t)R] > B.trig_cap) snap.status |= ST_TRIG_CAP;
        Ctl cur;
        rc = ck(cudaMemcpyAsync(&cur, c->ctl, sizeof cur, cudaMemcpyDeviceToHost, s));
        if (!rc) rc = ck(cudaStreamSynchronize(s));
        snap.status |= cur.status & ST_TRIG_ORDER;   // a redone run may have decreasing triggers
        snap.status &= ~ST_RUN_REDO;                 // done: a later sync has nothing to redo
        if (!rc) rc = ck(cudaMemcpyAsync(B.bt.run_rec_off, NO.data(), 8 * (size_t)(R + 1), cudaMemcpyHostToDevice, s));
        if (!rc) rc = ck(cudaMemcpyAsync(B.bt.run_trig_off, NTo.data(), 8 * (size_t)(R + 1), cudaMemcpyHostToDevice, s));
        if (!rc) rc = ck(cudaMemcpyAsync(B.n_cl, &NO[(size_t)R], 8, cudaMemcpyHostToDevice, s));
        if (!rc) rc = ck(cudaMemcpyAsync(B.n_trig, &NTo[(size_t)R], 8, cudaMemcpyHostToDevice, s));
        if (!rc) rc = ck(cudaMemcpyAsync(c->ctl, &snap, sizeof snap, cudaMemcpyHostToDevice, s));
        if (!rc) rc = ck(cudaStreamSynchronize(s));
    }
    cudaStreamSynchronize(s);
    cudaFree(hm);
    return rc;
}

}  // namespace tpxg

// ------------------------------------------------------------ C ABI
extern "C" int tpx_decode(tpx_ctx *c, const uint64_t *pk, int64_t n, int64_t base, const tpx_hits *hits,
                          int64_t cap, int64_t *d_n_hits, int64_t *trig, int64_t trig_cap, int64_t *d_n_trig) {
    if (!c || !hits || n < 0 || cap < 0 || trig_cap < 0 || !d_n_hits || !d_n_trig) return TPX_EINVAL;
    if (n > 0 && !pk) return TPX_EINVAL;
    if (n >= (1LL << 31)) return TPX_EINVAL;
    if (cap > 0 && (!hits->index || !hits->shot || !hits->t || !hits->tof || !hits->x || !hits->y || !hits->tot))
        return TPX_EINVAL;
    if (trig_cap > 0 && !trig) return TPX_EINVAL;
    c->last.valid = false;
    const tpxk::GAgg *E0 = nullptr;
    tpxk::GAgg *out = nullptr;
    take_state(c, &E0, &out);
    return tpxg::decode_impl(c, pk, n, base, *hits, cap, d_n_hits, trig, trig_cap, d_n_trig, true, E0, out, nullptr,
                             nullptr);
}

extern "C" int tpx_cluster(tpx_ctx *c, const tpx_hits *hits, int64_t n, int64_t *d_labels, uint8_t *d_is_peak) {
    if (!c || !hits || n < 0 || n >= (1LL << 31) || (n > 0 && !d_labels)) return TPX_EINVAL;
    c->last.valid = false;
    return tpxg::cluster_impl(c, *hits, n, d_labels, d_is_peak);
}

extern "C" int tpx_centroid(tpx_ctx *c, const tpx_hits *hits, const int64_t *d_labels, const uint8_t *d_is_peak,
                            int64_t n, tpx_record *d_clusters, int64_t cap, int64_t *d_n_clusters) {
    if (!c || !hits || n < 0 || n >= (1LL << 31) || cap < 0 || !d_n_clusters) return TPX_EINVAL;
    if ((n > 0 && !d_labels) || (cap > 0 && !d_clusters)) return TPX_EINVAL;
    c->last.valid = false;
    return tpxg::centroid_impl(c, *hits, d_labels, d_is_peak, n, d_clusters, cap, d_n_clusters);
}

namespace tpxg {
// one count per hit inside the ToF window (Sec. IV.C calibration histogram)
__global__ void k_tot_tof_hist(const int32_t *tof, const uint16_t *tot, long long n, int lo, int bin, int nb,
                               unsigned *hist) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long d = (long long)tof[i] - lo;
        if (d < 0) continue;
        const long long b = d / bin;
        if (b >= nb) continue;
        atomicAdd(&hist[(long long)tot[i] * nb + b], 1u);
    }
}
}  // namespace tpxg

extern "C" int tpx_tot_tof_histogram(tpx_ctx *c, const tpx_hits *hits, int64_t n, int32_t lo, int32_t bin, int32_t nb,
                                     uint32_t *d_hist) {
    if (!c || !hits || n < 0 || bin < 1 || nb < 1 || !d_hist) return TPX_EINVAL;
    if (n > 0 && (!hits->tof || !hits->tot)) return TPX_EINVAL;
    if (n == 0) return TPX_OK;
    tpxg::k_tot_tof_hist<<<tpxg::grid_for(n), tpxg::GT, 0, c->stream>>>(hits->tof, hits->tot, n, lo, bin, nb, d_hist);
    return tpxg::ck(cudaGetLastError());
}

extern "C" int tpx_summarize(tpx_ctx *c, const uint64_t *pk, int64_t n, tpx_chain_summary *out) {
    if (!c || !out || n < 0 || (n > 0 && !pk)) return TPX_EINVAL;
    using namespace tpxg;
    cudaStream_t s = c->stream;
    const long long tiles = (n + GTILE - 1) / GTILE;
    const size_t need = sz(tiles, sizeof(tpxk::GAgg)) * 2 + sz(tiles + 1, 8) * 2 + sz(1, sizeof(tpxk::GAgg)) + 4096;
    int rc = reserve(c, need);
    if (rc) return rc;
    Arena a{static_cast<char *>(c->g_mem), 0, c->g_bytes};
    tpxk::GAgg *tagg = a.take<tpxk::GAgg>(tiles), *tpre = a.take<tpxk::GAgg>(tiles);
    long long *tcnt = a.take<long long>(tiles + 1), *toff = a.take<long long>(tiles + 1);
    tpxk::GAgg *res = a.take<tpxk::GAgg>(1);
    long long *ntr = toff + tiles;
    tpxk::GAgg h;
    std::memset(&h, 0, sizeof h);
    if (n > 0) {
        const long long tp = c->cfg.wrap_thr_pix_ticks, tt = c->cfg.wrap_thr_tdc_ticks;
        k_tile_agg<<<(unsigned)tiles, GT, 0, s>>>(pk, n, tp, tt, tagg, tcnt);
        k_tile_prefix<<<1, PT, 0, s>>>(tagg, tpre, tcnt, toff, tiles, tp, tt, ntr, nullptr, res);
        if (ck(cudaMemcpyAsync(&h, res, sizeof h, cudaMemcpyDeviceToHost, s))) return TPX_ECUDA;
    }
    if (ck(cudaStreamSynchronize(s))) return TPX_ECUDA;
    out->pixels = h.pix.n;
    out->pix_first_raw = h.pix.first;
    out->pix_last_raw = h.pix.last;
    out->pix_wraps = h.pix.sum;
    out->triggers = h.tdc.n;
    out->tdc_first_raw = h.tdc.first;
    out->tdc_last_raw = h.tdc.last;
    out->tdc_wraps = h.tdc.sum;
    return TPX_OK;
}
