// tpx_general.cu -- the general (global-memory) path: tpx_decode,
// tpx_cluster, tpx_centroid, and the exact redo of a tpx_process call whose
// input the fused kernel cannot hold on chip.
//
// decode  : tile aggregates of the two unwrap chains (Sec. IV.A) -> serial
//           prefix over tiles -> per-packet unwrapped times and the trigger
//           list -> each pixel binned to the most recent trigger in time by
//           binary search, cut at tof_max (Sec. IV.B), timewalk table
//           subtracted (Sec. IV.C) -> kept pixels compacted in stream order.
// cluster : stable LSD radix sort of the hits on (shot, corrected ToF) --
//           ties keep stream order -- then, for every hit, a forward scan of
//           the hits within dt in that order; adjacent pairs (Sec. V.A box
//           rule) set the local-maximum flags (Sec. V.B) and are joined by a
//           lock-free union-find whose root is the smallest sorted position,
//           i.e. the earliest hit of the cluster.
// centroid: cluster ids in ascending label order, exact int64 moments by
//           global atomics, f64 final division (Sec. V.C); PAPER mode sums the
//           box neighbourhood of each local maximum.
// Nothing here is on the benchmark path; it trades speed for having no
// capacity limit besides 2^31 - 1 kept pixels per call.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cstring>

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

// exclusive prefix over tiles (one thread: this path is not on the benchmark)
__global__ void k_tile_prefix(const GAgg *tagg, GAgg *tpre, const long long *tcnt, long long *toff, long long tiles,
                              long long tp, long long tt, long long *n_trig_out, const GAgg *E0, GAgg *state_out) {
    GAgg acc = E0 ? *E0 : agg_id();
    long long off = 0;
    for (long long t = 0; t < tiles; ++t) {
        tpre[t] = acc;
        toff[t] = off;
        acc = acomb(acc, tagg[t], tp, tt);
        off += tcnt[t];
    }
    toff[tiles] = off;
    *n_trig_out = off;
    if (state_out) *state_out = acc;
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

__global__ void k_check_trig(const long long *trig, long long ntr, unsigned *status) {
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

__global__ void __launch_bounds__(GT) k_bin(const uint64_t *pk, long long n, const long long *t_all, const long long *trig,
                                            long long ntr, long long tof_max, long long *tile_kept,
                                            unsigned long long *counters) {
    __shared__ long long s_w[GW];
    __shared__ long long s_tot;
    const long long tile = blockIdx.x, q0 = tile * GTILE + threadIdx.x * GK;
    long long keep = 0, bg = 0, pre = 0, pix = 0, tdc = 0, bad = 0;
    for (int j = 0; j < GK; ++j) {
        const long long q = q0 + j;
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

__global__ void k_serial_prefix(const long long *cnt, long long *off, long long tiles, long long *total_out) {
    long long acc = 0;
    for (long long t = 0; t < tiles; ++t) {
        off[t] = acc;
        acc += cnt[t];
    }
    off[tiles] = acc;
    if (total_out) *total_out = acc;
}

__global__ void __launch_bounds__(GT) k_compact(const uint64_t *pk, long long n, long long idx_base, const long long *t_all,
                                                const long long *trig, long long ntr, long long tof_max,
                                                const int16_t *lut, const long long *tile_off, tpx_hits hits,
                                                long long cap, unsigned *status, const GAgg *E0) {
    const long long trig_base = E0 ? E0->tdc.n : 0;
    __shared__ long long s_w[GW];
    __shared__ long long s_tot;
    const long long tile = blockIdx.x, q0 = tile * GTILE + threadIdx.x * GK;
    long long mine = 0;
    for (int j = 0; j < GK; ++j) {
        const long long q = q0 + j;
        if (q >= n) break;
        long long s, f;
        mine += bin_pixel(pk[q], t_all[q], trig, ntr, tof_max, &s, &f) == 0;
    }
    long long o = tile_off[tile] + block_scan_ll(mine, s_w, &s_tot);
    for (int j = 0; j < GK; ++j) {
        const long long q = q0 + j;
        if (q >= n) break;
        const uint64_t w = pk[q];
        long long s, f;
        if (bin_pixel(w, t_all[q], trig, ntr, tof_max, &s, &f) != 0) continue;
        if (o < cap) {
            const int tot = pix_tot(w);
            const long long corr = lut ? (long long)lut[tot] : 0LL;
            hits.index[o] = idx_base + q;
            hits.shot[o] = s + trig_base;
            hits.t[o] = t_all[q] - corr;
            hits.tof[o] = (int32_t)(f - corr);
            hits.x[o] = (uint8_t)pix_x(w);
            hits.y[o] = (uint8_t)pix_y(w);
            hits.tot[o] = (uint16_t)tot;
        } else {
            atomicOr(status, ST_CLUSTER_CAP);
        }
        ++o;
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
__global__ void k_scan_bsum(unsigned *bsum, long long nb) {
    unsigned acc = 0;
    for (long long b = 0; b < nb; ++b) { const unsigned v = bsum[b]; bsum[b] = acc; acc += v; }
}
__global__ void k_scan_add(unsigned *out, long long n, const unsigned *bsum) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] += bsum[i / GTILE];
}

// ------------------------------------------------------------ cluster kernels
__global__ void k_make_keys(tpx_hits h, long long n, unsigned long long *keys, unsigned *vals) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        keys[i] = ((unsigned long long)h.shot[i] << 24) | (unsigned long long)(h.tof[i] + kBias);
        vals[i] = (unsigned)i;
    }
}
__global__ void k_max_shot(tpx_hits h, long long n, unsigned long long *mx) {
    unsigned long long m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)h.shot[i]);
    atomicMax(mx, m);
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

// every hit scans forward in sorted order while the shot is the same and the
// time gap is within dt: each adjacent pair is met once (from its earlier end)
__global__ void k_window(Sorted s, long long n, int rx, int ry, int dt, int cc, int *parent, unsigned char *notpeak) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long sh = s.shot[i];
        const int tb = s.tofb[i], xi = s.x[i], yi = s.y[i], ti = s.tot[i];
        const long long ii = s.index[i];
        for (long long j = i + 1; j < n; ++j) {
            if (s.shot[j] != sh || s.tofb[j] - tb > dt) break;
            const int dx = (int)s.x[j] - xi, dy = (int)s.y[j] - yi;
            if (dx < -rx || dx > rx || dy < -ry || dy > ry) continue;
            const int tj = s.tot[j];
            // local maxima: equal ToT goes to the later pixel in the stream (Sec. V.B)
            if (tj > ti || (tj == ti && s.index[j] > ii)) notpeak[i] = 1; else notpeak[j] = 1;
            if (cc) g_unite(parent, (int)i, (int)j);
        }
    }
}

__global__ void k_labels(Sorted s, long long n, int cc, int *parent, const unsigned char *notpeak, long long *labels,
                         unsigned char *is_peak) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned h = s.hit[i];
        labels[h] = cc ? s.index[g_find(parent, (int)i)] : s.index[i];
        if (is_peak) is_peak[h] = notpeak[i] ? 0 : 1;
    }
}

__global__ void k_iota(int *p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = (int)i;
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
        o.x = (double)o.s_x / (double)o.s_tot;
        o.y = (double)o.s_y / (double)o.s_tot;
        o.tof = (double)h.tof[i] + (double)o.s_t / (double)o.s_tot;
        out[c] = o;
    }
}

// PAPER mode: each local maximum sums its box neighbourhood (both directions
// in sorted order, within dt)
__global__ void k_paper(Sorted s, long long n, int rx, int ry, int dt, const unsigned char *is_peak_hit,
                        const unsigned *cid_hit, tpx_hits h, tpx_record *out, long long cap) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned hi = s.hit[i];
        if (!is_peak_hit[hi]) continue;
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
        o.x = (double)sx / (double)st;
        o.y = (double)sy / (double)st;
        o.tof = (double)tofc0 + (double)o.s_t / (double)st;
        out[c] = o;
    }
}

__global__ void k_count_from_scan(const unsigned *flags, const unsigned *cid, long long n, long long *out) {
    *out = n ? (long long)cid[n - 1] + flags[n - 1] : 0;
}

// ------------------------------------------------------------ host helpers
inline int ck(cudaError_t e) { return e == cudaSuccess ? TPX_OK : TPX_ECUDA; }
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
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return TPX_ECUDA;
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
    k_scan_bsum<<<1, 1, 0, s>>>(bsum, nb);
    k_scan_add<<<grid_for(n), GT, 0, s>>>(out, n, bsum);
    return ck(cudaGetLastError());
}

size_t sort_bytes(long long n) {
    const long long tiles = (n + GTILE - 1) / GTILE;
    return 2 * sz(n, 8) + 2 * sz(n, 4) + 2 * sz(256 * tiles, 4) + sz((256 * tiles + GTILE - 1) / GTILE + 1, 4) + 4096;
}

// sort the hits by (shot, corrected ToF); returns the sorted values buffer
int sort_hits(tpx_ctx *c, Arena &a, const tpx_hits &h, long long n, unsigned **vals_out) {
    cudaStream_t s = c->stream;
    const long long tiles = (n + GTILE - 1) / GTILE;
    unsigned long long *k0 = a.take<unsigned long long>(n), *k1 = a.take<unsigned long long>(n);
    unsigned *v0 = a.take<unsigned>(n), *v1 = a.take<unsigned>(n);
    unsigned *hist = a.take<unsigned>(256 * tiles), *offs = a.take<unsigned>(256 * tiles);
    unsigned long long *mx = a.take<unsigned long long>(1);
    if (cudaMemsetAsync(mx, 0, 8, s) != cudaSuccess) return TPX_ECUDA;
    k_make_keys<<<grid_for(n), GT, 0, s>>>(h, n, k0, v0);
    k_max_shot<<<grid_for(n), GT, 0, s>>>(h, n, mx);
    unsigned long long hmx = 0;
    if (cudaMemcpyAsync(&hmx, mx, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return TPX_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TPX_ECUDA;
    int bits = 24;
    while (bits < 64 && (hmx >> (bits - 24)) != 0) ++bits;
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

int decode_impl(tpx_ctx *c, const uint64_t *pk, int64_t n, int64_t base, const tpx_hits &h, int64_t cap,
                int64_t *d_n_hits, int64_t *trig, int64_t trig_cap, int64_t *d_n_trig, bool clear_ctl,
                const GAgg *E0, GAgg *state_out, long long *trig_pos, long long **t_all_out) {
    cudaStream_t s = c->stream;
    const long long tiles = (n + GTILE - 1) / GTILE;
    const size_t need = sz(tiles, sizeof(GAgg)) * 2 + sz(tiles + 1, 8) * 4 + sz(n, 8) + 4096;
    int rc = reserve(c, need);
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
    k_tile_agg<<<(unsigned)tiles, GT, 0, s>>>(pk, n, tp, tt, tagg, tcnt);
    k_tile_prefix<<<1, 1, 0, s>>>(tagg, tpre, tcnt, toff, tiles, tp, tt, reinterpret_cast<long long *>(d_n_trig),
                                  E0, state_out);
    k_unwrap<<<(unsigned)tiles, GT, 0, s>>>(pk, n, tpre, toff, tp, tt, t_all, reinterpret_cast<long long *>(trig),
                                            trig_cap, &c->ctl->status, trig_pos);
    long long ntr_h = 0;
    if (cudaMemcpyAsync(&ntr_h, d_n_trig, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return TPX_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TPX_ECUDA;
    if (ntr_h > trig_cap) return TPX_OK;   // status already latched; nothing to bin against
    k_check_trig<<<grid_for(ntr_h), GT, 0, s>>>(reinterpret_cast<long long *>(trig), ntr_h, &c->ctl->status);
    k_bin<<<(unsigned)tiles, GT, 0, s>>>(pk, n, t_all, reinterpret_cast<long long *>(trig), ntr_h,
                                         c->cfg.tof_max_ticks, tkept, c->ctl->counters);
    k_serial_prefix<<<1, 1, 0, s>>>(tkept, tkoff, tiles, reinterpret_cast<long long *>(d_n_hits));
    k_compact<<<(unsigned)tiles, GT, 0, s>>>(pk, n, base, t_all, reinterpret_cast<long long *>(trig), ntr_h,
                                             c->cfg.tof_max_ticks, c->cfg.d_timewalk_lut, tkoff, h, cap,
                                             &c->ctl->status, E0);
    const unsigned long long np = (unsigned long long)n;
    if (cudaMemcpyAsync(&c->ctl->counters[C_PACKETS], &np, 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TPX_ECUDA;
    return ck(cudaGetLastError());
}

int cluster_impl(tpx_ctx *c, const tpx_hits &h, int64_t n, int64_t *labels, uint8_t *is_peak) {
    cudaStream_t s = c->stream;
    if (n <= 0) return TPX_OK;
    const size_t need = sort_bytes(n) + sz(n, 4) + sz(n, 8) * 2 + sz(n, 4) + sz(n, 2) + 3 * sz(n, 1) + sz(n, 4) + 4096;
    int rc = reserve(c, need);
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
    unsigned char *notpeak = a.take<unsigned char>(n);
    int *parent = a.take<int>(n);
    unsigned *vals = nullptr;
    rc = sort_hits(c, a, h, n, &vals);
    if (rc) return rc;
    k_gather<<<grid_for(n), GT, 0, s>>>(h, vals, n, so);
    if (cudaMemsetAsync(notpeak, 0, (size_t)n, s) != cudaSuccess) return TPX_ECUDA;
    const int cc = c->cfg.mode == TPX_MODE_CC;
    k_iota<<<grid_for(n), GT, 0, s>>>(parent, n);
    k_window<<<grid_for(n), GT, 0, s>>>(so, n, c->cfg.rx, c->cfg.ry, c->cfg.dt_ticks, cc, parent, notpeak);
    k_labels<<<grid_for(n), GT, 0, s>>>(so, n, cc, parent, notpeak, reinterpret_cast<long long *>(labels), is_peak);
    return ck(cudaGetLastError());
}

int centroid_impl(tpx_ctx *c, const tpx_hits &h, const int64_t *labels, const uint8_t *is_peak, int64_t n,
                  tpx_record *out, int64_t cap, int64_t *d_n_clusters) {
    cudaStream_t s = c->stream;
    if (cudaMemsetAsync(d_n_clusters, 0, 8, s) != cudaSuccess) return TPX_ECUDA;
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
    k_count_from_scan<<<1, 1, 0, s>>>(flags, cid, n, reinterpret_cast<long long *>(d_n_clusters));
    long long ncl = 0;
    if (cudaMemcpyAsync(&ncl, d_n_clusters, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return TPX_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TPX_ECUDA;
    if (ncl > cap) {
        unsigned st = ST_CLUSTER_CAP, cur = 0;
        if (cudaMemcpy(&cur, &c->ctl->status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return TPX_ECUDA;
        cur |= st;
        if (cudaMemcpy(&c->ctl->status, &cur, 4, cudaMemcpyHostToDevice) != cudaSuccess) return TPX_ECUDA;
    }
    if (cc) {
        if (cudaMemsetAsync(acc, 0, sizeof(Acc) * (size_t)ncl, s) != cudaSuccess) return TPX_ECUDA;
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
        rc = sort_hits(c, a, h, n, &vals);
        if (rc) return rc;
        k_gather<<<grid_for(n), GT, 0, s>>>(h, vals, n, so);
        k_paper<<<grid_for(n), GT, 0, s>>>(so, n, c->cfg.rx, c->cfg.ry, c->cfg.dt_ticks, is_peak, cid, h, out, cap);
    }
    // counters of the clustering stage
    unsigned long long cl = (unsigned long long)ncl;
    if (cudaMemcpyAsync(&c->ctl->counters[C_CLUSTERS], &cl, 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TPX_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TPX_ECUDA;
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
        rc = cluster_impl(c, h, nh, reinterpret_cast<int64_t *>(hl), hp);
        if (!rc) rc = centroid_impl(c, h, reinterpret_cast<int64_t *>(hl), hp, nh, L.cl, L.cl_cap, L.n_cl);
        if (!rc && (L.labels || L.is_peak)) {
            if (L.labels) k_fill_ll<<<grid_for(n), GT, 0, s>>>(reinterpret_cast<long long *>(L.labels), n, -1);
            if (L.is_peak && cudaMemsetAsync(L.is_peak, 0, (size_t)n, s) != cudaSuccess) rc = TPX_ECUDA;
            k_packet_outputs<<<grid_for(nh), GT, 0, s>>>(h, hl, hp, nh, L.base, reinterpret_cast<long long *>(L.labels),
                                                        L.is_peak);
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
        k_tile_prefix<<<1, 1, 0, s>>>(tagg, tpre, tcnt, toff, tiles, tp, tt, ntr, nullptr, res);
        if (cudaMemcpyAsync(&h, res, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess) return TPX_ECUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return TPX_ECUDA;
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
