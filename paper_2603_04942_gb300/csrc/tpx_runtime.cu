// tpx_runtime.cu -- host side of the C ABI declared in include/tpx.h:
// context and scratch management, argument checks, launches, status words.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "tpx.h"
#include "tpx_ctx.h"
#include "tpx_fused.cuh"


void take_state(tpx_ctx *c, const tpxk::GAgg **E0, tpxk::GAgg **out) {
    *E0 = (c->cfg.chain || c->state_once) ? &c->d_state[c->cur] : nullptr;
    *out = &c->d_state[c->cur ^ 1];
    c->cur ^= 1;
    c->state_once = false;
}


// a failed CUDA call: true; with TPX_DEBUG set in the environment its error
// is printed to stderr
static inline bool ckr(cudaError_t e, int line = __builtin_LINE()) {
    if (e == cudaSuccess) return false;
    if (std::getenv("TPX_DEBUG")) std::fprintf(stderr, "tpx_runtime.cu:%d: %s\n", line, cudaGetErrorString(e));
    return true;
}

namespace {

constexpr int64_t kMaxTofMax = (1LL << 24) - 65537;

int check_cfg(const tpx_config *c) {
    if (!c) return TPX_EINVAL;
    if (c->rx < 0 || c->ry < 0 || c->rx > 7 || c->ry > 7) return TPX_EINVAL;
    if (c->dt_ticks < 0) return TPX_EINVAL;
    if (c->mode != TPX_MODE_CC && c->mode != TPX_MODE_PAPER) return TPX_EINVAL;
    if (c->tof_max_ticks < 0 || c->tof_max_ticks > kMaxTofMax) return TPX_EINVAL;
    if (c->wrap_thr_pix_ticks <= 0 || c->wrap_thr_tdc_ticks <= 0) return TPX_EINVAL;
    if (c->tile_geometry != TPX_TILE_DEFAULT && c->tile_geometry != TPX_TILE_4096 && c->tile_geometry != TPX_TILE_2048)
        return TPX_EINVAL;
    if (c->flags & ~(TPX_FLAG_HOST_DIRECT | TPX_FLAG_LABELS32 | TPX_FLAG_RECORDS64)) return TPX_EINVAL;
    return TPX_OK;
}

void free_scratch(tpx_ctx *c) {
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    c->stage = nullptr;
    std::memset(&c->ts, 0, sizeof c->ts);
    c->max_tiles = 0;
}

int alloc_scratch(tpx_ctx *c, int64_t max_packets) {
    // sized for either tile geometry: the smaller tiles need more tile records
    const int64_t T = tpxk::fused_tile_packets(tpxk::GEO_T2048);
    int64_t tiles = (max_packets + T - 1) / T;
    if (tiles < 1) tiles = 1;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_flags = al(sizeof(unsigned) * tiles), b_agg = al(sizeof(tpxk::GAgg) * tiles),
                 b_cnt = al(sizeof(long long) * tiles), b_blk = al(tpxk::unwrap_prepass_scratch_bytes(tiles));
    // record staging of the fused kernel: one range's records per CTA
    size_t stage_records = 0;   // the largest grid of a call times its range capacity
    for (int geo : {(int)tpxk::GEO_T4096, (int)tpxk::GEO_T2048}) {
        const int64_t tg = (max_packets + tpxk::fused_tile_packets(geo) - 1) / tpxk::fused_tile_packets(geo);
        int64_t ctas = (int64_t)c->num_sms * tpxk::fused_ctas_per_sm(geo);
        if (tg < ctas) ctas = tg < 1 ? 1 : tg;
        const size_t r = (size_t)ctas * (size_t)tpxk::fused_range_capacity(geo);
        if (r > stage_records) stage_records = r;
    }
    c->stage_records = (int64_t)stage_records;
    const size_t b_stage = al(sizeof(tpx_record) * stage_records);
    const size_t total = b_flags + b_blk + 2 * b_agg + 2 * b_cnt + b_stage;
    void *mem = nullptr;
    if (cudaMalloc(&mem, total) != cudaSuccess) { cudaGetLastError(); return TPX_ENOMEM; }
    if (cudaMemset(mem, 0, total) != cudaSuccess) { cudaFree(mem); return TPX_ECUDA; }
    char *p = static_cast<char *>(mem);
    c->ts.blk = reinterpret_cast<tpxk::GAgg *>(p); p += b_blk;
    c->ts.cflags = reinterpret_cast<unsigned *>(p); p += b_flags;
    c->ts.agg = reinterpret_cast<tpxk::GAgg *>(p); p += b_agg;
    c->ts.pre = reinterpret_cast<tpxk::GAgg *>(p); p += b_agg;
    c->ts.cagg = reinterpret_cast<long long *>(p); p += b_cnt;
    c->ts.cpre = reinterpret_cast<long long *>(p); p += b_cnt;
    c->stage = reinterpret_cast<tpx_record *>(p);
    c->scratch = mem;
    c->max_tiles = tiles;
    c->max_packets = tiles * T;
    c->seq = 0;   // fresh flags: any sequence number is new
    return TPX_OK;
}

template <class Tp>
int grow(Tp **ptr, int64_t *cap, int64_t want) {
    if (*ptr && *cap >= want) return TPX_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    if (want <= 0) want = 1;
    if (cudaMalloc(reinterpret_cast<void **>(ptr), sizeof(Tp) * (size_t)want) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return TPX_ENOMEM;
    }
    *cap = want;
    return TPX_OK;
}

}  // namespace

namespace {

// A call's failure bits (a range the tiles could not hold, a batch run to
// redo) are resolved by the tpx_sync after it. When a new call starts before
// that sync, the previous call's bits move to the sticky word, and tpx_sync
// reports them instead of leaving that call's outputs silently incomplete.
__global__ void k_keep_status(const tpxk::Ctl *ctl, unsigned *sticky) {
    const unsigned f = ctl->status & (tpxk::ST_CAPACITY | tpxk::ST_EXCEPTION | tpxk::ST_RUN_REDO);
    if (f) *sticky |= f;
}
int begin_call(tpx_ctx *c) {
    if (!c->synced) {
        k_keep_status<<<1, 1, 0, c->stream>>>(c->ctl, c->d_sticky);
        if (ckr(cudaGetLastError())) return TPX_ECUDA;
    }
    c->synced = false;
    c->redone_early = 0;
    return TPX_OK;
}

// ---- tile-geometry autotuner ----
constexpr int64_t kTuneMinPackets = 1LL << 20;   // smaller calls run untimed on the 4096 tiles
constexpr double kTunePenalty = 1e30;            // a sample whose call had to be redone

int tune_pick(const tpx_ctx *c, int64_t n) {
    if (c->cfg.tile_geometry != TPX_TILE_DEFAULT) return c->geo;
    if (c->tune.fixed) return c->tune.fixed;
    if (n < kTuneMinPackets) return tpxk::GEO_T4096;
    // alternate, the smaller tiles first
    return c->tune.issued[tpxk::GEO_T2048 - 1] <= c->tune.issued[tpxk::GEO_T4096 - 1] ? tpxk::GEO_T2048 : tpxk::GEO_T4096;
}

// device memory (not mapped host or managed memory): the fused kernel may
// prefetch such packets into L2 with the bulk-copy engine
bool device_memory(const void *ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice;
}

// kernel timing: add the oldest recorded launch's pre-pass and fused-kernel
// times to the sums (waits for it)
int ktime_collect_one(tpx_ctx *c) {
    auto &k = c->kt;
    cudaEvent_t *e = k.ev[k.head];
    if (ckr(cudaEventSynchronize(e[2]))) return TPX_ECUDA;
    float a = 0.f, b = 0.f;
    if (ckr(cudaEventElapsedTime(&a, e[0], e[1])) || ckr(cudaEventElapsedTime(&b, e[1], e[2]))) return TPX_ECUDA;
    k.pre_ms += a;
    k.fused_ms += b;
    k.launches += 1;
    k.head = (k.head + 1) % tpx_ctx::KTime::kRing;
    return TPX_OK;
}

// the events of the next fused launch on `s`, or null when timing is off or
// the stream is being captured; the first one is recorded here
cudaEvent_t *ktime_begin(tpx_ctx *c, cudaStream_t s) {
    auto &k = c->kt;
    if (!k.on) return nullptr;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return nullptr;
    }
    if ((k.tail + 1) % tpx_ctx::KTime::kRing == k.head && ktime_collect_one(c)) return nullptr;
    cudaEvent_t *e = k.ev[k.tail];
    if (cudaEventRecord(e[0], s) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    return e;
}

void ktime_end(tpx_ctx *c, cudaEvent_t *e, cudaStream_t s) {
    if (!e) return;
    if (cudaEventRecord(e[2], s) != cudaSuccess) { cudaGetLastError(); return; }
    c->kt.tail = (c->kt.tail + 1) % tpx_ctx::KTime::kRing;
}

// time the samples whose calls have completed (all of them after a sync);
// `redone_last` marks the newest one as redone by the general path
void tune_collect(tpx_ctx *c, bool redone_last) {
    auto &t = c->tune;
    while (t.head != t.tail) {
        auto &smp = t.ring[t.head];
        if (cudaEventQuery(smp.b) != cudaSuccess) { cudaGetLastError(); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, smp.a, smp.b);
        const bool newest = (t.head + 1) % 8 == t.tail;
        const double v = (smp.failed || (redone_last && newest)) ? kTunePenalty : (double)ms * 1e6 / (double)smp.n;
        const int k = smp.geo - 1;
        if (t.done[k] == 0 || v < t.best[k]) t.best[k] = v;
        t.done[k] += 1;
        t.head = (t.head + 1) % 8;
    }
    if (!t.fixed && t.done[0] > 0 && t.done[1] > 0)
        t.fixed = t.best[tpxk::GEO_T2048 - 1] < t.best[tpxk::GEO_T4096 - 1] ? tpxk::GEO_T2048 : tpxk::GEO_T4096;
}

}  // namespace

extern "C" {

void tpx_config_default(tpx_config *c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->rx = 1;
    c->ry = 1;
    c->dt_ticks = 32;
    c->mode = TPX_MODE_CC;
    c->tof_max_ticks = 64000;
    c->wrap_thr_pix_ticks = 12800000000LL;
    c->wrap_thr_tdc_ticks = 12800000000LL;
    c->d_timewalk_lut = nullptr;
    c->strict = 0;
}

int tpx_create(tpx_ctx **out, const tpx_config *cfg, int64_t max_packets, void *cuda_stream) {
    if (!out || max_packets < 0) return TPX_EINVAL;
    *out = nullptr;
    int rc = check_cfg(cfg);
    if (rc) return rc;
    tpx_ctx *c = new (std::nothrow) tpx_ctx;
    if (!c) return TPX_ENOMEM;
    std::memset(c, 0, sizeof *c);
    c->cfg = *cfg;
    c->geo = cfg->tile_geometry == TPX_TILE_2048 ? (int)tpxk::GEO_T2048 : (int)tpxk::GEO_T4096;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return TPX_ECUDA; }
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        delete c;
        return TPX_ECUDA;
    }
    if (cudaMalloc(&c->ctl, sizeof(tpxk::Ctl)) != cudaSuccess) { delete c; return TPX_ENOMEM; }
    if (cudaMallocHost(&c->h_ctl, sizeof(tpxk::Ctl)) != cudaSuccess) {
        cudaFree(c->ctl);
        delete c;
        return TPX_ENOMEM;
    }
    std::memset(c->h_ctl, 0, sizeof(tpxk::Ctl));
    cudaMemset(c->ctl, 0, sizeof(tpxk::Ctl));
    if (cudaMalloc(&c->d_state, 2 * sizeof(tpxk::GAgg)) != cudaSuccess) {
        cudaFree(c->ctl);
        cudaFreeHost(c->h_ctl);
        delete c;
        return TPX_ENOMEM;
    }
    cudaMemset(c->d_state, 0, 2 * sizeof(tpxk::GAgg));   // all zero = the start of a stream
    if (cudaMalloc(&c->d_sticky, sizeof(unsigned)) != cudaSuccess || cudaMemset(c->d_sticky, 0, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        tpx_destroy(c);
        return TPX_ENOMEM;
    }
    c->synced = true;
    for (auto &smp : c->tune.ring)
        if (cudaEventCreate(&smp.a) != cudaSuccess || cudaEventCreate(&smp.b) != cudaSuccess) {
            tpx_destroy(c);
            return TPX_ECUDA;
        }
    if (cudaEventCreateWithFlags(&c->batch.tab_copied, cudaEventDisableTiming) != cudaSuccess) {
        tpx_destroy(c);
        return TPX_ECUDA;
    }
    rc = alloc_scratch(c, max_packets);
    if (rc) {
        cudaFree(c->ctl);
        cudaFreeHost(c->h_ctl);
        delete c;
        return rc;
    }
    *out = c;
    return TPX_OK;
}

int tpx_reserve(tpx_ctx *c, int64_t max_packets) {
    if (!c || max_packets < 0) return TPX_EINVAL;
    if (max_packets <= c->max_packets) return TPX_OK;
    if (ckr(cudaStreamSynchronize(c->stream))) return TPX_ECUDA;
    free_scratch(c);
    return alloc_scratch(c, max_packets);
}

int tpx_destroy(tpx_ctx *c) {
    if (!c) return TPX_EINVAL;
    cudaStreamSynchronize(c->stream);
    free_scratch(c);
    if (c->ctl) cudaFree(c->ctl);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->st_pk) cudaFree(c->st_pk);
    if (c->st_labels) cudaFree(c->st_labels);
    if (c->st_peak) cudaFree(c->st_peak);
    if (c->st_cl) cudaFree(c->st_cl);
    if (c->st_trig) cudaFree(c->st_trig);
    if (c->st_counts) cudaFree(c->st_counts);
    if (c->g_mem) cudaFree(c->g_mem);
    if (c->d_state) cudaFree(c->d_state);
    if (c->d_sticky) cudaFree(c->d_sticky);
    for (auto &smp : c->tune.ring) {
        if (smp.a) cudaEventDestroy(smp.a);
        if (smp.b) cudaEventDestroy(smp.b);
    }
    for (auto &tri : c->kt.ev)
        for (cudaEvent_t ev : tri)
            if (ev) cudaEventDestroy(ev);
    if (c->pipe.ready) {
        cudaStreamSynchronize(c->pipe.s_in);
        cudaStreamSynchronize(c->pipe.s_out);
        for (int k = 0; k < tpx_ctx::Pipe::kMax; ++k) {
            cudaEventDestroy(c->pipe.ev_in[k]);
            cudaEventDestroy(c->pipe.ev_done[k]);
            cudaEventDestroy(c->pipe.ev_out[k]);
        }
        cudaStreamDestroy(c->pipe.s_in);
        cudaStreamDestroy(c->pipe.s_out);
        cudaFreeHost(c->pipe.h_slot);
        cudaFree(c->pipe.d_counts);
    }
    for (int b = 0; b < 2; ++b) {
        if (c->pipe.pk[b]) cudaFree(c->pipe.pk[b]);
        if (c->pipe.cl[b]) cudaFree(c->pipe.cl[b]);
        if (c->pipe.trig[b]) cudaFree(c->pipe.trig[b]);
    }
    if (c->batch.tab_copied) cudaEventDestroy(c->batch.tab_copied);
    for (auto *o = c->batch.graph_owned; o;) {
        auto *nx = o->next;
        cudaFree(o->dev);
        cudaFreeHost(o->host);
        delete o;
        o = nx;
    }
    if (c->batch.dev) cudaFree(c->batch.dev);
    if (c->batch.h_tab) cudaFreeHost(c->batch.h_tab);
    delete c;
    return TPX_OK;
}

int tpx_process(tpx_ctx *c, const uint64_t *d_packets, int64_t n, int64_t idx_base, int64_t *d_labels,
                uint8_t *d_is_peak, tpx_record *d_clusters, int64_t cl_cap, int64_t *d_n_clusters,
                int64_t *d_trig, int64_t trig_cap, int64_t *d_n_trig) {
    if (!c || n < 0 || cl_cap < 0 || trig_cap < 0 || !d_n_clusters || !d_n_trig) return TPX_EINVAL;
    if (n > c->max_packets) return TPX_EINVAL;
    if (n > 0 && !d_packets) return TPX_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_packets) & 15) != 0) return TPX_EINVAL;
    if (cl_cap > 0 && !d_clusters) return TPX_EINVAL;
    if (trig_cap > 0 && !d_trig) return TPX_EINVAL;
    const bool l32 = (c->cfg.flags & TPX_FLAG_LABELS32) != 0;
    const int64_t l32_base = c->lab32_outer ? c->lab32_base : idx_base;
    if (l32 && d_labels && idx_base - l32_base + n > (1LL << 31) - 1) return TPX_EINVAL;
    if (begin_call(c)) return TPX_ECUDA;
    c->last.valid = true;
    c->batch.last = false;
    c->last.pk = d_packets;
    c->last.n = n;
    c->last.base = idx_base;
    c->last.labels = d_labels;
    c->last.lab32 = l32;
    c->last.lab32_base = l32_base;
    c->last.is_peak = d_is_peak;
    c->last.cl = d_clusters;
    c->last.cl_cap = cl_cap;
    c->last.n_cl = d_n_clusters;
    c->last.trig = d_trig;
    c->last.trig_cap = trig_cap;
    c->last.n_trig = d_n_trig;
    const tpxk::GAgg *E0 = nullptr;
    tpxk::GAgg *state_out = nullptr;
    take_state(c, &E0, &state_out);
    c->last.E0 = E0;
    c->last.state_out = state_out;
    if (ckr(cudaMemsetAsync(c->ctl, 0, sizeof(tpxk::Ctl), c->stream))) return TPX_ECUDA;
    if (ckr(cudaMemsetAsync(d_n_clusters, 0, sizeof(int64_t), c->stream))) return TPX_ECUDA;
    if (ckr(cudaMemsetAsync(d_n_trig, 0, sizeof(int64_t), c->stream))) return TPX_ECUDA;
    if (n == 0) {   // the state passes through unchanged
        if (E0) return cudaMemcpyAsync(state_out, E0, sizeof(tpxk::GAgg), cudaMemcpyDeviceToDevice, c->stream)
                       == cudaSuccess ? TPX_OK : TPX_ECUDA;
        return cudaMemsetAsync(state_out, 0, sizeof(tpxk::GAgg), c->stream) == cudaSuccess ? TPX_OK : TPX_ECUDA;
    }
    c->seq = (c->seq + 1) & 0x3FFFFFFFu;
    if (c->seq == 0) {   // sequence numbers wrapped: clear the flags once
        c->seq = 1;
        cudaMemsetAsync(c->ts.cflags, 0, sizeof(unsigned) * c->max_tiles, c->stream);
    }
    tpxk::Params p;
    std::memset(&p, 0, sizeof p);
    p.pk = d_packets;
    p.n = n;
    p.idx_base = idx_base;
    p.labels = l32 ? nullptr : reinterpret_cast<long long *>(d_labels);
    p.labels32 = l32 ? reinterpret_cast<int *>(d_labels) : nullptr;
    p.lab32_base = l32_base;
    p.l2_prefetch = (!c->packets_on_host && device_memory(d_packets)) ? 1 : 0;
    p.rec64 = (c->cfg.flags & TPX_FLAG_RECORDS64) ? 1 : 0;
    p.is_peak = d_is_peak;
    p.clusters = d_clusters;
    p.cl_cap = cl_cap;
    p.n_clusters = reinterpret_cast<long long *>(d_n_clusters);
    p.trig = reinterpret_cast<long long *>(d_trig);
    p.trig_cap = trig_cap;
    p.n_trig = reinterpret_cast<long long *>(d_n_trig);
    p.lut = c->cfg.d_timewalk_lut;
    p.rx = c->cfg.rx;
    p.ry = c->cfg.ry;
    p.dt = c->cfg.dt_ticks;
    p.strict = c->cfg.strict;
    p.tof_max = c->cfg.tof_max_ticks;
    p.thr_pix = c->cfg.wrap_thr_pix_ticks;
    p.thr_tdc = c->cfg.wrap_thr_tdc_ticks;
    const int geo = tune_pick(c, n);
    const int64_t T = tpxk::fused_tile_packets(geo);
    p.n_tiles = (n + T - 1) / T;
    p.seq = c->seq;
    p.ts = c->ts;
    p.ctl = c->ctl;
    p.E0 = E0;
    p.state_out = state_out;
    p.stage = c->stage;
    p.hold = c->hold_next;
    c->hold_next = 0;
    int64_t grid = (int64_t)c->num_sms * tpxk::fused_ctas_per_sm(geo);   // persistent, all resident
    if (grid > p.n_tiles) grid = p.n_tiles;
    auto &t = c->tune;
    const bool timed = c->cfg.tile_geometry == TPX_TILE_DEFAULT && !t.fixed && n >= kTuneMinPackets &&
                       (t.tail + 1) % 8 != t.head;
    if (timed && cudaEventRecord(t.ring[t.tail].a, c->stream) != cudaSuccess) return TPX_ECUDA;
    cudaEvent_t *kte = ktime_begin(c, c->stream);
    cudaError_t e = tpxk::launch_fused(p, c->cfg.mode, geo, (int)grid, c->stream, kte ? kte[1] : nullptr);
    if (e != cudaSuccess) return TPX_ECUDA;
    ktime_end(c, kte, c->stream);
    if (timed) {
        // a sample runs synchronously: a geometry whose ranges could not hold
        // the input loses, and that call is redone at once, so that a later
        // call cannot leave it unresolved
        auto &smp = t.ring[t.tail];
        if (ckr(cudaEventRecord(smp.b, c->stream))) return TPX_ECUDA;
        smp.geo = geo;
        smp.n = n;
        smp.failed = false;
        t.tail = (t.tail + 1) % 8;
        t.issued[geo - 1] += 1;
        unsigned st = 0;
        if (ckr(cudaMemcpyAsync(&st, &c->ctl->status, 4, cudaMemcpyDeviceToHost, c->stream)) ||
            ckr(cudaStreamSynchronize(c->stream)))
            return TPX_ECUDA;
        if ((st & (tpxk::ST_CAPACITY | tpxk::ST_EXCEPTION)) && !(st & tpxk::ST_DEVTIMEOUT)) {
            smp.failed = true;
            const int rc = tpxg::redo_last(c);
            c->last.valid = false;
            c->redone_early = 1;
            if (rc) return rc;
        }
    }
    return TPX_OK;
}

int tpx_process_batch(tpx_ctx *c, const uint64_t *d_packets, const int64_t *h_run_offsets, int64_t n_runs,
                      int64_t *d_labels, uint8_t *d_is_peak, tpx_record *d_clusters, int64_t cl_cap,
                      int64_t *d_n_clusters, int64_t *d_run_clusters, int64_t *d_trig, int64_t trig_cap,
                      int64_t *d_n_trig, int64_t *d_run_trig) {
    if (!c || !h_run_offsets || n_runs < 1 || cl_cap < 0 || trig_cap < 0 || !d_n_clusters || !d_n_trig ||
        !d_run_clusters || !d_run_trig)
        return TPX_EINVAL;
    if (h_run_offsets[0] != 0) return TPX_EINVAL;
    if ((c->cfg.flags & TPX_FLAG_LABELS32) && d_labels) return TPX_EINVAL;   // batch labels are int64
    if (c->cfg.flags & TPX_FLAG_RECORDS64) return TPX_EINVAL;                // batch records are 88 bytes
    for (int64_t r = 0; r < n_runs; ++r)
        if (h_run_offsets[r + 1] < h_run_offsets[r]) return TPX_EINVAL;
    const int64_t n = h_run_offsets[n_runs];
    if (n > (1LL << 40) || n_runs > (1LL << 30)) return TPX_EINVAL;
    if (n > 0 && !d_packets) return TPX_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_packets) & 15) != 0) return TPX_EINVAL;
    if (cl_cap > 0 && !d_clusters) return TPX_EINVAL;
    if (trig_cap > 0 && !d_trig) return TPX_EINVAL;
    if (begin_call(c)) return TPX_ECUDA;
    cudaStream_t s = c->stream;
    // batches run on the larger ranges unless the configuration says
    // otherwise: a run whose shots overflow a range costs a general-path redo
    const int geo = c->cfg.tile_geometry == TPX_TILE_DEFAULT ? (int)tpxk::GEO_T4096 : c->geo;
    const int64_t T = tpxk::fused_tile_packets(geo), C = tpxk::fused_range_capacity(geo);
    // the tile queue: every run gets at least one tile (an empty run's tile
    // still records the run's offsets)
    int64_t n_tiles = 0;
    for (int64_t r = 0; r < n_runs; ++r) {
        const int64_t len = h_run_offsets[r + 1] - h_run_offsets[r];
        n_tiles += len > 0 ? (len + T - 1) / T : 1;
    }
    if (n_tiles >= (1LL << 31)) return TPX_EINVAL;
    int64_t grid = (int64_t)c->num_sms * tpxk::fused_ctas_per_sm(geo);
    if (grid > c->stage_records / C) grid = c->stage_records / C;
    if (grid > n_tiles) grid = n_tiles;
    if (grid < 1) return TPX_EINVAL;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    // CC mode: a range past the capacity goes through the big-range path,
    // with global scratch per CTA of the grid
    const size_t big_bytes = c->cfg.mode == TPX_MODE_CC ? (size_t)grid * tpxk::fused_big_scratch_bytes(geo) : 0;
    // a batch CTA holds up to kBatchRing staged tiles (records and triggers)
    constexpr int64_t RG = tpxk::kBatchRing;
    const size_t stage_bytes = sizeof(tpx_record) * (size_t)(grid * RG * C);
    // device scratch of the batch
    auto &B = c->batch;
    const size_t need_dev = al(4 * (size_t)n_tiles) + al(8 * (size_t)n_runs) + al(8 * (size_t)(n_runs + 1)) +
                            al(4 * (size_t)n_runs) + 4 * al(8 * (size_t)n_tiles) + al(8 * (size_t)(grid * T * RG)) +
                            al(tpxk::unwrap_prepass_scratch_bytes(n_tiles)) + al(4 * (size_t)n_tiles) +
                            2 * al(sizeof(tpxk::GAgg) * (size_t)n_tiles) + al(big_bytes) + al(stage_bytes);
    const size_t need_host = 8 * (size_t)(n_runs + 1) + 8 * (size_t)n_runs + 4 * (size_t)n_tiles + 64;
    // a call captured into a CUDA graph (relaxed capture mode) gets its own
    // device tables and pinned host tables, kept for the graph's replays
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (ckr(cudaStreamIsCapturing(s, &cap))) return TPX_ECUDA;
    const bool capturing = cap == cudaStreamCaptureStatusActive;
    void *dev = nullptr;
    int64_t *h_tab = nullptr;
    if (capturing) {
        auto *o = new (std::nothrow) tpx_ctx::Batch::Owned{nullptr, nullptr, B.graph_owned};
        if (!o) return TPX_ENOMEM;
        if (cudaMalloc(&o->dev, need_dev) != cudaSuccess || cudaMallocHost(&o->host, need_host) != cudaSuccess) {
            cudaGetLastError();
            if (o->dev) cudaFree(o->dev);
            delete o;
            return TPX_ENOMEM;
        }
        B.graph_owned = o;
        dev = o->dev;
        h_tab = static_cast<int64_t *>(o->host);
    }
    if (!capturing && need_dev > B.dev_bytes) {
        if (ckr(cudaStreamSynchronize(s))) return TPX_ECUDA;
        if (B.dev) cudaFree(B.dev);
        B.dev = nullptr;
        B.dev_bytes = 0;
        if (cudaMalloc(&B.dev, need_dev) != cudaSuccess) { cudaGetLastError(); return TPX_ENOMEM; }
        if (ckr(cudaMemset(B.dev, 0, need_dev))) return TPX_ECUDA;   // fresh flags
        B.dev_bytes = need_dev;
    }
    if (!capturing && B.h_tab) {   // the previous batch's tables may still be uploading
        if (ckr(cudaEventSynchronize(B.tab_copied))) return TPX_ECUDA;
    }
    if (!capturing && need_host > B.h_bytes) {
        if (B.h_tab) cudaFreeHost(B.h_tab);
        B.h_tab = nullptr;
        B.h_bytes = 0;
        if (cudaMallocHost(&B.h_tab, need_host) != cudaSuccess) { cudaGetLastError(); return TPX_ENOMEM; }
        B.h_bytes = need_host;
    }
    if (!capturing) {
        dev = B.dev;
        h_tab = B.h_tab;
    }
    char *m = static_cast<char *>(dev);
    auto take = [&](size_t bytes) { char *r = m; m += al(bytes); return r; };
    tpxk::BatchTable &bt = B.bt;
    bt.tile_run = reinterpret_cast<int *>(take(4 * (size_t)n_tiles));
    bt.run_tile0 = reinterpret_cast<long long *>(take(8 * (size_t)n_runs));
    bt.run_off = reinterpret_cast<long long *>(take(8 * (size_t)(n_runs + 1)));
    bt.run_failed = reinterpret_cast<unsigned *>(take(4 * (size_t)n_runs));
    bt.tcagg = reinterpret_cast<long long *>(take(8 * (size_t)n_tiles));
    bt.tcpre = reinterpret_cast<long long *>(take(8 * (size_t)n_tiles));
    B.ts.cagg = reinterpret_cast<long long *>(take(8 * (size_t)n_tiles));
    B.ts.cpre = reinterpret_cast<long long *>(take(8 * (size_t)n_tiles));
    bt.tstage = reinterpret_cast<long long *>(take(8 * (size_t)(grid * T * RG)));
    B.ts.blk = reinterpret_cast<tpxk::GAgg *>(take(tpxk::unwrap_prepass_scratch_bytes(n_tiles)));
    B.ts.cflags = reinterpret_cast<unsigned *>(take(4 * (size_t)n_tiles));
    B.ts.agg = reinterpret_cast<tpxk::GAgg *>(take(sizeof(tpxk::GAgg) * (size_t)n_tiles));
    B.ts.pre = reinterpret_cast<tpxk::GAgg *>(take(sizeof(tpxk::GAgg) * (size_t)n_tiles));
    unsigned char *big = big_bytes ? reinterpret_cast<unsigned char *>(take(big_bytes)) : nullptr;
    tpx_record *bstage = reinterpret_cast<tpx_record *>(take(stage_bytes));
    bt.run_rec_off = reinterpret_cast<long long *>(d_run_clusters);
    bt.run_trig_off = reinterpret_cast<long long *>(d_run_trig);
    bt.n_runs = n_runs;
    // the tables, built on the host and uploaded from pinned memory
    int64_t *h_off = h_tab, *h_t0 = h_tab + (n_runs + 1);
    int *h_tr = reinterpret_cast<int *>(h_tab + (n_runs + 1) + n_runs);
    std::memcpy(h_off, h_run_offsets, 8 * (size_t)(n_runs + 1));
    int64_t g = 0;
    for (int64_t r = 0; r < n_runs; ++r) {
        const int64_t len = h_off[r + 1] - h_off[r];
        const int64_t k = len > 0 ? (len + T - 1) / T : 1;
        h_t0[r] = g;
        for (int64_t i = 0; i < k; ++i) h_tr[g + i] = (int)r;
        g += k;
    }
    if (cudaMemcpyAsync(const_cast<long long *>(bt.run_off), h_off, 8 * (size_t)(n_runs + 1), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(const_cast<long long *>(bt.run_tile0), h_t0, 8 * (size_t)n_runs, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(const_cast<int *>(bt.tile_run), h_tr, 4 * (size_t)n_tiles, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return TPX_ECUDA;
    if (!capturing && ckr(cudaEventRecord(B.tab_copied, s))) return TPX_ECUDA;
    // the scratch layout follows the tile count: start every call's flags at zero
    if (ckr(cudaMemsetAsync(B.ts.cflags, 0, 4 * (size_t)n_tiles, s))) return TPX_ECUDA;
    if (ckr(cudaMemsetAsync(bt.run_failed, 0, 4 * (size_t)n_runs, s))) return TPX_ECUDA;
    if (ckr(cudaMemsetAsync(c->ctl, 0, sizeof(tpxk::Ctl), s))) return TPX_ECUDA;
    if (cudaMemsetAsync(d_n_clusters, 0, 8, s) != cudaSuccess || cudaMemsetAsync(d_n_trig, 0, 8, s) != cudaSuccess)
        return TPX_ECUDA;
    c->seq = (c->seq + 1) & 0x3FFFFFFFu;
    if (c->seq == 0) {   // sequence numbers wrapped: clear every flag once
        c->seq = 1;
        cudaMemsetAsync(c->ts.cflags, 0, sizeof(unsigned) * c->max_tiles, s);
        cudaMemsetAsync(B.ts.cflags, 0, 4 * (size_t)n_tiles, s);
    }
    tpxk::Params p;
    std::memset(&p, 0, sizeof p);
    p.pk = d_packets;
    p.n = n;
    p.idx_base = 0;
    p.labels = reinterpret_cast<long long *>(d_labels);
    p.is_peak = d_is_peak;
    p.clusters = d_clusters;
    p.cl_cap = cl_cap;
    p.n_clusters = reinterpret_cast<long long *>(d_n_clusters);
    p.trig = reinterpret_cast<long long *>(d_trig);
    p.trig_cap = trig_cap;
    p.n_trig = reinterpret_cast<long long *>(d_n_trig);
    p.lut = c->cfg.d_timewalk_lut;
    p.rx = c->cfg.rx;
    p.ry = c->cfg.ry;
    p.dt = c->cfg.dt_ticks;
    p.strict = c->cfg.strict;
    p.tof_max = c->cfg.tof_max_ticks;
    p.thr_pix = c->cfg.wrap_thr_pix_ticks;
    p.thr_tdc = c->cfg.wrap_thr_tdc_ticks;
    p.n_tiles = n_tiles;
    p.seq = c->seq;
    p.ts = B.ts;
    p.ctl = c->ctl;
    p.stage = bstage;
    p.bt = bt;
    p.big = big;
    cudaEvent_t *kte = ktime_begin(c, s);
    if (ckr(tpxk::launch_fused(p, c->cfg.mode, geo, (int)grid, s, kte ? kte[1] : nullptr))) return TPX_ECUDA;
    ktime_end(c, kte, s);
    // what a redo of failed runs needs
    c->last.valid = false;
    B.last = true;
    B.pk = d_packets;
    B.n_runs = n_runs;
    B.labels = d_labels;
    B.is_peak = d_is_peak;
    B.cl = d_clusters;
    B.cl_cap = cl_cap;
    B.n_cl = d_n_clusters;
    B.trig = d_trig;
    B.trig_cap = trig_cap;
    B.n_trig = d_n_trig;
    B.h_off = h_off;
    return TPX_OK;
}

int tpx_kernel_timing(tpx_ctx *c, int enable) {
    if (!c) return TPX_EINVAL;
    auto &k = c->kt;
    if (enable && !k.ev[0][0])
        for (auto &tri : k.ev)
            for (cudaEvent_t &ev : tri)
                if (ckr(cudaEventCreate(&ev))) return TPX_ECUDA;
    if (enable) {
        if (int rc = tpx_kernel_times(c, nullptr, nullptr, nullptr)) return rc;   // nothing left in flight
        k.pre_ms = k.fused_ms = 0.0;
        k.launches = 0;
    }
    k.on = enable != 0;
    return TPX_OK;
}

int tpx_kernel_times(tpx_ctx *c, double *prepass_ms, double *fused_ms, int64_t *launches) {
    if (!c) return TPX_EINVAL;
    auto &k = c->kt;
    while (k.head != k.tail)
        if (int rc = ktime_collect_one(c)) return rc;
    if (prepass_ms) *prepass_ms = k.pre_ms;
    if (fused_ms) *fused_ms = k.fused_ms;
    if (launches) *launches = k.launches;
    return TPX_OK;
}

int tpx_sync(tpx_ctx *c, tpx_counters *out) {
    if (!c) return TPX_EINVAL;
    int64_t redone = c->redone_early;
    c->redone_early = 0;
    c->synced = true;
    unsigned sticky = 0;
    if (ckr(cudaMemcpyAsync(&sticky, c->d_sticky, 4, cudaMemcpyDeviceToHost, c->stream)) ||
        ckr(cudaMemsetAsync(c->d_sticky, 0, 4, c->stream)))
        return TPX_ECUDA;
    if (cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(tpxk::Ctl), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return TPX_ECUDA;
    if (ckr(cudaStreamSynchronize(c->stream))) return TPX_ECUDA;
    // a checked build's index violation stays reported even when the call is redone
    const unsigned bounds = c->h_ctl->status & tpxk::ST_BOUNDS;
    if ((c->h_ctl->status & (tpxk::ST_CAPACITY | tpxk::ST_EXCEPTION)) && !(c->h_ctl->status & tpxk::ST_DEVTIMEOUT) &&
        c->last.valid) {
        // the fused kernel met an input it cannot hold on chip: redo the call
        // exactly with the general path, then report that run
        const int rc = tpxg::redo_last(c);
        c->last.valid = false;
        redone = 1;
        if (rc) return rc;
        if (cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(tpxk::Ctl), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            return TPX_ECUDA;
        if (ckr(cudaStreamSynchronize(c->stream))) return TPX_ECUDA;
    }
    if ((c->h_ctl->status & tpxk::ST_RUN_REDO) && !(c->h_ctl->status & tpxk::ST_DEVTIMEOUT) && c->batch.last) {
        // runs of the last batch that the tiles could not hold: redo them
        // exactly with the general path and splice their outputs in
        // (the batch stays the last call: a CUDA-graph replay of it sets the
        // redo bit again; the redo clears it, so a second sync does not redo)
        const int rc = tpxg::redo_batch(c, &redone);
        if (rc) return rc;
        if (cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(tpxk::Ctl), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            return TPX_ECUDA;
        if (ckr(cudaStreamSynchronize(c->stream))) return TPX_ECUDA;
    }
    tune_collect(c, redone != 0);
    c->h_ctl->status |= bounds;
    const tpxk::Ctl &h = *c->h_ctl;
    if (out) {
        out->packets = (int64_t)h.counters[tpxk::C_PACKETS];
        out->pixels = (int64_t)h.counters[tpxk::C_PIXELS];
        out->tdcs = (int64_t)h.counters[tpxk::C_TDCS];
        out->corrupt = (int64_t)h.counters[tpxk::C_CORRUPT];
        out->dropped_pre_trigger = (int64_t)h.counters[tpxk::C_DROP_PRE];
        out->dropped_background = (int64_t)h.counters[tpxk::C_DROP_BG];
        out->kept = (int64_t)h.counters[tpxk::C_KEPT];
        out->clusters = (int64_t)h.counters[tpxk::C_CLUSTERS];
        out->peaks = (int64_t)h.counters[tpxk::C_PEAKS];
        out->status_bits = (int64_t)h.status;
        out->redone = redone;
    }
    const unsigned s = h.status;
    if (s & tpxk::ST_DEVTIMEOUT) return TPX_EDEVTIMEOUT;
    if (s & tpxk::ST_BOUNDS) return TPX_EUNSUPPORTED;   // checked build: an access was skipped
    // an earlier call since the previous sync needed the general path, which
    // only the last call gets: its outputs are incomplete
    if (sticky) return TPX_EUNSUPPORTED;
    if (s & tpxk::ST_TRIG_ORDER) return TPX_ECORRUPT;
    if (s & (tpxk::ST_CAPACITY | tpxk::ST_EXCEPTION)) return TPX_EUNSUPPORTED;
    if (c->cfg.strict && h.counters[tpxk::C_CORRUPT]) return TPX_ECORRUPT;
    if (s & (tpxk::ST_CLUSTER_CAP | tpxk::ST_TRIG_CAP)) return TPX_EOVERFLOW;
    return TPX_OK;
}

namespace {

constexpr int64_t kPipeMinPackets = 1LL << 24;     // below this one call does it
constexpr int64_t kPipePiecePackets = 1LL << 23;   // smallest piece

int pipe_init(tpx_ctx *c) {
    auto &P = c->pipe;
    if (P.ready) return TPX_OK;
    if (ckr(cudaStreamCreateWithFlags(&P.s_in, cudaStreamNonBlocking)) ||
        ckr(cudaStreamCreateWithFlags(&P.s_out, cudaStreamNonBlocking)))
        return TPX_ECUDA;
    for (int k = 0; k < tpx_ctx::Pipe::kMax; ++k)
        if (ckr(cudaEventCreateWithFlags(&P.ev_in[k], cudaEventDisableTiming)) ||
            ckr(cudaEventCreateWithFlags(&P.ev_done[k], cudaEventDisableTiming)) ||
            ckr(cudaEventCreateWithFlags(&P.ev_out[k], cudaEventDisableTiming)))
            return TPX_ECUDA;
    if (ckr(cudaMallocHost(reinterpret_cast<void **>(&P.h_slot), sizeof(tpx_ctx::Pipe::Slot) * tpx_ctx::Pipe::kMax)))
        return TPX_ENOMEM;
    if (ckr(cudaMalloc(reinterpret_cast<void **>(&P.d_counts), sizeof(int64_t) * 2 * tpx_ctx::Pipe::kMax)))
        return TPX_ENOMEM;
    P.ready = true;
    return TPX_OK;
}

// piece boundaries: near k n / K, moved forward to the next trigger packet,
// so that each piece starts with its own shot; returns the number of pieces
int pipe_cuts(const uint64_t *h, int64_t n, int64_t *cut) {
    int K = (int)std::min<int64_t>(tpx_ctx::Pipe::kMax, n / kPipePiecePackets);
    int m = 0;
    cut[m++] = 0;
    for (int k = 1; k < K; ++k) {
        int64_t q = std::max(k * (n / K), cut[m - 1] + kPipePiecePackets / 2);
        while (q < n && (h[q] >> 60) != 0x6u) ++q;
        if (q >= n) break;
        cut[m++] = q;
    }
    cut[m] = n;
    return m;
}

}  // namespace

// The host call on a large input, pipelined: piece k's packets go up while
// piece k-1 runs and piece k-2's labels and records come down. The pieces are
// chained through the unwrap state exactly as consecutive calls; a cut is
// exact when no pixel after it belongs to the shot before it in time, and a
// piece whose fused kernel reports anything it cannot hold (such a pixel is
// one) sends the whole call back to the one-piece path. A state set by
// tpx_set_state starts the first piece (and is put back for the one-piece
// path). Returns 1 when it declined (the caller then runs the plain path),
// else a status.
static int process_host_pipelined(tpx_ctx *c, const uint64_t *h_packets, int64_t n, int64_t idx_base,
                                  int64_t *h_labels, uint8_t *h_is_peak, tpx_record *h_clusters, int64_t cl_cap,
                                  int64_t *h_n_clusters, int64_t *h_trig, int64_t trig_cap, int64_t *h_n_trig) {
    if (n < kPipeMinPackets || c->cfg.chain) return 1;
    const bool user_state = c->state_once;   // tpx_set_state before the call: the first piece starts there
    int64_t cut[tpx_ctx::Pipe::kMax + 1];
    const int K = pipe_cuts(h_packets, n, cut);
    if (K < 2) return 1;
    int rc = pipe_init(c);
    if (rc) return rc;
    auto &P = c->pipe;
    int64_t maxp = 0;
    for (int k = 0; k < K; ++k) maxp = std::max(maxp, cut[k + 1] - cut[k]);
    for (int b = 0; b < 2; ++b) {
        int64_t cap = P.pk_cap;
        if ((rc = grow(&P.pk[b], &cap, maxp))) return rc;
        cap = P.cl_cap;
        if ((rc = grow(&P.cl[b], &cap, cl_cap))) return rc;
        cap = P.trig_cap;
        if ((rc = grow(&P.trig[b], &cap, trig_cap))) return rc;
    }
    P.pk_cap = std::max(P.pk_cap, maxp);
    P.cl_cap = std::max(P.cl_cap, cl_cap);
    P.trig_cap = std::max(P.trig_cap, trig_cap);
    if (h_labels && (rc = grow(&c->st_labels, &c->st_labels_cap, n))) return rc;
    if (h_is_peak && (rc = grow(&c->st_peak, &c->st_peak_cap, n))) return rc;
    // int32 labels (TPX_FLAG_LABELS32) stay relative to the whole call
    const size_t les = (c->cfg.flags & TPX_FLAG_LABELS32) ? 4 : 8;
    const size_t rsz = (c->cfg.flags & TPX_FLAG_RECORDS64) ? sizeof(tpx_record64) : sizeof(tpx_record);
    char *st_lab = reinterpret_cast<char *>(c->st_labels);
    char *h_lab = reinterpret_cast<char *>(h_labels);
    cudaStream_t sc = c->stream;
    // all earlier work on the context stream is done before the copies start
    if (ckr(cudaEventRecord(P.ev_done[0], sc)) || ckr(cudaStreamWaitEvent(P.s_in, P.ev_done[0], 0)) ||
        ckr(cudaStreamWaitEvent(P.s_out, P.ev_done[0], 0)))
        return TPX_ECUDA;
    auto h2d = [&](int k) -> int {
        const int64_t m = cut[k + 1] - cut[k];
        if (k >= 2 && ckr(cudaStreamWaitEvent(P.s_in, P.ev_done[k - 2], 0))) return TPX_ECUDA;
        if (ckr(cudaMemcpyAsync(P.pk[k & 1], h_packets + cut[k], sizeof(uint64_t) * m, cudaMemcpyHostToDevice, P.s_in)) ||
            ckr(cudaEventRecord(P.ev_in[k], P.s_in)))
            return TPX_ECUDA;
        return TPX_OK;
    };
    int64_t rec_off = 0, trig_off = 0;
    bool failed = false;
    tpxk::Ctl total;
    std::memset(&total, 0, sizeof total);
    // records and triggers of piece k come down once its counts are known
    auto d2h_records = [&](int k) -> int {
        if (ckr(cudaEventSynchronize(P.ev_done[k]))) return TPX_ECUDA;
        const auto &sl = P.h_slot[k];
        total.status |= sl.ctl.status;
        for (int i = 0; i < tpxk::C_NUM; ++i) total.counters[i] += sl.ctl.counters[i];
        if (sl.ctl.status & (tpxk::ST_CAPACITY | tpxk::ST_EXCEPTION | tpxk::ST_DEVTIMEOUT)) failed = true;
        const int64_t ncl = sl.counts[0], ntr = sl.counts[1];
        const int64_t ccl = std::max<int64_t>(0, std::min(ncl, cl_cap - rec_off));
        const int64_t ctr = std::max<int64_t>(0, std::min(ntr, trig_cap - trig_off));
        if (!failed && ccl > 0 &&
            ckr(cudaMemcpyAsync(reinterpret_cast<char *>(h_clusters) + rsz * rec_off, P.cl[k & 1], rsz * ccl,
                                cudaMemcpyDeviceToHost, P.s_out)))
            return TPX_ECUDA;
        if (!failed && ctr > 0 &&
            ckr(cudaMemcpyAsync(h_trig + trig_off, P.trig[k & 1], sizeof(int64_t) * ctr, cudaMemcpyDeviceToHost, P.s_out)))
            return TPX_ECUDA;
        rec_off += ncl;
        trig_off += ntr;
        return ckr(cudaEventRecord(P.ev_out[k], P.s_out)) ? TPX_ECUDA : TPX_OK;
    };
    if ((rc = h2d(0))) return rc;
    for (int k = 0; k < K; ++k) {
        if (k + 1 < K && (rc = h2d(k + 1))) return rc;
        const int64_t m = cut[k + 1] - cut[k];
        if (ckr(cudaStreamWaitEvent(sc, P.ev_in[k], 0))) return TPX_ECUDA;
        if (k >= 2 && ckr(cudaStreamWaitEvent(sc, P.ev_out[k - 2], 0))) return TPX_ECUDA;
        c->state_once = k > 0 || user_state;   // continue from the previous piece's state
        c->lab32_outer = true;
        c->lab32_base = idx_base;
        rc = tpx_process(c, P.pk[k & 1], m, idx_base + cut[k],
                         h_labels ? reinterpret_cast<int64_t *>(st_lab + les * cut[k]) : nullptr,
                         h_is_peak ? c->st_peak + cut[k] : nullptr, P.cl[k & 1], cl_cap, P.d_counts + 2 * k,
                         P.trig[k & 1], trig_cap, P.d_counts + 2 * k + 1);
        c->lab32_outer = false;
        if (rc) return rc;
        // a piece the autotuner's sample already redid on the general path
        // cannot show whether its cut was exact
        if (c->redone_early) failed = true;
        if (ckr(cudaMemcpyAsync(P.h_slot[k].counts, P.d_counts + 2 * k, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, sc)) ||
            ckr(cudaMemcpyAsync(&P.h_slot[k].ctl, c->ctl, sizeof(tpxk::Ctl), cudaMemcpyDeviceToHost, sc)) ||
            ckr(cudaEventRecord(P.ev_done[k], sc)))
            return TPX_ECUDA;
        // piece k-1's records go down before piece k's labels: the kernel of
        // piece k+1 waits for them (it reuses their buffer), not for k's labels
        if (k >= 1 && (rc = d2h_records(k - 1))) return rc;
        if (ckr(cudaStreamWaitEvent(P.s_out, P.ev_done[k], 0))) return TPX_ECUDA;
        if (h_labels && ckr(cudaMemcpyAsync(h_lab + les * cut[k], st_lab + les * cut[k], les * m,
                                            cudaMemcpyDeviceToHost, P.s_out)))
            return TPX_ECUDA;
        if (h_is_peak && ckr(cudaMemcpyAsync(h_is_peak + cut[k], c->st_peak + cut[k], (size_t)m, cudaMemcpyDeviceToHost,
                                             P.s_out)))
            return TPX_ECUDA;
    }
    if ((rc = d2h_records(K - 1))) return rc;
    if (ckr(cudaStreamSynchronize(P.s_out)) || ckr(cudaStreamSynchronize(sc))) return TPX_ECUDA;
    if (failed) {
        // forget the pieces: no failure of theirs may reach the next sync
        if (ckr(cudaMemsetAsync(c->d_sticky, 0, 4, sc)) || ckr(cudaStreamSynchronize(sc))) return TPX_ECUDA;
        c->synced = true;
        c->last.valid = false;
        c->state_once = false;
        if (user_state) {   // the one-piece path starts from the same state
            if (ckr(cudaMemcpyAsync(&c->d_state[c->cur], &c->h_state, sizeof c->h_state, cudaMemcpyHostToDevice, sc)) ||
                ckr(cudaStreamSynchronize(sc)))
                return TPX_ECUDA;
            c->state_once = true;
        }
        return 1;
    }
    // the call's counters and status, as one call would leave them
    total.tile_counter = 0;
    if (ckr(cudaMemcpyAsync(c->ctl, &total, sizeof total, cudaMemcpyHostToDevice, sc)) ||
        ckr(cudaStreamSynchronize(sc)))
        return TPX_ECUDA;
    *h_n_clusters = rec_off;
    *h_n_trig = trig_off;
    rc = tpx_sync(c, nullptr);
    if (rc == TPX_OK && (rec_off > cl_cap || trig_off > trig_cap)) rc = TPX_EOVERFLOW;
    return rc;
}

// a host buffer the device reaches at the same address (pinned and mapped)
static bool host_mapped(const void *p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

// TPX_FLAG_HOST_DIRECT: the fused kernel on the mapped host buffers in place
// (counts in device memory); returns 1 when it declined
static int process_host_direct(tpx_ctx *c, const uint64_t *h_packets, int64_t n, int64_t idx_base, int64_t *h_labels,
                               uint8_t *h_is_peak, tpx_record *h_clusters, int64_t cl_cap, int64_t *h_n_clusters,
                               int64_t *h_trig, int64_t trig_cap, int64_t *h_n_trig) {
    if (!(c->cfg.flags & TPX_FLAG_HOST_DIRECT) || n == 0) return 1;
    if (!host_mapped(h_packets) || !host_mapped(h_labels) || !host_mapped(h_is_peak) || !host_mapped(h_clusters) ||
        !host_mapped(h_trig) || (reinterpret_cast<uintptr_t>(h_packets) & 15))
        return 1;
    int rc = grow(&c->st_counts, &c->st_counts_cap, 2);
    if (rc) return rc;
    c->packets_on_host = true;
    rc = tpx_process(c, h_packets, n, idx_base, h_labels, h_is_peak, h_clusters, cl_cap, c->st_counts, h_trig, trig_cap,
                     c->st_counts + 1);
    c->packets_on_host = false;
    if (rc) return rc;
    rc = tpx_sync(c, nullptr);
    int64_t cnt[2] = {0, 0};
    if (ckr(cudaMemcpy(cnt, c->st_counts, sizeof cnt, cudaMemcpyDeviceToHost))) return TPX_ECUDA;
    *h_n_clusters = cnt[0];
    *h_n_trig = cnt[1];
    return rc;
}

int tpx_process_host(tpx_ctx *c, const uint64_t *h_packets, int64_t n, int64_t idx_base, int64_t *h_labels,
                     uint8_t *h_is_peak, tpx_record *h_clusters, int64_t cl_cap, int64_t *h_n_clusters,
                     int64_t *h_trig, int64_t trig_cap, int64_t *h_n_trig) {
    if (!c || n < 0 || cl_cap < 0 || trig_cap < 0 || !h_n_clusters || !h_n_trig) return TPX_EINVAL;
    if (n > 0 && !h_packets) return TPX_EINVAL;
    if (n > c->max_packets) return TPX_EINVAL;
    if (cl_cap > 0 && !h_clusters) return TPX_EINVAL;
    if (trig_cap > 0 && !h_trig) return TPX_EINVAL;
    int rc = process_host_direct(c, h_packets, n, idx_base, h_labels, h_is_peak, h_clusters, cl_cap, h_n_clusters,
                                 h_trig, trig_cap, h_n_trig);
    if (rc != 1) return rc;
    rc = process_host_pipelined(c, h_packets, n, idx_base, h_labels, h_is_peak, h_clusters, cl_cap, h_n_clusters,
                                    h_trig, trig_cap, h_n_trig);
    if (rc != 1) return rc;
    if ((rc = grow(&c->st_pk, &c->st_n, n))) return rc;
    if (h_labels && (rc = grow(&c->st_labels, &c->st_labels_cap, n))) return rc;
    if (h_is_peak && (rc = grow(&c->st_peak, &c->st_peak_cap, n))) return rc;
    if ((rc = grow(&c->st_cl, &c->st_cl_cap, cl_cap))) return rc;
    if ((rc = grow(&c->st_trig, &c->st_trig_cap, trig_cap))) return rc;
    if ((rc = grow(&c->st_counts, &c->st_counts_cap, 2))) return rc;
    cudaStream_t s = c->stream;
    if (n && cudaMemcpyAsync(c->st_pk, h_packets, sizeof(uint64_t) * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TPX_ECUDA;
    rc = tpx_process(c, c->st_pk, n, idx_base, h_labels ? c->st_labels : nullptr, h_is_peak ? c->st_peak : nullptr,
                     c->st_cl, cl_cap, c->st_counts, c->st_trig, trig_cap, c->st_counts + 1);
    if (rc) return rc;
    int64_t counts[2] = {0, 0};
    if (ckr(cudaMemcpyAsync(counts, c->st_counts, sizeof counts, cudaMemcpyDeviceToHost, s))) return TPX_ECUDA;
    if (h_labels && n &&
        cudaMemcpyAsync(h_labels, c->st_labels, ((c->cfg.flags & TPX_FLAG_LABELS32) ? 4 : 8) * (size_t)n,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return TPX_ECUDA;
    if (h_is_peak && n && cudaMemcpyAsync(h_is_peak, c->st_peak, n, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return TPX_ECUDA;
    if (ckr(cudaStreamSynchronize(s))) return TPX_ECUDA;
    const int64_t ncl = counts[0] < cl_cap ? counts[0] : cl_cap;
    const int64_t ntr = counts[1] < trig_cap ? counts[1] : trig_cap;
    const size_t rsz = (c->cfg.flags & TPX_FLAG_RECORDS64) ? sizeof(tpx_record64) : sizeof(tpx_record);
    if (ncl > 0 && cudaMemcpyAsync(h_clusters, c->st_cl, rsz * ncl, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return TPX_ECUDA;
    if (ntr > 0 && cudaMemcpyAsync(h_trig, c->st_trig, sizeof(int64_t) * ntr, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return TPX_ECUDA;
    *h_n_clusters = counts[0];
    *h_n_trig = counts[1];
    return tpx_sync(c, nullptr);
}

int tpx_debug_hold_tile(tpx_ctx *c, int64_t tile) {
    if (!c) return TPX_EINVAL;
    c->hold_next = tile >= 0 ? tile + 1 : 0;
    return TPX_OK;
}

int tpx_tuning(tpx_ctx *c, int32_t *tile_geometry, double *ms_per_mpacket) {
    if (!c || !tile_geometry) return TPX_EINVAL;
    if (c->cfg.tile_geometry != TPX_TILE_DEFAULT) *tile_geometry = c->cfg.tile_geometry;
    else *tile_geometry = c->tune.fixed == tpxk::GEO_T2048 ? TPX_TILE_2048 : (c->tune.fixed ? TPX_TILE_4096 : TPX_TILE_DEFAULT);
    if (ms_per_mpacket) {
        ms_per_mpacket[0] = c->tune.done[tpxk::GEO_T4096 - 1] ? c->tune.best[tpxk::GEO_T4096 - 1] : 0.0;
        ms_per_mpacket[1] = c->tune.done[tpxk::GEO_T2048 - 1] ? c->tune.best[tpxk::GEO_T2048 - 1] : 0.0;
    }
    return TPX_OK;
}

int tpx_set_state(tpx_ctx *c, const tpx_stream_state *st) {
    if (!c) return TPX_EINVAL;
    tpxk::GAgg &g = c->h_state;
    std::memset(&g, 0, sizeof g);
    if (st) {
        if (st->pixels < 0 || st->triggers < 0) return TPX_EINVAL;
        g.pix.n = st->pixels;
        g.pix.first = st->pix_last_raw;
        g.pix.last = st->pix_last_raw;
        g.pix.sum = st->pix_wraps;
        g.tdc.n = st->triggers;
        g.tdc.first = st->tdc_last_raw;
        g.tdc.last = st->tdc_last_raw;
        g.tdc.sum = st->tdc_wraps;
    }
    if (cudaMemcpyAsync(&c->d_state[c->cur], &g, sizeof g, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return TPX_ECUDA;
    if (ckr(cudaStreamSynchronize(c->stream))) return TPX_ECUDA;
    c->state_once = true;
    return TPX_OK;
}

int tpx_get_state(tpx_ctx *c, tpx_stream_state *st) {
    if (!c || !st) return TPX_EINVAL;
    tpxk::GAgg &g = c->h_state;
    if (cudaMemcpyAsync(&g, &c->d_state[c->cur], sizeof g, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        return TPX_ECUDA;
    if (ckr(cudaStreamSynchronize(c->stream))) return TPX_ECUDA;
    st->pixels = g.pix.n;
    st->pix_last_raw = g.pix.last;
    st->pix_wraps = g.pix.sum;
    st->triggers = g.tdc.n;
    st->tdc_last_raw = g.tdc.last;
    st->tdc_wraps = g.tdc.sum;
    return TPX_OK;
}

const char *tpx_strerror(int code) {
    switch (code) {
        case TPX_OK: return "ok";
        case TPX_EINVAL: return "invalid argument or configuration";
        case TPX_ENOMEM: return "device memory allocation failed";
        case TPX_EOVERFLOW: return "output buffer too small (required count written)";
        case TPX_ECORRUPT: return "corrupt stream (unknown header in strict mode, or decreasing triggers)";
        case TPX_EAGAIN: return "admission refused";
        case TPX_ETIMEOUT: return "host wait timed out";
        case TPX_EDEVTIMEOUT: return "bounded device wait ran out";
        case TPX_ECUDA: return "CUDA runtime error";
        case TPX_EUNSUPPORTED: return "input outside the fused path's on-chip capacity";
        default: return "unknown status";
    }
}

const char *tpx_version(void) { return "tpx-gb300 0.1 (sm_103a)"; }

}  // extern "C"
