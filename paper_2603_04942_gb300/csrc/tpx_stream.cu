// tpx_stream.cu -- streaming: acquisition chunks in, closed shots' records out.
//
// A submit takes a free result slot and queues the chunk; it returns at once.
// The stream's worker thread processes the queued chunks in order: the held
// (open) packets plus the chunk are decoded by the general path starting from
// the unwrap state at the held part's start (device-resident); the hits are
// sorted and clustered, and records are written for the shots that closed
// (all but the last `hold_triggers`); the unwrap state at the first open
// shot's trigger packet is computed on the device and the open part is moved
// to the front of the other pending buffer for the next chunk. Two host
// round trips per chunk inside the worker: one for the counts after decoding,
// one for the record count. A poll waits for its chunk's slot. Independent
// streams run on their own CUDA streams and workers, so chunks of different
// acquisitions overlap on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "tpx.h"
#include "tpx_common.cuh"
#include "tpx_ctx.h"
#include "tpx_fused.cuh"


// a failed CUDA call: true; with TPX_DEBUG set in the environment its error
// is printed to stderr
static inline bool cks(cudaError_t e, int line = __builtin_LINE()) {
    if (e == cudaSuccess) return false;
    if (std::getenv("TPX_DEBUG")) std::fprintf(stderr, "tpx_stream.cu:%d: %s\n", line, cudaGetErrorString(e));
    return true;
}

namespace {

using Clock = std::chrono::steady_clock;

std::mutex g_budget_mu;
int64_t g_budget_used = 0;

struct Slot {
    bool busy = false;              // holds a queued, running or unpolled chunk
    bool ready = false;             // the worker is done with it (status in rc)
    int rc = 0;
    uint64_t ticket = 0;
    cudaEvent_t done = nullptr;
    tpx_record *h_cl = nullptr;
    int64_t cap_cl = 0;
    int64_t *h_trig = nullptr;
    int64_t cap_trig = 0;
    int64_t n_cl = 0, first_shot = 0, n_shots = 0, processed = 0;
    int32_t status = 0;
    Clock::time_point t_submit;
};

struct Job {                        // a queued submit or finish
    Slot *sl;
    const uint64_t *h;
    int64_t n;
    bool finishing;
};

struct Probe {                      // k_state_at scratch
    unsigned long long last_pix, last_tdc, n_pix, n_tdc;
};

}  // namespace

struct tpx_stream {
    tpx_stream_config cfg;
    tpx_ctx *ctx = nullptr;
    cudaStream_t s = nullptr;
    uint64_t *pend[2] = {nullptr, nullptr};
    int cur = 0;
    int64_t cap = 0;                // pending capacity (held + chunk)
    int64_t held = 0;
    int64_t index_base = 0;         // stream index of the first pending packet
    int64_t trig_base = 0;          // global index of the first pending trigger
    tpxk::GAgg *st[3] = {nullptr, nullptr, nullptr};   // state at pending start, scratch, next
    tpx_hits h{};
    void *dev_mem = nullptr;
    int64_t *d_counts = nullptr;    // n_hits, n_trig, n_cl, emit, p, status
    int64_t *d_trig = nullptr, *d_trig_pos = nullptr;
    tpx_record *d_cl = nullptr;
    Probe *d_probe = nullptr;
    int64_t *h_counts = nullptr;    // pinned copy of d_counts
    std::vector<Slot> slots;
    uint64_t next_ticket = 1;
    int64_t bytes = 0;
    bool finished = false;
    // the worker: queued chunks, processed in order on the stream's CUDA stream
    int device = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;     // a job was queued, a job finished, or stop
    std::deque<Job> q;
    bool busy_worker = false;       // processing a job now
    bool stop = false;
    // the same facts without the lock, for the short spins that keep a
    // thread wake-up out of a chunk's latency
    std::atomic<int> queued{0};
    std::atomic<uint64_t> done_ticket_max{0};   // tickets complete in order: every one up to this
};

namespace tpxs {

using namespace tpxk;
constexpr int BT = 256;

__global__ void k_probe(const uint64_t *pk, long long p, Probe *pr) {
    unsigned long long lp = 0, lt = 0, np = 0, nt = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < p; q += (long long)gridDim.x * blockDim.x) {
        const unsigned h = (unsigned)(pk[q] >> 60);
        if (h == 0xBu) { lp = max(lp, (unsigned long long)q + 1); ++np; }
        else if (h == 0x6u) { lt = max(lt, (unsigned long long)q + 1); ++nt; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lp = max(lp, __shfl_down_sync(0xffffffffu, lp, o));
        lt = max(lt, __shfl_down_sync(0xffffffffu, lt, o));
        np += __shfl_down_sync(0xffffffffu, np, o);
        nt += __shfl_down_sync(0xffffffffu, nt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (lp) atomicMax(&pr->last_pix, lp);
        if (lt) atomicMax(&pr->last_tdc, lt);
        if (np) atomicAdd(&pr->n_pix, np);
        if (nt) atomicAdd(&pr->n_tdc, nt);
    }
}

// unwrap state before position p of the pending buffer (t_all from the decode)
__global__ void k_state_at(const uint64_t *pk, const long long *t_all, const Probe *pr, const GAgg *E0, GAgg *out) {
    GAgg g = *E0;
    if (pr->last_pix) {
        const long long q = (long long)pr->last_pix - 1;
        const long long raw = pix_raw(pk[q]);
        g.pix.n += (long long)pr->n_pix;
        g.pix.last = raw;
        g.pix.first = raw;
        g.pix.sum = (t_all[q] - raw) / kPixPeriod;
    }
    if (pr->last_tdc) {
        const long long q = (long long)pr->last_tdc - 1;
        const long long raw = tdc_raw(pk[q]);
        g.tdc.n += (long long)pr->n_tdc;
        g.tdc.last = raw;
        g.tdc.first = raw;
        g.tdc.sum = (t_all[q] - raw) / kTdcPeriod;
    }
    *out = g;
}

// closed shots and where the open part starts: emit = shots to close,
// p = position of the first open shot's trigger packet (P when none is open)
__global__ void k_plan(long long *counts, const long long *trig_pos, long long hold, int finishing, long long P,
                       const unsigned *status) {
    const long long ntr = counts[1];
    const long long emit = finishing ? ntr : (ntr > hold ? ntr - hold : 0);
    counts[3] = emit;
    counts[4] = emit < ntr ? trig_pos[emit] : (finishing ? P : 0);
    counts[5] = (long long)*status;
}

inline unsigned gridn(long long n) {
    long long g = (n + BT - 1) / BT;
    if (g < 1) g = 1;
    if (g > 152 * 8) g = 152 * 8;
    return (unsigned)g;
}
inline size_t al(size_t b) { return (b + 255) & ~size_t(255); }

// grows a slot's pinned result buffers geometrically (freeing pinned memory
// synchronises the device, so growth must stay rare)
int grow_pinned(Slot &sl, int64_t ncl, int64_t ntr) {
    if (ncl > sl.cap_cl) ncl = std::max<int64_t>(ncl, 2 * sl.cap_cl);
    if (ntr > sl.cap_trig) ntr = std::max<int64_t>(ntr, 2 * sl.cap_trig);
    if (ncl > sl.cap_cl) {
        if (sl.h_cl) cudaFreeHost(sl.h_cl);
        sl.h_cl = nullptr;
        sl.cap_cl = 0;
        if (cudaMallocHost(&sl.h_cl, sizeof(tpx_record) * (size_t)ncl) != cudaSuccess) return TPX_ENOMEM;
        sl.cap_cl = ncl;
    }
    if (ntr > sl.cap_trig) {
        if (sl.h_trig) cudaFreeHost(sl.h_trig);
        sl.h_trig = nullptr;
        sl.cap_trig = 0;
        if (cudaMallocHost(&sl.h_trig, sizeof(int64_t) * (size_t)ntr) != cudaSuccess) return TPX_ENOMEM;
        sl.cap_trig = ntr;
    }
    return TPX_OK;
}

// one chunk, in the worker thread (the slot and ticket were taken at submit)
int process_job(tpx_stream *S, Slot *sl, const uint64_t *h_chunk, int64_t n, bool finishing) {
    cudaStream_t s = S->s;
    tpx_ctx *c = S->ctx;
    int rc = TPX_OK;
    const int64_t P = S->held + n;
    if (P > S->cap) return TPX_EOVERFLOW;
    uint64_t *pk = S->pend[S->cur];
    if (n > 0 && cudaMemcpyAsync(pk + S->held, h_chunk, sizeof(uint64_t) * (size_t)n, cudaMemcpyHostToDevice, s) !=
                     cudaSuccess)
        return TPX_ECUDA;
    long long *t_all = nullptr;
    long long *cnt_d = reinterpret_cast<long long *>(S->d_counts);
    rc = tpxg::decode_impl(c, pk, P, S->index_base, S->h, S->cap, S->d_counts, S->d_trig, S->cap, S->d_counts + 1,
                           true, S->st[0], S->st[1], reinterpret_cast<long long *>(S->d_trig_pos), &t_all);
    if (rc) return rc;
    k_plan<<<1, 1, 0, s>>>(cnt_d, reinterpret_cast<long long *>(S->d_trig_pos), S->cfg.hold_triggers, finishing ? 1 : 0,
                           P, &c->ctl->status);
    int64_t *hc = S->h_counts;
    if (cudaMemcpyAsync(hc, S->d_counts, 6 * sizeof(int64_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return TPX_ECUDA;
    if (cks(cudaStreamSynchronize(s))) return TPX_ECUDA;
    const int64_t n_hits = hc[0], ntr = hc[1], emit = hc[3], p = hc[4];
    const unsigned status = (unsigned)hc[5];
    if (status & ST_TRIG_ORDER) return TPX_ECORRUPT;
    if (status & (ST_TRIG_CAP | ST_CLUSTER_CAP)) return TPX_EOVERFLOW;
    // unwrap state at p, while the decode's per-packet times are still alive
    if (p == P) {
        if (cks(cudaMemcpyAsync(S->st[2], S->st[1], sizeof(GAgg), cudaMemcpyDeviceToDevice, s))) return TPX_ECUDA;
    } else if (p > 0) {
        if (cks(cudaMemsetAsync(S->d_probe, 0, sizeof(Probe), s))) return TPX_ECUDA;
        k_probe<<<gridn(p), BT, 0, s>>>(pk, p, S->d_probe);
        k_state_at<<<1, 1, 0, s>>>(pk, t_all, S->d_probe, S->st[0], S->st[2]);
    } else {
        if (cks(cudaMemcpyAsync(S->st[2], S->st[0], sizeof(GAgg), cudaMemcpyDeviceToDevice, s))) return TPX_ECUDA;
    }
    // cluster every hit; records only for the closed shots (shot < limit)
    int64_t n_cl = 0;
    if (emit > 0 && n_hits > 0) {
        rc = tpxg::cluster_all(c, S->h, n_hits, nullptr, nullptr, S->trig_base + emit, ntr, S->d_cl, S->cap,
                               S->d_counts + 2);
        if (rc) return rc;
        if (cks(cudaMemcpyAsync(&hc[2], S->d_counts + 2, 8, cudaMemcpyDeviceToHost, s))) return TPX_ECUDA;
        if (cks(cudaStreamSynchronize(s))) return TPX_ECUDA;
        n_cl = hc[2];
    }
    rc = grow_pinned(*sl, n_cl > 0 ? n_cl : 1, emit > 0 ? emit : 1);
    if (rc) return rc;
    if (n_cl > 0 && cudaMemcpyAsync(sl->h_cl, S->d_cl, sizeof(tpx_record) * (size_t)n_cl, cudaMemcpyDeviceToHost, s) !=
                        cudaSuccess)
        return TPX_ECUDA;
    if (emit > 0 && cudaMemcpyAsync(sl->h_trig, S->d_trig, sizeof(int64_t) * (size_t)emit, cudaMemcpyDeviceToHost, s) !=
                        cudaSuccess)
        return TPX_ECUDA;
    // move the open part to the front of the other pending buffer
    const int64_t rest = P - p;
    if (rest > S->cfg.max_hold_packets && !finishing) return TPX_EOVERFLOW;
    if (rest > 0 && cudaMemcpyAsync(S->pend[S->cur ^ 1], pk + p, sizeof(uint64_t) * (size_t)rest,
                                    cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return TPX_ECUDA;
    tpxk::GAgg *t = S->st[0];
    S->st[0] = S->st[2];
    S->st[2] = t;
    S->cur ^= 1;
    S->held = rest;
    S->index_base += p;
    sl->first_shot = S->trig_base;
    sl->n_shots = emit;
    S->trig_base += emit;
    sl->n_cl = n_cl;
    sl->processed = P;
    sl->status = 0;
    if (cks(cudaEventRecord(sl->done, s))) return TPX_ECUDA;
    return TPX_OK;
}

// spins before sleeping: about 0.2 ms of polling, then the condition variable
constexpr auto kSpinFor = std::chrono::microseconds(200);

void worker_loop(tpx_stream *S) {
    cudaSetDevice(S->device);
    for (;;) {
        Job j;
        {
            const auto t0 = Clock::now();
            while (S->queued.load(std::memory_order_acquire) == 0 && Clock::now() - t0 < kSpinFor)
                std::this_thread::yield();
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] { return S->stop || !S->q.empty(); });
            if (S->q.empty()) return;   // stop, nothing left
            j = S->q.front();
            S->q.pop_front();
            S->queued.fetch_sub(1, std::memory_order_acq_rel);
            S->busy_worker = true;
        }
        const int rc = process_job(S, j.sl, j.h, j.n, j.finishing);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            j.sl->rc = rc;
            j.sl->ready = true;
            S->busy_worker = false;
            S->done_ticket_max.store(j.sl->ticket, std::memory_order_release);
        }
        S->cv.notify_all();
    }
}

// queue a chunk (or the finish) into a free slot
int enqueue(tpx_stream *S, const uint64_t *h, int64_t n, bool finishing, uint64_t *ticket) {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->finished) return TPX_EINVAL;
    Slot *sl = nullptr;
    for (auto &x : S->slots)
        if (!x.busy) { sl = &x; break; }
    if (!sl) return TPX_EAGAIN;
    sl->busy = true;
    sl->ready = false;
    sl->rc = 0;
    sl->ticket = S->next_ticket++;
    sl->t_submit = Clock::now();
    S->q.push_back(Job{sl, h, n, finishing});
    S->queued.fetch_add(1, std::memory_order_acq_rel);
    if (finishing) S->finished = true;
    *ticket = sl->ticket;
    S->cv.notify_all();
    return TPX_OK;
}

// wait until the worker has nothing queued or running
void drain(tpx_stream *S) {
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv.wait(lk, [&] { return S->q.empty() && !S->busy_worker; });
}

}  // namespace tpxs

extern "C" {

using tpxs::al;

int tpx_stream_create(tpx_stream **out, const tpx_stream_config *cfg, void *cuda_stream) {
    if (!out || !cfg) return TPX_EINVAL;
    *out = nullptr;
    if (cfg->max_chunk_packets <= 0 || cfg->max_hold_packets < 0 || cfg->hold_triggers < 1 || cfg->slots < 1)
        return TPX_EINVAL;
    if (cfg->cfg.flags & (TPX_FLAG_LABELS32 | TPX_FLAG_RECORDS64)) return TPX_EINVAL;   // results are 88-byte records
    tpx_stream *S = new (std::nothrow) tpx_stream;
    if (!S) return TPX_ENOMEM;
    S->cfg = *cfg;
    S->cfg.cfg.chain = 0;
    S->s = static_cast<cudaStream_t>(cuda_stream);
    S->cap = cfg->max_chunk_packets + cfg->max_hold_packets;
    const int64_t C = S->cap;
    // device memory: pending x2, hits, records, triggers, trigger positions,
    // states, counts; plus the general path's scratch in the context
    const size_t hit_b = al(8 * C) * 3 + al(4 * C) + al(2 * C) + 2 * al(C);
    const size_t b = 2 * al(8 * (size_t)C) + hit_b + al(sizeof(tpx_record) * C) + 2 * al(8 * C) +
                     3 * al(sizeof(tpxk::GAgg)) + al(sizeof(Probe)) + al(64);
    size_t general = tpxg::decode_bytes(C);
    if (tpxg::cluster_bytes(C) > general) general = tpxg::cluster_bytes(C);
    S->bytes = (int64_t)(b + general);
    {
        std::lock_guard<std::mutex> lk(g_budget_mu);
        if (cfg->hbm_budget_bytes > 0 && g_budget_used + S->bytes > cfg->hbm_budget_bytes) {
            delete S;
            return TPX_EAGAIN;
        }
        g_budget_used += S->bytes;
    }
    int rc = tpx_create(&S->ctx, &S->cfg.cfg, 0, cuda_stream);
    if (!rc) rc = tpxg::reserve(S->ctx, general);
    if (!rc && cudaMalloc(&S->dev_mem, b) != cudaSuccess) { cudaGetLastError(); rc = TPX_ENOMEM; }
    if (!rc && cudaMallocHost(&S->h_counts, 8 * sizeof(int64_t)) != cudaSuccess) { cudaGetLastError(); rc = TPX_ENOMEM; }
    if (rc) {
        if (S->dev_mem) cudaFree(S->dev_mem);
        if (S->ctx) tpx_destroy(S->ctx);
        std::lock_guard<std::mutex> lk(g_budget_mu);
        g_budget_used -= S->bytes;
        delete S;
        return rc;
    }
    char *m = static_cast<char *>(S->dev_mem);
    auto take = [&](size_t bytes) { char *r = m; m += al(bytes); return r; };
    S->pend[0] = reinterpret_cast<uint64_t *>(take(8 * C));
    S->pend[1] = reinterpret_cast<uint64_t *>(take(8 * C));
    S->h.index = reinterpret_cast<int64_t *>(take(8 * C));
    S->h.shot = reinterpret_cast<int64_t *>(take(8 * C));
    S->h.t = reinterpret_cast<int64_t *>(take(8 * C));
    S->h.tof = reinterpret_cast<int32_t *>(take(4 * C));
    S->h.tot = reinterpret_cast<uint16_t *>(take(2 * C));
    S->h.x = reinterpret_cast<uint8_t *>(take(C));
    S->h.y = reinterpret_cast<uint8_t *>(take(C));
    S->d_cl = reinterpret_cast<tpx_record *>(take(sizeof(tpx_record) * C));
    S->d_trig = reinterpret_cast<int64_t *>(take(8 * C));
    S->d_trig_pos = reinterpret_cast<int64_t *>(take(8 * C));
    for (int i = 0; i < 3; ++i) S->st[i] = reinterpret_cast<tpxk::GAgg *>(take(sizeof(tpxk::GAgg)));
    S->d_probe = reinterpret_cast<Probe *>(take(sizeof(Probe)));
    S->d_counts = reinterpret_cast<int64_t *>(take(64));
    cudaMemsetAsync(S->st[0], 0, sizeof(tpxk::GAgg), S->s);
    S->slots.resize((size_t)cfg->slots);
    for (auto &sl : S->slots)
        if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            tpxs::grow_pinned(sl, std::max<int64_t>(1024, C / 16), std::max<int64_t>(64, C / 4096))) {
            tpx_stream_destroy(S);
            return TPX_ECUDA;
        }
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        tpx_stream_destroy(S);
        return TPX_ECUDA;
    }
    try {
        S->worker = std::thread(tpxs::worker_loop, S);
    } catch (...) {
        tpx_stream_destroy(S);
        return TPX_ENOMEM;
    }
    *out = S;
    return TPX_OK;
}

int tpx_stream_submit(tpx_stream *S, const uint64_t *h_chunk, int64_t n, uint64_t *ticket) {
    if (!S || !ticket || n < 0 || (n > 0 && !h_chunk) || n > S->cfg.max_chunk_packets) return TPX_EINVAL;
    return tpxs::enqueue(S, h_chunk, n, false, ticket);
}

int tpx_stream_finish(tpx_stream *S, uint64_t *ticket) {
    if (!S || !ticket) return TPX_EINVAL;
    return tpxs::enqueue(S, nullptr, 0, true, ticket);
}

int tpx_stream_poll(tpx_stream *S, uint64_t ticket, tpx_stream_result *out, int32_t timeout_us) {
    if (!S || !out) return TPX_EINVAL;
    Slot *sl = nullptr;
    const auto start = Clock::now();
    // a short spin first (tickets complete in order)
    while (S->done_ticket_max.load(std::memory_order_acquire) < ticket && Clock::now() - start < tpxs::kSpinFor &&
           (timeout_us < 0 || Clock::now() - start < std::chrono::microseconds(timeout_us)))
        std::this_thread::yield();
    {
        std::unique_lock<std::mutex> lk(S->mu);
        for (auto &x : S->slots)
            if (x.busy && x.ticket == ticket) { sl = &x; break; }
        if (!sl) return TPX_EINVAL;
        auto done = [&] { return sl->ready; };
        if (timeout_us < 0) S->cv.wait(lk, done);
        else if (!S->cv.wait_for(lk, std::chrono::microseconds(timeout_us), done)) return TPX_ETIMEOUT;
        if (sl->rc) {   // the chunk failed: the slot is free again, the status goes to the caller
            const int rc = sl->rc;
            sl->busy = false;
            return rc;
        }
    }
    for (;;) {
        const cudaError_t e = cudaEventQuery(sl->done);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return TPX_ECUDA;
        if (timeout_us >= 0 &&
            std::chrono::duration_cast<std::chrono::microseconds>(Clock::now() - start).count() >= timeout_us)
            return TPX_ETIMEOUT;
    }
    out->ticket = ticket;
    out->status = sl->status;
    out->reserved = 0;
    out->first_shot = sl->first_shot;
    out->n_shots = sl->n_shots;
    out->trig_t = sl->h_trig;
    out->n_clusters = sl->n_cl;
    out->clusters = sl->h_cl;
    out->packets_processed = sl->processed;
    out->latency_us = std::chrono::duration<double, std::micro>(Clock::now() - sl->t_submit).count();
    std::lock_guard<std::mutex> lk(S->mu);
    sl->busy = false;
    return TPX_OK;
}

// checkpoint: a fixed header, then the held packets
namespace {
constexpr uint64_t kSnapMagic = 0x31504E5358505454ull;   // "TTPXSNP1", little-endian
struct SnapHeader {
    uint64_t magic;
    int64_t held, index_base, trig_base, hold_triggers, max_hold_packets;
    int64_t rx, ry, dt, mode, tof_max, wrap_pix, wrap_tdc;   // the processing configuration
    tpxk::GAgg state;          // unwrap state and trigger count where the held packets start
};
void snap_cfg(const tpx_stream *S, SnapHeader &h) {
    const tpx_config &c = S->cfg.cfg;
    h.rx = c.rx; h.ry = c.ry; h.dt = c.dt_ticks; h.mode = c.mode; h.tof_max = c.tof_max_ticks;
    h.wrap_pix = c.wrap_thr_pix_ticks; h.wrap_tdc = c.wrap_thr_tdc_ticks;
}
}  // namespace

int64_t tpx_stream_snapshot_bytes(tpx_stream *S) {
    if (!S) return 0;
    tpxs::drain(S);
    return (int64_t)sizeof(SnapHeader) + 8 * S->held;
}

int tpx_stream_snapshot(tpx_stream *S, void *h_buf, int64_t capacity, int64_t *written) {
    if (!S || !h_buf || !written) return TPX_EINVAL;
    tpxs::drain(S);
    const int64_t need = tpx_stream_snapshot_bytes(S);
    *written = need;
    if (capacity < need) return TPX_EOVERFLOW;
    if (S->finished) return TPX_EINVAL;
    SnapHeader hd;
    std::memset(&hd, 0, sizeof hd);
    hd.magic = kSnapMagic;
    hd.held = S->held;
    hd.index_base = S->index_base;
    hd.trig_base = S->trig_base;
    hd.hold_triggers = S->cfg.hold_triggers;
    hd.max_hold_packets = S->cfg.max_hold_packets;
    snap_cfg(S, hd);
    char *dst = static_cast<char *>(h_buf);
    // the carry is written by the stream's own kernels and copies: read it behind them
    if (cks(cudaMemcpyAsync(&hd.state, S->st[0], sizeof(tpxk::GAgg), cudaMemcpyDeviceToHost, S->s))) return TPX_ECUDA;
    if (S->held > 0 && cks(cudaMemcpyAsync(dst + sizeof hd, S->pend[S->cur], 8 * (size_t)S->held,
                                           cudaMemcpyDeviceToHost, S->s)))
        return TPX_ECUDA;
    if (cks(cudaStreamSynchronize(S->s))) return TPX_ECUDA;
    std::memcpy(dst, &hd, sizeof hd);
    return TPX_OK;
}

int tpx_stream_restore(tpx_stream *S, const void *h_buf, int64_t n) {
    if (!S || !h_buf || n < (int64_t)sizeof(SnapHeader)) return TPX_EINVAL;
    tpxs::drain(S);
    SnapHeader hd;
    std::memcpy(&hd, h_buf, sizeof hd);
    if (hd.magic != kSnapMagic || hd.held < 0 || n != (int64_t)sizeof hd + 8 * hd.held) return TPX_EINVAL;
    SnapHeader mine;
    std::memset(&mine, 0, sizeof mine);
    snap_cfg(S, mine);
    if (hd.hold_triggers != S->cfg.hold_triggers || hd.rx != mine.rx || hd.ry != mine.ry || hd.dt != mine.dt ||
        hd.mode != mine.mode || hd.tof_max != mine.tof_max || hd.wrap_pix != mine.wrap_pix ||
        hd.wrap_tdc != mine.wrap_tdc)
        return TPX_EINVAL;
    // only into a stream that has not started
    if (S->next_ticket != 1 || S->held != 0 || S->finished) return TPX_EINVAL;
    if (hd.held > S->cfg.max_hold_packets) return TPX_EOVERFLOW;
    const char *src = static_cast<const char *>(h_buf);
    if (cks(cudaMemcpyAsync(S->st[0], &hd.state, sizeof(tpxk::GAgg), cudaMemcpyHostToDevice, S->s))) return TPX_ECUDA;
    if (hd.held > 0 && cks(cudaMemcpyAsync(S->pend[S->cur], src + sizeof hd, 8 * (size_t)hd.held,
                                           cudaMemcpyHostToDevice, S->s)))
        return TPX_ECUDA;
    if (cks(cudaStreamSynchronize(S->s))) return TPX_ECUDA;
    S->held = hd.held;
    S->index_base = hd.index_base;
    S->trig_base = hd.trig_base;
    return TPX_OK;
}

int tpx_stream_destroy(tpx_stream *S) {
    if (!S) return TPX_EINVAL;
    if (S->worker.joinable()) {   // the queued chunks are processed first
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stop = true;
        }
        S->cv.notify_all();
        S->worker.join();
    }
    if (S->s) cudaStreamSynchronize(S->s);
    for (auto &sl : S->slots) {
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.h_cl) cudaFreeHost(sl.h_cl);
        if (sl.h_trig) cudaFreeHost(sl.h_trig);
    }
    if (S->dev_mem) cudaFree(S->dev_mem);
    if (S->h_counts) cudaFreeHost(S->h_counts);
    if (S->ctx) tpx_destroy(S->ctx);
    {
        std::lock_guard<std::mutex> lk(g_budget_mu);
        g_budget_used -= S->bytes;
    }
    delete S;
    return TPX_OK;
}

}  // extern "C"
