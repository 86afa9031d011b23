// tpx_noalloc.cu -- tpx_process_noalloc: the fused path for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they process data:
// real-time acquisition loops that must not block in the allocator (a
// cudaMalloc can wait for the device or trigger an implicit synchronisation),
// and hosts that hand the library a fixed memory budget up front and account
// for every byte. tpx_create allocates the look-back scratch of a context, so
// those callers cannot use tpx_process. This entry point runs the same fused
// kernel with its scratch taken from one fixed array in device memory that is
// part of the library image, so it allocates nothing.
//
// The call reads the device status back and synchronises its stream before
// it returns, so it must not be made on a stream that is being captured into
// a CUDA graph. It has no redo: where tpx_sync would hand an input the fused
// kernel cannot hold (a shot longer than a tile's range, a pixel whose trigger
// lies outside its range) to the general path, this call returns
// TPX_EUNSUPPORTED and its outputs are incomplete.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it (about 2.4 MB) until the process exits, and all calls on a
// device share it. It keeps the contents of the last call; the per-call
// control block is cleared before each launch, and the look-back flags carry
// a per-device sequence number so stale flags from an earlier call never
// match. Calls that overlap on the GPU (on different streams, or from several
// host threads without ordering) race on the array and must not be made.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "tpx.h"
#include "tpx_fused.cuh"

namespace {

constexpr int64_t kTile = 4096;                            // packets per tile of the fused kernel
constexpr int64_t kMaxTiles = TPX_NOALLOC_MAX_PACKETS / kTile;
constexpr int kMaxDevices = 64;

// layout of the fixed scratch (all members naturally aligned); blk holds what
// unwrap_prepass_scratch_bytes(kMaxTiles) asks for: (tiles / 1024 + 1) block
// totals and flags, plus 256 bytes
static_assert(sizeof(tpxk::GAgg) * (kMaxTiles / 1024 + 8) >=
                  (kMaxTiles / 1024 + 1) * (sizeof(tpxk::GAgg) + sizeof(int)) + 256,
              "pre-pass block totals");
struct NoAllocScratch {
    tpxk::Ctl ctl;
    tpxk::GAgg blk[kMaxTiles / 1024 + 8];   // the unwrap pre-pass's block totals and flags
    unsigned cflags[kMaxTiles];
    tpxk::GAgg agg[kMaxTiles];
    tpxk::GAgg pre[kMaxTiles];
    long long cagg[kMaxTiles];
    long long cpre[kMaxTiles];
};

std::mutex g_mu;
void *g_dev_ptr[kMaxDevices];        // device address of the array, per device
unsigned g_dev_seq[kMaxDevices];     // last look-back sequence number, per device

int noalloc_check_cfg(const tpx_config *c) {
    if (!c) return TPX_EINVAL;
    if (c->rx < 0 || c->ry < 0 || c->rx > 7 || c->ry > 7) return TPX_EINVAL;
    if (c->dt_ticks < 0) return TPX_EINVAL;
    if (c->mode != TPX_MODE_CC && c->mode != TPX_MODE_PAPER) return TPX_EINVAL;
    if (c->tof_max_ticks < 0 || c->tof_max_ticks > (1LL << 24) - 65537) return TPX_EINVAL;
    if (c->wrap_thr_pix_ticks <= 0 || c->wrap_thr_tdc_ticks <= 0) return TPX_EINVAL;
    return TPX_OK;
}

}  // namespace

// The fixed scratch itself. Host code must not pass this symbol to a kernel:
// on the host it names a host-side stand-in, not device memory. Its device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

extern "C" int tpx_process_noalloc(const tpx_config *cfg, void *cuda_stream, const uint64_t *d_packets,
                                   int64_t n, int64_t idx_base, int64_t *d_labels, uint8_t *d_is_peak,
                                   tpx_record *d_clusters, int64_t cl_cap, int64_t *d_n_clusters,
                                   int64_t *d_trig, int64_t trig_cap, int64_t *d_n_trig,
                                   tpx_counters *h_counters) {
    int rc = noalloc_check_cfg(cfg);
    if (rc) return rc;
    if (n < 0 || n > TPX_NOALLOC_MAX_PACKETS) return TPX_EINVAL;   // beyond the fixed scratch
    if (cl_cap < 0 || trig_cap < 0 || !d_n_clusters || !d_n_trig) return TPX_EINVAL;
    if (n > 0 && !d_packets) return TPX_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_packets) & 15) != 0) return TPX_EINVAL;
    if (cl_cap > 0 && !d_clusters) return TPX_EINVAL;
    if (trig_cap > 0 && !d_trig) return TPX_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TPX_ECUDA;
    NoAllocScratch *scr = nullptr;
    unsigned seq = 0;
    bool wrapped = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_dev_ptr[dev]) {
            // first call on this device (with it current): look up the array's
            // device address once; this must happen before any stream capture
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return TPX_ECUDA;
            }
            g_dev_ptr[dev] = ptr;
        }
        scr = static_cast<NoAllocScratch *>(g_dev_ptr[dev]);
        seq = (g_dev_seq[dev] + 1) & 0x3FFFFFFFu;
        if (seq == 0) { seq = 1; wrapped = true; }
        g_dev_seq[dev] = seq;
    }

    // clear what must start at zero: the control block (tile counter, status,
    // counters) and the two output counts; flags only when sequence numbers wrap
    if (cudaMemsetAsync(&scr->ctl, 0, sizeof(tpxk::Ctl), s) != cudaSuccess) return TPX_ECUDA;
    if (cudaMemsetAsync(d_n_clusters, 0, sizeof(int64_t), s) != cudaSuccess) return TPX_ECUDA;
    if (cudaMemsetAsync(d_n_trig, 0, sizeof(int64_t), s) != cudaSuccess) return TPX_ECUDA;
    if (wrapped) {
        if (cudaMemsetAsync(scr->cflags, 0, sizeof scr->cflags, s) != cudaSuccess) return TPX_ECUDA;
    }

    if (n > 0) {
        int num_sms = 0;
        if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TPX_ECUDA;
        tpxk::Params p;
        std::memset(&p, 0, sizeof p);
        p.pk = d_packets;
        p.n = n;
        p.idx_base = idx_base;
        const bool l32 = (cfg->flags & TPX_FLAG_LABELS32) != 0;
        p.labels = l32 ? nullptr : reinterpret_cast<long long *>(d_labels);
        p.labels32 = l32 ? reinterpret_cast<int *>(d_labels) : nullptr;
        p.lab32_base = idx_base;
        p.rec64 = (cfg->flags & TPX_FLAG_RECORDS64) ? 1 : 0;
        p.is_peak = d_is_peak;
        p.clusters = d_clusters;
        p.cl_cap = cl_cap;
        p.n_clusters = reinterpret_cast<long long *>(d_n_clusters);
        p.trig = reinterpret_cast<long long *>(d_trig);
        p.trig_cap = trig_cap;
        p.n_trig = reinterpret_cast<long long *>(d_n_trig);
        p.lut = cfg->d_timewalk_lut;
        p.rx = cfg->rx;
        p.ry = cfg->ry;
        p.dt = cfg->dt_ticks;
        p.strict = cfg->strict;
        p.tof_max = cfg->tof_max_ticks;
        p.thr_pix = cfg->wrap_thr_pix_ticks;
        p.thr_tdc = cfg->wrap_thr_tdc_ticks;
        p.n_tiles = (n + kTile - 1) / kTile;
        p.seq = seq;
        p.ts.blk = scr->blk;
        p.ts.cflags = scr->cflags;
        p.ts.agg = scr->agg;
        p.ts.pre = scr->pre;
        p.ts.cagg = scr->cagg;
        p.ts.cpre = scr->cpre;
        p.ctl = &scr->ctl;
        int64_t grid = num_sms < p.n_tiles ? num_sms : p.n_tiles;
        if (tpxk::launch_fused(p, cfg->mode, tpxk::GEO_T4096, (int)grid, s) != cudaSuccess) return TPX_ECUDA;
    }

    // wait for the call and report its device status (a copy to pageable host
    // memory: no allocation)
    tpxk::Ctl h;
    if (cudaMemcpyAsync(&h, &scr->ctl, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess) return TPX_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TPX_ECUDA;
    if (h_counters) {
        h_counters->packets = (int64_t)h.counters[tpxk::C_PACKETS];
        h_counters->pixels = (int64_t)h.counters[tpxk::C_PIXELS];
        h_counters->tdcs = (int64_t)h.counters[tpxk::C_TDCS];
        h_counters->corrupt = (int64_t)h.counters[tpxk::C_CORRUPT];
        h_counters->dropped_pre_trigger = (int64_t)h.counters[tpxk::C_DROP_PRE];
        h_counters->dropped_background = (int64_t)h.counters[tpxk::C_DROP_BG];
        h_counters->kept = (int64_t)h.counters[tpxk::C_KEPT];
        h_counters->clusters = (int64_t)h.counters[tpxk::C_CLUSTERS];
        h_counters->peaks = (int64_t)h.counters[tpxk::C_PEAKS];
        h_counters->status_bits = (int64_t)h.status;
        h_counters->redone = 0;
    }
    const unsigned st = h.status;
    if (st & tpxk::ST_DEVTIMEOUT) return TPX_EDEVTIMEOUT;
    if (st & tpxk::ST_TRIG_ORDER) return TPX_ECORRUPT;
    if (st & (tpxk::ST_CAPACITY | tpxk::ST_EXCEPTION)) return TPX_EUNSUPPORTED;
    if (cfg->strict && h.counters[tpxk::C_CORRUPT]) return TPX_ECORRUPT;
    if (st & (tpxk::ST_CLUSTER_CAP | tpxk::ST_TRIG_CAP)) return TPX_EOVERFLOW;
    return TPX_OK;
}

extern "C" int tpx_debug_noalloc_seq(uint32_t last_seq) {
    if (last_seq > 0x3FFFFFFFu) return TPX_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TPX_ECUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    g_dev_seq[dev] = last_seq;
    return TPX_OK;
}
