// tpx_fused.cuh -- the fused single-pass TPX3 path for sm_103a.
//
// One persistent kernel reads the packet stream once.  Each CTA repeatedly
// claims the next tile of T packets (dynamic, in stream order), and:
//   1. loads the tile into shared memory; the exact state of the two ToA
//      unwrap chains (pixels, TDCs; Sec. IV.A: a step down by more than the
//      threshold adds a wrap, a step up by more removes one) at the tile start
//      comes from the unwrap pre-pass, which scans the tiles' chain
//      aggregates before the kernel starts (the chains are associative);
//   2. owns the laser shots whose TDC packet lies in the tile, reading past
//      the tile end up to the next TDC packet (its "range");
//   3. unwraps every packet of the range, bins each pixel to the most recent
//      trigger in time, applies the <= tof_max background cut and the optional
//      timewalk table (Sec. IV.B-C);
//   4. hashes kept pixels by (shot, x, y) and visits each adjacent pair once
//      under the box rule of Sec. V.A; a pair updates the local-maximum flags
//      (Sec. V.B, equal ToT resolved towards the later pixel) and, in CC mode,
//      a lock-free union-find whose root is the pair-wise minimum of the key
//      (corrected time, stream position) -- so each component's root is its
//      earliest pixel in sorted order without sorting the pixels;
//   5. accumulates exact integer sums per cluster in shared memory (Sec. V.C)
//      and writes per-packet labels and, after a second look-back over
//      cluster counts, the cluster records in ascending label order.
// Pixels whose trigger cannot be decided inside the range, and ranges that
// exceed the on-chip capacities, raise a status bit instead (the kernel never
// traps).  All device waits are bounded.
#pragma once

#include <cstdint>

#include "tpx.h"

namespace tpxk {

constexpr int64_t kPixPeriod = 1LL << 34;
constexpr int64_t kTdcPeriod = 1LL << 36;
constexpr int kTofBias = 32768;            // tof_c + bias >= 1 for int16 timewalk shifts
constexpr int kBatchRing = 4;              // staged tiles per CTA of a batch launch (records, triggers)

// status bits latched in Ctl::status
enum : unsigned {
    ST_CORRUPT = 1u << 0,      // unknown header (reported only when strict)
    ST_TRIG_ORDER = 1u << 1,   // trigger times decrease
    ST_CAPACITY = 1u << 2,     // a range exceeds shared-memory capacity
    ST_EXCEPTION = 1u << 3,    // a pixel's trigger lies outside its range
    ST_CLUSTER_CAP = 1u << 4,  // caller cluster buffer too small
    ST_TRIG_CAP = 1u << 5,     // caller trigger buffer too small
    ST_DEVTIMEOUT = 1u << 6,   // a look-back wait ran out
    ST_RUN_REDO = 1u << 7,     // batch: a run needs the general path (see run_failed)
    ST_BOUNDS = 1u << 8,       // checked build: an index outside its array (the access was skipped)
    ST_BIG = 1u << 9,          // a tile's range exceeds the capacity: the big-range path (never reported)
};

enum CounterIdx {
    C_PACKETS = 0, C_PIXELS, C_TDCS, C_CORRUPT, C_DROP_PRE, C_DROP_BG, C_KEPT, C_CLUSTERS, C_PEAKS,
    C_NUM
};

struct Ctl {                     // per-launch control block, cleared before each launch
    unsigned int tile_counter;
    unsigned int status;
    unsigned long long counters[C_NUM];
};

// one unwrap chain over a stretch of the stream (64-bit form)
struct GChain { long long n, first, last, sum; };
struct GAgg { GChain pix, tdc; };            // 64 bytes

// per-tile records: the unwrap pre-pass's tile aggregates and states, and
// the record-count look-back chain
struct TileScratch {
    GAgg *agg;               // [tiles] unwrap-chain aggregate of each tile
    GAgg *pre;               // [tiles] unwrap state before each tile
    GAgg *blk;               // unwrap_prepass_scratch_bytes(tiles): block totals of the scan
    unsigned int *cflags;    // [tiles] cluster-count chain: (seq<<2)|1 count, |2 inclusive prefix
    long long *cagg;         // [tiles]
    long long *cpre;         // [tiles]
};

// a batch of independent runs in one launch: the tile queue and per-run
// outputs (all device memory)
struct BatchTable {
    const int *tile_run;          // [tiles] run of each tile
    const long long *run_tile0;   // [runs] first tile of each run
    const long long *run_off;     // [runs + 1] packet offsets of the runs
    long long *run_rec_off;       // [runs + 1] out: record offsets
    long long *run_trig_off;      // [runs + 1] out: trigger offsets
    unsigned *run_failed;         // [runs] out: 1 = a range the tiles cannot hold
    long long *tcagg, *tcpre;     // [tiles] trigger-count chain
    long long *tstage;            // [grid * kBatchRing * tile packets] trigger staging
    long long n_runs;
};

struct Params {
    const uint64_t *pk;
    long long n;
    long long idx_base;
    long long *labels;
    int *labels32;            // TPX_FLAG_LABELS32: labels minus lab32_base, as int32 (labels NULL)
    int l2_prefetch;          // the packets are in device memory: prefetch the next tile into L2
    int rec64;                // TPX_FLAG_RECORDS64: clusters holds 64-byte records (no x, y, tof)
    long long lab32_base;
    uint8_t *is_peak;
    tpx_record *clusters;
    long long cl_cap;
    long long *n_clusters;
    long long *trig;
    long long trig_cap;
    long long *n_trig;
    const int16_t *lut;
    int rx, ry, dt, strict;
    long long tof_max;
    long long thr_pix, thr_tdc;
    long long n_tiles;
    unsigned int seq;
    TileScratch ts;
    Ctl *ctl;
    tpx_record *stage;       // per-CTA record staging (range-capacity records per
                             // CTA of the grid, kBatchRing slots of them in a batch,
                             // in label order), or NULL: inline offset look-back
    BatchTable bt;           // batch of runs (tile_run == NULL: one stream)
    long long hold;          // tile + 1 whose look-back flags stay unpublished (0: none): lets a
                             // test run its successors' bounded waits out (TPX_EDEVTIMEOUT)
    unsigned char *big;      // big-range scratch, fused_big_scratch_bytes per CTA of the grid (NULL:
                             // a range past the capacity sends its run to the general path)
    const GAgg *E0;          // unwrap state before the call (NULL: stream start)
    GAgg *state_out;         // state after the call, written by the pre-pass (or NULL)
};

}  // namespace tpxk

// launch entry points (defined in tpx_fused.cu)
namespace tpxk {
// tile geometries of the fused kernel
enum : int { GEO_T4096 = 1, GEO_T2048 = 2 };
int fused_tile_packets(int geo);
int fused_smem_bytes(int geo);
int fused_threads(int geo);
int fused_range_capacity(int geo);
int fused_ctas_per_sm(int geo);
// global scratch of the big-range path per CTA (batches in CC mode)
size_t fused_big_scratch_bytes(int geo);
// the unwrap pre-pass (tpx_prepass.cu): ts.pre[tile] = the state before each
// tile, *state_out = the state after the call; adds the pixel, TDC and
// corrupt-packet counters. launch_fused runs it before the fused kernel.
size_t unwrap_prepass_scratch_bytes(long long n_tiles);
cudaError_t launch_unwrap_prepass(const Params &p, int T, int grid, cudaStream_t s);
// `mid`, if given, is recorded on `s` between the pre-pass and the fused kernel
cudaError_t launch_fused(const Params &p, int mode, int geo, int grid, cudaStream_t s, cudaEvent_t mid = nullptr);
}  // namespace tpxk
