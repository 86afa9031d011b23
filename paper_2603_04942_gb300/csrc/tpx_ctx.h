// tpx_ctx.h -- the context behind the opaque tpx_ctx handle (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "tpx.h"
#include "tpx_fused.cuh"

struct tpx_ctx {
    tpx_config cfg;
    cudaStream_t stream;
    int device;
    int num_sms;
    int geo;                  // fused-kernel tile geometry (tpxk::GEO_*), when fixed by the config
    // tile-geometry autotuner (TPX_TILE_DEFAULT): the first large calls
    // alternate the geometries, timed with events; the faster one is kept
    struct Tune {
        int fixed;            // chosen tpxk::GEO_*, 0 while sampling
        int issued[2];        // samples launched per geometry (index geo - 1)
        int done[2];          // samples timed
        double best[2];       // lowest ms per million packets seen
        int head, tail;       // ring of launched, not yet timed samples
        struct Sample { cudaEvent_t a, b; int geo; int64_t n; bool failed; } ring[8];
    } tune;
    // kernel timing (tpx_kernel_timing): events before the pre-pass, between
    // it and the fused kernel, and after, for each fused launch
    struct KTime {
        static constexpr int kRing = 32;
        bool on;
        int head, tail;           // recorded, not yet collected
        cudaEvent_t ev[kRing][3];
        double pre_ms, fused_ms;
        int64_t launches;
    } kt;
    int64_t max_packets;
    int64_t max_tiles;
    unsigned seq;
    tpxk::TileScratch ts;
    void *scratch;            // one allocation for all tile records
    tpx_record *stage;        // fused-kernel record staging (inside scratch)
    int64_t stage_records;    // its capacity
    tpxk::Ctl *ctl;           // device control block
    tpxk::Ctl *h_ctl;         // pinned host copy
    unsigned *d_sticky;       // failure bits of calls that were not synchronised
    bool synced;              // tpx_sync ran after the last call
    int64_t redone_early;     // the last call was already redone (autotuner sample)
    int64_t hold_next;        // tile + 1 the next tpx_process call holds back (tpx_debug_hold_tile)
    // device staging for tpx_process_host
    uint64_t *st_pk;
    int64_t *st_labels;
    uint8_t *st_peak;
    int64_t st_n, st_labels_cap, st_peak_cap, st_counts_cap;
    tpx_record *st_cl;
    int64_t st_cl_cap;
    int64_t *st_trig;
    int64_t st_trig_cap;
    int64_t *st_counts;       // [2]: n_clusters, n_trig
    // tpx_process_host on large inputs: pieces cut at trigger packets, their
    // copies in and out overlapping the fused kernel of the neighbouring pieces
    struct Pipe {
        static constexpr int kMax = 16;
        cudaStream_t s_in, s_out;
        cudaEvent_t ev_in[kMax], ev_done[kMax], ev_out[kMax];
        struct Slot { int64_t counts[2]; tpxk::Ctl ctl; } *h_slot;   // pinned, [kMax]
        int64_t *d_counts;        // [kMax][2]
        uint64_t *pk[2];
        int64_t pk_cap;
        tpx_record *cl[2];
        int64_t cl_cap;
        int64_t *trig[2];
        int64_t trig_cap;
        bool ready;
    } pipe;
    // unwrap state before / after a call, on the device (ping-pong)
    tpxk::GAgg *d_state;      // [2]
    int cur;                  // d_state[cur]: state for the next call
    bool state_once;          // tpx_set_state was called for the next call
    bool packets_on_host;     // the next calls read mapped host packets (no L2 prefetch of them)
    bool lab32_outer;         // int32 labels of the next calls are relative to lab32_base
    int64_t lab32_base;       // (the pieces of one pipelined host call), not to their own base
    tpxk::GAgg h_state;       // host staging for tpx_set_state / tpx_get_state
    // scratch of the general (global-memory) path, grown on demand
    void *g_mem;
    size_t g_bytes;
    // the last tpx_process call, kept so tpx_sync can redo it exactly with the
    // general path when the fused kernel reports an input it cannot hold
    struct {
        bool valid;
        const uint64_t *pk;
        int64_t n, base;
        int64_t *labels;
        bool lab32;               // labels are int32, minus lab32_base (TPX_FLAG_LABELS32)
        int64_t lab32_base;
        uint8_t *is_peak;
        tpx_record *cl;
        int64_t cl_cap;
        int64_t *n_cl;
        int64_t *trig;
        int64_t trig_cap;
        int64_t *n_trig;
        const tpxk::GAgg *E0;
        tpxk::GAgg *state_out;
    } last;
    // batches of runs (tpx_process_batch): tile queue, run tables, their own
    // tile records and trigger staging, grown on demand; the last batch call
    struct Batch {
        void *dev;
        size_t dev_bytes;
        int64_t *h_tab;           // pinned: run offsets, run first tiles, tile runs
        size_t h_bytes;
        cudaEvent_t tab_copied;   // the tables' upload has run: the host copy may change
        tpxk::TileScratch ts;
        tpxk::BatchTable bt;
        bool last;                // the last call on the context was a batch
        const uint64_t *pk;
        int64_t n_runs;
        int64_t *labels;
        uint8_t *is_peak;
        tpx_record *cl;
        int64_t cl_cap;
        int64_t *n_cl;
        int64_t *trig;
        int64_t trig_cap;
        int64_t *n_trig;
        int64_t redone;           // runs redone by the last tpx_sync
        const int64_t *h_off;     // run offsets of the last batch call (its host table)
        // calls captured into a CUDA graph get tables of their own (the graph
        // reads them at every replay); freed with the context
        struct Owned { void *dev; void *host; Owned *next; } *graph_owned;
    } batch;
};

// state for the next call and where it leaves its final state (advances the
// ping-pong; tpx_runtime.cu)
void take_state(tpx_ctx *c, const tpxk::GAgg **E0, tpxk::GAgg **out);

// general (global-memory) path, tpx_general.cu
namespace tpxg {
// grow the context's general scratch to at least `bytes` (synchronises)
int reserve(tpx_ctx *c, size_t bytes);
// exact redo of the last tpx_process call with the general path; returns
// the status of the redone call
int redo_last(tpx_ctx *c);
// exact redo of the runs of the last batch call that the tiles could not
// hold, spliced into the call's outputs; *n_redone receives their number
int redo_batch(tpx_ctx *c, int64_t *n_redone);
int decode_impl(tpx_ctx *c, const uint64_t *pk, int64_t n, int64_t base, const tpx_hits &h, int64_t cap,
                int64_t *d_n_hits, int64_t *trig, int64_t trig_cap, int64_t *d_n_trig, bool clear_ctl,
                const tpxk::GAgg *E0, tpxk::GAgg *state_out, long long *trig_pos, long long **t_all_out);
int cluster_impl(tpx_ctx *c, const tpx_hits &h, int64_t n, int64_t *labels, uint8_t *is_peak);
// sort + cluster + (when out != NULL) records of the hits with shot < shot_limit;
// shot_span >= 0 bounds max - min shot of the hits (skips a host round trip)
int cluster_all(tpx_ctx *c, const tpx_hits &h, int64_t n, int64_t *labels, uint8_t *is_peak, long long shot_limit,
                long long shot_span, tpx_record *out, int64_t cap, int64_t *d_n_clusters);
// general-path scratch for n packets (decode) and n hits (cluster_all)
size_t decode_bytes(long long n);
size_t cluster_bytes(long long n);
int centroid_impl(tpx_ctx *c, const tpx_hits &h, const int64_t *labels, const uint8_t *is_peak, int64_t n,
                  tpx_record *out, int64_t cap, int64_t *d_n_clusters);
}  // namespace tpxg

// the refiners' shared loss and Adam step (tpx_refine.cu)
int tpxr_loss(cudaStream_t s, const float *out, const float *y, int n, float w_off, float *dout, float *loss);
int tpxr_adam(cudaStream_t s, float *p, const float *g, float *m, float *v, long long n, float lr, long long step);
