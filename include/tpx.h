/*
 * tpx.h -- C ABI of the GB300 TPX3 clustering / centroiding library (libtpx).
 *
 * The library turns a TimePix3-style packet stream (pixel events with X, Y,
 * ToA, ToT and TDC trigger events interleaved, paper Sec. III) into particle
 * hits: it decodes the 64-bit packets, unwraps ToA (Sec. IV.A), bins pixels
 * into laser shots by the most recent trigger and applies the background cut
 * (Sec. IV.B) and an optional timewalk table (Sec. IV.C, Eq. 1), groups pixels
 * by the box adjacency of Sec. V.A (connected components, or the paper's
 * per-maximum neighbourhoods), finds local maxima (Sec. V.B) and forms
 * ToT-weighted centroids (Sec. V.C).
 *
 * Conventions
 *   - Pointers named d_* are device pointers; h_* are host pointers.  The
 *     caller owns every buffer it passes in; the context owns its scratch.
 *     The fused path's scratch is sized by tpx_create / tpx_reserve, and
 *     tpx_process allocates nothing (tpx_process_noalloc not even scratch);
 *     the host-buffer, batch, general-path, streaming and refiner calls grow
 *     the context's scratch on demand and keep it for later calls.
 *   - Calls are asynchronous on the context's CUDA stream.  Device-side
 *     conditions (capacity, corrupt input, timeouts) are latched into a
 *     status word that tpx_sync() reads; the kernels never trap.
 *   - Every call returns TPX_OK (0) or a negative TPX_E* code.
 *   - Times are in ticks of 1.5625 ns (25/16 ns; 256 units of 25/4096 ns).
 *
 * Packet layout (project-defined, TPX3-style; the paper prints none):
 *   pixel : [63:60]=0xB [59:53]=dcol [52:47]=spix [46:44]=pix [43:30]=ToA
 *           [29:20]=ToT [19:16]=fToA [15:0]=spidr;
 *           x = 2*dcol + (pix>>2), y = 4*spix + (pix&3),
 *           raw time = ((spidr<<14 | ToA)*16 - fToA) mod 2^34 ticks
 *   TDC   : [63:60]=0x6 [43:9]=coarse (3.125 ns); raw time = 2*coarse mod 2^36
 *   any other header: counted as corrupt and skipped (an error if strict).
 */
#ifndef TPX_H
#define TPX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define TPX_OK 0
#define TPX_EINVAL (-1)        /* bad argument or configuration               */
#define TPX_ENOMEM (-2)        /* scratch allocation failed (create/reserve)  */
#define TPX_EOVERFLOW (-3)     /* a caller buffer is too small; the required
                                  count is in *d_n_clusters / *d_n_trig       */
#define TPX_ECORRUPT (-4)      /* strict mode saw an unknown header, or the
                                  trigger times decrease                      */
#define TPX_EAGAIN (-5)        /* admission refused (streaming)               */
#define TPX_ETIMEOUT (-6)      /* host-side wait ran out (streaming poll)     */
#define TPX_EDEVTIMEOUT (-7)   /* a bounded device-side wait ran out          */
#define TPX_ECUDA (-8)         /* a CUDA runtime call failed                  */
#define TPX_EUNSUPPORTED (-9)  /* input outside what the fused path handles   */

#define TPX_MODE_CC 0          /* connected components of the box adjacency   */
#define TPX_MODE_PAPER 1       /* box neighbourhood of each local maximum     */

/* Configuration.  Every paper parameter is a field (Sec. IV.A-C, V.A). */
typedef struct tpx_config {
    int32_t rx, ry;             /* spatial radii in pixels, inclusive, 0..7   */
    int32_t dt_ticks;           /* time radius in ticks, inclusive, >= 0      */
    int32_t mode;               /* TPX_MODE_CC or TPX_MODE_PAPER              */
    int64_t tof_max_ticks;      /* keep pixels with ToF <= this; 64000 = 100 us
                                   (Sec. IV.B).  At most 2^24 - 65537.        */
    int64_t wrap_thr_pix_ticks; /* unwrap threshold, pixel stream (20 s)      */
    int64_t wrap_thr_tdc_ticks; /* unwrap threshold, TDC stream (20 s)        */
    const int16_t *d_timewalk_lut; /* device, 1024 entries in ticks indexed by
                                   ToT, subtracted after the cut (Sec. IV.C);
                                   NULL = no correction                       */
    int32_t strict;             /* 1: unknown headers are an error            */
    int32_t chain;              /* 1: each tpx_process / tpx_decode continues
                                   the unwrap state and trigger count where
                                   the previous call on the context ended
                                   (kept on the device: a long stream can be
                                   fed in consecutive calls, each starting at
                                   a trigger packet); 0: each call starts a
                                   new stream unless tpx_set_state was used   */
    int32_t tile_geometry;      /* fused kernel tiles: TPX_TILE_4096 (1024-
                                   thread CTAs, one per SM, ranges of up to
                                   8192 positions), TPX_TILE_2048 (512-thread
                                   CTAs, two per SM, up to 4096 positions),
                                   or TPX_TILE_DEFAULT (the library's choice,
                                   TPX_TILE_4096).  Not a paper parameter:
                                   results are identical, only speed and the
                                   range limit differ.                        */
    int32_t flags;              /* TPX_FLAG_* bits, 0 by default              */
} tpx_config;

/* tpx_config.flags: TPX_FLAG_HOST_DIRECT -- tpx_process_host runs the fused
   kernel on the caller's host buffers in place (no device staging, no
   copies) when every one of them is pinned host memory mapped into the
   device at the same address (cudaHostAlloc / cudaHostRegister on a unified
   address space; checked with cudaPointerGetAttributes); the kernel then
   reads the packets and writes labels, records and triggers over the host
   link.  Otherwise the call stages through device memory as usual. */
#define TPX_FLAG_HOST_DIRECT 4
/* TPX_FLAG_LABELS32 -- the per-packet labels of tpx_process,
   tpx_process_host and tpx_process_noalloc are int32, not int64: the label
   minus the call's packet_index_base (for tpx_process_host, the base of the
   whole call), -1 where the packet is not a kept pixel.  The d_labels /
   h_labels argument then points to n_packets int32 values (the pointer type
   stays int64_t *).  Half the label bytes, the same information; a call whose
   labels would not fit 31 bits is rejected (TPX_EINVAL), as is a batch call
   with labels. */
#define TPX_FLAG_LABELS32 8
/* TPX_FLAG_RECORDS64 -- tpx_process, tpx_process_host and
   tpx_process_noalloc write the clusters as tpx_record64 (64 bytes: the
   record without the derived x, y and tof, which follow from the exact sums
   as x = s_x / s_tot, y = s_y / s_tot, tof = (t0 - t_trig[shot]) +
   s_t / s_tot); the d_clusters / h_clusters argument then points to cl_cap
   tpx_record64 (the pointer type stays tpx_record *).  A batch call is
   rejected (TPX_EINVAL). */
#define TPX_FLAG_RECORDS64 16

#define TPX_TILE_DEFAULT 0
#define TPX_TILE_4096 1
#define TPX_TILE_2048 2

/* One particle hit.  CC mode: one record per connected component; PAPER
   mode: one record per local maximum, summed over its box neighbourhood
   (Sec. V.C).  Records are written in ascending `label` order. */
typedef struct tpx_record {
    int64_t label;   /* stream index (packet_index_base + position) of the
                        cluster's earliest pixel in (time, stream index)
                        order; PAPER mode: of the local maximum              */
    int64_t shot;    /* trigger index (count of TDC packets before it)       */
    int64_t t0;      /* corrected time of the earliest pixel, ticks          */
    int64_t s_tot;   /* sum ToT                                              */
    int64_t s_x;     /* sum x*ToT                                            */
    int64_t s_y;     /* sum y*ToT                                            */
    int64_t s_t;     /* sum (t - t0)*ToT                                     */
    int32_t n;       /* pixel count                                          */
    int32_t n_peaks; /* local maxima among the pixels (Sec. V.B)             */
    double x;        /* s_x / s_tot                                          */
    double y;        /* s_y / s_tot                                          */
    double tof;      /* (t0 - t_trig[shot]) + s_t / s_tot, ticks             */
} tpx_record;        /* 88 bytes */

/* The compact record of TPX_FLAG_RECORDS64: the first 64 bytes of tpx_record. */
typedef struct tpx_record64 {
    int64_t label, shot, t0, s_tot, s_x, s_y, s_t;
    int32_t n, n_peaks;
} tpx_record64;      /* 64 bytes */

typedef struct tpx_counters {
    int64_t packets, pixels, tdcs, corrupt, dropped_pre_trigger, dropped_background,
            kept, clusters, peaks;
    int64_t status_bits;        /* raw device status word of the last call;
                                   bit 8: the checked build (libtpx_checked.so,
                                   -DTPX_CHECKED) met an index outside its array
                                   and skipped the access (tpx_sync then returns
                                   TPX_EUNSUPPORTED)                          */
    int64_t redone;             /* 1 if tpx_sync redid the last tpx_process
                                   call with the general path                 */
} tpx_counters;

typedef struct tpx_ctx tpx_ctx;

/* Unwrap state and trigger count before (or after) a call: what a call needs
   to continue a stream cut into several calls (Sec. IV.A wrap counting).  A
   call given a state behaves exactly as if the packets before it had been in
   the call, except that pixels before its first trigger packet are dropped
   (they belong to the previous call's last shot). */
typedef struct tpx_stream_state {
    int64_t pixels;        /* pixel packets before the call (0: none)         */
    int64_t pix_last_raw;  /* raw time of the last of them, ticks mod 2^34    */
    int64_t pix_wraps;     /* pixel wraps counted so far                      */
    int64_t triggers;      /* TDC packets before the call: trigger index base */
    int64_t tdc_last_raw;  /* raw time of the last of them, ticks mod 2^36    */
    int64_t tdc_wraps;     /* TDC wraps counted so far                        */
} tpx_stream_state;

/* Fill *cfg with the defaults: rx = ry = 1, dt = 32 ticks (50 ns),
   tof_max = 64000 ticks (100 us), both wrap thresholds 20 s, CC mode. */
void tpx_config_default(tpx_config *cfg);

/* Create a context bound to `cuda_stream` (a cudaStream_t; NULL = default
   stream) on the current device, with scratch for up to `max_packets`
   packets per call.  The configuration is copied; the timewalk table it
   points to must stay valid while the context is used.
   Errors: TPX_EINVAL (bad config), TPX_ENOMEM, TPX_ECUDA. */
int tpx_create(tpx_ctx **out, const tpx_config *cfg, int64_t max_packets, void *cuda_stream);

/* Grow the scratch to hold `max_packets` (synchronises the stream). */
int tpx_reserve(tpx_ctx *ctx, int64_t max_packets);

/* Destroy the context and free its scratch (synchronises the stream). */
int tpx_destroy(tpx_ctx *ctx);

/* The fused path (Sec. III - V.C, all steps in one pass over the stream).
     d_packets        [n_packets] uint64, device, stream order.
     packet_index_base  added to positions to form stream indices (labels),
                      so labels stay global when a long stream is cut into
                      calls.
     d_labels         [n_packets] int64 or NULL: per packet, the label of its
                      cluster (CC), its own stream index (PAPER) or -1 when
                      the packet is not a kept pixel.
     d_is_peak        [n_packets] uint8 or NULL: 1 for local maxima.
     d_clusters       [cluster_capacity] records, ascending label.
     d_n_clusters     device int64: number of records (if it exceeds the
                      capacity, only `capacity` are written and tpx_sync
                      returns TPX_EOVERFLOW).
     d_trig_t         [trig_capacity] int64: unwrapped trigger times.
     d_n_trig         device int64: number of triggers.
   Returns TPX_EINVAL for bad arguments or n_packets > reserved capacity;
   otherwise the work is queued and its outcome is read with tpx_sync. */
int tpx_process(tpx_ctx *ctx, const uint64_t *d_packets, int64_t n_packets,
                int64_t packet_index_base, int64_t *d_labels, uint8_t *d_is_peak,
                tpx_record *d_clusters, int64_t cluster_capacity, int64_t *d_n_clusters,
                int64_t *d_trig_t, int64_t trig_capacity, int64_t *d_n_trig);

/* The same with host buffers: copies h_packets to the device, processes
   them, copies the results back and synchronises.  h_labels / h_is_peak may
   be NULL.  *h_n_clusters and *h_n_trig receive the counts (the required
   ones when a buffer is short: TPX_EOVERFLOW).  Device staging is allocated
   on first use and kept by the context, grown for a larger call.  A call of
   at least 2^24 packets on a context with chain = 0 is pipelined (from the
   state of tpx_set_state, when one was set): cut into up to 16 pieces at
   trigger packets, chained through the unwrap state on the device, each
   piece's copy in
   overlapping the previous piece's kernel and its labels and records going
   out behind it (two more CUDA streams); a piece whose kernel meets anything
   it cannot hold -- a pixel after a cut that belongs in time to the shot
   before it is one -- sends the whole call back to the one-piece path, so
   the result always equals one call's.  Pinned host buffers let the copies
   overlap.  Returns the tpx_sync status. */
int tpx_process_host(tpx_ctx *ctx, const uint64_t *h_packets, int64_t n_packets,
                     int64_t packet_index_base, int64_t *h_labels, uint8_t *h_is_peak,
                     tpx_record *h_clusters, int64_t cluster_capacity, int64_t *h_n_clusters,
                     int64_t *h_trig_t, int64_t trig_capacity, int64_t *h_n_trig);

/* Kept pixels in stream order, as device arrays of one common capacity
   (structure of arrays, caller-owned), produced by tpx_decode. */
typedef struct tpx_hits {
    int64_t *index;   /* stream index: packet_index_base + packet position    */
    int64_t *shot;    /* trigger index (most recent trigger in time)          */
    int64_t *t;       /* unwrapped time after the timewalk table, ticks       */
    int32_t *tof;     /* t - t_trig[shot], ticks                              */
    uint8_t *x;
    uint8_t *y;
    uint16_t *tot;    /* time over threshold, 25 ns units                     */
} tpx_hits;

/* The same path in three separate calls, through global memory (no shot or
   range size limit; at most 2^31 - 1 kept pixels per call).  Each call
   queues its work on the context stream; scratch is taken from the
   context's general scratch, which these calls grow on first use (they may
   allocate, unlike tpx_process).

   tpx_decode: decode packets, unwrap ToA per stream (Sec. IV.A), bin each
   pixel to the most recent trigger in time and keep it if its ToF does not
   exceed tof_max (Sec. IV.B), subtract the timewalk table (Sec. IV.C).
     hits, hits_capacity   output arrays; kept pixels in stream order
     d_n_hits              device int64: number of kept pixels (if it exceeds
                           the capacity, only `capacity` are written and
                           tpx_sync returns TPX_EOVERFLOW)
     d_trig_t, d_n_trig    unwrapped trigger times and their number */
int tpx_decode(tpx_ctx *ctx, const uint64_t *d_packets, int64_t n_packets, int64_t packet_index_base,
               const tpx_hits *hits, int64_t hits_capacity, int64_t *d_n_hits,
               int64_t *d_trig_t, int64_t trig_capacity, int64_t *d_n_trig);

/* tpx_cluster: order the hits by ToA -- a stable device radix sort on
   (shot, corrected ToF), ties in stream order -- then join adjacent hits
   (Sec. V.A box rule) by union-find in that order, so that each cluster's
   root is its earliest hit; find the local maxima (Sec. V.B).
     n_hits        host count (read d_n_hits after tpx_decode)
     d_labels      [n_hits] int64: per hit, the stream index of its cluster's
                   earliest hit (CC mode) or its own stream index (PAPER mode)
     d_is_peak     [n_hits] uint8 or NULL: 1 for local maxima */
int tpx_cluster(tpx_ctx *ctx, const tpx_hits *hits, int64_t n_hits, int64_t *d_labels, uint8_t *d_is_peak);

/* tpx_centroid: cluster records in ascending label order (Sec. V.C).  CC
   mode: moments over the hits sharing a label; PAPER mode: over the box
   neighbourhood of each local maximum (d_is_peak required).  Same record
   layout and count/overflow rules as tpx_process. */
int tpx_centroid(tpx_ctx *ctx, const tpx_hits *hits, const int64_t *d_labels, const uint8_t *d_is_peak,
                 int64_t n_hits, tpx_record *d_clusters, int64_t cluster_capacity, int64_t *d_n_clusters);

/* Wait for the context's queued work and translate the device status word
   of the last call into a status code.  If counters != NULL, fill it.
   When the last call was tpx_process and the fused kernel met an input it
   cannot hold on chip (a range longer than the tiles' range capacity -- 8192
   positions for TPX_TILE_4096, 5120 for TPX_TILE_2048 -- or a pixel whose
   trigger lies outside its range), tpx_sync redoes that call exactly with the
   general path before returning (this may allocate general scratch); for a
   batch, the runs concerned.  Only the last call since the previous tpx_sync
   is redone: if an earlier one needed it, tpx_sync returns TPX_EUNSUPPORTED
   (call tpx_sync after each call whose input may be unusual). */
int tpx_sync(tpx_ctx *ctx, tpx_counters *counters);

/* Kernel timing (the measurement of the fused path, Sec. V).
   tpx_kernel_timing(ctx, 1) turns it on and resets the sums: every later
   fused launch of tpx_process / tpx_process_batch on the context records CUDA
   events on its stream before the unwrap pre-pass, between the pre-pass and
   the fused kernel, and after the fused kernel (not while the stream is being
   captured into a graph).  0 turns it off and keeps the sums.  The events
   are created on the first enable; TPX_ECUDA if that fails.
   tpx_kernel_times waits for the recorded launches and writes the summed
   pre-pass and fused-kernel milliseconds and the number of launches timed
   (any pointer may be NULL).  TPX_EINVAL for a NULL context. */
int tpx_kernel_timing(tpx_ctx *ctx, int enable);
int tpx_kernel_times(tpx_ctx *ctx, double *prepass_ms, double *fused_ms, int64_t *launches);

/* Per-phase cycle counters of the fused kernel (a measurement aid).  In the
   instrumented build (libtpx_phases.so, compiled with -DTPX_PHASE_TIMING)
   lane 0 of every warp adds the clock64 cycles of each phase of each tile to
   the phase's counter (a phase's time includes the barrier wait that ends
   it).  This call synchronises the device and copies the 32 counters of one
   tile geometry (TPX_TILE_4096 or TPX_TILE_2048) to h_cycles[32], zeroing
   them when `clear` is nonzero.  Phases: 0 tile start, 1 tile load,
   2 look-ahead, 3 walk 2 and its scan, 4 trigger times, 5 walk 4 (records),
   6 hash insert, 7 neighbour pass, 8 compression, 9 unions, 10 roots,
   11 member lists, 12 member-list walks (and the previous tile's copy-out),
   13 label ranks and staged stores, 14 labels and offsets, 15 tail,
   16 the CTA's end.  The normal build returns TPX_EUNSUPPORTED (zeros);
   TPX_EINVAL for another geometry or a NULL pointer. */
int tpx_debug_phase_times(int tile_geometry, uint64_t *h_cycles, int clear);

/* Upper bound on n_packets for tpx_process_noalloc (2^26 packets, 512 MB of
   input): the size of its fixed scratch array. */
#define TPX_NOALLOC_MAX_PACKETS (1LL << 26)

/* The fused path without any device allocation (no counterpart in the paper;
   it serves callers that cannot call cudaMalloc where they process data --
   real-time acquisition loops that must not block in the allocator, hosts
   that fix the library's memory up front).  Same inputs and outputs as
   tpx_process, but no context: the configuration and the CUDA stream are
   passed directly, and the look-back scratch is one fixed array in device
   memory that is part of the library (about 2.4 MB per device that loads it,
   held until exit).  The first call on each device, with that device current,
   looks up the array's device address (cudaGetSymbolAddress).  All calls on a
   device share the array and it keeps the last call's contents (the per-call
   control block is cleared first): calls that overlap on the GPU race and
   must not be made.  The call reads the device status back and synchronises
   the stream before it returns, so it must not be made on a stream that is
   being captured into a CUDA graph.  If h_counters is not NULL it receives
   the counters.
   Results equal tpx_process's when the fused kernel can hold the input.  The
   call has no redo: where tpx_sync would redo a call with the general path (a
   shot longer than the 8192-position range of the 4096-packet tiles, or a
   pixel whose trigger lies outside its range), this call returns
   TPX_EUNSUPPORTED and its outputs are incomplete.
   Errors: TPX_EINVAL for a bad configuration or argument, or n_packets above
   TPX_NOALLOC_MAX_PACKETS; TPX_EUNSUPPORTED as above; TPX_EDEVTIMEOUT,
   TPX_ECORRUPT, TPX_EOVERFLOW as for tpx_sync; TPX_ECUDA. */
int tpx_process_noalloc(const tpx_config *cfg, void *cuda_stream, const uint64_t *d_packets,
                        int64_t n_packets, int64_t packet_index_base, int64_t *d_labels,
                        uint8_t *d_is_peak, tpx_record *d_clusters, int64_t cluster_capacity,
                        int64_t *d_n_clusters, int64_t *d_trig_t, int64_t trig_capacity,
                        int64_t *d_n_trig, tpx_counters *h_counters);

/* ToT-ToF joint histogram for the timewalk calibration (Sec. IV.C: a
   narrow ToF slice around an ion peak, the ToF distribution of every ToT
   value; the fit of Eq. 1 to the per-ToT centres is host work).  Adds, for
   every hit whose tof lies in [tof_lo_ticks, tof_lo_ticks + n_tof_bins *
   tof_bin_ticks), one count to d_hist[tot * n_tof_bins + (tof - tof_lo_ticks)
   / tof_bin_ticks]; the caller zeroes d_hist (1024 * n_tof_bins uint32,
   device) and may accumulate several calls.  Hits as produced by tpx_decode
   on a context without a timewalk table (tof is then the measured ToF).
   Asynchronous on the context stream.  TPX_EINVAL for n_tof_bins < 1,
   tof_bin_ticks < 1 or NULL pointers with n_hits > 0. */
int tpx_tot_tof_histogram(tpx_ctx *ctx, const tpx_hits *hits, int64_t n_hits, int32_t tof_lo_ticks,
                          int32_t tof_bin_ticks, int32_t n_tof_bins, uint32_t *d_hist);

/* Failure detection without a GPU fault (no counterpart in the paper): the
   next tpx_process call leaves tile `tile`'s look-back flags unpublished
   (a negative tile clears the request), so the bounded waits of the tiles
   after it run out (about 0.5 s once; every later wait then gives up at
   once); the call completes, its outputs are not valid, and tpx_sync returns
   TPX_EDEVTIMEOUT.  The context stays usable.  For tests of the timeout
   path only. */
int tpx_debug_hold_tile(tpx_ctx *ctx, int64_t tile);

/* Test hook for tpx_process_noalloc (no counterpart in the paper): sets the
   look-back sequence number that the current device's last call used, so
   that a test can make the next calls cross the wrap of the 30-bit sequence
   (where the fixed array's flags are cleared) without 2^30 calls.  The next
   call uses last_seq + 1 (mod 2^30; 0 is skipped).  TPX_EINVAL if last_seq
   >= 2^30; TPX_ECUDA if the current device cannot be read. */
int tpx_debug_noalloc_seq(uint32_t last_seq);

/* ---- learned overlap refiner (not in the paper; its multi-hit discussion,
   Sec. VII.B, and the local-maximum count of Sec. V.B motivate it) ----
   A cluster may hold two particles. Its 9 x 9 patch (channel 0: ToT / 1023
   rounded to bf16; channel 1: ToA relative to the cluster's earliest pixel in
   units of 32 ticks, clamped to [-8, 8], rounded to fp16; empty cells 0;
   stored as fp32), centred on the centroid rounded half up, goes through a multilayer perceptron 162 -> H -> H -> 6 (ReLU):
   two logits (one or two particles) and (dx, dy) of each particle in pixels
   from the patch centre.  Parameters are one fp32 array (W1[162 x H], b1,
   W2[H x H], b2, W3[H x 6], b3; row-major). */

/* Patches of the CC-mode clusters with more than min_pixels pixels, from a
   tpx_process call's packets, per-packet labels and records (device, as
   that call wrote them).  d_patches [capacity x 162] floats, d_sel
   [capacity] record index of each patch, d_centre [capacity x 2] patch
   centre (x, y); *d_n_patches the number of such clusters (TPX_EOVERFLOW
   if above capacity: only `capacity` are written).  Synchronises. */
int tpx_refine_patches(tpx_ctx *ctx, const uint64_t *d_packets, int64_t n_packets, int64_t packet_index_base,
                       const int64_t *d_labels, const tpx_record *d_clusters, int64_t n_clusters, int32_t min_pixels,
                       float *d_patches, int64_t *d_sel, int32_t *d_centre, int64_t capacity, int64_t *d_n_patches);

/* Number of floats of the parameter array for H hidden units. */
int64_t tpx_refiner_params(int32_t hidden);

/* Forward pass of n patches: d_out [n x 6]; d_work [n x 2H] floats.
   Asynchronous (fp32 tiled GEMMs on the context stream). */
int tpx_refiner_forward(tpx_ctx *ctx, const float *d_params, int32_t hidden, const float *d_x, int64_t n,
                        float *d_work, float *d_out);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, step >= 1) on a minibatch of
   n <= 2^21 patches with targets d_y [n x 5] = (count 1 or 2, dx1, dy1, dx2,
   dy2): loss = mean softmax cross-entropy of the count + offset_weight x
   mean half squared error of the true particles' offsets.  d_grad,
   d_adam_m, d_adam_v: parameter-sized; d_work [n x (4H + 12)] floats;
   *d_loss the minibatch loss before the step.  Asynchronous. */
int tpx_refiner_train_step(tpx_ctx *ctx, float *d_params, float *d_adam_m, float *d_adam_v, float *d_grad,
                           int32_t hidden, int64_t step, const float *d_x, const float *d_y, int64_t n, float lr,
                           float offset_weight, float *d_work, float *d_loss);

/* Inference on the tensor cores (hidden = 64, 128 or 160, else
   TPX_EUNSUPPORTED): tpx_refiner_pack rounds the fp32 parameters to a bf16
   copy (d_packed, tpx_refiner_packed_bytes(hidden) bytes, 16-byte aligned;
   0 bytes for an unsupported width); tpx_refiner_infer runs all three
   layers in one kernel: inputs and weights in bf16 (the patch values are
   exact in bf16), fp32 accumulation and biases, each hidden activation
   rounded to bf16 after its ReLU.  d_x 8-byte aligned [n x 162], d_out
   [n x 6].  Asynchronous. */
int64_t tpx_refiner_packed_bytes(int32_t hidden);
int tpx_refiner_pack(tpx_ctx *ctx, const float *d_params, int32_t hidden, void *d_packed);
int tpx_refiner_infer(tpx_ctx *ctx, const void *d_packed, int32_t hidden, const float *d_x, int64_t n,
                      float *d_out);

/* Refined hits from the forward outputs: per patch d_hits[5] = (k, x1, y1,
   x2, y2): k = 2 when the probability of two particles reaches `threshold`
   (positions from the offsets); else (x1, y1) is the cluster's plain
   centroid (Sec. V.C) with k = 1 when the probability of one particle
   reaches `threshold`, k = 0 otherwise (x2 = y2 = 0).  The count is decided on the fp32 logit margin
   o1 - o0 against log(threshold / (1 - threshold)).  TPX_EINVAL unless
   0 < threshold < 1.  Asynchronous. */
int tpx_refine_decide(tpx_ctx *ctx, const float *d_out, const tpx_record *d_clusters, const int64_t *d_sel,
                      const int32_t *d_centre, int64_t n, float threshold, float *d_hits);

/* ---- the convolutional refiner (the same patch, count and offsets) ----
   The 2 x 9 x 9 patch through three 3 x 3 convolutions without padding and
   two dense layers: conv1 2 -> 16 channels (7 x 7), conv2 16 -> 16 (5 x 5),
   conv3 16 -> 32 (3 x 3), fc1 288 -> 144 (conv3's map flattened in channel,
   row, column order), fc2 144 -> 6; ReLU after every layer but the last.
   A convolution is out[co][y][x] = b[co] + sum W[co][ci][ky][kx]
   in[ci][y + ky][x + kx].  Parameters: one fp32 array of tpx_cnn_params()
   floats: W1 [16][2][3][3], b1, W2 [16][16][3][3], b2, W3 [32][16][3][3], b3,
   W4 [144][288], b4, W5 [6][144], b5. */

/* Number of parameters (49,750). */
int64_t tpx_cnn_params(void);

/* Floats of workspace tpx_cnn_forward and tpx_cnn_train_step need for n
   patches. */
int64_t tpx_cnn_work_floats(int64_t n);

/* fp32 forward pass of n <= 2^22 patches: d_x [n x 162] floats (channel 0,
   then channel 1, rows of 9), d_out [n x 6].  Asynchronous. */
int tpx_cnn_forward(tpx_ctx *ctx, const float *d_params, const float *d_x, int64_t n, float *d_work, float *d_out);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8, step >= 1) on a minibatch of
   1 <= n <= 2^20 patches, targets d_y [n x 5] and loss as in
   tpx_refiner_train_step; d_grad receives the gradient, *d_loss the loss
   before the step.  fp32 GEMMs over the layers' im2col matrices.
   Asynchronous. */
int tpx_cnn_train_step(tpx_ctx *ctx, float *d_params, float *d_adam_m, float *d_adam_v, float *d_grad, int64_t step,
                       const float *d_x, const float *d_y, int64_t n, float lr, float offset_weight, float *d_work,
                       float *d_loss);

/* Inference on the tensor cores (tcgen05, fp32 accumulation in tensor
   memory): tpx_cnn_pack writes a bf16 copy of the weights (and fp32 biases)
   to d_packed (tpx_cnn_packed_bytes() bytes, 256-byte aligned);
   tpx_cnn_infer runs the five layers over n <= 2^30 patches d_x [n x 162]
   bf16 (16-byte aligned; tpx_refine_patches_bf16) in one kernel: groups of
   48 patches per CTA, the layers as implicit GEMMs whose activations stay in
   shared memory, each hidden activation rounded to bf16 after its ReLU, into
   d_out [n x 6] floats.  d_work is not used (tpx_cnn_infer_work_bytes is
   kept for the interface: 256 bytes for n > 0); it may be NULL.
   Asynchronous; a tensor-core wait that runs out sets the context's status
   (TPX_EDEVTIMEOUT at tpx_sync). */
int64_t tpx_cnn_packed_bytes(void);
int tpx_cnn_pack(tpx_ctx *ctx, const float *d_params, void *d_packed);
int64_t tpx_cnn_infer_work_bytes(int64_t n);
/* Per-phase cycle counters of tpx_cnn_infer's kernel in the instrumented
   build (libtpx_phases.so, -DTPX_PHASE_TIMING): thread 0 of each CTA adds
   the clock64 cycles of each phase of each group of patches.  Synchronises
   the device, copies the 16 counters to h_cycles[16] (zeroing them when
   `clear` is nonzero).  Phases: 0 wait for the group's patches, 1 their
   conversion into the conv1 input map, then MMAs and epilogue of conv1 (2,
   3), conv2 (4, 5), conv3 (6, 7), fc1 (8, 9), fc2 (10, 11).  The normal
   build returns TPX_EUNSUPPORTED (zeros); TPX_EINVAL for a NULL pointer. */
int tpx_debug_cnn_phase_times(uint64_t *h_cycles, int clear);
int tpx_cnn_infer(tpx_ctx *ctx, const void *d_packed, const uint16_t *d_x, int64_t n, void *d_work, float *d_out);

/* tpx_refine_patches writing the patches as bf16 [capacity x 162] (the patch
   values are exact in bf16: 324 bytes a patch instead of 648). */
int tpx_refine_patches_bf16(tpx_ctx *ctx, const uint64_t *d_packets, int64_t n_packets, int64_t packet_index_base,
                            const int64_t *d_labels, const tpx_record *d_clusters, int64_t n_clusters,
                            int32_t min_pixels, uint16_t *d_patches, int64_t *d_sel, int32_t *d_centre,
                            int64_t capacity, int64_t *d_n_patches);

/* Batched runs (Sec. VI batches shots by zero-padding them to a rectangle;
   here nothing is padded): n_runs independent acquisitions concatenated in
   one device buffer, run r being packets [h_run_offsets[r],
   h_run_offsets[r+1]).  One persistent launch of the fused kernel works
   through a device queue of tiles of all runs; every run is a stream of its
   own (unwrap state and trigger count start from zero at its first packet),
   the context's configuration applies to all.  In CC mode a tile whose
   range (its shots up to the next trigger packet) is longer than the tile
   can hold on chip clusters it in the same launch with the big-range path:
   the whole range decoded into the CTA's global scratch, its kept pixels
   sorted by (shot, time bin), each pixel compared with its own and the
   previous bin (the same results as the tile's path).  A range even that
   cannot hold (more than 65,535 packets, more kept pixels than its shared
   scratch: 31,040, or 24,960 with 2048-packet tiles, more than 256 trigger
   packets), any range in PAPER mode, and a pixel whose trigger lies
   outside its range send the run to the general path: such runs are redone
   exactly at tpx_sync (counters.redone = the number of such runs) and
   spliced into the outputs.  The big-range scratch takes 13.3 MB per CTA of
   the grid (10.8 MB with 2048-packet tiles) of the batch scratch.
     h_run_offsets   host [n_runs + 1], h_run_offsets[0] = 0, non-decreasing
     d_labels, d_is_peak  per packet of the whole buffer, or NULL; labels are
                     positions in the whole buffer
     d_clusters, cluster_capacity, d_n_clusters   records of all runs, run
                     after run, each run's in ascending label order; `shot`
                     counts within the run
     d_run_clusters  device [n_runs + 1]: first record of each run and the
                     total (written by the call)
     d_trig_t, trig_capacity, d_n_trig, d_run_trig   trigger times of all
                     runs, run after run, with the same offsets layout
   Asynchronous like tpx_process; tpx_sync returns the status.  The call
   itself waits only until the previous batch's tables have been uploaded.
   The first call for a larger batch grows the context's batch scratch.
   Counters describe the tiles' pass (redone runs included as they ran).
   CUDA graphs: the call may be captured on the context's stream (relaxed
   capture mode, after one ordinary batch call on the context so that its
   kernels are set up); a captured call keeps device and pinned host tables
   of its own for the graph (freed with the context), and each replay
   re-uploads its run tables and launches the one persistent kernel.  Call
   tpx_sync after each replay (runs that need the general path are redone
   there, outside the graph), replay on the same context, and do not call
   tpx_reserve between capture and replay.
   TPX_EINVAL for bad offsets or pointers. */
int tpx_process_batch(tpx_ctx *ctx, const uint64_t *d_packets, const int64_t *h_run_offsets, int64_t n_runs,
                      int64_t *d_labels, uint8_t *d_is_peak, tpx_record *d_clusters, int64_t cluster_capacity,
                      int64_t *d_n_clusters, int64_t *d_run_clusters, int64_t *d_trig_t, int64_t trig_capacity,
                      int64_t *d_n_trig, int64_t *d_run_trig);

/* Tile-geometry autotuner (not in the paper).  With tile_geometry =
   TPX_TILE_DEFAULT the first calls of at least 2^20 packets alternate the
   two geometries, timed with CUDA events on the context stream; at the
   tpx_sync after both have run, the faster one per packet is kept for the
   context (a call that had to be redone by the general path counts as the
   slowest).  Results do not depend on the geometry.
     tile_geometry    out: TPX_TILE_4096 / TPX_TILE_2048 once chosen (or the
                      geometry fixed by the configuration), TPX_TILE_DEFAULT
                      while sampling
     ms_per_mpacket   out, may be NULL: [2] the best times seen, ms per 10^6
                      packets, for the 4096- and the 2048-packet tiles (0 if
                      not sampled)
   TPX_EINVAL for NULL ctx or tile_geometry. */
int tpx_tuning(tpx_ctx *ctx, int32_t *tile_geometry, double *ms_per_mpacket);

/* The next tpx_process / tpx_decode on the context starts from *state
   (NULL: the start of a stream).  Asynchronous on the context stream. */
int tpx_set_state(tpx_ctx *ctx, const tpx_stream_state *state);

/* The state after the last tpx_process / tpx_decode (synchronises). */
int tpx_get_state(tpx_ctx *ctx, tpx_stream_state *state);

/* Associative summary of a stretch of the stream's two unwrap chains
   (Sec. IV.A): counts, first and last raw times, and the wrap steps inside the
   stretch.  Summaries of consecutive stretches combine in order; the
   combination of all stretches before a shard is that shard's starting state
   (tpx_set_state), which is how ranks that each hold a contiguous range of
   shots agree on the unwrap state without exchanging packets. */
typedef struct tpx_chain_summary {
    int64_t pixels, pix_first_raw, pix_last_raw, pix_wraps;
    int64_t triggers, tdc_first_raw, tdc_last_raw, tdc_wraps;
} tpx_chain_summary;

/* Summarise d_packets[0, n_packets) (one read of the packets; synchronises). */
int tpx_summarize(tpx_ctx *ctx, const uint64_t *d_packets, int64_t n_packets, tpx_chain_summary *out);

/* ---- streaming: acquisition chunks in, particle hits out ---------------
   A stream takes the packet stream in consecutive chunks as they arrive
   (any sizes; a chunk need not end at a trigger).  Each submit processes
   everything held so far plus the new chunk through the general path and
   emits the records of every shot that is closed: all shots except the
   last `hold_triggers` ones, whose pixels may still arrive in a later chunk
   (a pixel reports after its light curve ends, Sec. III, so with a long ToF
   cut pixels of shot k follow trigger k+1 in the stream).  Clusters that
   straddle chunk boundaries are therefore complete when emitted, and the
   unwrap state of the held part stays on the device.  Results of a chunk are
   exactly those of processing the whole stream at once, restricted to the
   emitted shots, provided hold_triggers spans tof_max plus the readout
   delay.  Each result lists its records in ascending label order; across
   results the order is by shot (a late cluster of shot k, read out after
   trigger k+1, can carry a larger label than an early cluster of shot k+1).
   Per-packet labels are not produced by streams. */
typedef struct tpx_stream tpx_stream;

typedef struct tpx_stream_config {
    tpx_config cfg;               /* processing configuration (chain ignored) */
    int64_t max_chunk_packets;    /* largest chunk a submit accepts           */
    int64_t max_hold_packets;     /* largest held (open) part; exceeding it is
                                     TPX_EOVERFLOW                            */
    int32_t hold_triggers;        /* shots held open after each chunk (>= 1)  */
    int32_t slots;                /* chunks whose results may await poll      */
    int64_t hbm_budget_bytes;     /* process-wide device memory for all
                                     streams (0: no limit); create returns
                                     TPX_EAGAIN when a new stream exceeds it  */
} tpx_stream_config;

typedef struct tpx_stream_result {
    uint64_t ticket;
    int32_t status;               /* status of processing this chunk          */
    int32_t reserved;
    int64_t first_shot;           /* emitted shots: [first_shot, first_shot +  */
    int64_t n_shots;              /*                 n_shots), global indices  */
    const int64_t *trig_t;        /* their trigger times (host)               */
    int64_t n_clusters;
    const tpx_record *clusters;   /* host; valid until the slot is reused     */
    int64_t packets_processed;    /* packets the chunk's processing covered   */
    double latency_us;            /* submit entry to results on the host      */
} tpx_stream_result;

/* Create a stream on the current device, working on `cuda_stream`.
   Errors: TPX_EINVAL, TPX_ENOMEM, TPX_EAGAIN (budget). */
int tpx_stream_create(tpx_stream **out, const tpx_stream_config *cfg, void *cuda_stream);

/* Submit a chunk (host memory; pinned for best latency).  Returns a ticket at
   once: the chunk is queued in a free result slot and the stream's worker
   thread processes the queued chunks in order, so up to `slots` chunks are in
   flight.  The chunk's memory must stay valid and unchanged until its ticket
   has been polled.  TPX_EAGAIN when every slot holds a chunk not yet polled
   (admission); TPX_EINVAL when n_packets exceeds max_chunk_packets or after
   tpx_stream_finish.  Errors of the processing itself (TPX_EOVERFLOW when
   the open shots outgrow max_hold_packets, TPX_ECORRUPT for decreasing
   trigger times, TPX_ECUDA) are returned by the ticket's poll. */
int tpx_stream_submit(tpx_stream *st, const uint64_t *h_chunk, int64_t n_packets, uint64_t *ticket);

/* End of the stream: emit every held shot (returns a ticket like submit). */
int tpx_stream_finish(tpx_stream *st, uint64_t *ticket);

/* Wait up to timeout_us (negative: forever) for a ticket's results.
   TPX_ETIMEOUT if not ready in time, TPX_EINVAL for an unknown ticket; the
   processing error of a failed chunk (its slot is freed).  The result's
   buffers belong to the slot and stay valid until the slot is reused by a
   later submit. */
int tpx_stream_poll(tpx_stream *st, uint64_t ticket, tpx_stream_result *out, int32_t timeout_us);

int tpx_stream_destroy(tpx_stream *st);

/* Checkpoint and resume (no counterpart in the paper, which processes whole
   files): all that a stream carries from one submit to the next -- the
   packets of its open shots, the unwrap state and trigger count where they
   start, the stream index of the first -- as one host byte block of
   tpx_stream_snapshot_bytes() bytes (header + 8 bytes per held packet).
   tpx_stream_snapshot waits for the stream's queued work; results not yet
   polled are not part of the checkpoint (poll them first; they stay
   pollable).  TPX_EOVERFLOW (and *written = the size needed) if capacity is
   short; TPX_EINVAL after tpx_stream_finish.  tpx_stream_restore loads one
   into a stream created with the same configuration that has not been
   submitted to; its later submits continue the old stream exactly (the same
   shots, trigger times and records as if it had not stopped).  TPX_EINVAL for
   a damaged block, another configuration (radii, dt, mode, ToF cut, wrap
   thresholds, hold_triggers) or a stream already in use,
   TPX_EOVERFLOW if the held packets exceed max_hold_packets. */
int64_t tpx_stream_snapshot_bytes(tpx_stream *st);
int tpx_stream_snapshot(tpx_stream *st, void *h_buf, int64_t capacity, int64_t *written);
int tpx_stream_restore(tpx_stream *st, const void *h_buf, int64_t n_bytes);

/* Static description of a status code. */
const char *tpx_strerror(int code);

/* Library version string. */
const char *tpx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TPX_H */
