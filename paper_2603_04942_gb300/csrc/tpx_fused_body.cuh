// tpx_fused_body.cuh -- the fused kernel, included once per tile geometry
// by tpx_fused.cu inside a namespace that defines NT (threads per CTA),
// T (packets per tile), C (range capacity), HB (hash buckets), MS (trigger
// packets a range may hold) and MINB (CTAs per SM). No include guard: it
// is meant to be included repeatedly.
constexpr int NW = NT / 32;
constexpr int MAXSEG = MS;         // TDC packets a range may hold (more: the call is redone)
constexpr uint64_t INVALID = ~0ull;
constexpr uint32_t EMPTY = 0xFFFFu;
constexpr long long MAX_SPIN = 1LL << 22;   // bounded look-back waits (~0.5 s)
constexpr int LA0 = T / 2;         // look-ahead window loaded with the tile
static_assert(T + LA0 <= C, "the look-ahead window fits the range");

static_assert(T % NT == 0 && C % NT == 0 && T <= C && C <= 16384, "tile geometry");
static_assert(C < 0xFFFF && HB % 2 == 0 && (HB & (HB - 1)) == 0 && HB * 2 <= C * 4, "16-bit hash heads");

// ------------------------------------------------------------------ helpers
// Checked build (-DTPX_CHECKED): every data-dependent shared-memory or global
// index (hash chains, member lists, roots, cluster ids, output positions) is
// tested against its array before use; a violation sets ST_BOUNDS in the
// status word and skips the access. The normal build compiles the tests away.
#ifdef TPX_CHECKED
__device__ __forceinline__ bool in_bounds(long long i, long long n, const Params &p) {
    if (i >= 0 && i < n) return true;
    atomicOr(&p.ctl->status, ST_BOUNDS);
    return false;
}
#define TPX_IN(i, n) in_bounds((long long)(i), (long long)(n), p)
#else
#define TPX_IN(i, n) true
#endif

// Phase timing (-DTPX_PHASE_TIMING, the libtpx_phases.so build): lane 0 of
// every warp adds the clock64 cycles since the previous mark to the phase's
// counter; the kernel's end adds the CTA's counters to g_phase. A phase's
// time includes the barrier wait that ends it. The normal build compiles the
// marks away.
#ifdef TPX_PHASE_TIMING
__device__ unsigned long long g_phase[32];
#define TPX_PH(k)                                                                         \
    do {                                                                                  \
        const long long ph_now = clock64();                                               \
        if ((threadIdx.x & 31) == 0) atomicAdd(&S.ph[k], (unsigned long long)(ph_now - ph_t)); \
        ph_t = ph_now;                                                                    \
    } while (0)
#else
#define TPX_PH(k) do {} while (0)
#endif

__device__ __forceinline__ int pad(int p) { return p + (p >> 3); }   // conflict-free 8-wide walks

// kept-pixel record: [63:40] tof+bias | [39:30] ToT | [29:16] segment | [15:8] y | [7:0] x;
// the low 30 bits are the pixel's cell (segment, y, x)
__device__ __forceinline__ uint64_t mkrec(uint32_t tofb, uint32_t seg, uint32_t tot, uint32_t x, uint32_t y) {
    return ((uint64_t)tofb << 40) | ((uint64_t)tot << 30) | ((uint64_t)seg << 16) | ((uint64_t)y << 8) | x;
}
__device__ __forceinline__ int r_x(uint64_t r) { return (int)(r & 255); }
__device__ __forceinline__ int r_y(uint64_t r) { return (int)((r >> 8) & 255); }
__device__ __forceinline__ int r_seg(uint64_t r) { return (int)((r >> 16) & 0x3FFF); }
__device__ __forceinline__ int r_tot(uint64_t r) { return (int)((r >> 30) & 1023); }
__device__ __forceinline__ int r_tof(uint64_t r) { return (int)(r >> 40); }
__device__ __forceinline__ uint32_t r_cell(uint64_t r) { return (uint32_t)r & 0x3FFFFFFFu; }
// |d| <= dt, for 0 <= dt < 2^31
__device__ __forceinline__ bool within(int d, int dt) { return (uint32_t)d + (uint32_t)dt <= 2u * (uint32_t)dt; }

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_agg(GAgg *dst, const GAgg &a) {
    long long *d = reinterpret_cast<long long *>(dst);
    const long long *s = reinterpret_cast<const long long *>(&a);
#pragma unroll
    for (int i = 0; i < 8; i++) __stcg(d + i, s[i]);
}
__device__ __forceinline__ GAgg ld_agg(const GAgg *src) {
    GAgg a;
    const long long *s = reinterpret_cast<const long long *>(src);
    long long *d = reinterpret_cast<long long *>(&a);
#pragma unroll
    for (int i = 0; i < 8; i++) d[i] = __ldcg(s + i);
    return a;
}

// hash of a (segment, x, y) cell
__device__ __forceinline__ uint32_t hcell(int seg, int x, int y) {
    return (uint32_t)(x + 67 * y + 1543 * seg) & (HB - 1);
}

// Union-find over a shared-memory parent array, addressed explicitly in the
// shared window (32-bit addresses, ld/st.volatile.shared, atom.shared.cas).
__device__ __forceinline__ uint32_t sh_ld(uint32_t a) {
    uint32_t v;
    asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sh_st(uint32_t a, uint32_t v) {
    asm volatile("st.volatile.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t sh_cas(uint32_t a, uint32_t cmp, uint32_t v) {
    uint32_t o;
    asm volatile("atom.shared.cas.b32 %0, [%1], %2, %3;" : "=r"(o) : "r"(a), "r"(cmp), "r"(v) : "memory");
    return o;
}
__device__ __forceinline__ uint32_t find_ro(uint32_t pbase, uint32_t x) {
    uint32_t p;
    while ((p = sh_ld(pbase + 4 * x) & 0xFFFFu) != x) x = p;
    return x;
}

// --------------------------------------------------------------- smem layout
struct __align__(16) Smem {
    uint64_t buf[C + C / 8];                          // packets, then kept-pixel records
    uint32_t parent[C];                               // union-find; then member links and
                                                      // root positions (CC) / peak list (PAPER)
    union { uint16_t head[HB]; uint32_t mhead[C]; } u1; // hash heads (16-bit positions), then
                                                      // member-list heads
    union { uint16_t next[C]; uint16_t rootof[C]; } u2;
    uint8_t notpeak[C];
    uint32_t lbits[C / 32];       // CC: the tile's label positions, one bit each
    uint16_t lpre[C / 32];        // labels before each bitmap word
    long long tdc_t[MAXSEG];      // unwrapped trigger times of the range
    uint16_t tdc_pos[MAXSEG];     // their positions
    GAgg E;                       // unwrap state before the tile (from the pre-pass)
    long long j0;                 // pixel wrap step from the last pixel before the range to its first
    int warp_int[NW + 1];
    unsigned long long cnt[C_NUM];   // this tile's counters
    unsigned long long acc[C_NUM];   // this CTA's counters, added to the call's at its end
    long long next_tile;          // claimed while the current tile runs
    long long tile;
    long long clo;
    long long tlo;                // trigger offset of a batch tile
    // staged tiles awaiting their offsets: a ring, entry k staged in slot k
    // (one entry for a single stream, RING in a batch)
    struct Pend {
        long long tile, ntr;      // the tile; its trigger total (single streams)
        int ncl, ntdc, run;       // its records and triggers; its run
        bool first, big;          // the run's first tile; records in the big-range slot
    } pend[4];
    int pend_head, pend_count;
    int first_tdc;
    int first_pix;                // first pixel of the range
    int la_first[3];              // first TDC packet past the tile (window, then rotating chunk slots)
    int nroot;                    // CC: clusters of the tile (roots appended to the root list)
    unsigned status;
#ifdef TPX_PHASE_TIMING
    unsigned long long ph[32];
#endif
};

// MINB CTAs per SM within the SM's 228 KB of shared memory (1 KB of it is
// reserved per CTA)
static_assert(MINB * (sizeof(Smem) + 1024) <= 228 * 1024, "shared memory of the tile geometry");

// a batch keeps up to RING staged tiles per CTA waiting for their offsets (a
// tile behind a big range need not wait for it); a single stream keeps one
constexpr int RING = kBatchRing;
static_assert(RING >= 1 && RING <= 4, "the ring of staged tiles");

// ---------------------------------------------------- big-range constants
// (the path itself is described at big_range below)
constexpr int BR_L = 65535;          // positions of a big range (16-bit)
constexpr int BR_LW = (BR_L + 1) / 32;
constexpr int BR_S = 256;            // shots (trigger packets) of a big range
// sort keys (time bin, x stripe) shared out over its shots
constexpr int BR_BINS = C >= 8192 ? 12288 : 4096;
constexpr int BR_NS = 32;            // x stripes of 8 columns (16 when rx > 8, one when rx > 16)
struct BrMom { unsigned long long s_tot, s_x, s_y, s_tt, best; unsigned n, npk; };
static_assert(sizeof(BrMom) == 48, "moment record");
// shared scratch: the tile arrays in front of the trigger tables
constexpr int BR_REGION = (int)offsetof(Smem, tdc_t);
// the neighbour pass reads the sorted records through shared memory, BR_CH
// pixels at a time with the records before them that they can reach
constexpr int BR_CH = 2 * NT;
constexpr int BR_SB = 2 * BR_CH;
constexpr int BR_FIXED = 4 * (BR_BINS + 4) + 4 * BR_LW + 2 * BR_LW + 4 * 5 * BR_S + 4 * 16 + 8 * BR_SB;
// kept pixels: a 16-bit parent and a local-maximum bit each
constexpr int BR_N0 = ((BR_REGION - BR_FIXED) * 8 / 17) & ~63;
constexpr int BR_N = BR_N0 < 65472 ? BR_N0 : 65472;
static_assert(BR_N > C && BR_N % 64 == 0, "a big range holds more pixels than a tile");
static_assert(2 * BR_N + BR_N / 8 + BR_FIXED <= BR_REGION, "big-range shared scratch");
static_assert(BR_BINS % NT == 0 && BR_LW % NT == 0, "bins and label words split evenly over the CTA");
// per-CTA global scratch: records by position, sorted records and their
// positions, moments by root, and the staged cluster records (a big range
// may hold up to one cluster per kept pixel)
constexpr size_t BR_REC_OFF = ((size_t)8 * (BR_L + 1) + (size_t)58 * BR_N + 255) & ~(size_t)255;
// One record slot per ring entry: a big range's records wait in its entry's
// slot while the CTA goes on.
constexpr size_t BR_STRIDE = (BR_REC_OFF + RING * sizeof(tpx_record) * (size_t)BR_N + 255) & ~(size_t)255;
__device__ __forceinline__ tpx_record *br_stage(const Params &p, int slot) {
    return reinterpret_cast<tpx_record *>(p.big + (size_t)blockIdx.x * BR_STRIDE + BR_REC_OFF) + (size_t)slot * BR_N;
}


// block exclusive scan in thread order of two 16-bit halves added
// separately (__vadd2); each half's sums must fit it. Total in *total.
__device__ unsigned block_scan_vadd2(Smem &S, unsigned v, unsigned *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl = __vadd2(incl, u);
    }
    if (lane == 31) S.warp_int[w] = (int)incl;
    __syncthreads();
    if (w == 0) {
        const unsigned x = lane < NW ? (unsigned)S.warp_int[lane] : 0u;
        unsigned xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi = __vadd2(xi, u);
        }
        if (lane < NW) S.warp_int[lane] = (int)__vsub2(xi, x);
        if (lane == NW - 1) S.warp_int[NW] = (int)xi;
    }
    __syncthreads();
    const unsigned r = __vadd2((unsigned)S.warp_int[w], __vsub2(incl, v));
    *total = (unsigned)S.warp_int[NW];
    __syncthreads();
    return r;
}

// block exclusive scan of int; total in *total
__device__ int block_scan_int(Smem &S, int v, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) S.warp_int[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < NW ? S.warp_int[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += u;
        }
        if (lane < NW) S.warp_int[lane] = xi - x;
        if (lane == NW - 1) S.warp_int[NW] = xi;
    }
    __syncthreads();
    int r = S.warp_int[w] + incl - v;
    *total = S.warp_int[NW];
    __syncthreads();
    return r;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// once any wait has run out, every later wait gives up at once, so a broken
// chain costs one bounded wait, not one per tile
__device__ __forceinline__ bool timed_out(const Params &p) {
    return (*reinterpret_cast<volatile unsigned *>(&p.ctl->status) & ST_DEVTIMEOUT) != 0;
}

__device__ __forceinline__ GChain shfl_down_chain(const GChain &v, int o) {
    GChain u;
    u.n = __shfl_down_sync(0xffffffffu, v.n, o);
    u.first = __shfl_down_sync(0xffffffffu, v.first, o);
    u.last = __shfl_down_sync(0xffffffffu, v.last, o);
    u.sum = __shfl_down_sync(0xffffffffu, v.sum, o);
    return u;
}

// Bounded decoupled look-back, one warp. Each trip reads the flags of
// 32 * LB predecessors at once (lane l holds tiles hi - LB*l - j, j = 0 the
// latest), waits only for the tiles from hi down to the nearest inclusive
// prefix, and combines them in stream order. Two dependent L2 round trips
// per trip (flags, then values), so wide trips keep the chain short.
constexpr int LBC = 4;

// per lane: which of its LB tiles are needed this trip, given the flags
struct LbScan { unsigned need, inc; int stop; bool ok; };
template <int LB>
__device__ __forceinline__ LbScan lb_scan(const unsigned *flags, long long hi, long long lo, unsigned seq) {
    const int lane = threadIdx.x & 31;
    unsigned rdy = 0, inc = 0;
#pragma unroll
    for (int j = 0; j < LB; ++j) {
        const long long q = hi - LB * lane - j;
        if (q < lo) { rdy |= 1u << j; continue; }
        const unsigned f = ld_acquire(&flags[q]);
        if ((f >> 2) == seq && (f & 3u)) {
            rdy |= 1u << j;
            if ((f & 3u) == 2u) inc |= 1u << j;
        }
    }
    const unsigned im = __ballot_sync(0xffffffffu, inc != 0);
    LbScan r;
    r.stop = im ? __ffs(im) - 1 : 31;
    r.inc = inc;
    const unsigned all = (1u << LB) - 1u;
    r.need = lane < r.stop ? all : (lane == r.stop ? (inc ? ((inc & (0u - inc)) << 1) - 1u : all) : 0u);
    r.ok = (rdy & r.need) == r.need;
    return r;
}

// Decoupled look-back over the record counts of the tiles (and, in a batch,
// their trigger counts: .y), over all tiles of the call.
template <bool BATCH>
__device__ longlong2 lookback_count_warp(const Params &p, long long tile, unsigned seq, unsigned *status,
                                         bool block = true, bool *ready = nullptr) {
    const int lane = threadIdx.x & 31;
    longlong2 acc = make_longlong2(0, 0);
    for (long long hi = tile - 1; hi >= 0; hi -= 32 * LBC) {
        LbScan sc;
        long long spins = 0;
        for (;;) {
            sc = lb_scan<LBC>(p.ts.cflags, hi, 0, seq);
            if (__all_sync(0xffffffffu, sc.ok)) break;
            if (!block) { *ready = false; return acc; }   // not yet: the caller tries again later
            if (++spins > MAX_SPIN || timed_out(p)) {
                if (lane == 0) atomicOr(&p.ctl->status, ST_DEVTIMEOUT);
                *status |= ST_DEVTIMEOUT;
                return acc;
            }
            __nanosleep(64);
        }
        long long v = 0, w = 0;
#pragma unroll
        for (int j = 0; j < LBC; ++j) {
            const long long q = hi - LBC * lane - j;
            if (q < 0 || !((sc.need >> j) & 1u)) continue;
            const bool inc = (sc.inc >> j) & 1u;
            v += __ldcg(inc ? &p.ts.cpre[q] : &p.ts.cagg[q]);
            if (BATCH) w += __ldcg(inc ? &p.bt.tcpre[q] : &p.bt.tcagg[q]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
            if (BATCH) w += __shfl_xor_sync(0xffffffffu, w, o);
        }
        acc.x += v;
        acc.y += w;
        if (__any_sync(0xffffffffu, sc.inc != 0)) break;
    }
    return acc;
}

// The CC union-find array holds one 32-bit word per position: the parent in
// the lower half, in the upper half the pixel's second partner (NO_EXT: none;
// REWALK: more than two, re-walked at the unions). Finds look at the lower
// halves; writes keep the upper halves.
constexpr uint32_t NO_EXT = 0xFFFFu, REWALK = 0xFFFEu;
static_assert(C < (int)REWALK, "positions fit below the markers");
static_assert((C / 32) % 32 == 0, "the label bitmap splits evenly over a warp");

__device__ __forceinline__ uint32_t find_hw(uint32_t pbase, uint32_t x) {
    for (;;) {
        const uint32_t w = sh_ld(pbase + 4 * x);
        const uint32_t px = w & 0xFFFFu;
        if (px == x) return x;
        const uint32_t g = sh_ld(pbase + 4 * px) & 0xFFFFu;
        if (g == px) return px;
        sh_st(pbase + 4 * x, (w & 0xFFFF0000u) | g);   // path halving: g is an ancestor of x
        x = g;
    }
}

// lock-free union: the larger root position is linked under the smaller
__device__ void unite_hw(uint32_t pbase, uint32_t a, uint32_t b) {
    for (;;) {
        a = find_hw(pbase, a);
        b = find_hw(pbase, b);
        if (a == b) return;
        const uint32_t lo = min(a, b), hi = max(a, b);
        const uint32_t w = sh_ld(pbase + 4 * hi);
        if ((w & 0xFFFFu) == hi && sh_cas(pbase + 4 * hi, w, (w & 0xFFFF0000u) | lo) == w) return;
        a = lo;
        b = hi;   // hi was linked meanwhile: find again
    }
}

// a pixel with more than two partners: unite it with each partner in the
// forward half of its box (Sec. V.A), found again in the cell hash
template <int MODE>
__device__ void rewalk_unite(const Smem &S, const Params &p, uint32_t pbase, int q) {
    const uint64_t r = S.buf[pad(q)];
    const int x = r_x(r), y = r_y(r), sg = r_seg(r), tb = r_tof(r);
    for (int dx = 0; dx <= p.rx; ++dx) {
        const int cx = x + dx;
        if (cx > 255) break;
        for (int dy = (dx == 0 ? 0 : -p.ry); dy <= p.ry; ++dy) {
            const int cy = y + dy;
            if (cy < 0 || cy > 255) continue;
            for (uint32_t j = S.u1.head[hcell(sg, cx, cy)]; j != EMPTY; j = S.u2.next[j]) {
                if (!TPX_IN(j, C)) break;
                if (dx == 0 && dy == 0 && (int)j <= q) continue;
                const uint64_t rj = S.buf[pad((int)j)];
                if (r_x(rj) != cx || r_y(rj) != cy || r_seg(rj) != sg) continue;
                const int d = r_tof(rj) - tb;
                if (d < -p.dt || d > p.dt) continue;
                unite_hw(pbase, (uint32_t)q, j);
            }
        }
    }
}

// One warp resolves the record offset of tile tl holding nc records
// (decoupled look-back over the counts), publishes its inclusive count and,
// for the last tile, the call's totals; the offset is left in S.clo. In a
// batch the chain also carries the tile's nt triggers (offset in S.tlo), and a
// run's first tile records the run's record and trigger offsets.
// Without `block`, gives up (false, nothing published) when a predecessor's
// count is not out yet.
template <bool BATCH>
__device__ bool resolve_offset(Smem &S, const Params &p, unsigned seq, long long tl, int nc, long long ntr, int nt,
                               int run, bool run_first, bool block = true) {
    unsigned st2 = 0;
    longlong2 Ow = make_longlong2(0, 0);
    bool ready = true;
    if (tl > 0) Ow = lookback_count_warp<BATCH>(p, tl, seq, &st2, block, &ready);
    if (!ready) return false;
    if ((threadIdx.x & 31) == 0) {
        if (tl > 0 && tl + 1 != p.hold) {
            __stcg(&p.ts.cpre[tl], Ow.x + (long long)nc);
            if (BATCH) __stcg(&p.bt.tcpre[tl], Ow.y + (long long)nt);
            st_release(&p.ts.cflags[tl], (seq << 2) | 2u);
        }
        S.clo = Ow.x;
        S.tlo = Ow.y;
        if (st2) atomicOr(&S.status, st2);
        if (BATCH && run_first) {
            p.bt.run_rec_off[run] = Ow.x;
            p.bt.run_trig_off[run] = Ow.y;
        }
        if (tl == p.n_tiles - 1) {
            const long long nt_all = BATCH ? Ow.y + nt : ntr;
            *p.n_clusters = Ow.x + nc;
            *p.n_trig = nt_all;
            if (BATCH) {
                p.bt.run_rec_off[p.bt.n_runs] = Ow.x + nc;
                p.bt.run_trig_off[p.bt.n_runs] = nt_all;
            }
            if (Ow.x + nc > p.cl_cap) atomicOr(&p.ctl->status, ST_CLUSTER_CAP);
            if (nt_all > p.trig_cap) atomicOr(&p.ctl->status, ST_TRIG_CAP);
        }
    }
    return true;
}

// Staged output: a tile's records (in label order) and, in a batch, its
// trigger times wait in a staging slot of the CTA until a later tile of the
// CTA (or the end of the kernel) resolves their offset, when the
// predecessors' counts are long published; then one warp copies them out,
// coalesced, eight loads in flight per lane. The staged tiles form a ring
// (one entry for a single stream, RING in a batch): the oldest entries go out
// in order while their offsets resolve; the warp waits for the oldest only
// when the ring is full (the CTA needs the slot) or with `all` (the kernel's
// end). Called by one whole warp.
template <bool BATCH>
__device__ void flush_ring_warp(Smem &S, const Params &p, unsigned seq, bool all) {
    constexpr int NP = BATCH ? RING : 1;
    const int lane = threadIdx.x & 31;
    constexpr int WPR = (int)(sizeof(tpx_record) / 8);
    for (;;) {
        const int cnt = S.pend_count;
        if (cnt == 0) break;
        const int slot = S.pend_head;
        const long long pt = S.pend[slot].tile, ntr = S.pend[slot].ntr;
        const int nc = S.pend[slot].ncl, nt = S.pend[slot].ntdc, run = S.pend[slot].run;
        const bool first = S.pend[slot].first, big = S.pend[slot].big;
        if (!resolve_offset<BATCH>(S, p, seq, pt, nc, ntr, nt, run, first, all || cnt == NP)) break;
        __syncwarp();
        const long long O = S.clo;
        const long long keep = min((long long)nc, max(0LL, p.cl_cap - O));
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(
            (BATCH && big) ? br_stage(p, slot) : p.stage + ((long long)blockIdx.x * NP + slot) * C);
        if (p.rec64) {   // 64-byte records: the first 8 words of each staged record
            unsigned long long *d64 = reinterpret_cast<unsigned long long *>(p.clusters) + O * 8;
            const long long nw = keep * 8;
            for (long long w0 = lane; w0 < nw; w0 += 32 * 8) {
                unsigned long long v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const long long w = w0 + 32 * u;
                    v[u] = w < nw ? __ldcg(src + (w >> 3) * WPR + (w & 7)) : 0ull;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (w0 + 32 * u < nw) d64[w0 + 32 * u] = v[u];
            }
        }
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(p.clusters + O);
        const long long nw = p.rec64 ? 0 : keep * WPR;
        for (long long w0 = lane; w0 < nw; w0 += 32 * 8) {
            unsigned long long v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = w0 + 32 * u < nw ? __ldcg(src + w0 + 32 * u) : 0ull;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (w0 + 32 * u < nw) dst[w0 + 32 * u] = v[u];
        }
        if (BATCH) {
            const long long TO = S.tlo;
            const long long tkeep = min((long long)nt, max(0LL, p.trig_cap - TO));
            const long long *ts = p.bt.tstage + ((long long)blockIdx.x * NP + slot) * T;
            for (long long i = lane; i < tkeep; i += 32) p.trig[TO + i] = __ldcg(ts + i);
        }
        __syncwarp();
        if (lane == 0) {
            S.pend_head = (slot + 1) % NP;
            S.pend_count = cnt - 1;
        }
        __syncwarp();
    }
}

// the exact integer moments of one cluster from its member list (Sec. V.C)
// and its canonical label: the earliest member in (time, position) order
struct Moments {
    long long s_tot, s_x, s_y, s_tt;   // s_tt: sum of ToT x biased ToF
    int n, npk;
    uint32_t best_lo;                  // label position
    int tofb0;                         // its biased ToF
};

__device__ __forceinline__ Moments walk_members(const Smem &S, const Params &p, uint32_t head) {
    const uint16_t *mnext = reinterpret_cast<const uint16_t *>(S.parent);
    uint64_t best = ~0ull;
    Moments m{0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t k = head; k != EMPTY; k = mnext[k]) {
        if (!TPX_IN(k, C)) break;
        const uint64_t rm = S.buf[pad((int)k)];
        const long long tot = r_tot(rm);
        const int tf = r_tof(rm);
        best = min(best, ((uint64_t)tf << 16) | k);
        m.n += 1;
        m.npk += (S.notpeak[k] & 1) ? 0 : 1;
        m.s_tot += tot;
        m.s_x += tot * r_x(rm);
        m.s_y += tot * r_y(rm);
        m.s_tt += tot * (long long)tf;
    }
    m.best_lo = (uint32_t)(best & 0xFFFFu);
    m.tofb0 = (int)(best >> 16);
    return m;
}

// the record of a cluster whose label pixel lies at position best_lo of the
// tile at stream position base
__device__ __forceinline__ void put_record(tpx_record *dst, const Moments &m, const Smem &S, const Params &p,
                                           long long base, long long shot0) {
    const int seg = r_seg(S.buf[pad((int)m.best_lo)]);
    const long long tofc0 = (long long)m.tofb0 - kTofBias;
    const long long s_t = m.s_tt - (long long)m.tofb0 * m.s_tot;
    tpx_record o;
    o.label = p.idx_base + base + m.best_lo;
    o.shot = shot0 + seg;
    o.t0 = S.tdc_t[seg] + tofc0;
    o.s_tot = m.s_tot; o.s_x = m.s_x; o.s_y = m.s_y; o.s_t = s_t;
    o.n = m.n; o.n_peaks = m.npk;
    com_from_moments(m.s_x, m.s_y, s_t, m.s_tot, tofc0, &o.x, &o.y, &o.tof);
    *dst = o;
}

// a record at position idx of the caller's buffer (88 bytes, or its first 64
// with TPX_FLAG_RECORDS64)
__device__ __forceinline__ void out_record(const Params &p, long long idx, const tpx_record &o) {
    if (p.rec64) {
        const unsigned long long *w = reinterpret_cast<const unsigned long long *>(&o);
        unsigned long long *d = reinterpret_cast<unsigned long long *>(p.clusters) + idx * 8;
#pragma unroll
        for (int k = 0; k < 8; ++k) d[k] = w[k];
    } else {
        p.clusters[idx] = o;
    }
}

// rank of label position lp among the tile's labels (after the bitmap scan)
__device__ __forceinline__ int label_rank(const Smem &S, uint32_t lp) {
    return (int)S.lpre[lp >> 5] + __popc(S.lbits[lp >> 5] & ((1u << (lp & 31)) - 1u));
}

// ------------------------------------------------------------- big ranges
// A range longer than the range capacity C (in CC mode: a shot of more pixels
// than a tile holds) stays in the launch. The CTA decodes the whole range
// into its own global scratch (the tile's unwrap, binning and cut, Sec.
// IV.A-C), sorts the kept pixels by (shot, time bin, 8-column x stripe)
// with bins at least dt + 1 ticks wide, and compares each pixel with the
// pixels of the keys before its own that can hold a neighbour: the previous
// bin's three stripes around its own, its own bin's stripe to the left, and
// its own key up to itself. Two adjacent pixels (Sec. V.A: same shot, box
// neighbours, |dt| within the radius) lie in the same or consecutive bins
// and stripes, so every adjacent pair is seen once, as in the tile's
// neighbour pass. Union-find over the sorted order runs in shared
// memory (16-bit parents, roots linked by a hashed priority). The
// exact integer moments of each cluster (Sec. V.C) are gathered with
// warp-aggregated atomics, and the records are staged in label order in the
// scratch (copied out like a tile's). A range this cannot hold either goes
// back to the general path with its run: more than BR_L positions, BR_N
// kept pixels or BR_S shots.
// 16-bit parents addressed in the shared window (pb: the array's shared
// address), as the tile's union-find addresses its words
__device__ __forceinline__ unsigned br_ld(uint32_t pb, unsigned x) {
    unsigned short v;
    asm volatile("ld.volatile.shared.u16 %0, [%1];" : "=h"(v) : "r"(pb + 2 * x) : "memory");
    return v;
}
__device__ __forceinline__ void br_st(uint32_t pb, unsigned x, unsigned v) {
    asm volatile("st.volatile.shared.u16 [%0], %1;" ::"r"(pb + 2 * x), "h"((unsigned short)v) : "memory");
}
__device__ __forceinline__ unsigned br_cas(uint32_t pb, unsigned x, unsigned cmp, unsigned v) {
    unsigned short o;
    asm volatile("atom.shared.cas.b16 %0, [%1], %2, %3;"
                 : "=h"(o) : "r"(pb + 2 * x), "h"((unsigned short)cmp), "h"((unsigned short)v) : "memory");
    return o;
}
__device__ __forceinline__ void br_or(uint32_t a, unsigned v) {
    asm volatile("red.shared.or.b32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned br_find(uint32_t pb, unsigned x) {
    for (;;) {
        const unsigned px = br_ld(pb, x);
        if (px == x) return x;
        const unsigned g = br_ld(pb, px);
        if (g == px) return px;
        br_st(pb, x, g);   // path halving: g is an ancestor of x
        x = g;
    }
}
// The root of a big-range cluster need not be any particular pixel (its
// label comes from its moments), so roots are linked by a hashed priority,
// the lower under the higher: the sorted order puts a cluster's pixels on
// consecutive slots, and linking by slot would chain them. Links always rise
// in (priority, slot) order, so the forest stays acyclic.
__device__ __forceinline__ unsigned br_prio(unsigned x) { return ((x * 0x9E3779B1u) & 0xFFFF0000u) | x; }
__device__ __forceinline__ void br_unite(uint32_t pb, unsigned a, unsigned b) {
    for (;;) {
        a = br_find(pb, a);
        b = br_find(pb, b);
        if (a == b) return;
        const bool a_low = br_prio(a) < br_prio(b);
        const unsigned child = a_low ? a : b, up = a_low ? b : a;
        const unsigned old = br_cas(pb, child, child, up);
        if (old == child) return;
        if (a_low) a = old; else b = old;   // the child was linked meanwhile
    }
}

// The range of the tile at stream position `base` (first trigger packet at
// f): its cluster count, or -1 with a status bit set when it goes back to
// the general path. Called by every thread of the CTA after the tile's
// staging slot is free; writes the labels, local-maximum flags and staged
// records, and replaces the tile's keep / drop counts by the whole range's.
#ifdef TPX_PHASE_TIMING
#define BR_PH(k)                                                                          \
    do {                                                                                  \
        const long long ph_now = clock64();                                               \
        if ((threadIdx.x & 31) == 0) atomicAdd(&S.ph[k], (unsigned long long)(ph_now - br_t)); \
        br_t = ph_now;                                                                    \
    } while (0)
#else
#define BR_PH(k) do {} while (0)
#endif
template <bool BATCH>
__device__ __noinline__ int big_range(Smem &S, const Params &p, long long base, long long rend, int f,
                                      bool prev_global) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
#ifdef TPX_PHASE_TIMING
    long long br_t = clock64();
#endif
    const long long tp = p.thr_pix, tt = p.thr_tdc;
    unsigned char *R = reinterpret_cast<unsigned char *>(&S);
    uint16_t *par = reinterpret_cast<uint16_t *>(R);
    unsigned *npk = reinterpret_cast<unsigned *>(R + 2 * BR_N);
    unsigned *bins = npk + BR_N / 32;
    unsigned *lbits = bins + BR_BINS + 4;
    uint16_t *lpre = reinterpret_cast<uint16_t *>(lbits + BR_LW);
    int *sg_n = reinterpret_cast<int *>(lpre + BR_LW);
    int *sg_lo = sg_n + BR_S, *sg_hi = sg_lo + BR_S, *sg_b0 = sg_hi + BR_S, *sg_w = sg_b0 + BR_S;
    // misc: [0..2] range-end slots, [3] first pixel, [4] kept, [5] dropped
    // before a trigger, [6] background, [7] failure bits, [8] clusters, [9]
    // peaks, [12] the neighbour pass's task counter
    int *misc = sg_w + BR_S;
    uint64_t *sbuf = reinterpret_cast<uint64_t *>(misc + 16);   // [BR_SB] staged sorted records
    unsigned char *G = p.big + (size_t)blockIdx.x * BR_STRIDE;
    uint64_t *g_rec = reinterpret_cast<uint64_t *>(G);
    uint64_t *g_srec = g_rec + (BR_L + 1);
    uint16_t *g_spos = reinterpret_cast<uint16_t *>(g_srec + BR_N);
    BrMom *g_mom = reinterpret_cast<BrMom *>(g_spos + BR_N);
    const GAgg E = S.E;
    const uint32_t pb = (uint32_t)__cvta_generic_to_shared(par);      // shared addresses
    const uint32_t nb_sh = (uint32_t)__cvta_generic_to_shared(npk);
    const int rx = p.rx, ry = p.ry, dtr = p.dt;
    __syncthreads();
    if (tid < 16) misc[tid] = tid < 4 ? INT_MAX : 0;
    __syncthreads();

    // ---- the range end: the first TDC packet at or past C (the tile
    // searched the positions below C); four packets per thread per step, the
    // steps' minima rotating over three slots as in the tile's look-ahead ----
    int L = 0;
    bool term = false;
    {
        constexpr int STEP = 4 * NT;
        long long q0 = C;
        for (int k = 0;; ++k) {
            const long long lim = min((long long)BR_L, rend - base);
            if (q0 >= lim) { L = (int)lim; break; }
            if (tid == 0) misc[(k + 1) % 3] = INT_MAX;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long q = q0 + u * NT + tid;
                if (q < lim && (__ldcg(p.pk + base + q) >> 60) == 0x6u) atomicMin(&misc[k % 3], (int)q);
            }
            __syncthreads();
            const int lf = misc[k % 3];
            if (lf != INT_MAX) { L = lf + 1; term = true; break; }
            q0 += STEP;
        }
    }
    // not terminated before the position limit while the run goes on
    if (!term && base + L < rend) { if (tid == 0) atomicOr(&S.status, ST_CAPACITY); return -1; }

    // ---- walk 2 over [0, L): wrap steps and TDC counts per contiguous chunk ----
    const int kpd = (L + NT - 1) / NT;
    const int p0 = tid * kpd;
    int ntd = 0, jp = 0;
    {
        int lpx = -1, fpx = INT_MAX;
        long long lr = 0;
        for (int j = 0; j < kpd; ++j) {
            const int q = p0 + j;
            if (q >= L) break;
            const uint64_t w = __ldg(p.pk + base + q);
            const unsigned h = (unsigned)(w >> 60);
            if (h == 0xBu) {
                const long long r = pix_raw(w);
                if (lpx >= 0) jp += (int)jump(r - lr, tp); else fpx = q;
                lpx = q;
                lr = r;
            } else if (h == 0x6u) {
                ++ntd;
            }
        }
        if (lpx >= 0) {
            for (int q = p0 + kpd; q < L; ++q) {
                const uint64_t w = __ldg(p.pk + base + q);
                if ((w >> 60) == 0xBu) { jp += (int)jump(pix_raw(w) - lr, tp); break; }
            }
        }
        const int fw = (int)__reduce_min_sync(0xffffffffu, (unsigned)fpx);
        if (lane == 0 && fw != INT_MAX) atomicMin(&misc[3], fw);
    }
    unsigned pk_tot;
    const unsigned pk_ex = block_scan_vadd2(S, ((unsigned)ntd << 16) | ((unsigned)jp & 0xFFFFu), &pk_tot);
    const int li0 = (int)(pk_ex >> 16);
    const int nseg = (int)(pk_tot >> 16);
    const int jp_ex = (int)(short)(pk_ex & 0xFFFFu);
    if (nseg > BR_S || nseg > MAXSEG) { if (tid == 0) atomicOr(&S.status, ST_CAPACITY); return -1; }
    if (tid == 0) {
        const int fp = misc[3];
        S.j0 = (fp != INT_MAX && E.pix.n > 0) ? jump(pix_raw(__ldcg(p.pk + base + fp)) - E.pix.last, tp) : 0;
    }
    if (ntd) {
        int li = li0;
        for (int j = 0; j < kpd; ++j) {
            const int q = p0 + j;
            if (q >= L) break;
            if ((__ldg(p.pk + base + q) >> 60) != 0x6u) continue;
            S.tdc_pos[li] = (uint16_t)q;
            ++li;
        }
    }
    for (int s = tid; s < nseg; s += NT) { sg_n[s] = 0; sg_lo[s] = INT_MAX; sg_hi[s] = INT_MIN; }
    __syncthreads();
    // the trigger times (one warp, a scan of the TDC wrap steps)
    if (tid < 32) {
        bool has = E.tdc.n > 0;
        long long last = E.tdc.last, ep = E.tdc.sum, t_last = 0;
        for (int i0 = 0; i0 < nseg; i0 += 32) {
            const int i = i0 + lane;
            long long r = 0;
            if (i < nseg) r = tdc_raw(__ldcg(p.pk + base + S.tdc_pos[i]));
            const long long rp = __shfl_up_sync(0xffffffffu, r, 1);
            int st = 0;
            if (i < nseg && (lane > 0 || has)) st = (int)jump(r - (lane > 0 ? rp : last), tt);
            int inc = st;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            const long long t = r + (ep + inc) * kTdcPeriod;
            const long long tp_ = __shfl_up_sync(0xffffffffu, t, 1);
            if (i < nseg) {
                S.tdc_t[i] = t;
                if ((lane > 0 || i0 > 0) && t < (lane > 0 ? tp_ : t_last)) atomicOr(&p.ctl->status, ST_TRIG_ORDER);
            }
            const int lastl = min(31, nseg - 1 - i0);
            ep += __shfl_sync(0xffffffffu, inc, lastl);
            last = __shfl_sync(0xffffffffu, r, lastl);
            t_last = __shfl_sync(0xffffffffu, t, lastl);
            has = true;
        }
    }
    __syncthreads();

    BR_PH(20);
    // ---- walk 4 over [0, L): shot, cut, timewalk, packed record per position
    // (the tile's rule), and each shot's kept count and ToF span ----
    {
        long long ep = E.pix.sum + S.j0 + jp_ex;
        bool has = false;
        long long last = 0;
        int seg = li0 - 1;
        const long long t_prev_global = E.tdc.last + E.tdc.sum * kTdcPeriod;
        int c_keep = 0, c_pre = 0, c_bg = 0;
        bool exc = false;
        int cs = -1, cn = 0, clo = INT_MAX, chi = INT_MIN;   // the current shot's running stats
        for (int j = 0; j < kpd; ++j) {
            const int q = p0 + j;
            if (q >= L) break;
            const uint64_t w = __ldg(p.pk + base + q);
            const unsigned h = (unsigned)(w >> 60);
            uint64_t rec = INVALID;
            if (h == 0x6u) {
                ++seg;
            } else if (h == 0xBu) {
                const long long r = pix_raw(w);
                if (has) ep += jump(r - last, tp);
                has = true;
                last = r;
                const long long t = r + ep * kPixPeriod;
                if (seg < 0) {
                    if (!prev_global) ++c_pre;
                } else if (seg < nseg) {
                    const long long t_lo = S.tdc_t[seg];
                    const bool has_hi = seg + 1 < nseg;
                    int verdict;                      // 0 keep, 1 bg, 2 pre, 3 undecidable here
                    if (has_hi && t >= S.tdc_t[seg + 1]) verdict = 3;
                    else if (t >= t_lo) verdict = (t - t_lo > p.tof_max) ? 1 : 0;
                    else {
                        const bool hp = seg > 0 || prev_global;
                        const long long tprev = seg > 0 ? S.tdc_t[seg - 1] : t_prev_global;
                        if (!hp) verdict = 2;
                        else if (t >= tprev) verdict = (t - tprev > p.tof_max) ? 1 : 3;
                        else verdict = 3;
                    }
                    if (verdict == 0) {
                        const int tot = pix_tot(w);
                        const long long tc = t - (p.lut ? (long long)p.lut[tot] : 0LL);
                        const int tofb = (int)(tc - t_lo + kTofBias);
                        rec = mkrec((uint32_t)tofb, (uint32_t)seg, (uint32_t)tot, (uint32_t)pix_x(w), (uint32_t)pix_y(w));
                        ++c_keep;
                        if (seg != cs) {
                            if (cs >= 0) { atomicAdd(&sg_n[cs], cn); atomicMin(&sg_lo[cs], clo); atomicMax(&sg_hi[cs], chi); }
                            cs = seg; cn = 0; clo = INT_MAX; chi = INT_MIN;
                        }
                        ++cn;
                        clo = min(clo, tofb);
                        chi = max(chi, tofb);
                    } else if (verdict == 1) ++c_bg;
                    else if (verdict == 2) ++c_pre;
                    else exc = true;
                }
            }
            g_rec[q] = rec;
        }
        if (cs >= 0) { atomicAdd(&sg_n[cs], cn); atomicMin(&sg_lo[cs], clo); atomicMax(&sg_hi[cs], chi); }
        c_keep = (int)warp_sum((unsigned long long)c_keep);
        c_pre = (int)warp_sum((unsigned long long)c_pre);
        c_bg = (int)warp_sum((unsigned long long)c_bg);
        if (lane == 0) {
            atomicAdd(&misc[4], c_keep);
            atomicAdd(&misc[5], c_pre);
            atomicAdd(&misc[6], c_bg);
        }
        if (exc) atomicOr(&misc[7], (int)ST_EXCEPTION);
    }
    __syncthreads();
    const int N = misc[4];
    if (misc[7] || N > BR_N) {
        if (tid == 0) atomicOr(&S.status, misc[7] ? (unsigned)misc[7] : ST_CAPACITY);
        return -1;
    }

    BR_PH(21);
    // ---- time bins: each shot gets a share of the bins by its kept count,
    // each bin at least dt + 1 ticks wide (one warp); a key is a (bin,
    // stripe) pair ----
    // stripes at least rx wide; fewer when the shots need the time bins
    // (every shot takes at least one)
    int NS = rx <= 256 / BR_NS ? BR_NS : (rx <= 2 * 256 / BR_NS ? BR_NS / 2 : 1);
    while (NS > 1 && BR_BINS / NS < 2 * nseg) NS = NS > BR_NS / 2 ? BR_NS / 2 : 1;
    const int SW = 256 / NS;   // stripe width (columns)
    const int TB = BR_BINS / NS;   // time bins over all shots
    if (wid == 0) {
        constexpr int SPL = BR_S / 32;   // shots per lane
        int nb[SPL], tot = 0;
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
            const int s = lane * SPL + k;
            const int n = s < nseg ? sg_n[s] : 0;
            nb[k] = s < nseg ? (n > 0 ? 1 + (int)(((long long)(TB - nseg) * n) / N) : 1) : 0;
            tot += nb[k];
        }
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        int b0 = incl - tot;
#pragma unroll
        for (int k = 0; k < SPL; ++k) {
            const int s = lane * SPL + k;
            if (s < nseg) {
                sg_b0[s] = b0;
                const long long span = sg_n[s] > 0 ? (long long)sg_hi[s] - sg_lo[s] + 1 : 1;
                sg_w[s] = (int)max((long long)dtr + 1, (span + nb[k] - 1) / nb[k]);
                if (sg_n[s] == 0) sg_lo[s] = 0;
            }
            b0 += nb[k];
        }
    }
    for (int b = tid; b < BR_BINS; b += NT) bins[b] = 0u;
    __syncthreads();
    auto bin_of = [&](uint64_t r) -> int {
        const int s = r_seg(r);
        return (sg_b0[s] + (r_tof(r) - sg_lo[s]) / sg_w[s]) * NS + r_x(r) / SW;
    };
    // ---- counting sort of the kept pixels by bin ----
    for (int q = tid; q < L; q += NT) {
        const uint64_t r = g_rec[q];
        if (r != INVALID) atomicAdd(&bins[bin_of(r)], 1u);
    }
    __syncthreads();
    {
        constexpr int BPT = BR_BINS / NT;   // bins per thread, contiguous
        unsigned c[BPT], s = 0;
#pragma unroll
        for (int k = 0; k < BPT; ++k) { c[k] = bins[tid * BPT + k]; s += c[k]; }
        int total;
        unsigned run = (unsigned)block_scan_int(S, (int)s, &total);
#pragma unroll
        for (int k = 0; k < BPT; ++k) { bins[tid * BPT + k] = run; run += c[k]; }
    }
    __syncthreads();
    for (int q = tid; q < L; q += NT) {
        const uint64_t r = g_rec[q];
        if (r == INVALID) continue;
        const unsigned slot = atomicAdd(&bins[bin_of(r)], 1u);
        if (!TPX_IN(slot, N)) continue;
        g_srec[slot] = r;
        g_spos[slot] = (uint16_t)q;
    }
    // bins[b] is now the end of bin b (the start of bin b + 1)
    for (int i = tid; i < N; i += NT) par[i] = (uint16_t)i;
    for (int w = tid; w < BR_N / 32; w += NT) npk[w] = 0u;
    for (int w = tid; w < BR_LW; w += NT) lbits[w] = 0u;
    __syncthreads();

    BR_PH(22);
    // ---- neighbour pass: every pixel of the sorted order is checked against
    // the keys that can hold its earlier neighbours (the box rule, Sec. V.A);
    // an adjacent pair clears the loser's local-maximum flag (Sec. V.B: the
    // larger ToT wins, equal ToT goes to the later pixel) and unites. The
    // sorted records are read through shared memory: BR_CH pixels at a time,
    // staged with the records before them from the start of the first one's
    // previous time bin (or straight from the scratch when those do not fit) ----
    auto kstart = [&](int k) -> int { return k > 0 ? (int)bins[k - 1] : 0; };   // a key's first slot
    for (int a = 0; a < N; a += BR_CH) {
        const int e = min(N, a + BR_CH);
        int lo;
        {
            const uint64_t ra = g_srec[a];
            const int s = r_seg(ra);
            const int tbin = sg_b0[s] + (r_tof(ra) - sg_lo[s]) / sg_w[s];
            const int k0 = (tbin > sg_b0[s] ? tbin - 1 : tbin) * NS;
            lo = k0 > 0 ? (int)bins[k0 - 1] : 0;
        }
        const bool fits = e - lo <= BR_SB;
        if (tid == 0) misc[12] = 0;   // the chunk's task counter
        if (fits)
            for (int j = lo + tid; j < e; j += NT) sbuf[j - lo] = g_srec[j];
        __syncthreads();
        auto rec_at = [&](int j) -> uint64_t { return fits ? sbuf[j - lo] : g_srec[j]; };
        // A warp takes 32 consecutive pixels at a time, the next task from the
        // chunk's counter (dense stretches take longer). A pixel's candidates
        // are two runs of consecutive slots: the previous bin's stripes around
        // its own (consecutive keys), and its own bin's left stripe with its
        // own key up to itself. The warp spreads all its (pixel, candidate)
        // pairs evenly over its lanes: a prefix of the pixels' candidate
        // counts, and each lane finds the pixel of its pair by a search over
        // the lanes.
        const int ntask = (e - a + 31) >> 5;
        for (;;) {
            int task = 0;
            if (lane == 0) task = atomicAdd(&misc[12], 1);
            task = __shfl_sync(0xffffffffu, task, 0);
            if (task >= ntask) break;
            const int i0 = a + 32 * task;
            const int i = i0 + lane;
            int a0 = 0, la = 0, b0 = 0, lb = 0;
            if (i < e) {
                const uint64_t ri = rec_at(i);
                const int s = r_seg(ri);
                const int tbin = sg_b0[s] + (r_tof(ri) - sg_lo[s]) / sg_w[s];
                const int st = r_x(ri) / SW;
                if (tbin > sg_b0[s]) {
                    a0 = kstart((tbin - 1) * NS + max(st - 1, 0));
                    la = (int)bins[(tbin - 1) * NS + min(st + 1, NS - 1)] - a0;
                }
                b0 = kstart(tbin * NS + max(st - 1, 0));
                lb = i - b0;
            }
            const int n = la + lb;
            int incl = n;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            const int off = incl - n;
            const int W = __shfl_sync(0xffffffffu, incl, 31);
            for (int wb = 0; wb < W; wb += 32) {
                const int w = wb + lane;
                int q = 0;   // the last lane whose pairs start at or before w
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int o = __shfl_sync(0xffffffffu, off, q + step);
                    if (o <= w) q += step;
                }
                const int qa0 = __shfl_sync(0xffffffffu, a0, q), qla = __shfl_sync(0xffffffffu, la, q);
                const int qb0 = __shfl_sync(0xffffffffu, b0, q), qoff = __shfl_sync(0xffffffffu, off, q);
                if (w >= W) continue;
                const int c = w - qoff;
                const int ip = i0 + q;
                const int j = c < qla ? qa0 + c : qb0 + (c - qla);
                const uint64_t rp = rec_at(ip), rj = rec_at(j);
                const int dx = r_x(rj) - r_x(rp), dy = r_y(rj) - r_y(rp);
                if (dx < -rx || dx > rx || dy < -ry || dy > ry || !within(r_tof(rj) - r_tof(rp), dtr)) continue;
                const int tj = r_tot(rj), tp = r_tot(rp);
                const bool j_wins = tj > tp || (tj == tp && g_spos[j] > g_spos[ip]);
                const int loser = j_wins ? ip : j;
                br_or(nb_sh + 4 * (loser >> 5), 1u << (loser & 31));
                br_unite(pb, (unsigned)ip, (unsigned)j);
            }
        }
        __syncthreads();
    }
    BR_PH(23);
    // compress: every pixel points to its root
    for (int i = tid; i < N; i += NT) br_st(pb, (unsigned)i, br_find(pb, (unsigned)i));
    __syncthreads();
    // roots: their moment records cleared, counted
    {
        int k = 0;
        for (int i = tid; i < N; i += NT) {
            if (par[i] != i) continue;
            ++k;
            unsigned long long *m = reinterpret_cast<unsigned long long *>(&g_mom[i]);
#pragma unroll
            for (int u = 0; u < 5; ++u) __stcg(m + u, u == 4 ? ~0ull : 0ull);
            __stcg(m + 5, 0ull);
        }
        k = (int)warp_sum((unsigned long long)k);
        if (lane == 0 && k) atomicAdd(&misc[8], k);
    }
    __syncthreads();
    const int K = misc[8];

    BR_PH(24);
    // ---- moments: a warp's lanes sharing a root add up among themselves, one
    // lane per root adds to its record ----
    for (int i0 = wid * 32; i0 < N; i0 += NT) {
        const int i = i0 + lane;
        const bool v = i < N;
        const unsigned r = v ? par[i] : 0xFFFFFFFFu;
        const uint64_t ri = v ? g_srec[i] : 0ull;
        const unsigned pos = v ? g_spos[i] : 0u;
        const unsigned tot = (unsigned)r_tot(ri), tofb = (unsigned)r_tof(ri);
        const unsigned ux = tot * (unsigned)r_x(ri), uy = tot * (unsigned)r_y(ri);
        const unsigned long long utt = (unsigned long long)tot * tofb;
        const bool pk = v && !((npk[i >> 5] >> (i & 31)) & 1u);
        unsigned act = __ballot_sync(0xffffffffu, v);
        unsigned c_pk = 0;
        while (act) {
            const int ld = __ffs(act) - 1;
            const unsigned r0 = __shfl_sync(0xffffffffu, r, ld);
            const bool mine = v && r == r0;
            const unsigned grp = __ballot_sync(0xffffffffu, mine);
            const unsigned a_tot = __reduce_add_sync(0xffffffffu, mine ? tot : 0u);
            const unsigned a_x = __reduce_add_sync(0xffffffffu, mine ? ux : 0u);
            const unsigned a_y = __reduce_add_sync(0xffffffffu, mine ? uy : 0u);
            const unsigned a_tl = __reduce_add_sync(0xffffffffu, mine ? (unsigned)(utt & 0xFFFFFFu) : 0u);
            const unsigned a_th = __reduce_add_sync(0xffffffffu, mine ? (unsigned)(utt >> 24) : 0u);
            const unsigned m_t = __reduce_min_sync(0xffffffffu, mine ? tofb : 0xFFFFFFFFu);
            const unsigned m_p = __reduce_min_sync(0xffffffffu, (mine && tofb == m_t) ? pos : 0xFFFFFFFFu);
            const unsigned n_pk = __popc(__ballot_sync(0xffffffffu, mine && pk));
            if (lane == ld && TPX_IN(r0, N)) {
                BrMom &M = g_mom[r0];
                atomicAdd(&M.s_tot, (unsigned long long)a_tot);
                atomicAdd(&M.s_x, (unsigned long long)a_x);
                atomicAdd(&M.s_y, (unsigned long long)a_y);
                atomicAdd(&M.s_tt, ((unsigned long long)a_th << 24) + a_tl);
                atomicMin(&M.best, ((unsigned long long)m_t << 16) | m_p);
                atomicAdd(&M.n, (unsigned)__popc(grp));
                atomicAdd(&M.npk, n_pk);
            }
            c_pk += n_pk;
            act &= ~grp;
        }
        if (lane == 0 && c_pk) atomicAdd(&misc[9], (int)c_pk);
    }
    __syncthreads();
    BR_PH(25);
    // ---- the labels (each cluster's earliest pixel in (time, position)
    // order) marked in the bitmap, then their ranks ----
    for (int i = tid; i < N; i += NT) {
        if (par[i] != i) continue;
        const unsigned lp = (unsigned)(__ldcg(&g_mom[i].best) & 0xFFFFu);
        atomicOr(&lbits[lp >> 5], 1u << (lp & 31));
    }
    __syncthreads();
    {
        constexpr int WPT = BR_LW / NT;
        unsigned c[WPT], s = 0;
#pragma unroll
        for (int k = 0; k < WPT; ++k) { c[k] = (unsigned)__popc(lbits[tid * WPT + k]); s += c[k]; }
        int total;
        unsigned run = (unsigned)block_scan_int(S, (int)s, &total);
#pragma unroll
        for (int k = 0; k < WPT; ++k) { lpre[tid * WPT + k] = (uint16_t)run; run += c[k]; }
    }
    __syncthreads();
    // ---- records, staged in label order ----
    tpx_record *dst = br_stage(p, (S.pend_head + S.pend_count) % RING);   // the ring entry this tile takes
    for (int i = tid; i < N; i += NT) {
        if (par[i] != i) continue;
        const unsigned long long *m = reinterpret_cast<const unsigned long long *>(&g_mom[i]);
        const long long s_tot = (long long)__ldcg(m), s_x = (long long)__ldcg(m + 1), s_y = (long long)__ldcg(m + 2);
        const long long s_tt = (long long)__ldcg(m + 3);
        const unsigned long long best = __ldcg(m + 4), nn = __ldcg(m + 5);
        const unsigned lp = (unsigned)(best & 0xFFFFu);
        const int tofb0 = (int)(best >> 16);
        const int k = (int)lpre[lp >> 5] + __popc(lbits[lp >> 5] & ((1u << (lp & 31)) - 1u));
        if (!TPX_IN(k, K) || !TPX_IN(lp, L)) continue;
        const int seg = r_seg(g_rec[lp]);
        const long long tofc0 = (long long)tofb0 - kTofBias;
        tpx_record o;
        o.label = p.idx_base + base + lp;
        o.shot = E.tdc.n + seg;
        o.t0 = S.tdc_t[seg] + tofc0;
        o.s_tot = s_tot; o.s_x = s_x; o.s_y = s_y;
        o.s_t = s_tt - (long long)tofb0 * s_tot;
        o.n = (int)(nn & 0xFFFFFFFFu);
        o.n_peaks = (int)(nn >> 32);
        com_from_moments(o.s_x, o.s_y, o.s_t, s_tot, tofc0, &o.x, &o.y, &o.tof);
        dst[k] = o;
    }
    // ---- per-packet outputs over the range's label span ----
    if (p.labels || p.labels32 || p.is_peak) {
        for (int i = tid; i < N; i += NT) {
            const long long q = g_spos[i];
            const unsigned lp = (unsigned)(__ldcg(&g_mom[par[i]].best) & 0xFFFFu);
            const uint8_t pk = ((npk[i >> 5] >> (i & 31)) & 1u) ? 0 : 1;
            if (!TPX_IN(base + q, rend)) continue;
            if (p.labels) p.labels[base + q] = p.idx_base + base + lp;
            else if (p.labels32) p.labels32[base + q] = (int)(p.idx_base - p.lab32_base + base + lp);
            if (p.is_peak) p.is_peak[base + q] = pk;
        }
        const int W0 = prev_global ? f : 0, W1 = term ? L - 1 : L;
        for (int q = W0 + tid; q < W1; q += NT) {
            if (g_rec[q] != INVALID || !TPX_IN(base + q, rend)) continue;
            if (p.labels) p.labels[base + q] = -1LL;
            else if (p.labels32) p.labels32[base + q] = -1;
            if (p.is_peak) p.is_peak[base + q] = 0;
        }
    }
    __syncthreads();
    BR_PH(26);
    if (tid == 0) {
        S.cnt[C_KEPT] = (unsigned long long)misc[4];
        S.cnt[C_DROP_PRE] = (unsigned long long)misc[5];
        S.cnt[C_DROP_BG] = (unsigned long long)misc[6];
        S.cnt[C_PEAKS] += (unsigned long long)misc[9];
    }
    __syncthreads();
    return K;
}

// ------------------------------------------------------------------- kernel
template <int MODE, bool STAGED, bool BATCH>
__global__ void __launch_bounds__(NT, MINB) fused_kernel(const Params p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &S = *reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31;
    const long long tp = p.thr_pix, tt = p.thr_tdc;
    const unsigned seq = p.seq & 0x3FFFFFFFu;
    const uint32_t pbase = (uint32_t)__cvta_generic_to_shared(S.parent);
    // ranges past the capacity go through the big-range path (CC mode, batches)
    constexpr bool BIGR = BATCH && STAGED && MODE == TPX_MODE_CC;
    constexpr int NP = BATCH ? RING : 1;   // staged tiles a CTA may hold
    if (tid == 0) {
        S.pend_head = 0;
        S.pend_count = 0;
        S.tile = atomicAdd(&p.ctl->tile_counter, 1u);
        S.first_tdc = INT_MAX;
        S.first_pix = INT_MAX;
        S.nroot = 0;
        S.status = 0;
        S.la_first[0] = S.la_first[1] = S.la_first[2] = INT_MAX;
    }
    if (tid < C_NUM) S.cnt[tid] = 0;
    if (tid < C_NUM) S.acc[tid] = 0;
#ifdef TPX_PHASE_TIMING
    if (tid < 32) S.ph[tid] = 0;
    long long ph_t = clock64();
#endif
    __syncthreads();
    // the unwrap state before the first tile, from the pre-pass
    if (tid < 8 && S.tile < p.n_tiles)
        reinterpret_cast<long long *>(&S.E)[tid] = __ldcg(reinterpret_cast<const long long *>(&p.ts.pre[S.tile]) + tid);

    for (;;) {
        // the tile's number, its unwrap state and the reset per-tile fields
        // were written before this barrier (at the kernel's start or at the
        // previous tile's tail)
        __syncthreads();
        const long long tile = S.tile;
        // the next tile is claimed now; its number is needed only at the end
        unsigned long long claim = 0;
        if (tid == 0 && tile < p.n_tiles) {
            claim = atomicAdd(&p.ctl->tile_counter, 1u);
            // the claimed tile's packets (and its look-ahead window) start
            // moving into L2 now, a tile ahead of their loads (one bulk
            // prefetch; the start is 16-byte aligned, the size a multiple of 16)
            if (!BATCH && p.l2_prefetch && claim < (unsigned long long)p.n_tiles) {
                const long long b = (long long)claim * T;
                const long long m = min((long long)(T + LA0), p.n - b) & ~1LL;
                if (m > 0)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p.pk + b), "r"((unsigned)(8 * m))
                                 : "memory");
            }
        }
        if (tile >= p.n_tiles) {
            if (STAGED) {
                if (tid < 32) flush_ring_warp<BATCH>(S, p, seq, true);
                __syncthreads();
                if (tid == 0 && S.status) atomicOr(&p.ctl->status, S.status);
            }
            // this CTA's counters (packets of each class are counted by the
            // unwrap pre-pass)
            if (tid < C_NUM && tid != C_PIXELS && tid != C_TDCS && tid != C_CORRUPT && S.acc[tid])
                atomicAdd(&p.ctl->counters[tid], S.acc[tid]);
#ifdef TPX_PHASE_TIMING
            TPX_PH(16);
            __syncthreads();
            if (tid < 32 && S.ph[tid]) atomicAdd(&g_phase[tid], S.ph[tid]);
#endif
            break;
        }
        // the tile: in a batch, the tile queue names the run (each run is a
        // stream of its own: the chains start over at its first tile)
        int run = 0;
        long long tile0 = 0, rend = p.n, base;
        if (BATCH) {
            run = p.bt.tile_run[tile];
            tile0 = p.bt.run_tile0[run];
            base = p.bt.run_off[run] + (tile - tile0) * T;
            rend = p.bt.run_off[run + 1];
        } else {
            base = tile * T;
        }
        const int cnt = (int)max(0LL, min((long long)T, rend - base));
        TPX_PH(0);

        // ---- load the tile and a first look-ahead window past it:
        // coalesced 16-byte loads into the padded buffer; the tile's TDC
        // packets are counted and its first one found on the way, and the
        // first TDC packet of the window ----
        const int lw = (int)max(0LL, min((long long)min(LA0, C - cnt), rend - base - cnt));   // window length
        {
            int my_first = INT_MAX, my_la = INT_MAX, c_tdc = 0;
            const int ltot = cnt + lw;
            if (BATCH && (base & 1)) {   // a run starting at an odd packet: 8-byte loads
                for (int v = tid; v < ltot; v += NT) {
                    const uint64_t w = __ldcg(p.pk + base + v);
                    S.buf[pad(v)] = w;
                    if ((w >> 60) == 0x6u) {
                        if (v < cnt) { ++c_tdc; my_first = min(my_first, v); } else my_la = min(my_la, v);
                    }
                }
            } else {
                const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(p.pk + base);
                const int npair = ltot >> 1;
                for (int v = tid; v < npair; v += NT) {
                    ulonglong2 w = __ldcg(src + v);
                    S.buf[pad(2 * v)] = w.x;
                    S.buf[pad(2 * v + 1)] = w.y;
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int q = 2 * v + u;
                        if (((u ? w.y : w.x) >> 60) == 0x6u) {
                            if (q < cnt) { ++c_tdc; my_first = min(my_first, q); } else my_la = min(my_la, q);
                        }
                    }
                }
                if ((ltot & 1) && tid == 0) {
                    const uint64_t w = __ldcg(p.pk + base + ltot - 1);
                    S.buf[pad(ltot - 1)] = w;
                    if ((w >> 60) == 0x6u) {
                        if (ltot - 1 < cnt) { ++c_tdc; my_first = min(my_first, ltot - 1); }
                        else my_la = min(my_la, ltot - 1);
                    }
                }
            }
            for (int i = tid; i < HB / 2; i += NT) reinterpret_cast<uint32_t *>(S.u1.head)[i] = 0xFFFFFFFFu;
            if (__any_sync(0xffffffffu, c_tdc != 0 || my_la != INT_MAX)) {
                c_tdc = (int)warp_sum((unsigned long long)c_tdc);
                my_first = __reduce_min_sync(0xffffffffu, (unsigned)my_first);
                my_la = __reduce_min_sync(0xffffffffu, (unsigned)my_la);
                if (lane == 0) {
                    if (c_tdc) atomicAdd(&S.cnt[C_TDCS], (unsigned long long)c_tdc);
                    if (my_first != INT_MAX) atomicMin(&S.first_tdc, my_first);
                    if (my_la != INT_MAX) atomicMin(&S.la_first[0], my_la);
                }
            }
        }
        __syncthreads();

        TPX_PH(1);
        const int f = S.first_tdc;

        // ---- look ahead past the window up to the next TDC packet, one
        // barrier per chunk (the chunks' minima rotate over three slots: a
        // slot is reset two chunks after it was read) ----
        int L = f != INT_MAX ? cnt + lw : cnt;   // a tile without a TDC packet owns nothing
        bool term = false;
        if (f != INT_MAX) {
            const int lf0 = S.la_first[0];
            if (lf0 != INT_MAX) {
                L = lf0 + 1;
                term = true;
            } else {
                for (int k = 1; base + L < rend; ++k) {
                    const int room = C - L;
                    if (room <= 0) break;
                    const int chunk = (int)min((long long)min(NT, room), rend - (base + L));
                    const int slot = k % 3;
                    if (tid == 0) S.la_first[(k + 1) % 3] = INT_MAX;
                    if (tid < chunk) {
                        const uint64_t w = __ldcg(p.pk + base + L + tid);
                        if (TPX_IN(L + tid, C)) S.buf[pad(L + tid)] = w;
                        if ((w >> 60) == 0x6u) atomicMin(&S.la_first[slot], tid);
                    }
                    __syncthreads();
                    const int lf = S.la_first[slot];
                    if (lf != INT_MAX) { L += lf + 1; term = true; break; }
                    L += chunk;
                }
            }
            // a range past the capacity: the big-range path, or its run goes back
            if (!term && base + L < rend && tid == 0) atomicOr(&S.status, (BIGR && p.big) ? ST_BIG : ST_CAPACITY);
        }

        TPX_PH(2);
        // ---- walk 2: wrap steps and TDC counts over [0, L) ----
        // [0, L) is split evenly over all threads, in thread order (every
        // later per-thread walk and scan uses the same contiguous chunks). A
        // thread counts its TDC packets and the pixel wrap steps (Sec. IV.A)
        // between consecutive pixels from its first pixel up to the first
        // pixel after its chunk, so that one scan gives every chunk the wraps
        // before its first pixel.
        const int kpd = (L + NT - 1) / NT;
        const int p0 = tid * kpd;
        int ntd = 0, fpx = INT_MAX, jp = 0;
        {
            int lpx = -1;
            long long lr = 0;
            for (int j = 0; j < kpd; ++j) {
                const int q = p0 + j;
                if (q >= L) break;
                const uint64_t w = S.buf[pad(q)];
                const unsigned h = (unsigned)(w >> 60);
                if (h == 0xBu) {
                    const long long r = pix_raw(w);
                    if (lpx >= 0) jp += (int)jump(r - lr, tp); else fpx = q;
                    lpx = q;
                    lr = r;
                } else if (h == 0x6u) {
                    ++ntd;
                }
            }
            if (lpx >= 0) {   // the step to the next pixel after the chunk
                for (int q = p0 + kpd; q < L; ++q) {
                    const uint64_t w = S.buf[pad(q)];
                    if ((w >> 60) == 0xBu) { jp += (int)jump(pix_raw(w) - lr, tp); break; }
                }
            }
            const int fw = (int)__reduce_min_sync(0xffffffffu, (unsigned)fpx);
            if (lane == 0 && fw != INT_MAX) atomicMin(&S.first_pix, fw);
        }
        // one scan of (TDC count, wrap steps) packed as two 16-bit halves
        unsigned pk_tot;
        const unsigned pk_ex = block_scan_vadd2(S, ((unsigned)ntd << 16) | ((unsigned)jp & 0xFFFFu), &pk_tot);
        const int li0 = (int)(pk_ex >> 16);              // TDC packets before the chunk
        const int ntdc = (int)(pk_tot >> 16);            // in [0, L)
        const int jp_ex = (int)(short)(pk_ex & 0xFFFFu); // pixel wraps between the range's first pixel and the chunk
        TPX_PH(3);
        const GAgg E = S.E;
        // a call sees only its own triggers: "earlier" means earlier in this call
        const long long trig_base = (!BATCH && p.E0) ? p.E0->tdc.n : 0;
        const bool prev_global = E.tdc.n > trig_base;
        const int nseg = min(ntdc, MAXSEG);
        if (tid == 0) {
            if (ntdc > MAXSEG) atomicOr(&S.status, ST_CAPACITY);
            // the step into the range's first pixel, read while the buffer
            // still holds packets (walk 4 overwrites them with records)
            const int fp = S.first_pix;
            S.j0 = (fp != INT_MAX && E.pix.n > 0) ? jump(pix_raw(S.buf[pad(fp)]) - E.pix.last, tp) : 0;
        }
        // ---- TDC packets of the range in stream order, then their unwrapped
        // times (one warp, a scan of the wrap steps) ----
        if (ntd) {
            int li = li0;
            for (int j = 0; j < kpd; ++j) {
                const int q = p0 + j;
                if (q >= L) break;
                if ((S.buf[pad(q)] >> 60) != 0x6u) continue;
                if (li < MAXSEG) S.tdc_pos[li] = (uint16_t)q;
                ++li;
            }
        }
        __syncthreads();
        if (tid < 32) {
            bool has = E.tdc.n > 0;
            long long last = E.tdc.last, ep = E.tdc.sum, t_last = 0;
            for (int i0 = 0; i0 < nseg; i0 += 32) {
                const int i = i0 + lane;
                long long r = 0;
                if (i < nseg) r = tdc_raw(S.buf[pad((int)S.tdc_pos[i])]);
                const long long rp = __shfl_up_sync(0xffffffffu, r, 1);
                int st = 0;
                if (i < nseg && (lane > 0 || has)) st = (int)jump(r - (lane > 0 ? rp : last), tt);
                int inc = st;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += u;
                }
                const long long t = r + (ep + inc) * kTdcPeriod;
                const long long tp_ = __shfl_up_sync(0xffffffffu, t, 1);
                if (i < nseg) {
                    S.tdc_t[i] = t;
                    if ((lane > 0 || i0 > 0) && t < (lane > 0 ? tp_ : t_last)) atomicOr(&p.ctl->status, ST_TRIG_ORDER);
                    if (!BATCH && S.tdc_pos[i] < cnt) {   // a batch writes its triggers at the flush
                        const long long g = E.tdc.n - trig_base + i;
                        if (g >= 0 && g < p.trig_cap) p.trig[g] = t; else atomicOr(&p.ctl->status, ST_TRIG_CAP);
                    }
                }
                const int lastl = min(31, nseg - 1 - i0);
                ep += __shfl_sync(0xffffffffu, inc, lastl);
                last = __shfl_sync(0xffffffffu, r, lastl);
                t_last = __shfl_sync(0xffffffffu, t, lastl);
                has = true;
            }
        }
        __syncthreads();

        TPX_PH(4);
        // ---- walk 4: pixels -> shot, cut, timewalk, packed record ----
        {
            // wraps at the chunk's first pixel: before the range, the step from
            // the last pixel before it to the range's first pixel, the steps
            // inside the range before the chunk
            long long ep = E.pix.sum + S.j0 + jp_ex;
            bool has = false;
            long long last = 0;
            int seg = li0 - 1;
            const long long t_prev_global = E.tdc.last + E.tdc.sum * kTdcPeriod;
            unsigned long long c_keep = 0, c_pre = 0, c_bg = 0;
            bool exc = false;
            for (int j = 0; j < kpd; ++j) {
                const int q = p0 + j;
                if (q >= L) break;
                const uint64_t w = S.buf[pad(q)];
                const unsigned h = (unsigned)(w >> 60);
                uint64_t rec = INVALID;
                if (h == 0x6u) {
                    ++seg;
                } else if (h == 0xBu) {
                    const long long r = pix_raw(w);
                    if (has) ep += jump(r - last, tp);
                    has = true;
                    last = r;
                    const long long t = r + ep * kPixPeriod;
                    if (seg < 0) {
                        if (!prev_global) ++c_pre;        // no trigger before it anywhere
                    } else if (seg < nseg) {
                        const long long t_lo = S.tdc_t[seg];
                        const bool has_hi = seg + 1 < nseg;
                        int verdict;                      // 0 keep, 1 bg, 2 pre, 3 undecidable here
                        if (has_hi && t >= S.tdc_t[seg + 1]) verdict = 3;
                        else if (t >= t_lo) verdict = (t - t_lo > p.tof_max) ? 1 : 0;
                        else {
                            const bool hp = seg > 0 || prev_global;
                            const long long tprev = seg > 0 ? S.tdc_t[seg - 1] : t_prev_global;
                            if (!hp) verdict = 2;
                            else if (t >= tprev) verdict = (t - tprev > p.tof_max) ? 1 : 3;
                            else verdict = 3;
                        }
                        if (verdict == 0) {
                            const int tot = pix_tot(w);
                            const long long tc = t - (p.lut ? (long long)p.lut[tot] : 0LL);
                            const long long tofb = tc - t_lo + kTofBias;
                            rec = mkrec((uint32_t)tofb, (uint32_t)seg, (uint32_t)tot, (uint32_t)pix_x(w), (uint32_t)pix_y(w));
                            ++c_keep;
                        } else if (verdict == 1) ++c_bg;
                        else if (verdict == 2) ++c_pre;
                        else exc = true;
                    }
                }
                S.buf[pad(q)] = rec;
            }
            c_keep = warp_sum(c_keep); c_pre = warp_sum(c_pre); c_bg = warp_sum(c_bg);
            if (lane == 0) {
                atomicAdd(&S.cnt[C_KEPT], c_keep);
                atomicAdd(&S.cnt[C_DROP_PRE], c_pre);
                atomicAdd(&S.cnt[C_DROP_BG], c_bg);
            }
            if (exc) atomicOr(&S.status, ST_EXCEPTION);
        }
        __syncthreads();   // records written per contiguous chunk are read strided below

        TPX_PH(5);
        // a batch tile whose range the tiles cannot hold: its run is redone by
        // the general path, so it clusters nothing (its counts still flow)
        // (a big range clusters nothing here either: it has a path of its own)
        const bool skip = BATCH && (S.status & (ST_CAPACITY | ST_EXCEPTION | ST_BIG)) != 0;
        // a big range: its path runs before the previous tile is copied out
        // (that copy may wait for other CTAs' big ranges)
        const bool big_tile = BIGR && (S.status & ST_BIG) && !(S.status & (ST_CAPACITY | ST_EXCEPTION));
        // the range this CTA owns: [R0, R1)
        const int R0 = (f == INT_MAX || skip) ? 0 : f;
        const int R1 = (f == INT_MAX || skip) ? 0 : (term ? L - 1 : L);
        // label writes cover [W0, W1): the range, plus the packets before the
        // tile's first trigger when no trigger precedes them anywhere
        const int W0 = prev_global ? R0 : 0;
        const int W1 = skip ? 0 : ((f == INT_MAX) ? (prev_global ? 0 : cnt) : R1);

        // ---- hash insert ----
        for (int q = R0 + tid; q < R1; q += NT) {
            const uint64_t r = S.buf[pad(q)];
            S.parent[q] = (NO_EXT << 16) | (uint32_t)q;
            S.notpeak[q] = 0;
            if (r != INVALID) {
                const uint32_t b = hcell(r_seg(r), r_x(r), r_y(r));
                // push q on the bucket's list (16-bit exchange as a CAS loop)
                unsigned short old = S.u1.head[b], seen;
                do {
                    seen = old;
                    old = atomicCAS(&S.u1.head[b], seen, (unsigned short)q);
                } while (old != seen);
                S.u2.next[q] = old;
            }
        }
        __syncthreads();

        TPX_PH(6);
        // ---- neighbour pass: each adjacent pair once (Sec. V.A box rule) ----
        // The warp walks 32 consecutive positions at a time; each lane gathers
        // its pixel's partners in the forward half of the box -- a strict order
        // of the pairs: a larger x, or the same x and a larger y, or the same
        // cell and a later position -- and updates the local-maximum flags
        // (Sec. V.B). CC mode: the pixel points to its first partner (a plain
        // store: pointers only go forward, so they form a forest) and keeps its
        // second partner in the upper half of its pointer word; a pixel with
        // more partners marks its word for a re-walk.
        {
            for (int qb = R0 + (tid & ~31); qb < R1; qb += NT) {
                const int q = qb + lane;
                const uint64_t r = q < R1 ? S.buf[pad(q)] : INVALID;
                if (r == INVALID) continue;
                uint32_t e0 = (uint32_t)q, e1 = NO_EXT;
                int ne = 0;
                const int x = r_x(r), y = r_y(r), sg = r_seg(r), tb = r_tof(r), tot = r_tot(r);
                const uint32_t hb = (uint32_t)(x + 67 * y + 1543 * sg);   // hcell of (x, y), unmasked
                bool dim = false;
                if (MODE == TPX_MODE_CC && p.rx == 1 && p.ry == 1) {
                    // 8-neighbour box, its five forward cells unrolled. A diagonal
                    // partner (dx = 1, dy = -1 or +1) is held back and needs no
                    // union when the pixel's partner to the side (dx = 1, dy = 0),
                    // or above it (dx = 0, dy = +1) for dy = +1, is adjacent to it
                    // as well: that path of two axis-aligned pairs, which are never
                    // held back, joins them
                    uint32_t hold = 0xFFFFFFFFu;   // held partners: dy = -1 low half, dy = +1 high half
                    int tA = 0, tB = 0, tE = INT_MIN, tN = INT_MIN;
#pragma unroll
                    for (int c = 0; c < 5; ++c) {
                        const int dx = c < 2 ? 0 : 1;
                        const int dy = c == 0 ? 0 : (c == 1 ? 1 : c - 3);
                        if (x + dx > 255 || y + dy < 0 || y + dy > 255) continue;
                        const uint32_t ck = r_cell(r) + (uint32_t)(256 * dy + dx);
                        for (uint32_t j = S.u1.head[(hb + 67 * dy + dx) & (HB - 1)]; j != EMPTY; j = S.u2.next[j]) {
                            if (!TPX_IN(j, C)) break;
                            if (c == 0 && (int)j <= q) continue;
                            const uint64_t rj = S.buf[pad((int)j)];
                            if (r_cell(rj) != ck) continue;
                            const int tjt = r_tof(rj);
                            if (!within(tjt - tb, p.dt)) continue;
                            const int tj = r_tot(rj);
                            // local maxima: equal ToT goes to the later pixel (Sec. V.B)
                            if (tj > tot || (tj == tot && (int)j > q)) dim = true;
                            else S.notpeak[j] = 1;
                            if (c == 3 && tE == INT_MIN) tE = tjt;
                            if (c == 1 && tN == INT_MIN) tN = tjt;
                            if (c == 2 || c == 4) {
                                const int sh = c == 4 ? 16 : 0;
                                if (((hold >> sh) & 0xFFFFu) == 0xFFFFu) {
                                    hold = (hold & ~(0xFFFFu << sh)) | (j << sh);
                                    if (c == 4) tB = tjt; else tA = tjt;
                                    continue;
                                }
                            }
                            if (ne == 0) e0 = j; else if (ne == 1) e1 = j;
                            ++ne;
                        }
                    }
                    const uint32_t jA = hold & 0xFFFFu, jB = hold >> 16;
                    const bool skipA = tE != INT_MIN && within(tE - tA, p.dt);
                    const bool skipB = (tE != INT_MIN && within(tE - tB, p.dt)) || (tN != INT_MIN && within(tN - tB, p.dt));
                    if (jA != 0xFFFFu && !skipA) { if (ne == 0) e0 = jA; else if (ne == 1) e1 = jA; ++ne; }
                    if (jB != 0xFFFFu && !skipB) { if (ne == 0) e0 = jB; else if (ne == 1) e1 = jB; ++ne; }
                } else {
                    for (int dx = 0; dx <= p.rx; ++dx) {
                        const int cx = x + dx;
                        if (cx > 255) break;
                        for (int dy = (dx == 0 ? 0 : -p.ry); dy <= p.ry; ++dy) {
                            const int cy = y + dy;
                            if (cy < 0 || cy > 255) continue;
                            const uint32_t ck = r_cell(r) + (uint32_t)(256 * dy + dx);
                            for (uint32_t j = S.u1.head[(hb + 67 * dy + dx) & (HB - 1)]; j != EMPTY; j = S.u2.next[j]) {
                                if (!TPX_IN(j, C)) break;
                                if (dx == 0 && dy == 0 && (int)j <= q) continue;
                                const uint64_t rj = S.buf[pad((int)j)];
                                if (r_cell(rj) != ck) continue;
                                if (!within(r_tof(rj) - tb, p.dt)) continue;
                                const int tj = r_tot(rj);
                                // local maxima: equal ToT goes to the later pixel (Sec. V.B)
                                if (tj > tot || (tj == tot && (int)j > q)) dim = true;
                                else S.notpeak[j] = 1;
                                if (MODE == TPX_MODE_CC) {
                                    if (ne == 0) e0 = j; else if (ne == 1) e1 = j;
                                    ++ne;
                                }
                            }
                        }
                    }
                }
                if (dim) S.notpeak[q] = 1;
                // with two partners the pointer takes the later-found one (the
                // larger x when the two differ): pointers run along x first,
                // which keeps the trees of a compact cloud shallow
                if (MODE == TPX_MODE_CC)
                    S.parent[q] = ne > 2 ? ((REWALK << 16) | e0) : ne == 2 ? ((e0 << 16) | e1) : ((NO_EXT << 16) | e0);
            }
        }
        __syncthreads();

        TPX_PH(7);
        int ncl = 0;
        if (MODE == TPX_MODE_CC) {
            // compress: every pixel points to the root of its tree
            for (int q = R0 + tid; q < R1; q += NT) {
                const uint32_t w = sh_ld(pbase + 4 * q);
                if ((w & 0xFFFFu) == (uint32_t)q) continue;
                sh_st(pbase + 4 * q, (w & 0xFFFF0000u) | find_hw(pbase, w & 0xFFFFu));
            }
            __syncthreads();
            TPX_PH(8);
            // unions of the second partners, warp-synchronous: each trip
            // advances every active lane by one find hop (path halving) or one
            // link attempt, the larger root position linked under the smaller.
            // A pixel marked for a re-walk unites each of its partners in turn.
            for (int qb = R0 + (tid & ~31); qb < R1; qb += NT) {
                const int q = qb + lane;
                uint32_t b = q < R1 ? sh_ld(pbase + 4 * q) >> 16 : NO_EXT;
                if (b == REWALK) {
                    rewalk_unite<MODE>(S, p, pbase, q);
                    b = NO_EXT;
                }
                __syncwarp();
                uint32_t a = (uint32_t)q;
                bool active = b != NO_EXT && TPX_IN(b, C);
                while (__any_sync(0xffffffffu, active)) {
                    if (active) {
                        const uint32_t wa = sh_ld(pbase + 4 * a), wb = sh_ld(pbase + 4 * b);
                        const uint32_t pa = wa & 0xFFFFu, pb = wb & 0xFFFFu;
                        if (pa != a || pb != b) {
                            if (pa != a) {
                                const uint32_t ga = sh_ld(pbase + 4 * pa) & 0xFFFFu;
                                if (ga != pa) sh_st(pbase + 4 * a, (wa & 0xFFFF0000u) | ga);
                                a = ga;
                            }
                            if (pb != b) {
                                const uint32_t gb = sh_ld(pbase + 4 * pb) & 0xFFFFu;
                                if (gb != pb) sh_st(pbase + 4 * b, (wb & 0xFFFF0000u) | gb);
                                b = gb;
                            }
                        } else if (a == b) {
                            active = false;
                        } else {
                            const uint32_t lo = min(a, b), hi = max(a, b);
                            const uint32_t wh = hi == a ? wa : wb;
                            const uint32_t old = sh_cas(pbase + 4 * hi, wh, (wh & 0xFFFF0000u) | lo);
                            if (old == wh) active = false;
                            else { a = lo; b = old & 0xFFFFu; }   // hi was linked meanwhile: go on above it
                        }
                    }
                }
            }
            __syncthreads();
            TPX_PH(9);
            // roots; the hash is free now: member-list heads, cleared
            for (int q = R0 + tid; q < R1; q += NT) {
                S.u1.mhead[q] = EMPTY;
                if (S.buf[pad(q)] != INVALID) S.u2.rootof[q] = (uint16_t)find_ro(pbase, (uint32_t)q);
            }
            __syncthreads();
            TPX_PH(10);
            // member lists: each kept pixel joins its root's list (the links
            // take the first half of the union-find array); the roots are
            // appended to the root list (its second half) in any order, and
            // the label bitmap is cleared
            uint16_t *mnext = reinterpret_cast<uint16_t *>(S.parent);
            uint16_t *rootpos = reinterpret_cast<uint16_t *>(S.parent) + C;
            for (int w = tid; w < C / 32; w += NT) S.lbits[w] = 0u;
            for (int qb = R0 + (tid & ~31); qb < R1; qb += NT) {
                const int q = qb + lane;
                bool is_root = false;
                if (q < R1 && S.buf[pad(q)] != INVALID) {
                    const uint32_t rt = S.u2.rootof[q];
                    if (TPX_IN(rt, C)) mnext[q] = (uint16_t)atomicExch(&S.u1.mhead[rt], (uint32_t)q);
                    is_root = rt == (uint32_t)q;
                }
                const unsigned m = __ballot_sync(0xffffffffu, is_root);
                int at = 0;
                if (lane == 0 && m) at = atomicAdd(&S.nroot, __popc(m));
                at = __shfl_sync(0xffffffffu, at, 0) + __popc(m & ((1u << lane) - 1u));
                if (is_root && TPX_IN(at, C)) rootpos[at] = (uint16_t)q;
            }
            __syncthreads();
            TPX_PH(11);
            ncl = S.nroot;
            if (STAGED) {
                // The last warp copies the previous tile's staged records out
                // while the others walk this tile's member lists: one thread
                // per cluster forms the exact integer moments (Sec. V.C) and
                // finds the cluster's earliest pixel in (time, position) order
                // -- its canonical label -- which is kept in the upper half of
                // the list head and marked in the label bitmap. A thread keeps
                // its first cluster's moments in registers until the labels'
                // ranks are known; the records are staged in label order.
                constexpr int NWALK = NT - 32;
                Moments held{0, 0, 0, 0, 0, 0, 0, 0};
                if (tid >= NWALK) {
                    flush_ring_warp<BATCH>(S, p, seq, false);
                } else {
                    for (int i = tid; i < ncl; i += NWALK) {
                        if (!TPX_IN(i, C)) break;
                        const uint32_t rt = rootpos[i];
                        if (!TPX_IN(rt, C)) continue;
                        const uint32_t head = S.u1.mhead[rt] & 0xFFFFu;
                        const Moments m = walk_members(S, p, head);
                        if (!TPX_IN(m.best_lo, C)) continue;
                        S.u1.mhead[rt] = (m.best_lo << 16) | head;
                        atomicOr(&S.lbits[m.best_lo >> 5], 1u << (m.best_lo & 31));
                        if (i == tid) held = m;
                    }
                }
                __syncthreads();
                TPX_PH(12);
                // the labels' ranks: one warp scans the bitmap's counts
                if (tid < 32) {
                    constexpr int WPL = C / 32 / 32;   // bitmap words per lane
                    int c = 0;
#pragma unroll
                    for (int k = 0; k < WPL; ++k) c += __popc(S.lbits[lane * WPL + k]);
                    int incl = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += u;
                    }
                    int run = incl - c;
#pragma unroll
                    for (int k = 0; k < WPL; ++k) {
                        S.lpre[lane * WPL + k] = (uint16_t)run;
                        run += __popc(S.lbits[lane * WPL + k]);
                    }
                }
                __syncthreads();
                TPX_PH(19);
                tpx_record *dst = p.stage + ((long long)blockIdx.x * NP + (S.pend_head + S.pend_count) % NP) * C;
                if (tid < NWALK && tid < ncl && held.n > 0) {
                    const int k = label_rank(S, held.best_lo);
                    if (TPX_IN(k, C)) put_record(dst + k, held, S, p, base, E.tdc.n);
                }
                // clusters beyond one per walking thread: walked again
                for (int i = tid + NWALK; tid < NWALK && i < ncl; i += NWALK) {
                    if (!TPX_IN(i, C)) break;
                    const uint32_t rt = rootpos[i];
                    if (!TPX_IN(rt, C)) continue;
                    const Moments m = walk_members(S, p, S.u1.mhead[rt] & 0xFFFFu);
                    const int k = label_rank(S, m.best_lo);
                    if (TPX_IN(k, C) && TPX_IN(m.best_lo, C)) put_record(dst + k, m, S, p, base, E.tdc.n);
                }
            } else {
            // one thread per root walks its list for the cluster's earliest
            // pixel in (time, position) order -- its canonical label -- keeps
            // it in the upper half of the list head and flags it (bit 1 of
            // notpeak)
            for (int i = tid; i < ncl; i += NT) {
                if (!TPX_IN(i, C)) break;
                const uint32_t q = rootpos[i];
                if (!TPX_IN(q, C)) continue;
                const uint32_t head = S.u1.mhead[q] & 0xFFFFu;
                uint64_t best = ~0ull;
                for (uint32_t m = head; m != EMPTY; m = mnext[m]) {
                    if (!TPX_IN(m, C)) break;
                    best = min(best, ((uint64_t)r_tof(S.buf[pad((int)m)]) << 16) | m);
                }
                const uint32_t lp = (uint32_t)(best & 0xFFFFu);
                S.u1.mhead[q] = (lp << 16) | head;
                if (TPX_IN(lp, C)) S.notpeak[lp] |= 2;
            }
            __syncthreads();
            // cluster ids in ascending label position
            int c = 0;
            for (int j = 0; j < kpd; ++j) {
                const int q = p0 + j;
                if (q >= R0 && q < R1 && (S.notpeak[q] & 2)) ++c;
            }
            int excl = block_scan_int(S, c, &ncl);
            for (int j = 0; j < kpd; ++j) {
                const int q = p0 + j;
                if (q >= R0 && q < R1 && (S.notpeak[q] & 2)) {
                    if (TPX_IN(excl, C)) rootpos[excl] = (uint16_t)q;
                    ++excl;
                }
            }
            }
        } else {
            // PAPER mode: one record per local maximum (list kept in parent[])
            int c = 0;
            for (int j = 0; j < kpd; ++j) {
                const int q = p0 + j;
                if (q >= R0 && q < R1 && S.buf[pad(q)] != INVALID && !S.notpeak[q]) ++c;
            }
            int excl = block_scan_int(S, c, &ncl);
            for (int j = 0; j < kpd; ++j) {
                const int q = p0 + j;
                if (q >= R0 && q < R1 && S.buf[pad(q)] != INVALID && !S.notpeak[q]) {
                    if (TPX_IN(excl, C)) S.parent[excl] = (uint32_t)q;
                    ++excl;
                }
            }
        }
        bool big_done = false;   // this tile's records wait in the big-range scratch
        if constexpr (BIGR) {
            // a big range takes its own path once the staging slot is free
            // (the previous tile's records were copied out above)
            if (big_tile) {
                const int k = big_range<BATCH>(S, p, base, rend, f, prev_global);
                ncl = k > 0 ? k : 0;
                big_done = k >= 0;
                TPX_PH(17);
                if (tid < 32) flush_ring_warp<BATCH>(S, p, seq, false);
                __syncthreads();
                TPX_PH(18);
            }
        }

        TPX_PH(13);
        // ---- record offsets: publish this tile's count now, look back later ----
        if (tid == 0 && tile + 1 != p.hold) {
            if (tile > 0) {
                __stcg(&p.ts.cagg[tile], (long long)ncl);
                if (BATCH) __stcg(&p.bt.tcagg[tile], (long long)S.cnt[C_TDCS]);
                st_release(&p.ts.cflags[tile], (seq << 2) | 1u);
            } else {
                __stcg(&p.ts.cpre[0], (long long)ncl);
                if (BATCH) __stcg(&p.bt.tcpre[0], (long long)S.cnt[C_TDCS]);
                st_release(&p.ts.cflags[0], (seq << 2) | 2u);
            }
        }
        const long long ntr_here = E.tdc.n - trig_base + (long long)S.cnt[C_TDCS];
        // records go to the CTA's staging slot (STAGED) or straight to their
        // offset after an inline look-back
        auto record_target = [&](long long *lim) -> tpx_record * {
            if (STAGED) {
                if (tid < 32) flush_ring_warp<BATCH>(S, p, seq, false);
                __syncthreads();   // the peak list is complete
                *lim = C;
                return p.stage + ((long long)blockIdx.x * NP + (S.pend_head + S.pend_count) % NP) * C;
            }
            if (tid < 32) resolve_offset<false>(S, p, seq, tile, ncl, ntr_here, 0, 0, false);
            __syncthreads();
            *lim = p.cl_cap - S.clo;
            return p.clusters + S.clo;
        };

        if (MODE == TPX_MODE_CC) {
            // Each kept pixel writes its label (the stream index of its
            // cluster's earliest pixel); then one thread per cluster walks the
            // member list and forms the exact integer moments in registers
            // (Sec. V.C).
            const uint16_t *mnext = reinterpret_cast<const uint16_t *>(S.parent);
            const uint16_t *rootpos = mnext + C;
            __syncthreads();
            unsigned long long c_pk = 0;
            for (int q = W0 + tid; q < W1; q += NT) {
                const uint64_t r = S.buf[pad(q)];
                bool kept = q >= R0 && r != INVALID;
                uint32_t lp = 0;
                uint8_t pk = 0;
                if (kept && !TPX_IN(S.u2.rootof[q], C)) kept = false;
                if (kept) {
                    lp = S.u1.mhead[S.u2.rootof[q]] >> 16;
                    pk = (S.notpeak[q] & 1) ? 0 : 1;
                    c_pk += pk;
                }
                if (!TPX_IN(base + q, rend)) continue;
                if (p.labels) p.labels[base + q] = kept ? p.idx_base + base + (long long)lp : -1LL;
                else if (p.labels32) p.labels32[base + q] = kept ? (int)(p.idx_base - p.lab32_base + base + lp) : -1;
                if (p.is_peak) p.is_peak[base + q] = pk;
            }
            c_pk = warp_sum(c_pk);
            if (lane == 0) atomicAdd(&S.cnt[C_PEAKS], c_pk);
            long long lim = 0;
            tpx_record *dst = STAGED ? nullptr : record_target(&lim);
            // records (unstaged: after the inline look-back, in label order):
            // one thread per cluster walks its member list and forms the
            // exact integer moments in registers (Sec. V.C)
            for (int i = tid; !STAGED && i < ncl; i += NT) {
                if (i >= lim) break;
                const int q = rootpos[i];
                if (!TPX_IN(q, C) || !TPX_IN(S.u2.rootof[q], C)) continue;
                const uint64_t r = S.buf[pad(q)];
                const int tofb0 = r_tof(r);
                long long s_tot = 0, s_x = 0, s_y = 0, s_t = 0;
                int n = 0, npk = 0;
                for (uint32_t m = S.u1.mhead[S.u2.rootof[q]] & 0xFFFFu; m != EMPTY; m = mnext[m]) {
                    if (!TPX_IN(m, C)) break;
                    const uint64_t rm = S.buf[pad((int)m)];
                    const long long tot = r_tot(rm);
                    n += 1;
                    npk += (S.notpeak[m] & 1) ? 0 : 1;
                    s_tot += tot;
                    s_x += tot * r_x(rm);
                    s_y += tot * r_y(rm);
                    s_t += tot * (long long)(r_tof(rm) - tofb0);
                }
                const int seg = r_seg(r);
                const long long tofc0 = (long long)tofb0 - kTofBias;
                tpx_record o;
                o.label = p.idx_base + base + q;
                o.shot = E.tdc.n + seg;
                o.t0 = S.tdc_t[seg] + tofc0;
                o.s_tot = s_tot; o.s_x = s_x; o.s_y = s_y; o.s_t = s_t;
                o.n = n; o.n_peaks = npk;
                com_from_moments(s_x, s_y, s_t, s_tot, tofc0, &o.x, &o.y, &o.tof);
                out_record(p, S.clo + i, o);   // unstaged: straight to its offset
            }
        } else {
            unsigned long long c_pk = 0;
            for (int q = W0 + tid; q < W1; q += NT) {
                const uint64_t r = S.buf[pad(q)];
                long long lab = -1;
                uint8_t pk = 0;
                if (q >= R0 && r != INVALID) {
                    lab = p.idx_base + base + q;
                    pk = S.notpeak[q] ? 0 : 1;
                    c_pk += pk;
                }
                if (!TPX_IN(base + q, rend)) continue;
                if (p.labels) p.labels[base + q] = lab;
                else if (p.labels32) p.labels32[base + q] = lab < 0 ? -1 : (int)(lab - p.lab32_base);
                if (p.is_peak) p.is_peak[base + q] = pk;
            }
            c_pk = warp_sum(c_pk);
            if (lane == 0) atomicAdd(&S.cnt[C_PEAKS], c_pk);
            long long lim = 0;
            tpx_record *dst = record_target(&lim);
            // records: box neighbourhood sums of each local maximum (Sec. V.C)
            for (int i = tid; i < ncl; i += NT) {
                if (i >= lim) break;
                const int q = (int)S.parent[i];
                if (!TPX_IN(q, C)) continue;
                const uint64_t r = S.buf[pad(q)];
                const int x = r_x(r), y = r_y(r), sg = r_seg(r), tb = r_tof(r);
                long long n = 0, s_tot = 0, s_x = 0, s_y = 0, a2 = 0;
                int tmin = tb;
                for (int dx = -p.rx; dx <= p.rx; ++dx) {
                    const int cx = x + dx;
                    if (cx < 0 || cx > 255) continue;
                    for (int dy = -p.ry; dy <= p.ry; ++dy) {
                        const int cy = y + dy;
                        if (cy < 0 || cy > 255) continue;
                        for (uint32_t j = S.u1.head[hcell(sg, cx, cy)]; j != EMPTY; j = S.u2.next[j]) {
                            if (!TPX_IN(j, C)) break;
                            const uint64_t rj = S.buf[pad((int)j)];
                            if (r_x(rj) != cx || r_y(rj) != cy || r_seg(rj) != sg) continue;
                            const int d = r_tof(rj) - tb;
                            if (d < -p.dt || d > p.dt) continue;
                            const long long tj = r_tot(rj);
                            n += 1; s_tot += tj; s_x += tj * cx; s_y += tj * cy; a2 += tj * r_tof(rj);
                            tmin = min(tmin, r_tof(rj));
                        }
                    }
                }
                const long long s_t = a2 - (long long)tmin * s_tot;
                const long long tofc0 = (long long)tmin - kTofBias;
                tpx_record o;
                o.label = p.idx_base + base + q;
                o.shot = E.tdc.n + sg;
                o.t0 = S.tdc_t[sg] + tofc0;
                o.s_tot = s_tot; o.s_x = s_x; o.s_y = s_y; o.s_t = s_t;
                o.n = (int)n; o.n_peaks = 1;
                com_from_moments(s_x, s_y, s_t, s_tot, tofc0, &o.x, &o.y, &o.tof);
                if (STAGED) dst[i] = o;
                else out_record(p, S.clo + i, o);
            }
        }
        TPX_PH(14);
        if (BATCH) {   // this tile's trigger times wait with its records
            const int nt = min((int)S.cnt[C_TDCS], MAXSEG);
            long long *ts = p.bt.tstage + ((long long)blockIdx.x * NP + (S.pend_head + S.pend_count) % NP) * T;
            for (int i = tid; i < nt; i += NT) ts[i] = S.tdc_t[i];
            __syncthreads();   // every thread has its slot before the tile joins the ring
        }
        if (tid == 0) {
            S.cnt[C_CLUSTERS] = (unsigned long long)ncl;
            if (STAGED) {
                // a tile with nothing to write (no records, no triggers; not
                // a run's first tile nor the call's last) needs no offset: its
                // count is published, and the successors' look-backs add it up
                const bool first = tile == tile0;
                if (ncl != 0 || S.cnt[C_TDCS] != 0 || (BATCH && first) || tile == p.n_tiles - 1) {
                    const int e = (S.pend_head + S.pend_count) % NP;
                    S.pend[e].tile = tile;
                    S.pend[e].ncl = ncl;
                    S.pend[e].ntr = ntr_here;
                    S.pend[e].ntdc = (int)S.cnt[C_TDCS];
                    S.pend[e].run = run;
                    S.pend[e].first = first;
                    S.pend[e].big = big_done;
                    S.pend_count += 1;
                }
            }
        }
        __syncthreads();
        TPX_PH(15);
        // the tile's counters join the CTA's, and the per-tile fields are
        // reset for the next tile (which starts with a barrier)
        if (tid < C_NUM) {
            S.acc[tid] += tid == C_PACKETS ? (unsigned long long)cnt : S.cnt[tid];
            S.cnt[tid] = 0;
        }
        // the next tile and its unwrap state, by warp 0 alone: no other warp
        // reads S.tile or S.E before the next barrier
        if (tid == 0) S.next_tile = (long long)claim;
        __syncwarp();
        if (tid < 8 && S.next_tile < p.n_tiles)
            reinterpret_cast<long long *>(&S.E)[tid] =
                __ldcg(reinterpret_cast<const long long *>(&p.ts.pre[S.next_tile]) + tid);
        if (tid == 0) {
            S.tile = S.next_tile;
            unsigned st = S.status & ~ST_BIG;
            if (BATCH && (st & (ST_CAPACITY | ST_EXCEPTION))) {   // only this run is redone
                p.bt.run_failed[run] = 1u;
                st = (st & ~(ST_CAPACITY | ST_EXCEPTION)) | ST_RUN_REDO;
            }
            if (st) atomicOr(&p.ctl->status, st);
            S.status = 0;
            S.first_tdc = INT_MAX;
            S.first_pix = INT_MAX;
            S.nroot = 0;
            S.la_first[0] = S.la_first[1] = S.la_first[2] = INT_MAX;
        }
    }
}

int smem_bytes() { return (int)sizeof(Smem); }

// The shared-memory attribute belongs to each device's context: it is set
// once per device (and again on any device beyond the table).
template <int MODE, bool STAGED, bool BATCH>
cudaError_t launch_one(const Params &p, int grid, cudaStream_t s) {
    static std::atomic<bool> attr_done[kAttrDevices];
    const int smem = (int)sizeof(Smem);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool known = dev >= 0 && dev < kAttrDevices;
    if (!known || !attr_done[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(fused_kernel<MODE, STAGED, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        if (known) attr_done[dev].store(true, std::memory_order_release);
    }
    fused_kernel<MODE, STAGED, BATCH><<<grid, NT, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch(const Params &p, int mode, int grid, cudaStream_t s) {
    const bool cc = mode == TPX_MODE_CC;
    if (p.bt.tile_run)   // a batch always stages its output
        return cc ? launch_one<TPX_MODE_CC, true, true>(p, grid, s) : launch_one<TPX_MODE_PAPER, true, true>(p, grid, s);
    if (p.stage)
        return cc ? launch_one<TPX_MODE_CC, true, false>(p, grid, s) : launch_one<TPX_MODE_PAPER, true, false>(p, grid, s);
    return cc ? launch_one<TPX_MODE_CC, false, false>(p, grid, s) : launch_one<TPX_MODE_PAPER, false, false>(p, grid, s);
}
