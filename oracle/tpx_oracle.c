/*
 * tpx_oracle.c -- plain, slow, sequential CPU oracle for the TPX3 clustering /
 * centroiding path.  TEST INFRASTRUCTURE ONLY: only tests/, the smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * table with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   1. decode 64-bit packets (Sec. III: pixel events carry X, Y, ToA, ToT; TDC
 *      events carry the trigger ToA).  Bit layout: project-defined TPX3-style
 *      layout (the paper relies on a vendor converter and prints none):
 *        pixel [63:60]=0xB [59:53]=dcol [52:47]=spix [46:44]=pix [43:30]=ToA
 *              [29:20]=ToT [19:16]=fToA [15:0]=spidr;
 *              x = 2*dcol + (pix>>2), y = 4*spix + (pix&3),
 *              raw = ((spidr<<14 | ToA)*16 - fToA) mod 2^34   (1.5625 ns ticks)
 *        TDC   [63:60]=0x6 [43:9]=coarse (3.125 ns); raw = 2*coarse mod 2^36
 *      The pixel wrap 2^34 ticks * 1.5625 ns = 2^42 * 25/4096 ns = 26.84 s and
 *      the TDC wrap 2^36 ticks = 2^44 * 25/4096 ns = 107.37 s (Sec. IV.A).
 *   2. unwrap ToA separately for pixels and for TDCs in stream order
 *      (Sec. IV.A): a jump to a value more than `thr` below the previous one
 *      adds one wrap period to everything after it; a jump more than `thr`
 *      above it (a straggler reported after a wrap) removes one.
 *   3. triggers = TDC packets in stream order; they must be non-decreasing.
 *   4. each pixel belongs to the most recent trigger in time (last trigger
 *      with t_trig <= t); it is dropped if there is none or if its ToF exceeds
 *      tof_max (Sec. IV.B, "does not exceed" -> keep ToF <= tof_max).  An
 *      optional integer timewalk table indexed by ToT is subtracted after the
 *      cut (Sec. IV.C, Eq. 1, tabulated in ticks).
 *   5. kept pixels are stably sorted by (shot, corrected time); ties keep
 *      stream order.  The sorted rank is the canonical order.
 *   6. adjacency (Sec. V.A, the Hadamard product of per-axis box rules):
 *      same shot, |dx| <= rx, |dy| <= ry, |dt| <= dt_ticks, all inclusive.
 *      CC mode: clusters are the connected components of that adjacency,
 *      found by breadth-first search seeded at each unvisited pixel in sorted
 *      order, so every cluster is labelled by its earliest pixel in sorted
 *      order; the label value is that pixel's stream index.
 *   7. local maxima (Sec. V.B): a pixel is a local maximum iff no neighbour
 *      is brighter, where equal ToT is resolved in favour of the pixel that
 *      appears later in the stream (the paper's ascending 0.001*i offset,
 *      applied exactly as a lexicographic comparison on (ToT, stream index)).
 *   8. centroids (Sec. V.C, centre of mass with ToT as the mass):
 *      CC mode: sums over each cluster.  PAPER mode: for every local maximum
 *      i, sums over its box neighbourhood {j : A_ij = 1} (which contains i).
 *      Integer sums n, S_tot, S_x = sum x*ToT, S_y, t0 = earliest corrected
 *      time, S_t = sum (t - t0)*ToT; then x = S_x/S_tot, y = S_y/S_tot,
 *      tof = (t0 - t_trig) + S_t/S_tot in double precision.
 *   Output clusters in ascending label order; per-packet labels in stream
 *   order (-1 for anything that is not a kept pixel).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ECORRUPT (-4)

#define PIX_PERIOD (1LL << 34)
#define TDC_PERIOD (1LL << 36)

typedef struct orc_config {
    int32_t rx, ry, dt_ticks, mode;      /* mode 0 = CC, 1 = PAPER */
    int64_t tof_max_ticks;
    int64_t wrap_thr_pix_ticks, wrap_thr_tdc_ticks;
    const int16_t *timewalk_lut;         /* 1024 entries (ticks) or NULL */
    int32_t strict;                      /* unknown headers are an error */
    int32_t reserved;
    int64_t epoch0_pix, epoch0_tdc;      /* wraps before the first packet (a slice
                                            cut from the middle of a stream) */
    int32_t have_prev_pix, have_prev_tdc;/* the slice continues a stream: the step
                                            rule applies to its first packet too, */
    int64_t prev_pix_raw, prev_tdc_raw;  /* against these previous raw values    */
} orc_config;

typedef struct orc_cluster {
    int64_t label, shot, t0, s_tot, s_x, s_y, s_t;
    int32_t n, n_peaks;
    double x, y, tof;
} orc_cluster;

typedef struct orc_counters {
    int64_t packets, pixels, tdcs, corrupt, dropped_pre_trigger, dropped_background,
            kept, clusters, peaks;
} orc_counters;

/* per-packet diagnostic view */
typedef struct orc_packet_info {
    int32_t type;            /* 1 pixel, 2 TDC, 0 other */
    int32_t x, y, tot;
    int64_t t;               /* unwrapped time, ticks */
    int64_t shot;            /* -1 unless kept */
    int64_t tof;             /* t - t_trig[shot] before timewalk, kept only */
} orc_packet_info;

typedef struct kept_t {
    int64_t idx;     /* stream index (0-based within the call) */
    int64_t shot;
    int64_t t;       /* corrected time */
    int32_t x, y, tot;
    int32_t peak;
} kept_t;

static int cmp_kept(const void *a, const void *b) {
    const kept_t *p = (const kept_t *)a, *q = (const kept_t *)b;
    if (p->shot != q->shot) return p->shot < q->shot ? -1 : 1;
    if (p->t != q->t) return p->t < q->t ? -1 : 1;
    if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
    return 0;
}

static int adjacent(const orc_config *c, const kept_t *a, const kept_t *b) {
    if (a->shot != b->shot) return 0;
    int64_t dx = a->x - b->x, dy = a->y - b->y, dt = a->t - b->t;
    if (dx < 0) dx = -dx;
    if (dy < 0) dy = -dy;
    if (dt < 0) dt = -dt;
    return dx <= c->rx && dy <= c->ry && dt <= c->dt_ticks;
}

/* j outshines i: higher ToT, or equal ToT and later in the stream (Sec. V.B) */
static int brighter(const kept_t *j, const kept_t *i) {
    return j->tot > i->tot || (j->tot == i->tot && j->idx > i->idx);
}

int orc_run(const orc_config *cfg, const uint64_t *pk, int64_t n, int64_t idx_base,
            int64_t *labels, uint8_t *is_peak, orc_packet_info *info,
            orc_cluster **out_clusters, int64_t *out_n_clusters,
            int64_t **out_trig, int64_t *out_n_trig, orc_counters *cnt) {
    if (!cfg || (n > 0 && !pk) || n < 0 || cfg->rx < 0 || cfg->ry < 0 || cfg->dt_ticks < 0 ||
        cfg->rx > 255 || cfg->ry > 255 || cfg->tof_max_ticks < 0)
        return ORC_EINVAL;
    orc_counters c;
    memset(&c, 0, sizeof c);
    c.packets = n;

    if (labels) for (int64_t i = 0; i < n; i++) labels[i] = -1;
    if (is_peak) for (int64_t i = 0; i < n; i++) is_peak[i] = 0;

    /* ---- 1+2: decode and unwrap, sequentially, per stream ---- */
    int32_t *type = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
    int64_t *t = (int64_t *)calloc((size_t)(n + 1), sizeof(int64_t));
    int32_t *px = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
    int32_t *py = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
    int32_t *ptot = (int32_t *)calloc((size_t)(n + 1), sizeof(int32_t));
    if (!type || !t || !px || !py || !ptot) return ORC_ENOMEM;
    int have_pix = cfg->have_prev_pix != 0, have_tdc = cfg->have_prev_tdc != 0;
    int64_t prev_pix = cfg->prev_pix_raw, prev_tdc = cfg->prev_tdc_raw;
    int64_t epoch_pix = cfg->epoch0_pix, epoch_tdc = cfg->epoch0_tdc;
    for (int64_t i = 0; i < n; i++) {
        uint64_t w = pk[i];
        unsigned hdr = (unsigned)(w >> 60);
        if (hdr == 0xB) {
            uint64_t dcol = (w >> 53) & 0x7F, spix = (w >> 47) & 0x3F, pix = (w >> 44) & 0x7;
            uint64_t toa = (w >> 30) & 0x3FFF, tot = (w >> 20) & 0x3FF, ftoa = (w >> 16) & 0xF;
            uint64_t spidr = w & 0xFFFF;
            int64_t coarse = (int64_t)((spidr << 14) | toa);
            int64_t raw = (coarse * 16 - (int64_t)ftoa) % PIX_PERIOD;
            if (raw < 0) raw += PIX_PERIOD;
            if (have_pix) {
                int64_t d = raw - prev_pix;
                if (d < -cfg->wrap_thr_pix_ticks) epoch_pix += 1;
                else if (d > cfg->wrap_thr_pix_ticks) epoch_pix -= 1;
            }
            have_pix = 1;
            prev_pix = raw;
            type[i] = 1;
            px[i] = (int32_t)(2 * dcol + (pix >> 2));
            py[i] = (int32_t)(4 * spix + (pix & 3));
            ptot[i] = (int32_t)tot;
            t[i] = raw + epoch_pix * PIX_PERIOD;
            c.pixels++;
        } else if (hdr == 0x6) {
            int64_t coarse = (int64_t)((w >> 9) & ((1ULL << 35) - 1));
            int64_t raw = (2 * coarse) % TDC_PERIOD;
            if (have_tdc) {
                int64_t d = raw - prev_tdc;
                if (d < -cfg->wrap_thr_tdc_ticks) epoch_tdc += 1;
                else if (d > cfg->wrap_thr_tdc_ticks) epoch_tdc -= 1;
            }
            have_tdc = 1;
            prev_tdc = raw;
            type[i] = 2;
            t[i] = raw + epoch_tdc * TDC_PERIOD;
            c.tdcs++;
        } else {
            type[i] = 0;
            c.corrupt++;
        }
    }
    int status = ORC_OK;
    if (cfg->strict && c.corrupt) status = ORC_ECORRUPT;

    /* ---- 3: triggers ---- */
    int64_t ntrig = c.tdcs;
    int64_t *trig = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ntrig + 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++)
        if (type[i] == 2) trig[k++] = t[i];
    for (int64_t j = 1; j < ntrig; j++)
        if (trig[j] < trig[j - 1]) status = ORC_ECORRUPT;

    /* ---- 4: shot binning, background cut, timewalk ---- */
    kept_t *kp = (kept_t *)malloc(sizeof(kept_t) * (size_t)(c.pixels + 1));
    int64_t nk = 0;
    for (int64_t i = 0; i < n; i++) {
        if (info) {
            info[i].type = type[i]; info[i].x = px[i]; info[i].y = py[i]; info[i].tot = ptot[i];
            info[i].t = t[i]; info[i].shot = -1; info[i].tof = 0;
        }
        if (type[i] != 1) continue;
        /* upper_bound: first trigger strictly later than t */
        int64_t lo = 0, hi = ntrig;
        while (lo < hi) {
            int64_t mid = lo + (hi - lo) / 2;
            if (trig[mid] <= t[i]) lo = mid + 1; else hi = mid;
        }
        int64_t shot = lo - 1;
        if (shot < 0) { c.dropped_pre_trigger++; continue; }
        int64_t tof = t[i] - trig[shot];
        if (tof > cfg->tof_max_ticks) { c.dropped_background++; continue; }
        int64_t tc = t[i];
        if (cfg->timewalk_lut) tc -= cfg->timewalk_lut[ptot[i]];
        kp[nk].idx = i; kp[nk].shot = shot; kp[nk].t = tc;
        kp[nk].x = px[i]; kp[nk].y = py[i]; kp[nk].tot = ptot[i]; kp[nk].peak = 0;
        if (info) { info[i].shot = shot; info[i].tof = tof; }
        nk++;
    }
    c.kept = nk;

    /* ---- 5: stable order by (shot, corrected time, stream index) ---- */
    qsort(kp, (size_t)nk, sizeof(kept_t), cmp_kept);

    /* ---- 6+7: per shot, dense 256x256 grid of sorted ranks ---- */
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * 65536);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
    int64_t *root = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
    orc_cluster *pm = cfg->mode == 1 ? (orc_cluster *)calloc((size_t)(nk + 1), sizeof(orc_cluster)) : NULL;
    for (int q = 0; q < 65536; q++) head[q] = -1;
    for (int64_t s0 = 0; s0 < nk;) {
        int64_t s1 = s0;
        while (s1 < nk && kp[s1].shot == kp[s0].shot) s1++;
        /* insert in descending rank so each cell lists ranks ascending */
        for (int64_t r = s1 - 1; r >= s0; r--) {
            int q = kp[r].x * 256 + kp[r].y;
            next[r] = head[q];
            head[q] = r;
        }
        for (int64_t r = s0; r < s1; r++) root[r] = -1;
        /* local maxima over the box neighbourhood */
        for (int64_t r = s0; r < s1; r++) {
            int peak = 1;
            for (int xx = kp[r].x - cfg->rx; xx <= kp[r].x + cfg->rx && peak; xx++) {
                if (xx < 0 || xx > 255) continue;
                for (int yy = kp[r].y - cfg->ry; yy <= kp[r].y + cfg->ry && peak; yy++) {
                    if (yy < 0 || yy > 255) continue;
                    for (int64_t j = head[xx * 256 + yy]; j >= 0; j = next[j])
                        if (j != r && adjacent(cfg, &kp[r], &kp[j]) && brighter(&kp[j], &kp[r])) { peak = 0; break; }
                }
            }
            kp[r].peak = peak;
        }
        /* connected components: BFS from each unvisited pixel in sorted order */
        if (cfg->mode == 0) {
            for (int64_t r = s0; r < s1; r++) {
                if (root[r] >= 0) continue;
                int64_t qh = 0, qt = 0;
                root[r] = r;
                queue[qt++] = r;
                while (qh < qt) {
                    int64_t u = queue[qh++];
                    for (int xx = kp[u].x - cfg->rx; xx <= kp[u].x + cfg->rx; xx++) {
                        if (xx < 0 || xx > 255) continue;
                        for (int yy = kp[u].y - cfg->ry; yy <= kp[u].y + cfg->ry; yy++) {
                            if (yy < 0 || yy > 255) continue;
                            for (int64_t j = head[xx * 256 + yy]; j >= 0; j = next[j])
                                if (root[j] < 0 && adjacent(cfg, &kp[u], &kp[j])) {
                                    root[j] = r;
                                    queue[qt++] = j;
                                }
                        }
                    }
                }
            }
        }
        /* PAPER mode (Sec. V.C): for each local maximum r, sums over its box
           neighbourhood {j : A_rj = 1}, which contains r itself.  Gathered
           here, while the grid holds this shot; t0 is the earliest corrected
           time in the neighbourhood. */
        if (cfg->mode == 1) {
            for (int64_t r = s0; r < s1; r++) {
                if (!kp[r].peak) continue;
                orc_cluster *o = &pm[r];
                memset(o, 0, sizeof *o);
                o->label = idx_base + kp[r].idx;
                o->shot = kp[r].shot;
                o->n_peaks = 1;
                o->t0 = kp[r].t;
                for (int pass = 0; pass < 2; pass++)
                    for (int xx = kp[r].x - cfg->rx; xx <= kp[r].x + cfg->rx; xx++) {
                        if (xx < 0 || xx > 255) continue;
                        for (int yy = kp[r].y - cfg->ry; yy <= kp[r].y + cfg->ry; yy++) {
                            if (yy < 0 || yy > 255) continue;
                            for (int64_t j = head[xx * 256 + yy]; j >= 0; j = next[j]) {
                                if (!adjacent(cfg, &kp[r], &kp[j])) continue;
                                if (pass == 0) {            /* earliest time first */
                                    if (kp[j].t < o->t0) o->t0 = kp[j].t;
                                    continue;
                                }
                                o->n += 1;
                                o->s_tot += kp[j].tot;
                                o->s_x += (int64_t)kp[j].x * kp[j].tot;
                                o->s_y += (int64_t)kp[j].y * kp[j].tot;
                                o->s_t += (kp[j].t - o->t0) * kp[j].tot;
                            }
                        }
                    }
            }
        }
        for (int64_t r = s1 - 1; r >= s0; r--) head[kp[r].x * 256 + kp[r].y] = -1;
        s0 = s1;
    }

    /* ---- 8: sums ---- */
    orc_cluster *cl = NULL;
    int64_t ncl = 0;
    for (int64_t r = 0; r < nk; r++) c.peaks += kp[r].peak;
    if (cfg->mode == 0) {
        /* one cluster per root rank; order clusters by label (root stream index) */
        int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nk + 1));
        for (int64_t r = 0; r < nk; r++) slot[r] = -1;
        for (int64_t r = 0; r < nk; r++)
            if (root[r] == r) ncl++;
        cl = (orc_cluster *)calloc((size_t)(ncl + 1), sizeof(orc_cluster));
        /* list roots, then sort by stream index */
        int64_t *roots = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncl + 1));
        int64_t m = 0;
        for (int64_t r = 0; r < nk; r++)
            if (root[r] == r) roots[m++] = r;
        /* insertion into an array indexed by stream index order */
        int64_t *by_idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
        for (int64_t i = 0; i < n; i++) by_idx[i] = -1;
        for (int64_t a = 0; a < ncl; a++) by_idx[kp[roots[a]].idx] = roots[a];
        m = 0;
        for (int64_t i = 0; i < n; i++)
            if (by_idx[i] >= 0) slot[by_idx[i]] = m++;
        for (int64_t r = 0; r < nk; r++) {
            int64_t rr = root[r];
            orc_cluster *o = &cl[slot[rr]];
            if (o->n == 0) {
                o->label = idx_base + kp[rr].idx;
                o->shot = kp[rr].shot;
                o->t0 = kp[rr].t;
            }
            o->n += 1;
            o->s_tot += kp[r].tot;
            o->s_x += (int64_t)kp[r].x * kp[r].tot;
            o->s_y += (int64_t)kp[r].y * kp[r].tot;
            o->s_t += (kp[r].t - o->t0) * kp[r].tot;
            o->n_peaks += kp[r].peak;
        }
        if (labels)
            for (int64_t r = 0; r < nk; r++) labels[kp[r].idx] = idx_base + kp[root[r]].idx;
        free(slot); free(roots); free(by_idx);
    } else {
        /* PAPER mode: one record per local maximum, in ascending stream index */
        ncl = c.peaks;
        cl = (orc_cluster *)calloc((size_t)(ncl + 1), sizeof(orc_cluster));
        int64_t *by_idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
        for (int64_t i = 0; i < n; i++) by_idx[i] = -1;
        for (int64_t r = 0; r < nk; r++)
            if (kp[r].peak) by_idx[kp[r].idx] = r;
        int64_t m = 0;
        for (int64_t i = 0; i < n; i++)
            if (by_idx[i] >= 0) cl[m++] = pm[by_idx[i]];
        /* there is no partition in PAPER mode: each kept pixel is labelled
           with its own stream index */
        if (labels)
            for (int64_t r = 0; r < nk; r++) labels[kp[r].idx] = idx_base + kp[r].idx;
        free(by_idx);
        free(pm);
    }
    for (int64_t a = 0; a < ncl; a++) {
        orc_cluster *o = &cl[a];
        o->x = (double)o->s_x / (double)o->s_tot;
        o->y = (double)o->s_y / (double)o->s_tot;
        o->tof = (double)(o->t0 - trig[o->shot]) + (double)o->s_t / (double)o->s_tot;
    }
    c.clusters = ncl;
    if (is_peak)
        for (int64_t r = 0; r < nk; r++) is_peak[kp[r].idx] = (uint8_t)kp[r].peak;

    if (out_clusters) *out_clusters = cl; else free(cl);
    if (out_n_clusters) *out_n_clusters = ncl;
    if (out_trig) *out_trig = trig; else free(trig);
    if (out_n_trig) *out_n_trig = ntrig;
    if (cnt) *cnt = c;
    free(type); free(t); free(px); free(py); free(ptot); free(kp);
    free(head); free(next); free(root); free(queue);
    return status;
}

void orc_free(void *p) { free(p); }
