/*
 * tpx_synth.c -- seeded synthetic TimePix3-style packet streams.
 *
 * Input generator only: it draws charge clouds and encodes them as 64-bit
 * packets, and holds none of the decoding, unwrapping, binning, clustering or
 * centroiding arithmetic of the method. Both the CUDA path and the CPU oracle
 * consume its output; neither links it.
 *
 * Physical model (stand-in for the paper's argon ATI / ion data, which are not
 * available): laser triggers at a fixed period (1 kHz by default, Sec. II); per
 * trigger a number of particles, each an isotropic Gaussian MCP charge cloud
 * whose pixel ToT is floor(peak * exp(-r^2 / 2 sigma^2)) at integer pixel
 * centres, kept where ToT >= tot_min; ToA = trigger + time of flight + N(0,
 * jitter) rounded to 1.5625 ns ticks. A pixel reports once it falls back below
 * threshold (Sec. III), so the stream is ordered by readout time = ToA +
 * 16 * ToT ticks + U(0, readout_jitter). TDC trigger packets are emitted at
 * the trigger time.
 *
 * Packet layout (project-defined, TPX3-style; the paper relies on a vendor
 * converter and prints no bit layout):
 *   pixel : [63:60]=0xB, [59:53]=dcol, [52:47]=spix, [46:44]=pix,
 *           [43:30]=ToA (25 ns), [29:20]=ToT (25 ns), [19:16]=fToA, [15:0]=spidr
 *           x = 2*dcol + (pix>>2), y = 4*spix + (pix&3),
 *           time in 1.5625 ns ticks = ((spidr<<14 | ToA)*16 - fToA) mod 2^34
 *   TDC   : [63:60]=0x6, [59:56]=0xF, [55:44]=trigger counter, [43:9]=coarse
 *           (3.125 ns), time in ticks = 2*coarse mod 2^36
 *
 * Randomness: xoshiro256** streams seeded through splitmix64 from
 * (seed, shot, stream id), so any shot range regenerates identically and shots
 * can be generated in parallel.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_PIX_PERIOD (1LL << 34)
#define SYN_TDC_PERIOD (1LL << 36)

typedef struct synth_params {
    int64_t shot_begin;          /* first trigger index generated          */
    int64_t shot_end;            /* one past the last trigger index        */
    uint64_t seed;
    int32_t poisson;             /* 1: particles ~ Poisson(mean); 0: fixed */
    int32_t n_threads;
    double particles_per_shot;
    double sigma_px;
    double peak_lo, peak_hi;     /* peak ToT, 25 ns units                  */
    double tot_min;              /* keep pixel iff ToT >= tot_min          */
    double tof_lo_ns, tof_hi_ns; /* time of flight after the trigger       */
    double jitter_ns;            /* sigma of per-pixel ToA jitter          */
    double pair_frac;            /* probability a particle gets a partner  */
    double pair_sep_lo, pair_sep_hi;       /* px                            */
    double pair_dtoa_lo_ns, pair_dtoa_hi_ns;
    double pair_amp_lo, pair_amp_hi;       /* partner peak / primary peak   */
    double dark_per_shot;        /* mean dark counts per trigger period    */
    int64_t trig_period_ticks;   /* 640000 ticks = 1 ms                    */
    int64_t t_start_ticks;       /* time of trigger 0 (even)               */
    int64_t readout_jitter_ticks;/* U(0, this) added to the readout time   */
    double timewalk_a, timewalk_b, timewalk_c; /* optional ToA delay
                                    a/(ToT+b)+c ns added per pixel (0: off) */
} synth_params;

/* ---------------------------------------------------------------- RNG ---- */
static inline uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
typedef struct { uint64_t s[4]; int has_spare; double spare; } rng_t;
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t out = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return out;
}
static void rng_seed(rng_t *r, uint64_t seed, uint64_t shot, uint64_t stream) {
    uint64_t sm = seed * 0xD1B54A32D192ED03ULL ^ (shot + 0x632BE59BD9B4E019ULL) * 0x9E3779B97F4A7C15ULL
                  ^ (stream + 1) * 0xA24BAED4963EE407ULL;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&sm);
    r->has_spare = 0;
}
static inline double rng_u01(rng_t *r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static inline double rng_uniform(rng_t *r, double lo, double hi) { return lo + (hi - lo) * rng_u01(r); }
static double rng_normal(rng_t *r) {           /* Box-Muller */
    if (r->has_spare) { r->has_spare = 0; return r->spare; }
    double u1, u2;
    do { u1 = rng_u01(r); } while (u1 <= 0.0);
    u2 = rng_u01(r);
    double rad = sqrt(-2.0 * log(u1)), th = 6.283185307179586 * u2;
    r->spare = rad * sin(th); r->has_spare = 1;
    return rad * cos(th);
}
static int64_t rng_poisson(rng_t *r, double mean) {
    if (mean <= 0) return 0;
    if (mean < 60) {                            /* Knuth multiplication */
        double L = exp(-mean), p = 1.0; int64_t k = 0;
        do { k++; p *= rng_u01(r); } while (p > L);
        return k - 1;
    }
    double v = floor(mean + sqrt(mean) * rng_normal(r) + 0.5); /* large mean */
    return v < 0 ? 0 : (int64_t)v;
}

/* ------------------------------------------------------------ encoding ---- */
static inline uint64_t encode_pixel(int x, int y, int tot, int64_t t_ticks) {
    uint64_t raw = (uint64_t)(t_ticks & (SYN_PIX_PERIOD - 1));
    uint64_t coarse = (raw + 15) >> 4;          /* 25 ns units, ceil      */
    uint64_t ftoa = coarse * 16 - raw;           /* 0..15                  */
    coarse &= (1ULL << 30) - 1;
    uint64_t dcol = (uint64_t)(x >> 1), spix = (uint64_t)(y >> 2);
    uint64_t pix = (uint64_t)(((x & 1) << 2) | (y & 3));
    return (0xBULL << 60) | (dcol << 53) | (spix << 47) | (pix << 44) |
           ((coarse & 0x3FFF) << 30) | ((uint64_t)(tot & 0x3FF) << 20) |
           (ftoa << 16) | (coarse >> 14);
}
static inline uint64_t encode_tdc(int64_t t_ticks, int64_t counter) {
    uint64_t raw = (uint64_t)(t_ticks & (SYN_TDC_PERIOD - 1));
    return (0x6ULL << 60) | (0xFULL << 56) | ((uint64_t)(counter & 0xFFF) << 44) | ((raw >> 1) << 9);
}

/* ----------------------------------------------------------- shot data ---- */
typedef struct { int32_t q; int32_t tot; double amp; int64_t toa; int64_t readout; int64_t order; } hit_t;
typedef struct { int64_t shot; double cx, cy, t, peak; int32_t kind; } part_t;

typedef struct {
    uint64_t *pk; int64_t n_pk, cap_pk;
    part_t *pt; int64_t n_pt, cap_pt;
    hit_t *h; int64_t n_h, cap_h;
    hit_t *h2; int64_t cap_h2;
    int32_t *map_tag; int32_t *map_idx;  /* per-pixel last hit, tagged by shot */
    int64_t *rank_key; int64_t cap_rk;
    int64_t first_pix_t, first_tdc_t;    /* true times of the first emitted packets */
} worker_t;

#define GROW(ptr, n, cap, type)                                                        \
    do { if ((n) >= (cap)) { int64_t nc = (cap) ? (cap) * 2 : 4096; while (nc <= (n)) nc *= 2; \
        ptr = (type *)realloc(ptr, (size_t)nc * sizeof(type)); cap = nc; } } while (0)

static void add_hit(worker_t *w, int32_t tag, int q, double amp, int64_t toa) {
    /* A pixel fires once while it is over threshold: a second hit that arrives
       within the first one's ToT duration adds its amplitude and keeps the
       earlier ToA; otherwise it becomes a separate packet. */
    if (w->map_tag[q] == tag) {
        hit_t *e = &w->h[w->map_idx[q]];
        int64_t first = e->toa < toa ? e->toa : toa;
        double first_amp = e->toa <= toa ? e->amp : amp;
        int64_t busy = 16 * (int64_t)(first_amp > 1023 ? 1023 : floor(first_amp));
        int64_t second = e->toa < toa ? toa : e->toa;
        if (second < first + busy) { e->amp += amp; e->toa = first; return; }
    }
    GROW(w->h, w->n_h, w->cap_h, hit_t);
    hit_t *n = &w->h[w->n_h];
    n->q = q; n->amp = amp; n->toa = toa; n->tot = 0; n->readout = 0; n->order = w->n_h;
    w->map_tag[q] = tag; w->map_idx[q] = (int32_t)w->n_h;
    w->n_h++;
}

static void emit_cloud(worker_t *w, const synth_params *p, rng_t *r, int32_t tag,
                       double cx, double cy, double peak, double t_ticks) {
    if (peak < p->tot_min || peak <= 0) return;
    const double s2 = 2.0 * p->sigma_px * p->sigma_px;
    double R = sqrt(s2 * log(peak / (p->tot_min > 0 ? p->tot_min : 1e-9)));
    int x0 = (int)ceil(cx - R), x1 = (int)floor(cx + R);
    int y0 = (int)ceil(cy - R), y1 = (int)floor(cy + R);
    if (x0 < 0) x0 = 0; if (y0 < 0) y0 = 0; if (x1 > 255) x1 = 255; if (y1 > 255) y1 = 255;
    double ex[64], ey[64];
    if (x1 - x0 >= 64) x1 = x0 + 63; if (y1 - y0 >= 64) y1 = y0 + 63;
    for (int x = x0; x <= x1; x++) ex[x - x0] = exp(-((x - cx) * (x - cx)) / s2);
    for (int y = y0; y <= y1; y++) ey[y - y0] = exp(-((y - cy) * (y - cy)) / s2);
    const double jt = p->jitter_ns / 1.5625;
    for (int x = x0; x <= x1; x++)
        for (int y = y0; y <= y1; y++) {
            double a = peak * ex[x - x0] * ey[y - y0];
            if (floor(a) < p->tot_min) continue;
            double toa = t_ticks + jt * rng_normal(r);
            add_hit(w, tag, x * 256 + y, a, (int64_t)llround(toa));
        }
}

static int cmp_key(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* dark counts of trigger window k: uniform ToA over the period, random pixel */
static void gen_dark(worker_t *w, const synth_params *p, int64_t k, int64_t t_trig) {
    if (p->dark_per_shot <= 0) return;
    rng_t r; rng_seed(&r, p->seed, (uint64_t)k, 7);
    int64_t nd = rng_poisson(&r, p->dark_per_shot);
    for (int64_t i = 0; i < nd; i++) {
        int64_t toa = t_trig + (int64_t)(rng_u01(&r) * (double)p->trig_period_ticks);
        int q = (int)(rng_next(&r) & 0xFFFF);
        int tot = 10 + (int)(rng_next(&r) % 51);
        int64_t ro = toa + 16 * tot + (int64_t)(rng_next(&r) % (uint64_t)(p->readout_jitter_ticks + 1));
        GROW(w->h, w->n_h, w->cap_h, hit_t);
        hit_t *n = &w->h[w->n_h];
        n->q = q; n->amp = tot; n->tot = tot; n->toa = toa; n->readout = ro; n->order = -1;
        w->n_h++;
    }
}

/* all hits of shot k (its particles, its dark counts), appended to w->h with
   their readout times; the particles are recorded as truth if asked */
static void gen_hits(worker_t *w, const synth_params *p, int64_t k, int truth, int particles) {
    const int64_t t_trig = p->t_start_ticks + k * p->trig_period_ticks;
    const int32_t tag = (int32_t)(k & 0x3FFFFFFF) * 2 + 1 + (truth ? 0 : 1);
    rng_t r; rng_seed(&r, p->seed, (uint64_t)k, 0);
    const int64_t h0 = w->n_h;
    int64_t np = p->poisson ? rng_poisson(&r, p->particles_per_shot) : (int64_t)p->particles_per_shot;
    const double tick = 1.5625;
    for (int64_t i = 0; i < np && particles; i++) {
        double cx = rng_uniform(&r, 0.0, 256.0), cy = rng_uniform(&r, 0.0, 256.0);
        double peak = rng_uniform(&r, p->peak_lo, p->peak_hi);
        double tof = rng_uniform(&r, p->tof_lo_ns, p->tof_hi_ns);
        double t0 = (double)t_trig + tof / tick;
        int pair = p->pair_frac > 0 && rng_u01(&r) < p->pair_frac;
        if (truth) {
            GROW(w->pt, w->n_pt, w->cap_pt, part_t);
            w->pt[w->n_pt++] = (part_t){k, cx, cy, t0, peak, pair ? 1 : 0};
        }
        emit_cloud(w, p, &r, tag, cx, cy, peak, t0);
        if (pair) {
            double sep = rng_uniform(&r, p->pair_sep_lo, p->pair_sep_hi);
            double ang = rng_uniform(&r, 0.0, 6.283185307179586);
            double dt = rng_uniform(&r, p->pair_dtoa_lo_ns, p->pair_dtoa_hi_ns) / tick;
            double ratio = rng_uniform(&r, p->pair_amp_lo, p->pair_amp_hi);
            double cx2 = cx + sep * cos(ang), cy2 = cy + sep * sin(ang);
            if (truth) {
                GROW(w->pt, w->n_pt, w->cap_pt, part_t);
                w->pt[w->n_pt++] = (part_t){k, cx2, cy2, t0 + dt, peak * ratio, 2};
            }
            emit_cloud(w, p, &r, tag, cx2, cy2, peak * ratio, t0 + dt);
        }
    }
    /* finalise particle hits: ToT, optional timewalk delay, readout time */
    for (int64_t i = h0; i < w->n_h; i++) {
        hit_t *h = &w->h[i];
        int tot = (int)floor(h->amp);
        if (tot > 1023) tot = 1023;
        h->tot = tot;
        if (p->timewalk_a != 0 || p->timewalk_c != 0)
            h->toa += (int64_t)llround((p->timewalk_a / ((double)tot + p->timewalk_b) + p->timewalk_c) / tick);
        h->readout = h->toa + 16 * (int64_t)tot + (int64_t)(rng_next(&r) % (uint64_t)(p->readout_jitter_ticks + 1));
    }
    gen_dark(w, p, k, t_trig);
}

/* Trigger window k of the stream: its TDC packet, then -- in readout order --
   the hits of shot k read out before trigger k+1 and the hits of shot k-1
   read out after trigger k. */
static void gen_shot(worker_t *w, const synth_params *p, int64_t k) {
    const int64_t t_trig = p->t_start_ticks + k * p->trig_period_ticks;
    const int64_t t_next = t_trig + p->trig_period_ticks;
    const int last = k + 1 == p->shot_end;
    w->n_h = 0;
    gen_hits(w, p, k, 1, 1);
    int64_t j = 0;
    for (int64_t i = 0; i < w->n_h; i++)
        if (w->h[i].readout < t_next || last) w->h[j++] = w->h[i];
    w->n_h = j;
    if (k > 0) {
        /* particles of shot k-1 can only be late when their ToF plus the
           longest readout delay reaches the next trigger */
        const double max_delay = 16.0 * 1023 + (double)p->readout_jitter_ticks + 8.0 * p->jitter_ns / 1.5625;
        const int late_particles = p->tof_hi_ns / 1.5625 + max_delay >= (double)p->trig_period_ticks;
        if (late_particles || p->dark_per_shot > 0) {
            int64_t keep_from = w->n_h;
            gen_hits(w, p, k - 1, 0, late_particles);
            j = keep_from;
            for (int64_t i = keep_from; i < w->n_h; i++)
                if (w->h[i].readout >= t_trig) w->h[j++] = w->h[i];
            w->n_h = j;
        }
    }
    /* readout order: by readout time, ties by generation order */
    GROW(w->rank_key, w->n_h, w->cap_rk, int64_t);
    for (int64_t i = 0; i < w->n_h; i++) {
        int64_t rel = w->h[i].readout - t_trig + (1LL << 22);
        if (rel < 0) rel = 0;
        w->rank_key[i] = (rel << 24) | i;
    }
    qsort(w->rank_key, (size_t)w->n_h, sizeof(int64_t), cmp_key);
    GROW(w->pk, w->n_pk + w->n_h + 1, w->cap_pk, uint64_t);
    if (w->first_tdc_t < 0) w->first_tdc_t = t_trig;
    if (w->first_pix_t < 0 && w->n_h > 0) w->first_pix_t = w->h[w->rank_key[0] & 0xFFFFFF].toa;
    w->pk[w->n_pk++] = encode_tdc(t_trig, k);
    for (int64_t i = 0; i < w->n_h; i++) {
        hit_t *h = &w->h[w->rank_key[i] & 0xFFFFFF];
        w->pk[w->n_pk++] = encode_pixel(h->q >> 8, h->q & 255, h->tot, h->toa);
    }
}

typedef struct {
    const synth_params *p;
    int64_t s0, s1;
    worker_t w;
} job_t;

static void *run_job(void *arg) {
    job_t *j = (job_t *)arg;
    j->w.map_tag = (int32_t *)calloc(65536, sizeof(int32_t));
    j->w.map_idx = (int32_t *)calloc(65536, sizeof(int32_t));
    j->w.first_pix_t = -1;
    j->w.first_tdc_t = -1;
    for (int64_t k = j->s0; k < j->s1; k++) gen_shot(&j->w, j->p, k);
    free(j->w.map_tag); free(j->w.map_idx); free(j->w.h); free(j->w.rank_key);
    j->w.map_tag = NULL; j->w.map_idx = NULL; j->w.h = NULL; j->w.rank_key = NULL;
    return NULL;
}

typedef struct synth_result {
    int n_jobs;
    job_t *jobs;
    int64_t n_packets, n_particles;
} synth_result;

synth_result *synth_generate(const synth_params *p_in) {
    synth_result *res = (synth_result *)calloc(1, sizeof(synth_result));
    synth_params *p = (synth_params *)malloc(sizeof(synth_params));
    *p = *p_in;
    int64_t ns = p->shot_end - p->shot_begin;
    int nt = p->n_threads > 0 ? p->n_threads : 1;
    if (ns < nt) nt = ns > 0 ? (int)ns : 1;
    res->n_jobs = nt;
    res->jobs = (job_t *)calloc((size_t)nt, sizeof(job_t));
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nt);
    for (int i = 0; i < nt; i++) {
        res->jobs[i].p = p;
        res->jobs[i].s0 = p->shot_begin + ns * i / nt;
        res->jobs[i].s1 = p->shot_begin + ns * (i + 1) / nt;
        pthread_create(&th[i], NULL, run_job, &res->jobs[i]);
    }
    for (int i = 0; i < nt; i++) pthread_join(th[i], NULL);
    free(th);
    for (int i = 0; i < nt; i++) {
        res->n_packets += res->jobs[i].w.n_pk;
        res->n_particles += res->jobs[i].w.n_pt;
    }
    return res;
}

int64_t synth_n_packets(const synth_result *r) { return r->n_packets; }

/* true times of the first pixel and first TDC packet of the generated range
   (-1 if none): a slice's wrap counts before its first packet follow from them */
void synth_first_times(const synth_result *r, int64_t *pix_t, int64_t *tdc_t) {
    *pix_t = -1; *tdc_t = -1;
    for (int i = 0; i < r->n_jobs; i++) {
        if (*pix_t < 0 && r->jobs[i].w.first_pix_t >= 0) *pix_t = r->jobs[i].w.first_pix_t;
        if (*tdc_t < 0 && r->jobs[i].w.first_tdc_t >= 0) *tdc_t = r->jobs[i].w.first_tdc_t;
    }
}
int64_t synth_n_particles(const synth_result *r) { return r->n_particles; }

typedef struct { uint64_t *dst; const uint64_t *src; int64_t n; } cp_t;
static void *run_copy(void *a) { cp_t *c = (cp_t *)a; memcpy(c->dst, c->src, (size_t)c->n * 8); return NULL; }

void synth_copy_packets(const synth_result *r, uint64_t *dst) {
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)r->n_jobs);
    cp_t *cp = (cp_t *)malloc(sizeof(cp_t) * (size_t)r->n_jobs);
    int64_t off = 0;
    for (int i = 0; i < r->n_jobs; i++) {
        cp[i] = (cp_t){dst + off, r->jobs[i].w.pk, r->jobs[i].w.n_pk};
        off += r->jobs[i].w.n_pk;
        pthread_create(&th[i], NULL, run_copy, &cp[i]);
    }
    for (int i = 0; i < r->n_jobs; i++) pthread_join(th[i], NULL);
    free(th); free(cp);
}

void synth_copy_truth(const synth_result *r, int64_t *shot, double *cx, double *cy,
                      double *t, double *peak, int32_t *kind) {
    int64_t o = 0;
    for (int i = 0; i < r->n_jobs; i++)
        for (int64_t j = 0; j < r->jobs[i].w.n_pt; j++, o++) {
            const part_t *q = &r->jobs[i].w.pt[j];
            shot[o] = q->shot; cx[o] = q->cx; cy[o] = q->cy; t[o] = q->t; peak[o] = q->peak; kind[o] = q->kind;
        }
}

void synth_free(synth_result *r) {
    if (!r) return;
    for (int i = 0; i < r->n_jobs; i++) { free(r->jobs[i].w.pk); free(r->jobs[i].w.pt); }
    if (r->n_jobs) free((void *)r->jobs[0].p);
    free(r->jobs); free(r);
}

/* Encoders for hand-built test streams (same layout as above). */
void synth_encode_pixels(const int32_t *x, const int32_t *y, const int32_t *tot,
                         const int64_t *t_ticks, int64_t n, uint64_t *out) {
    for (int64_t i = 0; i < n; i++) out[i] = encode_pixel(x[i], y[i], tot[i], t_ticks[i]);
}
void synth_encode_tdcs(const int64_t *t_ticks, const int64_t *counter, int64_t n, uint64_t *out) {
    for (int64_t i = 0; i < n; i++) out[i] = encode_tdc(t_ticks[i], counter[i]);
}
