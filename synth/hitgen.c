/*
 * Seeded synthetic Timepix hit streams.
 *
 * This module only draws inputs: it holds none of the clustering arithmetic
 * and is shared, as the sole common piece, by the CPU oracle and the CUDA
 * path.  It stands in for the beam-test datasets of the paper (Section 4,
 * table of cluster sizes), which are not available: events are random-walk
 * blobs of 1 + Geometric(p) distinct 8-connected pixels and straight tracks
 * rastered 8-connectedly, arriving as a Poisson-like process.
 *
 * Record layout (16 B, little endian): x:u16, y:u16, tot:u16, reserved:u16,
 * toa:u64 (1 tick = 1.5625 ns).
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), one stream per call.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint16_t x, y, tot, reserved;
    uint64_t toa;
} hg_hit;

typedef struct {
    uint32_t width, height;
    uint64_t n;             /* hits to emit */
    uint64_t seed;
    double event_rate;      /* events per tick; 0 -> use hit_rate */
    double hit_rate;        /* hits per tick (used when event_rate == 0) */
    double track_frac;      /* fraction of events that are straight tracks */
    uint32_t track_min, track_max;  /* track length in pixels, U{min..max} */
    double max_gradient;    /* ticks per pixel along a track, g ~ U[0, max] */
    uint32_t toa_jitter;    /* per-pixel ToA = t_event + U[0, jitter] */
    double blob_p;          /* blob size = 1 + Geometric(p) */
    double tot_mean;        /* ToT = min(tot_max, 1 + round(Exp(mean))) */
    uint32_t tot_max;
    uint32_t dead_time;     /* 1: a refire inside the previous hit's ToT is re-timed */
    uint32_t shuffle_window;/* 0: time sorted; w: key_i = i + U[0, w), stable sort */
    uint64_t t0;            /* time of the first event */
} hg_params;

/* ---- SplitMix64 ---------------------------------------------------------- */
typedef struct { uint64_t s; } hg_rng;

static uint64_t rng_next(hg_rng *r) {
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double rng_unit(hg_rng *r) {             /* [0, 1) */
    return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}
static uint64_t rng_below(hg_rng *r, uint64_t m) { /* [0, m), m > 0 */
    return m ? (uint64_t)(rng_unit(r) * (double)m) % m : 0;
}
static double rng_exp(hg_rng *r, double mean) {
    return -mean * log(1.0 - rng_unit(r));
}

/* ---- growable hit vector ------------------------------------------------- */
typedef struct { hg_hit *v; uint64_t n, cap; } hitvec;

static int hv_push(hitvec *h, hg_hit e) {
    if (h->n == h->cap) {
        uint64_t nc = h->cap ? h->cap * 2 : 1024;
        hg_hit *nv = (hg_hit *)realloc(h->v, nc * sizeof(hg_hit));
        if (!nv) return -1;
        h->v = nv; h->cap = nc;
    }
    h->v[h->n++] = e;
    return 0;
}

/* ---- stable LSD radix sort of (key, payload) by 64-bit key ---------------- */
/* Sorts perm[0..n) so that key[perm[.]] is non-decreasing; ties keep order. */
static int sort_by_key(const uint64_t *key, uint32_t *perm, uint64_t n) {
    uint32_t *tmp = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    uint64_t *kbuf = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t *ktmp = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!tmp || !kbuf || !ktmp) { free(tmp); free(kbuf); free(ktmp); return -1; }
    for (uint64_t i = 0; i < n; ++i) kbuf[i] = key[perm[i]];
    for (int shift = 0; shift < 64; shift += 8) {
        uint64_t cnt[256] = {0};
        for (uint64_t i = 0; i < n; ++i) cnt[(kbuf[i] >> shift) & 255]++;
        int skip = 0;
        for (int d = 0; d < 256; ++d) if (cnt[d] == n) skip = 1;
        if (skip) continue;
        uint64_t off = 0;
        for (int d = 0; d < 256; ++d) { uint64_t c = cnt[d]; cnt[d] = off; off += c; }
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t d = (kbuf[i] >> shift) & 255, o = cnt[d]++;
            tmp[o] = perm[i]; ktmp[o] = kbuf[i];
        }
        memcpy(perm, tmp, n * sizeof(uint32_t));
        memcpy(kbuf, ktmp, n * sizeof(uint64_t));
    }
    free(tmp); free(kbuf); free(ktmp);
    return 0;
}

static int apply_perm(hg_hit *h, const uint32_t *perm, uint64_t n) {
    hg_hit *t = (hg_hit *)malloc((n ? n : 1) * sizeof(hg_hit));
    if (!t) return -1;
    for (uint64_t i = 0; i < n; ++i) t[i] = h[perm[i]];
    memcpy(h, t, n * sizeof(hg_hit));
    free(t);
    return 0;
}

static int sort_hits_by_toa(hg_hit *h, uint64_t n) {
    uint64_t *k = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    uint32_t *p = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!k || !p) { free(k); free(p); return -1; }
    for (uint64_t i = 0; i < n; ++i) { k[i] = h[i].toa; p[i] = (uint32_t)i; }
    int rc = sort_by_key(k, p, n);
    if (!rc) rc = apply_perm(h, p, n);
    free(k); free(p);
    return rc;
}

/* ---- event shapes -------------------------------------------------------- */
static uint16_t draw_tot(hg_rng *r, const hg_params *p) {
    double v = 1.0 + floor(rng_exp(r, p->tot_mean) + 0.5);
    if (v > (double)p->tot_max) v = (double)p->tot_max;
    return (uint16_t)v;
}

/* Random-walk blob of k distinct 8-connected pixels around (cx, cy). */
static int emit_blob(hg_rng *r, const hg_params *p, uint64_t t_ev, hitvec *out) {
    uint32_t k = 1;
    while (rng_unit(r) >= p->blob_p && k < 4096) k++;
    int32_t px[4096], py[4096];
    uint32_t m = 0;
    px[m] = (int32_t)rng_below(r, p->width);
    py[m] = (int32_t)rng_below(r, p->height);
    m = 1;
    for (uint32_t attempt = 0; m < k && attempt < 64u * k; ++attempt) {
        uint32_t j = (uint32_t)rng_below(r, m);
        uint32_t d = (uint32_t)rng_below(r, 8);
        static const int dx[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
        static const int dy[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
        int32_t nx = px[j] + dx[d], ny = py[j] + dy[d];
        if (nx < 0 || ny < 0 || nx >= (int32_t)p->width || ny >= (int32_t)p->height) continue;
        int seen = 0;
        for (uint32_t q = 0; q < m; ++q) if (px[q] == nx && py[q] == ny) { seen = 1; break; }
        if (seen) continue;
        px[m] = nx; py[m] = ny; m++;
    }
    for (uint32_t q = 0; q < m; ++q) {
        hg_hit e;
        e.x = (uint16_t)px[q]; e.y = (uint16_t)py[q];
        e.tot = draw_tot(r, p); e.reserved = 0;
        e.toa = t_ev + rng_below(r, (uint64_t)p->toa_jitter + 1);
        if (hv_push(out, e)) return -1;
    }
    return (int)m;
}

/* Straight track rastered with unit steps along its major axis (8-connected). */
static int emit_track(hg_rng *r, const hg_params *p, uint64_t t_ev, hitvec *out) {
    uint32_t len = p->track_min + (uint32_t)rng_below(r, (uint64_t)(p->track_max - p->track_min) + 1);
    double theta = rng_unit(r) * 3.14159265358979323846;
    double g = rng_unit(r) * p->max_gradient;
    double c = cos(theta), s = sin(theta);
    double mx = fabs(c) > fabs(s) ? fabs(c) : fabs(s);
    double sx = c / mx, sy = s / mx;
    double x0 = (double)rng_below(r, p->width), y0 = (double)rng_below(r, p->height);
    int m = 0;
    for (uint32_t k = 0; k < len; ++k) {
        double fx = floor(x0 + 0.5 + k * sx), fy = floor(y0 + 0.5 + k * sy);
        if (fx < 0 || fy < 0 || fx >= p->width || fy >= p->height) break;
        hg_hit e;
        e.x = (uint16_t)fx; e.y = (uint16_t)fy;
        e.tot = draw_tot(r, p); e.reserved = 0;
        e.toa = t_ev + (uint64_t)floor(k * g) + rng_below(r, (uint64_t)p->toa_jitter + 1);
        if (hv_push(out, e)) return -1;
        m++;
    }
    return m;
}

/*
 * Generate exactly p->n hits into out[0..n).  Returns 0 on success.
 * *max_disorder (if non-null) receives the smallest t >= 1 for which the
 * emitted sequence is t-ordered: toa[i] < toa[j] + t for all i < j.
 */
int hitgen_generate(const hg_params *p, hg_hit *out, uint64_t *max_disorder) {
    if (!p || (!out && p->n) || p->width == 0 || p->height == 0 ||
        p->width > 65536 || p->height > 65536) return -2;
    hg_rng r = { p->seed * 0x2545F4914F6CDD1Dull + 0x1234567ull };
    hitvec v = {0, 0, 0};
    uint64_t target = p->n + p->n / 50 + 64;
    double t = (double)p->t0;
    while (v.n < target) {
        int got;
        uint64_t t_ev = (uint64_t)t;
        if (rng_unit(&r) < p->track_frac) got = emit_track(&r, p, t_ev, &v);
        else got = emit_blob(&r, p, t_ev, &v);
        if (got < 0) { free(v.v); return -1; }
        if (p->event_rate > 0) t += rng_exp(&r, 1.0 / p->event_rate);
        else t += rng_exp(&r, 1.0) * (double)(got > 0 ? got : 1) / p->hit_rate;
    }
    if (sort_hits_by_toa(v.v, v.n)) { free(v.v); return -1; }
    if (p->dead_time) {
        /* per pixel in time order: a hit arriving while the pixel is still
           busy with the previous hit's ToT fires when the pixel frees up */
        uint64_t npx = (uint64_t)p->width * p->height;
        uint64_t *busy = (uint64_t *)calloc(npx, sizeof(uint64_t));
        if (!busy) { free(v.v); return -1; }
        for (uint64_t i = 0; i < v.n; ++i) {
            uint64_t q = (uint64_t)v.v[i].y * p->width + v.v[i].x;
            if (v.v[i].toa < busy[q]) v.v[i].toa = busy[q];
            busy[q] = v.v[i].toa + v.v[i].tot;
        }
        free(busy);
        if (sort_hits_by_toa(v.v, v.n)) { free(v.v); return -1; }
    }
    uint64_t n = p->n;
    if (p->shuffle_window > 1 && n > 1) {
        uint64_t *k = (uint64_t *)malloc(n * sizeof(uint64_t));
        uint32_t *pm = (uint32_t *)malloc(n * sizeof(uint32_t));
        if (!k || !pm) { free(k); free(pm); free(v.v); return -1; }
        for (uint64_t i = 0; i < n; ++i) { k[i] = i + rng_below(&r, p->shuffle_window); pm[i] = (uint32_t)i; }
        int rc = sort_by_key(k, pm, n);
        if (!rc) for (uint64_t i = 0; i < n; ++i) out[i] = v.v[pm[i]];
        free(k); free(pm);
        if (rc) { free(v.v); return -1; }
    } else if (n) {
        memcpy(out, v.v, n * sizeof(hg_hit));
    }
    free(v.v);
    if (max_disorder) {
        uint64_t run = 0, t_min = 1;   /* run = max ToA among earlier hits */
        for (uint64_t i = 0; i < n; ++i) {
            if (i > 0 && run > out[i].toa && run - out[i].toa + 1 > t_min) t_min = run - out[i].toa + 1;
            if (i == 0 || out[i].toa > run) run = out[i].toa;
        }
        *max_disorder = t_min;
    }
    return 0;
}

uint32_t hitgen_record_size(void) { return (uint32_t)sizeof(hg_hit); }
uint32_t hitgen_params_size(void) { return (uint32_t)sizeof(hg_params); }
