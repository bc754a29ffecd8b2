/*
 * Temporal-split parallel CPU clustering — a COMPARISON BASELINE.
 *
 * Not the oracle, and not part of the product: the CUDA library never calls
 * it.  It is the paper's multi-core CPU method for variant (iii)(a), timed by
 * the benchmark beside the GPU path, and tested against the oracle.
 *
 * Method (paper, Section 3.2 "Temporal splitting" and Section 3.3 "Merging
 * split clusters"):
 *   1. The hits are split by ToA into windows of `window` ticks; workers take
 *      contiguous runs of windows holding about the same number of hits.
 *   2. Each window is ordered by ToA and clustered by the data-driven sweep
 *      (Algorithm 1 with the union-find of Section 4.1): a matrix keeps the
 *      last hit seen on every pixel, and a hit is joined to the last hit of
 *      each of its 9 pixels (8 neighbours and its own) that is at most dt
 *      earlier.  That last hit suffices: any earlier hit of that pixel within
 *      dt is within dt of the last one, so already in its cluster.
 *   3. Only hits within dt of a window border can link across it, and only
 *      to hits of the adjacent window (window > dt), so for each border the
 *      clusters with a hit in the dt slab on either side are compared by the
 *      three-stage cascade: (1) temporal distance of the two clusters
 *      greater than dt: no merge; (2) bounding boxes, grown by one pixel, do
 *      not intersect: no merge; (3) full check: the larger cluster's slab
 *      hits inside the boxes' intersection go into a 2-D pixel array, and
 *      each slab hit of the smaller cluster looks for a hit within dt on its
 *      9 pixels.
 *   4. The merges are applied with a union-find over all clusters; a cluster's
 *      label is the smallest arrival index of its merged set, and the
 *      features (size, ToT sum, first ToA, ToT-weighted centroid in fp64 from
 *      exact integer sums) are summed over it.
 * Output matches the oracle exactly: labels are the smallest input index of
 * each cluster; records are ordered by label.
 *
 * Differences from the paper's pipeline, which streams: the whole input is
 * present, so windows are formed by a stable counting sort on the window
 * number (instead of a priority queue over a t-ordered stream), the per-pixel
 * matrix is invalidated by a per-window stamp (instead of clearing the
 * touched pixels), and each border is merged once by whichever worker takes
 * it (instead of one merging worker per border time in round robin).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint16_t x, y, tot, reserved;
    uint64_t toa;
} ts_hit;

typedef struct {
    uint64_t label;
    int64_t size;
    int64_t sum_tot;
    uint64_t first_toa;
    double cx, cy;
} ts_cluster;

enum { TS_OK = 0, TS_ERR_ARG = -1, TS_ERR_RANGE = -2, TS_ERR_NOMEM = -3 };
enum { TS_MAX_THREADS = 256 };

/* per-cluster summary, one per cluster found in a window */
typedef struct {
    uint64_t start, end;       /* first and last ToA */
    uint64_t sum_tot, swx, swy;
    uint32_t min_idx;          /* smallest arrival index */
    uint32_t size;
    uint16_t x0, x1, y0, y1;   /* bounding box */
} ts_stat;

typedef struct {
    uint64_t toa;
    uint32_t pos;              /* position in the window before ordering */
    uint32_t pad;
} ts_key;

/* ------------------------------------------------------------------------ */

typedef struct ts_job ts_job;

typedef struct {
    ts_job *job;
    int id;
    /* windows [w0, w1) */
    uint64_t w0, w1;
    /* clusters found by this worker */
    ts_stat *stat;
    uint64_t n_stat, cap_stat;
    /* merges found by this worker: pairs of global cluster ids */
    uint64_t *pairs;
    uint64_t n_pairs, cap_pairs;
    uint64_t cascade[4];       /* examined, cut by time, cut by box, merged */
    int err;
} ts_worker;

struct ts_job {
    const ts_hit *h;
    uint64_t n;
    uint32_t W, H;
    uint64_t dt, window, toa0;
    uint64_t nwin;
    int threads;
    /* window grouping */
    uint64_t *win_start;       /* nwin + 1 */
    uint32_t *hist;            /* threads * nwin */
    uint64_t *chunk0;          /* threads + 1: arrival chunks */
    /* hits grouped by window, each window in ToA order after clustering */
    ts_hit *g;
    uint32_t *gidx;            /* arrival index of each grouped hit */
    uint32_t *gcl;             /* worker-local cluster number */
    ts_worker *wk;
    uint64_t *cl_base;         /* threads + 1: first global cluster id of a worker */
    uint64_t *uf;              /* union-find over global cluster ids */
    uint64_t *label;
    uint32_t *root_of_hit;     /* by arrival index: the root cluster */
    uint64_t *heads;           /* threads + 1: records before each label range */
    ts_cluster *rec;
};

static int worker_of_window(const ts_job *j, uint64_t w) {
    int lo = 0, hi = j->threads - 1;
    while (lo < hi) {              /* last worker with w0 <= w */
        int mid = (lo + hi + 1) / 2;
        if (j->wk[mid].w0 <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

static int grow(void **p, uint64_t *cap, uint64_t need, size_t elem) {
    if (need <= *cap) return 0;
    uint64_t c = *cap ? *cap : 1024;
    while (c < need) c *= 2;
    void *q = realloc(*p, c * elem);
    if (!q) return -1;
    *p = q;
    *cap = c;
    return 0;
}

/* ordering of a window: ToA, ties in arrival order.  The hits of a window
   arrive in arrival order and their ToA offsets from the window start are
   below the window width, so a stable LSD radix sort by bytes of the offset
   orders them; `passes` bytes cover the width. */
static void sort_window(ts_key *a, ts_key *tmp, uint64_t n, int passes) {
    uint32_t cnt[256];
    for (int p = 0; p < passes; ++p) {
        const int sh = 8 * p;
        memset(cnt, 0, sizeof(cnt));
        for (uint64_t i = 0; i < n; ++i) cnt[(a[i].toa >> sh) & 255]++;
        uint32_t run = 0;
        for (int d = 0; d < 256; ++d) { uint32_t c = cnt[d]; cnt[d] = run; run += c; }
        for (uint64_t i = 0; i < n; ++i) tmp[cnt[(a[i].toa >> sh) & 255]++] = a[i];
        memcpy(a, tmp, n * sizeof(ts_key));
    }
}

static uint32_t uf_find32(uint32_t *p, uint32_t a) {
    while (p[a] != a) { p[a] = p[p[a]]; a = p[a]; }
    return a;
}

/* ------------------------------------------------------------------------ */
/* phase 0: arrival chunks -> per-window histograms                         */

static void *phase_hist(void *arg) {
    ts_worker *w = (ts_worker *)arg;
    ts_job *j = w->job;
    uint32_t *hist = j->hist + (uint64_t)w->id * j->nwin;
    for (uint64_t i = j->chunk0[w->id]; i < j->chunk0[w->id + 1]; ++i)
        hist[(j->h[i].toa - j->toa0) / j->window]++;
    return NULL;
}

static void *phase_scatter(void *arg) {
    ts_worker *w = (ts_worker *)arg;
    ts_job *j = w->job;
    uint32_t *off = j->hist + (uint64_t)w->id * j->nwin;   /* now running offsets */
    for (uint64_t i = j->chunk0[w->id]; i < j->chunk0[w->id + 1]; ++i) {
        uint64_t win = (j->h[i].toa - j->toa0) / j->window;
        uint64_t dst = j->win_start[win] + off[win]++;
        j->g[dst] = j->h[i];
        j->gidx[dst] = (uint32_t)i;
    }
    return NULL;
}

/* ------------------------------------------------------------------------ */
/* phase A: order and cluster each window                                   */

static void *phase_windows(void *arg) {
    ts_worker *w = (ts_worker *)arg;
    ts_job *j = w->job;
    const uint32_t W = j->W, H = j->H;
    uint64_t maxw = 0;
    for (uint64_t k = w->w0; k < w->w1; ++k) {
        uint64_t c = j->win_start[k + 1] - j->win_start[k];
        if (c > maxw) maxw = c;
    }
    uint32_t *stamp = (uint32_t *)calloc((size_t)W * H, sizeof(uint32_t));
    uint32_t *last = (uint32_t *)malloc((size_t)W * H * sizeof(uint32_t));
    ts_key *key = (ts_key *)malloc((maxw ? maxw : 1) * sizeof(ts_key));
    ts_key *key2 = (ts_key *)malloc((maxw ? maxw : 1) * sizeof(ts_key));
    uint64_t *last_toa = (uint64_t *)malloc((size_t)W * H * sizeof(uint64_t));
    uint32_t *par = (uint32_t *)malloc((maxw ? maxw : 1) * sizeof(uint32_t));
    uint32_t *ord = (uint32_t *)malloc((maxw ? maxw : 1) * sizeof(uint32_t));
    ts_hit *tmp_h = (ts_hit *)malloc((maxw ? maxw : 1) * sizeof(ts_hit));
    uint32_t *tmp_i = (uint32_t *)malloc((maxw ? maxw : 1) * sizeof(uint32_t));
    int passes = 0;
    for (uint64_t span = j->window - 1; span; span >>= 8) ++passes;
    if (!stamp || !last || !key || !key2 || !last_toa || !par || !ord || !tmp_h || !tmp_i) {
        w->err = TS_ERR_NOMEM;
        goto done;
    }
    uint32_t epoch = 0;
    for (uint64_t k = w->w0; k < w->w1; ++k) {
        const uint64_t s0 = j->win_start[k], m = j->win_start[k + 1] - s0;
        if (!m) continue;
        ts_hit *g = j->g + s0;
        uint32_t *gi = j->gidx + s0;
        /* ToA order (ties: arrival order, kept by the grouping) */
        const uint64_t w_start = j->toa0 + k * j->window;
        for (uint64_t i = 0; i < m; ++i) { key[i].toa = g[i].toa - w_start; key[i].pos = (uint32_t)i; }
        sort_window(key, key2, m, passes);
        for (uint64_t i = 0; i < m; ++i) { tmp_h[i] = g[key[i].pos]; tmp_i[i] = gi[key[i].pos]; }
        memcpy(g, tmp_h, m * sizeof(ts_hit));
        memcpy(gi, tmp_i, m * sizeof(uint32_t));
        /* the data-driven sweep with the last-hit matrix */
        if (++epoch == 0) {   /* stamp wrapped: clear it */
            memset(stamp, 0, (size_t)W * H * sizeof(uint32_t));
            epoch = 1;
        }
        for (uint64_t i = 0; i < m; ++i) {
            par[i] = (uint32_t)i;
            const int x = g[i].x, y = g[i].y;
            const uint64_t t = g[i].toa;
            for (int dy = -1; dy <= 1; ++dy) {
                const int py = y + dy;
                if (py < 0 || py >= (int)H) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int px = x + dx;
                    if (px < 0 || px >= (int)W) continue;
                    const uint64_t q = (uint64_t)py * W + px;
                    if (stamp[q] != epoch || t - last_toa[q] > j->dt) continue;
                    const uint32_t o = last[q];
                    /* union: the earlier position becomes the root */
                    uint32_t ra = uf_find32(par, o), rb = uf_find32(par, (uint32_t)i);
                    if (ra == rb) continue;
                    if (ra < rb) par[rb] = ra; else par[ra] = rb;
                }
            }
            const uint64_t p = (uint64_t)y * W + x;
            stamp[p] = epoch;
            last[p] = (uint32_t)i;
            last_toa[p] = t;
        }
        /* clusters: the root is the earliest position of its cluster */
        for (uint64_t i = 0; i < m; ++i) {
            const uint32_t r = uf_find32(par, (uint32_t)i);
            ts_stat *s;
            if (r == i) {
                if (grow((void **)&w->stat, &w->cap_stat, w->n_stat + 1, sizeof(ts_stat))) {
                    w->err = TS_ERR_NOMEM;
                    goto done;
                }
                ord[i] = (uint32_t)w->n_stat;
                s = &w->stat[w->n_stat++];
                s->start = s->end = g[i].toa;
                s->sum_tot = s->swx = s->swy = 0;
                s->min_idx = gi[i];
                s->size = 0;
                s->x0 = s->x1 = g[i].x;
                s->y0 = s->y1 = g[i].y;
            } else {
                ord[i] = ord[r];
                s = &w->stat[ord[i]];
            }
            const ts_hit *e = &g[i];
            if (e->toa > s->end) s->end = e->toa;
            if (gi[i] < s->min_idx) s->min_idx = gi[i];
            s->size++;
            s->sum_tot += e->tot;
            s->swx += (uint64_t)e->tot * e->x;
            s->swy += (uint64_t)e->tot * e->y;
            if (e->x < s->x0) s->x0 = e->x;
            if (e->x > s->x1) s->x1 = e->x;
            if (e->y < s->y0) s->y0 = e->y;
            if (e->y > s->y1) s->y1 = e->y;
            j->gcl[s0 + i] = ord[i];
        }
    }
done:
    free(stamp); free(last); free(last_toa); free(key); free(key2); free(par); free(ord); free(tmp_h);
    free(tmp_i);
    return NULL;
}

/* ------------------------------------------------------------------------ */
/* phase B: the merge cascade at each window border                         */

typedef struct {
    uint64_t id;               /* global cluster id */
    uint64_t first, count;     /* its slab hits: positions in a per-border list */
} ts_side;

static uint64_t global_id(const ts_job *j, uint64_t pos, int worker) {
    return j->cl_base[worker] + j->gcl[pos];
}

static const ts_stat *stat_of(const ts_job *j, uint64_t gid, int worker) {
    return &j->wk[worker].stat[gid - j->cl_base[worker]];
}

/* group slab positions [a, b) by cluster: side[] lists each distinct cluster
   with its hits, which are written consecutively into list[] */
static int slab_clusters(const ts_job *j, uint64_t a, uint64_t b, int worker, ts_side **side,
                         uint64_t *n_side, uint64_t *cap_side, uint64_t **list, uint64_t *cap_list) {
    *n_side = 0;
    if (grow((void **)list, cap_list, b - a, sizeof(uint64_t))) return -1;
    /* small slabs: a quadratic grouping keeps it simple */
    for (uint64_t p = a; p < b; ++p) {
        const uint64_t id = global_id(j, p, worker);
        uint64_t s = 0;
        while (s < *n_side && (*side)[s].id != id) ++s;
        if (s == *n_side) {
            if (grow((void **)side, cap_side, *n_side + 1, sizeof(ts_side))) return -1;
            (*side)[s].id = id;
            (*side)[s].first = 0;
            (*side)[s].count = 0;
            (*n_side)++;
        }
        (*side)[s].count++;
    }
    uint64_t off = 0;
    for (uint64_t s = 0; s < *n_side; ++s) { (*side)[s].first = off; off += (*side)[s].count; (*side)[s].count = 0; }
    for (uint64_t p = a; p < b; ++p) {
        const uint64_t id = global_id(j, p, worker);
        uint64_t s = 0;
        while ((*side)[s].id != id) ++s;
        (*list)[(*side)[s].first + (*side)[s].count++] = p;
    }
    return 0;
}

static void *phase_borders(void *arg) {
    ts_worker *w = (ts_worker *)arg;
    ts_job *j = w->job;
    const uint32_t W = j->W;
    const uint64_t dt = j->dt;
    uint32_t *stamp = (uint32_t *)calloc((size_t)W * j->H, sizeof(uint32_t));
    uint32_t *head = (uint32_t *)malloc((size_t)W * j->H * sizeof(uint32_t));
    uint32_t *next = NULL;
    uint64_t cap_next = 0;
    ts_side *ls = NULL, *rs = NULL;
    uint64_t nls = 0, nrs = 0, cap_ls = 0, cap_rs = 0, cap_ll = 0, cap_rl = 0;
    uint64_t *ll = NULL, *rl = NULL;
    uint32_t epoch = 0;
    if (!stamp || !head) { w->err = TS_ERR_NOMEM; goto done; }
    /* this worker merges the borders after each of its windows */
    for (uint64_t k = w->w0; k < w->w1 && k + 1 < j->nwin; ++k) {
        const uint64_t a0 = j->win_start[k], a1 = j->win_start[k + 1], b1 = j->win_start[k + 2];
        if (a0 == a1 || a1 == b1) continue;
        const uint64_t border = j->toa0 + (k + 1) * j->window;
        /* left slab: border - ToA <= dt (a suffix of window k, ToA ordered;
           its ToAs are below the border) */
        uint64_t ls0 = a1;
        while (ls0 > a0 && border - j->g[ls0 - 1].toa <= dt) --ls0;
        /* right slab: ToA - border < dt, i.e. within dt of some ToA before the
           border (a prefix of window k + 1, ToAs at or after the border);
           written as differences, so ToAs near 2^64 do not wrap */
        uint64_t rs1 = a1;
        while (rs1 < b1 && j->g[rs1].toa - border < dt) ++rs1;
        if (ls0 == a1 || rs1 == a1) continue;
        const int wl = worker_of_window(j, k), wr = worker_of_window(j, k + 1);
        if (slab_clusters(j, ls0, a1, wl, &ls, &nls, &cap_ls, &ll, &cap_ll) ||
            slab_clusters(j, a1, rs1, wr, &rs, &nrs, &cap_rs, &rl, &cap_rl)) {
            w->err = TS_ERR_NOMEM;
            goto done;
        }
        for (uint64_t u = 0; u < nls; ++u) {
            const ts_stat *c1 = stat_of(j, ls[u].id, wl);
            for (uint64_t v = 0; v < nrs; ++v) {
                const ts_stat *c2 = stat_of(j, rs[v].id, wr);
                w->cascade[0]++;
                /* (1) temporal distance of the two clusters */
                uint64_t tdist = 0;
                if (c2->start > c1->end) tdist = c2->start - c1->end;
                if (c1->start > c2->end && c1->start - c2->end > tdist) tdist = c1->start - c2->end;
                if (tdist > dt) { w->cascade[1]++; continue; }
                /* (2) bounding boxes: one grown by a pixel must meet the other;
                   every linking pair of hits lies in [ix0, ix1] x [iy0, iy1] */
                const int mx0 = c1->x0 > c2->x0 ? c1->x0 : c2->x0, mx1 = c1->x1 < c2->x1 ? c1->x1 : c2->x1;
                const int my0 = c1->y0 > c2->y0 ? c1->y0 : c2->y0, my1 = c1->y1 < c2->y1 ? c1->y1 : c2->y1;
                if (mx0 > mx1 + 1 || my0 > my1 + 1) { w->cascade[2]++; continue; }
                const int ix0 = mx0 - 1, ix1 = mx1 + 1, iy0 = my0 - 1, iy1 = my1 + 1;
                /* (3) full check on the slab hits: the larger side into the
                   pixel array, the smaller side looks up its 9 pixels */
                const ts_side *big = ls[u].count >= rs[v].count ? &ls[u] : &rs[v];
                const ts_side *small = big == &ls[u] ? &rs[v] : &ls[u];
                const uint64_t *bl = big == &ls[u] ? ll : rl, *sl = big == &ls[u] ? rl : ll;
                if (grow((void **)&next, &cap_next, big->count, sizeof(uint32_t))) {
                    w->err = TS_ERR_NOMEM;
                    goto done;
                }
                if (++epoch == 0) {
                    memset(stamp, 0, (size_t)W * j->H * sizeof(uint32_t));
                    epoch = 1;
                }
                for (uint64_t q = 0; q < big->count; ++q) {
                    const ts_hit *e = &j->g[bl[big->first + q]];
                    if (e->x < ix0 || e->x > ix1 || e->y < iy0 || e->y > iy1) continue;
                    const uint64_t p = (uint64_t)e->y * W + e->x;
                    next[q] = stamp[p] == epoch ? head[p] : UINT32_MAX;
                    head[p] = (uint32_t)q;
                    stamp[p] = epoch;
                }
                int linked = 0;
                for (uint64_t q = 0; q < small->count && !linked; ++q) {
                    const ts_hit *e = &j->g[sl[small->first + q]];
                    if (e->x < ix0 || e->x > ix1 || e->y < iy0 || e->y > iy1) continue;
                    for (int dy = -1; dy <= 1 && !linked; ++dy) {
                        const int py = e->y + dy;
                        if (py < 0 || py >= (int)j->H) continue;
                        for (int dx = -1; dx <= 1 && !linked; ++dx) {
                            const int px = e->x + dx;
                            if (px < 0 || px >= (int)W) continue;
                            const uint64_t p = (uint64_t)py * W + px;
                            if (stamp[p] != epoch) continue;
                            for (uint32_t r = head[p]; r != UINT32_MAX; r = next[r]) {
                                const uint64_t t2 = j->g[bl[big->first + r]].toa;
                                const uint64_t d = t2 > e->toa ? t2 - e->toa : e->toa - t2;
                                if (d <= dt) { linked = 1; break; }
                            }
                        }
                    }
                }
                if (!linked) continue;
                w->cascade[3]++;
                if (grow((void **)&w->pairs, &w->cap_pairs, 2 * (w->n_pairs + 1), sizeof(uint64_t))) {
                    w->err = TS_ERR_NOMEM;
                    goto done;
                }
                w->pairs[2 * w->n_pairs] = ls[u].id;
                w->pairs[2 * w->n_pairs + 1] = rs[v].id;
                w->n_pairs++;
            }
        }
    }
done:
    free(stamp); free(head); free(next); free(ls); free(rs); free(ll); free(rl);
    return NULL;
}

/* ------------------------------------------------------------------------ */
/* phases D and E: labels per hit, records in label order                   */

static uint64_t uf_find64(uint64_t *p, uint64_t a) {
    while (p[a] != a) a = p[a];
    return a;
}

static void *phase_labels(void *arg) {
    ts_worker *w = (ts_worker *)arg;
    ts_job *j = w->job;
    for (uint64_t k = w->w0; k < w->w1; ++k) {
        for (uint64_t p = j->win_start[k]; p < j->win_start[k + 1]; ++p) {
            /* every entry of uf is a root after the merge step */
            j->root_of_hit[j->gidx[p]] = (uint32_t)j->uf[global_id(j, p, w->id)];
        }
    }
    return NULL;
}

static int worker_of_cluster(const ts_job *j, uint64_t gid) {
    int lo = 0, hi = j->threads - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) / 2;
        if (j->cl_base[mid] <= gid) lo = mid; else hi = mid - 1;
    }
    return lo;
}

static const ts_stat *stat_global(const ts_job *j, uint64_t gid) {
    const int w = worker_of_cluster(j, gid);
    return &j->wk[w].stat[gid - j->cl_base[w]];
}

static void *phase_heads(void *arg) {
    ts_worker *w = (ts_worker *)arg;
    ts_job *j = w->job;
    uint64_t c = 0;
    for (uint64_t i = j->chunk0[w->id]; i < j->chunk0[w->id + 1]; ++i) {
        const ts_stat *s = stat_global(j, j->root_of_hit[i]);
        j->label[i] = s->min_idx;
        c += s->min_idx == i;
    }
    j->heads[w->id + 1] = c;
    return NULL;
}

static void *phase_records(void *arg) {
    ts_worker *w = (ts_worker *)arg;
    ts_job *j = w->job;
    uint64_t o = j->heads[w->id];
    for (uint64_t i = j->chunk0[w->id]; i < j->chunk0[w->id + 1]; ++i) {
        if (j->label[i] != i) continue;
        const ts_stat *s = stat_global(j, j->root_of_hit[i]);
        ts_cluster *r = &j->rec[o++];
        r->label = i;
        r->size = s->size;
        r->sum_tot = (int64_t)s->sum_tot;
        r->first_toa = s->start;
        r->cx = (double)s->swx / (double)s->sum_tot;
        r->cy = (double)s->swy / (double)s->sum_tot;
    }
    return NULL;
}

static int run_phase(ts_job *j, void *(*fn)(void *)) {
    pthread_t tid[TS_MAX_THREADS];
    int started = 0;
    for (int t = 1; t < j->threads; ++t) {
        if (pthread_create(&tid[t], NULL, fn, &j->wk[t]) != 0) break;
        started = t;
    }
    fn(&j->wk[0]);
    for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
    if (started != j->threads - 1) {
        /* could not start every thread: run the rest here */
        for (int t = started + 1; t < j->threads; ++t) fn(&j->wk[t]);
    }
    for (int t = 0; t < j->threads; ++t)
        if (j->wk[t].err) return j->wk[t].err;
    return TS_OK;
}

/* ------------------------------------------------------------------------ */

int tsplit_cluster(const ts_hit *h, uint64_t n, uint32_t W, uint32_t H, uint64_t dt,
                   uint64_t window, int threads, uint64_t *label, ts_cluster *rec,
                   uint64_t *n_clusters, uint64_t *cascade) {
    if ((n && (!h || !label || !rec)) || !n_clusters || W == 0 || H == 0 || n >= UINT32_MAX ||
        window <= dt || threads < 1)
        return TS_ERR_ARG;
    if (threads > TS_MAX_THREADS) threads = TS_MAX_THREADS;
    if (cascade) memset(cascade, 0, 4 * sizeof(uint64_t));
    *n_clusters = 0;
    if (!n) return TS_OK;
    uint64_t tmin = UINT64_MAX, tmax = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (h[i].x >= W || h[i].y >= H) return TS_ERR_RANGE;
        if (h[i].toa < tmin) tmin = h[i].toa;
        if (h[i].toa > tmax) tmax = h[i].toa;
    }
    if ((uint64_t)threads > n) threads = (int)n;
    ts_job J;
    memset(&J, 0, sizeof(J));
    ts_job *j = &J;
    j->h = h; j->n = n; j->W = W; j->H = H; j->dt = dt; j->toa0 = tmin; j->threads = threads;
    /* at most n / (2 threads) + 1 windows, so that the per-worker window
       histograms hold at most 2n counters: a sparse stream gets wider windows */
    uint64_t win = window;
    const uint64_t max_windows = n / (2 * (uint64_t)threads) + 1;
    if ((tmax - tmin) / win + 1 > max_windows) win = (tmax - tmin) / max_windows + 1;
    if (win <= dt) win = dt + 1;
    j->window = win;
    j->nwin = (tmax - tmin) / win + 1;
    int rc = TS_ERR_NOMEM;
    j->win_start = (uint64_t *)calloc(j->nwin + 2, sizeof(uint64_t));
    j->hist = (uint32_t *)calloc((size_t)threads * j->nwin, sizeof(uint32_t));
    j->chunk0 = (uint64_t *)malloc((threads + 1) * sizeof(uint64_t));
    j->g = (ts_hit *)malloc(n * sizeof(ts_hit));
    j->gidx = (uint32_t *)malloc(n * sizeof(uint32_t));
    j->gcl = (uint32_t *)malloc(n * sizeof(uint32_t));
    j->wk = (ts_worker *)calloc(threads, sizeof(ts_worker));
    j->cl_base = (uint64_t *)calloc(threads + 1, sizeof(uint64_t));
    j->root_of_hit = (uint32_t *)malloc(n * sizeof(uint32_t));
    j->heads = (uint64_t *)calloc(threads + 1, sizeof(uint64_t));
    if (!j->win_start || !j->hist || !j->chunk0 || !j->g || !j->gidx || !j->gcl || !j->wk ||
        !j->cl_base || !j->root_of_hit || !j->heads)
        goto out;
    for (int t = 0; t <= threads; ++t) j->chunk0[t] = n * (uint64_t)t / threads;
    for (int t = 0; t < threads; ++t) { j->wk[t].job = j; j->wk[t].id = t; }
    /* 1. group by window (stable counting sort) */
    if ((rc = run_phase(j, phase_hist))) goto out;
    {
        uint64_t run = 0;
        for (uint64_t k = 0; k < j->nwin; ++k) {
            j->win_start[k] = run;
            for (int t = 0; t < threads; ++t) {
                uint32_t c = j->hist[(uint64_t)t * j->nwin + k];
                j->hist[(uint64_t)t * j->nwin + k] = (uint32_t)(run - j->win_start[k]);
                run += c;
            }
        }
        j->win_start[j->nwin] = run;
        j->win_start[j->nwin + 1] = run;
    }
    if ((rc = run_phase(j, phase_scatter))) goto out;
    /* workers take runs of windows holding about n / threads hits */
    {
        uint64_t k = 0;
        for (int t = 0; t < threads; ++t) {
            j->wk[t].w0 = k;
            const uint64_t target = n * (uint64_t)(t + 1) / threads;
            while (k < j->nwin && (t == threads - 1 || j->win_start[k + 1] <= target)) ++k;
            if (k == j->wk[t].w0 && k < j->nwin && t < threads - 1) ++k;
            j->wk[t].w1 = k;
        }
        j->wk[threads - 1].w1 = j->nwin;
    }
    /* 2. cluster each window */
    if ((rc = run_phase(j, phase_windows))) goto out;
    for (int t = 0; t < threads; ++t) j->cl_base[t + 1] = j->cl_base[t] + j->wk[t].n_stat;
    const uint64_t ncl = j->cl_base[threads];
    /* 3. merge cascade at every border */
    if ((rc = run_phase(j, phase_borders))) goto out;
    /* 4. union-find over clusters; merged sets summed into their root */
    j->uf = (uint64_t *)malloc(ncl * sizeof(uint64_t));
    if (!j->uf) { rc = TS_ERR_NOMEM; goto out; }
    for (uint64_t c = 0; c < ncl; ++c) j->uf[c] = c;
    for (int t = 0; t < threads; ++t) {
        for (uint64_t q = 0; q < j->wk[t].n_pairs; ++q) {
            uint64_t a = uf_find64(j->uf, j->wk[t].pairs[2 * q]);
            uint64_t b = uf_find64(j->uf, j->wk[t].pairs[2 * q + 1]);
            if (a == b) continue;
            if (a < b) j->uf[b] = a; else j->uf[a] = b;
        }
        if (cascade)
            for (int s = 0; s < 4; ++s) cascade[s] += j->wk[t].cascade[s];
    }
    for (int t = 0; t < threads; ++t) {
        for (uint64_t q = 0; q < 2 * j->wk[t].n_pairs; ++q) {
            const uint64_t c = j->wk[t].pairs[q];
            const uint64_t r = uf_find64(j->uf, c);
            if (r == c) continue;
            /* add cluster c into root r once: c then points at r directly and
               is marked done by its stat's size becoming 0 */
            const int wc = worker_of_cluster(j, c), wr = worker_of_cluster(j, r);
            ts_stat *sc = &j->wk[wc].stat[c - j->cl_base[wc]];
            ts_stat *sr = &j->wk[wr].stat[r - j->cl_base[wr]];
            if (sc->size) {
                if (sc->start < sr->start) sr->start = sc->start;
                if (sc->end > sr->end) sr->end = sc->end;
                if (sc->min_idx < sr->min_idx) sr->min_idx = sc->min_idx;
                sr->size += sc->size;
                sr->sum_tot += sc->sum_tot;
                sr->swx += sc->swx;
                sr->swy += sc->swy;
                sc->size = 0;
            }
            j->uf[c] = r;
        }
    }
    /* 5. labels and records */
    if ((rc = run_phase(j, phase_labels))) goto out;
    j->label = label;
    if ((rc = run_phase(j, phase_heads))) goto out;
    for (int t = 0; t < threads; ++t) j->heads[t + 1] += j->heads[t];
    j->rec = rec;
    if ((rc = run_phase(j, phase_records))) goto out;
    *n_clusters = j->heads[threads];
    rc = TS_OK;
out:
    if (j->wk)
        for (int t = 0; t < threads; ++t) { free(j->wk[t].stat); free(j->wk[t].pairs); }
    free(j->win_start); free(j->hist); free(j->chunk0); free(j->g); free(j->gidx); free(j->gcl);
    free(j->wk); free(j->cl_base); free(j->uf); free(j->root_of_hit); free(j->heads);
    return rc;
}

uint32_t tsplit_hit_size(void) { return (uint32_t)sizeof(ts_hit); }
uint32_t tsplit_cluster_size(void) { return (uint32_t)sizeof(ts_cluster); }
