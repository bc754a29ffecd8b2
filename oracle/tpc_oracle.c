/*
 * CPU oracle for Timepix hit clustering — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code, header, table or helper with the CUDA
 * library; the two meet only in the 16-byte hit record drawn by the input
 * generator.  Plain, sequential and slow on purpose: each function states the
 * definition it follows and takes its steps in that order.
 *
 * Definitions (paper, Section 2, conditions (i)-(iii)):
 *   A cluster is a maximal (i) set of hits that is spatially 8-connected (ii)
 *   and satisfies one of three temporal conditions (iii):
 *   (a) dynamic local-time neighbourhood: consecutive hits on a connecting
 *       path are at most dt apart in ToA;
 *   (b) dynamic global-time neighbourhood: every hit but the first has another
 *       cluster hit at most dt earlier;
 *   (c) static time neighbourhood: all pairwise ToA differences are <= dt.
 *   The GPU step that looks for neighbours visits "the 8 neighbouring pixels
 *   plus the pixel itself" (Section 4.1), so a pixel is its own neighbour.
 *
 * Readings taken where the text leaves room (each is also stated in the
 * design notes):
 *   - (a) is read as "there exists a path" whose every step is 8-adjacent
 *     (Chebyshev distance <= 1) with |dToA| <= dt, i.e. connected components
 *     of that graph.  Comparisons are inclusive.
 *   - (b) and (c) define properties, not a unique partition; they are read
 *     as the time sweep of Algorithm 1 (Section 2.2) in (toa, index) order:
 *     a hit joins, and merges, every cluster that has a member on one of its
 *     9 pixels and is still open; (b) open = last ToA >= toa(h) - dt,
 *     (c) open = first ToA >= toa(h) - dt; otherwise the hit starts a new
 *     cluster.
 *   - Labels are canonical: the smallest input index in each cluster.
 *   - Features: size, sum ToT (exact integers), first ToA (min ToA), and the
 *     ToT-weighted centroid sum(tot*x)/sum(tot) of integer pixel coordinates,
 *     evaluated in fp64 from exact integer sums (0/0 gives NaN).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint16_t x, y, tot, reserved;
    uint64_t toa;
} or_hit;

typedef struct {
    uint64_t label;
    int64_t size;
    int64_t sum_tot;
    uint64_t first_toa;
    double cx, cy;
} or_cluster;

enum { OR_OK = 0, OR_ERR_ARG = -1, OR_ERR_RANGE = -2, OR_ERR_NOMEM = -3 };

static const uint64_t NONE = UINT64_MAX;

/* |a - b| <= dt without overflow */
static int within(uint64_t a, uint64_t b, uint64_t dt) {
    return (a >= b ? a - b : b - a) <= dt;
}

static int check_range(const or_hit *h, uint64_t n, uint32_t W, uint32_t H) {
    for (uint64_t i = 0; i < n; ++i)
        if (h[i].x >= W || h[i].y >= H) return OR_ERR_RANGE;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* per-pixel hit lists, each sorted by (toa, index)                         */

typedef struct {
    uint64_t *start;   /* W*H + 1 offsets */
    uint64_t *idx;     /* n hit indices grouped by pixel */
} pixel_lists;

/* qsort has no context argument; one per thread, so that calls from
   several threads (the full-size tests run two at once) do not mix */
static _Thread_local const or_hit *g_sort_hits;

static int cmp_toa_idx(const void *a, const void *b) {
    uint64_t i = *(const uint64_t *)a, j = *(const uint64_t *)b;
    uint64_t ti = g_sort_hits[i].toa, tj = g_sort_hits[j].toa;
    if (ti != tj) return ti < tj ? -1 : 1;
    return i < j ? -1 : (i > j ? 1 : 0);
}

static int build_pixel_lists(const or_hit *h, uint64_t n, uint32_t W, uint32_t H,
                             pixel_lists *pl) {
    uint64_t npx = (uint64_t)W * H;
    pl->start = (uint64_t *)calloc(npx + 1, sizeof(uint64_t));
    pl->idx = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!pl->start || !pl->idx) return OR_ERR_NOMEM;
    for (uint64_t i = 0; i < n; ++i) pl->start[(uint64_t)h[i].y * W + h[i].x + 1]++;
    for (uint64_t p = 0; p < npx; ++p) pl->start[p + 1] += pl->start[p];
    uint64_t *fill = (uint64_t *)malloc((npx ? npx : 1) * sizeof(uint64_t));
    if (!fill) return OR_ERR_NOMEM;
    memcpy(fill, pl->start, npx * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; ++i) pl->idx[fill[(uint64_t)h[i].y * W + h[i].x]++] = i;
    free(fill);
    g_sort_hits = h;
    for (uint64_t p = 0; p < npx; ++p) {
        uint64_t len = pl->start[p + 1] - pl->start[p];
        if (len > 1) qsort(pl->idx + pl->start[p], len, sizeof(uint64_t), cmp_toa_idx);
    }
    return OR_OK;
}

static void free_pixel_lists(pixel_lists *pl) {
    free(pl->start); free(pl->idx);
    pl->start = pl->idx = NULL;
}

/* first position in the (toa-sorted) list [lo, hi) whose toa >= t */
static uint64_t lower_bound_toa(const or_hit *h, const uint64_t *idx, uint64_t lo,
                                uint64_t hi, uint64_t t) {
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (h[idx[mid]].toa < t) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* ------------------------------------------------------------------------ */
/* Variant (a): connected components by breadth-first search.               */
/* label[i] = smallest index in i's component.                              */

int oracle_labels_local(const or_hit *h, uint64_t n, uint32_t W, uint32_t H,
                        uint64_t dt, uint64_t *label) {
    if ((n && (!h || !label)) || W == 0 || H == 0) return OR_ERR_ARG;
    int rc = check_range(h, n, W, H);
    if (rc) return rc;
    pixel_lists pl;
    rc = build_pixel_lists(h, n, W, H, &pl);
    uint64_t *queue = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    if (rc || !queue) { free_pixel_lists(&pl); free(queue); return OR_ERR_NOMEM; }
    for (uint64_t i = 0; i < n; ++i) label[i] = NONE;

    for (uint64_t s = 0; s < n; ++s) {
        if (label[s] != NONE) continue;
        /* every smaller index is already labelled, so s is the component's minimum */
        uint64_t head = 0, tail = 0;
        label[s] = s;
        queue[tail++] = s;
        while (head < tail) {
            uint64_t u = queue[head++];
            uint64_t t = h[u].toa;
            uint64_t t_lo = t >= dt ? t - dt : 0;
            for (int dy = -1; dy <= 1; ++dy) {
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t px = (int64_t)h[u].x + dx, py = (int64_t)h[u].y + dy;
                    if (px < 0 || py < 0 || px >= (int64_t)W || py >= (int64_t)H) continue;
                    uint64_t p = (uint64_t)py * W + (uint64_t)px;
                    uint64_t k = lower_bound_toa(h, pl.idx, pl.start[p], pl.start[p + 1], t_lo);
                    for (; k < pl.start[p + 1]; ++k) {
                        uint64_t v = pl.idx[k];
                        if (!within(h[v].toa, t, dt)) break;   /* list is toa sorted */
                        if (label[v] == NONE) { label[v] = s; queue[tail++] = v; }
                    }
                }
            }
        }
    }
    free(queue);
    free_pixel_lists(&pl);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Variants (b) and (c): time sweep (Algorithm 1) with union-find over       */
/* clusters.  mode 1 = (b) open iff toa(h) - last <= dt,                     */
/*            mode 2 = (c) open iff toa(h) - first <= dt.                    */

typedef struct {
    uint64_t *parent;
    uint64_t *first, *last;   /* valid at roots */
} sweep_uf;

static uint64_t uf_find(sweep_uf *u, uint64_t a) {
    uint64_t r = a;
    while (u->parent[r] != r) r = u->parent[r];
    while (u->parent[a] != r) { uint64_t nx = u->parent[a]; u->parent[a] = r; a = nx; }
    return r;
}

/* per-pixel vector of hit indices whose clusters had a member there */
typedef struct { uint64_t *v; uint32_t n, cap; } pix_vec;

static int pv_push(pix_vec *p, uint64_t e) {
    if (p->n == p->cap) {
        uint32_t nc = p->cap ? p->cap * 2 : 4;
        uint64_t *nv = (uint64_t *)realloc(p->v, nc * sizeof(uint64_t));
        if (!nv) return -1;
        p->v = nv; p->cap = nc;
    }
    p->v[p->n++] = e;
    return 0;
}

static int sweep_labels(const or_hit *h, uint64_t n, uint32_t W, uint32_t H,
                        uint64_t dt, int mode, uint64_t *label) {
    if ((n && (!h || !label)) || W == 0 || H == 0) return OR_ERR_ARG;
    int rc = check_range(h, n, W, H);
    if (rc) return rc;
    uint64_t npx = (uint64_t)W * H;
    uint64_t *order = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    sweep_uf u;
    u.parent = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    u.first = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    u.last = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    pix_vec *pix = (pix_vec *)calloc(npx, sizeof(pix_vec));
    uint64_t *cand = (uint64_t *)malloc(1024 * sizeof(uint64_t));
    uint64_t cand_cap = 1024;
    if (!order || !u.parent || !u.first || !u.last || !pix || !cand) { rc = OR_ERR_NOMEM; goto done; }

    for (uint64_t i = 0; i < n; ++i) order[i] = i;
    g_sort_hits = h;
    qsort(order, n, sizeof(uint64_t), cmp_toa_idx);

    for (uint64_t k = 0; k < n; ++k) {
        uint64_t hi = order[k];
        uint64_t t = h[hi].toa;
        uint64_t nc = 0;
        /* findNeighborClusters: open clusters with a member on one of the 9 pixels */
        for (int dy = -1; dy <= 1; ++dy) {
            for (int dx = -1; dx <= 1; ++dx) {
                int64_t px = (int64_t)h[hi].x + dx, py = (int64_t)h[hi].y + dy;
                if (px < 0 || py < 0 || px >= (int64_t)W || py >= (int64_t)H) continue;
                pix_vec *pv = &pix[(uint64_t)py * W + (uint64_t)px];
                uint32_t keep = 0;
                for (uint32_t e = 0; e < pv->n; ++e) {
                    uint64_t r = uf_find(&u, pv->v[e]);
                    uint64_t ref = mode == 1 ? u.last[r] : u.first[r];
                    /* sweep order gives ref <= t */
                    if (t - ref > dt) continue;          /* closed: can never reopen */
                    pv->v[keep++] = r;
                    int dup = 0;
                    for (uint64_t c = 0; c < nc; ++c) if (cand[c] == r) { dup = 1; break; }
                    if (!dup) {
                        if (nc == cand_cap) {
                            uint64_t *ncand = (uint64_t *)realloc(cand, 2 * cand_cap * sizeof(uint64_t));
                            if (!ncand) { rc = OR_ERR_NOMEM; goto done; }
                            cand = ncand; cand_cap *= 2;
                        }
                        cand[nc++] = r;
                    }
                }
                pv->n = keep;
            }
        }
        /* createNewCluster / addHitToCluster / mergeClusters */
        u.parent[hi] = hi;
        u.first[hi] = t;
        u.last[hi] = t;
        uint64_t root = hi;
        for (uint64_t c = 0; c < nc; ++c) {
            uint64_t r = cand[c];
            uint64_t f = u.first[r] < u.first[root] ? u.first[r] : u.first[root];
            /* chain the clusters: the accumulated root hangs under r */
            u.parent[root] = r;
            root = r;
            u.first[root] = f;
            u.last[root] = t;
        }
        /* record this cluster on the hit's pixel (once per cluster) */
        pix_vec *own = &pix[(uint64_t)h[hi].y * W + h[hi].x];
        int present = 0;
        for (uint32_t e = 0; e < own->n; ++e) if (uf_find(&u, own->v[e]) == root) { present = 1; break; }
        if (!present && pv_push(own, hi)) { rc = OR_ERR_NOMEM; goto done; }
    }
    /* canonical labels: smallest input index per cluster */
    {
        uint64_t *minidx = u.first;   /* reuse: first[] no longer needed */
        for (uint64_t i = 0; i < n; ++i) minidx[i] = NONE;
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t r = uf_find(&u, i);
            if (i < minidx[r]) minidx[r] = i;
        }
        for (uint64_t i = 0; i < n; ++i) label[i] = minidx[uf_find(&u, i)];
    }
    rc = OR_OK;
done:
    if (pix) for (uint64_t p = 0; p < npx; ++p) free(pix[p].v);
    free(pix); free(order); free(u.parent); free(u.first); free(u.last); free(cand);
    return rc;
}

int oracle_labels_global(const or_hit *h, uint64_t n, uint32_t W, uint32_t H,
                         uint64_t dt, uint64_t *label) {
    return sweep_labels(h, n, W, H, dt, 1, label);
}

int oracle_labels_static(const or_hit *h, uint64_t n, uint32_t W, uint32_t H,
                         uint64_t dt, uint64_t *label) {
    return sweep_labels(h, n, W, H, dt, 2, label);
}

/* ------------------------------------------------------------------------ */
/* Per-cluster features, records ordered by label.                          */
/* out must hold n records; *n_clusters receives the count.                 */

int oracle_features(const or_hit *h, uint64_t n, const uint64_t *label,
                    or_cluster *out, uint64_t *n_clusters) {
    if ((n && (!h || !label || !out)) || !n_clusters) return OR_ERR_ARG;
    uint64_t *slot = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t *swx = (uint64_t *)calloc(n ? n : 1, sizeof(uint64_t));
    uint64_t *swy = (uint64_t *)calloc(n ? n : 1, sizeof(uint64_t));
    if (!slot || !swx || !swy) { free(slot); free(swx); free(swy); return OR_ERR_NOMEM; }
    /* a label is the smallest member index, so labels appear in increasing
       order the first time each is seen, scanning indices upward */
    uint64_t m = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (label[i] >= n || label[label[i]] != label[i]) {
            free(slot); free(swx); free(swy); return OR_ERR_ARG;
        }
        if (label[i] == i) {
            slot[i] = m;
            out[m].label = i; out[m].size = 0; out[m].sum_tot = 0;
            out[m].first_toa = UINT64_MAX;
            m++;
        }
    }
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t c = slot[label[i]];
        out[c].size += 1;
        out[c].sum_tot += h[i].tot;
        if (h[i].toa < out[c].first_toa) out[c].first_toa = h[i].toa;
        swx[c] += (uint64_t)h[i].tot * h[i].x;
        swy[c] += (uint64_t)h[i].tot * h[i].y;
    }
    for (uint64_t c = 0; c < m; ++c) {
        double w = (double)out[c].sum_tot;
        out[c].cx = (double)swx[c] / w;
        out[c].cy = (double)swy[c] / w;
    }
    *n_clusters = m;
    free(slot); free(swx); free(swy);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Hit buffer filling (Algorithm 2, Section 4.1): the host-side procedure     */
/* storeHit(hit, buffer, nextBuffer), called once per hit in arrival order.  */
/*   b         maximum buffer size                                           */
/*   b_t       room kept free at the end of a buffer for late hits            */
/*   t         the stream's disorder bound (the stream is t-ordered)          */
/*   t_closing slack added to toa_max to place the buffer's closing time      */
/* A buffer takes hits freely while it holds fewer than b - b_t; after that   */
/* only hits earlier than toa_max + t_closing, the rest go to the next        */
/* buffer; a hit later than toa_max + t + t_closing sends the buffer, and the */
/* next buffer becomes the current one.  toa_max is one variable for the      */
/* whole stream, updated only by hits taken while the buffer has room, as the */
/* procedure states.                                                          */
/* Readings where the procedure is silent: b caps the closing phase, so a    */
/* hit that qualifies for a full buffer (b hits) goes to the next buffer (the */
/* next buffer itself has no cap in the procedure); at the end of the stream */
/* the current buffer and then a non-empty next buffer are sent.             */
/* Output: buffer_of[i] = number of the buffer hit i lands in (buffers are    */
/* numbered in the order they are sent; inside a buffer hits keep arrival    */
/* order); cut[k] = toa_max + t_closing when buffer k was sent (saturating;  */
/* UINT64_MAX for buffers sent at the end); *n_buffers = buffers sent.        */
/* cut must hold n + 1 entries.                                               */

static uint64_t sat_add(uint64_t a, uint64_t b) { return a > UINT64_MAX - b ? UINT64_MAX : a + b; }

int oracle_fill_buffers(const or_hit *h, uint64_t n, uint64_t b, uint64_t b_t, uint64_t t,
                        uint64_t t_closing, uint64_t *buffer_of, uint64_t *cut,
                        uint64_t *n_buffers) {
    if ((n && (!h || !buffer_of)) || !cut || !n_buffers || b == 0 || b_t >= b) return OR_ERR_ARG;
    uint64_t toa_max = 0;
    uint64_t cur = 0;          /* number of the current buffer; the next one is cur + 1 */
    uint64_t size_cur = 0, size_next = 0;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t toa = h[i].toa;
        if (size_cur < b - b_t) {
            buffer_of[i] = cur;
            size_cur++;
            if (toa > toa_max) toa_max = toa;
        } else if (toa < sat_add(toa_max, t_closing) && size_cur < b) {
            buffer_of[i] = cur;
            size_cur++;
        } else {
            buffer_of[i] = cur + 1;
            size_next++;
        }
        if (toa > toa_max && toa - toa_max > sat_add(t, t_closing)) {
            cut[cur] = sat_add(toa_max, t_closing);   /* sendToDevice(buffer) */
            cur++;                                     /* buffer <- nextBuffer */
            size_cur = size_next;
            size_next = 0;
        }
    }
    uint64_t sent = cur;
    if (size_cur) cut[sent++] = UINT64_MAX;
    if (size_next) cut[sent++] = UINT64_MAX;
    *n_buffers = sent;
    return OR_OK;
}

uint32_t oracle_hit_size(void) { return (uint32_t)sizeof(or_hit); }
uint32_t oracle_cluster_size(void) { return (uint32_t)sizeof(or_cluster); }
