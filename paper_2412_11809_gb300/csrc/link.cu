// Neighbour search and union-find hooking (Algorithm 3 steps 4-5, Section 4.1)
// for the edge-connectivity variant (iii)(a).
//
// Hits are in (ToA, position) order ("rank" order).  Every edge (j, i) of
// the hit graph — 8-adjacent or same pixel, |dToA| <= dt — has its earlier
// end j among the hits within dt before i, so each hit looks only at that
// time window and joins every adjacent hit in it (the complete edge set, so
// the components are exact by construction).
//
// k_tile_link_table (the main path): one CTA per tile of TILE ranks with a
//   per-pixel list table in shared memory (the paper's pixel matrix), for
//   sensors the table covers in at most TAB_MAX_BANDS bands of rows; see the
//   comment above the kernel.
// k_tile_link (sensors the table cannot cover, and tiles the table kernel
//   gave back): the tile staged in shared memory, then
//   window mode (sparse tiles: few hits within dt of a hit, on average):
//     every pair (k, j < k) within dt is checked for adjacency, the pairs
//     spread evenly over the threads by a prefix sum of the window lengths;
//   bucket mode (dense tiles): the tile is counting-sorted into buckets of
//     4x4-pixel cells (hashed onto NBUCKETS buckets) and hit k scans the (at
//     most four) buckets covering its 3x3 neighbourhood.
//   Unions run on a shared-memory forest; the smallest rank of each
//   component (its earliest hit) becomes the tile root in the global forest.
//
// k_border_fast / k_border_link: edges whose earlier end lies before the tile
// (the paper's step 5, "border hits at the start of the next chunk").  The
// halo is every earlier hit within dt of the tile's first hit; the front is
// every tile hit within dt of the halo's last hit.  One warp per border from
// staged windows when both are small; otherwise block-wide, pairwise or with
// the halo bucketed by cell.  Unions run on the global forest.
//
// k_sorted_roots (variants (b) and (c) only): the root of every sorted
// position after the (a) links, into the idle radix buffer (the forest is
// left as it is; every root is a tile root, whose slot the tile kernels
// zeroed).  k_init_roots (after the (b)/(c) merges): the slots of the final
// roots, which (c) can pick among non-roots.
#include "tpc_internal.cuh"

namespace tpc {

constexpr int LINK_THREADS = 512;
constexpr uint32_t TAB_CAP = 68u << 10;        // table entries: sensor plus a 1-pixel frame
constexpr uint32_t TAB_MAX_BANDS = 16;

// Table mode: the sensor, with a frame of empty pixels around it, is covered
// by the shared-memory table in at most TAB_MAX_BANDS bands of rows (one band
// for a 256 x 256 sensor, 258 x 258 entries; four for 448 x 512).  Rows per
// band (a band's table also holds the row above and the row below it);
// 0 when the sensor does not qualify.
__device__ __forceinline__ uint32_t table_rows(uint32_t W, uint32_t H) {
    const uint32_t W2 = W + 2;
    if (W2 * 3 > TAB_CAP) return 0;
    const uint32_t rpb = TAB_CAP / W2 - 2;
    return (H + rpb - 1) / rpb <= TAB_MAX_BANDS ? rpb : 0;
}
__device__ __forceinline__ bool table_mode(uint32_t W, uint32_t H) { return table_rows(W, H) != 0; }

// Host view of the same rule: bands of the table for a W x H sensor (0 =
// the sensor takes k_tile_link).
int link_bands(uint32_t W, uint32_t H) {
    const uint32_t W2 = W + 2;
    if (W2 * 3 > TAB_CAP) return 0;
    const uint32_t rpb = TAB_CAP / W2 - 2;
    const uint32_t nb = (H + rpb - 1) / rpb;
    return nb <= TAB_MAX_BANDS ? (int)nb : 0;
}
constexpr int NBUCKETS = 2048;                // hashed 4x4-pixel cells
constexpr int HALO_BATCH = 2048;
constexpr int BORDER_THREADS = 256;
constexpr uint32_t BORDER_PAIRS_DIRECT = 1u << 12;

__device__ __forceinline__ bool adjacent(uint32_t a, uint32_t b) {
    const int dx = (int)(a & 0xFFFFu) - (int)(b & 0xFFFFu);
    const int dy = (int)(a >> 16) - (int)(b >> 16);
    return dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1;
}

// Shared-memory forest with randomised linking: the root with the lower
// pseudo-random priority is hooked under the other, which keeps the expected
// tree depth logarithmic however the edges arrive (linking by index would
// chain a 300-hit track whose edges are joined in parallel).  The smallest
// rank of each component is found afterwards.
__device__ __forceinline__ uint32_t link_prio(uint32_t k) {
    uint32_t h = k * 0x9E3779B1u;
    h ^= h >> 15;
    h *= 0x85EBCA77u;
    return h ^ (h >> 13);
}

__device__ __forceinline__ void sunion_prio(uint32_t *parent, uint32_t a, uint32_t b) {
    while (true) {
        a = sfind(parent, a);
        b = sfind(parent, b);
        if (a == b) return;
        const uint32_t pa = link_prio(a), pb = link_prio(b);
        if (pa < pb || (pa == pb && a < b)) { uint32_t t = a; a = b; b = t; }
        // b has the lower priority: hook it under a
        if (atomicCAS(parent + b, b, a) == b) return;
    }
}

// Bucket of the 4x4-pixel cell holding (x, y); cells are hashed onto
// NBUCKETS buckets (a collision only adds candidates, never drops one).
__device__ __forceinline__ uint32_t cell_bucket(uint32_t x, uint32_t y, uint32_t cw) {
    return ((y >> 2) * cw + (x >> 2)) & (NBUCKETS - 1);
}

// The (up to four) distinct buckets covering the 3x3 neighbourhood of (x, y).
__device__ __forceinline__ int neighbour_buckets(uint32_t pix, uint32_t W, uint32_t H, uint32_t cw,
                                                 uint32_t b[4]) {
    const uint32_t x = pix & 0xFFFFu, y = pix >> 16;
    const uint32_t x0 = x ? x - 1 : 0, x1 = x + 1 < W ? x + 1 : x;
    const uint32_t y0 = y ? y - 1 : 0, y1 = y + 1 < H ? y + 1 : y;
    int n = 0;
    const uint32_t cand[4] = {cell_bucket(x0, y0, cw), cell_bucket(x1, y0, cw),
                              cell_bucket(x0, y1, cw), cell_bucket(x1, y1, cw)};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        bool dup = false;
        for (int j = 0; j < n; ++j) dup |= b[j] == cand[i];
        if (!dup) b[n++] = cand[i];
    }
    return n;
}

// Counting sort of entries 0..n of s_pix into cell buckets: bucket q holds
// s_seg[s_start[q] .. s_start[q+1]).  Order inside a bucket is arbitrary
// (the scans below compare ranks explicitly).
__device__ void bucket_sort(const uint32_t *s_pix, uint32_t n, uint32_t cw, uint32_t *s_start,
                            uint32_t *s_cur, uint16_t *s_seg, uint32_t *s_warp) {
    for (uint32_t q = threadIdx.x; q <= NBUCKETS; q += blockDim.x) s_start[q] = 0;
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x)
        atomicAdd(&s_start[cell_bucket(s_pix[k] & 0xFFFFu, s_pix[k] >> 16, cw) + 1], 1u);
    __syncthreads();
    // inclusive scan of s_start[1..NBUCKETS]: each thread owns `per` consecutive entries
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t per = (NBUCKETS + blockDim.x - 1) / blockDim.x;
    const uint32_t i0 = 1 + threadIdx.x * per;
    uint32_t local = 0;
    for (uint32_t i = i0; i < i0 + per && i <= NBUCKETS; ++i) local += s_start[i];
    uint32_t x = local;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t run = x - local;
    for (int q = 0; q < warp; ++q) run += s_warp[q];
    __syncthreads();
    for (uint32_t i = i0; i < i0 + per && i <= NBUCKETS; ++i) {
        run += s_start[i];
        s_start[i] = run;
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < NBUCKETS; q += blockDim.x) s_cur[q] = s_start[q];
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
        const uint32_t q = cell_bucket(s_pix[k] & 0xFFFFu, s_pix[k] >> 16, cw);
        s_seg[atomicAdd(&s_cur[q], 1u)] = (uint16_t)k;
    }
    __syncthreads();
}

// Load-balanced window scan: every pair (k, j) with j < k and
// key(k) - key(j) <= dt is one unit of work; a prefix sum over the window
// lengths hands each thread an equal slice of the pairs, so lanes neither
// wait on long windows (bursty tracks) nor on each other.
constexpr uint32_t EDGE_BUF = 256;   // queued adjacent pairs per warp

__device__ void link_window(const uint32_t *s_key, const uint32_t *s_pix, uint32_t *s_par,
                            uint16_t *s_lo, uint32_t *s_pref, uint32_t *s_warp, uint32_t *s_edges,
                            uint32_t n_t, uint32_t dt) {
    constexpr uint32_t PER = TILE / LINK_THREADS;
    const uint32_t k0 = threadIdx.x * PER;
    uint32_t sum = 0;
    if (k0 < n_t) {
        const uint32_t key0 = s_key[k0], tgt = key0 >= dt ? key0 - dt : 0;
        uint32_t lo = 0, hi = k0;           // first rank with key >= tgt
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_key[mid] < tgt) lo = mid + 1; else hi = mid;
        }
        for (uint32_t k = k0; k < k0 + PER && k < n_t; ++k) {
            const uint32_t key = s_key[k];
            while (key - s_key[lo] > dt) ++lo;
            s_lo[k] = (uint16_t)lo;
            sum += k - lo;
        }
    }
    // exclusive prefix of the window lengths: s_pref[k], s_pref[n_t] = total
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t run = x - sum;
    for (int q = 0; q < warp; ++q) run += s_warp[q];
    for (uint32_t k = k0; k < k0 + PER && k < n_t; ++k) {
        s_pref[k] = run;
        run += k - s_lo[k];
    }
    if (threadIdx.x == LINK_THREADS - 1) {
        uint32_t tot = 0;
        for (int q = 0; q < LINK_THREADS / 32; ++q) tot += s_warp[q];
        s_pref[n_t] = tot;
    }
    __syncthreads();
    const uint32_t total = s_pref[n_t];
    // each warp takes a contiguous range of pairs; lane i handles pair
    // base + i, so lanes share the hit k (broadcast reads) and read
    // consecutive earlier hits j (no bank conflicts)
    constexpr uint32_t NW = LINK_THREADS / 32;
    const uint32_t w0 = (uint32_t)((uint64_t)total * warp / NW);
    const uint32_t w1 = (uint32_t)((uint64_t)total * (warp + 1) / NW);
    uint32_t k = 0;
    if (w0 + lane < w1) {
        uint32_t lo = 0, hi = n_t;          // last k with s_pref[k] <= p
        const uint32_t p = w0 + lane;
        while (lo + 1 < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_pref[mid] <= p) lo = mid; else hi = mid;
        }
        k = lo;
    }
    // adjacent pairs are queued per warp and joined by all 32 lanes at once
    // (a round has only a few adjacent pairs; joining them where they are
    // found would leave most lanes idle behind a latency-bound union)
    uint32_t *buf = s_edges + warp * EDGE_BUF;
    uint32_t count = 0;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t pb = w0; pb < w1; pb += 32) {
        const uint32_t p = pb + lane;
        bool adj = false;
        uint32_t j = 0;
        if (p < w1) {
            while (p >= s_pref[k + 1]) ++k;
            j = s_lo[k] + (p - s_pref[k]);
            adj = adjacent(s_pix[k], s_pix[j]);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, adj);
        if (adj) buf[count + __popc(m & lt)] = (k << 16) | j;
        count += __popc(m);
        if (count > EDGE_BUF - 32) {
            __syncwarp();
            for (uint32_t i = lane; i < count; i += 32) sunion_prio(s_par, buf[i] >> 16, buf[i] & 0xFFFFu);
            __syncwarp();
            count = 0;
        }
    }
    __syncwarp();
    for (uint32_t i = lane; i < count; i += 32) sunion_prio(s_par, buf[i] >> 16, buf[i] & 0xFFFFu);
}

__global__ void __launch_bounds__(LINK_THREADS) k_tile_link(Work w) {
    extern __shared__ uint32_t smem[];
    uint32_t *s_key = smem;                  // [TILE]
    uint32_t *s_pix = s_key + TILE;          // [TILE] x | y << 16
    uint32_t *s_par = s_pix + TILE;          // [TILE] shared-memory forest
    uint32_t *s_start = s_par + TILE;        // [NBUCKETS + 1] (window mode: prefix, TILE + 1)
    uint32_t *s_cur = s_start + NBUCKETS + 1;  // [NBUCKETS]
    uint32_t *s_warp = s_cur + NBUCKETS;     // [32]
    uint16_t *s_seg = reinterpret_cast<uint16_t *>(s_warp + 32);  // [TILE] (window mode: lo)
    uint32_t *s_edges = reinterpret_cast<uint32_t *>(s_seg + TILE);  // [warps * EDGE_BUF]
    static_assert(2 * NBUCKETS + 1 >= TILE + 1, "prefix array size");

    const Prob &P = *w.prob;
    const uint32_t *skey = pick(w.keys, sorted_sel(P));
    // tiles of large sensors, then the tiles the table kernel gave back
    const uint32_t n_large = P.ntiles, n_all = P.ntiles + P.redo_count;
    for (uint32_t u = blockIdx.x; u < n_all; u += gridDim.x) {
        const uint32_t t = u < n_large ? u : w.redo[u - n_large];
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint32_t n_t = end - begin, W = g.width, H = g.height, dt = g.dt;
        if (u < n_large && table_mode(W, H) && !g.link_general) continue;   // done by k_tile_link_table
        const uint32_t cw = (W + 3) >> 2;
        {
            constexpr int ITEMS = TILE / LINK_THREADS;
            uint32_t kv[ITEMS], pv[ITEMS];
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {   // every load in flight before any use
                const uint32_t k = q * LINK_THREADS + threadIdx.x;
                if (k < n_t) { kv[q] = skey[begin + k]; pv[q] = w.spix[begin + k]; }
            }
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const uint32_t k = q * LINK_THREADS + threadIdx.x;
                if (k < n_t) { s_key[k] = kv[q]; s_pix[k] = pv[q]; s_par[k] = k; }
            }
        }
        __syncthreads();
        // mean window length (hits within dt before a hit) decides the mode
        const uint64_t span = (uint64_t)(s_key[n_t - 1] - s_key[0]) + 1;
        const uint64_t window = (uint64_t)n_t * ((uint64_t)dt + 1) / span;
        if (window <= 48) {
            link_window(s_key, s_pix, s_par, s_seg, s_start, s_warp, s_edges, n_t, dt);
        } else {
            bucket_sort(s_pix, n_t, cw, s_start, s_cur, s_seg, s_warp);
            for (uint32_t k = threadIdx.x; k < n_t; k += LINK_THREADS) {
                const uint32_t key = s_key[k], pix = s_pix[k];
                uint32_t b[4];
                const int nb = neighbour_buckets(pix, W, H, cw, b);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (i >= nb) break;
                    for (uint32_t q = s_start[b[i]]; q < s_start[b[i] + 1]; ++q) {
                        const uint32_t j = s_seg[q];
                        if (j < k && key - s_key[j] <= dt && adjacent(pix, s_pix[j])) sunion_prio(s_par, k, j);
                    }
                }
            }
        }
        __syncthreads();
        // smallest rank per component; the bucket arrays are free again
        // (s_start and s_cur are contiguous: 2 * NBUCKETS + 1 >= TILE entries)
        static_assert(2 * NBUCKETS + 1 >= TILE, "min array size");
        uint32_t *s_min = s_start;
        for (uint32_t k = threadIdx.x; k < n_t; k += LINK_THREADS) s_min[k] = 0xFFFFFFFFu;
        __syncthreads();
        uint32_t *s_root = s_key;   // keys are no longer needed; only k's thread writes s_root[k]
        for (uint32_t k = threadIdx.x; k < n_t; k += LINK_THREADS) {
            const uint32_t r = sfind(s_par, k);
            s_root[k] = r;
            atomicMin(&s_min[r], k);
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < n_t; k += LINK_THREADS) {
            const uint32_t m = s_min[s_root[k]];
            w.parent[begin + k] = begin + m;
            if (m == k) init_slot(w, begin + k);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Table mode, for sensors that fit TAB_CAP with a frame: a direct-mapped
// per-pixel table in shared memory (the paper's per-pixel matrix with 2-byte
// entries, Algorithm 3 step 4 and Section 4.2) heads a lock-free list of the
// tile's hits on each pixel (16-bit compare-and-swap pushes).  Hit k walks the
// lists of its 9 pixels; every earlier hit there within dt is an edge.  The
// table has a frame of never-used entries around the sensor, so the 9
// lookups need no bounds checks.
//
// Components: each hit points to the smallest earlier neighbour it found (a
// forest, since parents have smaller ranks, whose roots are the smallest
// ranks of their trees); further neighbours go to an edge list.  Each listed
// edge is then a lock-free union that hooks the larger root under the
// smaller with compare-and-swap (Jaiganesh & Burtscher's ECL-CC hooking),
// straight on that forest: the finds halve the paths they walk, which
// shortens them for the finds after (a separate pointer-jumping pass over
// every hit first measured slower), so the surviving root of a component is
// its smallest rank, i.e. its earliest hit.  A list longer than
// TAB_WALK (a pile on one pixel) or more edges than the list holds send the
// tile to k_tile_link instead.  Only the table entries a tile touched are
// reset afterwards (Algorithm 3 step 7).
constexpr int TAB_THREADS = 1024;
constexpr uint16_t TAB_NONE = 0x7FFFu;   // empty list / end of list
constexpr uint32_t TAB_MORE = 0x8000u;   // table entry flag: the list holds a second hit
constexpr int TAB_WALK = 64;
constexpr int TAB_EDGES = 3 * TILE / 2;

struct TabShared {
    uint16_t tab[TAB_CAP];           // head of each pixel's list (rank), or TAB_NONE
    uint32_t key[TILE];              // per rank: key
    uint16_t next[TILE];             // per rank: next rank on the same pixel
    uint32_t par[TILE];              // forest over ranks
    uint32_t edges[TAB_EDGES];       // banded: extra-edge buffers, then the shared list (k << 16 | j)
    uint32_t pix[TILE];              // per rank: pixel (banded sensors)
    uint16_t wl[TILE];               // ranks walked in the current band
    uint32_t wl_count[TAB_MAX_BANDS];
    uint32_t nedges;
    uint32_t overflow;
};
constexpr int TAB_SMEM = (int)sizeof(TabShared);

// table entry of pixel (x, y): row y + 1, column x + 1 of a (W + 2)-wide table
__device__ __forceinline__ uint32_t tab_pid(uint32_t pix, uint32_t W) {
    return ((pix >> 16) + 1) * (W + 2) + (pix & 0xFFFFu) + 1;
}

// push rank k on pixel pid's list; returns the previous head (a rank, or
// TAB_NONE).  The new head entry carries TAB_MORE when the list already held
// a hit, so walks see multi-hit lists without reading the link array.
__device__ __forceinline__ uint16_t tab_push(uint16_t *tab, uint32_t pid, uint16_t k) {
    uint32_t *word = reinterpret_cast<uint32_t *>(tab) + (pid >> 1);
    const uint32_t shift = (pid & 1u) * 16u;
    uint32_t old = *reinterpret_cast<volatile uint32_t *>(word);
    while (true) {
        const uint32_t prev = (old >> shift) & 0x7FFFu;
        const uint32_t ent = (uint32_t)k | (prev != TAB_NONE ? TAB_MORE : 0u);
        const uint32_t nv = (old & ~(0xFFFFu << shift)) | (ent << shift);
        const uint32_t seen = atomicCAS(word, old, nv);
        if (seen == old) return (uint16_t)prev;
        old = seen;
    }
}

// root of x with path halving: every other node on the way is pointed at its
// grandparent (parents only ever move towards the root, so this is safe
// against concurrent hooks, which only ever rewrite roots)
__device__ __forceinline__ uint32_t tab_root(volatile uint32_t *par, uint32_t x) {
    while (true) {
        const uint32_t p = par[x];
        const uint32_t gp = par[p];
        if (p == gp) return p;
        par[x] = gp;
        x = gp;
    }
}

// Union of the components of a and b: hook the larger root under the
// smaller.  A failed compare-and-swap means another thread hooked that root
// first (each retry follows one completed hook, so there are fewer retries
// than ranks); returns false only if that bound is exceeded.
__device__ __forceinline__ bool tab_union(volatile uint32_t *par, uint32_t a, uint32_t b) {
    uint32_t ra = tab_root(par, a), rb = tab_root(par, b);
    for (int it = 0; it < TILE; ++it) {
        if (ra == rb) return true;
        if (ra > rb) { const uint32_t t = ra; ra = rb; rb = t; }
        const uint32_t old = atomicCAS(const_cast<uint32_t *>(par) + rb, rb, ra);
        if (old == rb) return true;
        rb = tab_root(par, old);
        ra = tab_root(par, ra);
    }
    return false;
}

// Extra edges.  Each thread lists the extra edges of the hits it walks into
// a buffer of its own as soon as they are known, so no warp-wide pass lists
// them; the union phase then takes each thread's buffer.  One-band sensors:
// a thread walks its own hits q * TAB_THREADS + t, so an entry is
// q << 12 | j (16 bits, TAB_EB per thread in the pixel array, which only
// banded sensors use).  Banded sensors: a thread walks listed hits, so an
// entry is k << 12 | j (32 bits, TAB_EBB per thread in the first part of the
// edge array).  Entry s of thread t sits at [s * TAB_THREADS + t].  Edges
// beyond a buffer go to the shared list (the rest of the edge array).
constexpr int TAB_EB = 8;
constexpr int TAB_EBB = 3;
constexpr uint32_t TAB_LIST_BAND = TAB_EDGES - TAB_EBB * TAB_THREADS;   // shared-list entries, banded
static_assert(TAB_EB * TAB_THREADS * 2 <= TILE * 4, "one-band buffers fit the pixel array");
static_assert(TAB_LIST_BAND > 0, "banded buffers leave a shared list");

template <bool BAND>
__device__ __forceinline__ uint32_t *tab_list(TabShared &S) { return BAND ? S.edges + TAB_EBB * TAB_THREADS : S.edges; }
template <bool BAND>
__device__ __forceinline__ uint32_t tab_list_cap() { return BAND ? TAB_LIST_BAND : (uint32_t)TAB_EDGES; }

// The walk of hit k (key `key`; `centre` = its pixel's table entry, rows W2
// entries apart; q: its item when the thread walks its own hits).  Returns
// its parent: the smallest earlier neighbour within dt, or k if it has none.
// Every other earlier neighbour within dt is an extra edge (k, j), listed
// at the neighbour that reveals it (the neighbour itself, or the parent it
// displaces).  The heads of the 9 lists are read first (independent loads),
// then tested without branches: an empty head (TAB_NONE) is a rank above
// every hit.  Lists whose head entry carries TAB_MORE hold further hits (a
// pixel hit more than once in the tile: rare) and are walked afterwards.
template <bool BAND>
__device__ __forceinline__ uint32_t tab_walk(TabShared &S, uint32_t q, uint32_t k, uint32_t key, uint32_t centre,
                                             uint32_t W2, uint32_t dt, uint32_t &ecnt) {
    auto edge = [&](uint32_t e) {
        if (BAND) {
            if (ecnt < TAB_EBB) S.edges[ecnt * TAB_THREADS + threadIdx.x] = k << 12 | e;
        } else {
            if (ecnt < TAB_EB) reinterpret_cast<uint16_t *>(S.pix)[ecnt * TAB_THREADS + threadIdx.x] = (uint16_t)(q << 12 | e);
        }
        if (ecnt >= (BAND ? TAB_EBB : TAB_EB)) {   // the shared list
            const uint32_t slot = atomicAdd(&S.nedges, 1u);
            if (slot < tab_list_cap<BAND>()) tab_list<BAND>(S)[slot] = (k << 16) | e;
        }
        ++ecnt;
    };
    uint32_t hd[9];
#pragma unroll
    for (int n = 0; n < 9; ++n) hd[n] = S.tab[centre + (n / 3 - 1) * (int)W2 + (n % 3 - 1)];
    uint32_t more = 0, mn = TAB_NONE;
#pragma unroll
    for (int n = 0; n < 9; ++n) {
        more |= (hd[n] >> 15) << n;           // TAB_MORE
        hd[n] &= 0x7FFFu;
        const uint32_t j = hd[n];
        bool ok = false;                           // an empty head (TAB_NONE) is never below k
        if (j < k) ok = key - S.key[j] <= dt;
        const uint32_t e = j < mn ? mn : j;        // the new edge: the old parent, or j
        if (ok && e != TAB_NONE) edge(e);
        mn = ok && j < mn ? j : mn;
    }
    while (more) {   // lists holding more than one hit
        const int n = __ffs(more) - 1;
        more &= more - 1;
        uint32_t h = hd[0];
#pragma unroll
        for (int m = 1; m < 9; ++m)   // a select, not an indexed load: hd stays in registers
            if (m == n) h = hd[m];
        uint32_t j = S.next[h];
        int steps = 1;
        for (; j != TAB_NONE && steps < TAB_WALK; j = S.next[j], ++steps) {
            if (j < k && key - S.key[j] <= dt) {
                const uint32_t e = j < mn ? mn : j;
                if (e != TAB_NONE) edge(e);
                mn = j < mn ? j : mn;
            }
        }
        if (j != TAB_NONE) S.overflow = 1;
    }
    return mn == TAB_NONE ? k : mn;
}

__global__ void __launch_bounds__(TAB_THREADS, 1) k_tile_link_table(Work w) {
    extern __shared__ __align__(16) unsigned char tab_raw[];
    TabShared &S = *reinterpret_cast<TabShared *>(tab_raw);
    volatile uint32_t *vpar = S.par;
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    const uint32_t *skey = pick(w.keys, sorted_sel(P));
    const int lane = threadIdx.x & 31;
    for (uint32_t i = threadIdx.x; i < TAB_CAP / 2; i += TAB_THREADS)
        reinterpret_cast<uint32_t *>(S.tab)[i] = 0x7FFF7FFFu;
    __syncthreads();
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        const uint32_t W = g.width, H = g.height, dt = g.dt;
        const uint32_t rpb = g.link_general ? 0u : table_rows(W, H);
        if (!rpb) continue;   // k_tile_link handles sensors the table cannot cover
        const uint32_t nb = (H + rpb - 1) / rpb, W2 = W + 2;
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint32_t n_t = end - begin;
        constexpr int ITEMS = TILE / TAB_THREADS;   // 4
        uint32_t kv[ITEMS], pv[ITEMS];
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {
            const uint32_t k = q * TAB_THREADS + threadIdx.x;
            if (k < n_t) { kv[q] = skey[begin + k]; pv[q] = w.spix[begin + k]; }
        }
        if (threadIdx.x == 0) { S.overflow = 0; S.nedges = 0; }
        uint32_t ecnt = 0;   // one band: this thread's buffered extra edges
        if (nb == 1) {
            // the whole sensor in one table: push every hit, then walk each
            // from registers
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const uint32_t k = q * TAB_THREADS + threadIdx.x;
                if (k < n_t) {
                    S.key[k] = kv[q];
                    S.next[k] = tab_push(S.tab, tab_pid(pv[q], W), (uint16_t)k);
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const uint32_t k = q * TAB_THREADS + threadIdx.x;
                if (k < n_t) S.par[k] = tab_walk<false>(S, q, k, kv[q], tab_pid(pv[q], W), W2, dt, ecnt);
            }
        } else {
            // band by band: a band's table holds its rows and the rows just
            // above and below; its hits are listed and walked by all lanes,
            // then the entries it pushed are cleared for the next band
            if (threadIdx.x < TAB_MAX_BANDS) S.wl_count[threadIdx.x] = 0;
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const uint32_t k = q * TAB_THREADS + threadIdx.x;
                if (k < n_t) { S.key[k] = kv[q]; S.pix[k] = pv[q]; }
            }
            __syncthreads();
            for (uint32_t b = 0; b < nb; ++b) {
                const uint32_t y0 = b * rpb, y1 = y0 + rpb < H ? y0 + rpb : H;
#pragma unroll
                for (int q = 0; q < ITEMS; ++q) {
                    const uint32_t k = q * TAB_THREADS + threadIdx.x;
                    const uint32_t y = pv[q] >> 16;
                    const bool in = k < n_t && y + 1 >= y0 && y <= y1;   // rows y0 - 1 .. y1
                    if (in)
                        S.next[k] = tab_push(S.tab, (y + 1 - y0) * W2 + (pv[q] & 0xFFFFu) + 1, (uint16_t)k);
                    const bool own = in && y >= y0 && y < y1;
                    const uint32_t m = __ballot_sync(0xffffffffu, own);
                    uint32_t slot0 = 0;
                    if (lane == 0 && m) slot0 = atomicAdd(&S.wl_count[b], (uint32_t)__popc(m));
                    slot0 = __shfl_sync(0xffffffffu, slot0, 0);
                    if (own) S.wl[slot0 + __popc(m & ((1u << lane) - 1u))] = (uint16_t)k;
                }
                __syncthreads();
                const uint32_t cnt = S.wl_count[b];
                for (uint32_t base = 0; base < cnt; base += TAB_THREADS) {
                    const uint32_t idx = base + threadIdx.x;
                    if (idx < cnt) {
                        const uint32_t k = S.wl[idx];
                        const uint32_t pix = S.pix[k];
                        S.par[k] = tab_walk<true>(S, 0, k, S.key[k],
                                                  ((pix >> 16) + 1 - y0) * W2 + (pix & 0xFFFFu) + 1, W2, dt, ecnt);
                    }
                }
                __syncthreads();
#pragma unroll
                for (int q = 0; q < ITEMS; ++q) {
                    const uint32_t k = q * TAB_THREADS + threadIdx.x;
                    const uint32_t y = pv[q] >> 16;
                    if (k < n_t && y + 1 >= y0 && y <= y1) S.tab[(y + 1 - y0) * W2 + (pv[q] & 0xFFFFu) + 1] = TAB_NONE;
                }
                __syncthreads();
            }
        }
        __syncthreads();
        const uint32_t *list = nb == 1 ? tab_list<false>(S) : tab_list<true>(S);
        bool redo = S.overflow || S.nedges > (nb == 1 ? tab_list_cap<false>() : tab_list_cap<true>());
        if (!redo) {
            const uint32_t ne = S.nedges;
            bool ok = true;
            // the shared list (edges beyond the threads' buffers) is filled
            // warp by warp, so neighbouring entries tend to share roots:
            // lanes take entries ne / 32 apart (fewer colliding
            // compare-and-swaps within a warp)
            const uint32_t ccol = (ne + 31) >> 5;
            for (uint32_t e = threadIdx.x; e < 32 * ccol; e += TAB_THREADS) {
                const uint32_t idx = (e & 31) * ccol + (e >> 5);
                if (idx >= ne) continue;
                const uint32_t ed = list[idx];
                ok &= tab_union(vpar, ed >> 16, ed & 0xFFFFu);
            }
            if (nb == 1) {   // this thread's buffered edges
                const uint16_t *eb = reinterpret_cast<const uint16_t *>(S.pix);
                for (uint32_t i = 0; i < ecnt && i < TAB_EB; ++i) {
                    const uint32_t e = eb[i * TAB_THREADS + threadIdx.x];
                    ok &= tab_union(vpar, (e >> 12) * TAB_THREADS + threadIdx.x, e & (TILE - 1));
                }
            } else {
                for (uint32_t i = 0; i < ecnt && i < TAB_EBB; ++i) {
                    const uint32_t e = S.edges[i * TAB_THREADS + threadIdx.x];
                    ok &= tab_union(vpar, e >> 12, e & (TILE - 1));
                }
            }
            redo = !__syncthreads_and(ok);
        }
        if (redo) {   // leave this tile to k_tile_link
            if (threadIdx.x == 0) {
                const uint32_t slot = atomicAdd(&w.prob->redo_count, 1u);
                w.redo[slot] = t;
            }
            if (nb == 1) {   // (banded tables were cleared band by band)
#pragma unroll
                for (int q = 0; q < ITEMS; ++q) {
                    const uint32_t k = q * TAB_THREADS + threadIdx.x;
                    if (k < n_t) S.tab[tab_pid(pv[q], W)] = TAB_NONE;
                }
            }
            __syncthreads();
            continue;
        }
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {
            const uint32_t k = q * TAB_THREADS + threadIdx.x;
            if (k < n_t) {
                const uint32_t r = tab_root(vpar, k);
                w.parent[begin + k] = begin + r;
                if (r == k) init_slot(w, begin + k);
                if (nb == 1) S.tab[tab_pid(pv[q], W)] = TAB_NONE;   // reset only what this tile touched
            }
        }
        __syncthreads();
    }
}

// One warp per tile border, for the usual case of a halo and a front of at
// most BF_WIN hits each: keys, pixels and tile roots of both are staged by
// one round of loads, the halo and front counted with ballots, and every
// (front, halo) pair within dt is checked from shared memory, newest halo
// hit first.  An adjacent pair contributes the edge between the two hits'
// tile roots (the tile links left every hit one step from its tile root);
// each lane drops repeats of its previous edge and the warp then runs one
// union per listed edge, so a dense border does not pay a chain of global
// finds per pair.  Borders with a larger halo or front are listed for
// k_border_link.
constexpr int BF_WARPS = 8;
constexpr int BF_WIN = 128;
constexpr int BF_PER_LANE = BF_WIN / 32;
constexpr int BF_EDGES = 64;

__global__ void __launch_bounds__(BF_WARPS * 32, 4) k_border_fast(Work w) {
    __shared__ uint32_t s_hk[BF_WARPS][BF_WIN];
    __shared__ uint32_t s_hp[BF_WARPS][BF_WIN];
    __shared__ uint32_t s_hr[BF_WARPS][BF_WIN];
    __shared__ uint32_t s_ea[BF_WARPS][BF_EDGES], s_eb[BF_WARPS][BF_EDGES];
    __shared__ uint32_t s_ne[BF_WARPS];
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    const uint32_t *skey = pick(w.keys, sorted_sel(P));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *hk = s_hk[warp], *hp = s_hp[warp], *hr = s_hr[warp], *ea = s_ea[warp], *eb = s_eb[warp];
    if (lane == 0) s_ne[warp] = 0;
    __syncwarp();
    for (uint32_t t = blockIdx.x * BF_WARPS + warp; t < nt; t += gridDim.x * BF_WARPS) {
        const Seg &g = w.seg[w.tile_seg[t]];
        if (t == g.tile0) continue;   // nothing before the segment's first tile
        uint32_t s0, end;
        tile_range(g, t, s0, end);
        const uint32_t dt = g.dt;
        const uint32_t nwh = s0 - g.off < (uint32_t)BF_WIN ? s0 - g.off : BF_WIN;
        const uint32_t nwf = end - s0 < (uint32_t)BF_WIN ? end - s0 : BF_WIN;
        const uint32_t hb = s0 - nwh;
        uint32_t fk[BF_PER_LANE], fp[BF_PER_LANE], fr[BF_PER_LANE];
#pragma unroll
        for (int u = 0; u < BF_PER_LANE; ++u) {
            const uint32_t j = u * 32 + lane;
            if (j < nwh) {
                hk[j] = skey[hb + j];
                hp[j] = w.spix[hb + j];
                hr[j] = w.parent[hb + j];
            }
            fk[u] = j < nwf ? skey[s0 + j] : 0xFFFFFFFFu;
            fp[u] = j < nwf ? w.spix[s0 + j] : 0;
            fr[u] = j < nwf ? w.parent[s0 + j] : 0;
        }
        __syncwarp();
        const uint32_t k0 = __shfl_sync(0xffffffffu, fk[0], 0);
        const uint32_t lo_key = k0 >= dt ? k0 - dt : 0;
        const uint64_t hi64 = (uint64_t)hk[nwh - 1] + dt;
        const uint32_t hi_key = hi64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)hi64;
        uint32_t nh = 0, nf = 0;
#pragma unroll
        for (int u = 0; u < BF_PER_LANE; ++u) {
            const uint32_t j = u * 32 + lane;
            nh += __popc(__ballot_sync(0xffffffffu, j < nwh && hk[j] >= lo_key));
            nf += __popc(__ballot_sync(0xffffffffu, j < nwf && fk[u] <= hi_key));
        }
        const bool halo_in = nh < nwh || hb == g.off, front_in = nf < nwf || s0 + nwf == end;
        if (halo_in && front_in) {
            uint32_t la = 0xFFFFFFFFu, lb = 0xFFFFFFFFu;   // this lane's previous edge
#pragma unroll
            for (int u = 0; u < BF_PER_LANE; ++u) {
                const uint32_t j = u * 32 + lane;
                if (j >= nf) continue;
                const uint32_t key = fk[u], pix = fp[u], a = fr[u];
                for (uint32_t h = nwh; h-- > nwh - nh;) {
                    if (key - hk[h] > dt) break;
                    if (!adjacent(pix, hp[h])) continue;
                    const uint32_t b = hr[h];
                    if (a == la && b == lb) continue;
                    la = a;
                    lb = b;
                    const uint32_t slot = atomicAdd(&s_ne[warp], 1u);
                    if (slot < (uint32_t)BF_EDGES) {
                        ea[slot] = a;
                        eb[slot] = b;
                    } else {
                        gunion(w.parent, a, b);
                    }
                }
            }
            __syncwarp();
            const uint32_t ne = s_ne[warp] < (uint32_t)BF_EDGES ? s_ne[warp] : BF_EDGES;
            for (uint32_t e = lane; e < ne; e += 32) gunion(w.parent, ea[e], eb[e]);
        } else if (lane == 0) {
            w.border_list[atomicAdd(&w.prob->border_count, 1u)] = t;
        }
        __syncwarp();   // the staging is rewritten for the next border
        if (lane == 0) s_ne[warp] = 0;
        __syncwarp();
    }
}

// The borders k_border_fast listed: halo and front searched block-wide.
__global__ void __launch_bounds__(BORDER_THREADS) k_border_link(Work w) {
    __shared__ uint32_t b_key[HALO_BATCH];
    __shared__ uint32_t b_pix[HALO_BATCH];
    __shared__ uint32_t b_root[HALO_BATCH];
    __shared__ uint32_t b_start[NBUCKETS + 1];
    __shared__ uint32_t b_cur[NBUCKETS];
    __shared__ uint32_t b_warp[32];
    __shared__ uint16_t b_seg[HALO_BATCH];
    const Prob &P = *w.prob;
    const uint32_t nlist = P.border_count;
    const uint32_t *skey = pick(w.keys, sorted_sel(P));
    for (uint32_t u = blockIdx.x; u < nlist; u += gridDim.x) {
        const uint32_t t = w.border_list[u];
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t s0, end;
        tile_range(g, t, s0, end);
        const uint32_t W = g.width, H = g.height, dt = g.dt, cw = (W + 3) >> 2;
        const uint32_t k0 = skey[s0];
        const uint32_t lo_key = k0 >= dt ? k0 - dt : 0;
        const uint64_t hi64 = (uint64_t)skey[s0 - 1] + dt;
        const uint32_t hi_key = hi64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)hi64;
        // halo: [h0, s0) = earlier hits with key >= key(s0) - dt (a suffix)
        uint32_t h0 = s0;
        while (h0 > g.off) {
            const uint32_t chunk = h0 - g.off < BORDER_THREADS ? h0 - g.off : BORDER_THREADS;
            const uint32_t p = h0 - 1 - threadIdx.x;
            const bool in = threadIdx.x < chunk && skey[p] >= lo_key;
            const uint32_t cnt = (uint32_t)__syncthreads_count(in);
            h0 -= cnt;
            if (cnt < chunk) break;
        }
        if (h0 == s0) continue;
        // front: [s0, e0) = tile hits with key <= key(s0 - 1) + dt (a prefix)
        uint32_t e0 = s0;
        while (e0 < end) {
            const uint32_t chunk = end - e0 < BORDER_THREADS ? end - e0 : BORDER_THREADS;
            const uint32_t p = e0 + threadIdx.x;
            const bool in = threadIdx.x < chunk && skey[p] <= hi_key;
            const uint32_t cnt = (uint32_t)__syncthreads_count(in);
            e0 += cnt;
            if (cnt < chunk) break;
        }
        // halo staged in batches with keys, pixels and tile roots; small
        // borders scan every (front, halo) pair within dt, large ones bucket
        // the batch by cell.  Unions join tile roots, skipping a repeat of
        // the thread's previous one.
        const uint32_t nh = s0 - h0, nf = e0 - s0;
        const bool direct = nh * (uint64_t)nf <= BORDER_PAIRS_DIRECT;
        for (uint32_t hb = h0; hb < s0; hb += HALO_BATCH) {
            const uint32_t n_b = s0 - hb < HALO_BATCH ? s0 - hb : HALO_BATCH;
            for (uint32_t j = threadIdx.x; j < n_b; j += BORDER_THREADS) {
                b_key[j] = skey[hb + j];
                b_pix[j] = w.spix[hb + j];
                b_root[j] = w.parent[hb + j];
            }
            __syncthreads();
            if (!direct) bucket_sort(b_pix, n_b, cw, b_start, b_cur, b_seg, b_warp);
            for (uint32_t i = s0 + threadIdx.x; i < e0; i += BORDER_THREADS) {
                const uint32_t key = skey[i], pix = w.spix[i], a = w.parent[i];
                uint32_t lb = 0xFFFFFFFFu;
                if (direct) {   // newest halo hit first
                    for (uint32_t j = n_b; j-- > 0;) {
                        if (key - b_key[j] > dt) break;
                        if (adjacent(pix, b_pix[j]) && b_root[j] != lb) {
                            lb = b_root[j];
                            gunion(w.parent, a, lb);
                        }
                    }
                } else {
                    uint32_t b[4];
                    const int nb = neighbour_buckets(pix, W, H, cw, b);
                    for (int q2 = 0; q2 < nb; ++q2) {
                        for (uint32_t q = b_start[b[q2]]; q < b_start[b[q2] + 1]; ++q) {
                            const uint32_t j = b_seg[q];
                            if (key - b_key[j] <= dt && adjacent(pix, b_pix[j]) && b_root[j] != lb) {
                                lb = b_root[j];
                                gunion(w.parent, a, lb);
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_sorted_roots(Work w) {
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    uint32_t *sroot = pick(w.keys, sorted_sel(P) ^ 1u);   // the idle radix buffer
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        constexpr int ITEMS = TILE / 256;
        uint32_t par[ITEMS], p2[ITEMS];
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {   // every load in flight before any use
            const uint32_t s = begin + q * 256 + threadIdx.x;
            par[q] = s < end ? w.parent[s] : s;
        }
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {   // the second hop for every item at once (most paths end there)
            const uint32_t s = begin + q * 256 + threadIdx.x;
            p2[q] = par[q] != s ? w.parent[par[q]] : s;
        }
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {
            const uint32_t s = begin + q * 256 + threadIdx.x;
            if (s < end) sroot[s] = p2[q] == par[q] ? p2[q] : gfind(w.parent, p2[q]);
        }
    }
}

constexpr int TILE_LINK_SMEM = (3 * TILE + 2 * NBUCKETS + 1 + 32) * (int)sizeof(uint32_t) +
                               TILE * (int)sizeof(uint16_t) +
                               (LINK_THREADS / 32) * EDGE_BUF * (int)sizeof(uint32_t);

cudaError_t init_features_attributes();

cudaError_t init_kernel_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_tile_link, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_LINK_SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tile_link_table, cudaFuncAttributeMaxDynamicSharedMemorySize, TAB_SMEM);
    if (e == cudaSuccess) e = init_features_attributes();
    if (e == cudaSuccess) e = init_variants_attributes();
    return e == cudaSuccess ? init_sortfast_attributes() : e;
}

void launch_tile_border(const Work &w, const Launch &L) {
    const int smem = TILE_LINK_SMEM;
    k_tile_link_table<<<L.fit(k_tile_link_table, TAB_THREADS, TAB_SMEM, G_LINK), TAB_THREADS, TAB_SMEM,
                        L.stream>>>(w);
    L.mark("k_tile_link_table");
    k_tile_link<<<L.fit(k_tile_link, LINK_THREADS, smem, G_LINK), LINK_THREADS, smem, L.stream>>>(w);
    L.mark("k_tile_link");
    k_border_fast<<<L.fit(k_border_fast, BF_WARPS * 32, 0, G_LINK), BF_WARPS * 32, 0, L.stream>>>(w);
    L.mark("k_border_fast");
    k_border_link<<<L.fit(k_border_link, BORDER_THREADS, 0), BORDER_THREADS, 0, L.stream>>>(w);
    L.mark("k_border_link");
}

void launch_sorted_roots(const Work &w, const Launch &L) {
    k_sorted_roots<<<L.fit(k_sorted_roots, 256, 0), 256, 0, L.stream>>>(w);
    L.mark("k_sorted_roots");
}

// After the (b)/(c) merges: zero the feature slot of every root (parent[s]
// == s); k_accumulate finds each position's root itself.
__global__ void __launch_bounds__(256) k_init_roots(Work w) {
    const uint32_t nt = w.prob->ntiles;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        for (uint32_t s = begin + threadIdx.x; s < end; s += blockDim.x)
            if (w.parent[s] == s) init_slot(w, s);
    }
}

void launch_init_roots(const Work &w, const Launch &L) {
    k_init_roots<<<L.fit(k_init_roots, 256, 0), 256, 0, L.stream>>>(w);
    L.mark("k_init_roots");
}

// Tile links and border links; roots are found by k_accumulate.
void launch_link(const Work &w, const Launch &L) {
    launch_tile_border(w, L);
}

}  // namespace tpc
