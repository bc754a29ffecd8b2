// Internal layout shared by the kernels and the host orchestration of libtpc.
//
// Positions.  A processing step clusters one or more independent segments
// (one per sensor / context).  Their hits live in separate input buffers but
// every work array is indexed by a single "position" space in which segment
// s occupies [off, off + n) and off is a multiple of TILE, so that tiles,
// 32-position flag words and warps never straddle two segments.
//
// Within a segment, position p stands for input hit (p - off).  After the
// ToA sort, sorted position s holds the hit whose position is sidx[s]; the
// union-find forest lives on sorted positions and a root is the earliest hit
// of its cluster in (ToA, index) order, the paper's "time invariant"
// toa(h) >= toa(parent(h)) (Section 4.1).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "tpc.h"

namespace tpc {

constexpr int TILE = 4096;          // positions per tile (sort, link, flags)
constexpr int TILE_WORDS = TILE / 32;
constexpr int MAX_SEGS = 256;
constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;
constexpr uint32_t MAX_PIXELS = 1u << 20;   // width*height bound (packed smem keys)

enum ErrBits : uint32_t {
    E_RANGE = 1u,     // hit outside the sensor
    E_SPAN = 2u,      // ToA span of a segment >= 2^32
    E_LATE = 4u,      // streaming: chunk ToA below the last watermark
    E_TIMEOUT = 8u,   // a bounded wait gave up
    E_CAP = 16u,      // internal capacity exceeded
};

// Carried state of a streaming context (device resident across steps).
struct StreamState {
    uint32_t n_carry;         // open hits carried into the next step
    uint32_t has_seen;        // seen_max is valid
    uint64_t seen_max;        // max ToA over all pushed hits
    uint64_t watermark;       // clusters with last ToA <= watermark are final
};

enum CloseMode : uint32_t { CLOSE_NONE = 0, CLOSE_ALL = 1, CLOSE_WM = 2 };

struct Seg {
    // ---- set by the host ----------------------------------------------
    const tpc_hit *hits;       // input hits [0, n); for streaming: set on device
    const tpc_hit *carry_in;   // streaming: buffer whose [cap - n_carry, cap) holds the carry
    const uint64_t *carry_gidx_in;
    tpc_hit *carry_out;        // streaming: next step's buffer (carry written right aligned)
    uint64_t *carry_gidx_out;
    StreamState *ss;           // streaming state, null when not streaming
    uint64_t *out_labels;      // finalised labels (u64), ordered by global index
    uint64_t *out_index;       // their global indices (streaming only; may be null)
    tpc_cluster *out_rec;      // finalised cluster records ordered by label
    uint64_t gidx_base;        // global index of the first new hit
    uint64_t max_disorder;     // UINT64_MAX: not streaming (everything closes)
    uint32_t carry_cap;        // streaming: capacity of the carry region
    uint32_t n_new;            // hits pushed in this step
    uint32_t width, height;
    uint32_t dt;               // time window, clamped to 32 bits
    uint32_t variant;
    uint32_t out_cap;          // capacity of out_labels/out_index and out_rec
    uint32_t close_mode;       // CloseMode, derived on the device
    // ---- derived on the device ------------------------------------------
    const uint64_t *carry_gidx;  // global indices of hits [0, n_carry)
    uint32_t n_carry;
    uint32_t n;                // n_carry + n_new
    uint32_t off;              // first position
    uint32_t tile0, ntiles;
    uint32_t npasses;          // radix passes this segment needs
    uint64_t toa_min, toa_max;
    uint64_t key_base;         // sort keys are ToA - key_base (32 bits)
    uint64_t fast_base;        // the tile sort's key base (fast_key_base, set by k_setup)
    uint64_t chunk_min;        // min ToA of the new hits
    uint64_t watermark;        // CLOSE_WM: close clusters whose last ToA <= watermark
    uint64_t seen_after;       // streaming: max ToA seen after this step
    // ---- outputs -------------------------------------------------------
    uint32_t n_final;          // hits finalised
    uint32_t n_clusters;       // clusters finalised
    uint32_t n_open;           // hits carried forward
    uint32_t link_general;     // set by the host (a tuning choice): link every tile with
                               // k_tile_link instead of the shared-memory table kernel
};

struct Prob {
    uint32_t nsegs;
    uint32_t ntiles;
    uint32_t npasses;      // radix passes run; sorted data in buffer npasses % 2
    uint32_t err;          // ErrBits
    uint32_t tile_cap;
    uint32_t pos_cap;
    uint32_t fallback;     // the tile sort + merge did not order the input: radix sort
    uint32_t lsd_passes;   // passes the radix sort needs (max over segments)
    uint32_t redo_count;   // tiles the table-mode link left to the general link kernel
    uint32_t border_count; // tile borders k_border_fast left to k_border_link
    uint32_t merge_count;  // tile borders k_tile_merge left to its whole-window form (listed in redo)
};

// Feature sums of one cluster, kept at its root's sorted position.  One
// 40-byte record (8-byte aligned, so exactly two 32-byte sectors) instead of
// six arrays: the scattered per-root accesses touch 2 sectors, not 6.
struct Slot {
    unsigned long long tot, wx, wy;   // sum ToT, sum ToT*x, sum ToT*y
    uint32_t size;
    uint32_t min;                     // smallest position
    uint32_t maxkey;                  // largest key (last ToA - toa_min)
    uint32_t pad;
};
static_assert(sizeof(Slot) == 40, "slot layout");

// Work arrays (device), sized for pos_cap positions and tile_cap tiles.
struct Work {
    Seg *seg;
    Prob *prob;
    uint32_t *tile_seg;        // [tile_cap]
    uint32_t *border_list;     // [tile_cap] tiles whose border needs the block-wide search
    uint32_t *redo;            // [tile_cap] tiles handed from table mode to k_tile_link
    uint32_t *keys[2];         // radix ping-pong: ToA - toa_min
    uint32_t *vals[2];         // radix ping-pong: position
    uint32_t *spix;            // sorted positions: x | y << 16
    uint16_t *stot;            // sorted positions: ToT
    uint32_t *parent;          // union-find over sorted positions
    uint32_t *root_of;         // per position: root (a sorted position)
    Slot *slot;                // per root: its cluster's features
    uint64_t *lab_tmp;         // streaming: label per position
    uint32_t *flag_label;      // bit per position: label hit of a finalised cluster
    uint32_t *flag_closed;     // bit per position: hit of a finalised cluster
    uint32_t *tile_cnt;        // [2][tile_cap] counts of the two flag kinds
    uint32_t *tile_base;       // [2][tile_cap] exclusive per-segment prefix
    uint32_t *hist;            // [RADIX][tile_cap]
    uint32_t *segtot;          // [MAX_SEGS][RADIX]
};

// Extra arrays of the (b)/(c) variants (single-segment steps only).
struct VarWork {
    uint32_t *k[2], *v[2];     // grouping radix sort: keys / sorted positions
    uint32_t *cpar;            // (c): forest over the root-grouped order
    uint32_t *pix_start;       // (b): per pixel, start of its timeline (W*H + 1)
    uint32_t *tcnt, *tbase;    // (b): (a) components per tile and their exclusive prefix
    uint32_t *ncomp;           // (b): number of (a) components (dense ids 0 .. ncomp - 1)
    uint32_t *cid_at;          // (b): per sorted position that is an (a) root: its dense id
    uint32_t *croot;           // (b): per dense id: the root's sorted position
    uint32_t *cpar_d;          // (b): forest over dense ids (a group's root: its smallest id)
    uint32_t *clast0, *clast;  // (b): per dense id: its component's last key; at a group's root, the group's
    uint4 *pstate, *tline;     // (b): before a full round, per sorted position and per pixel-timeline
                               //      entry: (sorted position, id of its group's root, the group's last
                               //      key, its key)
    uint32_t *changed;         // (b): [0] a round merged something, [1] the edge list overflowed;
                               // (c): [0] windowed components, [1] of those swept again by a CTA,
                               //      [2] of those swept from global memory
    unsigned long long *ecount;  // (b): edges pushed to lists 0 and 1 (beyond edge_cap: overflow)
    uint2 *edges[2];           // (b): edges not merged yet (an id of h's group, an id of its neighbour's)
    uint32_t *ekey[2];         // (b): h's key of each edge
    uint32_t edge_cap;         // (b): entries each edge list holds
    uint32_t *work;            // (c): next chunk of the grouped order to sweep
    uint2 *big;                // (c): (first grouped position, hits) of components for the big window
    Prob *prob;                // problem view of the grouping sort
};

// ---------------------------------------------------------------------------
// device helpers

__device__ __forceinline__ uint32_t seg_of_tile(const Work &w, uint32_t t) { return w.tile_seg[t]; }

__device__ __forceinline__ void tile_range(const Seg &s, uint32_t t, uint32_t &begin, uint32_t &end) {
    begin = s.off + (t - s.tile0) * (uint32_t)TILE;
    uint32_t e = begin + (uint32_t)TILE, last = s.off + s.n;
    end = e < last ? e : last;
}

__device__ __forceinline__ uint64_t gidx_of(const Seg &s, uint32_t local) {
    return local < s.n_carry ? s.carry_gidx[local] : s.gidx_base + (local - s.n_carry);
}

__device__ __forceinline__ uint32_t sorted_sel(const Prob &p) { return p.npasses & 1u; }

// One of a pair of buffers by a runtime bit, as a select: indexing a kernel
// parameter's array with a runtime value would copy the parameter to local
// memory.
template <class T>
__device__ __forceinline__ T *pick(T *const (&a)[2], uint32_t sel) { return sel ? a[1] : a[0]; }

// Zero the feature slot of root r (a tile root; every global root is one).
__device__ __forceinline__ void init_slot(const Work &w, uint32_t r) {
    unsigned long long *q = reinterpret_cast<unsigned long long *>(w.slot + r);
    q[0] = 0;
    q[1] = 0;
    q[2] = 0;
    q[3] = 0xFFFFFFFF00000000ull;   // size = 0, min = all ones
    q[4] = 0;                       // maxkey = 0
}

// Union-find on global memory over sorted positions.  Roots are the smaller
// position (hook the larger root under the smaller, Jaiganesh & Burtscher,
// "A high-performance connected components implementation for GPUs", 2018);
// path halving on every find.
__device__ __forceinline__ uint32_t gfind(uint32_t *parent, uint32_t x) {
    volatile uint32_t *par = parent;
    while (true) {
        uint32_t p = par[x];
        if (p == x) return x;
        uint32_t gp = par[p];
        if (gp == p) return p;
        par[x] = gp;
        x = gp;
    }
}

__device__ __forceinline__ void gunion(uint32_t *parent, uint32_t a, uint32_t b) {
    while (true) {
        a = gfind(parent, a);
        b = gfind(parent, b);
        if (a == b) return;
        if (a > b) { uint32_t t = a; a = b; b = t; }
        uint32_t old = atomicCAS(parent + b, b, a);
        if (old == b) return;
    }
}

__device__ __forceinline__ uint32_t sfind(uint32_t *parent, uint32_t x) {
    volatile uint32_t *par = parent;
    while (true) {
        uint32_t p = par[x];
        if (p == x) return x;
        uint32_t gp = par[p];
        if (gp == p) return p;
        par[x] = gp;
        x = gp;
    }
}

__device__ __forceinline__ void sunion(uint32_t *parent, uint32_t a, uint32_t b) {
    while (true) {
        a = sfind(parent, a);
        b = sfind(parent, b);
        if (a == b) return;
        if (a > b) { uint32_t t = a; a = b; b = t; }
        uint32_t old = atomicCAS(parent + b, b, a);
        if (old == b) return;
    }
}

__device__ __forceinline__ uint4 ld_hit(const tpc_hit *h) {
    return __ldg(reinterpret_cast<const uint4 *>(h));
}
__device__ __forceinline__ uint32_t hit_x(uint4 v) { return v.x & 0xFFFFu; }
__device__ __forceinline__ uint32_t hit_y(uint4 v) { return v.x >> 16; }
__device__ __forceinline__ uint32_t hit_tot(uint4 v) { return v.y & 0xFFFFu; }
__device__ __forceinline__ uint64_t hit_toa(uint4 v) { return ((uint64_t)v.w << 32) | v.z; }

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
    for (int o = 16; o; o >>= 1) {
        uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}
__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
    for (int o = 16; o; o >>= 1) {
        uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}

// Key base of the tile sort, known before any pass over the hits: 2^31 ticks
// before the segment's first hit.  Its keys are exact when every ToA lies
// within 2^31 ticks of that hit (checked once the extremes are known; the
// general sort, with base = minimum ToA, takes over otherwise).
__device__ __forceinline__ uint64_t fast_key_base(const Seg &g) {
    const uint64_t t0 = g.n ? hit_toa(ld_hit(g.hits)) : 0;
    return t0 > (1ull << 31) ? t0 - (1ull << 31) : 0;
}

// Pixel clamped into the sensor.  The tile sort reports hits outside it
// (E_RANGE) but the step still runs to its end, and the link kernels index
// per-pixel tables with the sorted pixels, so the sorts store them clamped.
__device__ __forceinline__ uint32_t clamp_pix(uint32_t pix, uint32_t W, uint32_t H) {
    uint32_t x = pix & 0xFFFFu, y = pix >> 16;
    x = x < W ? x : W - 1;
    y = y < H ? y : H - 1;
    return x | y << 16;
}

// ---------------------------------------------------------------------------
// host-side launchers (one translation unit each)

// Optional per-kernel tracing: an event after every launch.
struct Tracer {
    static constexpr int MAX = 64;
    cudaEvent_t ev[MAX + 1];
    const char *names[MAX];
    int n = 0;
    void mark(const char *name, cudaStream_t st) {
        if (n < MAX) {
            names[n] = name;
            cudaEventRecord(ev[++n], st);
        }
    }
};

// CTAs of `kernel` one SM holds at once with this block size and dynamic
// shared memory (registers included); cached per device.
int occupancy(const void *kernel, int threads, size_t smem);

// Launch choices a tuner may change (tpc_tuning at the ABI): CTAs per SM of
// each group of persistent kernels and the feature kernel's span.  Results
// never depend on them.
enum TuneGroup { G_SORT = 0, G_LINK = 1, G_ACC = 2, G_OUT = 3, NGROUPS = 4 };
struct Tuning {
    uint8_t cap[NGROUPS] = {0, 0, 0, 0};   // CTAs per SM per group, 0 = as many as fit
    uint16_t acc_span = 1024;              // k_accumulate positions per pass: 512, 1024, 2048
    uint8_t general_link = 0;              // bit 0: single-band sensors, bit 1: banded sensors
                                           // take k_tile_link instead of the table kernel
    uint8_t order = 0;                     // 1: batch segments largest first
};

struct Launch {
    int grid;          // fallback grid when the SM count is unknown
    cudaStream_t stream;
    Tracer *tr = nullptr;
    int sms = 0;       // SM count
    int cap = 0;       // at most this many CTAs per SM (0 = as many as fit)
    Tuning tune{};
    void mark(const char *name) const { if (tr) tr->mark(name, stream); }
    // Grid of a persistent kernel (a strided loop over tiles): exactly one
    // wave, every SM filled to the kernel's occupancy (or to its group's
    // tuned cap).  A grid that is not a whole multiple of the resident CTAs
    // would leave a partial second wave running on a fraction of each SM.
    template <class K>
    int fit(K *kernel, int threads, size_t smem, int group = -1) const {
        if (sms <= 0) return grid;
        int per_sm = occupancy(reinterpret_cast<const void *>(kernel), threads, smem);
        if (cap > 0 && per_sm > cap) per_sm = cap;
        if (group >= 0 && tune.cap[group] > 0 && per_sm > tune.cap[group]) per_sm = tune.cap[group];
        return sms * (per_sm > 0 ? per_sm : 1);
    }
};

cudaError_t init_kernel_attributes();   // once per process and device, before capture
cudaError_t init_variants_attributes();
void launch_setup(const Work &w, int nsegs, const Launch &L);
void launch_seg_finalize(const Work &w, const Launch &L);
void launch_make_keys(const Work &w, const Launch &L);
void launch_sort_fast(const Work &w, const Launch &L);
cudaError_t init_sortfast_attributes();
void launch_radix_pass(const Work &w, int pass, const Launch &L);
void launch_gather(const Work &w, const Launch &L);
void launch_link(const Work &w, const Launch &L);          // tile + border links
void launch_tile_border(const Work &w, const Launch &L);
int link_bands(uint32_t W, uint32_t H);   // table bands of a sensor, 0 = general link kernel
void launch_sorted_roots(const Work &w, const Launch &L);
void launch_init_roots(const Work &w, const Launch &L);
void launch_variant_keys(const Work &w, const VarWork &v, int by_pixel, const Launch &L);
Work variant_view(const Work &w, const VarWork &v);
void launch_static_sweep(const Work &w, const VarWork &v, const Launch &L);
void launch_pixel_timelines(const Work &w, const VarWork &v, uint32_t npixels, const Launch &L);
void launch_components(const Work &w, const VarWork &v, const Launch &L);
void launch_group_last(const VarWork &v, const Launch &L);
void launch_comp_parents(const Work &w, const VarWork &v, const Launch &L);
void launch_global_edges(const Work &w, const VarWork &v, int full, int flat, int in_list, const Launch &L);
void launch_features(const Work &w, const Launch &L);
void launch_outputs(const Work &w, const Launch &L);

}  // namespace tpc
