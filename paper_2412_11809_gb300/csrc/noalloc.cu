// tpc_cluster_static: one-shot clustering of a small batch of hits that
// allocates nothing.
//
// Some callers cannot call cudaMalloc: real-time readout loops that must not
// block (cudaMalloc can synchronise the device and take unbounded time), and
// code that runs under a fixed memory plan, such as a host framework that
// reserved the device memory up front and hands out only buffers from its
// own pool.  They hand over device buffers for the inputs and outputs; the
// working memory comes from the fixed array below, which every GPU that
// loads the library holds until the process exits.
//
// The kernels are the library's own (the same launch sequence as
// tpc_flush); only the source of their scratch differs.  Every call shares
// the one array and leaves its last contents behind: nothing in it has to
// start at zero, because each call first rewrites the segment and problem
// descriptors and every other array is fully written before it is read.
// Calls whose work overlaps on the GPU (different streams, or different
// threads without ordering) race on the array and give wrong results;
// order them on one stream.
#include <mutex>

#include "tpc_internal.cuh"

namespace tpc {
namespace {

constexpr uint32_t NA_MAX = TPC_STATIC_MAX_HITS;   // one segment, tiles of TILE
constexpr uint32_t NA_POS = NA_MAX;
constexpr uint32_t NA_TILES = NA_POS / TILE;
static_assert(NA_MAX % TILE == 0, "whole tiles");

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// byte offsets of every work array inside the scratch array
struct Layout {
    size_t seg, prob, tile_seg, redo, border_list, keys0, keys1, vals0, vals1, spix, stot, parent, root_of,
        slot, flag_label, flag_closed,
        tile_cnt, tile_base, hist, segtot, total;
};

constexpr Layout make_layout() {
    Layout l{};
    size_t o = 0;
    l.seg = o; o += align256(sizeof(Seg));
    l.prob = o; o += align256(sizeof(Prob));
    l.tile_seg = o; o += align256(NA_TILES * 4);
    l.redo = o; o += align256(NA_TILES * 4);
    l.border_list = o; o += align256(NA_TILES * 4);
    l.keys0 = o; o += align256(NA_POS * 4);
    l.keys1 = o; o += align256(NA_POS * 4);
    l.vals0 = o; o += align256(NA_POS * 4);
    l.vals1 = o; o += align256(NA_POS * 4);
    l.spix = o; o += align256(NA_POS * 4);
    l.stot = o; o += align256(NA_POS * 2);
    l.parent = o; o += align256(NA_POS * 4);
    l.root_of = o; o += align256(NA_POS * 4);
    l.slot = o; o += align256(NA_POS * sizeof(Slot));
    l.flag_label = o; o += align256((NA_POS / 32 + 1) * 4);
    l.flag_closed = o; o += align256((NA_POS / 32 + 1) * 4);
    l.tile_cnt = o; o += align256(2 * NA_TILES * 4);
    l.tile_base = o; o += align256(2 * NA_TILES * 4);
    l.hist = o; o += align256((size_t)RADIX * NA_TILES * 4);
    l.segtot = o; o += align256((size_t)MAX_SEGS * RADIX * 4);
    l.total = o;
    return l;
}

constexpr Layout NA = make_layout();

// The scratch.  In host code this name is only a stand-in for the device
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char na_scratch[NA.total];

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mu;
void *na_ptr[NA_MAX_DEVICES] = {};
int na_sms[NA_MAX_DEVICES] = {};

// Per device, once, with that device current: the scratch's device address,
// the SM count and the kernels' shared-memory limits.
int na_setup(int dev, unsigned char **base, int *sms) {
    std::lock_guard<std::mutex> lk(na_mu);
    if (!na_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || !p) return TPC_ERR_CUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TPC_ERR_CUDA;
        if (init_kernel_attributes() != cudaSuccess) return TPC_ERR_CUDA;
        na_sms[dev] = n > 0 ? n : 1;
        na_ptr[dev] = p;
    }
    *base = static_cast<unsigned char *>(na_ptr[dev]);
    *sms = na_sms[dev];
    return TPC_OK;
}

__global__ void k_na_begin(Work w, Seg s, uint32_t tile_cap, uint32_t pos_cap) {
    w.seg[0] = s;
    Prob p{};
    p.tile_cap = tile_cap;
    p.pos_cap = pos_cap;
    *w.prob = p;
}

// counts[1] keeps the public bits only (TPC_STATIC_E_*); with no record
// buffer (record_cap == 0) the caller asked for labels alone, so more
// clusters than records is not an error then.
__global__ void k_na_end(Work w, uint64_t *counts, uint32_t keep) {
    counts[0] = w.seg[0].n_clusters;
    counts[1] = w.prob->err & keep;
}

__global__ void k_na_empty(uint64_t *counts) {
    counts[0] = 0;
    counts[1] = 0;
}

}  // namespace
}  // namespace tpc

using namespace tpc;

extern "C" int tpc_cluster_static(const tpc_hit *hits, size_t n, uint32_t width, uint32_t height,
                                  uint64_t dt, uint64_t *labels, tpc_cluster *records,
                                  size_t record_cap, uint64_t *counts, void *stream) {
    if (n > NA_MAX) return TPC_ERR_ARG;   // larger batches need tpc_create/tpc_flush
    if (!counts || (n && (!hits || !labels || (record_cap && !records)))) return TPC_ERR_ARG;
    if (width == 0 || height == 0 || width > 65536 || height > 65536 ||
        (uint64_t)width * height > MAX_PIXELS)
        return TPC_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n == 0) {
        k_na_empty<<<1, 1, 0, st>>>(counts);
        return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return TPC_ERR_CUDA;
    unsigned char *base = nullptr;
    int sms = 1;
    int rc = na_setup(dev, &base, &sms);
    if (rc) return rc;

    Work w{};
    w.seg = reinterpret_cast<Seg *>(base + NA.seg);
    w.prob = reinterpret_cast<Prob *>(base + NA.prob);
    w.tile_seg = reinterpret_cast<uint32_t *>(base + NA.tile_seg);
    w.redo = reinterpret_cast<uint32_t *>(base + NA.redo);
    w.border_list = reinterpret_cast<uint32_t *>(base + NA.border_list);
    w.keys[0] = reinterpret_cast<uint32_t *>(base + NA.keys0);
    w.keys[1] = reinterpret_cast<uint32_t *>(base + NA.keys1);
    w.vals[0] = reinterpret_cast<uint32_t *>(base + NA.vals0);
    w.vals[1] = reinterpret_cast<uint32_t *>(base + NA.vals1);
    w.spix = reinterpret_cast<uint32_t *>(base + NA.spix);
    w.stot = reinterpret_cast<uint16_t *>(base + NA.stot);
    w.parent = reinterpret_cast<uint32_t *>(base + NA.parent);
    w.root_of = reinterpret_cast<uint32_t *>(base + NA.root_of);
    w.slot = reinterpret_cast<Slot *>(base + NA.slot);
    w.lab_tmp = nullptr;   // streaming only
    w.flag_label = reinterpret_cast<uint32_t *>(base + NA.flag_label);
    w.flag_closed = reinterpret_cast<uint32_t *>(base + NA.flag_closed);
    w.tile_cnt = reinterpret_cast<uint32_t *>(base + NA.tile_cnt);
    w.tile_base = reinterpret_cast<uint32_t *>(base + NA.tile_base);
    w.hist = reinterpret_cast<uint32_t *>(base + NA.hist);
    w.segtot = reinterpret_cast<uint32_t *>(base + NA.segtot);

    Seg s{};
    s.hits = hits;
    s.out_labels = labels;
    s.out_rec = records;
    s.out_cap = (uint32_t)(record_cap < NA_MAX ? record_cap : NA_MAX);
    s.gidx_base = 0;
    s.max_disorder = ~0ull;
    s.n_new = (uint32_t)n;
    s.width = width;
    s.height = height;
    s.dt = dt > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)dt;
    s.variant = TPC_LOCAL;

    const Launch L{sms * 4, st, nullptr, sms};
    k_na_begin<<<1, 1, 0, st>>>(w, s, NA_TILES, NA_POS);
    launch_setup(w, 1, L);
    launch_sort_fast(w, L);
    launch_seg_finalize(w, L);
    launch_make_keys(w, L);
    for (int pass = 0; pass < 4; ++pass) launch_radix_pass(w, pass, L);
    launch_gather(w, L);
    launch_link(w, L);
    launch_features(w, L);
    launch_outputs(w, L);
    static_assert(E_RANGE == TPC_STATIC_E_RANGE && E_SPAN == TPC_STATIC_E_SPAN && E_CAP == TPC_STATIC_E_CAP,
                  "public error bits");
    const uint32_t keep = TPC_STATIC_E_RANGE | TPC_STATIC_E_SPAN | (record_cap ? TPC_STATIC_E_CAP : 0u);
    k_na_end<<<1, 1, 0, st>>>(w, counts, keep);
    return cudaGetLastError() == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}
