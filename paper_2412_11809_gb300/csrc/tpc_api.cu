// C ABI of libtpc: contexts, device memory, the launch sequence of one
// processing step, streaming carry, batching and CUDA-graph replay.
//
// A processing step (tpc_flush, a streaming tpc_push, or tpc_batch_flush)
// enqueues the same fixed kernel sequence on one CUDA stream:
//   setup -> tile sort -> tile merge -> sort check -> segment finalize ->
//   (general-order fallback: keys -> radix passes 0..3 -> gather) ->
//   table link -> tile link (redo tiles) -> border fast -> border link ->
//   accumulate (finds the roots) -> labels -> tile scan -> records ->
//   stream compact -> stream end.
// Streaming contexts also checkpoint and restore their open state here
// (tpc_snapshot / tpc_restore).
// Every size the kernels need is read from device memory and every kernel is
// a persistent grid over (segment, tile) work items, so no step waits for the
// host and the sequence is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ctx_internal.h"
#include "tpc_internal.cuh"

using namespace tpc;

namespace {

constexpr int SEG_RING = 8;

// occupancy(): cudaOccupancyMaxActiveBlocksPerMultiprocessor, remembered per
// (device, kernel, block size, shared memory) so that launches and graph
// captures do not repeat the query.
struct OccEntry {
    int dev;
    const void *kernel;
    int threads;
    size_t smem;
    int blocks;
};
std::mutex occ_mu;
std::vector<OccEntry> occ_cache;


// Device memory of every context comes from one stream-ordered pool per
// device (cudaMallocFromPoolAsync / cudaFreeAsync on the context's stream).
// Growing or dropping one context's arrays is ordered after that context's
// own queued work and never synchronises the device, so contexts serving
// other streams keep running.  The pool keeps up to POOL_KEEP bytes of freed
// memory for reuse instead of returning it to the driver.
constexpr int MAX_DEVICES = 64;
constexpr uint64_t POOL_KEEP = 8ull << 30;
std::mutex pool_mu;
cudaMemPool_t pools[MAX_DEVICES] = {};

cudaMemPool_t device_pool(int dev) {
    if (dev < 0 || dev >= MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lk(pool_mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        uint64_t keep = POOL_KEEP;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

// Every allocation of a context goes through these two.  `fault` is the
// context's TPC_OPT_FAIL_ALLOC countdown (a test hook): while positive it
// counts the allocations still to succeed, and the one that brings it to
// zero fails as an out-of-memory would, without calling CUDA.
bool injected_failure(int64_t *fault) { return fault && *fault > 0 && --*fault == 0; }

// Device memory, usable by work queued on `st` after this call (and by other
// streams once they wait for `st`).
cudaError_t dev_alloc(int64_t *fault, void **p, size_t bytes, cudaStream_t st, int dev) {
    *p = nullptr;
    if (injected_failure(fault)) return cudaErrorMemoryAllocation;
    cudaMemPool_t pool = device_pool(dev);
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

// Free after the work already queued on `st` (which must include every use).
void dev_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

cudaError_t host_alloc(int64_t *fault, void **p, size_t bytes) {
    *p = nullptr;
    if (injected_failure(fault)) return cudaErrorMemoryAllocation;
    return cudaMallocHost(p, bytes);
}

struct DevMem {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    int64_t *fault = nullptr;
    cudaStream_t stream = nullptr;   // the owning context's stream
    int dev = 0;
    template <class T>
    T *alloc(size_t count, cudaError_t &err) {
        void *p = nullptr;
        if (err != cudaSuccess) return nullptr;
        size_t b = std::max<size_t>(count, 1) * sizeof(T);
        b = (b + 255) & ~size_t(255);
        err = dev_alloc(fault, &p, b, stream, dev);
        if (err != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        bytes += b;
        return static_cast<T *>(p);
    }
    void release() {
        for (void *p : ptrs) dev_free(p, stream);
        ptrs.clear();
        bytes = 0;
    }
};

// Device work arrays for up to pos_cap positions in up to seg_cap segments.
struct Workspace {
    size_t pos_cap = 0, tile_cap = 0;
    uint64_t gen = 0;   // bumped by every (re)allocation: a graph captured on older arrays is stale
    Work w{};
    DevMem mem;

    size_t alloc_need = 0;   // positions the arrays were sized for (whole tiles, spare tile excluded)

    static size_t round_tiles(size_t positions) {
        return std::max<size_t>(((positions + TILE - 1) / TILE) * TILE, TILE);
    }

    // Positions ensure(positions) sizes the arrays for: the need itself on
    // the first allocation; on growth at least double the old size (at most
    // 2^26 positions more), so that a sequence of growing steps regrows, and
    // re-captures its graph, only a few times.
    size_t grown(size_t positions) const {
        const size_t need = round_tiles(positions);
        if (!w.seg || !alloc_need) return need;
        if (need <= alloc_need) return alloc_need;
        return std::max(need, round_tiles(std::min(2 * alloc_need, alloc_need + (size_t(1) << 26))));
    }

    // Bytes of the arrays for `need` positions (the same arrays ensure()
    // allocates, each rounded up to 256 bytes as DevMem does).
    static size_t bytes_for_need(size_t need) {
        const size_t P = need + TILE, T = need / TILE + MAX_SEGS;
        auto r = [](size_t count, size_t size) { return ((std::max<size_t>(count, 1) * size) + 255) & ~size_t(255); };
        return r(MAX_SEGS, sizeof(Seg)) + r(1, sizeof(Prob)) + 3 * r(T, 4) + 5 * r(P, 4) + r(P, 2) +
               2 * r(P, 4) + r(P, sizeof(Slot)) + r(P, 8) + 2 * r(P / 32 + 1, 4) + 2 * r(2 * T, 4) +
               r((size_t)RADIX * T, 4) + r((size_t)MAX_SEGS * RADIX, 4);
    }

    // Bytes held once ensure(positions) has run.
    size_t bytes_after(size_t positions) const {
        const size_t need = grown(positions);
        return w.seg && need == alloc_need ? mem.bytes : bytes_for_need(need);
    }

    cudaError_t ensure(size_t positions) {
        size_t need = grown(positions);
        if (w.seg && need == alloc_need) return cudaSuccess;
        mem.release();   // freed after the steps already queued on the owner's stream
        alloc_need = need;
        pos_cap = need;
        tile_cap = need / TILE + MAX_SEGS;   // segments pad to whole tiles
        // segments are laid out on whole tiles, so `need` (a sum of whole
        // tiles) covers every position a step uses; one spare tile
        const size_t P = pos_cap + TILE, T = tile_cap;
        pos_cap = P;
        cudaError_t e = cudaSuccess;
        w.seg = mem.alloc<Seg>(MAX_SEGS, e);
        w.prob = mem.alloc<Prob>(1, e);
        w.tile_seg = mem.alloc<uint32_t>(T, e);
        w.redo = mem.alloc<uint32_t>(T, e);
        w.border_list = mem.alloc<uint32_t>(T, e);
        w.keys[0] = mem.alloc<uint32_t>(P, e);
        w.keys[1] = mem.alloc<uint32_t>(P, e);
        w.vals[0] = mem.alloc<uint32_t>(P, e);
        w.vals[1] = mem.alloc<uint32_t>(P, e);
        w.spix = mem.alloc<uint32_t>(P, e);
        w.stot = mem.alloc<uint16_t>(P, e);
        w.parent = mem.alloc<uint32_t>(P, e);
        w.root_of = mem.alloc<uint32_t>(P, e);
        w.slot = mem.alloc<Slot>(P, e);
        w.lab_tmp = mem.alloc<uint64_t>(P, e);
        w.flag_label = mem.alloc<uint32_t>(P / 32 + 1, e);
        w.flag_closed = mem.alloc<uint32_t>(P / 32 + 1, e);
        w.tile_cnt = mem.alloc<uint32_t>(2 * T, e);
        w.tile_base = mem.alloc<uint32_t>(2 * T, e);
        w.hist = mem.alloc<uint32_t>((size_t)RADIX * T, e);
        w.segtot = mem.alloc<uint32_t>((size_t)MAX_SEGS * RADIX, e);
        if (e == cudaSuccess) {
            Prob p{};
            p.tile_cap = (uint32_t)T;
            p.pos_cap = (uint32_t)P;
            e = cudaMemcpyAsync(w.prob, &p, sizeof(Prob), cudaMemcpyHostToDevice, mem.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(mem.stream);   // &p is on this stack
        }
        if (e != cudaSuccess) {
            mem.release();
            w = Work{};
            pos_cap = tile_cap = alloc_need = 0;
        }
        ++gen;
        return e;
    }
};

// Arrays of the (b)/(c) variants, allocated on first use: the grouping
// sort's for both, then each variant's own.
struct VarSpace {
    VarWork v{};
    DevMem mem;
    size_t pos_cap = 0, pixels = 0;
    cudaError_t ensure(size_t positions, size_t npixels, bool global) {
        if (v.k[0] && positions <= pos_cap && npixels <= pixels) return cudaSuccess;
        mem.release();
        v = VarWork{};
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < 2; ++i) {
            v.k[i] = mem.alloc<uint32_t>(positions, e);
            v.v[i] = mem.alloc<uint32_t>(positions, e);
        }
        v.changed = mem.alloc<uint32_t>(4, e);
        v.prob = mem.alloc<Prob>(1, e);
        if (global) {
            const size_t tiles = positions / TILE + 2;
            v.pix_start = mem.alloc<uint32_t>(npixels + 1, e);
            v.tcnt = mem.alloc<uint32_t>(tiles, e);
            v.tbase = mem.alloc<uint32_t>(tiles, e);
            v.ncomp = mem.alloc<uint32_t>(1, e);
            v.cid_at = mem.alloc<uint32_t>(positions, e);
            v.croot = mem.alloc<uint32_t>(positions, e);
            v.cpar_d = mem.alloc<uint32_t>(positions, e);
            v.clast0 = mem.alloc<uint32_t>(positions, e);
            v.clast = mem.alloc<uint32_t>(positions, e);
            v.pstate = mem.alloc<uint4>(positions, e);
            v.tline = mem.alloc<uint4>(positions, e);
            v.ecount = mem.alloc<unsigned long long>(2, e);
            // open edges: 2 per position per list (the first round of the
            // 2.5 Ghits/s Timepix4 stream leaves 0.64 per hit open, later
            // rounds fewer); a round that finds more marks the overflow and
            // the next round reads every hit's 9 again
            v.edge_cap = (uint32_t)std::min<size_t>(2 * positions, 0xFFFFFFFFull);
            for (int i = 0; i < 2; ++i) {
                v.edges[i] = mem.alloc<uint2>(v.edge_cap, e);
                v.ekey[i] = mem.alloc<uint32_t>(v.edge_cap, e);
            }
        } else {
            v.cpar = mem.alloc<uint32_t>(positions, e);
            v.work = mem.alloc<uint32_t>(1, e);
            v.big = mem.alloc<uint2>(positions / 512 + 1, e);   // components of more than 512 hits
        }
        if (e != cudaSuccess) {
            mem.release();
            v = VarWork{};
            pos_cap = pixels = 0;
            return e;
        }
        pos_cap = positions;
        pixels = npixels;
        return cudaSuccess;
    }
};

int num_sms(int dev) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

int map_err(uint32_t bits) {
    if (bits & E_RANGE) return TPC_ERR_RANGE;
    if (bits & E_SPAN) return TPC_ERR_SPAN;
    if (bits & E_TIMEOUT) return TPC_ERR_TIMEOUT;
    if (bits & E_CAP) return TPC_ERR_NOMEM;
    if (bits & E_LATE) return TPC_ERR_LATE;
    return TPC_OK;
}

__global__ void k_iota_u64(uint64_t *out, uint64_t base, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = base + i;
}

}  // namespace

struct tpc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint32_t width = 0, height = 0, dt32 = 0;
    uint64_t dt = 0;
    int variant = 0;
    uint64_t max_disorder = ~0ull;
    uint64_t budget = 0;
    int ctas_per_sm = 0;
    int sms = 1;
    int64_t fail_alloc = 0;        // TPC_OPT_FAIL_ALLOC countdown (0: off)

    // non-streaming pending hits
    const tpc_hit *zc = nullptr;   // zero-copy: one device push
    size_t pending = 0;
    tpc_hit *in = nullptr;         // materialised pending hits
    size_t in_cap = 0;
    uint64_t pushed = 0;           // global index of the next pushed hit
    uint64_t base = 0;             // global index of the first pending hit

    // streaming buffers: [carry_cap | chunk_cap] each, double buffered
    tpc_hit *sbuf[2] = {nullptr, nullptr};
    uint64_t *sgidx[2] = {nullptr, nullptr};
    size_t carry_cap = 0, chunk_cap = 0;
    int scur = 1;
    size_t carry_ub = 0;           // upper bound on the device-side carry count
    StreamState *ss = nullptr;

    Workspace ws;
    VarSpace vs;                   // variants (b), (c)
    uint32_t *h_flag = nullptr;    // pinned: (b) round result ([0..1]) and list size ([2..3]); (c) counters
    DevMem outmem;                 // output buffers
    uint64_t *d_labels = nullptr, *d_index = nullptr;
    tpc_cluster *d_rec = nullptr;
    // caller device buffers one-shot steps write into (tpc_bind_outputs)
    uint64_t *bound_labels = nullptr;
    tpc_cluster *bound_rec = nullptr;
    size_t bound_cap = 0;
    // where the last step's labels and records are
    uint64_t *res_labels = nullptr;
    tpc_cluster *res_rec = nullptr;
    size_t out_cap = 0;

    // where the last step's results live: the own workspace after a flush or
    // push, the context's own result block after a batch (never another
    // context's memory, which may be freed before this one is read)
    Seg *res_seg = nullptr;
    Prob *res_prob = nullptr;
    Seg *own_res_seg = nullptr;
    Prob *own_res_prob = nullptr;
    bool has_result = false;
    bool res_streaming = false;
    uint64_t res_base = 0;

    // pinned staging
    Seg *h_seg = nullptr;          // SEG_RING * MAX_SEGS
    cudaEvent_t seg_ev[SEG_RING] = {};
    int seg_slot = 0;
    tpc_hit *h_stage = nullptr;
    size_t stage_cap = 0;
    cudaEvent_t stage_ev = nullptr;
    cudaEvent_t done_ev = nullptr;

    // launch choices (tpc_set_tuning / tpc_tune_batch); a batch uses its lead's
    Tuning tune{};
    tpc_variant_stats vstats{};    // the last (b)/(c) flush (tpc_variant_stats)
    bool vstats_pending = false;   // (c) counters still in h_flag

    // graph of the step sequence
    cudaGraphExec_t graph = nullptr;
    int graph_nsegs = 0;
    uint64_t graph_gen = 0;        // workspace generation the graph was captured on
    int graph_grid = 0;
    Tuning graph_tune{};           // launch choices the graph was captured with

    std::mutex mu;

    size_t device_bytes() const {
        return ws.mem.bytes + outmem.bytes + in_cap * sizeof(tpc_hit) +
               (sbuf[0] ? 2 * (carry_cap + chunk_cap) * (sizeof(tpc_hit) + sizeof(uint64_t)) : 0);
    }
};

// Point the context's device-memory holders at its current stream.
static void bind_mem(tpc_ctx *c) {
    for (DevMem *m : {&c->ws.mem, &c->vs.mem, &c->outmem}) {
        m->stream = c->stream;
        m->dev = c->device;
    }
}

int tpc::occupancy(const void *kernel, int threads, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(occ_mu);
    for (const OccEntry &e : occ_cache)
        if (e.dev == dev && e.kernel == kernel && e.threads == threads && e.smem == smem) return e.blocks;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, smem) != cudaSuccess || blocks < 1)
        blocks = 1;
    occ_cache.push_back({dev, kernel, threads, smem, blocks});
    return blocks;
}

namespace {

int grid_of(const tpc_ctx *c) {
    int k = c->ctas_per_sm > 0 ? c->ctas_per_sm : 4;
    return c->sms * k;
}

// Entries ensure_out(c, n) sizes the output buffers for: n (at least 1024);
// on growth at least double the old size (at most 2^26 entries more).
size_t out_grown(const tpc_ctx *c, size_t n) {
    const size_t cap = std::max<size_t>(n, 1024);
    if (!c->d_labels || !c->out_cap) return cap;
    if (cap <= c->out_cap) return c->out_cap;
    return std::max(cap, std::min(2 * c->out_cap, c->out_cap + (size_t(1) << 26)));
}

cudaError_t ensure_out(tpc_ctx *c, size_t n) {
    if (n <= c->out_cap && c->d_labels) return cudaSuccess;
    const size_t cap = out_grown(c, n);
    c->outmem.release();
    cudaError_t e = cudaSuccess;
    c->d_labels = c->outmem.alloc<uint64_t>(cap, e);
    c->d_index = c->outmem.alloc<uint64_t>(cap, e);
    c->d_rec = c->outmem.alloc<tpc_cluster>(cap, e);
    if (e != cudaSuccess) {
        c->outmem.release();
        c->d_labels = c->d_index = nullptr;
        c->d_rec = nullptr;
        c->out_cap = 0;
        return e;
    }
    c->out_cap = cap;
    return cudaSuccess;
}

// Upload the host copy of the segment table through a pinned ring slot.
cudaError_t upload_segs(tpc_ctx *c, const Work &w, const Seg *segs, int nsegs, cudaStream_t st) {
    const int slot = c->seg_slot;
    c->seg_slot = (c->seg_slot + 1) % SEG_RING;
    cudaError_t e = cudaEventSynchronize(c->seg_ev[slot]);
    if (e != cudaSuccess) return e;
    Seg *h = c->h_seg + (size_t)slot * MAX_SEGS;
    std::memcpy(h, segs, nsegs * sizeof(Seg));
    e = cudaMemcpyAsync(w.seg, h, nsegs * sizeof(Seg), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(c->seg_ev[slot], st);
}

void enqueue_kernels(const Work &w, int nsegs, const Launch &L) {
    launch_setup(w, nsegs, L);
    launch_sort_fast(w, L);
    launch_seg_finalize(w, L);
    launch_make_keys(w, L);
    for (int pass = 0; pass < 4; ++pass) launch_radix_pass(w, pass, L);
    launch_gather(w, L);
    launch_link(w, L);
    launch_features(w, L);
    launch_outputs(w, L);
}

// Run the fixed kernel sequence, from a CUDA graph captured on first use
// (and re-captured when the workspace or the segment count changes).
cudaError_t run_step(tpc_ctx *owner, Workspace &ws, int nsegs, cudaStream_t st, Tracer *tr = nullptr) {
    Launch L{grid_of(owner), st, nullptr, owner->sms, owner->ctas_per_sm};
    L.tune = owner->tune;
    if (tr) {   // kernels one by one with an event after each (no graph)
        cudaEventRecord(tr->ev[0], st);
        Launch T = L;
        T.tr = tr;
        enqueue_kernels(ws.w, nsegs, T);
        return cudaGetLastError();
    }
    if (!owner->graph || owner->graph_nsegs != nsegs || owner->graph_gen != ws.gen ||
        owner->graph_grid != L.grid || std::memcmp(&owner->graph_tune, &owner->tune, sizeof(Tuning)) != 0) {
        if (owner->graph) {
            cudaGraphExecDestroy(owner->graph);
            owner->graph = nullptr;
        }
        cudaStream_t cap_st;
        cudaError_t e = cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            Launch C = L;
            C.stream = cap_st;
            enqueue_kernels(ws.w, nsegs, C);
            e = cudaStreamEndCapture(cap_st, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&owner->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap_st);
        if (e != cudaSuccess) {
            owner->graph = nullptr;
            return e;
        }
        owner->graph_nsegs = nsegs;
        owner->graph_gen = ws.gen;
        owner->graph_grid = L.grid;
        owner->graph_tune = owner->tune;
    }
    return cudaGraphLaunch(owner->graph, st);
}

// Outputs of a one-shot step: the caller's bound buffers, else the
// context's own; the retrieval calls read them from where they went.
void set_outputs(tpc_ctx *c, Seg &s) {
    const bool bound = c->bound_labels != nullptr;
    s.out_labels = c->res_labels = bound ? c->bound_labels : c->d_labels;
    s.out_rec = c->res_rec = bound ? c->bound_rec : c->d_rec;
    s.out_cap = (uint32_t)(bound ? c->bound_cap : c->out_cap);
}

// Whether a sensor takes k_tile_link instead of the table kernel under the
// launch choices t (bit 0: single-band sensors, bit 1: banded ones).
uint32_t link_general(const Tuning &t, uint32_t W, uint32_t H) {
    const int nb = link_bands(W, H);
    if (nb == 1) return t.general_link & 1u;
    if (nb > 1) return (t.general_link >> 1) & 1u;
    return 0;
}

Seg base_seg(const tpc_ctx *c, const Tuning &t) {
    Seg s{};
    s.width = c->width;
    s.height = c->height;
    s.dt = c->dt32;
    s.variant = (uint32_t)c->variant;
    s.max_disorder = ~0ull;
    s.link_general = link_general(t, c->width, c->height);
    return s;
}

Seg base_seg(const tpc_ctx *c) { return base_seg(c, c->tune); }

cudaError_t stage_host(tpc_ctx *c, tpc_hit *dst, const tpc_hit *src, size_t n) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, src) == cudaSuccess && a.type == cudaMemoryTypeHost)
        return cudaMemcpyAsync(dst, src, n * sizeof(tpc_hit), cudaMemcpyHostToDevice, c->stream);
    cudaGetLastError();   // clear a possible "not a device pointer" error
    const size_t chunk = size_t(1) << 20;
    if (!c->h_stage) {
        cudaError_t e = host_alloc(&c->fail_alloc, (void **)&c->h_stage, chunk * sizeof(tpc_hit));
        if (e != cudaSuccess) return e;
        c->stage_cap = chunk;
    }
    for (size_t done = 0; done < n; done += chunk) {
        const size_t m = std::min(chunk, n - done);
        cudaError_t e = cudaEventSynchronize(c->stage_ev);
        if (e != cudaSuccess) return e;
        std::memcpy(c->h_stage, src + done, m * sizeof(tpc_hit));
        e = cudaMemcpyAsync(dst + done, c->h_stage, m * sizeof(tpc_hit), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return e;
        e = cudaEventRecord(c->stage_ev, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool over_budget(const tpc_ctx *c, size_t extra) {
    return c->budget && c->device_bytes() + extra > c->budget;
}

// Make the pending hits of a non-streaming context live in c->in with room
// for `more` additional hits.
int materialise(tpc_ctx *c, size_t more) {
    const size_t need = c->pending + more;
    if (need > c->in_cap || (c->zc && !c->in)) {
        size_t cap = std::max(need, c->in_cap * 2);
        if (over_budget(c, (cap - c->in_cap) * sizeof(tpc_hit))) return TPC_ERR_BUSY;
        tpc_hit *nb = nullptr;
        if (dev_alloc(&c->fail_alloc, (void **)&nb, cap * sizeof(tpc_hit), c->stream, c->device) != cudaSuccess)
            return TPC_ERR_NOMEM;
        const tpc_hit *src = c->zc ? c->zc : c->in;
        if (c->pending &&
            cudaMemcpyAsync(nb, src, c->pending * sizeof(tpc_hit), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
            dev_free(nb, c->stream);
            return TPC_ERR_CUDA;
        }
        dev_free(c->in, c->stream);   // after the copy out of it
        c->in = nb;
        c->in_cap = cap;
    } else if (c->zc) {
        if (c->pending &&
            cudaMemcpyAsync(c->in, c->zc, c->pending * sizeof(tpc_hit), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            return TPC_ERR_CUDA;
    }
    c->zc = nullptr;
    return TPC_OK;
}

int ensure_stream_buffers(tpc_ctx *c, size_t chunk) {
    if (chunk > c->chunk_cap || c->carry_ub + chunk > c->carry_cap) {
        // learn the true carry size before growing anything
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return TPC_ERR_CUDA;
        uint32_t nc = 0;
        if (c->ss && cudaMemcpy(&nc, &c->ss->n_carry, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return TPC_ERR_CUDA;
        c->carry_ub = nc;
    }
    if (chunk <= c->chunk_cap && c->carry_ub + chunk <= c->carry_cap && c->sbuf[0]) return TPC_OK;
    size_t ncarry = std::max<size_t>({c->carry_cap, 2 * (c->carry_ub + chunk), 1 << 16});
    size_t nchunk = std::max<size_t>({c->chunk_cap, chunk, 1 << 16});
    size_t extra = 2 * ((ncarry + nchunk) - (c->carry_cap + c->chunk_cap)) * (sizeof(tpc_hit) + sizeof(uint64_t));
    if (over_budget(c, extra)) return TPC_ERR_BUSY;
    tpc_hit *nb[2] = {nullptr, nullptr};
    uint64_t *ng[2] = {nullptr, nullptr};
    for (int i = 0; i < 2; ++i) {
        if (dev_alloc(&c->fail_alloc, (void **)&nb[i], (ncarry + nchunk) * sizeof(tpc_hit), c->stream, c->device) !=
                cudaSuccess ||
            dev_alloc(&c->fail_alloc, (void **)&ng[i], (ncarry + nchunk) * sizeof(uint64_t), c->stream, c->device) !=
                cudaSuccess) {
            for (int j = 0; j < 2; ++j) { dev_free(nb[j], c->stream); dev_free(ng[j], c->stream); }
            return TPC_ERR_NOMEM;
        }
    }
    // move the current carry (right aligned in the buffer the next step reads)
    const int next = 1 - c->scur;
    if (c->sbuf[next] && c->carry_ub) {
        const size_t nc = c->carry_ub;   // exact after the synchronisation above
        cudaMemcpyAsync(nb[next] + (ncarry - nc), c->sbuf[next] + (c->carry_cap - nc), nc * sizeof(tpc_hit),
                        cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(ng[next] + (ncarry - nc), c->sgidx[next] + (c->carry_cap - nc), nc * sizeof(uint64_t),
                        cudaMemcpyDeviceToDevice, c->stream);
    }
    for (int i = 0; i < 2; ++i) {   // freed after the copies above, in stream order
        dev_free(c->sbuf[i], c->stream);
        dev_free(c->sgidx[i], c->stream);
        c->sbuf[i] = nb[i];
        c->sgidx[i] = ng[i];
    }
    c->carry_cap = ncarry;
    c->chunk_cap = nchunk;
    return TPC_OK;
}

// One streaming step over the carry plus `n` new hits already copied into
// the chunk region of the next input buffer.  close_all: end of stream.
int stream_step(tpc_ctx *c, size_t n, bool close_all) {
    const int in = 1 - c->scur;
    const size_t positions = c->carry_ub + n;
    c->has_result = false;   // the workspace may move: the last result is gone
    if (c->ws.ensure(positions) != cudaSuccess) return TPC_ERR_NOMEM;
    if (ensure_out(c, positions) != cudaSuccess) return TPC_ERR_NOMEM;   // >= hits this step can finalise
    Seg s = base_seg(c);
    s.carry_in = c->sbuf[in];
    s.carry_gidx_in = c->sgidx[in];
    s.carry_out = c->sbuf[c->scur];
    s.carry_gidx_out = c->sgidx[c->scur];
    s.ss = c->ss;
    s.out_labels = c->res_labels = c->d_labels;
    s.out_index = c->d_index;
    s.out_rec = c->res_rec = c->d_rec;
    s.out_cap = (uint32_t)c->out_cap;
    s.gidx_base = c->pushed;
    s.max_disorder = close_all ? ~0ull : c->max_disorder;
    s.carry_cap = (uint32_t)c->carry_cap;
    s.n_new = (uint32_t)n;
    if (upload_segs(c, c->ws.w, &s, 1, c->stream) != cudaSuccess) return TPC_ERR_CUDA;
    if (run_step(c, c->ws, 1, c->stream) != cudaSuccess) return TPC_ERR_CUDA;
    c->scur = in;
    c->pushed += n;
    c->carry_ub = close_all ? 0 : positions;
    c->res_seg = c->ws.w.seg;
    c->res_prob = c->ws.w.prob;
    c->has_result = true;
    c->res_streaming = true;
    return TPC_OK;
}

struct ResultInfo {
    Seg seg;
    Prob prob;
};

int read_result(tpc_ctx *c, ResultInfo &r) {
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return TPC_ERR_CUDA;
    if (!c->has_result) {
        std::memset(&r, 0, sizeof(r));
        return TPC_OK;
    }
    if (cudaMemcpy(&r.seg, c->res_seg, sizeof(Seg), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&r.prob, c->res_prob, sizeof(Prob), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TPC_ERR_CUDA;
    // the last streaming step's open hits are the exact carry: the next push
    // sizes its arrays from it instead of the running upper bound
    if (c->res_streaming && c->ss && !r.prob.err && r.seg.n_open <= c->carry_ub) c->carry_ub = r.seg.n_open;
    return map_err(r.prob.err);
}

}  // namespace

extern "C" {

int tpc_create(uint32_t width, uint32_t height, uint64_t dt, int variant, tpc_ctx **out) {
    if (!out) return TPC_ERR_ARG;
    *out = nullptr;
    if (width == 0 || height == 0 || width > 65536 || height > 65536 ||
        (uint64_t)width * height > MAX_PIXELS)
        return TPC_ERR_ARG;
    if (variant != TPC_LOCAL && variant != TPC_GLOBAL && variant != TPC_STATIC) return TPC_ERR_ARG;
    tpc_ctx *c = new (std::nothrow) tpc_ctx();
    if (!c) return TPC_ERR_NOMEM;
    c->width = width;
    c->height = height;
    c->dt = dt;
    c->dt32 = dt > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)dt;
    c->variant = variant;
    c->ws.mem.fault = c->vs.mem.fault = c->outmem.fault = &c->fail_alloc;
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return TPC_ERR_CUDA; }
    c->sms = num_sms(c->device);
    if (init_kernel_attributes() != cudaSuccess) { delete c; return TPC_ERR_CUDA; }
    bool ok = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) == cudaSuccess;
    c->own_stream = ok;
    bind_mem(c);
    ok = ok && device_pool(c->device) != nullptr;
    ok = ok && cudaMallocHost(&c->h_seg, sizeof(Seg) * MAX_SEGS * SEG_RING) == cudaSuccess;
    for (int i = 0; ok && i < SEG_RING; ++i)
        ok = cudaEventCreateWithFlags(&c->seg_ev[i], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->stage_ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&c->own_res_seg, sizeof(Seg)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->own_res_prob, sizeof(Prob)) == cudaSuccess;
    if (!ok) { tpc_destroy(c); return TPC_ERR_CUDA; }
    *out = c;
    return TPC_OK;
}

int tpc_set_option(tpc_ctx *c, int key, uint64_t value) {
    if (!c) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    const bool busy = c->pending || c->zc || (c->ss && c->carry_ub);
    switch (key) {
    case TPC_OPT_MAX_DISORDER:
        if (busy) return TPC_ERR_STATE;
        if (value == 0) return TPC_ERR_ARG;
        if (value != ~0ull && !c->ss) {   // the stream state first: the option stands only with it
            StreamState *ss = nullptr;
            if (dev_alloc(&c->fail_alloc, (void **)&ss, sizeof(StreamState), c->stream, c->device) != cudaSuccess)
                return TPC_ERR_NOMEM;
            if (cudaMemsetAsync(ss, 0, sizeof(StreamState), c->stream) != cudaSuccess) {
                dev_free(ss, c->stream);
                return TPC_ERR_CUDA;
            }
            c->ss = ss;
            c->scur = 1;
            c->carry_ub = 0;
        }
        c->max_disorder = value;
        return TPC_OK;
    case TPC_OPT_MEM_BUDGET:
        c->budget = value;
        return TPC_OK;
    case TPC_OPT_STREAM: {
        if (busy) return TPC_ERR_STATE;
        cudaStreamSynchronize(c->stream);
        if (c->own_stream) cudaStreamDestroy(c->stream);
        c->own_stream = false;
        c->stream = reinterpret_cast<cudaStream_t>(value);
        if (!value) {
            if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return TPC_ERR_CUDA;
            c->own_stream = true;
        }
        bind_mem(c);   // the old stream is idle: later frees may go on the new one
        return TPC_OK;
    }
    case TPC_OPT_CTAS_PER_SM:
        if (value > 64) return TPC_ERR_ARG;
        c->ctas_per_sm = (int)value;
        return TPC_OK;
    case TPC_OPT_FAIL_ALLOC:
        if (value > (uint64_t)INT64_MAX) return TPC_ERR_ARG;
        c->fail_alloc = (int64_t)value;
        return TPC_OK;
    default:
        return TPC_ERR_ARG;
    }
}

int tpc_push(tpc_ctx *c, const tpc_hit *hits, size_t n, int where) {
    if (!c || (n && !hits) || (where != TPC_HOST && where != TPC_DEVICE)) return TPC_ERR_ARG;
    if (n > 0x7FFFFFFFull) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->max_disorder != ~0ull) {
        // streaming: copy the chunk behind the carry and cluster it now
        if (c->variant != TPC_LOCAL) return TPC_ERR_ARG;
        if (c->budget && over_budget(c, c->ws.bytes_after(c->carry_ub + n) > c->ws.mem.bytes
                                            ? c->ws.bytes_after(c->carry_ub + n) - c->ws.mem.bytes : 0))
            return TPC_ERR_BUSY;
        int rc = ensure_stream_buffers(c, n);
        if (rc) return rc;
        tpc_hit *dst = c->sbuf[1 - c->scur] + c->carry_cap;
        cudaError_t e = where == TPC_HOST
            ? stage_host(c, dst, hits, n)
            : cudaMemcpyAsync(dst, hits, n * sizeof(tpc_hit), cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TPC_ERR_NOMEM : TPC_ERR_CUDA;
        return stream_step(c, n, false);
    }
    if (n == 0) return TPC_OK;
    if (where == TPC_DEVICE && c->pending == 0 && !c->zc) {
        c->zc = hits;   // zero copy: read in place by the next flush
        c->pending = n;
        return TPC_OK;
    }
    int rc = materialise(c, n);
    if (rc) return rc;
    cudaError_t e = where == TPC_HOST
        ? stage_host(c, c->in + c->pending, hits, n)
        : cudaMemcpyAsync(c->in + c->pending, hits, n * sizeof(tpc_hit), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TPC_ERR_NOMEM : TPC_ERR_CUDA;
    c->pending += n;
    return TPC_OK;
}

// Variants (b) and (c): the (a) forest and its roots first, then the
// variant's kernels (csrc/variants.cu), then the shared feature / output
// kernels.
// Launched without a graph; (b) waits for the host between rounds.
static int flush_variant(tpc_ctx *c, Tracer *tr) {
    const size_t n = c->pending;
    c->has_result = false;   // the workspace may move: the last result is gone
    if (c->bound_labels && n > c->bound_cap) return TPC_ERR_CAP;
    if (c->ws.ensure(n) != cudaSuccess) return TPC_ERR_NOMEM;
    if (c->vs.ensure(c->ws.pos_cap, (size_t)c->width * c->height, c->variant == TPC_GLOBAL) != cudaSuccess)
        return TPC_ERR_NOMEM;
    if (!c->bound_labels && ensure_out(c, n) != cudaSuccess) return TPC_ERR_NOMEM;
    if (!c->h_flag && host_alloc(&c->fail_alloc, (void **)&c->h_flag, 8 * sizeof(uint32_t)) != cudaSuccess)
        return TPC_ERR_NOMEM;
    Seg s = base_seg(c);
    s.hits = c->zc ? c->zc : c->in;
    set_outputs(c, s);
    s.gidx_base = c->pushed;
    s.n_new = (uint32_t)n;
    if (upload_segs(c, c->ws.w, &s, 1, c->stream) != cudaSuccess) return TPC_ERR_CUDA;
    const Work &w = c->ws.w;
    const VarWork &v = c->vs.v;
    Launch L{grid_of(c), c->stream, tr, c->sms, c->ctas_per_sm};
    L.tune = c->tune;
    if (tr) cudaEventRecord(tr->ev[0], c->stream);
    launch_setup(w, 1, L);
    launch_sort_fast(w, L);
    launch_seg_finalize(w, L);
    launch_make_keys(w, L);
    for (int pass = 0; pass < 4; ++pass) launch_radix_pass(w, pass, L);
    launch_gather(w, L);
    launch_tile_border(w, L);
    launch_sorted_roots(w, L);
    const Work wv = variant_view(w, v);
    if (c->variant == TPC_STATIC) {
        launch_variant_keys(w, v, 0, L);
        for (int pass = 0; pass < 4; ++pass) launch_radix_pass(wv, pass, L);
        launch_static_sweep(w, v, L);
        c->vstats = tpc_variant_stats{};
        if (cudaMemcpyAsync(c->h_flag, v.changed, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess)
            return TPC_ERR_CUDA;
        c->vstats_pending = true;   // read at tpc_variant_stats, after the stream
    } else {
        launch_variant_keys(w, v, 1, L);
        for (int pass = 0; pass < 3; ++pass) launch_radix_pass(wv, pass, L);
        launch_pixel_timelines(w, v, c->width * c->height, L);
        // Rounds of the rule until the partition is closed under it, on the
        // (a) components' dense ids: the first over every hit's 9 latest
        // neighbours, the later ones over the edges left open (all hits
        // again after an overflow of the list); the groups' last keys are
        // exact at the start (each group one component) and kept at the
        // roots by the unions (never above the exact value), and recomputed
        // exactly when a round merges nothing: the end is a round without
        // merges on exact values.
        launch_components(w, v, L);
        bool full = true, exact = true;
        int in = 0;
        c->vstats = tpc_variant_stats{};
        c->vstats_pending = false;
        for (int round = 0;; ++round) {
            if (round > 4096) return TPC_ERR_TIMEOUT;
            launch_global_edges(w, v, full, round == 0, in, L);   // round 0: k_sorted_roots' roots hold
            ++c->vstats.rounds;
            if (full) ++c->vstats.full_rounds;
            if (cudaMemcpyAsync(c->h_flag, v.changed, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream) !=
                    cudaSuccess ||
                (round == 0 && cudaMemcpyAsync(c->h_flag + 2, v.ecount, sizeof(unsigned long long),
                                               cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                return TPC_ERR_CUDA;
            if (round == 0) {
                const unsigned long long listed = *reinterpret_cast<unsigned long long *>(c->h_flag + 2);
                c->vstats.first_open_edges = (uint32_t)std::min<unsigned long long>(listed, v.edge_cap);
            }
            const bool merged = c->h_flag[0] != 0, overflow = c->h_flag[1] != 0;
            in = full ? 0 : 1 - in;   // the list just written
            full = overflow;
            if (merged) {
                exact = false;
                continue;
            }
            if (exact) break;
            launch_group_last(v, L);
            ++c->vstats.exact_checks;
            exact = true;
        }
        launch_comp_parents(w, v, L);
    }
    // (b) only merges, so its roots are (a) roots, whose slots the tile
    // kernels zeroed; a (c) root can be any hit.  k_accumulate finds the
    // roots (the parents may be deep).
    if (c->variant == TPC_STATIC) launch_init_roots(w, L);
    launch_features(w, L);
    launch_outputs(w, L);
    if (cudaGetLastError() != cudaSuccess) return TPC_ERR_CUDA;
    c->res_base = c->pushed;
    c->pushed += n;
    c->pending = 0;
    c->zc = nullptr;
    c->res_seg = c->ws.w.seg;
    c->res_prob = c->ws.w.prob;
    c->has_result = true;
    c->res_streaming = false;
    return TPC_OK;
}

static int flush_impl(tpc_ctx *c, Tracer *tr) {
    if (c->max_disorder != ~0ull) {
        if (tr) return TPC_ERR_STATE;
        int rc = ensure_stream_buffers(c, 0);
        if (rc) return rc;
        return stream_step(c, 0, true);
    }
    if (c->variant != TPC_LOCAL) return flush_variant(c, tr);
    const size_t n = c->pending;
    c->has_result = false;   // the workspace may move: the last result is gone
    if (over_budget(c, c->ws.bytes_after(n) > c->ws.mem.bytes ? c->ws.bytes_after(n) - c->ws.mem.bytes : 0))
        return TPC_ERR_BUSY;
    if (c->bound_labels && n > c->bound_cap) return TPC_ERR_CAP;
    if (c->ws.ensure(n) != cudaSuccess) return TPC_ERR_NOMEM;
    if (!c->bound_labels && ensure_out(c, n) != cudaSuccess) return TPC_ERR_NOMEM;
    Seg s = base_seg(c);
    s.hits = c->zc ? c->zc : c->in;
    set_outputs(c, s);
    s.gidx_base = c->pushed;
    s.n_new = (uint32_t)n;
    if (upload_segs(c, c->ws.w, &s, 1, c->stream) != cudaSuccess) return TPC_ERR_CUDA;
    if (run_step(c, c->ws, 1, c->stream, tr) != cudaSuccess) return TPC_ERR_CUDA;
    c->res_base = c->pushed;
    c->pushed += n;
    c->pending = 0;
    c->zc = nullptr;
    c->res_seg = c->ws.w.seg;
    c->res_prob = c->ws.w.prob;
    c->has_result = true;
    c->res_streaming = false;
    return TPC_OK;
}

int tpc_flush(tpc_ctx *c) {
    if (!c) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    return flush_impl(c, nullptr);
}

int tpc_profile_flush(tpc_ctx *c, const char **names, float *ms, int cap, int *n_out) {
    if (!c || !n_out || cap < 0 || (cap && (!names || !ms))) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    Tracer tr;
    for (int i = 0; i <= Tracer::MAX; ++i)
        if (cudaEventCreate(&tr.ev[i]) != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaEventDestroy(tr.ev[j]);
            return TPC_ERR_CUDA;
        }
    int rc = flush_impl(c, &tr);
    if (rc == TPC_OK && cudaEventSynchronize(tr.ev[tr.n]) != cudaSuccess) rc = TPC_ERR_CUDA;
    if (rc == TPC_OK) {
        *n_out = tr.n;
        for (int i = 0; i < tr.n && i < cap; ++i) {
            names[i] = tr.names[i];
            cudaEventElapsedTime(&ms[i], tr.ev[i], tr.ev[i + 1]);
        }
        if (tr.n > cap) rc = TPC_ERR_CAP;
    }
    for (int i = 0; i <= Tracer::MAX; ++i) cudaEventDestroy(tr.ev[i]);
    return rc;
}

int tpc_sync(tpc_ctx *c) {
    if (!c) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    ResultInfo r;
    return read_result(c, r);
}

int tpc_counts(tpc_ctx *c, size_t *n_hits, size_t *n_clusters, size_t *n_open) {
    if (!c) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    ResultInfo r;
    int rc = read_result(c, r);
    if (n_hits) *n_hits = r.seg.n_final;
    if (n_clusters) *n_clusters = r.seg.n_clusters;
    if (n_open) *n_open = r.seg.n_open;
    return rc;
}

int tpc_labels(tpc_ctx *c, uint64_t *labels, uint64_t *indices, size_t cap, size_t *n_out, int where) {
    if (!c || !n_out || (where != TPC_HOST && where != TPC_DEVICE)) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    ResultInfo r;
    int rc = read_result(c, r);
    if (rc) return rc;
    const size_t n = r.seg.n_final;
    *n_out = n;
    if (n > cap) return TPC_ERR_CAP;
    if (n && !labels) return TPC_ERR_ARG;
    if (!n) return TPC_OK;
    const cudaMemcpyKind kind = where == TPC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (labels != c->res_labels &&
        cudaMemcpyAsync(labels, c->res_labels, n * sizeof(uint64_t), kind, c->stream) != cudaSuccess)
        return TPC_ERR_CUDA;
    if (indices) {
        if (c->res_streaming) {
            if (cudaMemcpyAsync(indices, c->d_index, n * sizeof(uint64_t), kind, c->stream) != cudaSuccess)
                return TPC_ERR_CUDA;
        } else if (where == TPC_DEVICE) {
            k_iota_u64<<<c->sms * 4, 256, 0, c->stream>>>(indices, c->res_base, n);
        } else {
            for (size_t i = 0; i < n; ++i) indices[i] = c->res_base + i;
        }
    }
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}

int tpc_labels_async(tpc_ctx *c, uint64_t *labels, size_t cap, size_t *n_out, int where) {
    if (!c || !n_out || (where != TPC_HOST && where != TPC_DEVICE)) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->has_result || c->res_streaming) return TPC_ERR_STATE;
    const size_t n = c->pushed - c->res_base;   // every hit of a one-shot step is final
    *n_out = n;
    if (n > cap) return TPC_ERR_CAP;
    if (!n) return TPC_OK;
    if (!labels) return TPC_ERR_ARG;
    const cudaMemcpyKind kind = where == TPC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (labels == c->res_labels) return TPC_OK;   // written there by the step
    return cudaMemcpyAsync(labels, c->res_labels, n * sizeof(uint64_t), kind, c->stream) == cudaSuccess
               ? TPC_OK : TPC_ERR_CUDA;
}

int tpc_cluster_features(tpc_ctx *c, tpc_cluster *out, size_t cap, size_t *n_out, int where) {
    if (!c || !n_out || (where != TPC_HOST && where != TPC_DEVICE)) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    ResultInfo r;
    int rc = read_result(c, r);
    if (rc) return rc;
    const size_t n = r.seg.n_clusters;
    *n_out = n;
    if (n > cap) return TPC_ERR_CAP;
    if (n && !out) return TPC_ERR_ARG;
    if (!n) return TPC_OK;
    const cudaMemcpyKind kind = where == TPC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (out != c->res_rec &&
        cudaMemcpyAsync(out, c->res_rec, n * sizeof(tpc_cluster), kind, c->stream) != cudaSuccess)
        return TPC_ERR_CUDA;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? TPC_OK : TPC_ERR_CUDA;
}

}  // extern "C"

int tpc::check_batch(tpc_ctx **ctxs, int n) {
    if (!ctxs || n <= 0 || n > MAX_SEGS) return TPC_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || ctxs[i]->max_disorder != ~0ull || ctxs[i]->variant != TPC_LOCAL) return TPC_ERR_ARG;
        for (int j = 0; j < i; ++j) if (ctxs[j] == ctxs[i]) return TPC_ERR_ARG;
        if (ctxs[i]->device != ctxs[0]->device) return TPC_ERR_ARG;
    }
    return TPC_OK;
}

int tpc::batch_step(tpc_ctx **ctxs, int n, bool consume) {
    tpc_ctx *lead = ctxs[0];
    const Tuning &t = lead->tune;
    for (int i = 0; i < n; ++i) ctxs[i]->has_result = false;   // workspaces may move
    size_t positions = 0;
    for (int i = 0; i < n; ++i) positions += ((ctxs[i]->pending + TILE - 1) / TILE) * TILE;
    // output buffers first (allocated on each context's own stream), then
    // every context's pending copies and allocations must land before the
    // lead stream uses them
    for (int i = 0; i < n; ++i)
        if (ctxs[i]->bound_labels && ctxs[i]->pending > ctxs[i]->bound_cap) return TPC_ERR_CAP;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i]->bound_labels && ensure_out(ctxs[i], ctxs[i]->pending) != cudaSuccess) return TPC_ERR_NOMEM;
    for (int i = 1; i < n; ++i) {
        if (cudaEventRecord(ctxs[i]->done_ev, ctxs[i]->stream) != cudaSuccess ||
            cudaStreamWaitEvent(lead->stream, ctxs[i]->done_ev, 0) != cudaSuccess)
            return TPC_ERR_CUDA;
    }
    if (lead->ws.ensure(positions) != cudaSuccess) return TPC_ERR_NOMEM;
    // segment order: as given, or (a tuning choice) most pending hits first,
    // so that the big sensors' tiles start in the first wave
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    if (t.order == 1)
        std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return ctxs[a]->pending > ctxs[b]->pending; });
    std::vector<Seg> segs(n);
    for (int k = 0; k < n; ++k) {
        tpc_ctx *c = ctxs[perm[k]];
        Seg s = base_seg(c, t);
        s.hits = c->zc ? c->zc : c->in;
        set_outputs(c, s);
        s.gidx_base = c->pushed;
        s.n_new = (uint32_t)c->pending;
        segs[k] = s;
    }
    if (upload_segs(lead, lead->ws.w, segs.data(), n, lead->stream) != cudaSuccess) return TPC_ERR_CUDA;
    if (run_step(lead, lead->ws, n, lead->stream) != cudaSuccess) return TPC_ERR_CUDA;
    for (int k = 0; k < n; ++k) {   // each context keeps its own copy of its results
        tpc_ctx *c = ctxs[perm[k]];
        if (cudaMemcpyAsync(c->own_res_seg, lead->ws.w.seg + k, sizeof(Seg), cudaMemcpyDeviceToDevice,
                            lead->stream) != cudaSuccess ||
            cudaMemcpyAsync(c->own_res_prob, lead->ws.w.prob, sizeof(Prob), cudaMemcpyDeviceToDevice,
                            lead->stream) != cudaSuccess)
            return TPC_ERR_CUDA;
    }
    if (cudaEventRecord(lead->done_ev, lead->stream) != cudaSuccess) return TPC_ERR_CUDA;
    for (int i = 0; i < n; ++i) {
        tpc_ctx *c = ctxs[i];
        if (i && cudaStreamWaitEvent(c->stream, lead->done_ev, 0) != cudaSuccess) return TPC_ERR_CUDA;
        if (!consume) continue;   // a tuning trial: the hits stay pending
        c->res_base = c->pushed;
        c->pushed += c->pending;
        c->pending = 0;
        c->zc = nullptr;
        c->res_seg = c->own_res_seg;
        c->res_prob = c->own_res_prob;
        c->has_result = true;
        c->res_streaming = false;
    }
    return TPC_OK;
}

extern "C" {

int tpc_batch_flush(tpc_ctx **ctxs, int n) {
    int rc = check_batch(ctxs, n);
    if (rc) return rc;
    std::vector<std::unique_lock<std::mutex>> locks;
    for (int i = 0; i < n; ++i) locks.emplace_back(ctxs[i]->mu);
    return batch_step(ctxs, n, true);
}

int tpc_forest(tpc_ctx *c, uint32_t *parent, uint32_t *input_pos, size_t cap, size_t *n_out) {
    if (!c || !n_out) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    *n_out = 0;
    ResultInfo r;
    int rc = read_result(c, r);
    if (rc) return rc;
    if (!c->has_result || c->res_seg != c->ws.w.seg) return TPC_ERR_STATE;
    const size_t n = r.seg.n;
    *n_out = n;
    if (n > cap) return TPC_ERR_CAP;
    if (!n) return TPC_OK;
    if (!parent || !input_pos) return TPC_ERR_ARG;
    // the sorted order lives in the buffer the step's last sort pass wrote
    const uint32_t sel = r.prob.npasses & 1u;
    if (cudaMemcpy(parent, c->ws.w.parent + r.seg.off, n * sizeof(uint32_t), cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(input_pos, c->ws.w.vals[sel] + r.seg.off, n * sizeof(uint32_t), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return TPC_ERR_CUDA;
    for (size_t i = 0; i < n; ++i) {   // positions and input indices relative to the step
        parent[i] -= r.seg.off;
        input_pos[i] -= r.seg.off;
    }
    return TPC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Internal interface of the serving loop (server.cu).

size_t tpc::ctx_projected_bytes(tpc_ctx *c, size_t n) {
    std::lock_guard<std::mutex> lk(c->mu);
    // the growth rules of ensure_stream_buffers, stream_step and ensure_out,
    // with the carry at its upper bound (the device holds the exact count)
    size_t carry_cap = c->carry_cap, chunk_cap = c->chunk_cap;
    if (n > chunk_cap || c->carry_ub + n > carry_cap || !c->sbuf[0]) {
        carry_cap = std::max<size_t>({carry_cap, 2 * (c->carry_ub + n), 1 << 16});
        chunk_cap = std::max<size_t>({chunk_cap, n, 1 << 16});
    }
    const size_t stream_bytes = 2 * (carry_cap + chunk_cap) * (sizeof(tpc_hit) + sizeof(uint64_t));
    const size_t positions = c->carry_ub + n;
    const size_t ws = c->ws.bytes_after(positions);
    const size_t out_n = out_grown(c, positions);
    const size_t out = out_n == c->out_cap && c->d_labels ? c->outmem.bytes
                                                          : 2 * ((out_n * 8 + 255) & ~size_t(255)) +
                                                                ((out_n * sizeof(tpc_cluster) + 255) & ~size_t(255));
    return ws + out + stream_bytes + c->in_cap * sizeof(tpc_hit);
}

size_t tpc::ctx_held_bytes(tpc_ctx *c) {
    std::lock_guard<std::mutex> lk(c->mu);
    return c->device_bytes();
}

void tpc::ctx_release_scratch(tpc_ctx *c) {
    std::lock_guard<std::mutex> lk(c->mu);
    c->ws.mem.release();   // stream-ordered: after the context's queued work
    c->ws.w = Work{};
    c->ws.pos_cap = c->ws.tile_cap = c->ws.alloc_need = 0;
    ++c->ws.gen;
    c->outmem.release();
    c->d_labels = c->d_index = nullptr;
    c->d_rec = nullptr;
    c->out_cap = 0;
    c->vs.mem.release();
    c->vs.v = VarWork{};
    c->vs.pos_cap = c->vs.pixels = 0;
    c->has_result = false;
}

int tpc::ctx_settle(tpc_ctx *c) {
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->ss || !c->carry_ub) return TPC_OK;
    uint32_t nc = 0;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(&nc, &c->ss->n_carry, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return TPC_ERR_CUDA;
    c->carry_ub = nc;   // the exact count: the next push's sizes follow it
    return TPC_OK;
}

cudaStream_t tpc::ctx_stream(tpc_ctx *c) { return c->stream; }
Tuning &tpc::ctx_tuning(tpc_ctx *c) { return c->tune; }
std::mutex &tpc::ctx_mutex(tpc_ctx *c) { return c->mu; }
size_t tpc::ctx_pending(tpc_ctx *c) { return c->pending; }
void tpc::ctx_sensor(tpc_ctx *c, uint32_t *width, uint32_t *height) {
    *width = c->width;
    *height = c->height;
}
int tpc::ctx_device(tpc_ctx *c) { return c->device; }

extern "C" {

int tpc_bind_outputs(tpc_ctx *c, uint64_t *labels, tpc_cluster *records, size_t cap) {
    if (!c || (labels == nullptr) != (records == nullptr) || (labels && !cap)) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->max_disorder != ~0ull) return TPC_ERR_STATE;   // one-shot steps only
    if (labels) {   // device memory of the context's device
        cudaPointerAttributes a{};
        for (const void *p : {(const void *)labels, (const void *)records})
            if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice ||
                a.device != c->device) {
                cudaGetLastError();
                return TPC_ERR_ARG;
            }
    }
    c->bound_labels = labels;
    c->bound_rec = records;
    c->bound_cap = labels ? cap : 0;
    return TPC_OK;
}

int tpc_variant_stats_get(tpc_ctx *c, tpc_variant_stats *out) {
    if (!c || !out) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->vstats_pending) {
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return TPC_ERR_CUDA;
        c->vstats.windowed = c->h_flag[0];
        c->vstats.window_fallbacks = c->h_flag[1];
        c->vstats.global_sweeps = c->h_flag[2];
        c->vstats_pending = false;
    }
    *out = c->vstats;
    return TPC_OK;
}

int tpc_device_bytes(tpc_ctx *c, size_t *bytes) {
    if (!c || !bytes) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    *bytes = c->device_bytes();
    return TPC_OK;
}

static_assert(sizeof(tpc_snapshot_header) == 64, "snapshot header layout");

int tpc_snapshot(tpc_ctx *c, void *buf, size_t cap, size_t *n_out) {
    if (!c || !n_out) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->max_disorder == ~0ull || !c->ss) return TPC_ERR_STATE;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return TPC_ERR_CUDA;
    if (c->has_result) {
        Prob p;
        if (cudaMemcpy(&p, c->res_prob, sizeof(Prob), cudaMemcpyDeviceToHost) != cudaSuccess) return TPC_ERR_CUDA;
        if (p.err) return map_err(p.err);
    }
    StreamState st;
    if (cudaMemcpy(&st, c->ss, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return TPC_ERR_CUDA;
    const size_t nc = c->sbuf[0] ? st.n_carry : 0;
    const size_t bytes = sizeof(tpc_snapshot_header) + nc * (sizeof(tpc_hit) + sizeof(uint64_t));
    *n_out = bytes;
    if (bytes > cap) return TPC_ERR_CAP;
    if (!buf) return TPC_ERR_ARG;
    tpc_snapshot_header h;
    std::memset(&h, 0, sizeof(h));
    h.magic = TPC_SNAPSHOT_MAGIC;
    h.version = TPC_SNAPSHOT_VERSION;
    h.width = c->width;
    h.height = c->height;
    h.dt = c->dt;
    h.max_disorder = c->max_disorder;
    h.pushed = c->pushed;
    h.seen_max = st.seen_max;
    h.watermark = st.watermark;
    h.has_seen = st.has_seen ? 1u : 0u;
    h.n_carry = (uint32_t)nc;
    char *out = static_cast<char *>(buf);
    std::memcpy(out, &h, sizeof(h));
    if (nc) {
        // the carry sits right-aligned in the buffer the next step reads
        const int next = 1 - c->scur;
        if (cudaMemcpy(out + sizeof(h), c->sbuf[next] + (c->carry_cap - nc), nc * sizeof(tpc_hit),
                       cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(out + sizeof(h) + nc * sizeof(tpc_hit), c->sgidx[next] + (c->carry_cap - nc),
                       nc * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return TPC_ERR_CUDA;
    }
    return TPC_OK;
}

int tpc_restore(tpc_ctx *c, const void *buf, size_t n) {
    if (!c || !buf || n < sizeof(tpc_snapshot_header)) return TPC_ERR_ARG;
    tpc_snapshot_header h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != TPC_SNAPSHOT_MAGIC || h.version != TPC_SNAPSHOT_VERSION) return TPC_ERR_ARG;
    if (n != sizeof(h) + (size_t)h.n_carry * (sizeof(tpc_hit) + sizeof(uint64_t))) return TPC_ERR_ARG;
    if (h.max_disorder == 0 || h.max_disorder == ~0ull || h.has_seen > 1) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(c->mu);
    if (h.width != c->width || h.height != c->height || h.dt != c->dt || c->variant != TPC_LOCAL)
        return TPC_ERR_ARG;
    if (c->pending || c->zc) return TPC_ERR_STATE;
    if (c->ss && c->carry_ub) {
        // carry_ub only bounds the carry: read the exact count
        uint32_t open = 0;
        if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
            cudaMemcpy(&open, &c->ss->n_carry, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            return TPC_ERR_CUDA;
        if (open) return TPC_ERR_STATE;
        c->carry_ub = 0;
    }
    if (!c->ss) {
        if (dev_alloc(&c->fail_alloc, (void **)&c->ss, sizeof(StreamState), c->stream, c->device) != cudaSuccess)
            return TPC_ERR_NOMEM;
        if (cudaMemsetAsync(c->ss, 0, sizeof(StreamState), c->stream) != cudaSuccess) return TPC_ERR_CUDA;
        c->scur = 1;
        c->carry_ub = 0;
    }
    // Room for the restored carry, grown while the device still holds an empty
    // carry (nothing is moved); then the open hits and the stream state.
    const size_t nc = h.n_carry;
    int rc = ensure_stream_buffers(c, nc);
    if (rc) return rc;
    StreamState st;
    std::memset(&st, 0, sizeof(st));
    st.n_carry = h.n_carry;
    st.has_seen = h.has_seen;
    st.seen_max = h.seen_max;
    st.watermark = h.watermark;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess ||
        cudaMemcpy(c->ss, &st, sizeof(st), cudaMemcpyHostToDevice) != cudaSuccess)
        return TPC_ERR_CUDA;
    if (nc) {
        const char *src = static_cast<const char *>(buf) + sizeof(h);
        const int next = 1 - c->scur;
        if (cudaMemcpy(c->sbuf[next] + (c->carry_cap - nc), src, nc * sizeof(tpc_hit), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(c->sgidx[next] + (c->carry_cap - nc), src + nc * sizeof(tpc_hit), nc * sizeof(uint64_t),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return TPC_ERR_CUDA;
    }
    c->max_disorder = h.max_disorder;
    c->carry_ub = nc;
    c->pushed = h.pushed;
    c->base = h.pushed;
    c->has_result = false;
    c->res_streaming = false;
    c->res_base = h.pushed;
    return TPC_OK;
}

const char *tpc_strerror(int status) {
    switch (status) {
    case TPC_OK: return "ok";
    case TPC_ERR_ARG: return "invalid argument";
    case TPC_ERR_RANGE: return "hit outside the sensor";
    case TPC_ERR_NOMEM: return "out of device or pinned memory";
    case TPC_ERR_BUSY: return "memory budget exceeded";
    case TPC_ERR_TIMEOUT: return "bounded device wait timed out";
    case TPC_ERR_CUDA: return "CUDA runtime error";
    case TPC_ERR_CAP: return "output buffer too small";
    case TPC_ERR_SPAN: return "ToA span of one step is 2^32 ticks or more";
    case TPC_ERR_LATE: return "hit later than max_disorder allows";
    case TPC_ERR_STATE: return "call not valid in the current state";
    default: return "unknown status";
    }
}

void tpc_destroy(tpc_ctx *c) {
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->ws.mem.release();   // stream-ordered frees, after the context's queued work
    c->outmem.release();
    c->vs.mem.release();
    dev_free(c->in, c->stream);
    for (int i = 0; i < 2; ++i) { dev_free(c->sbuf[i], c->stream); dev_free(c->sgidx[i], c->stream); }
    dev_free(c->ss, c->stream);
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->own_res_seg);
    cudaFree(c->own_res_prob);
    if (c->h_flag) cudaFreeHost(c->h_flag);
    if (c->h_seg) cudaFreeHost(c->h_seg);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    for (int i = 0; i < SEG_RING; ++i) if (c->seg_ev[i]) cudaEventDestroy(c->seg_ev[i]);
    if (c->stage_ev) cudaEventDestroy(c->stage_ev);
    if (c->done_ev) cudaEventDestroy(c->done_ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
