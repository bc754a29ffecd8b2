// Per-cluster features, canonical labels and stream compaction.
//
// k_accumulate walks the hits in (ToA, position) order and reduces size,
// sum ToT, sum ToT*x, sum ToT*y, smallest position and largest key into the
// root's slot, privatised in shared memory per span of sorted positions.
// Integer sums are exact; the centroid is one division of exact sums
// (features are the purpose named in Section 1: on-the-fly filtering and
// compression; Algorithm 3 step 6 orders clusters by time, here records are
// ordered by label instead).
//
// k_labels writes label = global index of the smallest position of the
// cluster and sets two bit flags per position (label hit of a finalised
// cluster; hit of a finalised cluster) with one ballot per warp.
// k_tile_scan turns per-tile flag counts into per-segment offsets;
// k_records and k_stream_compact write the compacted outputs and, when
// streaming, the carry of open hits for the next step.
#include "tpc_internal.cuh"

namespace tpc {

constexpr int ACC_THREADS = 512;
// Sorted positions per pass (ACC_SPAN): 1024 by default (measured best on
// the 256x256 stream); 512 and 2048 are tuning choices.
template <int ACC_SPAN>
constexpr int acc_smem() {
    return 2 * ACC_SPAN * (int)sizeof(uint32_t) + 3 * ACC_SPAN * (int)sizeof(unsigned long long);
}

// Roots and features in (ToA, position) order, where a cluster's hits sit
// close together.  Each pass over ACC_SPAN sorted positions finds every
// position's root (the global forest is shallow after the tile links),
// records it by input position for the label pass, and sums into shared-
// memory slots of the roots inside the span (a root precedes its cluster's
// hits); hits of one cluster within a warp are combined first (match.any +
// redux) when there are three or more of them, so a burst of one track does
// not serialise on one slot, while the small groups of a dense stream (where
// each group's reductions would run one group after another) add their hits
// one by one.  One
// partial per root then goes to the global slots; hits whose root lies
// before the span go there directly.  The global slots of tile roots were
// zeroed by the tile-link kernels.  Size and sum ToT share one 64-bit
// shared-memory counter (size << 32 | sum ToT: a span holds at most ACC_SPAN
// hits of ToT < 2^16, so neither part overflows), and the last key is kept
// only when a streaming watermark needs it.
template <int ACC_SPAN>
__global__ void __launch_bounds__(ACC_THREADS, ACC_SPAN >= 2048 ? 2 : 4) k_accumulate(Work w) {
    constexpr int ACC_ITEMS = ACC_SPAN / ACC_THREADS;
    extern __shared__ __align__(16) unsigned char acc_raw[];
    unsigned long long *a_wx = reinterpret_cast<unsigned long long *>(acc_raw);
    unsigned long long *a_wy = a_wx + ACC_SPAN, *a_st = a_wy + ACC_SPAN;
    uint32_t *a_min = reinterpret_cast<uint32_t *>(a_st + ACC_SPAN), *a_max = a_min + ACC_SPAN;
    static_assert((unsigned long long)ACC_SPAN * 0xFFFFu < (1ull << 32), "packed sum ToT fits 32 bits");
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    const uint32_t *skey = pick(w.keys, sorted_sel(P));
    const uint32_t *sidx = pick(w.vals, sorted_sel(P));
    const int lane = threadIdx.x & 31;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const bool want_max = g.close_mode == CLOSE_WM;
        for (uint32_t b = begin; b < end; b += ACC_SPAN) {
            const uint32_t e = b + ACC_SPAN < end ? b + ACC_SPAN : end;
            uint32_t rr[ACC_ITEMS], px[ACC_ITEMS], tt[ACC_ITEMS], kk[ACC_ITEMS], ps[ACC_ITEMS];
#pragma unroll
            for (int q = 0; q < ACC_ITEMS; ++q) {   // every load in flight before any use
                const uint32_t s = b + q * ACC_THREADS + threadIdx.x;
                if (s < e) {
                    rr[q] = w.parent[s];
                    px[q] = w.spix[s];
                    tt[q] = w.stot[s];
                    kk[q] = want_max ? skey[s] : 0u;   // the last key only matters when streaming
                    ps[q] = sidx[s];
                }
            }
            uint32_t p2[ACC_ITEMS];
#pragma unroll
            for (int q = 0; q < ACC_ITEMS; ++q) {   // second hop for every item at once
                const uint32_t s = b + q * ACC_THREADS + threadIdx.x;
                p2[q] = s < e && rr[q] != s ? w.parent[rr[q]] : rr[q];
            }
#pragma unroll
            for (int q = 0; q < ACC_ITEMS; ++q) {
                const uint32_t s = b + q * ACC_THREADS + threadIdx.x;
                if (s >= e) continue;
                // parent[s] is s's tile root; that root is global unless a border
                // link hooked it (then follow the rest of the path)
                const uint32_t r = p2[q] == rr[q] ? rr[q] : gfind(w.parent, p2[q]);
                rr[q] = r;
                w.root_of[ps[q]] = r;
                if (r == s) {
                    const uint32_t k = s - b;
                    a_st[k] = a_wx[k] = a_wy[k] = 0;
                    a_min[k] = 0xFFFFFFFFu;
                    a_max[k] = 0;
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < ACC_ITEMS; ++q) {
                const uint32_t s = b + q * ACC_THREADS + threadIdx.x;
                const bool valid = s < e;
                const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
                if (!valid) continue;
                const uint32_t r = rr[q], pix = px[q], tot = tt[q];
                const uint32_t peers = __match_any_sync(vmask, r);
                const uint32_t cnt = __popc(peers);
                uint32_t sum_tot = tot, mn = ps[q], mx = kk[q];
                unsigned long long wx = (unsigned long long)tot * (pix & 0xFFFFu);
                unsigned long long wy = (unsigned long long)tot * (pix >> 16);
                // combine this cluster's hits of the warp when there are
                // enough of them to contend; smaller groups add their hits
                // one by one (a group reduction runs once per distinct group)
                const bool agg = cnt >= 3u;
                uint32_t c = 1;
                if (agg) {
                    const uint32_t wx32 = tot * (pix & 0xFFFFu), wy32 = tot * (pix >> 16);
                    sum_tot = __reduce_add_sync(peers, tot);
                    wx = ((unsigned long long)__reduce_add_sync(peers, wx32 >> 16) << 16) +
                         __reduce_add_sync(peers, wx32 & 0xFFFFu);
                    wy = ((unsigned long long)__reduce_add_sync(peers, wy32 >> 16) << 16) +
                         __reduce_add_sync(peers, wy32 & 0xFFFFu);
                    mn = __reduce_min_sync(peers, mn);
                    if (want_max) mx = __reduce_max_sync(peers, mx);
                    c = cnt;
                    if (lane != __ffs(peers) - 1) continue;
                }
                if (r >= b) {
                    const uint32_t k = r - b;
                    atomicAdd(&a_st[k], (unsigned long long)c << 32 | sum_tot);
                    atomicAdd(&a_wx[k], wx);
                    atomicAdd(&a_wy[k], wy);
                    atomicMin(&a_min[k], mn);
                    if (want_max) atomicMax(&a_max[k], mx);
                } else {
                    Slot &sl = w.slot[r];
                    atomicAdd(&sl.size, c);
                    atomicAdd(&sl.tot, (unsigned long long)sum_tot);
                    atomicAdd(&sl.wx, wx);
                    atomicAdd(&sl.wy, wy);
                    atomicMin(&sl.min, mn);
                    if (want_max) atomicMax(&sl.maxkey, mx);
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < ACC_ITEMS; ++q) {
                const uint32_t k = q * ACC_THREADS + threadIdx.x;
                const uint32_t r = b + k;
                if (r < e && rr[q] == r) {
                    Slot &sl = w.slot[r];
                    const unsigned long long st = a_st[k];
                    atomicAdd(&sl.size, (uint32_t)(st >> 32));
                    atomicAdd(&sl.tot, st & 0xFFFFFFFFull);
                    atomicAdd(&sl.wx, a_wx[k]);
                    atomicAdd(&sl.wy, a_wy[k]);
                    atomicMin(&sl.min, a_min[k]);
                    if (want_max) atomicMax(&sl.maxkey, a_max[k]);
                }
            }
            // no barrier here: the next span re-initialises shared slot k only in
            // the thread that has just flushed it (the same k = q * ACC_THREADS +
            // thread mapping), before its first barrier, and no other thread
            // touches slot k until after that barrier
        }
    }
}

__device__ __forceinline__ bool cluster_closed(const Seg &g, uint32_t maxkey) {
    if (g.close_mode == CLOSE_ALL) return true;
    if (g.close_mode == CLOSE_NONE) return false;
    return g.key_base + (uint64_t)maxkey <= g.watermark;
}

__global__ void __launch_bounds__(256) k_labels(Work w) {
    __shared__ uint32_t s_cnt[2];
    const uint32_t nt = w.prob->ntiles;
    const int lane = threadIdx.x & 31;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const bool direct = g.ss == nullptr;   // one-shot: every hit is final
        if (threadIdx.x < 2) s_cnt[threadIdx.x] = 0;
        __syncthreads();
        uint32_t c_label = 0, c_closed = 0;
        constexpr int PARTS = 4;                 // fewer registers, more resident warps
        constexpr int ITEMS = TILE / 256 / PARTS;
        for (int part = 0; part < PARTS; ++part) {
            const uint32_t base = begin + part * (ITEMS * 256);
            uint32_t rr[ITEMS], ll[ITEMS], mk[ITEMS];
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const uint32_t pos = base + q * 256 + threadIdx.x;
                rr[q] = pos < end ? w.root_of[pos] : 0;
            }
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const uint32_t pos = base + q * 256 + threadIdx.x;
                ll[q] = pos < end ? w.slot[rr[q]].min : 0;
                mk[q] = pos < end && g.close_mode == CLOSE_WM ? w.slot[rr[q]].maxkey : 0;
            }
#pragma unroll
            for (int q = 0; q < ITEMS; ++q) {
                const uint32_t pos = base + q * 256 + threadIdx.x;
                const bool valid = pos < end;
                bool is_label = false, closed = false;
                if (valid) {
                    const uint32_t l = ll[q];
                    closed = cluster_closed(g, mk[q]);
                    is_label = closed && l == pos;
                    const uint64_t lab = gidx_of(g, l - g.off);
                    if (direct) g.out_labels[pos - g.off] = lab;
                    else w.lab_tmp[pos] = lab;
                }
                const uint32_t bl = __ballot_sync(0xffffffffu, is_label);
                const uint32_t bc = __ballot_sync(0xffffffffu, valid && closed);
                if (lane == 0) {
                    w.flag_label[pos >> 5] = bl;
                    w.flag_closed[pos >> 5] = bc;
                    c_label += __popc(bl);
                    c_closed += __popc(bc);
                }
            }
        }
        if (lane == 0) {
            atomicAdd(&s_cnt[0], c_label);
            atomicAdd(&s_cnt[1], c_closed);
        }
        __syncthreads();
        if (threadIdx.x < 2) w.tile_cnt[threadIdx.x * w.prob->tile_cap + t] = s_cnt[threadIdx.x];
        __syncthreads();
    }
}

// One CTA per segment: exclusive scans of the tile counts; totals.
__global__ void __launch_bounds__(1024) k_tile_scan(Work w) {
    __shared__ uint32_t s_warp[32];
    const uint32_t s = blockIdx.x;
    if (s >= w.prob->nsegs) return;
    Seg &g = w.seg[s];
    const uint32_t cap = w.prob->tile_cap;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int kind = 0; kind < 2; ++kind) {
        uint32_t running = 0;
        for (uint32_t c = 0; c < g.ntiles; c += blockDim.x) {
            const uint32_t t = g.tile0 + c + threadIdx.x;
            const bool valid = c + threadIdx.x < g.ntiles;
            const uint32_t v = valid ? w.tile_cnt[kind * cap + t] : 0;
            uint32_t x = v;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_warp[warp] = x;
            __syncthreads();
            if (warp == 0) {
                uint32_t q = s_warp[lane];
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(0xffffffffu, q, o);
                    if (lane >= o) q += y;
                }
                s_warp[lane] = q;
            }
            __syncthreads();
            const uint32_t ex = (warp ? s_warp[warp - 1] : 0) + x - v;
            if (valid) w.tile_base[kind * cap + t] = running + ex;
            running += s_warp[31];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (kind == 0) g.n_clusters = running;
            else { g.n_final = running; g.n_open = g.n - running; }
        }
    }
    if (threadIdx.x == 0 && g.n_clusters > g.out_cap) atomicOr(&w.prob->err, E_CAP);
}

// One thread per flag word (TILE / 32 = 128 words per tile).
__global__ void __launch_bounds__(TILE_WORDS) k_records(Work w) {
    __shared__ uint32_t s_warp[TILE_WORDS / 32];
    const uint32_t nt = w.prob->ntiles, cap = w.prob->tile_cap;
    const uint32_t *skey = pick(w.keys, sorted_sel(*w.prob));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint32_t nwords = (end - begin + 31) >> 5;
        uint32_t bits = threadIdx.x < nwords ? w.flag_label[(begin >> 5) + threadIdx.x] : 0;
        const uint32_t c = __popc(bits);
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (int q = 0; q < warp; ++q) wpre += s_warp[q];
        uint32_t ord = w.tile_base[t] + wpre + x - c;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const uint32_t pos = begin + (threadIdx.x << 5) + b;
            const uint32_t r = w.root_of[pos];
            if (ord < g.out_cap) {
                tpc_cluster rec;
                rec.label = gidx_of(g, pos - g.off);
                const Slot sl = w.slot[r];
                rec.size = (int64_t)sl.size;
                rec.sum_tot = (int64_t)sl.tot;
                rec.first_toa = g.key_base + skey[r];
                // fp32 quotient of the exact integer sums: three roundings, each
                // at most 2^-24 relative (FP64 is a slow pipe on this GPU)
                const float sw = (float)sl.tot;
                rec.cx = (float)sl.wx / sw;
                rec.cy = (float)sl.wy / sw;
                g.out_rec[ord] = rec;
            }
            ++ord;
        }
        __syncthreads();
    }
    (void)cap;
}

// Streaming: finalised hits -> (label, index) in increasing global index;
// open hits -> the next step's carry, right aligned in its carry region.
__global__ void __launch_bounds__(TILE_WORDS) k_stream_compact(Work w) {
    __shared__ uint32_t s_warp[TILE_WORDS / 32];
    const uint32_t nt = w.prob->ntiles, cap = w.prob->tile_cap;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        if (!g.ss) continue;
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint32_t nwords = (end - begin + 31) >> 5;
        const bool vw = threadIdx.x < nwords;
        const uint32_t bits = vw ? w.flag_closed[(begin >> 5) + threadIdx.x] : 0;
        const uint32_t c = __popc(bits);
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t wpre = 0;
        for (int q = 0; q < warp; ++q) wpre += s_warp[q];
        const uint32_t closed_before = w.tile_base[cap + t] + wpre + x - c;
        const bool carry_fits = g.n_open <= g.carry_cap;
        if (!carry_fits && threadIdx.x == 0) atomicOr(&w.prob->err, E_CAP);
        if (vw) {
            const uint32_t first = begin + (threadIdx.x << 5);
            const uint32_t last = first + 32 < end ? first + 32 : end;
            uint32_t k_closed = 0;
            for (uint32_t pos = first; pos < last; ++pos) {
                const uint32_t local = pos - g.off;
                const bool cl = (bits >> (pos - first)) & 1u;
                if (cl) {
                    const uint32_t ord = closed_before + k_closed++;
                    if (ord < g.out_cap) {
                        g.out_labels[ord] = w.lab_tmp[pos];
                        if (g.out_index) g.out_index[ord] = gidx_of(g, local);
                    }
                } else if (carry_fits) {
                    const uint32_t open_rank = local - (closed_before + k_closed);
                    const uint32_t dst = g.carry_cap - g.n_open + open_rank;
                    g.carry_out[dst] = g.hits[local];
                    g.carry_gidx_out[dst] = gidx_of(g, local);
                }
            }
        }
        __syncthreads();
    }
}

__global__ void k_stream_end(Work w) {
    const uint32_t nsegs = w.prob->nsegs;
    for (uint32_t s = threadIdx.x; s < nsegs; s += blockDim.x) {
        Seg &g = w.seg[s];
        if (!g.ss) continue;
        StreamState &ss = *g.ss;
        if (g.n_open > g.carry_cap) atomicOr(&w.prob->err, E_CAP);
        ss.n_carry = g.n_open <= g.carry_cap ? g.n_open : 0;
        ss.seen_max = g.seen_after;
        ss.has_seen = ss.has_seen || g.n != 0;
        if (g.close_mode == CLOSE_WM) ss.watermark = g.watermark;
    }
}

cudaError_t init_features_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_accumulate<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         acc_smem<512>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_accumulate<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, acc_smem<1024>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_accumulate<2048>, cudaFuncAttributeMaxDynamicSharedMemorySize, acc_smem<2048>());
    return e;
}

template <int SPAN>
static void launch_accumulate(const Work &w, const Launch &L) {
    k_accumulate<SPAN><<<L.fit(k_accumulate<SPAN>, ACC_THREADS, acc_smem<SPAN>(), G_ACC), ACC_THREADS,
                         acc_smem<SPAN>(), L.stream>>>(w);
}

void launch_features(const Work &w, const Launch &L) {
    if (L.tune.acc_span == 512) launch_accumulate<512>(w, L);
    else if (L.tune.acc_span == 2048) launch_accumulate<2048>(w, L);
    else launch_accumulate<1024>(w, L);
    L.mark("k_accumulate");
}

void launch_outputs(const Work &w, const Launch &L) {
    k_labels<<<L.fit(k_labels, 256, 0, G_OUT), 256, 0, L.stream>>>(w);
    L.mark("k_labels");
    k_tile_scan<<<MAX_SEGS, 1024, 0, L.stream>>>(w);
    L.mark("k_tile_scan");
    k_records<<<L.fit(k_records, TILE_WORDS, 0, G_OUT), TILE_WORDS, 0, L.stream>>>(w);
    L.mark("k_records");
    k_stream_compact<<<L.fit(k_stream_compact, TILE_WORDS, 0, G_OUT), TILE_WORDS, 0, L.stream>>>(w);
    L.mark("k_stream_compact");
    k_stream_end<<<1, 256, 0, L.stream>>>(w);
    L.mark("k_stream_end");
}

}  // namespace tpc
