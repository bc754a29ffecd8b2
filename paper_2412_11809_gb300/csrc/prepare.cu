// Step set-up (Algorithm 3, steps 1-2: the hits arrive on the device), the
// per-segment decisions taken once the tile sort has seen every hit, and the
// general sort's keys and post-sort gather of pixel coordinates.
#include "tpc_internal.cuh"

namespace tpc {

// One CTA: lay the segments out in position space, reset per-step state and
// fill the tile -> segment table.  Streaming segments pick up the carry left
// by the previous step: it sits right-aligned in the carry region of their
// input buffer, immediately followed by the new chunk.
__global__ void k_setup(Work w, int nsegs) {
    __shared__ uint32_t s_tile0[MAX_SEGS + 1];
    if (threadIdx.x == 0) {
        uint32_t off = 0, tile = 0;
        for (int s = 0; s < nsegs; ++s) {
            Seg &g = w.seg[s];
            if (g.ss) {
                g.n_carry = g.ss->n_carry;
                g.hits = g.carry_in + (g.carry_cap - g.n_carry);
                g.carry_gidx = g.carry_gidx_in + (g.carry_cap - g.n_carry);
            } else {
                g.n_carry = 0;
                g.carry_gidx = nullptr;
            }
            g.n = g.n_carry + g.n_new;
            g.fast_base = fast_key_base(g);
            g.off = off;
            g.tile0 = tile;
            g.ntiles = (g.n + TILE - 1) / TILE;
            off += g.ntiles * TILE;
            tile += g.ntiles;
            g.toa_min = ~0ull;
            g.toa_max = 0;
            g.chunk_min = ~0ull;
            g.npasses = 0;
            g.watermark = 0;
            g.close_mode = CLOSE_NONE;
            g.seen_after = 0;
            g.n_final = g.n_clusters = g.n_open = 0;
            s_tile0[s] = g.tile0;
        }
        s_tile0[nsegs] = tile;
        Prob &p = *w.prob;
        p.nsegs = (uint32_t)nsegs;
        p.npasses = 0;
        p.fallback = 0;
        p.lsd_passes = 0;
        p.redo_count = 0;
        p.border_count = 0;
        p.merge_count = 0;
        p.err = 0;
        p.ntiles = tile;
        if (tile > p.tile_cap || off > p.pos_cap) {
            p.err |= E_CAP;
            p.ntiles = 0;
        }
    }
    __syncthreads();
    const uint32_t nt = w.prob->ntiles;
    for (uint32_t t = threadIdx.x; t < nt; t += blockDim.x) {
        int lo = 0, hi = nsegs - 1;   // last segment whose first tile <= t
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (s_tile0[mid] <= t) lo = mid; else hi = mid - 1;
        }
        w.tile_seg[t] = (uint32_t)lo;
    }
}

// One CTA, after the tile sort, merge and check: per-segment radix pass
// count, the ToA span check, the choice of sort (the tile sort's keys are
// relative to fast_key_base; if a ToA lies outside 2^32 ticks of that base,
// or the check found the tiles out of order, every segment takes the
// general sort with keys relative to its minimum ToA) and the streaming
// watermark.  A later hit j satisfies toa_j > seen_max - max_disorder (the
// t-ordered property, Section 3.1), and can join hit i only if
// toa_j - toa_i <= dt, so every cluster whose last ToA <=
// seen_max - max_disorder - dt is final.
__global__ void k_seg_finalize(Work w) {
    __shared__ uint32_t s_fallback;
    const uint32_t nsegs = w.prob->nsegs;
    if (threadIdx.x == 0) s_fallback = w.prob->fallback;
    __syncthreads();
    for (uint32_t s = threadIdx.x; s < nsegs; s += blockDim.x) {
        Seg &g = w.seg[s];
        uint32_t passes = 0;
        if (g.n) {
            uint64_t span = g.toa_max - g.toa_min;
            if (span >> 32) {
                atomicOr(&w.prob->err, E_SPAN);
            } else if (span) {
                uint32_t bits = 64 - __clzll((long long)span);
                passes = (bits + RADIX_BITS - 1) / RADIX_BITS;
            }
            const uint64_t fb = g.fast_base;
            if (g.toa_min < fb || g.toa_max - fb > 0xFFFFFFFFull) atomicOr(&s_fallback, 1u);
        }
        g.npasses = passes;
        atomicMax(&w.prob->lsd_passes, passes);   // used only by the general sort
        if (!g.ss) {
            g.close_mode = CLOSE_ALL;   // one-shot: the end of the stream
            continue;
        }
        StreamState &ss = *g.ss;
        const uint64_t md = g.max_disorder;   // ~0: a flush of a streaming context
        if (md != ~0ull && g.n_new && ss.has_seen && ss.seen_max >= md &&
            g.chunk_min <= ss.seen_max - md)
            atomicOr(&w.prob->err, E_LATE);
        uint64_t seen = ss.has_seen ? ss.seen_max : 0;
        if (g.n && g.toa_max > seen) seen = g.toa_max;
        g.seen_after = seen;
        const uint64_t lag = md + (uint64_t)g.dt;
        if (md == ~0ull) {
            g.close_mode = CLOSE_ALL;
        } else if (lag >= md && seen >= lag) {
            g.close_mode = CLOSE_WM;
            g.watermark = seen - lag;
        } else {
            g.close_mode = CLOSE_NONE;
        }
    }
    __syncthreads();
    const uint32_t fallback = s_fallback;
    for (uint32_t s = threadIdx.x; s < nsegs; s += blockDim.x) {
        Seg &g = w.seg[s];
        g.key_base = fallback || !g.n ? g.toa_min : g.fast_base;
    }
    if (threadIdx.x == 0 && fallback) {
        w.prob->fallback = 1u;
        w.prob->npasses = w.prob->lsd_passes;
    }
}

// Fallback path: keys[pos] = ToA - toa_min (32 bits), vals[pos] = pos.
__global__ void __launch_bounds__(256) k_make_keys(Work w) {
    if (!w.prob->fallback) return;
    const uint32_t nt = w.prob->ntiles;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint64_t base = g.toa_min;
        constexpr int U = 4;
        for (uint32_t p0 = begin + threadIdx.x; p0 < end; p0 += U * blockDim.x) {
            uint4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t pos = p0 + u * blockDim.x;
                if (pos < end) v[u] = ld_hit(g.hits + (pos - g.off));
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t pos = p0 + u * blockDim.x;
                if (pos < end) {
                    w.keys[0][pos] = (uint32_t)(hit_toa(v[u]) - base);
                    w.vals[0][pos] = pos;
                }
            }
        }
    }
}

// Fallback path: spix[s], stot[s] = pixel and ToT of the hit at sorted position s.
__global__ void __launch_bounds__(256) k_gather(Work w) {
    if (!w.prob->fallback) return;   // the tile sort wrote pixels and ToTs already
    const uint32_t nt = w.prob->ntiles;
    const uint32_t *vals = pick(w.vals, sorted_sel(*w.prob));
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        constexpr int ITEMS = TILE / 256;
        uint32_t pv[ITEMS];
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t s = begin + r * 256 + threadIdx.x;
            pv[r] = s < end ? vals[s] : 0;
        }
        uint2 px[ITEMS];
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t s = begin + r * 256 + threadIdx.x;
            px[r] = s < end ? __ldg(reinterpret_cast<const uint2 *>(g.hits + (pv[r] - g.off))) : make_uint2(0, 0);
        }
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t s = begin + r * 256 + threadIdx.x;
            if (s < end) {
                w.spix[s] = clamp_pix(px[r].x, g.width, g.height);   // x | y << 16
                w.stot[s] = (uint16_t)(px[r].y & 0xFFFFu);
            }
        }
    }
}

void launch_setup(const Work &w, int nsegs, const Launch &L) {
    k_setup<<<1, 1024, 0, L.stream>>>(w, nsegs);
    L.mark("k_setup");
}
void launch_seg_finalize(const Work &w, const Launch &L) {
    k_seg_finalize<<<1, 256, 0, L.stream>>>(w);
    L.mark("k_seg_finalize");
}
void launch_make_keys(const Work &w, const Launch &L) {
    k_make_keys<<<L.fit(k_make_keys, 256, 0), 256, 0, L.stream>>>(w);
    L.mark("k_make_keys");
}
void launch_gather(const Work &w, const Launch &L) {
    k_gather<<<L.fit(k_gather, 256, 0), 256, 0, L.stream>>>(w);
    L.mark("k_gather");
}

}  // namespace tpc
