// Neighbour search and union-find hooking (Algorithm 3 steps 4-5, Section 4.1)
// for the edge-connectivity variant (iii)(a).
//
// Hits are in (ToA, position) order.  For hit i and each of its 9 pixels p
// (8 neighbours plus its own), let L(i, p) be the latest earlier hit on p.
// Joining i to L(i, p) whenever toa(i) - toa(L) <= dt yields the same
// components as joining every pair within dt: an earlier hit j on p with
// toa(i) - toa(j) <= dt reaches L(i, p) through the chain of consecutive
// hits on p, all of which lie between toa(j) and toa(i) and are therefore
// joined to one another.  This is the paper's "reference to the last hit at
// each pixel" (Algorithm 3 step 4) made data parallel.
//
// k_tile_link: one CTA per tile of TILE sorted hits.  The tile's pixels are
// staged in shared memory as packed keys (pixel << 12 | rank), sorted, and
// L(i, p) inside the tile is a binary search for the predecessor of
// (p, rank(i)).  Unions run on a shared-memory forest and the tile's roots
// are written to the global forest (roots = earliest hit).
//
// k_border_link: edges whose earlier end lies before the tile (the paper's
// step 5, "border hits at the start of the next chunk").  The halo is every
// earlier hit within dt of the tile's first hit; the front is every tile hit
// within dt of the halo's last hit.  The latest halo hit on each pixel is
// found in a shared-memory sorted copy of the halo, processed in batches when
// the halo is large; unions run on the global forest.
//
// k_flatten: full path compression; records each position's root and
// initialises the per-root feature slots.
#include "tpc_internal.cuh"

namespace tpc {

constexpr int LINK_THREADS = 512;
constexpr int LINK_RANK_BITS = 12;            // TILE = 4096 ranks
constexpr int HALO_BATCH = 2048;
constexpr int HALO_RANK_BITS = 11;
constexpr int BORDER_THREADS = 256;

static_assert((1 << LINK_RANK_BITS) == TILE, "tile rank bits");

// In-place ascending bitonic sort of n (power of two) 32-bit keys.
__device__ __forceinline__ void bitonic_sort(uint32_t *v, uint32_t n) {
    for (uint32_t k = 2; k <= n; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const uint32_t a = v[i], b = v[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { v[i] = b; v[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

// Number of entries of the ascending array v[0..n) that are < target (n a
// power of two).
__device__ __forceinline__ uint32_t count_less(const uint32_t *v, uint32_t n, uint32_t target) {
    uint32_t pos = 0;
    for (uint32_t step = n >> 1; step > 0; step >>= 1)
        if (v[pos + step - 1] < target) pos += step;
    if (v[pos] < target) pos += 1;
    return pos;
}

__global__ void __launch_bounds__(LINK_THREADS) k_tile_link(Work w) {
    extern __shared__ uint32_t smem[];
    uint32_t *s_key = smem;             // [TILE] keys of the tile (rank order)
    uint32_t *s_pix = s_key + TILE;     // [TILE] x | y << 16
    uint32_t *s_v = s_pix + TILE;       // [TILE] pixel << 12 | rank, sorted
    uint32_t *s_par = s_v + TILE;       // [TILE] shared-memory forest

    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    const uint32_t *skey = w.keys[sorted_sel(P)];
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint32_t n_t = end - begin, W = g.width, H = g.height, dt = g.dt;
        for (uint32_t k = threadIdx.x; k < TILE; k += LINK_THREADS) {
            if (k < n_t) {
                const uint32_t pix = w.spix[begin + k];
                const uint32_t pid = (pix >> 16) * W + (pix & 0xFFFFu);
                s_key[k] = skey[begin + k];
                s_pix[k] = pix;
                s_v[k] = (pid << LINK_RANK_BITS) | k;
            } else {
                s_v[k] = 0xFFFFFFFFu;
            }
            s_par[k] = k;
        }
        __syncthreads();
        bitonic_sort(s_v, TILE);
        for (uint32_t k = threadIdx.x; k < n_t; k += LINK_THREADS) {
            const uint32_t pix = s_pix[k], key = s_key[k];
            const int x = (int)(pix & 0xFFFFu), y = (int)(pix >> 16);
            for (int dy = -1; dy <= 1; ++dy) {
                const int ny = y + dy;
                if (ny < 0 || ny >= (int)H) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int nx = x + dx;
                    if (nx < 0 || nx >= (int)W) continue;
                    const uint32_t p = (uint32_t)ny * W + (uint32_t)nx;
                    const uint32_t c = count_less(s_v, TILE, (p << LINK_RANK_BITS) | k);
                    if (c == 0) continue;
                    const uint32_t e = s_v[c - 1];
                    if ((e >> LINK_RANK_BITS) != p) continue;
                    const uint32_t j = e & (TILE - 1);
                    if (key - s_key[j] <= dt) sunion(s_par, k, j);
                }
            }
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < n_t; k += LINK_THREADS)
            w.parent[begin + k] = begin + sfind(s_par, k);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(BORDER_THREADS) k_border_link(Work w) {
    __shared__ uint32_t b_v[HALO_BATCH];
    __shared__ uint32_t b_key[HALO_BATCH];
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    const uint32_t *skey = w.keys[sorted_sel(P)];
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        if (t == g.tile0) continue;   // nothing before the segment's first tile
        uint32_t s0, end;
        tile_range(g, t, s0, end);
        const uint32_t W = g.width, H = g.height, dt = g.dt;
        // halo: [h0, s0) = earlier hits with key >= key(s0) - dt (a suffix)
        const uint32_t k0 = skey[s0];
        const uint32_t lo_key = k0 >= dt ? k0 - dt : 0;
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
        const uint64_t hi64 = (uint64_t)skey[s0 - 1] + dt;
        const uint32_t hi_key = hi64 > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)hi64;
        uint32_t e0 = s0;
        while (e0 < end) {
            const uint32_t chunk = end - e0 < BORDER_THREADS ? end - e0 : BORDER_THREADS;
            const uint32_t p = e0 + threadIdx.x;
            const bool in = threadIdx.x < chunk && skey[p] <= hi_key;
            const uint32_t cnt = (uint32_t)__syncthreads_count(in);
            e0 += cnt;
            if (cnt < chunk) break;
        }
        for (uint32_t hb = h0; hb < s0; hb += HALO_BATCH) {
            const uint32_t nb = s0 - hb < HALO_BATCH ? s0 - hb : HALO_BATCH;
            uint32_t np2 = 2;
            while (np2 < nb) np2 <<= 1;
            for (uint32_t j = threadIdx.x; j < np2; j += BORDER_THREADS) {
                if (j < nb) {
                    const uint32_t pix = w.spix[hb + j];
                    const uint32_t pid = (pix >> 16) * W + (pix & 0xFFFFu);
                    b_v[j] = (pid << HALO_RANK_BITS) | j;
                    b_key[j] = skey[hb + j];
                } else {
                    b_v[j] = 0xFFFFFFFFu;
                }
            }
            __syncthreads();
            bitonic_sort(b_v, np2);
            for (uint32_t i = s0 + threadIdx.x; i < e0; i += BORDER_THREADS) {
                const uint32_t pix = w.spix[i], key = skey[i];
                const int x = (int)(pix & 0xFFFFu), y = (int)(pix >> 16);
                for (int dy = -1; dy <= 1; ++dy) {
                    const int ny = y + dy;
                    if (ny < 0 || ny >= (int)H) continue;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int nx = x + dx;
                        if (nx < 0 || nx >= (int)W) continue;
                        const uint32_t p = (uint32_t)ny * W + (uint32_t)nx;
                        // latest halo hit on p: the largest entry below (p + 1) << bits
                        const uint32_t c = count_less(b_v, np2, (p + 1) << HALO_RANK_BITS);
                        if (c == 0) continue;
                        const uint32_t e = b_v[c - 1];
                        if ((e >> HALO_RANK_BITS) != p) continue;
                        const uint32_t j = e & (HALO_BATCH - 1);
                        if (key - b_key[j] <= dt) gunion(w.parent, i, hb + j);
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_flatten(Work w) {
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    const uint32_t *sidx = w.vals[sorted_sel(P)];
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        for (uint32_t s = begin + threadIdx.x; s < end; s += blockDim.x) {
            const uint32_t r = gfind(w.parent, s);
            w.root_of[sidx[s]] = r;
            if (r == s) {
                w.slot_size[r] = 0;
                w.slot_min[r] = 0xFFFFFFFFu;
                w.slot_maxkey[r] = 0;
                w.slot_tot[r] = 0;
                w.slot_wx[r] = 0;
                w.slot_wy[r] = 0;
            }
        }
    }
}

constexpr int TILE_LINK_SMEM = 4 * TILE * (int)sizeof(uint32_t);

cudaError_t init_kernel_attributes() {
    return cudaFuncSetAttribute(k_tile_link, cudaFuncAttributeMaxDynamicSharedMemorySize, TILE_LINK_SMEM);
}

void launch_link(const Work &w, const Launch &L) {
    const int smem = TILE_LINK_SMEM;
    k_tile_link<<<L.grid, LINK_THREADS, smem, L.stream>>>(w);
    k_border_link<<<L.grid, BORDER_THREADS, 0, L.stream>>>(w);
    k_flatten<<<L.grid, 256, 0, L.stream>>>(w);
}

}  // namespace tpc
