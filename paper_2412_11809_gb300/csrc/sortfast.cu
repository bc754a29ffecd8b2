// ToA ordering for t-ordered streams (Section 3.1: each hit arrives at most
// t late), in three kernels, with the general LSD radix sort (radix.cu) as
// the fallback:
//
//   k_tile_sort   every tile of TILE input positions is read once, whole
//                 records into shared memory, and sorted there by a block
//                 radix sort over the key bits
//                 that vary inside the tile; the sorted keys, positions,
//                 pixels and ToTs are written out, so no separate gather is
//                 needed.  Being the first pass over the hits, it also
//                 reduces the segment's ToA extremes and checks the pixels
//                 against the sensor (Algorithm 3, steps 1-2).
//   k_tile_merge  the second half of tile t-1 and the first half of tile t
//                 are merged.  If every hit lies less than TILE/2 positions
//                 from its place in (ToA, position) order, this completes the
//                 sort: after the first kernel, the prefix ending in the
//                 middle of any tile holds exactly the hits that belong
//                 there, so the windows straddling tile borders only need
//                 their own contents ordered.
//   k_sort_check  compares the neighbours at every window border; on any
//                 inversion the step is marked for the fallback (k_seg_finalize
//                 also sends it there when a ToA lies outside the tile sort's
//                 key range), whose kernels (make_keys, radix passes, gather)
//                 otherwise return at once.  The result is therefore exact
//                 for any input order.
#include "tpc_internal.cuh"

namespace tpc {

constexpr int LS_THREADS = 256;
constexpr int LS_WARPS = LS_THREADS / 32;
constexpr int LS_ITEMS = TILE / LS_THREADS;    // 16
constexpr int LS_WARP_SPAN = TILE / LS_WARPS;  // 512
constexpr uint16_t LS_NONE = 0xFFFFu;
constexpr int LS_BITS = 9;                     // digit width of the in-tile sort
constexpr int LS_RADIX = 1 << LS_BITS;         // 512 buckets: a 17-bit tile span in 2 passes

__device__ __forceinline__ uint32_t ls_lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t ls_match_digit(uint32_t d, uint32_t vmask) {
    uint32_t peers = vmask;
#pragma unroll
    for (int b = 0; b < LS_BITS; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

struct LsShared {
    uint32_t key[TILE];
    uint32_t pix[TILE];          // per local input index: x | y << 16 (read once, with the ToA)
    uint16_t tot[TILE];          // per local input index: ToT
    uint16_t idx[TILE];          // local input index of the element at each rank
    uint16_t wcnt[LS_WARPS][LS_RADIX];
    uint16_t dstart[LS_RADIX];
    uint32_t warp[32];
    uint32_t kmin[LS_WARPS], kmax[LS_WARPS];
    unsigned long long tmin[LS_WARPS], tmax[LS_WARPS], cmin[LS_WARPS];
};

constexpr int LS_SMEM = (int)sizeof(LsShared);

// Each record is read once, whole (16-byte loads); keys, pixels, ToTs and
// the permutation live in shared memory, and the output pass writes the
// sorted arrays from there, checking the pixels against the sensor.  The
// load phase also reduces the segment's ToA extremes (this pass is the
// first to see every hit).  Per pass a thread
// holds its 16 elements' local indices two to a register and each digit
// with its rank among the warp's equal digits in one register.
__global__ void __launch_bounds__(LS_THREADS, 3) k_tile_sort(Work w) {
    extern __shared__ __align__(16) unsigned char ls_raw[];
    LsShared &S = *reinterpret_cast<LsShared *>(ls_raw);
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = ls_lanemask_lt();
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint32_t n_t = end - begin;
        const tpc_hit *hits = g.hits + (begin - g.off);
        const uint64_t base = g.fast_base;
        const uint32_t new0 = g.n_carry > begin - g.off ? g.n_carry - (begin - g.off) : 0;   // first new hit
        uint32_t kmin = 0xFFFFFFFFu, kmax = 0;
        uint64_t tmin = ~0ull, tmax = 0, cmin = ~0ull;   // ToA extremes; minimum of the new hits
        constexpr int HALF = LS_ITEMS / 4;   // four batches of whole-record loads keep registers in bounds
#pragma unroll
        for (int hb = 0; hb < LS_ITEMS / HALF; ++hb) {
            uint4 tv[HALF];   // whole records: the pixel and ToT go to shared memory for the output
#pragma unroll
            for (int r = 0; r < HALF; ++r) {
                const uint32_t li = (hb * HALF + r) * LS_THREADS + threadIdx.x;
                if (li < n_t) tv[r] = ld_hit(hits + li);
            }
#pragma unroll
            for (int r = 0; r < HALF; ++r) {
                const uint32_t li = (hb * HALF + r) * LS_THREADS + threadIdx.x;
                if (li < n_t) {
                    const uint64_t toa = hit_toa(tv[r]);
                    S.pix[li] = tv[r].x;
                    S.tot[li] = (uint16_t)hit_tot(tv[r]);
                    const uint32_t key = (uint32_t)(toa - base);
                    tmin = toa < tmin ? toa : tmin;
                    tmax = toa > tmax ? toa : tmax;
                    if (li >= new0) cmin = toa < cmin ? toa : cmin;
                    S.key[li] = key;
                    S.idx[li] = (uint16_t)li;
                    kmin = key < kmin ? key : kmin;
                    kmax = key > kmax ? key : kmax;
                } else {
                    S.idx[li] = LS_NONE;
                }
            }
        }
        for (int o = 16; o; o >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
        }
        tmin = warp_min_u64(tmin);
        tmax = warp_max_u64(tmax);
        cmin = warp_min_u64(cmin);
        if (lane == 0) {
            S.kmin[warp] = kmin;
            S.kmax[warp] = kmax;
            S.tmin[warp] = tmin;
            S.tmax[warp] = tmax;
            S.cmin[warp] = cmin;
        }
        __syncthreads();
        for (int q = 0; q < LS_WARPS; ++q) { kmin = min(kmin, S.kmin[q]); kmax = max(kmax, S.kmax[q]); }
        if (threadIdx.x == 0) {   // the segment's ToA extremes (Algorithm 3, step 2)
            for (int q = 1; q < LS_WARPS; ++q) {
                tmin = S.tmin[q] < tmin ? S.tmin[q] : tmin;
                tmax = S.tmax[q] > tmax ? S.tmax[q] : tmax;
                cmin = S.cmin[q] < cmin ? S.cmin[q] : cmin;
            }
            Seg &gw = w.seg[w.tile_seg[t]];
            atomicMin(reinterpret_cast<unsigned long long *>(&gw.toa_min), (unsigned long long)tmin);
            atomicMax(reinterpret_cast<unsigned long long *>(&gw.toa_max), (unsigned long long)tmax);
            atomicMin(reinterpret_cast<unsigned long long *>(&gw.chunk_min), (unsigned long long)cmin);
        }
        const uint32_t span = kmax - kmin;
        const int passes = span ? (32 - __clz(span) + LS_BITS - 1) / LS_BITS : 0;

        for (int pass = 0; pass < passes; ++pass) {
            const int shift = pass * LS_BITS;
            uint32_t ii2[LS_ITEMS / 2];   // local indices, two per register
            uint32_t dr[LS_ITEMS];        // digit << 16 | rank among the warp's equal digits
#pragma unroll
            for (int r = 0; r < LS_ITEMS; ++r) {
                const uint32_t e = warp * LS_WARP_SPAN + r * 32 + lane;
                const uint32_t i = S.idx[e];
                if (r & 1) ii2[r >> 1] |= i << 16; else ii2[r >> 1] = i;
                // padding sorts last: digit RADIX-1 in every pass, after all real entries
                dr[r] = i == LS_NONE ? LS_RADIX - 1 : ((S.key[i] - kmin) >> shift) & (LS_RADIX - 1);
            }
            for (int i = threadIdx.x; i < LS_WARPS * LS_RADIX / 2; i += LS_THREADS)
                reinterpret_cast<uint32_t *>(&S.wcnt[0][0])[i] = 0;
            __syncthreads();
#pragma unroll
            for (int r = 0; r < LS_ITEMS; ++r) {
                const uint32_t d = dr[r];
                const uint32_t peers = ls_match_digit(d, 0xffffffffu);
                const uint32_t rank = __popc(peers & lt);
                const uint32_t pre = S.wcnt[warp][d];
                __syncwarp();
                if (rank == 0) S.wcnt[warp][d] = (uint16_t)(pre + __popc(peers));
                __syncwarp();
                dr[r] = d << 16 | (pre + rank);
            }
            __syncthreads();
            {   // per digit: prefix over warps; then exclusive scan of the digit totals
                // (LS_RADIX / LS_THREADS = 2 consecutive digits per thread)
                const uint32_t d0 = 2 * threadIdx.x;
                uint32_t tot2[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    uint32_t sum = 0;
#pragma unroll
                    for (int q = 0; q < LS_WARPS; ++q) {
                        const uint32_t c = S.wcnt[q][d0 + u];
                        S.wcnt[q][d0 + u] = (uint16_t)sum;
                        sum += c;
                    }
                    tot2[u] = sum;
                }
                const uint32_t both = tot2[0] + tot2[1];
                uint32_t x = both;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (lane == 31) S.warp[warp] = x;
                __syncthreads();
                uint32_t pre = 0;
                for (int q = 0; q < warp; ++q) pre += S.warp[q];
                S.dstart[d0] = (uint16_t)(pre + x - both);
                S.dstart[d0 + 1] = (uint16_t)(pre + x - both + tot2[0]);
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < LS_ITEMS; ++r) {
                const uint32_t d = dr[r] >> 16;
                const uint32_t i = (ii2[r >> 1] >> ((r & 1) * 16)) & 0xFFFFu;
                S.idx[S.dstart[d] + S.wcnt[warp][d] + (dr[r] & 0xFFFFu)] = (uint16_t)i;
            }
            __syncthreads();
        }
        bool bad = false;   // a hit outside the sensor
        const uint32_t W = g.width, H = g.height;
        for (uint32_t j = threadIdx.x; j < n_t; j += LS_THREADS) {
            const uint32_t li = S.idx[j];
            const uint32_t px = S.pix[li];   // x | y << 16
            bad |= (px & 0xFFFFu) >= W || (px >> 16) >= H;
            w.keys[0][begin + j] = S.key[li];
            w.vals[0][begin + j] = begin + li;
            w.spix[begin + j] = clamp_pix(px, W, H);
            w.stot[begin + j] = S.tot[li];
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&w.prob->err, E_RANGE);
    }
}

// Merge the second half of tile t-1 with the first half of tile t (both
// sorted by (key, position)), in place.
template <uint32_t CAP>
struct LmShared {
    uint32_t key[CAP];
    uint32_t pos[CAP];
    uint32_t pix[CAP];
    uint16_t tot[CAP];
    uint16_t rank[CAP];          // output rank of each moving element
    uint32_t cut[2];
};

// (key, position) of a below (key, position) of b
__device__ __forceinline__ bool lm_below(uint32_t ka, uint32_t pa, uint32_t kb, uint32_t pb) {
    return ka < kb || (ka == kb && pa < pb);
}

// Only the part of the window where the two halves interleave moves: A's
// elements above B's first and B's elements below A's last.  Keys and
// positions of a band of MERGE_BAND entries on each side of the border are
// read first, and the two cut points counted (A sorted, so the number of its
// elements below B's first is where B's first goes); the whole window is
// taken when the overlap reaches the band's edge.  Each moving element's
// output rank = its index in its own part + the number of the other part's
// elements that sort before it (binary search; the lanes of a warp search
// for neighbouring values, so their probes mostly coincide).  The moving
// elements' pixels and ToTs are staged in shared memory, so that the final
// pass can write every array straight to its output position.
constexpr uint32_t MERGE_BAND = TILE / 4;
// k_tile_merge<false> stages two bands (a small CTA, many per SM) and lists
// the borders whose overlap is wider than a band; k_tile_merge<true> takes
// those with the whole window (TILE / 2 on each side).
template <bool BIG>
constexpr int lm_smem() { return (int)sizeof(LmShared<BIG ? (uint32_t)TILE : 2 * MERGE_BAND>); }

template <bool BIG>
__global__ void __launch_bounds__(LS_THREADS) k_tile_merge(Work w) {
    extern __shared__ __align__(16) unsigned char lm_raw[];
    LmShared<BIG ? (uint32_t)TILE : 2 * MERGE_BAND> &S =
        *reinterpret_cast<LmShared<BIG ? (uint32_t)TILE : 2 * MERGE_BAND> *>(lm_raw);
    const Prob &P = *w.prob;
    const uint32_t nt = BIG ? P.merge_count : P.ntiles;   // the big kernel: the listed borders
    for (uint32_t u = blockIdx.x; u < nt; u += gridDim.x) {
        const uint32_t t = BIG ? w.redo[u] : u;
        const Seg &g = w.seg[w.tile_seg[t]];
        if (t == g.tile0) continue;
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint32_t nb_all = end - begin < TILE / 2 ? end - begin : TILE / 2;
        {   // already in order across the border?
            const uint32_t ka = w.keys[0][begin - 1], kb = w.keys[0][begin];
            if (ka < kb || (ka == kb && w.vals[0][begin - 1] < w.vals[0][begin])) continue;
        }
        {
            const uint32_t band = BIG ? TILE / 2 : MERGE_BAND;
            const uint32_t na = band, nb = band < nb_all ? band : nb_all;
            const uint32_t a0 = begin - na;   // A = [a0, begin), B = [begin, begin + nb)
            if (threadIdx.x < 2) S.cut[threadIdx.x] = 0;
            for (uint32_t j = threadIdx.x; j < na + nb; j += LS_THREADS) {
                S.key[j] = w.keys[0][a0 + j];
                S.pos[j] = w.vals[0][a0 + j];
            }
            __syncthreads();
            {   // ia = A elements below B[0]; ib = B elements below A[last]
                const uint32_t kb0 = S.key[na], pb0 = S.pos[na], kal = S.key[na - 1], pal = S.pos[na - 1];
                uint32_t ca = 0, cb = 0;
                for (uint32_t j = threadIdx.x; j < na; j += LS_THREADS)
                    ca += lm_below(S.key[j], S.pos[j], kb0, pb0);
                for (uint32_t j = threadIdx.x; j < nb; j += LS_THREADS)
                    cb += lm_below(S.key[na + j], S.pos[na + j], kal, pal);
                for (int o = 16; o; o >>= 1) {
                    ca += __shfl_xor_sync(0xffffffffu, ca, o);
                    cb += __shfl_xor_sync(0xffffffffu, cb, o);
                }
                if ((threadIdx.x & 31) == 0) {
                    if (ca) atomicAdd(&S.cut[0], ca);
                    if (cb) atomicAdd(&S.cut[1], cb);
                }
            }
            __syncthreads();
            const uint32_t ia = S.cut[0], ib = S.cut[1];
            const bool contained = (ia > 0 || na == TILE / 2) && (ib < nb || nb == nb_all);
            if (!BIG && !contained) {   // overlap wider than the band: the whole window, later
                if (threadIdx.x == 0) w.redo[atomicAdd(&w.prob->merge_count, 1u)] = t;
                __syncthreads();
                continue;
            }
            // moving part: A[ia, na) then B[0, ib) (indices in S); outputs a0 + ia ...
            const uint32_t ma = na - ia, m = ma + ib;
            for (uint32_t j = threadIdx.x; j < m; j += LS_THREADS) {
                const bool in_a = j < ma;
                const uint32_t src = in_a ? ia + j : na + (j - ma);
                const uint32_t kk = S.key[src], pp = S.pos[src];
                uint32_t lo = in_a ? na : ia, hi = in_a ? na + ib : na;   // the other part
                const uint32_t first = lo;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (lm_below(S.key[mid], S.pos[mid], kk, pp)) lo = mid + 1; else hi = mid;
                }
                S.rank[j] = (uint16_t)((in_a ? j : j - ma) + (lo - first));
                S.pix[src] = w.spix[a0 + src];
                S.tot[src] = w.stot[a0 + src];
            }
            __syncthreads();
            const uint32_t o0 = a0 + ia;
            for (uint32_t j = threadIdx.x; j < m; j += LS_THREADS) {
                const uint32_t src = j < ma ? ia + j : na + (j - ma);
                const uint32_t o = o0 + S.rank[j];
                w.keys[0][o] = S.key[src];
                w.vals[0][o] = S.pos[src];
                w.spix[o] = S.pix[src];
                w.stot[o] = S.tot[src];
            }
            __syncthreads();
        }
    }
}

// Borders between the sorted runs: mid-tile positions.  Any inversion sends
// the step to the general radix sort.
__global__ void __launch_bounds__(256) k_sort_check(Work w) {
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    bool bad = false;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint32_t s = begin + TILE / 2 - 1;
        if (s + 1 >= end) continue;
        const uint32_t ka = w.keys[0][s], kb = w.keys[0][s + 1];
        bad |= ka > kb || (ka == kb && w.vals[0][s] > w.vals[0][s + 1]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) w.prob->fallback = 1u;
}

cudaError_t init_sortfast_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_tile_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, LS_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tile_merge<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lm_smem<false>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_tile_merge<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lm_smem<true>());
}

void launch_sort_fast(const Work &w, const Launch &L) {
    k_tile_sort<<<L.fit(k_tile_sort, LS_THREADS, LS_SMEM, G_SORT), LS_THREADS, LS_SMEM, L.stream>>>(w);
    L.mark("k_tile_sort");
    k_tile_merge<false><<<L.fit(k_tile_merge<false>, LS_THREADS, lm_smem<false>(), G_SORT), LS_THREADS,
                          lm_smem<false>(), L.stream>>>(w);
    L.mark("k_tile_merge");
    k_tile_merge<true><<<L.fit(k_tile_merge<true>, LS_THREADS, lm_smem<true>(), G_SORT), LS_THREADS,
                         lm_smem<true>(), L.stream>>>(w);
    L.mark("k_tile_merge_big");
    k_sort_check<<<L.fit(k_sort_check, 256, 0), 256, 0, L.stream>>>(w);
    L.mark("k_sort_check");
}

}  // namespace tpc
