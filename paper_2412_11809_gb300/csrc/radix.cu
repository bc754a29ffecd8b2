// Stable LSD radix sort of (ToA key, position) pairs, 8 bits per pass, per
// segment (Algorithm 3 step 3 names a parallel radix sort).  Reduce-then-scan
// with no inter-CTA waits: an upsweep counts digits per tile, a scan turns the
// [digit][tile] counts into per-segment offsets, a downsweep ranks each tile
// stably (warp match + popc), sorts it in shared memory and writes every
// digit run contiguously.  Passes beyond a segment's key width are skipped on
// the device, so the launch sequence does not depend on the data.
#include "tpc_internal.cuh"

namespace tpc {

constexpr int DS_THREADS = 256;
constexpr int DS_WARPS = DS_THREADS / 32;
constexpr int DS_ITEMS = TILE / DS_THREADS;   // 16
constexpr int DS_WARP_SPAN = TILE / DS_WARPS;  // 512 consecutive elements per warp

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of `vmask` holding the same 8-bit digit as this lane, from eight
// ballots (cheaper than match.any on this hardware).
__device__ __forceinline__ uint32_t match_digit(uint32_t d, uint32_t vmask) {
    uint32_t peers = vmask;
#pragma unroll
    for (int b = 0; b < RADIX_BITS; ++b) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// Exclusive scan of one value per thread over a CTA of NT threads.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = lane < NT / 32 ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < NT / 32) s_warp[lane] = s;
    }
    __syncthreads();
    total = s_warp[NT / 32 - 1];
    uint32_t prefix = (warp ? s_warp[warp - 1] : 0) + x - v;
    __syncthreads();
    return prefix;
}

__global__ void __launch_bounds__(256) k_radix_upsweep(Work w, int pass) {
    if ((uint32_t)pass >= w.prob->npasses) return;
    __shared__ uint32_t cnt[RADIX];
    const uint32_t nt = w.prob->ntiles, cap = w.prob->tile_cap;
    const uint32_t *keys = w.keys[pass & 1];
    const int shift = pass * RADIX_BITS;
    constexpr int ITEMS = TILE / 256;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        uint32_t kk[ITEMS];
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {   // all loads in flight before any use
            const uint32_t pos = begin + r * 256 + threadIdx.x;
            kk[r] = pos < end ? keys[pos] : 0;
        }
        cnt[threadIdx.x] = 0;
        __syncthreads();
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const uint32_t pos = begin + r * 256 + threadIdx.x;
            const bool valid = pos < end;
            const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
            const uint32_t d = (kk[r] >> shift) & (RADIX - 1);
            const uint32_t peers = match_digit(d, vmask);
            if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&cnt[d], __popc(peers));
        }
        __syncthreads();
        w.hist[threadIdx.x * cap + t] = cnt[threadIdx.x];
        __syncthreads();
    }
}

// One CTA per digit: exclusive scan of that digit's tile counts within each
// segment; per-segment digit totals go to segtot.
__global__ void __launch_bounds__(1024) k_radix_scan(Work w, int pass) {
    if ((uint32_t)pass >= w.prob->npasses) return;
    __shared__ uint32_t s_warp[32];
    const uint32_t d = blockIdx.x, cap = w.prob->tile_cap, nsegs = w.prob->nsegs;
    uint32_t *h = w.hist + d * cap;
    for (uint32_t s = 0; s < nsegs; ++s) {
        const Seg &g = w.seg[s];
        uint32_t running = 0;
        for (uint32_t c = 0; c < g.ntiles; c += blockDim.x) {
            const uint32_t t = g.tile0 + c + threadIdx.x;
            const bool valid = c + threadIdx.x < g.ntiles;
            uint32_t v = valid ? h[t] : 0, total;
            uint32_t ex = block_exclusive_scan<1024>(v, s_warp, total);
            if (valid) h[t] = running + ex;
            running += total;
        }
        if (threadIdx.x == 0) w.segtot[s * RADIX + d] = running;
    }
}

__global__ void __launch_bounds__(DS_THREADS) k_radix_downsweep(Work w, int pass) {
    if ((uint32_t)pass >= w.prob->npasses) return;
    __shared__ uint32_t s_keys[TILE];
    __shared__ uint32_t s_vals[TILE];
    __shared__ uint32_t s_wcnt[DS_WARPS][RADIX];
    __shared__ uint32_t s_dstart[RADIX];
    __shared__ uint32_t s_gbase[RADIX];
    __shared__ uint32_t s_warp[32];
    const uint32_t nt = w.prob->ntiles, cap = w.prob->tile_cap;
    const uint32_t *keys_in = w.keys[pass & 1], *vals_in = w.vals[pass & 1];
    uint32_t *keys_out = w.keys[(pass + 1) & 1], *vals_out = w.vals[(pass + 1) & 1];
    const int shift = pass * RADIX_BITS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = lanemask_lt();

    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const uint32_t si = w.tile_seg[t];
        const Seg &g = w.seg[si];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        const uint32_t n_t = end - begin;
        {   // global base of each digit run of this tile
            uint32_t tot, segex = block_exclusive_scan<DS_THREADS>(w.segtot[si * RADIX + threadIdx.x], s_warp, tot);
            s_gbase[threadIdx.x] = g.off + segex + w.hist[threadIdx.x * cap + t];
        }
        for (int i = threadIdx.x; i < DS_WARPS * RADIX; i += DS_THREADS) (&s_wcnt[0][0])[i] = 0;
        __syncthreads();

        uint32_t kk[DS_ITEMS], vv[DS_ITEMS], rr[DS_ITEMS];
#pragma unroll
        for (int r = 0; r < DS_ITEMS; ++r) {   // all loads in flight before the ranking
            const uint32_t idx = warp * DS_WARP_SPAN + r * 32 + lane;
            kk[r] = idx < n_t ? keys_in[begin + idx] : 0;
            vv[r] = idx < n_t ? vals_in[begin + idx] : 0;
        }
#pragma unroll
        for (int r = 0; r < DS_ITEMS; ++r) {
            const uint32_t idx = warp * DS_WARP_SPAN + r * 32 + lane;
            const bool valid = idx < n_t;
            const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
            const uint32_t key = kk[r], d = (key >> shift) & (RADIX - 1);
            const uint32_t peers = match_digit(d, vmask);
            uint32_t pre = 0, rank = 0;
            if (valid) {
                rank = __popc(peers & lt);
                pre = s_wcnt[warp][d];
            }
            __syncwarp();
            if (valid && rank == 0) s_wcnt[warp][d] = pre + __popc(peers);
            __syncwarp();
            rr[r] = pre + rank;
        }
        __syncthreads();
        {   // digit-major prefix over warps, then tile-local digit starts
            const uint32_t d = threadIdx.x;
            uint32_t sum = 0;
#pragma unroll
            for (int q = 0; q < DS_WARPS; ++q) {
                uint32_t c = s_wcnt[q][d];
                s_wcnt[q][d] = sum;
                sum += c;
            }
            uint32_t tot;
            s_dstart[d] = block_exclusive_scan<DS_THREADS>(sum, s_warp, tot);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < DS_ITEMS; ++r) {
            const uint32_t idx = warp * DS_WARP_SPAN + r * 32 + lane;
            if (idx < n_t) {
                const uint32_t d = (kk[r] >> shift) & (RADIX - 1);
                const uint32_t lpos = s_dstart[d] + s_wcnt[warp][d] + rr[r];
                s_keys[lpos] = kk[r];
                s_vals[lpos] = vv[r];
            }
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < n_t; j += DS_THREADS) {
            const uint32_t key = s_keys[j];
            const uint32_t d = (key >> shift) & (RADIX - 1);
            const uint32_t gpos = s_gbase[d] + (j - s_dstart[d]);
            keys_out[gpos] = key;
            vals_out[gpos] = s_vals[j];
        }
        __syncthreads();
    }
}

void launch_radix_pass(const Work &w, int pass, const Launch &L) {
    static const char *up[4] = {"k_radix_upsweep0", "k_radix_upsweep1", "k_radix_upsweep2", "k_radix_upsweep3"};
    static const char *sc[4] = {"k_radix_scan0", "k_radix_scan1", "k_radix_scan2", "k_radix_scan3"};
    static const char *dn[4] = {"k_radix_downsweep0", "k_radix_downsweep1", "k_radix_downsweep2",
                                "k_radix_downsweep3"};
    k_radix_upsweep<<<L.fit(k_radix_upsweep, 256, 0), 256, 0, L.stream>>>(w, pass);
    L.mark(up[pass & 3]);
    k_radix_scan<<<RADIX, 1024, 0, L.stream>>>(w, pass);
    L.mark(sc[pass & 3]);
    k_radix_downsweep<<<L.fit(k_radix_downsweep, DS_THREADS, 0), DS_THREADS, 0, L.stream>>>(w, pass);
    L.mark(dn[pass & 3]);
}

}  // namespace tpc
