// Variants (iii)(b) and (iii)(c) of the cluster definition (paper Section 2),
// read as the time sweep of Algorithm 1: in (ToA, index) order a hit merges
// every still-open cluster with a member on one of its 9 pixels; (b) open =
// last ToA >= toa - dt, (c) open = first ToA >= toa - dt.  Both start from
// the components of variant (a), already in the global forest.
//
// (c): every (c) join is an (a) edge (the joined member lies between the
// cluster's first hit and the new hit, so within dt of it), hence (c)
// clusters split (a) components and each component can be swept on its own.
// Components are grouped by a stable radix sort on their root (keeping ToA
// order inside); one thread sweeps each component, looking back only over
// hits within dt (older members belong to clusters that are closed).
//
// (b): a closed cluster never reopens, so at any moment every open cluster
// with a member on pixel p also contains the latest hit on p (that hit joined
// it on arrival), and a (b) cluster is open exactly on [first, last + dt].
// The sweep's result is therefore the least partition, reached from the (a)
// components by merging, in which hit h is joined to L = the latest earlier
// hit on each of its 9 pixels whenever toa(h) <= last(group(L)) + dt.
// Rounds apply that rule: the first to every hit's 9 latest neighbours, the
// later ones to the edges still open, with the groups' last ToA kept at the
// roots by the unions (a lagging value only postpones a merge) and
// recomputed exactly when a round merges nothing; the partition is final
// after a round without merges on exact values.  The rounds join (a)
// components, each by a dense id; per-pixel timelines come from a stable
// radix sort of the hits by pixel.
#include "tpc_internal.cuh"

namespace tpc {

__device__ __forceinline__ bool adjacent_v(uint32_t a, uint32_t b) {
    const int dx = (int)(a & 0xFFFFu) - (int)(b & 0xFFFFu);
    const int dy = (int)(a >> 16) - (int)(b >> 16);
    return dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1;
}

// grouping keys: (c) the (a) root of each sorted position; (b) its pixel id
__global__ void __launch_bounds__(256) k_var_keys(Work w, VarWork v, int by_pixel) {
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    const uint32_t *sroot = pick(w.keys, sorted_sel(P) ^ 1u);
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        for (uint32_t s = begin + threadIdx.x; s < end; s += blockDim.x) {
            const uint32_t pix = w.spix[s];
            v.k[0][s] = by_pixel ? (pix >> 16) * g.width + (pix & 0xFFFFu) : sroot[s];
            v.v[0][s] = s;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *v.prob = P;
        v.prob->npasses = by_pixel ? 3 : 4;   // pixel ids < 2^20; roots < 2^32
    }
}

// find with path halving, for a forest owned by one thread
__device__ __forceinline__ uint32_t seq_find(uint32_t *par, uint32_t x) {
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

// (c): one warp per component of the root-grouped order (components are
// contiguous there, in ToA order).  The sweep is sequential over the
// component's hits, but each step is warp-wide: for hit i the lanes take the
// earlier hits within dt (32 at a time, newest first), test adjacency and
// whether the cluster of that hit is still open (its root, the earliest hit,
// within dt of i), and every open cluster found is joined under the earliest
// of their roots, together with i.  Whether a cluster is open does not
// depend on the joins made for i itself (a join only unites open clusters,
// and the result is open), so the lanes may test their candidates at once.
// Components of up to SW_CAP hits are staged in shared memory; larger ones
// run on the grouped arrays in global memory.  Warps take chunks of SW_CHUNK
// grouped positions from a counter and sweep every component that starts in
// their chunk.
constexpr int SW_WARPS = 8;
constexpr uint32_t SW_CAP = 512;
constexpr uint32_t SW_CHUNK = 32;

template <bool STAGED>
struct SweepView {
    const uint32_t *sk, *sp;   // staged keys and pixels (STAGED)
    uint32_t *sc;              // parent per component index (staged or global)
    const uint32_t *skey, *spix, *gv;
    uint32_t q;                // first grouped position of the component
    __device__ uint32_t key(uint32_t i) const { return STAGED ? sk[i] : skey[gv[q + i]]; }
    __device__ uint32_t pix(uint32_t i) const { return STAGED ? sp[i] : spix[gv[q + i]]; }
    __device__ uint32_t find(uint32_t x) const {   // path halving
        volatile uint32_t *c = sc;
        while (true) {
            const uint32_t p = c[x];
            if (p == x) return x;
            const uint32_t gp = c[p];
            if (gp == p) return p;
            c[x] = gp;
            x = gp;
        }
    }
};

template <bool STAGED>
__device__ void sweep_component(const SweepView<STAGED> &V, uint32_t n, uint32_t dt, int lane) {
    for (uint32_t i = lane; i < n; i += 32) V.sc[i] = i;
    __syncwarp();
    for (uint32_t i = 1; i < n; ++i) {
        const uint32_t ki = V.key(i), pi = V.pix(i);
        uint32_t root = 0xFFFFFFFFu;   // the earliest open root joined so far
        for (uint32_t base = 0; base < i; base += 32) {
            const bool valid = base + lane < i;
            const uint32_t j = valid ? i - 1 - base - lane : 0;
            const bool in = valid && ki - V.key(j) <= dt;
            if (!__any_sync(0xffffffffu, in)) break;   // keys only fall further back
            uint32_t r = 0xFFFFFFFFu;
            if (in && adjacent_v(pi, V.pix(j))) {
                const uint32_t rj = V.find(j);
                if (ki - V.key(rj) <= dt) r = rj;   // that cluster is still open
            }
            const uint32_t m = __reduce_min_sync(0xffffffffu, r);
            __syncwarp();
            if (m != 0xFFFFFFFFu) {
                const uint32_t target = m < root ? m : root;
                if (r != 0xFFFFFFFFu && r != target) V.sc[r] = target;
                if (lane == 0 && root != 0xFFFFFFFFu && root != target) V.sc[root] = target;
                root = target;
            }
            __syncwarp();
        }
        if (lane == 0 && root != 0xFFFFFFFFu) V.sc[i] = root;
        __syncwarp();
    }
}

// Components of more than SW_CAP hits: the same sweep over a sliding window
// of the component's last SW_CAP hits in shared memory (slot = index mod
// SW_CAP).  A (c) cluster spans at most dt, so while every hit within dt of
// the hit being swept is still in the window, a hit that leaves it belongs
// to a cluster that is closed for every later hit: its root is final.  On
// leaving, its root goes to global memory (cpar, by component index, and
// the parent array); finds that reach a hit that has left read it there.  A
// batch of 32 hits enters every 32 steps, pushing the 32 oldest out; if one
// of those is within dt of the first newcomer, the window is too small
// (returns false): the component is listed for k_static_sweep_big, which
// sweeps it again with a whole CTA, staged in shared memory up to BIG_CAP
// hits, from global memory beyond.
template <uint32_t CAP>
struct WindowView {
    uint32_t *wk, *wp, *wc;    // window: key, pixel, parent (component index)
    uint32_t *cpar;            // global: final root of each hit that left
    uint32_t lo;               // first component index still in the window
    __device__ uint32_t key(uint32_t i) const { return wk[i % CAP]; }
    __device__ uint32_t pix(uint32_t i) const { return wp[i % CAP]; }
    __device__ uint32_t find(uint32_t x) const {
        volatile uint32_t *c = wc;
        while (true) {
            if (x < lo) return *reinterpret_cast<volatile uint32_t *>(&cpar[x]);
            const uint32_t p = c[x % CAP];
            if (p == x) return x;
            if (p < lo) return *reinterpret_cast<volatile uint32_t *>(&cpar[p]);
            const uint32_t gp = c[p % CAP];
            if (gp == p) return p;
            c[x % CAP] = gp;
            x = gp;
        }
    }
};

template <uint32_t CAP>
__device__ bool sweep_windowed(WindowView<CAP> V, const uint32_t *skey, const uint32_t *spix, const uint32_t *gv,
                               uint32_t *parent, uint32_t q0, uint32_t n, uint32_t dt, int lane) {
    for (uint32_t i = 0; i < n; ++i) {
        if ((i & 31u) == 0) {   // hits [i, i + 32) enter, [i - CAP, i - CAP + 32) leave
            const uint32_t ki = skey[gv[q0 + i]];
            if (i >= CAP) {
                const uint32_t j = i - CAP + lane;   // < i <= n - 1
                if (__any_sync(0xffffffffu, ki - V.key(j) <= dt)) return false;
                const uint32_t r = V.find(j);
                __syncwarp();
                V.cpar[j] = r;
                parent[gv[q0 + j]] = gv[q0 + r];
                __syncwarp();
                V.lo = i - CAP + 32;
            }
            const uint32_t e = i + lane;
            if (e < n) {
                const uint32_t se = gv[q0 + e];
                V.wk[e % CAP] = skey[se];
                V.wp[e % CAP] = spix[se];
                V.wc[e % CAP] = e;
            }
            __syncwarp();
        }
        if (i == 0) continue;
        const uint32_t ki = V.key(i), pi = V.pix(i);
        uint32_t root = 0xFFFFFFFFu;   // the earliest open root joined so far
        for (uint32_t base = 0; base < i; base += 32) {
            const bool valid = base + lane < i && i - 1 - base - lane >= V.lo;
            const uint32_t j = valid ? i - 1 - base - lane : i;
            const bool in = valid && ki - V.key(j) <= dt;
            if (!__any_sync(0xffffffffu, in)) break;   // keys only fall further back
            uint32_t r = 0xFFFFFFFFu;
            if (in && adjacent_v(pi, V.pix(j))) {
                const uint32_t rj = V.find(j);
                if (rj >= V.lo && ki - V.key(rj) <= dt) r = rj;   // that cluster is still open
            }
            const uint32_t m = __reduce_min_sync(0xffffffffu, r);
            __syncwarp();
            if (m != 0xFFFFFFFFu) {
                const uint32_t target = m < root ? m : root;
                if (r != 0xFFFFFFFFu && r != target) V.wc[r % CAP] = target;
                if (lane == 0 && root != 0xFFFFFFFFu && root != target) V.wc[root % CAP] = target;
                root = target;
            }
            __syncwarp();
        }
        if (lane == 0 && root != 0xFFFFFFFFu) V.wc[i % CAP] = root;
        __syncwarp();
    }
    // the hits still in the window
    const uint32_t first = V.lo;
    for (uint32_t j = first + lane; j < n; j += 32) {
        const uint32_t r = V.find(j);
        parent[gv[q0 + j]] = gv[q0 + r];
    }
    return true;
}

__global__ void __launch_bounds__(SW_WARPS * 32) k_static_sweep(Work w, VarWork v) {
    __shared__ uint32_t s_k[SW_WARPS][SW_CAP], s_p[SW_WARPS][SW_CAP], s_c[SW_WARPS][SW_CAP];
    const uint32_t *skey = pick(w.keys, sorted_sel(*w.prob));
    const uint32_t sel = v.prob->npasses & 1u;
    const uint32_t *gk = pick(v.k, sel), *gv = pick(v.v, sel);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Seg &g = w.seg[0];
    const uint32_t first = g.off, last = g.off + g.n, dt = g.dt;
    const uint32_t nchunks = (g.n + SW_CHUNK - 1) / SW_CHUNK;
    while (true) {
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(v.work, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= nchunks) break;
        const uint32_t q = first + c * SW_CHUNK + lane;
        uint32_t starts = __ballot_sync(0xffffffffu, q < last && (q == first || gk[q] != gk[q - 1]));
        while (starts) {
            const uint32_t q0 = first + c * SW_CHUNK + (__ffs(starts) - 1);
            starts &= starts - 1;
            // the component's end: the first grouped position with another root
            const uint32_t key0 = gk[q0];
            uint32_t n = 0;
            for (uint32_t p0 = q0 + 1;; p0 += 32) {
                const uint32_t p = p0 + lane;
                const uint32_t stop = __ballot_sync(0xffffffffu, p >= last || gk[p] != key0);
                if (stop) { n = p0 + (__ffs(stop) - 1) - q0; break; }
            }
            if (n == 1) {
                if (lane == 0) w.parent[gv[q0]] = gv[q0];
                continue;
            }
            if (n <= SW_CAP) {
                for (uint32_t i = lane; i < n; i += 32) {
                    const uint32_t si = gv[q0 + i];
                    s_k[warp][i] = skey[si];
                    s_p[warp][i] = w.spix[si];
                }
                __syncwarp();
                const SweepView<true> V{s_k[warp], s_p[warp], s_c[warp], skey, w.spix, gv, q0};
                sweep_component(V, n, dt, lane);
                for (uint32_t i = lane; i < n; i += 32) w.parent[gv[q0 + i]] = gv[q0 + V.find(i)];
            } else {
                const WindowView<SW_CAP> WV{s_k[warp], s_p[warp], s_c[warp], v.cpar + q0, 0};
                if (lane == 0) atomicAdd(&v.changed[0], 1u);   // diagnostics: windowed components
                if (!sweep_windowed(WV, skey, w.spix, gv, w.parent, q0, n, dt, lane)) {
                    if (lane == 0) {   // more than the window within dt: the big window's list
                        const uint32_t k = atomicAdd(&v.changed[1], 1u);
                        v.big[k] = make_uint2(q0, n);   // k < positions / SW_CAP: each has > SW_CAP hits
                    }
                    __syncwarp();
                }
            }
            __syncwarp();   // the staging is rewritten for the next component
        }
    }
}

// (c): components whose hits within dt outgrew the warp's window.  One CTA
// per component, the component staged whole in dynamic shared memory (up to
// BIG_CAP hits; from global memory beyond): the same sweep, with each
// step's candidates (the earlier hits within dt) spread over the CTA's
// threads instead of one warp's lanes, the earliest open root found by a
// shared-memory minimum.
constexpr int BIG_THREADS = 512;
constexpr uint32_t BIG_CAP = 8192;
constexpr int BIG_SMEM = 3 * BIG_CAP * (int)sizeof(uint32_t);

template <bool STAGED>
__device__ void sweep_block(const SweepView<STAGED> &V, uint32_t n, uint32_t dt, uint32_t *s_min) {
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) V.sc[i] = i;
    if (threadIdx.x < 2) s_min[threadIdx.x] = 0xFFFFFFFFu;
    __syncthreads();
    uint32_t it = 0;   // iterations so far: s_min[it & 1] collects this one's minimum
    for (uint32_t i = 1; i < n; ++i) {
        const uint32_t ki = V.key(i), pi = V.pix(i);
        uint32_t root = 0xFFFFFFFFu;   // the earliest open root joined so far (the same in every thread)
        for (uint32_t base = 0; base < i; base += blockDim.x, ++it) {
            const bool valid = base + threadIdx.x < i;
            const uint32_t j = valid ? i - 1 - base - threadIdx.x : 0;
            const bool in = valid && ki - V.key(j) <= dt;
            uint32_t r = 0xFFFFFFFFu;
            if (in && adjacent_v(pi, V.pix(j))) {
                const uint32_t rj = V.find(j);
                if (ki - V.key(rj) <= dt) r = rj;   // that cluster is still open
            }
            uint32_t *mn = s_min + (it & 1u);
            if (r != 0xFFFFFFFFu) atomicMin(mn, r);
            const bool any_in = __syncthreads_or(in);
            const uint32_t m = *reinterpret_cast<volatile uint32_t *>(mn);
            if (threadIdx.x == 0) s_min[(it + 1) & 1u] = 0xFFFFFFFFu;   // read by nobody until the next barrier
            if (m != 0xFFFFFFFFu) {
                const uint32_t target = m < root ? m : root;
                if (r != 0xFFFFFFFFu && r != target) V.sc[r] = target;
                if (threadIdx.x == 0 && root != 0xFFFFFFFFu && root != target) V.sc[root] = target;
                root = target;
            }
            __syncthreads();
            if (!any_in) { ++it; break; }   // keys only fall further back
        }
        if (threadIdx.x == 0 && root != 0xFFFFFFFFu) V.sc[i] = root;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(BIG_THREADS) k_static_sweep_big(Work w, VarWork v) {
    extern __shared__ uint32_t big_raw[];
    __shared__ uint32_t s_min[2];
    const uint32_t *skey = pick(w.keys, sorted_sel(*w.prob));
    const uint32_t *gv = pick(v.v, v.prob->npasses & 1u);
    const uint32_t dt = w.seg[0].dt, nbig = v.changed[1];
    for (uint32_t k = blockIdx.x; k < nbig; k += gridDim.x) {
        const uint2 job = v.big[k];
        const uint32_t q0 = job.x, n = job.y;
        if (n <= BIG_CAP) {
            uint32_t *sk = big_raw, *sp = big_raw + BIG_CAP, *sc = big_raw + 2 * BIG_CAP;
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                const uint32_t si = gv[q0 + i];
                sk[i] = skey[si];
                sp[i] = w.spix[si];
            }
            __syncthreads();
            const SweepView<true> V{sk, sp, sc, skey, w.spix, gv, q0};
            sweep_block(V, n, dt, s_min);
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) w.parent[gv[q0 + i]] = gv[q0 + V.find(i)];
        } else {
            if (threadIdx.x == 0) atomicAdd(&v.changed[2], 1u);   // diagnostics: swept from global memory
            const SweepView<false> V{nullptr, nullptr, v.cpar + q0, skey, w.spix, gv, q0};
            sweep_block(V, n, dt, s_min);
            for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) w.parent[gv[q0 + i]] = gv[q0 + V.find(i)];
        }
        __syncthreads();   // the staging is rewritten for the next component
    }
}

cudaError_t init_variants_attributes() {
    return cudaFuncSetAttribute(k_static_sweep_big, cudaFuncAttributeMaxDynamicSharedMemorySize, BIG_SMEM);
}

// (b): pixel histogram and its exclusive scan (single segment).
__global__ void __launch_bounds__(256) k_pixel_hist(Work w, VarWork v) {
    const Prob &P = *w.prob;
    const uint32_t nt = P.ntiles;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        for (uint32_t s = begin + threadIdx.x; s < end; s += blockDim.x) {
            const uint32_t pix = w.spix[s];
            atomicAdd(&v.pix_start[(pix >> 16) * g.width + (pix & 0xFFFFu) + 1], 1u);
        }
    }
}

__global__ void __launch_bounds__(1024) k_pixel_scan(Work w, VarWork v) {
    __shared__ uint32_t s_warp[32];
    const Seg &g = w.seg[0];
    const uint32_t np = g.width * g.height;   // entries 1..np hold counts
    const uint32_t per = (np + blockDim.x - 1) / blockDim.x;
    const uint32_t i0 = 1 + threadIdx.x * per;
    uint32_t local = 0;
    for (uint32_t i = i0; i < i0 + per && i <= np; ++i) local += v.pix_start[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t run = x - local;
    for (int q = 0; q < warp; ++q) run += s_warp[q];
    for (uint32_t i = i0; i < i0 + per && i <= np; ++i) {
        run += v.pix_start[i];
        v.pix_start[i] = run;
    }
}

// (b) takes the (a) components as its units: they get dense ids in the
// order of their roots (sorted positions), and the rounds find and join on
// a forest over those ids (cpar_d, with each group's last key at its root
// in clast), a tenth of the hits' count, mostly held in L2, instead of on
// the forest over sorted positions.  A component's own last key (clast0)
// is fixed.  The roots of the sorted positions after the (a) links are
// those k_sorted_roots left in the idle radix buffer.

// Components per tile: the roots among its positions.
__global__ void __launch_bounds__(256) k_comp_count(Work w, VarWork v) {
    __shared__ uint32_t s_cnt;
    const uint32_t nt = w.prob->ntiles;
    const uint32_t *sroot = pick(w.keys, sorted_sel(*w.prob) ^ 1u);
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        if (threadIdx.x == 0) s_cnt = 0;
        __syncthreads();
        uint32_t c = 0;
        for (uint32_t s = begin + threadIdx.x; s < end; s += blockDim.x) c += sroot[s] == s ? 1u : 0u;
        c = __reduce_add_sync(0xffffffffu, c);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s_cnt, c);
        __syncthreads();
        if (threadIdx.x == 0) v.tcnt[t] = s_cnt;
        __syncthreads();   // s_cnt is reset for the next tile
    }
}

// One CTA: exclusive scan of the tile counts; the total is the id count.
__global__ void __launch_bounds__(1024) k_comp_scan(Work w, VarWork v) {
    __shared__ uint32_t s_warp[32];
    const uint32_t nt = w.prob->ntiles;
    const uint32_t per = (nt + blockDim.x - 1) / blockDim.x;
    const uint32_t i0 = threadIdx.x * per;
    uint32_t local = 0;
    for (uint32_t i = i0; i < i0 + per && i < nt; ++i) local += v.tcnt[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t run = x - local;
    for (int q = 0; q < warp; ++q) run += s_warp[q];
    for (uint32_t i = i0; i < i0 + per && i < nt; ++i) {
        v.tbase[i] = run;
        run += v.tcnt[i];
    }
    if (threadIdx.x == blockDim.x - 1) *v.ncomp = run;
}

// Dense ids in root order: a root's id is the roots before it.  Each id
// starts as its own group.
__global__ void __launch_bounds__(256) k_comp_ids(Work w, VarWork v) {
    constexpr int ITEMS = TILE / 256;
    __shared__ uint32_t s_pre[TILE / 32];   // roots per 32 positions, then their exclusive prefix
    const uint32_t nt = w.prob->ntiles;
    const uint32_t *sroot = pick(w.keys, sorted_sel(*w.prob) ^ 1u);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const Seg &g = w.seg[w.tile_seg[t]];
        uint32_t begin, end;
        tile_range(g, t, begin, end);
        uint32_t m[ITEMS];
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {   // position begin + q * 256 + threadIdx.x: word q * 8 + warp
            const uint32_t s = begin + q * 256 + threadIdx.x;
            m[q] = __ballot_sync(0xffffffffu, s < end && sroot[s] == s);
            if (lane == 0) s_pre[q * 8 + warp] = __popc(m[q]);
        }
        __syncthreads();
        if (warp == 0) {   // 128 words, 4 per lane
            uint32_t c[4], sum = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) { c[k] = s_pre[lane * 4 + k]; sum += c[k]; }
            uint32_t x = sum;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            uint32_t run = x - sum;
#pragma unroll
            for (int k = 0; k < 4; ++k) { s_pre[lane * 4 + k] = run; run += c[k]; }
        }
        __syncthreads();
        const uint32_t base = v.tbase[t];
#pragma unroll
        for (int q = 0; q < ITEMS; ++q) {
            if (!((m[q] >> lane) & 1u)) continue;
            const uint32_t s = begin + q * 256 + threadIdx.x;
            const uint32_t c = base + s_pre[q * 8 + warp] + __popc(m[q] & ((1u << lane) - 1u));
            v.cid_at[s] = c;
            v.croot[c] = s;
            v.cpar_d[c] = c;
            v.clast0[c] = 0;
        }
        __syncthreads();   // s_pre is rewritten for the next tile
    }
}

// Each component's last key; only hits that could raise the stored value
// issue the atomic (a long component would serialise on one address).
__global__ void __launch_bounds__(256) k_comp_last(Work w, VarWork v) {
    const Seg &g = w.seg[0];
    const uint32_t *skey = pick(w.keys, sorted_sel(*w.prob));
    const uint32_t *sroot = pick(w.keys, sorted_sel(*w.prob) ^ 1u);
    for (uint32_t s = g.off + blockIdx.x * blockDim.x + threadIdx.x; s < g.off + g.n; s += gridDim.x * blockDim.x) {
        const uint32_t c = v.cid_at[sroot[s]], k = skey[s];
        if (*reinterpret_cast<volatile uint32_t *>(&v.clast0[c]) < k) atomicMax(&v.clast0[c], k);
    }
}

// Before a full round: each hit's state, (sorted position, id of its
// group's root, that group's last key, its key), first in position order
// (coalesced but for the ids, whose roots lie near), then gathered into
// pixel-timeline order, one 16-byte read per hit.  The groups and last keys
// are those of the moment (the last keys exact at the first round, lagging
// later): every rule applied to them is one the sweep applies.  flat: the
// first round, where every group is one component (and starts here).
__global__ void __launch_bounds__(256) k_position_state(Work w, VarWork v, int flat) {
    const Seg &g = w.seg[0];
    const uint32_t *skey = pick(w.keys, sorted_sel(*w.prob));
    const uint32_t *sroot = pick(w.keys, sorted_sel(*w.prob) ^ 1u);
    for (uint32_t s = g.off + blockIdx.x * blockDim.x + threadIdx.x; s < g.off + g.n; s += gridDim.x * blockDim.x) {
        const uint32_t r = sroot[s], c0 = v.cid_at[r];
        uint32_t c = c0, last;
        if (flat) {
            last = v.clast0[c0];
            if (r == s) v.clast[c0] = last;
        } else {
            c = gfind(v.cpar_d, c0);
            last = *reinterpret_cast<volatile uint32_t *>(&v.clast[c]);
        }
        v.pstate[s] = make_uint4(s, c, last, skey[s]);
    }
}

__global__ void __launch_bounds__(256) k_timeline_state(Work w, VarWork v) {
    const Seg &g = w.seg[0];
    const uint32_t *tl = pick(v.v, v.prob->npasses & 1u) + g.off;
    uint4 *T = v.tline + g.off;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < g.n; j += gridDim.x * blockDim.x)
        T[j] = v.pstate[tl[j]];
}

// Exact last keys of the groups (when a round merged nothing): reset at
// the roots, then each id's own last key raised into its root's.
__global__ void __launch_bounds__(256) k_group_last_reset(VarWork v) {
    const uint32_t n = *v.ncomp;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        if (v.cpar_d[c] == c) v.clast[c] = 0;
}

__global__ void __launch_bounds__(256) k_group_last(VarWork v) {
    const uint32_t n = *v.ncomp;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const uint32_t f = gfind(v.cpar_d, c), k = v.clast0[c];
        if (*reinterpret_cast<volatile uint32_t *>(&v.clast[f]) < k) atomicMax(&v.clast[f], k);
    }
}

// The result on the hits' forest: each component's root hooked under its
// group's root (an earlier position: ids follow the roots' order).
__global__ void __launch_bounds__(256) k_comp_parents(Work w, VarWork v) {
    const uint32_t n = *v.ncomp;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const uint32_t f = gfind(v.cpar_d, c);
        if (f != c) w.parent[v.croot[c]] = v.croot[f];
    }
}

// (b) with the groups' last keys kept at their roots during the unions: when
// root b is hooked under a, a's last key takes b's (atomicMax).  A value can
// lag behind its group's (a concurrent hook of a loses it), never exceed it,
// so every union made on it is one the sweep makes; an exact recomputation
// when a round merges nothing decides the end.
__device__ __forceinline__ bool gunion_last(uint32_t *parent, uint32_t *glast, uint32_t a, uint32_t b) {
    while (true) {
        a = gfind(parent, a);
        b = gfind(parent, b);
        if (a == b) return false;
        if (a > b) { const uint32_t t = a; a = b; b = t; }
        if (atomicCAS(parent + b, b, a) == b) {
            const uint32_t lb = *reinterpret_cast<volatile uint32_t *>(&glast[b]);
            if (*reinterpret_cast<volatile uint32_t *>(&glast[a]) < lb) atomicMax(&glast[a], lb);
            return true;
        }
    }
}

// Append the warp's open edges (a node of h's group, a node of its
// neighbour's group, h's key) to list `out` (one atomic per warp); on
// overflow the list is marked and the next round takes every hit again.
__device__ __forceinline__ void push_edges(const VarWork &v, int out, bool keep, uint32_t a, uint32_t b,
                                           uint32_t key) {
    uint2 *list = pick(v.edges, out);
    uint32_t *keys = pick(v.ekey, out);
    const uint32_t m = __ballot_sync(0xffffffffu, keep);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;   // 64 bits: a full round can push more than 2^32 edges
    if (lane == __ffs(m) - 1) base = atomicAdd(&v.ecount[out], (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    const unsigned long long slot = base + __popc(m & ((1u << lane) - 1u));
    if (keep) {
        if (slot < v.edge_cap) {
            list[slot] = make_uint2(a, b);
            keys[slot] = key;
        } else {
            v.changed[1] = 1u;
        }
    }
}

// The latest entry of timeline [q0, q1) (ascending positions) before
// position s, for the 32 lanes of a warp whose positions ascend with the
// lane index: a 32-way search for lane 0's, then a window of the 32 entries
// from the one before it, each lane's answer in it by five shuffles; a lane
// whose answer lies past the window searches the rest alone.  All lanes
// call it with the same q0, q1.
__device__ __forceinline__ void lane_latest(const uint32_t *tl, const uint4 *T, uint32_t a, uint32_t b,
                                            uint32_t s, uint4 &nb, bool &has) {
    const uint32_t a0 = a;
    while (a < b) {   // first entry of [a, b) at or after s
        const uint32_t mid = (a + b) >> 1;
        if (tl[mid] < s) a = mid + 1; else b = mid;
    }
    if (a > a0) {
        nb = T[a - 1];
        has = true;
    }
}

__device__ __forceinline__ void warp_latest(const uint32_t *tl, const uint4 *T, uint32_t q0, uint32_t q1,
                                            uint32_t s, int lane, uint4 &nb, bool &has) {
    const uint32_t s0 = __shfl_sync(0xffffffffu, s, 0);
    uint32_t lo = q0, hi = q1;   // the first entry at or after s0 lies in [lo, hi] (hi = q1: none)
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) >> 5, idx = lo + (uint32_t)lane * step;
        const int c = __popc(__ballot_sync(0xffffffffu, idx < hi && tl[idx] < s0));   // a prefix of the lanes
        if (c == 0) { hi = lo; break; }
        const uint32_t below = lo + (uint32_t)(c - 1) * step;
        lo = below + 1;
        hi = min(below + step, hi);
    }
    if (hi > lo) lo += __popc(__ballot_sync(0xffffffffu, lo + lane < hi && tl[lo + lane] < s0));
    // window lane j holds entry lo - 1 + j (lane 0: none if lo = q0; past q1: +inf)
    const bool in = (lane > 0 || lo > q0) && lo + lane - 1 < q1;
    const uint4 e = in ? T[lo + lane - 1] : make_uint4(0, 0, 0, 0);
    const uint32_t wpos = in ? e.x : 0xFFFFFFFFu;   // lane 0's is never compared
    int c = 0;   // entries of lanes 1..31 before s
#pragma unroll
    for (int st = 16; st > 0; st >>= 1)
        if (__shfl_sync(0xffffffffu, wpos, c + st) < s) c += st;
    nb.x = __shfl_sync(0xffffffffu, e.x, c);
    nb.y = __shfl_sync(0xffffffffu, e.y, c);
    nb.z = __shfl_sync(0xffffffffu, e.z, c);
    nb.w = __shfl_sync(0xffffffffu, e.w, c);
    has = c > 0 || lo > q0;
    if (c == 31 && lo + 31 < q1) lane_latest(tl, T, lo + 31, q1, s, nb, has);
}

// A round over every hit's 9 latest neighbours (the first round, and any
// round after an overflow of the edge list), in pixel-timeline order: a warp
// takes 32 consecutive entries, which mostly share a pixel, and finds their
// latest earlier entries on each neighbour pixel together (warp_latest;
// lane by lane where the warp straddles pixels), with their state from the
// snapshot: the snapshot root starts the find of the neighbour's group (one
// step shorter than from the hit), its last key decides most rules without
// a read.  Merges what the rule allows and lists the rest, as (hit, root of
// the neighbour's group).
__global__ void __launch_bounds__(256) k_global_first(Work w, VarWork v, int out) {
    const Seg &g = w.seg[0];
    const uint32_t W = g.width, H = g.height, n = g.n, dt = g.dt;
    const uint32_t sel = v.prob->npasses & 1u;
    const uint32_t *tl = pick(v.v, sel) + g.off;   // sorted positions grouped by pixel
    const uint32_t *tk = pick(v.k, sel) + g.off;   // their pixel ids
    const uint4 *T = v.tline + g.off;
    const uint32_t *ps = v.pix_start;
    const int lane = threadIdx.x & 31;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    bool changed = false;
    for (uint32_t i0 = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32u; i0 < n; i0 += warps * 32u) {
        const uint32_t i = i0 + (uint32_t)lane;
        const bool valid = i < n;
        const uint4 me = valid ? T[i] : make_uint4(0, 0, 0, 0);   // position, group id, its last key, key
        const uint32_t p = valid ? tk[i] : 0xFFFFFFFFu;
        const uint32_t p0 = __shfl_sync(0xffffffffu, p, 0);
        const bool uniform = __all_sync(0xffffffffu, p == p0);
        const int px = (int)(p % W), py = (int)(p / W);
        uint32_t rh = me.y;   // an id of h's group, moved towards its root as the round goes
#pragma unroll 1
        for (int d = 0; d < 9; ++d) {
            uint4 nb = make_uint4(0, 0, 0, 0);
            bool has = false;
            const int x = px + d % 3 - 1, y = py + d / 3 - 1;
            const bool inside = valid && x >= 0 && x < (int)W && y >= 0 && y < (int)H;
            if (d == 4) {
                if (valid && i > ps[p]) {
                    nb = T[i - 1];
                    has = true;
                }
            } else if (uniform) {   // inside is the same for every lane
                if (inside) {
                    const uint32_t q = (uint32_t)y * W + (uint32_t)x;
                    warp_latest(tl, T, ps[q], ps[q + 1], me.x, lane, nb, has);
                }
            } else if (inside) {
                const uint32_t q = (uint32_t)y * W + (uint32_t)x;
                lane_latest(tl, T, ps[q], ps[q + 1], me.x, nb, has);
            }
            // Any two nodes found equal are in one group (groups only
            // merge), so stale roots only cost a find; the last keys used
            // are lower bounds of the group's (nb.z: its part at the
            // snapshot), so the rule never merges more than the sweep.
            int r = 0;
            uint32_t rl = nb.y;
            if (has && rl != rh) {
                rl = gfind(v.cpar_d, rl);
                if (rl != rh) rh = gfind(v.cpar_d, rh);   // h's group may have been joined since
                if (rl != rh) {
                    bool ok = (uint64_t)me.w <= (uint64_t)nb.z + dt;
                    if (!ok) ok = (uint64_t)me.w <= (uint64_t)*reinterpret_cast<volatile uint32_t *>(&v.clast[rl]) + dt;
                    if (ok) {
                        if (gunion_last(v.cpar_d, v.clast, rh, rl)) r = 1;
                        rh = min(rh, rl);
                    } else {
                        r = 2;
                    }
                }
            }
            changed |= r == 1;
            push_edges(v, out, r == 2, rh, rl, me.w);
        }
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&v.changed[0], 1u);
}

// A round over the open edges of list `in` only: both ends' first steps
// up the forest at once.
__global__ void __launch_bounds__(256) k_global_list(Work w, VarWork v, int in) {
    const uint2 *list = pick(v.edges, in);
    const uint32_t *keys = pick(v.ekey, in);
    const uint32_t dt = w.seg[0].dt;
    const unsigned long long n = v.ecount[in];
    const uint32_t cnt = n < v.edge_cap ? (uint32_t)n : v.edge_cap;
    bool changed = false;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t e0 = blockIdx.x * blockDim.x; e0 < cnt; e0 += stride) {
        const uint32_t e = e0 + threadIdx.x;
        const bool valid = e < cnt;
        uint2 ed = make_uint2(0, 0);
        uint32_t ks = 0, ux = 0, uy = 0;
        if (valid) {
            ed = list[e];
            ks = keys[e];
            ux = v.cpar_d[ed.x];
            uy = v.cpar_d[ed.y];
        }
        int r = 0;
        uint32_t rh = ed.x, rl = ed.y;
        if (valid) {
            rh = ux == ed.x ? ux : gfind(v.cpar_d, ux);
            rl = uy == ed.y ? uy : gfind(v.cpar_d, uy);
            if (rl != rh) {   // the rule on the group's last key as it stands (a lower bound)
                const uint32_t last = *reinterpret_cast<volatile uint32_t *>(&v.clast[rl]);
                if ((uint64_t)ks <= (uint64_t)last + dt) r = gunion_last(v.cpar_d, v.clast, rh, rl) ? 1 : 0;
                else r = 2;
            }
        }
        changed |= r == 1;
        push_edges(v, 1 - in, r == 2, rh, rl, ks);
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicOr(&v.changed[0], 1u);
}

void launch_components(const Work &w, const VarWork &v, const Launch &L) {
    k_comp_count<<<L.fit(k_comp_count, 256, 0), 256, 0, L.stream>>>(w, v);
    k_comp_scan<<<1, 1024, 0, L.stream>>>(w, v);
    k_comp_ids<<<L.fit(k_comp_ids, 256, 0), 256, 0, L.stream>>>(w, v);
    k_comp_last<<<L.fit(k_comp_last, 256, 0), 256, 0, L.stream>>>(w, v);
    L.mark("k_components");
}

void launch_group_last(const VarWork &v, const Launch &L) {
    k_group_last_reset<<<L.fit(k_group_last_reset, 256, 0), 256, 0, L.stream>>>(v);
    k_group_last<<<L.fit(k_group_last, 256, 0), 256, 0, L.stream>>>(v);
    L.mark("k_group_last");
}

void launch_comp_parents(const Work &w, const VarWork &v, const Launch &L) {
    k_comp_parents<<<L.fit(k_comp_parents, 256, 0), 256, 0, L.stream>>>(w, v);
    L.mark("k_comp_parents");
}

// One round: list `1 - in` (or, if full, every hit) into list `in`'s
// partner.  full: out = list 0 after reading every hit.
void launch_global_edges(const Work &w, const VarWork &v, int full, int flat, int in, const Launch &L) {
    const int out = full ? 0 : 1 - in;
    cudaMemsetAsync(v.changed, 0, 2 * sizeof(uint32_t), L.stream);
    cudaMemsetAsync(v.ecount + out, 0, sizeof(unsigned long long), L.stream);
    if (full) {
        k_position_state<<<L.fit(k_position_state, 256, 0), 256, 0, L.stream>>>(w, v, flat);
        k_timeline_state<<<L.fit(k_timeline_state, 256, 0), 256, 0, L.stream>>>(w, v);
        L.mark("k_timeline_state");
        k_global_first<<<L.fit(k_global_first, 256, 0), 256, 0, L.stream>>>(w, v, out);
        L.mark("k_global_first");
    } else {
        k_global_list<<<L.fit(k_global_list, 256, 0), 256, 0, L.stream>>>(w, v, in);
        L.mark("k_global_list");
    }
}

void launch_variant_keys(const Work &w, const VarWork &v, int by_pixel, const Launch &L) {
    k_var_keys<<<L.fit(k_var_keys, 256, 0), 256, 0, L.stream>>>(w, v, by_pixel);
    L.mark(by_pixel ? "k_var_keys_pixel" : "k_var_keys_root");
}

Work variant_view(const Work &w, const VarWork &v) {
    Work wv = w;
    wv.keys[0] = v.k[0];
    wv.keys[1] = v.k[1];
    wv.vals[0] = v.v[0];
    wv.vals[1] = v.v[1];
    wv.prob = v.prob;
    return wv;
}

void launch_static_sweep(const Work &w, const VarWork &v, const Launch &L) {
    cudaMemsetAsync(v.work, 0, sizeof(uint32_t), L.stream);
    cudaMemsetAsync(v.changed, 0, 3 * sizeof(uint32_t), L.stream);
    k_static_sweep<<<L.fit(k_static_sweep, SW_WARPS * 32, 0), SW_WARPS * 32, 0, L.stream>>>(w, v);
    L.mark("k_static_sweep");
    k_static_sweep_big<<<L.fit(k_static_sweep_big, BIG_THREADS, BIG_SMEM), BIG_THREADS, BIG_SMEM, L.stream>>>(w, v);
    L.mark("k_static_sweep_big");
}

void launch_pixel_timelines(const Work &w, const VarWork &v, uint32_t npixels, const Launch &L) {
    cudaMemsetAsync(v.pix_start, 0, (npixels + 1) * sizeof(uint32_t), L.stream);
    k_pixel_hist<<<L.fit(k_pixel_hist, 256, 0), 256, 0, L.stream>>>(w, v);
    k_pixel_scan<<<1, 1024, 0, L.stream>>>(w, v);
    L.mark("k_pixel_hist_scan");
}


}  // namespace tpc
