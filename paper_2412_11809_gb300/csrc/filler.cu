// Hit buffer filling (Algorithm 2, Section 4.1): the host side of the
// pipeline that cuts the arriving hit stream into device buffers.  Host code
// only; it hands a finished buffer to a context with tpc_push.
//
// The procedure is applied hit by hit where it branches (the closing phase),
// and run by run where it cannot: while the current buffer holds fewer than
// b - b_t hits every hit is appended and only raises toa_max, and such a hit
// can never trigger a send (its ToA is at most the new toa_max), so a whole
// run of them is one copy and one max-reduction.
#include <algorithm>
#include <cstring>
#include <deque>
#include <new>
#include <utility>
#include <vector>

#include "tpc.h"

namespace {

struct FillBuf {
    std::vector<tpc_hit> hits;
    std::vector<uint64_t> idx;   // arrival number of each hit
    uint64_t cut = 0;
    void clear() {
        hits.clear();
        idx.clear();
        cut = 0;
    }
};

uint64_t sat_add(uint64_t a, uint64_t b) { return a > ~0ull - b ? ~0ull : a + b; }

}  // namespace

struct tpc_filler {
    uint64_t b = 0, b_t = 0, t = 0, t_closing = 0;
    uint64_t toa_max = 0;        // one value for the whole stream
    uint64_t arrived = 0;        // hits stored so far
    bool finished = false;
    FillBuf cur, next;
    std::deque<FillBuf> sent;    // sent, not yet taken (oldest first)
    std::vector<FillBuf> spare;  // taken buffers kept for their capacity

    FillBuf fresh() {
        if (spare.empty()) return FillBuf{};
        FillBuf f = std::move(spare.back());
        spare.pop_back();
        f.clear();
        return f;
    }

    // the current buffer is filled to about b hits: size it once instead of
    // growing it (and copying it) step by step
    void reserve_current() {
        const size_t r = (size_t)std::min<uint64_t>(b, 1ull << 24);
        if (cur.hits.capacity() < r) {
            cur.hits.reserve(r);
            cur.idx.reserve(r);
        }
    }

    // sendToDevice(buffer); buffer <- nextBuffer
    void send_current(uint64_t cut) {
        cur.cut = cut;
        sent.push_back(std::move(cur));
        cur = std::move(next);
        next = fresh();
        reserve_current();
    }

    void store(const tpc_hit *h, size_t n) {
        const uint64_t room = b - b_t;
        const uint64_t t_send = sat_add(t, t_closing);
        size_t i = 0;
        while (i < n) {
            if (cur.hits.size() < room) {
                // filling phase: a run of appends that only raise toa_max
                const size_t m = (size_t)std::min<uint64_t>(n - i, room - cur.hits.size());
                cur.hits.insert(cur.hits.end(), h + i, h + i + m);
                uint64_t mx = toa_max;
                for (size_t k = 0; k < m; ++k) mx = std::max(mx, h[i + k].toa);
                toa_max = mx;
                const size_t base = cur.idx.size();
                cur.idx.resize(base + m);
                for (size_t k = 0; k < m; ++k) cur.idx[base + k] = arrived + i + k;
                i += m;
                continue;
            }
            // closing phase: the room b_t is for hits before toa_max + t_closing
            const tpc_hit &x = h[i];
            if (x.toa < sat_add(toa_max, t_closing) && cur.hits.size() < b) {
                cur.hits.push_back(x);
                cur.idx.push_back(arrived + i);
            } else {
                next.hits.push_back(x);
                next.idx.push_back(arrived + i);
                if (x.toa > toa_max && x.toa - toa_max > t_send) send_current(sat_add(toa_max, t_closing));
            }
            ++i;
        }
        arrived += n;
    }
};

extern "C" {

int tpc_filler_create(uint64_t b, uint64_t b_t, uint64_t t, uint64_t t_closing, tpc_filler **out) {
    if (!out) return TPC_ERR_ARG;
    *out = nullptr;
    if (b == 0 || b_t >= b) return TPC_ERR_ARG;
    tpc_filler *f = new (std::nothrow) tpc_filler();
    if (!f) return TPC_ERR_NOMEM;
    f->b = b;
    f->b_t = b_t;
    f->t = t;
    f->t_closing = t_closing;
    try {
        f->reserve_current();
    } catch (const std::bad_alloc &) {
        delete f;
        return TPC_ERR_NOMEM;
    }
    *out = f;
    return TPC_OK;
}

int tpc_filler_store(tpc_filler *f, const tpc_hit *hits, size_t n) {
    if (!f || (n && !hits)) return TPC_ERR_ARG;
    if (f->finished) return TPC_ERR_STATE;
    try {
        f->store(hits, n);
    } catch (const std::bad_alloc &) {
        return TPC_ERR_NOMEM;
    }
    return TPC_OK;
}

int tpc_filler_finish(tpc_filler *f) {
    if (!f) return TPC_ERR_ARG;
    if (f->finished) return TPC_OK;
    try {
        if (!f->cur.hits.empty()) {
            f->cur.cut = ~0ull;
            f->sent.push_back(std::move(f->cur));
        }
        if (!f->next.hits.empty()) {
            f->next.cut = ~0ull;
            f->sent.push_back(std::move(f->next));
        }
    } catch (const std::bad_alloc &) {
        return TPC_ERR_NOMEM;
    }
    f->cur = FillBuf{};
    f->next = FillBuf{};
    f->finished = true;
    return TPC_OK;
}

int tpc_filler_ready(tpc_filler *f, size_t *n_buffers, size_t *front_hits) {
    if (!f) return TPC_ERR_ARG;
    if (n_buffers) *n_buffers = f->sent.size();
    if (front_hits) *front_hits = f->sent.empty() ? 0 : f->sent.front().hits.size();
    return TPC_OK;
}

static void pop_front(tpc_filler *f, uint64_t *indices, uint64_t *cut) {
    FillBuf &fb = f->sent.front();
    if (indices && !fb.idx.empty()) std::memcpy(indices, fb.idx.data(), fb.idx.size() * sizeof(uint64_t));
    if (cut) *cut = fb.cut;
    FillBuf done = std::move(fb);
    f->sent.pop_front();
    if (f->spare.size() < 4) {
        try {
            f->spare.push_back(std::move(done));
        } catch (const std::bad_alloc &) {
        }
    }
}

int tpc_filler_take(tpc_filler *f, tpc_hit *hits, uint64_t *indices, size_t cap, size_t *n_out, uint64_t *cut) {
    if (!f || !n_out) return TPC_ERR_ARG;
    if (f->sent.empty()) {
        *n_out = 0;
        return TPC_ERR_STATE;
    }
    const FillBuf &fb = f->sent.front();
    const size_t n = fb.hits.size();
    *n_out = n;
    if (n > cap) return TPC_ERR_CAP;
    if (!hits) return TPC_ERR_ARG;
    std::memcpy(hits, fb.hits.data(), n * sizeof(tpc_hit));
    pop_front(f, indices, cut);
    return TPC_OK;
}

int tpc_filler_send(tpc_filler *f, tpc_ctx *ctx, uint64_t *indices, size_t cap, size_t *n_out, uint64_t *cut) {
    if (!f || !ctx || !n_out) return TPC_ERR_ARG;
    if (f->sent.empty()) {
        *n_out = 0;
        return TPC_ERR_STATE;
    }
    const FillBuf &fb = f->sent.front();
    const size_t n = fb.hits.size();
    *n_out = n;
    if (indices && n > cap) return TPC_ERR_CAP;
    const int rc = tpc_push(ctx, fb.hits.data(), n, TPC_HOST);
    if (rc != TPC_OK) return rc;
    pop_front(f, indices, cut);
    return TPC_OK;
}

void tpc_filler_destroy(tpc_filler *f) { delete f; }

}  // extern "C"
