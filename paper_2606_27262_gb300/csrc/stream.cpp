// stream.cpp -- real-time streaming search (arXiv 2606.27262, Sec. 2-3.1:
// beams arrive as continuous streams read in overlapping blocks; each block
// must be searched before the next one arrives).
//
// Per beam a device ring holds the last gulp + max_delay samples (time-major).
// Gulp k of a beam is searched over output samples [k*gulp, (k+1)*gulp) from
// the ring window [k*gulp, k*gulp + gulp + max_delay).  Pushed gulps wait in
// a FIFO; whenever a launch stream and enough in-flight slots are free, the
// oldest pending gulps become one batch: their samples are copied into the
// rings, each window is staged into a slot, all of them are dedispersed in
// one persistent launch (or one grid launch per gulp), searched, and the
// candidates are copied back.  With two launch streams a new batch is
// admitted while the previous one is still on the GPU (continuous batching).
// No threads: all progress happens in sp_stream_push / sp_stream_poll.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "sp_internal.h"

using namespace sp;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

constexpr int kMaxStreams = 2;

struct Gulp {
    int32_t beam = 0;
    int64_t seq = 0;
    const uint8_t *h = nullptr;
    double t_push = 0.0;
};

struct Slot {
    uint8_t *d_staged = nullptr;
    int32_t *d_dmt = nullptr;
    void *d_sps = nullptr;
    sp_cand *d_cands = nullptr;
    int64_t *d_count = nullptr;
    sp_cand *h_cands = nullptr;  // pinned
    int64_t *h_count = nullptr;  // pinned
};

struct Launch {  // one batch in flight on one launch stream
    bool busy = false;
    std::vector<Gulp> gulps;
    std::vector<int> slots;
    cudaEvent_t done = nullptr;
    std::atomic<int> finished{0};
    double t_done = 0.0;
    BatchBeamDev *h_table = nullptr;  // pinned [max_batch]
    int64_t *h_begin = nullptr;       // pinned [max_batch + 1]
    BatchBeamDev *d_table = nullptr;
    int64_t *d_begin = nullptr;
    unsigned long long *d_counter = nullptr;
};

void CUDART_CB mark_done(void *p) {  // host callback: no CUDA calls here
    Launch *l = static_cast<Launch *>(p);
    l->t_done = now_s();
    l->finished.store(1, std::memory_order_release);
}

struct Result {
    sp_gulp_result info;
    std::vector<sp_cand> cands;
};

}  // namespace

struct sp_stream {
    const sp_plan *plan = nullptr;
    int device = 0;
    int32_t nbeams = 0;
    int64_t gulp = 0, n_in = 0, pitch = 0;
    int32_t widths[SP_MAX_WIDTHS] = {0};
    int32_t nw = 0;
    float threshold = 0.f;
    int64_t norm_block = 0;
    int64_t cap = 0;
    int32_t max_batch = 0;
    int32_t flags = 0;
    int nstreams = kMaxStreams;
    int64_t device_bytes = 0;
    // beams
    uint8_t *d_rings = nullptr;      // [nbeams][n_in][nchan]
    int64_t ring_bytes = 0;
    std::vector<int64_t> next_seq;   // gulps pushed so far
    std::vector<char> has_history;
    std::vector<cudaEvent_t> staged_ev;  // last staging of each beam's ring
    std::vector<char> staged_ev_used;
    // slots and launches
    std::vector<Slot> slots;
    std::vector<int> free_slots;
    Launch launches[kMaxStreams];
    cudaStream_t streams[kMaxStreams] = {nullptr, nullptr};
    BatchLaunch geometry{};
    std::deque<Gulp> pending;
    std::deque<Result> results;
};

namespace {

int alloc_dev(void **p, int64_t bytes, int64_t *tot) {
    const int64_t b = std::max<int64_t>(align256(bytes), 256);
    if (cudaMalloc(p, (size_t)b) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SP_ENOMEM;
    }
    *tot += b;
    return SP_OK;
}

int alloc_host(void **p, int64_t bytes) {
    if (cudaMallocHost(p, (size_t)std::max<int64_t>(bytes, 64)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SP_ENOMEM;
    }
    return SP_OK;
}

void stream_free(sp_stream *s) {
    for (int i = 0; i < kMaxStreams; ++i) {
        Launch &l = s->launches[i];
        if (l.done) cudaEventDestroy(l.done);
        cudaFreeHost(l.h_table);
        cudaFreeHost(l.h_begin);
        cudaFree(l.d_table);
        cudaFree(l.d_begin);
        cudaFree(l.d_counter);
        if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    }
    for (Slot &sl : s->slots) {
        cudaFree(sl.d_staged);
        cudaFree(sl.d_dmt);
        cudaFree(sl.d_sps);
        cudaFree(sl.d_cands);
        cudaFree(sl.d_count);
        cudaFreeHost(sl.h_cands);
        cudaFreeHost(sl.h_count);
    }
    for (cudaEvent_t e : s->staged_ev)
        if (e) cudaEventDestroy(e);
    cudaFree(s->d_rings);
}

int64_t slot_bytes(const sp_stream *s) {
    const sp_plan *p = s->plan;
    return align256(p->nchan * s->pitch) + align256((int64_t)p->ndm * s->gulp * 4) +
           align256(sps_workspace_bytes(p->ndm, s->gulp, s->nw, s->norm_block)) +
           align256(std::max<int64_t>(s->cap, 1) * (int64_t)sizeof(sp_cand)) + 256;
}

// Copies gulp g's samples into its beam's ring (after the beam's previous
// window was staged) and stages its window into slot `sl`, on stream st.
int stage_gulp(sp_stream *s, const Gulp &g, const Slot &sl, cudaStream_t st) {
    const sp_plan *p = s->plan;
    const int64_t row_bytes = p->nchan;
    uint8_t *ring = s->d_rings + (int64_t)g.beam * s->ring_bytes;
    if (s->staged_ev_used[g.beam] && cudaStreamWaitEvent(st, s->staged_ev[g.beam], 0) != cudaSuccess)
        return SP_ECUDA;
    // Samples [max_delay + seq*gulp, + gulp) of the stream; sample i lives in
    // ring row i mod n_in.
    const int64_t first = (p->max_delay + g.seq * s->gulp) % s->n_in;
    const int64_t n1 = std::min(s->gulp, s->n_in - first);
    if (cudaMemcpyAsync(ring + first * row_bytes, g.h, (size_t)(n1 * row_bytes), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return SP_ECUDA;
    if (n1 < s->gulp && cudaMemcpyAsync(ring, g.h + n1 * row_bytes, (size_t)((s->gulp - n1) * row_bytes),
                                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SP_ECUDA;
    // Window of gulp seq: stream samples [seq*gulp, seq*gulp + n_in).
    const int64_t row0 = (g.seq * s->gulp) % s->n_in;
    int rc = launch_stage_input(ring, s->n_in, p->nchan, sl.d_staged, s->pitch, st, row0, s->n_in);
    if (rc) return rc;
    if (cudaEventRecord(s->staged_ev[g.beam], st) != cudaSuccess) return SP_ECUDA;
    s->staged_ev_used[g.beam] = 1;
    return SP_OK;
}

int search_slot(sp_stream *s, const Slot &sl, cudaStream_t st) {
    SpsArgs a;
    std::memset(&a, 0, sizeof a);
    a.dmt = sl.d_dmt;
    a.ndm = s->plan->ndm;
    a.n_out = s->gulp;
    for (int k = 0; k < s->nw; ++k) a.widths[k] = s->widths[k];
    a.nw = s->nw;
    a.threshold = s->threshold;
    a.norm_block = s->norm_block;
    a.nblk = sps_nblocks(s->gulp, s->norm_block);
    a.work = sl.d_sps;
    a.cands = sl.d_cands;
    a.cap = s->cap;
    a.count = sl.d_count;
    return launch_sps(a, st);
}

// Starts one batch of the oldest pending gulps on launch stream li.
int launch_batch(sp_stream *s, int li) {
    Launch &L = s->launches[li];
    cudaStream_t st = s->streams[li];
    const int n = (int)std::min<int64_t>({(int64_t)s->max_batch, (int64_t)s->free_slots.size(),
                                          (int64_t)s->pending.size()});
    L.gulps.clear();
    L.slots.clear();
    for (int i = 0; i < n; ++i) {
        L.gulps.push_back(s->pending.front());
        s->pending.pop_front();
        L.slots.push_back(s->free_slots.back());
        s->free_slots.pop_back();
    }
    const sp_plan *p = s->plan;
    int rc = SP_OK;
    for (int i = 0; i < n && !rc; ++i) rc = stage_gulp(s, L.gulps[i], s->slots[L.slots[i]], st);
    if (!rc && (s->flags & SP_STREAM_PER_GULP)) {
        for (int i = 0; i < n && !rc; ++i) {
            const Slot &sl = s->slots[L.slots[i]];
            rc = launch_dedisperse(p, sl.d_staged, s->pitch, s->gulp, sl.d_dmt, st);
        }
    } else if (!rc) {
        const int64_t items = (int64_t)p->ntiles * dedisp_time_tiles(p, s->gulp);
        L.h_begin[0] = 0;
        for (int i = 0; i < n; ++i) {
            const Slot &sl = s->slots[L.slots[i]];
            BatchBeamDev &d = L.h_table[i];
            d.xt = sl.d_staged;
            d.pitch = s->pitch;
            d.n_out = s->gulp;
            d.out = sl.d_dmt;
            d.tile_first = p->d_tile_first;
            d.tile_count = p->d_tile_count;
            d.geo = p->d_chunk_geo;
            d.off = p->d_chunk_off;
            d.nchan = p->nchan;
            d.nchunks = p->nchunks;
            d.ntiles = p->ntiles;
            d.ntime = (int32_t)dedisp_time_tiles(p, s->gulp);
            L.h_begin[i + 1] = L.h_begin[i] + items;
        }
        // Pinned sources: the copies are asynchronous; the buffers are
        // rewritten only after this launch has completed.
        if (cudaMemcpyAsync(L.d_table, L.h_table, (size_t)n * sizeof(BatchBeamDev), cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(L.d_begin, L.h_begin, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st) !=
                cudaSuccess)
            rc = SP_ECUDA;
        BatchLaunch B = s->geometry;
        B.nbeams = n;
        B.nitems = L.h_begin[n];
        B.d_beams = L.d_table;
        B.d_item_begin = L.d_begin;
        B.d_counter = L.d_counter;
        B.d_status = p->d_status;
        if (!rc) rc = launch_dedisperse_batch(B, st, true);
    }
    for (int i = 0; i < n && !rc; ++i) {
        const Slot &sl = s->slots[L.slots[i]];
        rc = search_slot(s, sl, st);
        if (!rc && (cudaMemcpyAsync(sl.h_count, sl.d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st) !=
                        cudaSuccess ||
                    cudaMemcpyAsync(sl.h_cands, sl.d_cands, (size_t)s->cap * sizeof(sp_cand),
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess))
            rc = SP_ECUDA;
    }
    L.finished.store(0, std::memory_order_relaxed);
    if (!rc && (cudaLaunchHostFunc(st, mark_done, &L) != cudaSuccess || cudaEventRecord(L.done, st) != cudaSuccess))
        rc = SP_ECUDA;
    L.busy = true;  // even on error: its slots return when the stream has drained
    if (rc) {
        L.t_done = now_s();
        L.finished.store(1, std::memory_order_release);
    }
    return rc;
}

// Collects finished launches, then starts new ones while possible.
int progress(sp_stream *s) {
    for (int li = 0; li < s->nstreams; ++li) {
        Launch &L = s->launches[li];
        if (!L.busy) continue;
        const cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return SP_ECUDA;
        // The host callback precedes the event on the stream, so it has run;
        // the bound only guards against a launch that failed to enqueue it.
        for (long spins = 0; !L.finished.load(std::memory_order_acquire) && spins < (1L << 26); ++spins) {
        }
        if (!L.finished.load(std::memory_order_acquire)) L.t_done = now_s();
        for (size_t i = 0; i < L.gulps.size(); ++i) {
            const Slot &sl = s->slots[L.slots[i]];
            Result r;
            r.info.beam = L.gulps[i].beam;
            r.info.seq = L.gulps[i].seq;
            r.info.t0 = L.gulps[i].seq * s->gulp;
            r.info.count = *sl.h_count;
            r.info.status = *sl.h_count > s->cap ? SP_EOVERFLOW : SP_OK;
            r.info.t_push = L.gulps[i].t_push;
            r.info.t_done = L.t_done;
            r.cands.assign(sl.h_cands, sl.h_cands + std::min(*sl.h_count, s->cap));
            s->results.push_back(std::move(r));
            s->free_slots.push_back(L.slots[i]);
        }
        L.busy = false;
    }
    for (int li = 0; li < s->nstreams; ++li) {
        if (s->pending.empty() || s->free_slots.empty()) break;
        if (s->launches[li].busy) continue;
        const int rc = launch_batch(s, li);
        if (rc) return rc;
    }
    return SP_OK;
}

}  // namespace

extern "C" double sp_stream_now(void) { return now_s(); }

extern "C" int sp_stream_create(const sp_plan *plan, int32_t nbeams, int64_t gulp, const int32_t *h_widths,
                                int32_t nw, float threshold, int64_t norm_block, int64_t cand_cap,
                                int64_t hbm_budget_bytes, int32_t max_batch, int32_t flags, sp_stream **out) {
    if (!out) return SP_EINVAL;
    *out = nullptr;
    if (!plan || nbeams <= 0 || gulp <= 0 || cand_cap < 1 || max_batch < 1 || hbm_budget_bytes <= 0 ||
        (flags & ~(SP_STREAM_PER_GULP | SP_STREAM_ONE_STREAM)))
        return SP_EINVAL;
    int rc = check_widths(h_widths, nw);
    if (rc) return rc;
    if (!on_plan_device(plan)) return SP_EINVAL;
    if (plan->ndm > 65535 || gulp + plan->max_delay > (int64_t)INT32_MAX - 4096 ||
        dedisp_time_tiles(plan, gulp) > 65535)
        return SP_ELIMIT;
    sp_stream *s = new (std::nothrow) sp_stream();
    if (!s) return SP_ENOMEM;
    s->plan = plan;
    s->device = plan->device;
    s->nbeams = nbeams;
    s->gulp = gulp;
    s->n_in = gulp + plan->max_delay;
    s->pitch = dedisp_pitch(s->n_in);
    std::copy(h_widths, h_widths + nw, s->widths);
    s->nw = nw;
    s->threshold = threshold;
    s->norm_block = norm_block;
    s->cap = cand_cap;
    s->max_batch = max_batch;
    s->flags = flags;
    s->nstreams = (flags & SP_STREAM_ONE_STREAM) ? 1 : kMaxStreams;
    s->ring_bytes = align256(s->n_in * plan->nchan);
    s->next_seq.assign(nbeams, 0);
    s->has_history.assign(nbeams, 0);
    s->staged_ev.assign(nbeams, nullptr);
    s->staged_ev_used.assign(nbeams, 0);
    // Memory: the rings first, then as many slots as the budget allows (at
    // most one batch per launch stream is useful).
    const int64_t tables = s->nstreams * (align256((int64_t)max_batch * sizeof(BatchBeamDev)) +
                                          align256((int64_t)(max_batch + 1) * 8) + 256);
    const int64_t rings = (int64_t)nbeams * s->ring_bytes;
    const int64_t per_slot = slot_bytes(s);
    const int64_t nslots = std::min<int64_t>((hbm_budget_bytes - rings - tables) / per_slot,
                                             (int64_t)max_batch * s->nstreams);
    if (nslots < 1) rc = SP_ENOMEM;
    if (!rc) rc = alloc_dev((void **)&s->d_rings, rings, &s->device_bytes);
    if (!rc && cudaMemset(s->d_rings, 0, (size_t)rings) != cudaSuccess) rc = SP_ECUDA;
    for (int64_t i = 0; i < nslots && !rc; ++i) {
        s->slots.emplace_back();
        Slot &sl = s->slots.back();
        rc = alloc_dev((void **)&sl.d_staged, plan->nchan * s->pitch, &s->device_bytes);
        if (!rc) rc = alloc_dev((void **)&sl.d_dmt, (int64_t)plan->ndm * gulp * 4, &s->device_bytes);
        if (!rc) rc = alloc_dev(&sl.d_sps, sps_workspace_bytes(plan->ndm, gulp, nw, norm_block), &s->device_bytes);
        if (!rc) rc = alloc_dev((void **)&sl.d_cands, cand_cap * (int64_t)sizeof(sp_cand), &s->device_bytes);
        if (!rc) rc = alloc_dev((void **)&sl.d_count, 8, &s->device_bytes);
        if (!rc) rc = alloc_host((void **)&sl.h_cands, cand_cap * (int64_t)sizeof(sp_cand));
        if (!rc) rc = alloc_host((void **)&sl.h_count, 8);
        s->free_slots.push_back((int)i);
    }
    for (int li = 0; li < s->nstreams && !rc; ++li) {
        Launch &L = s->launches[li];
        rc = alloc_host((void **)&L.h_table, (int64_t)max_batch * sizeof(BatchBeamDev));
        if (!rc) rc = alloc_host((void **)&L.h_begin, (int64_t)(max_batch + 1) * 8);
        if (!rc) rc = alloc_dev((void **)&L.d_table, (int64_t)max_batch * sizeof(BatchBeamDev), &s->device_bytes);
        if (!rc) rc = alloc_dev((void **)&L.d_begin, (int64_t)(max_batch + 1) * 8, &s->device_bytes);
        if (!rc) rc = alloc_dev((void **)&L.d_counter, 8, &s->device_bytes);
        if (!rc && (cudaStreamCreateWithFlags(&s->streams[li], cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess)) {
            cudaGetLastError();
            rc = SP_ECUDA;
        }
    }
    for (int32_t b = 0; b < nbeams && !rc; ++b)
        if (cudaEventCreateWithFlags(&s->staged_ev[b], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            rc = SP_ECUDA;
        }
    if (!rc) {
        BatchLaunch &G = s->geometry;
        G.shape = plan->shape;
        G.copies_max = plan->copies_max;
        G.raw_max = plan->raw_max;
        G.smem_bytes = plan->smem_bytes;
        rc = batch_grid(G);
    }
    if (!rc) rc = dedisp_configure(plan);
    if (!rc) rc = sps_configure(h_widths[nw - 1]);
    if (rc) {
        stream_free(s);
        delete s;
        return rc;
    }
    *out = s;
    return SP_OK;
}

extern "C" int sp_stream_destroy(sp_stream *s) {
    if (!s) return SP_EINVAL;
    for (int li = 0; li < s->nstreams; ++li)
        if (s->streams[li]) cudaStreamSynchronize(s->streams[li]);
    stream_free(s);
    delete s;
    return SP_OK;
}

extern "C" int sp_stream_info(const sp_stream *s, int32_t *slots, int64_t *device_bytes, int64_t *n_in) {
    if (!s) return SP_EINVAL;
    if (slots) *slots = (int32_t)s->slots.size();
    if (device_bytes) *device_bytes = s->device_bytes;
    if (n_in) *n_in = s->n_in;
    return SP_OK;
}

extern "C" int sp_stream_history(sp_stream *s, int32_t beam, const uint8_t *h_hist) {
    if (!s || beam < 0 || beam >= s->nbeams || !h_hist) return SP_EINVAL;
    for (const Gulp &g : s->pending)
        if (g.beam == beam) return SP_EINVAL;
    for (int li = 0; li < s->nstreams; ++li)
        for (const Gulp &g : s->launches[li].gulps)
            if (s->launches[li].busy && g.beam == beam) return SP_EINVAL;
    const int64_t n = s->plan->max_delay;
    if (n > 0 && cudaMemcpy(s->d_rings + (int64_t)beam * s->ring_bytes, h_hist, (size_t)(n * s->plan->nchan),
                            cudaMemcpyHostToDevice) != cudaSuccess)
        return SP_ECUDA;
    s->has_history[beam] = 1;
    s->next_seq[beam] = 0;
    return SP_OK;
}

extern "C" int sp_stream_push(sp_stream *s, int32_t beam, const uint8_t *h_gulp, int64_t *seq) {
    if (!s || beam < 0 || beam >= s->nbeams || !h_gulp || !s->has_history[beam]) return SP_EINVAL;
    Gulp g;
    g.beam = beam;
    g.seq = s->next_seq[beam]++;
    g.h = h_gulp;
    g.t_push = now_s();
    s->pending.push_back(g);
    if (seq) *seq = g.seq;
    return progress(s);
}

extern "C" int sp_stream_poll(sp_stream *s, int32_t wait, sp_gulp_result *out, sp_cand *cands, int32_t max_results,
                              int32_t *n_results) {
    if (!s || !n_results || max_results < 0 || (max_results > 0 && !out)) return SP_EINVAL;
    *n_results = 0;
    int rc = progress(s);
    if (rc) return rc;
    if (wait && s->results.empty()) {
        // Wait for the launch that finishes first (the older one).
        for (int li = 0; li < s->nstreams; ++li)
            if (s->launches[li].busy) {
                if (cudaEventSynchronize(s->launches[li].done) != cudaSuccess) return SP_ECUDA;
                break;
            }
        rc = progress(s);
        if (rc) return rc;
    }
    int32_t n = 0;
    while (n < max_results && !s->results.empty()) {
        Result &r = s->results.front();
        out[n] = r.info;
        if (cands && !r.cands.empty())
            std::memcpy(cands + (int64_t)n * s->cap, r.cands.data(), r.cands.size() * sizeof(sp_cand));
        s->results.pop_front();
        ++n;
    }
    *n_results = n;
    return SP_OK;
}

extern "C" int sp_stream_pending(const sp_stream *s, int64_t *queued, int64_t *in_flight, int64_t *ready) {
    if (!s) return SP_EINVAL;
    int64_t f = 0;
    for (int li = 0; li < s->nstreams; ++li)
        if (s->launches[li].busy) f += (int64_t)s->launches[li].gulps.size();
    if (queued) *queued = (int64_t)s->pending.size();
    if (in_flight) *in_flight = f;
    if (ready) *ready = (int64_t)s->results.size();
    return SP_OK;
}
