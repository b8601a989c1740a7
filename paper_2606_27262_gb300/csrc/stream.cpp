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
//
// With a sifter (and classifier) attached, each finished gulp's candidates
// are clustered on the host (sp_sift) and the kept peaks are scored from the
// gulp's staged window on a classifier stream while later batches run; the
// slot is recycled after that, and the result is returned when the scores
// are on the host (Sec. 3.2: sifting and classification of each block).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
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
    uint64_t order = 0;  // launches started before this one
    std::vector<Gulp> gulps;
    std::vector<int> slots;
    cudaEvent_t done = nullptr;
    cudaEvent_t dedispersed = nullptr;
    std::atomic<int> finished{0};
    double t_done = 0.0;
    BatchBeamDev *h_table = nullptr;  // pinned [max_batch]
    int64_t *h_begin = nullptr;       // pinned [max_batch + 1]
    BatchBeamDev *d_table = nullptr;
    int64_t *d_begin = nullptr;
    unsigned long long *d_counter = nullptr;
    // Status word of this batch's dedispersion (SP_STATUS_* bits), cleared
    // before each launch and read back with the candidates: a bounded wait
    // that ran out in any CTA invalidates every gulp of the batch.
    int32_t *d_status = nullptr;
    int32_t *h_status = nullptr;      // pinned
};

void CUDART_CB mark_done(void *p) {  // host callback: no CUDA calls here
    Launch *l = static_cast<Launch *>(p);
    l->t_done = now_s();
    l->finished.store(1, std::memory_order_release);
}

struct Result {
    sp_gulp_result info;
    std::vector<sp_cand> cands;
    std::vector<sp_cand> kept;
    std::vector<float> prob;
};

// Peaks scored by one classification job: the kept peaks of the gulps of
// one finished batch, cut, imaged and scored together.
constexpr int32_t kClsCap = SP_CNN_MAX_BATCH;

struct Searched {  // a gulp whose candidates are on the host, not yet sifted
    Result r;
    int slot = 0;
};

struct JobRec {  // a classification job (FIFO on the classifier stream)
    std::atomic<int> finished{0};  // set by a host callback after the scores' copy
    double t_done = 0.0;
    cudaEvent_t done = nullptr;
    sp_cand *h_kept = nullptr;     // pinned [kClsCap]
    float *h_prob = nullptr;       // pinned [kClsCap]
    std::vector<Result> rs;        // the gulps it scores, their slots and first peaks
    std::vector<int> slots;
    std::vector<int32_t> first;
    int32_t total = 0;
};

void CUDART_CB mark_classified(void *p) {  // host callback: no CUDA calls here
    JobRec *j = static_cast<JobRec *>(p);
    j->t_done = now_s();
    j->finished.store(1, std::memory_order_release);
}

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
    // Searches and result copies of every batch (highest priority), unless
    // SP_STREAM_ONE_STREAM keeps all of a batch on its launch stream.
    cudaStream_t search_stream = nullptr;
    BatchLaunch geometry{};
    std::deque<Gulp> pending;
    std::deque<Searched> searched;
    std::deque<Result> results;
    uint64_t launches_started = 0;
    bool pushed = false;
    // sifting and classification (sp_stream_attach)
    bool attached = false;
    sp_sift_params sift{};
    sp_cnn *clf = nullptr;
    int32_t t_in = 0, kept_cap = 0;
    cudaStream_t cls_stream = nullptr;
    sp_cand *d_kept = nullptr;     // [kClsCap]
    float *d_sub = nullptr;        // [kClsCap][256][t_in]
    void *d_ft = nullptr;          // bf16 [kClsCap][256][256]
    void *d_img = nullptr;         // bf16 [kClsCap][256][256] (DM-time)
    void *d_work = nullptr;
    int64_t work_bytes = 0;
    int32_t *d_shift = nullptr;    // [256][256]
    float *d_prob = nullptr;       // [kClsCap]
    std::unique_ptr<JobRec[]> recs;  // [slots]: a job holds at least one slot
    std::vector<int> free_recs;
    std::deque<int> jobs;          // dispatched, in order
    int open_job = -1;             // being filled
    std::vector<sp_cand> sift_buf;
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

// Releases the classifier stage of sp_stream_attach (also after a failed
// attach, which leaves the stream as it was).
void cls_free(sp_stream *s) {
    for (size_t i = 0; s->recs && i < s->slots.size(); ++i) {
        JobRec &j = s->recs[i];
        cudaFreeHost(j.h_kept);
        cudaFreeHost(j.h_prob);
        if (j.done) cudaEventDestroy(j.done);
    }
    s->recs.reset();
    s->free_recs.clear();
    if (s->cls_stream) cudaStreamDestroy(s->cls_stream);
    for (void *q : {(void *)s->d_kept, (void *)s->d_sub, s->d_ft, s->d_img, s->d_work, (void *)s->d_shift,
                    (void *)s->d_prob})
        cudaFree(q);
    s->cls_stream = nullptr;
    s->d_kept = nullptr;
    s->d_sub = nullptr;
    s->d_ft = s->d_img = s->d_work = nullptr;
    s->d_shift = nullptr;
    s->d_prob = nullptr;
}

void stream_free(sp_stream *s) {
    for (int i = 0; i < kMaxStreams; ++i) {
        Launch &l = s->launches[i];
        if (l.done) cudaEventDestroy(l.done);
        if (l.dedispersed) cudaEventDestroy(l.dedispersed);
        cudaFreeHost(l.h_table);
        cudaFreeHost(l.h_begin);
        cudaFree(l.d_table);
        cudaFree(l.d_begin);
        cudaFree(l.d_counter);
        cudaFree(l.d_status);
        cudaFreeHost(l.h_status);
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
    if (s->search_stream) cudaStreamDestroy(s->search_stream);
    cls_free(s);
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
    if (cudaMemsetAsync(L.d_status, 0, sizeof(int32_t), st) != cudaSuccess) rc = SP_ECUDA;
    for (int i = 0; i < n && !rc; ++i) rc = stage_gulp(s, L.gulps[i], s->slots[L.slots[i]], st);
    if (!rc && (s->flags & SP_STREAM_PER_GULP)) {
        for (int i = 0; i < n && !rc; ++i) {
            const Slot &sl = s->slots[L.slots[i]];
            rc = launch_dedisperse(p, sl.d_staged, s->pitch, s->gulp, sl.d_dmt, st, L.d_status);
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
        B.d_status = L.d_status;
        // One CTA per work item: CTAs retire, so the search's and the
        // classifier's high-priority CTAs take SMs as items finish (a
        // persistent grid would hold every SM until the batch is done), and
        // with eight DMs per thread the per-item kernel is also the faster
        // one (the persistent loop's extra state spills registers).
        if (!rc) rc = launch_dedisperse_batch(B, st, false);
    }
    // The searches go to the high-priority search stream: the next batch's
    // dedispersion (already queued on the other launch stream) would
    // otherwise take the SMs first and hold this batch's results back until
    // it ends.
    if (!rc && cudaMemcpyAsync(L.h_status, L.d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = SP_ECUDA;
    cudaStream_t ss = st;
    if (!rc && s->search_stream) {
        if (cudaEventRecord(L.dedispersed, st) != cudaSuccess ||
            cudaStreamWaitEvent(s->search_stream, L.dedispersed, 0) != cudaSuccess)
            rc = SP_ECUDA;
        ss = s->search_stream;
    }
    for (int i = 0; i < n && !rc; ++i) {
        const Slot &sl = s->slots[L.slots[i]];
        rc = search_slot(s, sl, ss);
        if (!rc && (cudaMemcpyAsync(sl.h_count, sl.d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, ss) !=
                        cudaSuccess ||
                    cudaMemcpyAsync(sl.h_cands, sl.d_cands, (size_t)s->cap * sizeof(sp_cand),
                                    cudaMemcpyDeviceToHost, ss) != cudaSuccess))
            rc = SP_ECUDA;
    }
    L.finished.store(0, std::memory_order_relaxed);
    if (!rc && (cudaLaunchHostFunc(ss, mark_done, &L) != cudaSuccess || cudaEventRecord(L.done, ss) != cudaSuccess))
        rc = SP_ECUDA;
    L.busy = true;  // even on error: its slots return when the stream has drained
    L.order = s->launches_started++;
    if (rc) {
        L.t_done = now_s();
        L.finished.store(1, std::memory_order_release);
    }
    return rc;
}

// Queues the open classification job on the classifier stream: each gulp's
// peaks are cut from its own staged window, then all of them are imaged and
// scored together and the scores copied back.  On failure its gulps are
// finished with the error (after whatever was queued has drained).
int dispatch_job(sp_stream *s) {
    if (s->open_job < 0) return SP_OK;
    const int id = s->open_job;
    s->open_job = -1;
    JobRec &j = s->recs[id];
    const sp_plan *p = s->plan;
    cudaStream_t st = s->cls_stream;
    j.finished.store(0, std::memory_order_relaxed);
    int rc = SP_OK;
    if (cudaMemcpyAsync(s->d_kept, j.h_kept, (size_t)j.total * sizeof(sp_cand), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        rc = SP_ECUDA;
    for (size_t g = 0; g < j.rs.size() && !rc; ++g)
        rc = sp_cnn_extract(p, s->slots[(size_t)j.slots[g]].d_staged, s->pitch, s->n_in, s->d_kept + j.first[g],
                            (int32_t)j.rs[g].kept.size(), s->widths, s->nw, s->t_in,
                            s->d_sub + (int64_t)j.first[g] * 256 * s->t_in, st);
    if (!rc)
        rc = sp_cnn_features(s->d_sub, j.total, 256, s->t_in, s->d_shift, s->d_ft, s->d_img, s->d_work,
                             s->work_bytes, st);
    const int32_t bmax = cnn_max_batch(s->clf);
    const int64_t img = (int64_t)256 * 256 * 2;  // bytes of one bf16 image
    for (int32_t i = 0; i < j.total && !rc; i += bmax)
        rc = sp_cnn_forward(s->clf, static_cast<uint8_t *>(s->d_ft) + i * img,
                            static_cast<uint8_t *>(s->d_img) + i * img, std::min(bmax, j.total - i), s->d_prob + i,
                            st);
    if (!rc &&
        (cudaMemcpyAsync(j.h_prob, s->d_prob, (size_t)j.total * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaLaunchHostFunc(st, mark_classified, &j) != cudaSuccess || cudaEventRecord(j.done, st) != cudaSuccess))
        rc = SP_ECUDA;
    if (!rc) {
        s->jobs.push_back(id);
        return SP_OK;
    }
    cudaStreamSynchronize(st);
    cudaGetLastError();
    for (size_t g = 0; g < j.rs.size(); ++g) {
        Result &r = j.rs[g];
        r.info.status = rc;
        r.prob.assign(r.kept.size(), -1.0f);
        s->results.push_back(std::move(r));
        s->free_slots.push_back(j.slots[g]);
    }
    j.rs.clear();
    j.slots.clear();
    j.first.clear();
    j.total = 0;
    s->free_recs.push_back(id);
    return SP_ECUDA;
}

// A gulp whose search candidates are on the host: without an attached stage
// it is finished; else its candidates are sifted, and with a classifier the
// kept peaks join the open classification job.  Slot si was freed already
// unless a classifier is attached; then it is held until the gulp's job has
// finished (or freed here when the gulp has no peak to score).
int finish_search(sp_stream *s, Result &&r, int si) {
    if (!s->attached) {
        s->results.push_back(std::move(r));
        return SP_OK;
    }
    const sp_plan *p = s->plan;
    int64_t nk = 0;
    int rc = sp_sift(r.cands.empty() ? nullptr : r.cands.data(), (int64_t)r.cands.size(), p->dms.data(), p->ndm,
                     s->widths, s->nw, p->tsamp, &s->sift, s->sift_buf.data(), s->kept_cap, &nk, nullptr);
    if (rc == SP_EOVERFLOW) {
        r.info.status = SP_EOVERFLOW;
        rc = SP_OK;
    }
    const int32_t n = rc ? 0 : (int32_t)std::min<int64_t>(nk, s->kept_cap);
    if (rc) r.info.status = rc;
    r.info.kept = rc ? 0 : nk;
    r.kept.assign(s->sift_buf.begin(), s->sift_buf.begin() + n);
    if (!s->clf || n == 0) {
        r.prob.assign((size_t)n, -1.0f);
        r.info.accepted = s->clf ? 0 : n;
        s->results.push_back(std::move(r));
        if (s->clf) s->free_slots.push_back(si);  // held only for the classifier
        return SP_OK;
    }
    if (s->open_job >= 0 && s->recs[s->open_job].total + n > kClsCap) {
        rc = dispatch_job(s);
        if (rc) return rc;
    }
    if (s->open_job < 0) {  // a record is free: every job holds at least one slot
        s->open_job = s->free_recs.back();
        s->free_recs.pop_back();
    }
    JobRec &j = s->recs[s->open_job];
    std::memcpy(j.h_kept + j.total, r.kept.data(), (size_t)n * sizeof(sp_cand));
    j.first.push_back(j.total);
    j.total += n;
    j.slots.push_back(si);
    j.rs.push_back(std::move(r));
    return SP_OK;
}

// Collects finished classifications and launches, then starts new launches
// while possible.
int progress(sp_stream *s) {
    while (!s->jobs.empty()) {
        const int id = s->jobs.front();
        JobRec &j = s->recs[id];
        const cudaError_t q = cudaEventQuery(j.done);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return SP_ECUDA;
        for (long spins = 0; !j.finished.load(std::memory_order_acquire) && spins < (1L << 26); ++spins) {
        }
        const double t_done = j.finished.load(std::memory_order_acquire) ? j.t_done : now_s();
        for (size_t g = 0; g < j.rs.size(); ++g) {
            Result &r = j.rs[g];
            r.prob.assign(j.h_prob + j.first[g], j.h_prob + j.first[g] + r.kept.size());
            r.info.accepted = 0;
            for (float v : r.prob) r.info.accepted += v >= 0.5f;
            r.info.t_done = t_done;
            s->results.push_back(std::move(r));
            s->free_slots.push_back(j.slots[g]);
        }
        j.rs.clear();
        j.slots.clear();
        j.first.clear();
        j.total = 0;
        s->free_recs.push_back(id);
        s->jobs.pop_front();
    }
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
        L.busy = false;
        // The candidates are on the host now: unless the classifier will read
        // the staged window, the slot is free for the next batch at once.
        const bool hold = s->attached && s->clf;
        for (size_t i = 0; i < L.gulps.size(); ++i) {
            const Slot &sl = s->slots[L.slots[i]];
            Searched g;
            std::memset(&g.r.info, 0, sizeof g.r.info);
            g.r.info.beam = L.gulps[i].beam;
            g.r.info.seq = L.gulps[i].seq;
            g.r.info.t0 = L.gulps[i].seq * s->gulp;
            g.r.info.count = *sl.h_count;
            g.r.info.status = *sl.h_count > s->cap ? SP_EOVERFLOW : SP_OK;
            if (*L.h_status & SP_STATUS_STAGING_TIMEOUT) {  // the whole batch is void
                g.r.info.status = SP_ETIMEOUT;
                g.r.info.count = 0;
            }
            g.r.info.t_push = L.gulps[i].t_push;
            g.r.info.t_done = L.t_done;
            g.r.info.t_search = L.t_done;
            if (g.r.info.status != SP_ETIMEOUT)
                g.r.cands.assign(sl.h_cands, sl.h_cands + std::min(*sl.h_count, s->cap));
            g.slot = L.slots[i];
            if (!hold) s->free_slots.push_back(g.slot);
            s->searched.push_back(std::move(g));
        }
    }
    // New batches first, then the host-side sifting and the classification
    // of the searched gulps, so that the GPU is never waiting for the sifter.
    for (int li = 0; li < s->nstreams; ++li) {
        if (s->pending.empty() || s->free_slots.empty()) break;
        if (s->launches[li].busy) continue;
        const int rc = launch_batch(s, li);
        if (rc) return rc;
    }
    int rc = SP_OK;
    while (!s->searched.empty()) {
        Searched &g = s->searched.front();
        const int e = finish_search(s, std::move(g.r), g.slot);
        if (e && !rc) rc = e;
        s->searched.pop_front();
    }
    const int e = dispatch_job(s);
    if (e && !rc) rc = e;
    return rc;
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
    // Memory: the rings first, then as many slots as the budget allows: one
    // batch per launch stream, plus one batch more so that a batch can be
    // admitted while the slots of an earlier one are still held by its
    // classification (sp_stream_attach).
    const int64_t tables = s->nstreams * (align256((int64_t)max_batch * sizeof(BatchBeamDev)) +
                                          align256((int64_t)(max_batch + 1) * 8) + 256);
    const int64_t rings = (int64_t)nbeams * s->ring_bytes;
    const int64_t per_slot = slot_bytes(s);
    const int64_t nslots = std::min<int64_t>((hbm_budget_bytes - rings - tables) / per_slot,
                                             (int64_t)max_batch * (s->nstreams + 1));
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
        if (!rc) rc = alloc_dev((void **)&L.d_status, 4, &s->device_bytes);
        if (!rc) rc = alloc_host((void **)&L.h_status, 4);
        if (!rc && (cudaStreamCreateWithFlags(&s->streams[li], cudaStreamNonBlocking) != cudaSuccess ||
                    cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
                    cudaEventCreateWithFlags(&L.dedispersed, cudaEventDisableTiming) != cudaSuccess)) {
            cudaGetLastError();
            rc = SP_ECUDA;
        }
    }
    if (!rc && !(flags & SP_STREAM_ONE_STREAM)) {
        int prio_lo = 0, prio_hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&s->search_stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
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
    if (s->search_stream) cudaStreamSynchronize(s->search_stream);
    if (s->cls_stream) cudaStreamSynchronize(s->cls_stream);
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
    s->pushed = true;
    if (seq) *seq = g.seq;
    return progress(s);
}

namespace {

int poll_impl(sp_stream *s, int32_t wait, sp_gulp_result *out, sp_cand *cands, sp_cand *kept, float *prob,
              int32_t max_results, int32_t *n_results) {
    if (!s || !n_results || max_results < 0 || (max_results > 0 && !out)) return SP_EINVAL;
    *n_results = 0;
    int rc = progress(s);
    if (rc) return rc;
    // Wait for the oldest classification, else the older launch, until a
    // result is ready or nothing is in flight (each wait ends with the work
    // it waits for).
    while (wait && s->results.empty()) {
        cudaEvent_t e = nullptr;
        if (!s->jobs.empty()) {
            e = s->recs[s->jobs.front()].done;
        } else {
            const Launch *oldest = nullptr;
            for (int li = 0; li < s->nstreams; ++li)
                if (s->launches[li].busy && (!oldest || s->launches[li].order < oldest->order))
                    oldest = &s->launches[li];
            if (oldest) e = oldest->done;
        }
        if (!e) break;
        if (cudaEventSynchronize(e) != cudaSuccess) return SP_ECUDA;
        rc = progress(s);
        if (rc) return rc;
    }
    int32_t n = 0;
    while (n < max_results && !s->results.empty()) {
        Result &r = s->results.front();
        out[n] = r.info;
        if (cands && !r.cands.empty())
            std::memcpy(cands + (int64_t)n * s->cap, r.cands.data(), r.cands.size() * sizeof(sp_cand));
        if (kept && !r.kept.empty())
            std::memcpy(kept + (int64_t)n * s->kept_cap, r.kept.data(), r.kept.size() * sizeof(sp_cand));
        if (prob && !r.prob.empty())
            std::memcpy(prob + (int64_t)n * s->kept_cap, r.prob.data(), r.prob.size() * sizeof(float));
        s->results.pop_front();
        ++n;
    }
    *n_results = n;
    return SP_OK;
}

}  // namespace

extern "C" int sp_stream_poll(sp_stream *s, int32_t wait, sp_gulp_result *out, sp_cand *cands, int32_t max_results,
                              int32_t *n_results) {
    return poll_impl(s, wait, out, cands, nullptr, nullptr, max_results, n_results);
}

extern "C" int sp_stream_poll_sifted(sp_stream *s, int32_t wait, sp_gulp_result *out, sp_cand *cands, sp_cand *kept,
                                     float *prob, int32_t max_results, int32_t *n_results) {
    if (s && !s->attached) return SP_EINVAL;
    return poll_impl(s, wait, out, cands, kept, prob, max_results, n_results);
}

extern "C" int sp_stream_pending(const sp_stream *s, int64_t *queued, int64_t *in_flight, int64_t *ready) {
    if (!s) return SP_EINVAL;
    int64_t f = (int64_t)s->jobs.size();
    for (int li = 0; li < s->nstreams; ++li)
        if (s->launches[li].busy) f += (int64_t)s->launches[li].gulps.size();
    if (queued) *queued = (int64_t)s->pending.size();
    if (in_flight) *in_flight = f;
    if (ready) *ready = (int64_t)s->results.size();
    return SP_OK;
}

extern "C" int sp_stream_attach(sp_stream *s, const sp_sift_params *params, sp_cnn *clf, int32_t t_in,
                                int32_t kept_cap) {
    if (!s || !params || s->attached || s->pushed || kept_cap < 1 || kept_cap > kClsCap) return SP_EINVAL;
    const sp_plan *p = s->plan;
    if (clf && (p->nchan % 256 || t_in < 256 || t_in > 4096 || (t_in & 1) || cnn_device(clf) != s->device))
        return SP_EINVAL;
    int64_t dummy = 0;  // the sifter's own argument checks, on no candidates
    int rc = sp_sift(nullptr, 0, p->dms.data(), p->ndm, s->widths, s->nw, p->tsamp, params, nullptr, 0, &dummy, nullptr);
    if (rc) return rc;
    if (!on_plan_device(p)) return SP_EINVAL;
    s->sift_buf.assign((size_t)kept_cap, sp_cand{});
    if (clf) {
        const int64_t nimg = (int64_t)kClsCap * 256 * 256;
        const int64_t bytes0 = s->device_bytes;
        s->work_bytes = sp_cnn_features_workspace_bytes(kClsCap);
        rc = alloc_dev((void **)&s->d_kept, (int64_t)kClsCap * (int64_t)sizeof(sp_cand), &s->device_bytes);
        if (!rc) rc = alloc_dev((void **)&s->d_sub, (int64_t)kClsCap * 256 * t_in * 4, &s->device_bytes);
        if (!rc) rc = alloc_dev(&s->d_ft, nimg * 2, &s->device_bytes);
        if (!rc) rc = alloc_dev(&s->d_img, nimg * 2, &s->device_bytes);
        if (!rc) rc = alloc_dev(&s->d_work, s->work_bytes, &s->device_bytes);
        if (!rc) rc = alloc_dev((void **)&s->d_shift, 256 * 256 * 4, &s->device_bytes);
        if (!rc) rc = alloc_dev((void **)&s->d_prob, (int64_t)kClsCap * 4, &s->device_bytes);
        if (!rc) {
            s->recs.reset(new (std::nothrow) JobRec[s->slots.size()]);
            if (!s->recs) rc = SP_ENOMEM;
        }
        for (size_t i = 0; i < s->slots.size() && !rc; ++i) {
            JobRec &j = s->recs[i];
            rc = alloc_host((void **)&j.h_kept, (int64_t)kClsCap * (int64_t)sizeof(sp_cand));
            if (!rc) rc = alloc_host((void **)&j.h_prob, (int64_t)kClsCap * 4);
            if (!rc && cudaEventCreateWithFlags(&j.done, cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                rc = SP_ECUDA;
            }
            s->free_recs.push_back((int)i);
        }
        std::vector<int32_t> shift((size_t)256 * 256);
        if (!rc) rc = sp_dmt_shifts(p->freqs.data(), p->nchan, 256, (t_in - 256) / 2, shift.data());
        if (!rc && cudaMemcpy(s->d_shift, shift.data(), shift.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = SP_ECUDA;
        // The classifier's kernels are few and short: the highest priority lets
        // them take SMs as soon as any free up instead of queueing behind the
        // CTAs of the next dedispersion batch.
        int prio_lo = 0, prio_hi = 0;
        if (!rc && (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
                    cudaStreamCreateWithPriority(&s->cls_stream, cudaStreamNonBlocking, prio_hi) != cudaSuccess)) {
            cudaGetLastError();
            rc = SP_ECUDA;
        }
        if (rc) {
            cls_free(s);
            s->device_bytes = bytes0;
            return rc;
        }
    }
    s->sift = *params;
    s->clf = clf;
    s->t_in = t_in;
    s->kept_cap = kept_cap;
    s->attached = true;
    return SP_OK;
}
