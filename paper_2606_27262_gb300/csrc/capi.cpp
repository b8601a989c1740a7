// capi.cpp -- argument checking and the extern "C" entry points of
// libspotlight (declared and documented in include/spotlight.h).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>

#include "sp_internal.h"

using namespace sp;

namespace sp {

bool on_plan_device(const sp_plan *p) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return dev == p->device;
}

int check_widths(const int32_t *w, int32_t nw) {
    if (!w || nw <= 0) return SP_EINVAL;
    if (nw > SP_MAX_WIDTHS) return SP_ELIMIT;
    for (int32_t k = 0; k < nw; ++k) {
        if (w[k] < 1) return SP_EINVAL;
        if (w[k] > SP_MAX_WIDTH) return SP_ELIMIT;
        if (k > 0 && !(w[k] > w[k - 1])) return SP_EINVAL;
    }
    return SP_OK;
}

}  // namespace sp

namespace {

int sps_common(const int32_t *d_dmt, int32_t ndm, int64_t n_out, const int32_t *h_widths, int32_t nw,
               int64_t norm_block, void *d_work, int64_t work_bytes, SpsArgs &a) {
    if (!d_dmt || ndm <= 0 || n_out <= 0) return SP_EINVAL;
    int rc = check_widths(h_widths, nw);
    if (rc) return rc;
    if (ndm > 65535 || n_out > (int64_t)INT32_MAX) return SP_ELIMIT;
    const int64_t need = sps_workspace_bytes(ndm, n_out, nw, norm_block);
    if (!d_work || work_bytes < need || (reinterpret_cast<uintptr_t>(d_work) & 255)) return SP_EWORKSPACE;
    std::memset(&a, 0, sizeof(a));
    a.dmt = d_dmt;
    a.ndm = ndm;
    a.n_out = n_out;
    for (int k = 0; k < nw; ++k) a.widths[k] = h_widths[k];
    a.nw = nw;
    a.norm_block = norm_block;
    a.nblk = sps_nblocks(n_out, norm_block);
    a.work = d_work;
    return SP_OK;
}

}  // namespace

namespace sp {
namespace {
std::atomic<uint64_t> g_launches{0};
thread_local bool t_capturing = false;  // launches go into a graph, not to the GPU
thread_local uint64_t t_captured = 0;
}  // namespace
void note_launch(uint64_t n) {
    if (t_capturing)
        t_captured += n;
    else
        g_launches.fetch_add(n, std::memory_order_relaxed);
}
void capture_begin() {
    t_capturing = true;
    t_captured = 0;
}
uint64_t capture_end() {
    t_capturing = false;
    return t_captured;
}
}  // namespace sp

extern "C" uint64_t sp_launch_count(void) { return sp::g_launches.load(std::memory_order_relaxed); }

extern "C" const char *sp_strerror(int code) {
    switch (code) {
        case SP_OK: return "ok";
        case SP_EINVAL: return "invalid argument";
        case SP_ESHAPE: return "inconsistent sizes (n_out must equal n_in - max_delay)";
        case SP_ECUDA: return "CUDA runtime error";
        case SP_EOVERFLOW: return "more candidates than the capacity";
        case SP_ENOMEM: return "allocation failed";
        case SP_EWORKSPACE: return "workspace missing, misaligned or too small";
        case SP_ELIMIT: return "size beyond a library limit";
        case SP_ETIMEOUT: return "a bounded wait in a kernel ran out; its outputs are void";
        default: return "unknown error";
    }
}

extern "C" int sp_debug_staging_fault(int32_t extra_bytes, int64_t wait_limit_cycles) {
    if (extra_bytes < 0 || (extra_bytes & 15) || extra_bytes > (1 << 20) || wait_limit_cycles < 1024 ||
        wait_limit_cycles > (1LL << 40))
        return SP_EINVAL;
    return set_staging_fault((uint32_t)extra_bytes, (long long)wait_limit_cycles);
}

extern "C" int64_t sp_staged_pitch(int64_t n_in) { return n_in > 0 ? dedisp_pitch(n_in) : -1; }

extern "C" int64_t sp_staged_bytes(int32_t nchan, int64_t n_in) {
    if (nchan <= 0 || n_in <= 0) return -1;
    return align256((int64_t)nchan * dedisp_pitch(n_in));
}

extern "C" int64_t sp_dedisperse_workspace_bytes(const sp_plan *p, int64_t n_in) {
    if (!p || n_in <= 0) return -1;
    return sp_staged_bytes(p->nchan, n_in);
}

static int check_dedisp_shape(const sp_plan *p, int64_t n_in, int64_t n_out) {
    if (!on_plan_device(p)) return SP_EINVAL;
    if (n_out != n_in - p->max_delay) return SP_ESHAPE;
    if (n_in > (int64_t)INT32_MAX - 4096 || dedisp_time_tiles(p, n_out) > 65535) return SP_ELIMIT;
    return SP_OK;
}

extern "C" int sp_dedisperse(const sp_plan *p, const uint8_t *d_in, int64_t n_in, int32_t *d_out, int64_t n_out,
                             void *d_work, int64_t work_bytes, void *stream) {
    if (!p || !d_in || !d_out || n_in <= 0 || n_out <= 0) return SP_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_in) & 15) return SP_EINVAL;
    int rc = check_dedisp_shape(p, n_in, n_out);
    if (rc) return rc;
    const int64_t pitch = dedisp_pitch(n_in);
    if (!d_work || work_bytes < sp_staged_bytes(p->nchan, n_in) || (reinterpret_cast<uintptr_t>(d_work) & 255))
        return SP_EWORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint8_t *staged = reinterpret_cast<uint8_t *>(d_work);
    rc = launch_stage_input(d_in, n_in, p->nchan, staged, pitch, s);
    if (rc) return rc;
    return launch_dedisperse(p, staged, pitch, n_out, d_out, s);
}

extern "C" int sp_stage_input(const uint8_t *d_in, int64_t n_in, int32_t nchan, uint8_t *d_staged, int64_t pitch,
                              void *stream) {
    if (!d_in || !d_staged || n_in <= 0 || nchan <= 0) return SP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_in) & 15) || (reinterpret_cast<uintptr_t>(d_staged) & 255)) return SP_EINVAL;
    if (pitch < dedisp_pitch(n_in) || (pitch & 63)) return SP_EINVAL;
    if (n_in > (int64_t)INT32_MAX - 4096 || (nchan + 63) / 64 > 65535) return SP_ELIMIT;
    return launch_stage_input(d_in, n_in, nchan, d_staged, pitch, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sp_dedisperse_staged(const sp_plan *p, const uint8_t *d_staged, int64_t pitch, int64_t n_in,
                                    int32_t *d_out, int64_t n_out, void *stream) {
    if (!p || !d_staged || !d_out || n_in <= 0 || n_out <= 0) return SP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_staged) & 255) || pitch < dedisp_pitch(n_in) || (pitch & 63))
        return SP_EINVAL;
    const int rc = check_dedisp_shape(p, n_in, n_out);
    if (rc) return rc;
    return launch_dedisperse(p, d_staged, pitch, n_out, d_out, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int64_t sp_sps_workspace_bytes(int32_t ndm, int64_t n_out, int32_t nw, int64_t norm_block) {
    if (ndm <= 0 || n_out <= 0 || nw <= 0) return -1;
    return sps_workspace_bytes(ndm, n_out, nw, norm_block);
}

extern "C" int sp_single_pulse_search(const int32_t *d_dmt, int32_t ndm, int64_t n_out, const int32_t *h_widths,
                                      int32_t nw, float threshold, int64_t norm_block, void *d_work,
                                      int64_t work_bytes, sp_cand *d_cands, int64_t cap, int64_t *d_count,
                                      void *stream) {
    SpsArgs a;
    int rc = sps_common(d_dmt, ndm, n_out, h_widths, nw, norm_block, d_work, work_bytes, a);
    if (rc) return rc;
    if (!d_count || cap < 0 || (cap > 0 && !d_cands)) return SP_EINVAL;
    a.threshold = threshold;
    a.cands = d_cands;
    a.cap = cap;
    a.count = d_count;
    return launch_sps(a, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int64_t sp_sps_window_workspace_bytes(int32_t ndm, int64_t n_out, int32_t nw, int64_t norm_block,
                                                 int32_t peak_radius) {
    if (ndm <= 0 || n_out <= 0 || nw <= 0 || peak_radius < 1 || peak_radius > kMaxPeakRadius) return -1;
    return sps_window_workspace_bytes(ndm, n_out, nw, norm_block, peak_radius);
}

extern "C" int sp_single_pulse_search_window(const int32_t *d_dmt, int32_t ndm, int64_t n_out,
                                             const int32_t *h_widths, int32_t nw, float threshold,
                                             int64_t norm_block, int32_t peak_radius, void *d_work,
                                             int64_t work_bytes, sp_cand *d_cands, int64_t cap, int64_t *d_count,
                                             void *stream) {
    if (peak_radius < 1 || peak_radius > kMaxPeakRadius) return SP_EINVAL;
    SpsArgs a;
    int rc = sps_common(d_dmt, ndm, n_out, h_widths, nw, norm_block, d_work, work_bytes, a);
    if (rc) return rc;
    if (work_bytes < sps_window_workspace_bytes(ndm, n_out, nw, norm_block, peak_radius)) return SP_EWORKSPACE;
    if (!d_count || cap < 0 || (cap > 0 && !d_cands)) return SP_EINVAL;
    a.threshold = threshold;
    a.cands = d_cands;
    a.cap = cap;
    a.count = d_count;
    return launch_sps_window(a, peak_radius, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int sp_best_snr_map(const int32_t *d_dmt, int32_t ndm, int64_t n_out, const int32_t *h_widths,
                               int32_t nw, int64_t norm_block, void *d_work, int64_t work_bytes, float *d_best,
                               int8_t *d_wbest, void *stream) {
    SpsArgs a;
    int rc = sps_common(d_dmt, ndm, n_out, h_widths, nw, norm_block, d_work, work_bytes, a);
    if (rc) return rc;
    if (!d_best || !d_wbest) return SP_EINVAL;
    a.map_best = d_best;
    a.map_wbest = d_wbest;
    return launch_sps(a, reinterpret_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------- searcher --
struct sp_searcher {
    const sp_plan *plan = nullptr;
    int64_t n_out = 0, n_in = 0;
    int32_t widths[SP_MAX_WIDTHS] = {0};
    int32_t nw = 0;
    float threshold = 0.f;
    int64_t norm_block = 0;
    int64_t cap = 0;
    uint8_t *d_in = nullptr;
    void *d_work = nullptr;
    int64_t work_bytes = 0;
    int32_t *d_dmt = nullptr;
    void *d_sps = nullptr;
    int64_t sps_bytes = 0;
    sp_cand *d_cands = nullptr;
    int64_t *d_count = nullptr;
    // Pipelined host runs (sp_searcher_submit_host): two slots, each with
    // its device input, candidates and count, a page-locked count, and the
    // events that order the input copy after the slot's last staging and
    // the collection after the slot's search.  Slot 0 uses d_in, d_cands
    // and d_count above.
    bool pipe_ready = false;
    uint8_t *p_in[2] = {nullptr, nullptr};
    sp_cand *p_cands[2] = {nullptr, nullptr};
    int64_t *p_count[2] = {nullptr, nullptr};
    int64_t *h_count = nullptr;      // page-locked [2]
    cudaStream_t copy_stream = nullptr, result_stream = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr}, staged[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool staged_used[2] = {false, false};
    int head = 0, queued = 0;        // oldest uncollected slot, uncollected beams
};

static void searcher_free(sp_searcher *s) {
    cudaFree(s->d_in);
    cudaFree(s->d_work);
    cudaFree(s->d_dmt);
    cudaFree(s->d_sps);
    cudaFree(s->d_cands);
    cudaFree(s->d_count);
    cudaFree(s->p_in[1]);
    cudaFree(s->p_cands[1]);
    cudaFree(s->p_count[1]);
    cudaFreeHost(s->h_count);
    for (int i = 0; i < 2; ++i) {
        if (s->copied[i]) cudaEventDestroy(s->copied[i]);
        if (s->staged[i]) cudaEventDestroy(s->staged[i]);
        if (s->done[i]) cudaEventDestroy(s->done[i]);
    }
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->result_stream) cudaStreamDestroy(s->result_stream);
}

extern "C" int sp_searcher_create(const sp_plan *p, int64_t n_out, const int32_t *h_widths, int32_t nw,
                                  float threshold, int64_t norm_block, int64_t cand_cap, sp_searcher **out) {
    if (!out) return SP_EINVAL;
    *out = nullptr;
    if (!p || n_out <= 0 || cand_cap < 0) return SP_EINVAL;
    int rc = check_widths(h_widths, nw);
    if (rc) return rc;
    if (!on_plan_device(p)) return SP_EINVAL;
    sp_searcher *s = new (std::nothrow) sp_searcher();
    if (!s) return SP_ENOMEM;
    s->plan = p;
    s->n_out = n_out;
    s->n_in = n_out + p->max_delay;
    std::copy(h_widths, h_widths + nw, s->widths);
    s->nw = nw;
    s->threshold = threshold;
    s->norm_block = norm_block;
    s->cap = cand_cap;
    s->work_bytes = sp_dedisperse_workspace_bytes(p, s->n_in);
    s->sps_bytes = sps_workspace_bytes(p->ndm, n_out, nw, norm_block);
    bool ok = cudaMalloc((void **)&s->d_in, (size_t)(s->n_in * p->nchan)) == cudaSuccess &&
              cudaMalloc(&s->d_work, (size_t)s->work_bytes) == cudaSuccess &&
              cudaMalloc((void **)&s->d_dmt, (size_t)p->ndm * n_out * 4) == cudaSuccess &&
              cudaMalloc(&s->d_sps, (size_t)s->sps_bytes) == cudaSuccess &&
              cudaMalloc((void **)&s->d_cands, (size_t)std::max<int64_t>(1, cand_cap) * sizeof(sp_cand)) ==
                  cudaSuccess &&
              cudaMalloc((void **)&s->d_count, sizeof(int64_t)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        searcher_free(s);
        delete s;
        return SP_ENOMEM;
    }
    *out = s;
    return SP_OK;
}

extern "C" int sp_searcher_destroy(sp_searcher *s) {
    if (!s) return SP_EINVAL;
    searcher_free(s);
    delete s;
    return SP_OK;
}

extern "C" int sp_searcher_run(sp_searcher *s, const uint8_t *d_in, sp_cand *d_cands, int64_t cap,
                               int64_t *d_count, void *stream) {
    if (!s) return SP_EINVAL;
    int rc = sp_dedisperse(s->plan, d_in, s->n_in, s->d_dmt, s->n_out, s->d_work, s->work_bytes, stream);
    if (rc) return rc;
    return sp_single_pulse_search(s->d_dmt, s->plan->ndm, s->n_out, s->widths, s->nw, s->threshold,
                                  s->norm_block, s->d_sps, s->sps_bytes, d_cands, cap, d_count, stream);
}

extern "C" int sp_searcher_run_host(sp_searcher *s, const uint8_t *h_in, sp_cand *h_cands, int64_t cap,
                                    int64_t *h_count, void *stream) {
    if (!s || !h_in || !h_count || cap < 0 || (cap > 0 && !h_cands)) return SP_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t cap_eff = std::min(cap, s->cap);
    if (cudaMemcpyAsync(s->d_in, h_in, (size_t)(s->n_in * s->plan->nchan), cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return SP_ECUDA;
    int rc = sp_searcher_run(s, s->d_in, s->d_cands, cap_eff, s->d_count, stream);
    if (rc) return rc;
    int64_t total = 0;
    if (cudaMemcpyAsync(&total, s->d_count, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SP_ECUDA;
    *h_count = total;
    const int64_t n = std::min(total, cap_eff);
    if (n > 0) {
        if (cudaMemcpyAsync(h_cands, s->d_cands, (size_t)n * sizeof(sp_cand), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return SP_ECUDA;
    }
    return total > cap_eff ? SP_EOVERFLOW : SP_OK;
}

// Second slot, streams and events of the pipelined host path (first submit).
static int searcher_pipe_init(sp_searcher *s) {
    if (s->pipe_ready) return SP_OK;
    const size_t in_bytes = (size_t)(s->n_in * s->plan->nchan);
    s->p_in[0] = s->d_in;
    s->p_cands[0] = s->d_cands;
    s->p_count[0] = s->d_count;
    bool ok = cudaMalloc((void **)&s->p_in[1], in_bytes) == cudaSuccess &&
              cudaMalloc((void **)&s->p_cands[1], (size_t)std::max<int64_t>(1, s->cap) * sizeof(sp_cand)) ==
                  cudaSuccess &&
              cudaMalloc((void **)&s->p_count[1], sizeof(int64_t)) == cudaSuccess &&
              cudaMallocHost((void **)&s->h_count, 2 * sizeof(int64_t)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return SP_ENOMEM;
    }
    ok = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&s->result_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < 2; ++i)
        ok = cudaEventCreateWithFlags(&s->copied[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->staged[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->done[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    s->pipe_ready = true;
    return SP_OK;
}

extern "C" int sp_searcher_submit_host(sp_searcher *s, const uint8_t *h_in, void *stream) {
    if (!s || !h_in || s->queued >= 2) return SP_EINVAL;
    int rc = check_dedisp_shape(s->plan, s->n_in, s->n_out);
    if (!rc) rc = searcher_pipe_init(s);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int i = (s->head + s->queued) % 2;
    // The slot's input is rewritten only after its previous beam was staged.
    if (s->staged_used[i] && cudaStreamWaitEvent(s->copy_stream, s->staged[i], 0) != cudaSuccess) return SP_ECUDA;
    if (cudaMemcpyAsync(s->p_in[i], h_in, (size_t)(s->n_in * s->plan->nchan), cudaMemcpyHostToDevice,
                        s->copy_stream) != cudaSuccess ||
        cudaEventRecord(s->copied[i], s->copy_stream) != cudaSuccess ||
        cudaStreamWaitEvent(st, s->copied[i], 0) != cudaSuccess)
        return SP_ECUDA;
    const int64_t pitch = dedisp_pitch(s->n_in);
    uint8_t *staged = static_cast<uint8_t *>(s->d_work);
    rc = launch_stage_input(s->p_in[i], s->n_in, s->plan->nchan, staged, pitch, st);
    if (!rc && cudaEventRecord(s->staged[i], st) != cudaSuccess) rc = SP_ECUDA;
    if (rc) return rc;
    s->staged_used[i] = true;
    rc = sp_dedisperse_staged(s->plan, staged, pitch, s->n_in, s->d_dmt, s->n_out, stream);
    if (!rc)
        rc = sp_single_pulse_search(s->d_dmt, s->plan->ndm, s->n_out, s->widths, s->nw, s->threshold,
                                    s->norm_block, s->d_sps, s->sps_bytes, s->p_cands[i], s->cap, s->p_count[i],
                                    stream);
    if (rc) return rc;
    if (cudaMemcpyAsync(s->h_count + i, s->p_count[i], sizeof(int64_t), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaEventRecord(s->done[i], st) != cudaSuccess)
        return SP_ECUDA;
    ++s->queued;
    return SP_OK;
}

extern "C" int sp_searcher_collect(sp_searcher *s, sp_cand *h_cands, int64_t cap, int64_t *h_count) {
    if (!s || !h_count || cap < 0 || (cap > 0 && !h_cands) || s->queued == 0) return SP_EINVAL;
    const int i = s->head;
    s->head = (s->head + 1) % 2;
    --s->queued;
    if (cudaEventSynchronize(s->done[i]) != cudaSuccess) return SP_ECUDA;
    const int64_t total = s->h_count[i];
    const int64_t cap_eff = std::min(cap, s->cap);
    *h_count = total;
    const int64_t n = std::min(total, cap_eff);
    if (n > 0 && (cudaMemcpyAsync(h_cands, s->p_cands[i], (size_t)n * sizeof(sp_cand), cudaMemcpyDeviceToHost,
                                  s->result_stream) != cudaSuccess ||
                  cudaStreamSynchronize(s->result_stream) != cudaSuccess))
        return SP_ECUDA;
    return total > cap_eff ? SP_EOVERFLOW : SP_OK;
}
