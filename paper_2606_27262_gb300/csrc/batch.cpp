// batch.cpp -- many beams per launch (arXiv 2606.27262, Sec. 2 and 3.1:
// every GPU searches many independent beams in real time).
//
//   sp_dedisperse_batch  one persistent dedispersion launch over the
//                        (beam, DM tile, time tile) items of several beams.
//   sp_batch             a fixed set of beams searched as one step: beams are
//                        grouped so that a group's DM transforms fit a memory
//                        budget; per group one staging pass, one persistent
//                        dedispersion launch, then the per-beam searches on a
//                        second stream (overlapping the next group's
//                        dedispersion).  The step can be captured into a CUDA
//                        graph; a per-beam mode runs the same work with one
//                        launch per step and beam for comparison.
#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <vector>

#include "sp_internal.h"

using namespace sp;

namespace {

constexpr int64_t kCounterBytes = 256;

// Device layout of one launch's tables: [work-queue head][beam table][item
// offsets].
int64_t table_bytes(int32_t nbeams) {
    return kCounterBytes + align256((int64_t)nbeams * (int64_t)sizeof(BatchBeamDev)) +
           align256((int64_t)(nbeams + 1) * 8);
}

// Checks one beam and fills its kernel descriptor; *items = its work items.
int describe(const sp_plan *p, const uint8_t *staged, int64_t pitch, int64_t n_in, int32_t *out, int64_t n_out,
             BatchBeamDev &d, int64_t *items) {
    if (!p || !staged || !out || n_in <= 0 || n_out <= 0) return SP_EINVAL;
    if (!on_plan_device(p)) return SP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(staged) & 255) || pitch < dedisp_pitch(n_in) || (pitch & 63)) return SP_EINVAL;
    if (n_out != n_in - p->max_delay) return SP_ESHAPE;
    if (n_in > (int64_t)INT32_MAX - 4096) return SP_ELIMIT;
    const int64_t nt = dedisp_time_tiles(p, n_out);
    if (nt > 65535) return SP_ELIMIT;
    d.xt = staged;
    d.pitch = pitch;
    d.n_out = n_out;
    d.out = out;
    d.tile_first = p->d_tile_first;
    d.tile_count = p->d_tile_count;
    d.geo = p->d_chunk_geo;
    d.off = p->d_chunk_off;
    d.nchan = p->nchan;
    d.nchunks = p->nchunks;
    d.ntiles = p->ntiles;
    d.ntime = (int32_t)nt;
    *items = (int64_t)p->ntiles * nt;
    return SP_OK;
}

// Shape, staging sizes and shared memory of a launch over these plans (all
// of one shape); persistent grid size for it on the current device.
int launch_geometry(const std::vector<const sp_plan *> &plans, BatchLaunch &L) {
    if (plans.empty()) return SP_EINVAL;
    const sp_plan *p0 = plans[0];
    L.shape = p0->shape;
    L.copies_max = 0;
    L.raw_max = 0;
    for (const sp_plan *p : plans) {
        if (p->shape != L.shape) return SP_EINVAL;
        L.copies_max = std::max(L.copies_max, p->copies_max);
        L.raw_max = std::max(L.raw_max, p->raw_max);
    }
    L.smem_bytes = dedisp_header_bytes(p0->chan_chunk, p0->dm_tile) + kDedispRawSlots * L.raw_max + 2 * L.copies_max;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    if (L.smem_bytes > optin) return SP_ELIMIT;
    return batch_grid(L);
}

}  // namespace

extern "C" int64_t sp_dedisperse_batch_workspace_bytes(int32_t nbeams) {
    return nbeams > 0 ? table_bytes(nbeams) : -1;
}

extern "C" int sp_dedisperse_batch(const sp_batch_beam *h_beams, int32_t nbeams, void *d_work, int64_t work_bytes,
                                   void *stream) {
    if (!h_beams || nbeams <= 0) return SP_EINVAL;
    if (!d_work || work_bytes < table_bytes(nbeams) || (reinterpret_cast<uintptr_t>(d_work) & 255))
        return SP_EWORKSPACE;
    std::vector<BatchBeamDev> dev((size_t)nbeams);
    std::vector<int64_t> begin((size_t)nbeams + 1, 0);
    std::vector<const sp_plan *> plans;
    for (int32_t b = 0; b < nbeams; ++b) {
        const sp_batch_beam &x = h_beams[b];
        int64_t items = 0;
        const int rc = describe(x.plan, x.d_staged, x.pitch, x.n_in, x.d_out, x.n_out, dev[b], &items);
        if (rc) return rc;
        begin[b + 1] = begin[b] + items;
        plans.push_back(x.plan);
    }
    BatchLaunch L{};
    int rc = launch_geometry(plans, L);
    if (rc) return rc;
    uint8_t *w = reinterpret_cast<uint8_t *>(d_work);
    L.nbeams = nbeams;
    L.nitems = begin[nbeams];
    L.d_counter = reinterpret_cast<unsigned long long *>(w);
    L.d_beams = reinterpret_cast<const BatchBeamDev *>(w + kCounterBytes);
    L.d_item_begin =
        reinterpret_cast<const int64_t *>(w + kCounterBytes + align256((int64_t)nbeams * sizeof(BatchBeamDev)));
    L.d_status = h_beams[0].plan->d_status;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // Host arrays are pageable: each copy has read its source when it returns.
    if (cudaMemcpyAsync(const_cast<BatchBeamDev *>(L.d_beams), dev.data(), dev.size() * sizeof(BatchBeamDev),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(const_cast<int64_t *>(L.d_item_begin), begin.data(), begin.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SP_ECUDA;
    return launch_dedisperse_batch(L, st);
}

// ------------------------------------------------------------------ batch --
struct sp_batch {
    int device = 0;
    std::vector<const sp_plan *> plans;
    int32_t nbeams = 0;
    std::vector<int32_t> beam_plan;
    std::vector<int64_t> n_out, n_in, pitch;
    int32_t widths[SP_MAX_WIDTHS] = {0};
    int32_t nw = 0;
    float threshold = 0.f;
    int64_t norm_block = 0;
    int64_t cap = 0;
    // Groups: beams [first, last) share one persistent launch; their staged
    // inputs and DM transforms sit at the offsets below in arena g & 1.
    struct Group {
        int32_t first = 0, last = 0;
        BatchLaunch launch{};
    };
    std::vector<Group> groups;
    std::vector<int64_t> staged_off, dmt_off;  // per beam, within its group's arena
    int64_t staged_arena = 0, dmt_arena = 0;
    // Device memory.
    uint8_t *d_in = nullptr;                   // every beam's input
    std::vector<int64_t> in_off;
    uint8_t *d_staged[2] = {nullptr, nullptr};
    int32_t *d_dmt[2] = {nullptr, nullptr};
    void *d_sps = nullptr;
    int64_t sps_bytes = 0;
    sp_cand *d_cands = nullptr;                // [nbeams][cap]
    int64_t *d_counts = nullptr;               // [nbeams]
    uint8_t *d_tables = nullptr;               // per group: counter, beam table, item offsets
    int32_t *d_status = nullptr;
    int64_t device_bytes = 0;
    // Execution.
    cudaStream_t side = nullptr;               // search stream of the grouped mode
    cudaStream_t copy = nullptr;               // host input copies of sp_batch_run_host
    std::vector<cudaEvent_t> ev_in;            // per group: its beams' inputs are on the device
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_dd[2] = {nullptr, nullptr}, ev_sps[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev_t0, ev_t1;     // per group, around its persistent launch (timed runs)
    bool timed_valid = false;
    cudaGraphExec_t graph = nullptr;
    uint64_t graph_kernels = 0;  // kernels recorded in the graph
    int last_mode = -1;
};

namespace {

void batch_free(sp_batch *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaEvent_t e : {b->ev_fork, b->ev_join, b->ev_dd[0], b->ev_dd[1], b->ev_sps[0], b->ev_sps[1]})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_t0) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_t1) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_in) if (e) cudaEventDestroy(e);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->copy) cudaStreamDestroy(b->copy);
    cudaFree(b->d_in);
    cudaFree(b->d_staged[0]);
    cudaFree(b->d_staged[1]);
    cudaFree(b->d_dmt[0]);
    cudaFree(b->d_dmt[1]);
    cudaFree(b->d_sps);
    cudaFree(b->d_cands);
    cudaFree(b->d_counts);
    cudaFree(b->d_tables);
    cudaFree(b->d_status);
}

int dev_alloc(void **p, int64_t bytes, int64_t *total) {
    if (cudaMalloc(p, (size_t)std::max<int64_t>(bytes, 256)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SP_ENOMEM;
    }
    *total += std::max<int64_t>(bytes, 256);
    return SP_OK;
}

const sp_plan *plan_of(const sp_batch *b, int32_t beam) { return b->plans[b->beam_plan[beam]]; }

int search_beam(sp_batch *b, int32_t beam, const int32_t *dmt, cudaStream_t st) {
    const sp_plan *p = plan_of(b, beam);
    SpsArgs a;
    std::memset(&a, 0, sizeof a);
    a.dmt = dmt;
    a.ndm = p->ndm;
    a.n_out = b->n_out[beam];
    for (int k = 0; k < b->nw; ++k) a.widths[k] = b->widths[k];
    a.nw = b->nw;
    a.threshold = b->threshold;
    a.norm_block = b->norm_block;
    a.nblk = sps_nblocks(a.n_out, b->norm_block);
    a.work = b->d_sps;
    a.cands = b->d_cands + (int64_t)beam * b->cap;
    a.cap = b->cap;
    a.count = b->d_counts + beam;
    return launch_sps(a, st);
}

// h_in != nullptr: the beams' inputs come from host memory first, group by
// group on the copy stream, so that group g + 1's copies overlap group g's
// work and each group waits only for its own.
int run_grouped(sp_batch *b, cudaStream_t s0, bool timed, bool persistent, const uint8_t *const *h_in = nullptr) {
    if (cudaEventRecord(b->ev_fork, s0) != cudaSuccess || cudaStreamWaitEvent(b->side, b->ev_fork, 0) != cudaSuccess)
        return SP_ECUDA;
    if (h_in) {
        if (cudaStreamWaitEvent(b->copy, b->ev_fork, 0) != cudaSuccess) return SP_ECUDA;
        for (size_t g = 0; g < b->groups.size(); ++g) {
            for (int32_t beam = b->groups[g].first; beam < b->groups[g].last; ++beam) {
                const size_t bytes = (size_t)(b->n_in[beam] * plan_of(b, beam)->nchan);
                if (cudaMemcpyAsync(b->d_in + b->in_off[beam], h_in[beam], bytes, cudaMemcpyHostToDevice, b->copy) !=
                    cudaSuccess)
                    return SP_ECUDA;
            }
            if (cudaEventRecord(b->ev_in[g], b->copy) != cudaSuccess) return SP_ECUDA;
        }
    }
    for (size_t g = 0; g < b->groups.size(); ++g) {
        const sp_batch::Group &G = b->groups[g];
        const int slot = (int)(g & 1);
        if (g >= 2 && cudaStreamWaitEvent(s0, b->ev_sps[slot], 0) != cudaSuccess) return SP_ECUDA;
        if (h_in && cudaStreamWaitEvent(s0, b->ev_in[g], 0) != cudaSuccess) return SP_ECUDA;
        for (int32_t beam = G.first; beam < G.last; ++beam) {
            const int rc = launch_stage_input(b->d_in + b->in_off[beam], b->n_in[beam], plan_of(b, beam)->nchan,
                                              b->d_staged[slot] + b->staged_off[beam], b->pitch[beam], s0);
            if (rc) return rc;
        }
        if (timed && cudaEventRecord(b->ev_t0[g], s0) != cudaSuccess) return SP_ECUDA;
        int rc = launch_dedisperse_batch(G.launch, s0, persistent);
        if (rc) return rc;
        if (timed && cudaEventRecord(b->ev_t1[g], s0) != cudaSuccess) return SP_ECUDA;
        if (cudaEventRecord(b->ev_dd[slot], s0) != cudaSuccess ||
            cudaStreamWaitEvent(b->side, b->ev_dd[slot], 0) != cudaSuccess)
            return SP_ECUDA;
        for (int32_t beam = G.first; beam < G.last; ++beam) {
            rc = search_beam(b, beam, b->d_dmt[slot] + b->dmt_off[beam], b->side);
            if (rc) return rc;
        }
        if (cudaEventRecord(b->ev_sps[slot], b->side) != cudaSuccess) return SP_ECUDA;
    }
    if (cudaEventRecord(b->ev_join, b->side) != cudaSuccess || cudaStreamWaitEvent(s0, b->ev_join, 0) != cudaSuccess)
        return SP_ECUDA;
    return SP_OK;
}

int run_per_beam(sp_batch *b, cudaStream_t s0) {
    for (int32_t beam = 0; beam < b->nbeams; ++beam) {
        const sp_plan *p = plan_of(b, beam);
        int rc = launch_stage_input(b->d_in + b->in_off[beam], b->n_in[beam], p->nchan, b->d_staged[0],
                                    b->pitch[beam], s0);
        if (!rc) rc = launch_dedisperse(p, b->d_staged[0], b->pitch[beam], b->n_out[beam], b->d_dmt[0], s0);
        if (!rc) rc = search_beam(b, beam, b->d_dmt[0], s0);
        if (rc) return rc;
    }
    return SP_OK;
}

int run_mode(sp_batch *b, int32_t mode, cudaStream_t s0, bool timed = false) {
    int rc = SP_EINVAL;
    if (mode == SP_BATCH_GROUPED) rc = run_grouped(b, s0, timed, true);
    else if (mode == SP_BATCH_GROUPED_GRID) rc = run_grouped(b, s0, timed, false);
    else if (mode == SP_BATCH_PER_BEAM) rc = run_per_beam(b, s0);
    if (!rc) b->last_mode = mode;
    b->timed_valid = !rc && timed;
    return rc;
}

bool on_device(const sp_batch *b) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return dev == b->device;
}

}  // namespace

extern "C" int sp_batch_create(const sp_plan *const *plans, int32_t nplans, const int32_t *h_beam_plan,
                               const int64_t *h_beam_n_out, int32_t nbeams, const int32_t *h_widths, int32_t nw,
                               float threshold, int64_t norm_block, int64_t cand_cap, int64_t dmt_budget_bytes,
                               sp_batch **out) {
    if (!out) return SP_EINVAL;
    *out = nullptr;
    if (!plans || nplans <= 0 || !h_beam_plan || !h_beam_n_out || nbeams <= 0 || cand_cap < 0 ||
        dmt_budget_bytes <= 0)
        return SP_EINVAL;
    int rc = check_widths(h_widths, nw);
    if (rc) return rc;
    for (int32_t i = 0; i < nplans; ++i)
        if (!plans[i] || !on_plan_device(plans[i]) || plans[i]->shape != plans[0]->shape) return SP_EINVAL;
    sp_batch *b = new (std::nothrow) sp_batch();
    if (!b) return SP_ENOMEM;
    b->device = plans[0]->device;
    b->plans.assign(plans, plans + nplans);
    b->nbeams = nbeams;
    std::copy(h_widths, h_widths + nw, b->widths);
    b->nw = nw;
    b->threshold = threshold;
    b->norm_block = norm_block;
    b->cap = cand_cap;
    int64_t in_total = 0, sps_max = 0;
    for (int32_t beam = 0; beam < nbeams; ++beam) {
        const int32_t pi = h_beam_plan[beam];
        const int64_t n_out = h_beam_n_out[beam];
        if (pi < 0 || pi >= nplans || n_out <= 0) rc = SP_EINVAL;
        if (rc) break;
        const sp_plan *p = plans[pi];
        const int64_t n_in = n_out + p->max_delay;
        if (n_in > (int64_t)INT32_MAX - 4096 || dedisp_time_tiles(p, n_out) > 65535 || p->ndm > 65535) {
            rc = SP_ELIMIT;
            break;
        }
        b->beam_plan.push_back(pi);
        b->n_out.push_back(n_out);
        b->n_in.push_back(n_in);
        b->pitch.push_back(dedisp_pitch(n_in));
        b->in_off.push_back(in_total);
        in_total += align256(n_in * p->nchan);
        sps_max = std::max(sps_max, sps_workspace_bytes(p->ndm, n_out, nw, norm_block));
    }
    // Groups: beams in order while their DM transforms fit the budget.
    if (!rc) {
        b->staged_off.assign(nbeams, 0);
        b->dmt_off.assign(nbeams, 0);
        int32_t first = 0;
        int64_t dmt_acc = 0, st_acc = 0;
        for (int32_t beam = 0; beam <= nbeams; ++beam) {
            int64_t dmt_b = 0, st_b = 0;
            if (beam < nbeams) {
                const sp_plan *p = plan_of(b, beam);
                dmt_b = align256((int64_t)p->ndm * b->n_out[beam] * 4);
                st_b = align256((int64_t)p->nchan * b->pitch[beam]);
            }
            if (beam == nbeams || (beam > first && dmt_acc + dmt_b > dmt_budget_bytes)) {
                sp_batch::Group G;
                G.first = first;
                G.last = beam;
                b->groups.push_back(G);
                b->dmt_arena = std::max(b->dmt_arena, dmt_acc);
                b->staged_arena = std::max(b->staged_arena, st_acc);
                first = beam;
                dmt_acc = st_acc = 0;
            }
            if (beam < nbeams) {
                b->dmt_off[beam] = dmt_acc / 4;
                b->staged_off[beam] = st_acc;
                dmt_acc += dmt_b;
                st_acc += st_b;
            }
        }
    }
    int64_t &tot = b->device_bytes;
    int64_t tables_total = 0;
    for (const sp_batch::Group &G : b->groups) tables_total += table_bytes(G.last - G.first);
    b->sps_bytes = sps_max;
    if (!rc) rc = dev_alloc((void **)&b->d_in, in_total, &tot);
    for (int s = 0; s < 2 && !rc; ++s) {
        rc = dev_alloc((void **)&b->d_staged[s], b->staged_arena, &tot);
        if (!rc) rc = dev_alloc((void **)&b->d_dmt[s], b->dmt_arena, &tot);
    }
    if (!rc) rc = dev_alloc(&b->d_sps, sps_max, &tot);
    if (!rc) rc = dev_alloc((void **)&b->d_cands, (int64_t)nbeams * std::max<int64_t>(cand_cap, 1) * sizeof(sp_cand), &tot);
    if (!rc) rc = dev_alloc((void **)&b->d_counts, (int64_t)nbeams * 8, &tot);
    if (!rc) rc = dev_alloc((void **)&b->d_tables, tables_total, &tot);
    if (!rc) rc = dev_alloc((void **)&b->d_status, 4, &tot);
    if (!rc && (cudaMemset(b->d_status, 0, 4) != cudaSuccess || cudaMemset(b->d_counts, 0, (size_t)nbeams * 8) != cudaSuccess))
        rc = SP_ECUDA;
    // Per-group launch tables, pointing into the group's arena.
    int64_t toff = 0;
    for (size_t g = 0; g < b->groups.size() && !rc; ++g) {
        sp_batch::Group &G = b->groups[g];
        const int slot = (int)(g & 1);
        const int32_t n = G.last - G.first;
        std::vector<BatchBeamDev> dev((size_t)n);
        std::vector<int64_t> begin((size_t)n + 1, 0);
        std::vector<const sp_plan *> gp;
        for (int32_t i = 0; i < n && !rc; ++i) {
            const int32_t beam = G.first + i;
            int64_t items = 0;
            rc = describe(plan_of(b, beam), b->d_staged[slot] + b->staged_off[beam], b->pitch[beam], b->n_in[beam],
                          b->d_dmt[slot] + b->dmt_off[beam], b->n_out[beam], dev[i], &items);
            begin[i + 1] = begin[i] + items;
            gp.push_back(plan_of(b, beam));
        }
        if (!rc) rc = launch_geometry(gp, G.launch);
        if (rc) break;
        uint8_t *w = b->d_tables + toff;
        G.launch.nbeams = n;
        G.launch.nitems = begin[n];
        G.launch.d_counter = reinterpret_cast<unsigned long long *>(w);
        G.launch.d_beams = reinterpret_cast<const BatchBeamDev *>(w + kCounterBytes);
        G.launch.d_item_begin =
            reinterpret_cast<const int64_t *>(w + kCounterBytes + align256((int64_t)n * sizeof(BatchBeamDev)));
        G.launch.d_status = b->d_status;
        if (cudaMemcpy(const_cast<BatchBeamDev *>(G.launch.d_beams), dev.data(), dev.size() * sizeof(BatchBeamDev),
                       cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(const_cast<int64_t *>(G.launch.d_item_begin), begin.data(), begin.size() * sizeof(int64_t),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            rc = SP_ECUDA;
        toff += table_bytes(n);
    }
    // Kernel attributes are set now so that no run, in or out of a graph
    // capture, has to set them.
    for (int32_t i = 0; i < nplans && !rc; ++i) rc = dedisp_configure(plans[i]);
    if (!rc) rc = sps_configure(h_widths[nw - 1]);
    int prio_lo = 0, prio_hi = 0;  // the search stream gets the device's highest priority
    if (!rc && (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
                cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
                cudaStreamCreateWithFlags(&b->copy, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_dd[0], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_dd[1], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_sps[0], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_sps[1], cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        rc = SP_ECUDA;
    }
    if (!rc) {
        b->ev_t0.assign(b->groups.size(), nullptr);
        b->ev_t1.assign(b->groups.size(), nullptr);
        b->ev_in.assign(b->groups.size(), nullptr);
        for (size_t g = 0; g < b->groups.size() && !rc; ++g)
            if (cudaEventCreate(&b->ev_t0[g]) != cudaSuccess || cudaEventCreate(&b->ev_t1[g]) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->ev_in[g], cudaEventDisableTiming) != cudaSuccess) {
                cudaGetLastError();
                rc = SP_ECUDA;
            }
    }
    if (rc) {
        batch_free(b);
        delete b;
        return rc;
    }
    *out = b;
    return SP_OK;
}

extern "C" int sp_batch_destroy(sp_batch *b) {
    if (!b) return SP_EINVAL;
    batch_free(b);
    delete b;
    return SP_OK;
}

extern "C" int sp_batch_info(const sp_batch *b, int32_t *ngroups, int64_t *device_bytes) {
    if (!b) return SP_EINVAL;
    if (ngroups) *ngroups = (int32_t)b->groups.size();
    if (device_bytes) *device_bytes = b->device_bytes;
    return SP_OK;
}

extern "C" int sp_batch_input(sp_batch *b, int32_t beam, uint8_t **d_in, int64_t *n_in) {
    if (!b || beam < 0 || beam >= b->nbeams || !d_in) return SP_EINVAL;
    *d_in = b->d_in + b->in_off[beam];
    if (n_in) *n_in = b->n_in[beam];
    return SP_OK;
}

extern "C" int sp_batch_run(sp_batch *b, int32_t mode, void *stream) {
    if (!b || !on_device(b)) return SP_EINVAL;
    const bool timed = (mode & SP_BATCH_TIMED) != 0;
    return run_mode(b, mode & ~SP_BATCH_TIMED, reinterpret_cast<cudaStream_t>(stream), timed);
}

extern "C" int sp_batch_group_ms(const sp_batch *b, float *h_ms) {
    if (!b || !h_ms || !b->timed_valid) return SP_EINVAL;
    for (size_t g = 0; g < b->groups.size(); ++g)
        if (cudaEventSynchronize(b->ev_t1[g]) != cudaSuccess ||
            cudaEventElapsedTime(&h_ms[g], b->ev_t0[g], b->ev_t1[g]) != cudaSuccess)
            return SP_ECUDA;
    return SP_OK;
}

extern "C" int sp_batch_capture(sp_batch *b, int32_t mode, void *stream) {
    if (!b || !stream || !on_device(b) ||
        (mode != SP_BATCH_GROUPED && mode != SP_BATCH_PER_BEAM && mode != SP_BATCH_GROUPED_GRID))
        return SP_EINVAL;
    b->timed_valid = false;
    cudaStream_t s0 = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    capture_begin();
    const int rc = run_mode(b, mode, s0);
    const uint64_t kernels = capture_end();
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(s0, &graph);
    if (rc || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc ? rc : SP_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = exec;
    b->graph_kernels = kernels;
    return SP_OK;
}

extern "C" int sp_batch_launch(sp_batch *b, void *stream) {
    if (!b || !b->graph || !on_device(b)) return SP_EINVAL;
    if (cudaGraphLaunch(b->graph, reinterpret_cast<cudaStream_t>(stream)) != cudaSuccess) return SP_ECUDA;
    note_launch(b->graph_kernels);
    return SP_OK;
}

extern "C" int sp_batch_results(sp_batch *b, int32_t beam, sp_cand *h_cands, int64_t cap, int64_t *h_count,
                                void *stream) {
    if (!b || beam < 0 || beam >= b->nbeams || !h_count || cap < 0 || (cap > 0 && !h_cands)) return SP_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int64_t total = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess ||
        cudaMemcpy(&total, b->d_counts + beam, sizeof total, cudaMemcpyDeviceToHost) != cudaSuccess)
        return SP_ECUDA;
    *h_count = total;
    const int64_t lim = std::min(cap, b->cap);
    const int64_t n = std::min(total, lim);
    if (n > 0 && cudaMemcpy(h_cands, b->d_cands + (int64_t)beam * b->cap, (size_t)n * sizeof(sp_cand),
                            cudaMemcpyDeviceToHost) != cudaSuccess)
        return SP_ECUDA;
    return total > lim ? SP_EOVERFLOW : SP_OK;
}

extern "C" int sp_batch_dmt(const sp_batch *b, int32_t beam, const int32_t **d_dmt) {
    if (!b || beam < 0 || beam >= b->nbeams || !d_dmt) return SP_EINVAL;
    if (b->last_mode == SP_BATCH_PER_BEAM) {
        if (beam != b->nbeams - 1) return SP_EINVAL;
        *d_dmt = b->d_dmt[0];
        return SP_OK;
    }
    if (b->last_mode != SP_BATCH_GROUPED && b->last_mode != SP_BATCH_GROUPED_GRID) return SP_EINVAL;
    const int32_t ng = (int32_t)b->groups.size();
    for (int32_t g = std::max(0, ng - 2); g < ng; ++g) {
        const sp_batch::Group &G = b->groups[g];
        if (beam >= G.first && beam < G.last) {
            *d_dmt = b->d_dmt[g & 1] + b->dmt_off[beam];
            return SP_OK;
        }
    }
    return SP_EINVAL;
}

extern "C" int sp_batch_run_host(sp_batch *b, const uint8_t *const *h_in, sp_cand *h_cands, int64_t cap_per_beam,
                                 int64_t *h_counts, void *stream) {
    if (!b || !h_in || !h_counts || cap_per_beam < 0 || (cap_per_beam > 0 && !h_cands) || !on_device(b))
        return SP_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    for (int32_t beam = 0; beam < b->nbeams; ++beam)
        if (!h_in[beam]) return SP_EINVAL;
    int rc = run_grouped(b, st, false, false, h_in);  // one CTA per work item
    b->last_mode = rc ? b->last_mode : SP_BATCH_GROUPED_GRID;
    b->timed_valid = false;
    if (rc) return rc;
    if (cudaMemcpyAsync(h_counts, b->d_counts, (size_t)b->nbeams * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SP_ECUDA;
    const int64_t lim = std::min(cap_per_beam, b->cap);
    bool over = false;
    for (int32_t beam = 0; beam < b->nbeams; ++beam) {
        const int64_t n = std::min(h_counts[beam], lim);
        over = over || h_counts[beam] > lim;
        if (n > 0 && cudaMemcpyAsync(h_cands + (int64_t)beam * cap_per_beam, b->d_cands + (int64_t)beam * b->cap,
                                     (size_t)n * sizeof(sp_cand), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return SP_ECUDA;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return SP_ECUDA;
    return over ? SP_EOVERFLOW : SP_OK;
}

extern "C" int sp_batch_status(const sp_batch *b, int32_t *h_status, int32_t clear) {
    if (!b || !h_status || !on_device(b)) return SP_EINVAL;
    if (cudaDeviceSynchronize() != cudaSuccess) return SP_ECUDA;
    int32_t acc = 0, v = 0;
    if (cudaMemcpy(&v, b->d_status, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return SP_ECUDA;
    acc |= v;
    if (clear && cudaMemset(b->d_status, 0, 4) != cudaSuccess) return SP_ECUDA;
    for (const sp_plan *p : b->plans) {
        int32_t s = 0;
        const int rc = sp_plan_status(p, &s, clear);
        if (rc) return rc;
        acc |= s;
    }
    *h_status = acc;
    return SP_OK;
}
