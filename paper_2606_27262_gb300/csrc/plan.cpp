// plan.cpp -- dedispersion plan: the delay table of Eq. 1 and the DM-tile
// layout of the dedispersion kernel.  Built with -ffp-contract=off so that
// the binary64 expression is evaluated exactly as written (no fused
// multiply-add), left to right.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>

#include "sp_internal.h"

namespace sp {

// Eq. 1 of arXiv 2606.27262 (Sec. 3.1.1): dispersion delay of frequency f
// relative to the highest frequency of the band, in samples, rounded half up.
// The dispersion constant is Eq. 1's 4.1488064239e3 rounded to 4.148808e3
// MHz^2 pc^-1 cm^3 s.
static const double kDispersionConstant = 4.148808e3;

int compute_delays(const double *freqs, int32_t nchan, double tsamp, const double *dms,
                   int32_t ndm, std::vector<int32_t> &out, int32_t *max_delay) {
    if (!freqs || !dms || nchan <= 0 || ndm <= 0 || !(tsamp > 0.0)) return SP_EINVAL;
    for (int32_t c = 0; c < nchan; ++c) {
        if (!(freqs[c] > 0.0) || !std::isfinite(freqs[c])) return SP_EINVAL;
        if (c > 0 && !(freqs[c] < freqs[c - 1])) return SP_EINVAL;
    }
    for (int32_t d = 0; d < ndm; ++d)
        if (!(dms[d] >= 0.0) || !std::isfinite(dms[d])) return SP_EINVAL;
    if ((int64_t)ndm * nchan > (int64_t)INT32_MAX) return SP_ELIMIT;
    out.resize((size_t)ndm * nchan);
    const double ftop = freqs[0];
    int32_t mx = 0;
    for (int32_t d = 0; d < ndm; ++d) {
        const double dm = dms[d];
        for (int32_t c = 0; c < nchan; ++c) {
            const double f = freqs[c];
            const double x = kDispersionConstant * dm * (1.0 / (f * f) - 1.0 / (ftop * ftop)) / tsamp;
            const double r = std::floor(x + 0.5);
            if (!(r < 1.0e9)) return SP_ELIMIT;
            const int32_t v = (int32_t)r;
            out[(size_t)d * nchan + c] = v;
            mx = std::max(mx, v);
        }
    }
    *max_delay = mx;
    return SP_OK;
}

// Staging tables of the dedispersion kernel, per (DM tile, channel chunk).
// Time tiles start at multiples of the time tile (a multiple of 16), so the
// 16-byte-aligned window start of a channel relative to the time tile is
// (min delay over the tile) rounded down to 16 and does not depend on the
// time tile; neither do the offsets derived from it.  A channel occupies
// R + 16 bytes of a raw staging slot (the window plus the 16 bytes its
// shifted copies reach past it) and 4 R bytes of a copies buffer (its four
// byte-shifted copies, stride R).
void build_chunk_tables(const sp_plan &p, std::vector<int32_t> &geo, std::vector<int32_t> &off,
                        int32_t *copies_max, int32_t *raw_max) {
    const int32_t CH = p.chan_chunk, DT = p.dm_tile;
    geo.assign((size_t)p.ntiles * p.nchunks * CH * 4, 0);
    off.assign((size_t)p.ntiles * p.nchunks * CH * DT, 0);
    int32_t cmax = 0, rmax = 0;
    for (int32_t j = 0; j < p.ntiles; ++j) {
        const int32_t d0 = p.tile_first[j], cnt = p.tile_count[j];
        for (int32_t k = 0; k < p.nchunks; ++k) {
            const int32_t c0 = k * CH;
            const int32_t nc = std::min(CH, p.nchan - c0);
            int32_t soff = 0, roff = 0;
            for (int32_t i = 0; i < nc; ++i) {
                const int32_t c = c0 + i;
                int32_t lo = INT32_MAX, hi = 0;
                for (int32_t dl = 0; dl < cnt; ++dl) {
                    const int32_t v = p.delays[(size_t)(d0 + dl) * p.nchan + c];
                    lo = std::min(lo, v);
                    hi = std::max(hi, v);
                }
                const int32_t rel_base = lo & ~15;
                const int32_t R = dedisp_row_bytes(hi - lo, p.time_tile);
                const int32_t stride = R;  // copies are derived from the raw slot: no tail needed
                int32_t *g = &geo[(((size_t)j * p.nchunks + k) * CH + i) * 4];
                g[0] = rel_base;
                g[1] = R;
                g[2] = soff;
                g[3] = roff;
                int32_t *o = &off[(((size_t)j * p.nchunks + k) * CH + i) * DT];
                for (int32_t dl = 0; dl < DT; ++dl) {
                    const int32_t dd = std::min(dl, cnt - 1);  // idle slots repeat the last DM
                    const int32_t shift = p.delays[(size_t)(d0 + dd) * p.nchan + c] - rel_base;
                    o[dl] = soff + (shift & 3) * stride + (shift & ~3);
                }
                soff += 4 * stride;
                roff += R + 16;
            }
            cmax = std::max(cmax, soff);
            rmax = std::max(rmax, roff);
        }
    }
    *copies_max = cmax;
    *raw_max = rmax;
}

}  // namespace sp

using namespace sp;

static void free_plan_device(sp_plan *p) {
    cudaFree(p->d_delays);
    cudaFree(p->d_tile_first);
    cudaFree(p->d_tile_count);
    cudaFree(p->d_chunk_geo);
    cudaFree(p->d_chunk_off);
    cudaFree(p->d_status);
    p->d_delays = p->d_tile_first = p->d_tile_count = p->d_chunk_off = p->d_status = nullptr;
    p->d_chunk_geo = nullptr;
}

template <class T>
static int upload(T **dst, const T *src, size_t n) {
    if (cudaMalloc((void **)dst, n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return SP_ENOMEM;
    }
    if (cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return SP_ECUDA;
    return SP_OK;
}

// The host half of a plan: delays, DM tiles, staging tables and the
// kernel's shared-memory size; no device memory.
static int build_host_plan(const double *freqs_mhz, int32_t nchan, double tsamp_s, const double *dms, int32_t ndm,
                           int32_t shape, sp_plan *p, std::vector<int32_t> &geo, std::vector<int32_t> &off) {
    if (shape < 0 || shape >= kDedispNumShapes) return SP_EINVAL;
    int rc = compute_delays(freqs_mhz, nchan, tsamp_s, dms, ndm, p->delays, &p->max_delay);
    if (rc) return rc;
    p->nchan = nchan;
    p->ndm = ndm;
    p->tsamp = tsamp_s;
    p->freqs.assign(freqs_mhz, freqs_mhz + nchan);
    p->dms.assign(dms, dms + ndm);
    p->shape = shape;
    p->chan_chunk = kDedispShapeCh[shape];
    p->dm_tile = kDedispShapeNdt[shape] * p->chan_chunk;
    p->time_tile = 32 * kDedispShapeSpt[shape];
    const int32_t max_span = kDedispShapeMaxSpan[shape];
    const int32_t half_tile = 4 * p->chan_chunk;  // 4 DMs per thread

    // DM tiles: greedy runs of consecutive trial DMs (list order) with at
    // most dm_tile members and a per-channel delay spread (max - min over
    // the run) of at most the shape's span.  A single DM has spread 0, so
    // every plan tiles.  For a shape of 8 DMs per thread a run that cannot
    // reach 3/4 of the tile is cut to 4 DMs per thread instead (a tile of
    // 33..47 DMs would leave a quarter or more of its threads' DMs idle).
    std::vector<int32_t> lo(nchan), hi(nchan);
    int32_t d = 0;
    while (d < ndm) {
        const int32_t *row = &p->delays[(size_t)d * nchan];
        std::copy(row, row + nchan, lo.begin());
        std::copy(row, row + nchan, hi.begin());
        int32_t cnt = 1;
        while (cnt < p->dm_tile && d + cnt < ndm) {
            const int32_t *r2 = &p->delays[(size_t)(d + cnt) * nchan];
            bool ok = true;
            for (int32_t c = 0; c < nchan && ok; ++c) {
                const int32_t l = std::min(lo[c], r2[c]), h = std::max(hi[c], r2[c]);
                ok = (h - l) <= max_span;
            }
            if (!ok) break;
            for (int32_t c = 0; c < nchan; ++c) {
                lo[c] = std::min(lo[c], r2[c]);
                hi[c] = std::max(hi[c], r2[c]);
            }
            ++cnt;
        }
        if (p->dm_tile > half_tile && cnt > half_tile && 4 * cnt < 3 * p->dm_tile) cnt = half_tile;
        p->tile_first.push_back(d);
        p->tile_count.push_back(cnt);
        d += cnt;
    }
    p->ntiles = (int32_t)p->tile_first.size();
    p->nchunks = (nchan + p->chan_chunk - 1) / p->chan_chunk;
    build_chunk_tables(*p, geo, off, &p->copies_max, &p->raw_max);
    p->smem_bytes = dedisp_header_bytes(p->chan_chunk, p->dm_tile) + kDedispRawSlots * p->raw_max + 2 * p->copies_max;
    return SP_OK;
}

static int create_plan(const double *freqs_mhz, int32_t nchan, double tsamp_s, const double *dms, int32_t ndm,
                       int32_t shape, sp_plan **out) {
    if (!out) return SP_EINVAL;
    *out = nullptr;
    if (shape < 0 || shape >= kDedispNumShapes) return SP_EINVAL;
    sp_plan *p = new (std::nothrow) sp_plan();
    if (!p) return SP_ENOMEM;
    std::vector<int32_t> geo, off;
    int rc = build_host_plan(freqs_mhz, nchan, tsamp_s, dms, ndm, shape, p, geo, off);
    if (rc) {
        delete p;
        return rc;
    }

    int smem_optin = 0;
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return SP_ECUDA;
    }
    if (p->smem_bytes > smem_optin) {  // cannot happen with the compiled shapes and their spans
        delete p;
        return SP_ELIMIT;
    }
    rc = upload(&p->d_delays, p->delays.data(), p->delays.size());
    if (!rc) rc = upload(&p->d_tile_first, p->tile_first.data(), p->tile_first.size());
    if (!rc) rc = upload(&p->d_tile_count, p->tile_count.data(), p->tile_count.size());
    if (!rc) rc = upload(reinterpret_cast<int32_t **>(&p->d_chunk_geo), geo.data(), geo.size());
    if (!rc) rc = upload(&p->d_chunk_off, off.data(), off.size());
    const int32_t zero = 0;
    if (!rc) rc = upload(&p->d_status, &zero, 1);
    if (!rc) rc = dedisp_configure(p);
    if (rc) {
        free_plan_device(p);
        delete p;
        return rc;
    }
    *out = p;
    return SP_OK;
}

extern "C" int sp_plan_create(const double *freqs_mhz, int32_t nchan, double tsamp_s, const double *dms,
                              int32_t ndm, sp_plan **out) {
    return create_plan(freqs_mhz, nchan, tsamp_s, dms, ndm, 0, out);
}

extern "C" int sp_plan_create_shaped(const double *freqs_mhz, int32_t nchan, double tsamp_s, const double *dms,
                                     int32_t ndm, int32_t shape, sp_plan **out) {
    if (shape == SP_SHAPE_AUTO) {
        float ms[SP_DEDISP_NUM_SHAPES];
        const int rc = sp_autotune_dedisperse(freqs_mhz, nchan, tsamp_s, dms, ndm, SP_AUTOTUNE_SAMPLES,
                                              SP_AUTOTUNE_REPS, ms, &shape, nullptr);
        if (rc) return rc;
    }
    return create_plan(freqs_mhz, nchan, tsamp_s, dms, ndm, shape, out);
}

extern "C" int sp_dedisp_shape_info(int32_t shape, int32_t *dm_tile, int32_t *time_tile, int32_t *chan_chunk) {
    if (shape < 0 || shape >= kDedispNumShapes) return SP_EINVAL;
    if (dm_tile) *dm_tile = kDedispShapeNdt[shape] * kDedispShapeCh[shape];
    if (time_tile) *time_tile = 32 * kDedispShapeSpt[shape];
    if (chan_chunk) *chan_chunk = kDedispShapeCh[shape];
    return SP_OK;
}

extern "C" int sp_plan_shape(const sp_plan *p, int32_t *shape, int32_t *ntiles, int32_t *smem_bytes) {
    if (!p) return SP_EINVAL;
    if (shape) *shape = p->shape;
    if (ntiles) *ntiles = p->ntiles;
    if (smem_bytes) *smem_bytes = p->smem_bytes;
    return SP_OK;
}

extern "C" int sp_plan_destroy(sp_plan *p) {
    if (!p) return SP_EINVAL;
    free_plan_device(p);
    delete p;
    return SP_OK;
}

extern "C" int sp_plan_info(const sp_plan *p, int32_t *max_delay, int32_t *nchan, int32_t *ndm) {
    if (!p) return SP_EINVAL;
    if (max_delay) *max_delay = p->max_delay;
    if (nchan) *nchan = p->nchan;
    if (ndm) *ndm = p->ndm;
    return SP_OK;
}

extern "C" int sp_compute_delays(const double *freqs_mhz, int32_t nchan, double tsamp_s, const double *dms,
                                 int32_t ndm, int32_t *h_out, int32_t *max_delay) {
    if (!h_out) return SP_EINVAL;
    std::vector<int32_t> tab;
    int32_t mx = 0;
    const int rc = compute_delays(freqs_mhz, nchan, tsamp_s, dms, ndm, tab, &mx);
    if (rc) return rc;
    std::memcpy(h_out, tab.data(), tab.size() * sizeof(int32_t));
    if (max_delay) *max_delay = mx;
    return SP_OK;
}

extern "C" int sp_plan_status(const sp_plan *p, int32_t *h_status, int32_t clear) {
    if (!p || !h_status) return SP_EINVAL;
    if (cudaMemcpy(h_status, p->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SP_ECUDA;
    if (clear && cudaMemset(p->d_status, 0, sizeof(int32_t)) != cudaSuccess) return SP_ECUDA;
    return SP_OK;
}

extern "C" int sp_plan_delays(const sp_plan *p, int32_t *h_out) {
    if (!p || !h_out) return SP_EINVAL;
    std::memcpy(h_out, p->delays.data(), p->delays.size() * sizeof(int32_t));
    return SP_OK;
}

// Host-side check of the staging tables against every access the
// dedispersion kernel makes with them (see dedisperse.cu): bulk copies of
// raw windows (16-byte aligned, inside the staged row and the raw slot),
// the four shifted copies (inside the copies buffer, rows 16-byte aligned),
// and every shared load of the sums (inside the channel's copy, within the
// R + 16 bytes its copy was built from).
extern "C" int sp_plan_check_tables(const double *freqs_mhz, int32_t nchan, double tsamp_s, const double *dms,
                                    int32_t ndm, int32_t shape, int64_t n_out, int64_t *h_report) {
    if (!h_report || n_out <= 0) return SP_EINVAL;
    sp_plan p;
    std::vector<int32_t> geo, off;
    int rc = build_host_plan(freqs_mhz, nchan, tsamp_s, dms, ndm, shape, &p, geo, off);
    if (rc) return rc;
    const int32_t CH = p.chan_chunk, DT = p.dm_tile, T = p.time_tile;
    const int64_t n_in = n_out + p.max_delay;
    const int64_t pitch = dedisp_pitch(n_in);
    const int64_t ntime = (n_out + T - 1) / T;
    int64_t bad = 0;
    for (int32_t j = 0; j < p.ntiles; ++j) {
        for (int32_t k = 0; k < p.nchunks; ++k) {
            const int32_t nc = std::min(CH, p.nchan - k * CH);
            for (int32_t i = 0; i < nc; ++i) {
                const int32_t *g = &geo[(((size_t)j * p.nchunks + k) * CH + i) * 4];
                const int32_t rel = g[0], R = g[1], soff = g[2], roff = g[3];
                bad += (rel < 0) + (rel % 16 != 0) + (R % 16 != 0) + (R < T) + (soff % 16 != 0) + (roff % 16 != 0);
                bad += (roff + R + 16 > p.raw_max) + (soff + 4 * R > p.copies_max);
                // the last time tile's window must end inside the staged row
                bad += ((ntime - 1) * T + rel + R + 16 > pitch);
                const int32_t *o = &off[(((size_t)j * p.nchunks + k) * CH + i) * DT];
                for (int32_t dl = 0; dl < DT; ++dl) {
                    const int32_t dd = std::min(dl, p.tile_count[j] - 1);
                    const int32_t shift = p.delays[(size_t)(p.tile_first[j] + dd) * p.nchan + k * CH + i] - rel;
                    const int32_t r = shift & 3, w0 = shift & ~3;
                    bad += (shift < 0) + (o[dl] != soff + r * R + w0);
                    // words w0/4 .. (w0 + T)/4 - 1 of copy r: inside the copy
                    // and built from bytes below R + 16 of the raw window
                    bad += (w0 + T > R) + (w0 + T + r > R + 16);
                }
            }
        }
    }
    h_report[0] = p.ntiles;
    h_report[1] = p.nchunks;
    h_report[2] = p.copies_max;
    h_report[3] = p.raw_max;
    h_report[4] = p.smem_bytes;
    h_report[5] = bad;
    h_report[6] = p.max_delay;
    h_report[7] = pitch;
    return SP_OK;
}
