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

}  // namespace sp

using namespace sp;

static void free_plan_device(sp_plan *p) {
    cudaFree(p->d_delays);
    cudaFree(p->d_tile_first);
    cudaFree(p->d_tile_count);
    cudaFree(p->d_tile_dlo);
    cudaFree(p->d_tile_span);
    p->d_delays = p->d_tile_first = p->d_tile_count = p->d_tile_dlo = p->d_tile_span = nullptr;
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

extern "C" int sp_plan_create(const double *freqs_mhz, int32_t nchan, double tsamp_s,
                              const double *dms, int32_t ndm, sp_plan **out) {
    if (!out) return SP_EINVAL;
    *out = nullptr;
    sp_plan *p = new (std::nothrow) sp_plan();
    if (!p) return SP_ENOMEM;
    int rc = compute_delays(freqs_mhz, nchan, tsamp_s, dms, ndm, p->delays, &p->max_delay);
    if (rc) {
        delete p;
        return rc;
    }
    p->nchan = nchan;
    p->ndm = ndm;
    p->tsamp = tsamp_s;

    // DM tiles: greedy runs of consecutive trial DMs (list order) with at
    // most kDedispDmTile members and a per-channel delay spread (max - min
    // over the run) of at most kDedispMaxSpan samples.  A single DM has
    // spread 0, so every plan tiles.
    std::vector<int32_t> lo(nchan), hi(nchan), tile_dlo, tile_span;
    int32_t d = 0;
    int32_t worst_chunk = 0;
    while (d < ndm) {
        const int32_t *row = &p->delays[(size_t)d * nchan];
        std::copy(row, row + nchan, lo.begin());
        std::copy(row, row + nchan, hi.begin());
        int32_t cnt = 1;
        while (cnt < kDedispDmTile && d + cnt < ndm) {
            const int32_t *r2 = &p->delays[(size_t)(d + cnt) * nchan];
            bool ok = true;
            for (int32_t c = 0; c < nchan && ok; ++c) {
                const int32_t l = std::min(lo[c], r2[c]), h = std::max(hi[c], r2[c]);
                ok = (h - l) <= kDedispMaxSpan;
            }
            if (!ok) break;
            for (int32_t c = 0; c < nchan; ++c) {
                lo[c] = std::min(lo[c], r2[c]);
                hi[c] = std::max(hi[c], r2[c]);
            }
            ++cnt;
        }
        p->tile_first.push_back(d);
        p->tile_count.push_back(cnt);
        for (int32_t c = 0; c < nchan; ++c) {
            tile_dlo.push_back(lo[c]);
            tile_span.push_back(hi[c] - lo[c]);
        }
        for (int32_t c0 = 0; c0 < nchan; c0 += kDedispChanChunk) {
            int32_t bytes = 0;
            for (int32_t c = c0; c < std::min(nchan, c0 + kDedispChanChunk); ++c)
                bytes += 4 * dedisp_row_bytes(hi[c] - lo[c]);
            worst_chunk = std::max(worst_chunk, bytes);
        }
        d += cnt;
    }
    p->ntiles = (int32_t)p->tile_first.size();
    p->smem_bytes = worst_chunk + kDedispChanChunk * kDedispDmTile * 4;

    if (cudaGetDevice(&p->device) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return SP_ECUDA;
    }
    rc = upload(&p->d_delays, p->delays.data(), p->delays.size());
    if (!rc) rc = upload(&p->d_tile_first, p->tile_first.data(), p->tile_first.size());
    if (!rc) rc = upload(&p->d_tile_count, p->tile_count.data(), p->tile_count.size());
    if (!rc) rc = upload(&p->d_tile_dlo, tile_dlo.data(), tile_dlo.size());
    if (!rc) rc = upload(&p->d_tile_span, tile_span.data(), tile_span.size());
    if (rc) {
        free_plan_device(p);
        delete p;
        return rc;
    }
    *out = p;
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

extern "C" int sp_plan_delays(const sp_plan *p, int32_t *h_out) {
    if (!p || !h_out) return SP_EINVAL;
    std::memcpy(h_out, p->delays.data(), p->delays.size() * sizeof(int32_t));
    return SP_OK;
}
