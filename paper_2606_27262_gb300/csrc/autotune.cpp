// autotune.cpp -- picks the dedispersion kernel shape (DM tile x time tile x
// channel chunk) for a plan by timing every compiled shape on a bounded
// sample of the plan's own work.  The shapes compute identical results; only
// their speed differs, and it depends on the channel count, the spread of
// the delays across a DM tile and the GPU, so it is measured rather than
// modelled.
#include <cmath>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "sp_internal.h"

using namespace sp;

namespace {

std::mutex g_tune_lock;
std::map<std::string, std::vector<float>> g_tune_cache;  // key: device + every input byte

std::string tune_key(int dev, const double *freqs, int32_t nchan, double tsamp, const double *dms, int32_t ndm,
                     int64_t n_out, int32_t reps) {
    std::string k;
    auto put = [&k](const void *p, size_t n) { k.append(reinterpret_cast<const char *>(p), n); };
    put(&dev, sizeof dev);
    put(&nchan, sizeof nchan);
    put(&ndm, sizeof ndm);
    put(&tsamp, sizeof tsamp);
    put(&n_out, sizeof n_out);
    put(&reps, sizeof reps);
    put(freqs, sizeof(double) * (size_t)nchan);
    put(dms, sizeof(double) * (size_t)ndm);
    return k;
}

// Mean milliseconds per launch of one shape, +inf if the shape cannot run.
int time_shape(int32_t shape, const double *freqs, int32_t nchan, double tsamp, const double *dms, int32_t ndm,
               int64_t n_out, int32_t reps, cudaStream_t st, float *ms_out) {
    *ms_out = std::numeric_limits<float>::infinity();
    sp_plan *p = nullptr;
    int rc = sp_plan_create_shaped(freqs, nchan, tsamp, dms, ndm, shape, &p);
    if (rc == SP_ELIMIT) return SP_OK;  // this shape cannot hold the plan's tiles
    if (rc) return rc;
    const int64_t n_in = n_out + p->max_delay;
    const int64_t pitch = dedisp_pitch(n_in);
    uint8_t *staged = nullptr;
    int32_t *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (dedisp_time_tiles(p, n_out) > 65535) {
        sp_plan_destroy(p);
        return SP_OK;
    }
    bool ok = cudaMalloc((void **)&staged, (size_t)(nchan * pitch)) == cudaSuccess &&
              cudaMalloc((void **)&out, (size_t)p->ndm * n_out * 4) == cudaSuccess &&
              cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        rc = SP_ENOMEM;
    }
    // Timing does not depend on the byte values; any fixed pattern serves.
    if (!rc && cudaMemsetAsync(staged, 0x5a, (size_t)(nchan * pitch), st) != cudaSuccess) rc = SP_ECUDA;
    if (!rc) rc = launch_dedisperse(p, staged, pitch, n_out, out, st);  // warm-up
    if (!rc && cudaEventRecord(e0, st) != cudaSuccess) rc = SP_ECUDA;
    for (int32_t r = 0; !rc && r < reps; ++r) rc = launch_dedisperse(p, staged, pitch, n_out, out, st);
    if (!rc && cudaEventRecord(e1, st) != cudaSuccess) rc = SP_ECUDA;
    float ms = 0.f;
    if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = SP_ECUDA;
    int32_t status = 0;
    if (!rc && cudaMemcpy(&status, p->d_status, sizeof status, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = SP_ECUDA;
    if (!rc && status == 0) *ms_out = ms / (float)reps;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(staged);
    cudaFree(out);
    sp_plan_destroy(p);
    return rc;
}

}  // namespace

extern "C" int sp_autotune_dedisperse(const double *freqs_mhz, int32_t nchan, double tsamp_s, const double *dms,
                                      int32_t ndm, int64_t n_out_sample, int32_t reps, float *h_ms, int32_t *best,
                                      void *stream) {
    if (!freqs_mhz || !dms || nchan <= 0 || ndm <= 0 || n_out_sample < 1 || reps < 1 || !h_ms || !best)
        return SP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    const std::string key = tune_key(dev, freqs_mhz, nchan, tsamp_s, dms, ndm, n_out_sample, reps);
    std::vector<float> ms;
    {
        std::lock_guard<std::mutex> guard(g_tune_lock);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) ms = it->second;
    }
    if (ms.empty()) {
        cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
        ms.assign(kDedispNumShapes, std::numeric_limits<float>::infinity());
        for (int32_t s = 0; s < kDedispNumShapes; ++s) {
            const int rc = time_shape(s, freqs_mhz, nchan, tsamp_s, dms, ndm, n_out_sample, reps, st, &ms[s]);
            if (rc) return rc;
        }
        std::lock_guard<std::mutex> guard(g_tune_lock);
        g_tune_cache[key] = ms;
    }
    int32_t b = -1;
    for (int32_t s = 0; s < kDedispNumShapes; ++s) {
        h_ms[s] = ms[s];
        if (std::isfinite(ms[s]) && (b < 0 || ms[s] < ms[b])) b = s;
    }
    if (b < 0) return SP_ELIMIT;
    *best = b;
    return SP_OK;
}
