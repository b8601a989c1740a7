// sps_noalloc.cu -- sp_single_pulse_search_noalloc: the single-pulse search
// with its scratch (per-row, per-block statistics) in a fixed array that is
// part of the library's device image instead of a caller-allocated workspace.
//
// For callers that cannot allocate device memory when they search: a
// real-time loop that claimed its whole memory budget at start-up and must
// not block or fail on an allocation later, a host application whose device
// memory is owned entirely by its own pool allocator, or a plug-in that is
// not permitted to call cudaMalloc.  They still pass the DM transform and
// the candidate/count outputs; only the scratch comes from here.
//
// The array below exists once per device that loads the library and stays
// resident until the process exits.  Host code cannot use its name as a
// device address; the address is looked up per device with
// cudaGetSymbolAddress the first time the entry point runs on that device
// and kept for the life of the process.  It belongs to the device's primary
// context: a cudaDeviceReset destroys that context, and the kept address is
// stale afterwards, so this entry point must not be used on a device after
// it was reset.
#include <mutex>

#include "sp_internal.h"

namespace {

constexpr int64_t kNoAllocScratchBytes = SP_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_sps_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_sps_scratch on the current device (looked up once per
// device, with that device current).
int scratch_for_current_device(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return SP_ELIMIT;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sps_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SP_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SP_OK;
}

}  // namespace

extern "C" int sp_single_pulse_search_noalloc(const int32_t *d_dmt, int32_t ndm, int64_t n_out,
                                              const int32_t *h_widths, int32_t nw, float threshold,
                                              int64_t norm_block, sp_cand *d_cands, int64_t cap,
                                              int64_t *d_count, void *stream) {
    if (!d_dmt || ndm <= 0 || n_out <= 0 || nw <= 0 || nw > SP_MAX_WIDTHS) return SP_EINVAL;
    if (sp::sps_workspace_bytes(ndm, n_out, nw, norm_block) > kNoAllocScratchBytes) return SP_ELIMIT;
    void *scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    // The statistics kernel overwrites every scratch entry the search reads,
    // and the candidate count is zeroed on the stream before the search, so
    // nothing left from an earlier call is used.
    return sp_single_pulse_search(d_dmt, ndm, n_out, h_widths, nw, threshold, norm_block, scratch,
                                  kNoAllocScratchBytes, d_cands, cap, d_count, stream);
}
