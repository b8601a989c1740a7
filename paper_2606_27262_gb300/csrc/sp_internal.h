// sp_internal.h -- shared declarations of libspotlight's translation units.
// Not installed; the public interface is include/spotlight.h.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/spotlight.h"

namespace sp {

// Dedispersion tiling (see dedisperse.cu for the kernel these describe).
constexpr int kDedispDmPerThread = 4;                     // trial DMs per thread
constexpr int kDedispWarps = 8;                           // warps per CTA
constexpr int kDedispDmTile = kDedispDmPerThread * kDedispWarps;  // 32 DMs per CTA
constexpr int kDedispTimeTile = 512;                      // output samples per CTA
constexpr int kDedispChanChunk = 16;                      // channels staged per pass
constexpr int kDedispMaxSpan = 1024;                      // max delay spread in a DM tile
// Channel-major workspace row pitch: room for a full time tile and the
// 16-byte staging overrun past n_in, rounded to 64 bytes.
__host__ __device__ inline int64_t dedisp_pitch(int64_t n_in) {
    return ((n_in + kDedispTimeTile + 64 + 63) / 64) * 64;
}
// Staged bytes of one channel for a tile whose delay spread is `span`:
// four byte-shifted copies of a window that covers the time tile, the spread
// and the 16-byte alignment slack.
__host__ __device__ inline int32_t dedisp_row_bytes(int32_t span) {
    return ((15 + span + kDedispTimeTile + 15) / 16) * 16;
}

}  // namespace sp

struct sp_plan {
    int device = 0;
    int32_t nchan = 0, ndm = 0, max_delay = 0;
    double tsamp = 0.0;
    std::vector<int32_t> delays;  // host copy [ndm][nchan]
    // DM tiles: consecutive runs of at most kDedispDmTile trial DMs whose
    // per-channel delay spread stays within kDedispMaxSpan.
    int32_t ntiles = 0;
    std::vector<int32_t> tile_first, tile_count;
    int32_t smem_bytes = 0;       // dynamic shared memory of the dedispersion kernel
    // device copies
    int32_t *d_delays = nullptr;      // [ndm][nchan]
    int32_t *d_tile_first = nullptr;  // [ntiles]
    int32_t *d_tile_count = nullptr;  // [ntiles]
    int32_t *d_tile_dlo = nullptr;    // [ntiles][nchan] min delay over the tile
    int32_t *d_tile_span = nullptr;   // [ntiles][nchan] max - min delay over the tile
};

namespace sp {

// Host-side delay evaluation of Eq. 1 (plan.cpp, compiled -ffp-contract=off).
int compute_delays(const double *freqs, int32_t nchan, double tsamp, const double *dms,
                   int32_t ndm, std::vector<int32_t> &out, int32_t *max_delay);

// Kernel launchers (return SP_OK or SP_ECUDA).
int launch_transpose(const uint8_t *d_in, int64_t n_in, int32_t nchan, uint8_t *d_xt,
                     int64_t pitch, cudaStream_t stream);
int launch_dedisperse(const sp_plan *plan, const uint8_t *d_xt, int64_t pitch, int64_t n_out,
                      int32_t *d_out, cudaStream_t stream);

struct SpsArgs {
    const int32_t *dmt;
    int32_t ndm;
    int64_t n_out;
    int32_t widths[SP_MAX_WIDTHS];
    int32_t nw;
    float threshold;
    int64_t norm_block;
    int64_t nblk;
    void *work;
    sp_cand *cands;
    int64_t cap;
    int64_t *count;
    float *map_best;
    int8_t *map_wbest;
};
int64_t sps_nblocks(int64_t n_out, int64_t norm_block);
int64_t sps_workspace_bytes(int32_t ndm, int64_t n_out, int32_t nw, int64_t norm_block);
int launch_sps(const SpsArgs &a, cudaStream_t stream);

inline int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }

}  // namespace sp
