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
constexpr int kDedispChanChunk = 8;                       // channels staged per pass
constexpr int kDedispMaxSpan = 1024;                      // max delay spread in a DM tile
constexpr int kDedispTileGroup = 24;                      // DM tiles per raster group
// Shared-memory header of the dedispersion kernel: one mbarrier per raw
// staging slot, then per slot the geometry and the (channel, DM) offset table
// of the chunk it holds.
constexpr int kDedispGeoOffset = 64;
constexpr int kDedispOffTabOffset = 512;
constexpr int kDedispOffTabInts = kDedispChanChunk * kDedispDmTile;
constexpr int kDedispRawSlots = 3;                        // raw chunks in flight (two ahead)
constexpr int kDedispHeaderBytes = kDedispOffTabOffset + kDedispRawSlots * kDedispOffTabInts * 4;
// Staged-input row pitch: room for the last time tile's window past n_in,
// rounded to 64 bytes.
__host__ __device__ inline int64_t dedisp_pitch(int64_t n_in) {
    return ((n_in + kDedispTimeTile + 64 + 63) / 64) * 64;
}
// Bytes of one shifted copy of one channel for a tile whose delay spread is
// `span`: a window that covers the time tile, the spread and the 16-byte
// alignment slack of its start.
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
    int32_t nchunks = 0;          // channel chunks of kDedispChanChunk
    std::vector<int32_t> tile_first, tile_count;
    int32_t copies_max = 0;       // largest shifted-copy staging of one chunk (bytes)
    int32_t raw_max = 0;          // largest raw staging of one chunk (bytes)
    int32_t smem_bytes = 0;       // dynamic shared memory of the dedispersion kernel
    // device copies
    int32_t *d_delays = nullptr;      // [ndm][nchan]
    int32_t *d_tile_first = nullptr;  // [ntiles]
    int32_t *d_tile_count = nullptr;  // [ntiles]
    // Per (tile, chunk, channel): {window start relative to the time tile,
    // bytes R read from one copy, offset of the channel's copies, 0}.
    int4 *d_chunk_geo = nullptr;      // [ntiles][nchunks][kDedispChanChunk]
    // Per (tile, chunk, channel, DM): byte offset of the DM's first sample in
    // the chunk's copies (copy (shift & 3), word shift >> 2).
    int32_t *d_chunk_off = nullptr;   // [ntiles][nchunks][kDedispChanChunk][kDedispDmTile]
    int32_t *d_status = nullptr;      // device status word (bit 0: a staging wait timed out)
};

namespace sp {

// Host-side delay evaluation of Eq. 1 (plan.cpp, compiled -ffp-contract=off).
int compute_delays(const double *freqs, int32_t nchan, double tsamp, const double *dms,
                   int32_t ndm, std::vector<int32_t> &out, int32_t *max_delay);

// Kernel launchers (return SP_OK or SP_ECUDA).
int launch_stage_input(const uint8_t *d_in, int64_t n_in, int32_t nchan, uint8_t *d_staged,
                       int64_t pitch, cudaStream_t stream);
int launch_dedisperse(const sp_plan *plan, const uint8_t *d_xt, int64_t pitch, int64_t n_out,
                      int32_t *d_out, cudaStream_t stream);
// Host-side layout of the per-(tile, chunk) staging tables (plan.cpp).
void build_chunk_tables(const sp_plan &p, std::vector<int32_t> &geo, std::vector<int32_t> &off,
                        int32_t *copies_max, int32_t *raw_max);

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
