// sp_internal.h -- shared declarations of libspotlight's translation units.
// Not installed; the public interface is include/spotlight.h.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/spotlight.h"

namespace sp {

// Dedispersion tiling (see dedisperse.cu for the kernel these describe).
// A kernel shape is (channels per chunk CH, samples per thread SPT, trial
// DMs per thread NDT): CH warps of NDT DMs each, so a DM tile holds up to
// NDT*CH DMs, and a time tile holds 32*SPT output samples.  A shape with
// NDT = 8 also runs tiles of at most 4*CH DMs with 4 DMs per thread.  The
// shapes below are compiled; the autotuner picks one per plan.
constexpr int kDedispNumShapes = 4;
constexpr int kDedispShapeCh[kDedispNumShapes] = {8, 8, 8, 4};
constexpr int kDedispShapeSpt[kDedispNumShapes] = {16, 16, 8, 16};
constexpr int kDedispShapeNdt[kDedispNumShapes] = {8, 4, 4, 4};
// Largest per-channel delay spread of a DM tile: for the 8-DM shape the
// bound that keeps two CTAs' staging (8 windows of 512 + spread samples,
// raw and as four shifted copies, plus a 64-DM offset table) in one SM's
// shared memory.
constexpr int kDedispShapeMaxSpan[kDedispNumShapes] = {680, 1024, 1024, 1024};
constexpr int kDedispMaxChanChunk = 8;
constexpr int kDedispMaxTimeTile = 512;                   // largest time tile of any shape
constexpr int kDedispMaxSpan = 1024;                      // largest spread of any shape
constexpr int kDedispTileGroupDms = 768;                  // DMs per raster group (24 tiles of 32)
// 8-DM tiles keep 16-bit partial sums: at most 257 channels of bytes fit
// a 16-bit lane, so the partials are added to the output every 256 channels.
constexpr int kDedispPackedChannels = 256;
// Shared-memory header of the dedispersion kernel: one mbarrier per raw
// staging slot, then per slot the geometry and the (channel, DM) offset table
// of the chunk it holds.
constexpr int kDedispItemOffset = 32;                     // persistent CTA's current work item
constexpr int kDedispGeoOffset = 64;
constexpr int kDedispOffTabOffset = 512;
constexpr int kDedispRawSlots = 3;                        // raw chunks in flight (two ahead)
__host__ __device__ constexpr int dedisp_header_bytes(int ch, int dm_tile) {
    return kDedispOffTabOffset + kDedispRawSlots * ch * dm_tile * 4;
}
// Staged-input row pitch: room for the last time tile's window past n_in,
// rounded to 64 bytes.
__host__ __device__ inline int64_t dedisp_pitch(int64_t n_in) {
    return ((n_in + kDedispMaxTimeTile + 64 + 63) / 64) * 64;
}
// Bytes of one shifted copy of one channel for a tile whose delay spread is
// `span`: a window that covers the time tile, the spread and the 16-byte
// alignment slack of its start.
__host__ __device__ inline int32_t dedisp_row_bytes(int32_t span, int32_t time_tile) {
    return ((15 + span + time_tile + 15) / 16) * 16;
}

}  // namespace sp

struct sp_plan {
    int device = 0;
    int32_t nchan = 0, ndm = 0, max_delay = 0;
    double tsamp = 0.0;
    std::vector<double> freqs;    // host copy of the channel axis [nchan] (MHz)
    std::vector<double> dms;      // host copy of the trial DMs [ndm]
    std::vector<int32_t> delays;  // host copy [ndm][nchan]
    // Kernel shape (index into kDedispShapeCh/Spt/Ndt) and its tile sizes.
    int32_t shape = 0;
    int32_t dm_tile = 0, time_tile = 0, chan_chunk = 0;
    // DM tiles: consecutive runs of at most dm_tile trial DMs whose
    // per-channel delay spread stays within the shape's maximum span.
    int32_t ntiles = 0;
    int32_t nchunks = 0;          // channel chunks of chan_chunk
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
    int4 *d_chunk_geo = nullptr;      // [ntiles][nchunks][chan_chunk]
    // Per (tile, chunk, channel, DM): byte offset of the DM's first sample in
    // the chunk's copies (copy (shift & 3), word shift >> 2).
    int32_t *d_chunk_off = nullptr;   // [ntiles][nchunks][chan_chunk][dm_tile]
    int32_t *d_status = nullptr;      // device status word (bit 0: a staging wait timed out)
};

namespace sp {

// Host-side delay evaluation of Eq. 1 (plan.cpp, compiled -ffp-contract=off).
int compute_delays(const double *freqs, int32_t nchan, double tsamp, const double *dms,
                   int32_t ndm, std::vector<int32_t> &out, int32_t *max_delay);

// Kernel launchers (return SP_OK or SP_ECUDA).
// Sample t comes from input row (row0 + t) mod ring_rows (ring_rows 0 = a
// plain input of n_in rows).
int launch_stage_input(const uint8_t *d_in, int64_t n_in, int32_t nchan, uint8_t *d_staged,
                       int64_t pitch, cudaStream_t stream, int64_t row0 = 0, int64_t ring_rows = 0);
// status: the device word a timed-out wait flags (nullptr: the plan's own).
int launch_dedisperse(const sp_plan *plan, const uint8_t *d_xt, int64_t pitch, int64_t n_out,
                      int32_t *d_out, cudaStream_t stream, int32_t *status = nullptr);
// One beam of a batched dedispersion launch, as the kernel reads it.
struct BatchBeamDev {
    const uint8_t *xt;             // staged beam
    int64_t pitch;
    int64_t n_out;
    int32_t *out;                  // [ndm][n_out]
    const int32_t *tile_first;
    const int32_t *tile_count;
    const int4 *geo;
    const int32_t *off;
    int32_t nchan, nchunks, ntiles, ntime;
};
// Host view of a batch launch: every beam's plan must have the same shape.
struct BatchLaunch {
    int32_t shape;
    int32_t nbeams;
    int64_t nitems;                // sum over beams of ntiles * ntime
    int32_t copies_max, raw_max, smem_bytes;
    const BatchBeamDev *d_beams;   // [nbeams]
    const int64_t *d_item_begin;   // [nbeams + 1]
    unsigned long long *d_counter; // work-queue head, zeroed by the launcher
    int32_t *d_status;
    int32_t grid;                  // persistent CTAs (batch_grid)
};
// Configures the shape's kernels and sets b.grid to the number of CTAs that
// fit on the current device at once (no CUDA call is left for the launch).
int batch_grid(BatchLaunch &b);
// persistent: a resident grid draining the work queue; else one CTA per item.
int launch_dedisperse_batch(const BatchLaunch &b, cudaStream_t stream, bool persistent = true);
int64_t dedisp_time_tiles(const sp_plan *plan, int64_t n_out);
// Test hook of the dedispersion kernel's bounded waits on the current device.
int set_staging_fault(uint32_t extra_bytes, long long wait_limit);
// Sets the dynamic shared-memory limit of the plan's kernels on the current
// device (once per device and size); called before any launch or capture.
int dedisp_configure(const sp_plan *plan);
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
// Windowed peak filter of radius 1..kMaxPeakRadius (radius 1 = launch_sps).
constexpr int kMaxPeakRadius = 5;
int64_t sps_window_workspace_bytes(int32_t ndm, int64_t n_out, int32_t nw, int64_t norm_block, int32_t radius);
int launch_sps_window(SpsArgs a, int32_t radius, cudaStream_t stream);
// Sets the boxcar kernels' shared-memory limit for widths up to maxw on the
// current device (launch_sps does it on first use otherwise).
int sps_configure(int32_t maxw);

inline int64_t align256(int64_t x) { return (x + 255) & ~int64_t(255); }

// Argument checks shared by the entry points (capi.cpp).
bool on_plan_device(const sp_plan *p);
int check_widths(const int32_t *w, int32_t nw);

// Kernel launches issued by the library (sp_launch_count); every launcher
// adds its launches, a CUDA-graph replay adds the kernels of the graph.
// Between capture_begin and capture_end the calling thread's launches are
// recorded into a graph: they are counted for the graph (capture_end
// returns how many) instead of as launches.
void note_launch(uint64_t n = 1);
void capture_begin();
uint64_t capture_end();

// Facts about a classifier that the streaming search needs (cnn.cpp).
int32_t cnn_max_batch(const sp_cnn *c);
int cnn_device(const sp_cnn *c);

}  // namespace sp
