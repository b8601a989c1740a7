/*
 * spotlight.h -- C ABI of libspotlight, the GB300 (sm_103a) search hot path
 * of the SPOTLIGHT real-time transient pipeline (arXiv 2606.27262, Sec. 3.1):
 * brute-force incoherent dedispersion of an 8-bit filterbank beam over a list
 * of trial DMs, then a multi-width boxcar single-pulse search with per-block
 * mean/sigma normalisation, a threshold and a 3x3 peak filter that emit a
 * candidate list.
 *
 * Conventions shared by every call
 *   - All functions return SP_OK (0) or a negative SP_E* code; sp_strerror()
 *     names it.  Arguments are checked on the host before anything is
 *     launched; a failed check launches nothing and writes nothing.
 *   - "d_" pointers are device pointers (memory of the current CUDA device),
 *     "h_" pointers are host pointers.  The caller owns every buffer it
 *     passes; the library keeps no pointer to them after the call returns.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *     work is enqueued on it and the call returns without waiting, except
 *     where a call says it synchronises.  Buffers must stay valid until the
 *     stream has executed the work.
 *   - Only the create calls and the autotuner allocate device memory; the
 *     other calls allocate nothing.  Calls on different streams may overlap
 *     as long as they do not share output or workspace buffers.
 *   - Filterbank layout: uint8 [n_in][nchan], time-major (the order a
 *     filterbank file or ring block stores samples), channel 0 = the highest
 *     frequency (the band is flipped highest-first, Sec. 2).
 *   - DM-transform layout: int32 [ndm][n_out], row d = trial DM d.
 */
#ifndef SPOTLIGHT_H
#define SPOTLIGHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SP_OK 0
#define SP_EINVAL (-1)     /* invalid argument (null pointer, bad value)      */
#define SP_ESHAPE (-2)     /* sizes inconsistent (n_in < n_out + max delay)   */
#define SP_ECUDA (-3)      /* a CUDA runtime call failed                      */
#define SP_EOVERFLOW (-4)  /* more candidates than the caller's capacity      */
#define SP_ENOMEM (-5)     /* device or host allocation failed                */
#define SP_EWORKSPACE (-6) /* workspace pointer null or too small             */
#define SP_ELIMIT (-7)     /* a size is beyond a documented library limit     */
#define SP_ETIMEOUT (-8)   /* a kernel gave up a bounded wait: outputs void   */

/* Library limits. */
#define SP_MAX_WIDTHS 16        /* trial boxcar widths per search           */
#define SP_MAX_WIDTH 1024       /* largest trial boxcar width, samples      */

typedef struct sp_plan sp_plan;
typedef struct sp_searcher sp_searcher;

/* One single-pulse candidate (Sec. 3.1.2): trial-DM row, first sample of the
 * boxcar window [t, t + w), index of the best width in the caller's width
 * list, and that width's S/N. */
typedef struct {
    int32_t dm_idx;
    int32_t t;
    int32_t width_idx;
    float snr;
} sp_cand;

const char *sp_strerror(int code);

/* Kernel launches the library has issued in this process, for measurement
 * (no counterpart in the paper): every kernel a call launches counts once;
 * kernels that sp_batch_capture records count once per sp_batch_launch, not
 * at capture.  (A graph the caller captures around library calls counts its
 * kernels once, when they are recorded.)  Never fails. */
uint64_t sp_launch_count(void);

/* ------------------------------------------------------------------ plan --
 * Dedispersion plan (Sec. 3.1.1).  For trial DM d and channel c the delay is
 *   delay[d][c] = floor(x + 0.5),
 *   x = 4.148808e3 * dms[d] * (1/freqs[c]^2 - 1/freqs[0]^2) / tsamp_s
 * evaluated in IEEE binary64 from left to right (Eq. 1 with the highest
 * frequency as reference; 4.148808e3 MHz^2 pc^-1 cm^3 s is Eq. 1's
 * dispersion constant rounded).  The plan computes the table on the host,
 * uploads it once and derives the DM-tile layout the kernels use.
 *   freqs_mhz [nchan]  host, copied; > 0 and strictly decreasing.
 *   dms [ndm]          host, copied; >= 0 (any order).
 *   tsamp_s            sampling time, > 0.
 *   out                receives a library-owned plan; free with sp_plan_destroy.
 * Errors: SP_EINVAL for invalid values, SP_ELIMIT if a delay or a size does
 * not fit int32, SP_ENOMEM / SP_ECUDA if the device upload fails.  Uses the
 * current CUDA device; the plan must be used on that device only. */
int sp_plan_create(const double *freqs_mhz, int32_t nchan, double tsamp_s,
                   const double *dms, int32_t ndm, sp_plan **out);
int sp_plan_destroy(sp_plan *plan);
/* max_delay = the largest delay[d][c] (D_max, samples); any out pointer may
 * be NULL. */
int sp_plan_info(const sp_plan *plan, int32_t *max_delay, int32_t *nchan, int32_t *ndm);
/* Device status word of the plan's kernels: 0, or SP_STATUS_* bits set by
 * a kernel that gave up a bounded wait.  A set bit voids every output of
 * every launch that flagged it since the last clear -- the whole DM
 * transform, and for a batched launch every beam of the batch, not only the
 * tile whose wait ran out: a CTA that gives up twice may leave copies in
 * flight that land in shared memory a later CTA of the same launch uses.
 * Reads it after synchronising the device; clear != 0 resets it. */
#define SP_STATUS_STAGING_TIMEOUT 1
int sp_plan_status(const sp_plan *plan, int32_t *h_status, int32_t clear);
/* Test hook of the failure path above (the paper has no counterpart): on
 * the current device, every later dedispersion CTA's first chunk expects
 * extra_bytes (a multiple of 16, <= 1 MiB) more than its bulk copies bring,
 * and every staging wait gives up after wait_limit_cycles SM cycles (>=
 * 1024).  With extra_bytes > 0 the first wait of every CTA runs out, the CTA
 * waits once more (bounded) and leaves, and the status word gets
 * SP_STATUS_STAGING_TIMEOUT; no access leaves its buffers and the device
 * stays usable.  sp_debug_staging_fault(0, 1LL << 31) restores the
 * defaults.  Not for use while dedispersion kernels are in flight. */
int sp_debug_staging_fault(int32_t extra_bytes, int64_t wait_limit_cycles);
/* Copies the delay table, int32 [ndm][nchan], to host memory. */
int sp_plan_delays(const sp_plan *plan, int32_t *h_out);
/* The same delay table computed on the host only (no device, no plan):
 * h_out [ndm][nchan] int32 and *max_delay (may be NULL).  Lets a caller size
 * n_in = n_out + max_delay before touching a GPU.  Same errors as
 * sp_plan_create's argument checks. */
int sp_compute_delays(const double *freqs_mhz, int32_t nchan, double tsamp_s,
                      const double *dms, int32_t ndm, int32_t *h_out, int32_t *max_delay);

/* ------------------------------------------- kernel shapes, autotuner --
 * The dedispersion kernel is compiled for SP_DEDISP_NUM_SHAPES tile shapes,
 * each a (DM tile, time tile, channel chunk) triple: shape 0 = 32 trial DMs
 * x 512 samples x 8 channels (the shape of sp_plan_create), 1 = 32 x 256 x 8,
 * 2 = 16 x 512 x 4.  A plan is built for one shape (its DM tiles and staging
 * tables depend on it).  The shape changes speed only: every shape computes
 * the same DM transform, bit for bit.  Choosing it by measurement has no
 * counterpart in the paper (whose kernels come from its dedispersion
 * library); it exists because the best tile shape depends on the channel
 * count, the DM list and the GPU.
 * sp_dedisp_shape_info: the triple of a shape (out pointers may be NULL).
 * sp_plan_create_shaped: sp_plan_create for a given shape, or for
 *   SP_SHAPE_AUTO: the shape sp_autotune_dedisperse picks with
 *   SP_AUTOTUNE_SAMPLES searched samples and SP_AUTOTUNE_REPS repetitions.
 * sp_plan_shape: the plan's shape, DM-tile count and the dedispersion
 *   kernel's dynamic shared memory in bytes (out pointers may be NULL).
 * sp_autotune_dedisperse: for each shape, builds a plan for (freqs, dms),
 *   stages a synthetic input of n_out_sample searched samples
 *   (n_in = n_out_sample + max_delay) and times `reps` launches of the
 *   dedispersion kernel after one warm-up launch, with CUDA events on
 *   `stream`; h_ms [SP_DEDISP_NUM_SHAPES] receives the mean milliseconds per
 *   launch (+inf for a shape that cannot run this plan) and *best the
 *   fastest shape.  Synchronous; allocates and frees temporary device
 *   memory (n_in * nchan + ndm * n_out_sample * 4 bytes).  The result is
 *   cached for the process per (device, inputs): a repeated call returns the
 *   cached timings without launching anything.
 * Errors: SP_EINVAL (bad shape or arguments, n_out_sample < 1, reps < 1),
 *   the plan-creation errors, SP_ENOMEM, SP_ECUDA. */
#define SP_DEDISP_NUM_SHAPES 4
#define SP_SHAPE_AUTO (-1)
#define SP_AUTOTUNE_SAMPLES 16384
#define SP_AUTOTUNE_REPS 3
int sp_dedisp_shape_info(int32_t shape, int32_t *dm_tile, int32_t *time_tile, int32_t *chan_chunk);
int sp_plan_create_shaped(const double *freqs_mhz, int32_t nchan, double tsamp_s,
                          const double *dms, int32_t ndm, int32_t shape, sp_plan **out);
int sp_plan_shape(const sp_plan *plan, int32_t *shape, int32_t *ntiles, int32_t *smem_bytes);
/* Host-only check of a plan's staging tables (no counterpart in the paper;
 * no device is touched): builds the plan of (freqs, tsamp, dms, shape) on
 * the host and checks, for a beam of n_out searched samples, every access
 * the dedispersion kernel makes with its tables -- 16-byte alignment and
 * bounds of the bulk copies (inside the staged row of pitch
 * sp_staged_pitch(n_out + max_delay) and inside the raw slot), the four
 * shifted copies inside the copies buffer, and every shared load of the
 * sums inside its channel's copy.  h_report [8] (host): DM tiles, channel
 * chunks, copies bytes, raw bytes, dynamic shared memory bytes of the
 * kernel, number of violated conditions (0 for a sound plan), max delay,
 * staged pitch.  Errors: SP_EINVAL (the sp_plan_create argument checks,
 * shape, n_out < 1, h_report NULL). */
int sp_plan_check_tables(const double *freqs_mhz, int32_t nchan, double tsamp_s, const double *dms,
                         int32_t ndm, int32_t shape, int64_t n_out, int64_t *h_report);
int sp_autotune_dedisperse(const double *freqs_mhz, int32_t nchan, double tsamp_s,
                           const double *dms, int32_t ndm, int64_t n_out_sample, int32_t reps,
                           float *h_ms, int32_t *best, void *stream);

/* ----------------------------------------------------------- dedisperse --
 * Brute-force incoherent dedispersion (Sec. 3.1.1, the DM transform):
 *   d_out[d][t] = sum_{c < nchan} d_in[t + delay[d][c]][c],  0 <= t < n_out,
 * exact in int32 (every sum is at most 255 * nchan).  The input must hold
 * the overlap of the maximum sweep (Sec. 3.1 overlap-read):
 * n_out = n_in - max_delay is required, else SP_ESHAPE.
 *   d_in  [n_in][nchan] uint8, device, 16-byte aligned.
 *   d_out [ndm][n_out]  int32, device.
 *   d_work / work_bytes: device scratch of at least
 *         sp_dedisperse_workspace_bytes(plan, n_in) bytes, 256-byte aligned
 *         (holds the staged input, see sp_stage_input); contents on entry
 *         are ignored, on return they hold the staged input.
 * Errors: SP_EINVAL, SP_ESHAPE, SP_EWORKSPACE, SP_ELIMIT, SP_ECUDA (launch). */
int64_t sp_dedisperse_workspace_bytes(const sp_plan *plan, int64_t n_in);
int sp_dedisperse(const sp_plan *plan, const uint8_t *d_in, int64_t n_in,
                  int32_t *d_out, int64_t n_out, void *d_work, int64_t work_bytes,
                  void *stream);

/* The two steps of sp_dedisperse, for callers that stage an input once and
 * search it several times, or keep it staged in a ring buffer.
 * The staged form is the input rearranged for the dedispersion kernel; its
 * layout belongs to the library (currently channel-major uint8
 * [nchan][pitch], zero at and past n_in) and is produced by sp_stage_input.
 * It takes sp_staged_bytes(nchan, n_in) bytes, 256-byte aligned, with row
 * pitch sp_staged_pitch(n_in).
 * sp_stage_input: d_in [n_in][nchan] (time-major, 16-byte aligned) ->
 *   d_staged.  sp_dedisperse_staged: the DM transform of d_staged, same
 *   definition, shape rule and errors as sp_dedisperse. */
int64_t sp_staged_pitch(int64_t n_in);
int64_t sp_staged_bytes(int32_t nchan, int64_t n_in);
int sp_stage_input(const uint8_t *d_in, int64_t n_in, int32_t nchan, uint8_t *d_staged,
                   int64_t pitch, void *stream);
int sp_dedisperse_staged(const sp_plan *plan, const uint8_t *d_staged, int64_t pitch, int64_t n_in,
                         int32_t *d_out, int64_t n_out, void *stream);

/* Many beams in one launch (the multi-beam operation of Sec. 2 and 3.1:
 * every beam is searched independently; beams may differ in length, DM list
 * and channel count).  One persistent kernel takes (beam, DM tile, time
 * tile) items from a work queue until all beams are done; each beam's result
 * is exactly that of sp_dedisperse_staged.
 *   h_beams [nbeams]  host array, read during the call:
 *     plan      the beam's plan; every plan must have the same shape and
 *               belong to the current device;
 *     d_staged  the staged beam (sp_stage_input), 256-byte aligned;
 *     pitch     its row pitch, >= sp_staged_pitch(n_in), a multiple of 64;
 *     n_in      input samples;
 *     d_out     [plan ndm][n_out] int32 device, disjoint from the others;
 *     n_out     must equal n_in - the plan's max delay (else SP_ESHAPE).
 *   d_work / work_bytes  device scratch of at least
 *     sp_dedisperse_batch_workspace_bytes(nbeams) bytes, 256-byte aligned
 *     (the work queue and the beam table, copied there from host memory on
 *     `stream`, so this call cannot be captured into a CUDA graph; the batch
 *     object below can).
 * A staging wait that runs out sets SP_STATUS_STAGING_TIMEOUT in the status
 * word of h_beams[0].plan; it voids the outputs of every beam of the call.
 * Errors: SP_EINVAL, SP_ESHAPE, SP_EWORKSPACE, SP_ELIMIT, SP_ECUDA. */
typedef struct {
    const sp_plan *plan;
    const uint8_t *d_staged;
    int64_t pitch;
    int64_t n_in;
    int32_t *d_out;
    int64_t n_out;
} sp_batch_beam;
int64_t sp_dedisperse_batch_workspace_bytes(int32_t nbeams);
int sp_dedisperse_batch(const sp_batch_beam *h_beams, int32_t nbeams, void *d_work,
                        int64_t work_bytes, void *stream);

/* ------------------------------------------------- single-pulse search --
 * Boxcar matched-filter search of a DM transform (Sec. 3.1.2).
 * Normalisation: each row is cut into nblk = max(1, n_out / norm_block)
 * blocks [b*L, (b+1)*L) (the last also takes the remainder; norm_block <= 0
 * or >= n_out means one block).  With n, Sx, Sxx the count, sum and sum of
 * squares of block b (population variance), the S/N of the window [t, t+w)
 * whose first sample t lies in block b is
 *   snr_w(d, t) = (n*S - w*Sx) / (sqrt(w) * sqrt(n*Sxx - Sx^2)),
 *   S = sum_{k<w} dmt[d][t+k]        (windows never cross n_out),
 * and 0 for a zero-variance block.  best(d,t) is the maximum over the
 * widths (smallest width index on ties); -inf where no width fits.
 * A candidate is (d,t) with best(d,t) >= threshold that is a 3x3 local
 * maximum of best in the DM-time plane: strictly greater than each in-range
 * neighbour that precedes it in (d,t) order and >= each one after it.
 *   d_dmt [ndm][n_out] int32 device.
 *   h_widths [nw]      host, strictly increasing, 1..SP_MAX_WIDTH,
 *                      nw <= SP_MAX_WIDTHS.
 *   d_work/work_bytes  device scratch of sp_sps_workspace_bytes(...) bytes,
 *                      256-byte aligned (per-row block statistics,
 *                      pre-filter constants and tile lists).
 *   d_cands [cap]      device; receives min(count, cap) candidates in an
 *                      unspecified order (sort by (dm_idx, t) for a
 *                      canonical list).
 *   d_count            device int64; receives the total number found, which
 *                      exceeds cap on overflow (then only cap are written).
 * S/N is evaluated in float32 from an exact integer numerator; it agrees
 * with an exact evaluation to about 1e-6 relative.
 * Errors: SP_EINVAL, SP_ELIMIT, SP_EWORKSPACE, SP_ECUDA. */
int64_t sp_sps_workspace_bytes(int32_t ndm, int64_t n_out, int32_t nw, int64_t norm_block);
int sp_single_pulse_search(const int32_t *d_dmt, int32_t ndm, int64_t n_out,
                           const int32_t *h_widths, int32_t nw, float threshold,
                           int64_t norm_block, void *d_work, int64_t work_bytes,
                           sp_cand *d_cands, int64_t cap, int64_t *d_count,
                           void *stream);
/* sp_single_pulse_search with a (2 peak_radius + 1)^2 peak-filter window
 * instead of 3 x 3 (Sec. 3.1.2: a window slides over the DM-time plane and
 * keeps only its highest S/N; the paper uses 3 x 3 and 11 x 11 stencils,
 * peak_radius 1 and 5).  A point at or above the threshold is kept when its
 * best S/N is above every in-range neighbour of the window that precedes it
 * in (dm_idx, t) order and not below any that follows.  peak_radius in
 * 1..5; 1 is exactly sp_single_pulse_search.  For peak_radius > 1 the best-S/N
 * map is written into the workspace first (ndm * n_out * 5 more bytes), so
 * the workspace must hold sp_sps_window_workspace_bytes(...) bytes.
 * Same arguments, outputs and errors otherwise (SP_EINVAL for a radius out of
 * range). */
int64_t sp_sps_window_workspace_bytes(int32_t ndm, int64_t n_out, int32_t nw, int64_t norm_block,
                                      int32_t peak_radius);
int sp_single_pulse_search_window(const int32_t *d_dmt, int32_t ndm, int64_t n_out,
                                  const int32_t *h_widths, int32_t nw, float threshold,
                                  int64_t norm_block, int32_t peak_radius, void *d_work,
                                  int64_t work_bytes, sp_cand *d_cands, int64_t cap,
                                  int64_t *d_count, void *stream);
/* Allocation-free variant of sp_single_pulse_search.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * when they search -- a real-time loop that claimed its whole memory budget
 * at start-up and must not block or fail on an allocation mid-stream, a host
 * whose device memory belongs entirely to its own pool allocator, a plug-in
 * that is not permitted to call cudaMalloc.  Same arguments, arithmetic,
 * outputs and errors as sp_single_pulse_search, minus the workspace: the
 * block statistics live in a library-owned device array of
 * SP_NOALLOC_SCRATCH_BYTES (16 MiB), present on every GPU that loads the
 * library until the process exits.  Requests whose statistics need more
 * (sp_sps_workspace_bytes(ndm, n_out, nw, norm_block) > 16 MiB; config 2,
 * 5751 DMs x 131072 samples / 8192-sample blocks x 9 widths, needs 15.9 MB)
 * return SP_ELIMIT.  The call allocates nothing: no cudaMalloc, no cudaFree.
 * The first call on a device looks up the array's device address with that
 * device current (make that first call before any stream capture) and keeps
 * it for the life of the process; it does not survive cudaDeviceReset, so do
 * not call this entry point on a device after resetting it.  Every
 * call on a device shares the one array and it keeps the last call's
 * contents (each call overwrites what it reads); calls whose GPU work
 * overlaps -- on different streams or different host threads -- race on it
 * and must be serialised by the caller. */
#define SP_NOALLOC_SCRATCH_BYTES (16 << 20)
int sp_single_pulse_search_noalloc(const int32_t *d_dmt, int32_t ndm, int64_t n_out,
                                   const int32_t *h_widths, int32_t nw, float threshold,
                                   int64_t norm_block, sp_cand *d_cands, int64_t cap,
                                   int64_t *d_count, void *stream);
/* The map the candidates are picked from: d_best [ndm][n_out] float (best
 * S/N, -inf where no width fits) and d_wbest [ndm][n_out] int8 (index of the
 * best width, -1 where none fits).  Same arguments and arithmetic as
 * sp_single_pulse_search. */
int sp_best_snr_map(const int32_t *d_dmt, int32_t ndm, int64_t n_out,
                    const int32_t *h_widths, int32_t nw, int64_t norm_block,
                    void *d_work, int64_t work_bytes, float *d_best, int8_t *d_wbest,
                    void *stream);

/* -------------------------------------------------------------- searcher --
 * The whole per-beam path -- dedispersion, normalisation, boxcars, 3x3
 * peaks -- with every device buffer it needs allocated once up front, for a
 * fixed plan, searched length n_out (n_in = n_out + max_delay), width list,
 * threshold, normalisation block and candidate capacity.  The run calls
 * allocate nothing.
 * Errors from create: SP_EINVAL, SP_ELIMIT, SP_ENOMEM, SP_ECUDA. */
int sp_searcher_create(const sp_plan *plan, int64_t n_out, const int32_t *h_widths,
                       int32_t nw, float threshold, int64_t norm_block, int64_t cand_cap,
                       sp_searcher **out);
int sp_searcher_destroy(sp_searcher *s);
/* Device-resident run: d_in [n_in][nchan] uint8 device (16-byte aligned),
 * d_cands [cap] / d_count as in sp_single_pulse_search.  Asynchronous. */
int sp_searcher_run(sp_searcher *s, const uint8_t *d_in, sp_cand *d_cands, int64_t cap,
                    int64_t *d_count, void *stream);
/* End-to-end run from host memory: copies h_in [n_in][nchan] to the device
 * (page-locked memory makes this copy asynchronous and fast), searches,
 * copies min(count, cap) candidates to h_cands and the total to *h_count,
 * and synchronises the stream before returning.  Returns SP_EOVERFLOW
 * (after filling h_cands) when the total exceeds min(cap, cand_cap). */
int sp_searcher_run_host(sp_searcher *s, const uint8_t *h_in, sp_cand *h_cands, int64_t cap,
                         int64_t *h_count, void *stream);
/* Pipelined end-to-end runs from host memory, for a sequence of beams: the
 * copy of one beam's input overlaps the search of the beam before it
 * (Sec. 2: beams arrive continuously and each GPU searches them back to
 * back).  sp_searcher_submit_host queues one beam and returns at once: its
 * h_in [n_in][nchan] is copied on a copy stream of the searcher into one of
 * two device input buffers (after the beam that last used that buffer has
 * been staged), then dedispersed and searched on `stream`, and its count
 * copied to page-locked memory of the searcher.  h_in must be page-locked
 * for the copy to overlap, and must stay unchanged until that beam has been
 * collected.  At most two beams are uncollected at a time (SP_EINVAL for a
 * third).  sp_searcher_collect waits for the oldest uncollected beam and
 * copies its first min(count, cap, cand_cap) candidates to h_cands and its
 * total to *h_count; SP_EOVERFLOW (after copying) when the total exceeds
 * that, SP_EINVAL when nothing is queued.  The first submit allocates the
 * second input buffer, the second candidate buffer, two streams and four
 * events; later calls allocate nothing.  Results come back in submission
 * order, each equal to sp_searcher_run_host of the same input. */
int sp_searcher_submit_host(sp_searcher *s, const uint8_t *h_in, void *stream);
int sp_searcher_collect(sp_searcher *s, sp_cand *h_cands, int64_t cap, int64_t *h_count);

/* ----------------------------------------------------------------- batch --
 * A fixed set of beams searched as one step: the multi-beam workload of one
 * GPU (Sec. 2: each GPU searches many beams in real time).  Beam b has plan
 * plans[h_beam_plan[b]] and n_out = h_beam_n_out[b] searched samples
 * (n_in = n_out + that plan's max delay); all beams share the width list,
 * threshold, normalisation block and candidate capacity, and all plans must
 * have the same shape (sp_plan_shape) and belong to the current device.
 * The batch owns every device buffer of the step: each beam's input,
 * staged inputs, DM transforms, search workspace, candidates and counts.
 * DM transforms are not all held at once: beams are taken in order into
 * groups whose transforms fit in dmt_budget_bytes (a beam larger than the
 * budget forms a group alone), and two group arenas alternate.
 *
 * A run (mode SP_BATCH_GROUPED) does, per group: stage the group's beams,
 * dedisperse all of them in one persistent launch (sp_dedisperse_batch),
 * then search each beam (sp_single_pulse_search) on a second stream owned
 * by the batch (at the device's highest stream priority), so that group
 * g's search overlaps group g+1's dedispersion.  SP_BATCH_GROUPED_GRID is
 * the same with one CTA per work item instead of a persistent grid, so that
 * the block scheduler can run search CTAs between retiring dedispersion
 * CTAs.  Mode SP_BATCH_PER_BEAM does the same work beam by beam on `stream`
 * with one launch per step (stage, sp_dedisperse_staged, search): the
 * comparison the batch exists to beat.  Every mode gives every beam the
 * result its own sp_searcher would give.
 *
 * sp_batch_input: device pointer and n_in of beam b's input buffer (uint8
 *   [n_in][nchan], time-major, 256-byte aligned), which the caller fills
 *   before a run.
 * sp_batch_run: enqueues one run on `stream` (asynchronous).  Adding
 *   SP_BATCH_TIMED to a grouped mode also records CUDA events around each
 *   group's persistent dedispersion launch on `stream`; sp_batch_group_ms
 *   then waits for them and writes each group's launch time in ms to
 *   h_ms [ngroups] (SP_EINVAL if the last run or capture was not timed).
 * sp_batch_capture: records one run of `mode` on `stream` into a CUDA graph
 *   held by the batch (replacing any earlier one); nothing executes.
 *   sp_batch_launch enqueues that graph on `stream`.  Make the first run or
 *   capture before any other capture is active on the device.
 * sp_batch_results: after the run, waits for `stream` and copies beam b's
 *   total count to *h_count and min(count, cap, cand_cap) candidates
 *   (unspecified order) to h_cands; SP_EOVERFLOW (after copying) if the
 *   count exceeds min(cap, cand_cap).
 * sp_batch_dmt: beam b's DM transform [ndm][n_out] as left by the last run,
 *   if the arenas still hold it (beams of the last two groups of a grouped
 *   run, the last beam of a per-beam run); else SP_EINVAL.
 * sp_batch_run_host: end to end from host memory: copies h_in[b] (n_in *
 *   nchan bytes each; page-locked memory makes the copies asynchronous) into
 *   the beams' inputs group by group on a copy stream of the batch (group
 *   g + 1's copies overlap group g's work; each group waits only for its
 *   own), runs SP_BATCH_GROUPED_GRID, then copies every beam's count
 *   to h_counts [nbeams] and its first min(count, cap_per_beam, cand_cap)
 *   candidates to h_cands + b * cap_per_beam.  Synchronises `stream`;
 *   SP_EOVERFLOW (after copying) if any beam overflowed.
 * sp_batch_status: OR of the status words of the batch and of its plans
 *   (SP_STATUS_*), after synchronising the device; clear != 0 resets them.
 * sp_batch_info: group count and total device bytes the batch holds.
 * Errors: SP_EINVAL, SP_ESHAPE, SP_ELIMIT, SP_ENOMEM, SP_ECUDA. */
typedef struct sp_batch sp_batch;
#define SP_BATCH_GROUPED 0
#define SP_BATCH_PER_BEAM 1
#define SP_BATCH_GROUPED_GRID 2
#define SP_BATCH_TIMED 16
int sp_batch_create(const sp_plan *const *plans, int32_t nplans, const int32_t *h_beam_plan,
                    const int64_t *h_beam_n_out, int32_t nbeams, const int32_t *h_widths,
                    int32_t nw, float threshold, int64_t norm_block, int64_t cand_cap,
                    int64_t dmt_budget_bytes, sp_batch **out);
int sp_batch_destroy(sp_batch *b);
int sp_batch_info(const sp_batch *b, int32_t *ngroups, int64_t *device_bytes);
int sp_batch_input(sp_batch *b, int32_t beam, uint8_t **d_in, int64_t *n_in);
int sp_batch_run(sp_batch *b, int32_t mode, void *stream);
int sp_batch_group_ms(const sp_batch *b, float *h_ms);
int sp_batch_capture(sp_batch *b, int32_t mode, void *stream);
int sp_batch_launch(sp_batch *b, void *stream);
int sp_batch_results(sp_batch *b, int32_t beam, sp_cand *h_cands, int64_t cap, int64_t *h_count,
                     void *stream);
int sp_batch_dmt(const sp_batch *b, int32_t beam, const int32_t **d_dmt);
int sp_batch_run_host(sp_batch *b, const uint8_t *const *h_in, sp_cand *h_cands,
                      int64_t cap_per_beam, int64_t *h_counts, void *stream);
int sp_batch_status(const sp_batch *b, int32_t *h_status, int32_t clear);

/* --------------------------------------------------------------- injector --
 * Signal injection into quantised data (Appendix B; used to add simulated
 * bursts to beams that are already quantised, for validation).  With
 * L = 2^bits states, state k covers noise values [lo_k, hi_k),
 * lo_k = mu + (k - L/2) * level * sigma, hi_k = lo_k + level * sigma, state
 * 0 extends to -inf and state L-1 to +inf.  A sample in state n receiving a
 * signal S >= 0 (in the units of mu and sigma) moves to the state k >= n
 * of highest probability
 *   P(n -> k) = max(0, phi(min(hi_k - S, hi_n)) - phi(max(lo_k - S, lo_n)))
 *               / (phi(hi_n) - phi(lo_n)),
 * phi the Gaussian CDF with mean mu and deviation sigma (Appendix B's
 * general formula with its boundary states); exact ties go to the lower
 * state.  Evaluated in double precision.
 *   d_data [n] uint8 device, one sample per byte (values < 2^bits), updated
 *           in place; samples with S <= 0, in the top state, or with a
 *           value >= 2^bits are left unchanged.
 *   d_signal [n] float32 device.
 *   bits 1..8; sigma > 0; level > 0 (Appendix B's l; 0.030765 for its 8-bit
 *   data; 1/16 for data quantised as round(128 + 16 z), with mu = 127.5 and
 *   sigma = 16).
 * Errors: SP_EINVAL, SP_ECUDA (launch). */
int sp_inject_quantised(uint8_t *d_data, const float *d_signal, int64_t n, int32_t bits, double mu,
                        double sigma, double level, void *stream);

/* ----------------------------------------------------------------- sifter --
 * Candidate sifting after the single-pulse search (Sec. 3.2.1), host code:
 * DBSCAN clustering of one beam's candidates in the DM-time plane, the
 * highest-S/N member of each cluster kept, then thresholds.  Coordinates
 * are the trial DM in pc cm^-3 (h_dms[dm_idx]) and the arrival time in
 * seconds (t * tsamp_s); two candidates are neighbours when their Euclidean
 * distance is at most eps; a core candidate has at least min_points
 * neighbours (itself included); clusters grow breadth first from the first
 * unclustered core candidate in (dm_idx, t) order, and a border candidate
 * near two clusters joins the one that reaches it first.  Candidates in no
 * cluster are dropped.  A cluster's peak (highest S/N, first in (dm_idx, t)
 * order on ties) is kept when snr >= snr_min, DM >= dm_min and width
 * (h_widths[width_idx] * tsamp_s) <= width_max_s.
 *   h_cands [n]        host candidates (any order).
 *   h_dms [ndm], h_widths [nw]  the search's trial DMs and widths (samples).
 *   h_out [cap]        receives the kept peaks in (dm_idx, t) order;
 *   *n_out             how many were kept (SP_EOVERFLOW if more than cap).
 *   h_labels [n]       optional (NULL): cluster id of each input candidate
 *                      (clusters numbered in discovery order), -1 for noise.
 * SP_SIFT_DEFAULTS are the values of Sec. 3.2.1: eps 0.5, 5 points,
 * S/N 10, DM 10 pc cm^-3, width 100 ms.  Synchronous; touches no GPU.
 * Errors: SP_EINVAL (bad arguments or a candidate index out of range). */
typedef struct {
    float eps;
    int32_t min_points;
    float snr_min;
    float dm_min;
    float width_max_s;
} sp_sift_params;
#define SP_SIFT_DEFAULTS {0.5f, 5, 10.0f, 10.0f, 0.1f}
int sp_sift(const sp_cand *h_cands, int64_t n, const double *h_dms, int32_t ndm,
            const int32_t *h_widths, int32_t nw, double tsamp_s, const sp_sift_params *params,
            sp_cand *h_out, int64_t cap, int64_t *n_out, int32_t *h_labels);

/* ------------------------------------------------------------ classifier --
 * Candidate classifier (Sec. 3.2.2: a convolutional network scores each
 * sifted candidate from two images -- its dynamic spectrum dedispersed at
 * the candidate DM and its DM transform over a narrow DM range -- with one
 * network per image fused multiplicatively into one probability; candidates
 * pass at p >= 0.5).  The paper's pretrained networks are not available;
 * this one is trained by the library's own kernels.
 *
 * Images: bf16 [batch][256][256] (rows = subbands or DM offsets, columns =
 * time bins), device, 16-byte aligned.  sp_cnn_features makes both from
 * subband dynamic spectra d_sub fp32 [batch][nsub = 256][t_in] that are
 * already dedispersed at the candidate DM within each subband: the
 * frequency-time image is the centre 256 bins, u0 = (t_in - 256) / 2, and
 * DM-time row j is sum_s d_sub[s][u0 + u + shift[j][s]] (out-of-range bins
 * count 0), shift from sp_dmt_shifts; each image is then scaled to zero
 * mean and unit variance.  d_work: sp_cnn_features_workspace_bytes(batch)
 * bytes, 256-byte aligned.
 * sp_dmt_shifts: h_shift [256][nsub] for a band freqs_mhz [nchan] (strictly
 *   decreasing, nchan a multiple of nsub): row j is a residual dispersion
 *   sweep of max_sweep * (2j/255 - 1) time bins across the band, i.e.
 *   shift[j][s] = round(sweep_j * (f_s^-2 - f_0^-2) / (f_last^-2 - f_0^-2))
 *   with f_s the mean frequency of subband s (Eq. 1 in time bins).
 *   t_in = 256 + 2 * max_sweep keeps every shifted bin inside d_sub.
 * Network (per image): five 3x3 convolutions, stride 2, padding 1, with
 *   1->16->32->64->128->256 channels and ReLU; global average pooling; a
 *   linear head to one logit l; p = sigmoid(l_ft) * sigmoid(l_dmt).  bf16
 *   activations and GEMM operands, fp32 accumulation (tensor cores), fp32
 *   master weights.  Training minimises the binary cross-entropy of p
 *   (mean over the batch) with Adam (beta 0.9 / 0.999, eps 1e-8).
 * sp_cnn_create: He-normal weights from `seed`, batch <= max_batch <=
 *   SP_CNN_MAX_BATCH; allocates all buffers.
 * sp_cnn_num_params: length of the flat fp32 parameter vector: per image
 *   (frequency-time first) and per layer W [Cout][9 Cin] (k = (ky*3 +
 *   kx)*Cin + c) then b [Cout], then the head w [256] and b [1].
 * sp_cnn_get_params / _set_params / _get_grads: that vector (host); grads
 *   are those of the last sp_cnn_backward (SP_EINVAL before one).
 * sp_cnn_forward: d_prob [batch] fp32 device.  sp_cnn_backward: forward with
 *   d_labels [batch] (1 = astrophysical, 0 = not), gradients, and the loss
 *   in *h_loss (synchronises; NULL = no copy).  sp_cnn_adam_step applies the
 *   stored gradients; sp_cnn_train_step = backward + adam step.
 * Errors: SP_EINVAL, SP_ENOMEM, SP_EWORKSPACE, SP_ECUDA. */
typedef struct sp_cnn sp_cnn;
#define SP_CNN_MAX_BATCH 256
int64_t sp_cnn_num_params(void);
int sp_cnn_create(int32_t max_batch, uint64_t seed, sp_cnn **out);
int sp_cnn_destroy(sp_cnn *c);
int sp_cnn_get_params(const sp_cnn *c, float *h_params);
int sp_cnn_set_params(sp_cnn *c, const float *h_params);
int sp_cnn_get_grads(const sp_cnn *c, float *h_grads);
int sp_cnn_forward(sp_cnn *c, const void *d_ft, const void *d_dmt, int32_t batch, float *d_prob,
                   void *stream);
int sp_cnn_backward(sp_cnn *c, const void *d_ft, const void *d_dmt, const float *d_labels,
                    int32_t batch, float *h_loss, void *stream);
int sp_cnn_adam_step(sp_cnn *c, float lr, void *stream);
int sp_cnn_train_step(sp_cnn *c, const void *d_ft, const void *d_dmt, const float *d_labels,
                      int32_t batch, float lr, float *h_loss, void *stream);
int64_t sp_cnn_features_workspace_bytes(int32_t batch);
int sp_cnn_features(const float *d_sub, int32_t batch, int32_t nsub, int32_t t_in,
                    const int32_t *d_shift, void *d_ft, void *d_dmt, void *d_work,
                    int64_t work_bytes, void *stream);
int sp_dmt_shifts(const double *freqs_mhz, int32_t nchan, int32_t nsub, int32_t max_sweep,
                  int32_t *h_shift);
/* Subband dynamic spectra of candidates (the input of sp_cnn_features),
 * cut from a staged beam (sp_stage_input) searched with `plan`: for
 * candidate q with boxcar width w = h_widths[width_idx], decimation dec =
 * max(1, w / 4) and centre t0 = t + w / 2,
 *   d_sub[q][s][u] = sum over the nchan/256 channels c of subband s and
 *                    i < dec of staged[c][t0 + (u - t_in/2) dec + i + delay[dm_idx][c]]
 * (samples outside [0, n_in) count 0): each subband dedispersed at the
 * candidate's DM by Eq. 1's delays.  d_cands [ncand] device sp_cand;
 * d_sub fp32 [ncand][256][t_in] device; nchan a multiple of 256;
 * ncand <= 65535, t_in <= 4096; every candidate's width_idx < nw.
 * Asynchronous.  Errors: SP_EINVAL, SP_ECUDA. */
int sp_cnn_extract(const sp_plan *plan, const uint8_t *d_staged, int64_t pitch, int64_t n_in,
                   const sp_cand *d_cands, int32_t ncand, const int32_t *h_widths, int32_t nw,
                   int32_t t_in, float *d_sub, void *stream);

/* ---------------------------------------------------------------- stream --
 * Real-time streaming search (Sec. 2 and 3.1: each beam arrives as a
 * continuous stream that is read in blocks overlapping by the largest
 * dispersion sweep, and each block must be searched before the next one
 * arrives).  Beam b's samples arrive in order: first max_delay samples of
 * history (sp_stream_history), then gulps of `gulp` samples
 * (sp_stream_push).  Gulp k of a beam (k = 0, 1, ...) is searched over
 * output samples [k*gulp, (k+1)*gulp) of that beam, from the n_in =
 * gulp + max_delay input samples [k*gulp, k*gulp + n_in): exactly
 * sp_dedisperse and sp_single_pulse_search of that window (a beam of n_out
 * = gulp; one normalisation block when gulp <= norm_block).
 *
 * Device memory: one ring per beam holding the last n_in samples (uint8,
 * time-major), then as many in-flight slots (staged window, DM transform,
 * search scratch, candidates) as fit in hbm_budget_bytes beside the rings,
 * at most max_batch per launch stream plus max_batch more (so that a batch
 * can be admitted while an earlier batch's slots are still held by its
 * classification).  SP_ENOMEM if not even one fits.
 * Scheduling (continuous batching): pushed gulps wait in a FIFO.  Whenever
 * a launch stream and slots are free, the oldest pending gulps (at most
 * max_batch) form a batch: each gulp is copied into its ring (after the
 * beam's previous window was staged), its window is staged into a slot, all
 * of the batch is dedispersed in one persistent launch, each gulp is
 * searched and its candidates are copied back.  Two launch streams let a
 * batch be admitted while the previous one is still on the GPU.  Flags:
 * SP_STREAM_PER_GULP dedisperses each gulp with its own launch;
 * SP_STREAM_ONE_STREAM uses a single launch stream (per-gulp launches on
 * one stream is the per-beam comparison).
 * All progress happens inside sp_stream_push and sp_stream_poll: there are
 * no threads, and one host thread must drive a stream object.
 *
 * sp_stream_history: copies h_hist [max_delay][nchan] (host) into the beam's
 *   ring and restarts its gulp count at 0; synchronous; SP_EINVAL while the
 *   beam has gulps pending or in flight.
 * sp_stream_push: queues gulp h_gulp [gulp][nchan] (host; page-locked
 *   memory makes its copy asynchronous) of the beam, stamps its arrival time
 *   (sp_stream_now's clock) and writes its sequence number to *seq (may be
 *   NULL); the buffer must stay valid and unchanged until poll has returned
 *   that gulp's result.  SP_EINVAL before the beam's history.
 * sp_stream_poll: makes progress, then moves up to max_results finished
 *   gulps (in completion order) to out[] and their candidates to
 *   cands + i * cand_cap (cands may be NULL); *n_results = how many.  wait
 *   != 0 blocks until at least one result is ready or nothing is in flight.
 * sp_gulp_result: beam, seq, t0 = seq * gulp (first searched sample of the
 *   window in the beam's output time), count (total candidates; only
 *   min(count, cand_cap) are returned; status SP_EOVERFLOW when it exceeds),
 *   t_push and t_done (host seconds: arrival, and when all of the gulp's
 *   results were on the host), t_search (when its search candidates were;
 *   = t_done without sp_stream_attach), kept and accepted (below; 0
 *   without sp_stream_attach).
 * sp_stream_pending: gulps queued, in flight (searching or classifying) and
 *   finished-but-not-polled.
 * sp_stream_info: slot count, device bytes held, window length n_in.
 * sp_stream_now: the clock of t_push / t_done (seconds, monotonic).
 *
 * Sifting and classification in the stream (Sec. 3.2: each searched block's
 * candidates are clustered and thresholded, and the surviving cluster peaks
 * are scored by the classifier before the block's results are final).
 * sp_stream_attach: from now on each finished gulp's candidates are sifted
 *   on the host (sp_sift with *params, the gulp's candidates as returned);
 *   with clf != NULL the kept peaks (the first kept_cap in (dm_idx, t)
 *   order) are then cut from the gulp's staged window (sp_cnn_extract,
 *   t_in bins), made into images (sp_cnn_features with the sp_dmt_shifts
 *   table of sweep (t_in - 256) / 2) and scored (sp_cnn_forward) on a
 *   high-priority stream of the library's own while later gulps are
 *   searched; the peaks of all gulps of one finished batch are imaged and
 *   scored together (up to SP_CNN_MAX_BATCH per job).  The gulp's slot is
 *   reused only after its classification has finished, and its result is
 *   returned once the probabilities are on the host.  clf must outlive the
 *   stream and must not run on another stream meanwhile.  With clf: nchan
 *   a multiple of 256, 256 <= t_in <= 4096, t_in even.  1 <= kept_cap <=
 *   SP_CNN_MAX_BATCH.  Allowed once, before the first push (SP_EINVAL
 *   otherwise).
 * sp_stream_poll_sifted: sp_stream_poll, plus per result i its kept peaks
 *   in kept + i * kept_cap and their probabilities p in prob + i * kept_cap
 *   (-1 without a classifier); either may be NULL.  Result fields: kept =
 *   total peaks the sifter kept (status SP_EOVERFLOW when above kept_cap);
 *   accepted = how many of the returned ones have p >= 0.5 (all of them
 *   without a classifier).
 * Every batch has its own status word: if a bounded wait of its
 *   dedispersion ran out, each gulp of that batch is returned with status
 *   SP_ETIMEOUT, count 0 and no candidates (its outputs are void). */
typedef struct sp_stream sp_stream;
typedef struct {
    int32_t beam;
    int32_t status;
    int64_t seq;
    int64_t t0;
    int64_t count;
    double t_push;
    double t_done;
    double t_search;
    int64_t kept;
    int64_t accepted;
} sp_gulp_result;
#define SP_STREAM_PER_GULP 1
#define SP_STREAM_ONE_STREAM 2
int sp_stream_create(const sp_plan *plan, int32_t nbeams, int64_t gulp, const int32_t *h_widths,
                     int32_t nw, float threshold, int64_t norm_block, int64_t cand_cap,
                     int64_t hbm_budget_bytes, int32_t max_batch, int32_t flags, sp_stream **out);
int sp_stream_destroy(sp_stream *s);
int sp_stream_info(const sp_stream *s, int32_t *slots, int64_t *device_bytes, int64_t *n_in);
int sp_stream_history(sp_stream *s, int32_t beam, const uint8_t *h_hist);
int sp_stream_push(sp_stream *s, int32_t beam, const uint8_t *h_gulp, int64_t *seq);
int sp_stream_poll(sp_stream *s, int32_t wait, sp_gulp_result *out, sp_cand *cands,
                   int32_t max_results, int32_t *n_results);
int sp_stream_pending(const sp_stream *s, int64_t *queued, int64_t *in_flight, int64_t *ready);
double sp_stream_now(void);
int sp_stream_attach(sp_stream *s, const sp_sift_params *params, sp_cnn *clf, int32_t t_in, int32_t kept_cap);
int sp_stream_poll_sifted(sp_stream *s, int32_t wait, sp_gulp_result *out, sp_cand *cands, sp_cand *kept,
                          float *prob, int32_t max_results, int32_t *n_results);

#ifdef __cplusplus
}
#endif
#endif /* SPOTLIGHT_H */
