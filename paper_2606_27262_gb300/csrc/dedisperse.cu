// dedisperse.cu -- brute-force incoherent dedispersion on sm_103a
// (arXiv 2606.27262, Sec. 3.1.1: shift every channel by its Eq.-1 delay and
// sum, for every trial DM; the result is the DM transform).
//
//   out[d][t] = sum_c in[t + delay[d][c]][c]
//
// Kernels:
//   stage_input_kernel  time-major [n_in][nchan] -> channel-major
//                       [nchan][pitch] (zero padded), so that one channel's
//                       time series is contiguous.
//   dedisperse_kernel   one CTA = up to DT = 4*CH consecutive trial DMs (a "DM
//                       tile" from the plan) x T = 32*SPT output samples, for
//                       a compiled shape (CH, SPT).  Channels go in chunks of
//                       CH: per channel the CTA stages the window of input
//                       samples the tile's delays reach (T + delay spread +
//                       alignment slack).  Warp 0 fetches chunk k+2 with bulk
//                       asynchronous copies (TMA) into a ring of three raw
//                       slots while the CTA sums chunk k, so every fetch has
//                       two chunks of work to land in; each warp expands one
//                       channel of chunk k+1 into four copies shifted by 0..3
//                       bytes (double-buffered), so that any 4 consecutive
//                       samples are one aligned 32-bit load.  One barrier per
//                       chunk.  One staged byte serves up to DT DMs.
//   dedisperse_batch_kernel  the same tile body in a persistent grid that
//                       takes (beam, DM tile, time tile) items from a work
//                       queue: many beams of uneven length and DM range in
//                       one launch.
//
// Arithmetic: the sum is a pure integer add of bytes (no tensor-core
// contraction exists here).  Each thread owns 4 DMs x 16 samples.  For every
// group of four channels it loads one word (4 consecutive samples) per
// channel, transposes the 4x4 bytes with byte permutes, and adds each
// 4-channel word into an int32 accumulator with one 4-way byte dot product:
// four channel adds per instruction, exact (every sum is at most 255*nchan).
#include <algorithm>
#include <mutex>

#include "sp_internal.h"

namespace sp {
namespace {

constexpr int kStTime = 64;
constexpr int kStChan = 64;

// 64 samples x 64 channels per CTA through shared memory.  Positions of the
// output at and past n_in (up to the pitch) are written as zeros.  Sample t
// is read from input row row0 + t, wrapped at ring_rows (a ring buffer of
// ring_rows samples; row0 = 0 and ring_rows = n_in for a plain input).
__global__ void __launch_bounds__(256) stage_input_kernel(const uint8_t *__restrict__ in, int64_t n_in,
                                                          int32_t nchan, uint8_t *__restrict__ xt,
                                                          int64_t pitch, int64_t row0, int64_t ring_rows) {
    __shared__ __align__(16) uint8_t tile[kStTime][kStChan + 4];
    const int64_t t0 = (int64_t)blockIdx.x * kStTime;
    const int c0 = blockIdx.y * kStChan;
    {
        const int r = threadIdx.x >> 2;
        const int g = (threadIdx.x & 3) * 16;
        const int64_t t = t0 + r;
        uint32_t v[4] = {0u, 0u, 0u, 0u};
        if (t < n_in) {
            int64_t row = row0 + t;  // row0 < ring_rows and t < n_in <= ring_rows: one wrap at most
            if (row >= ring_rows) row -= ring_rows;
            const uint8_t *src = in + row * nchan + c0 + g;
            if ((nchan & 15) == 0 && c0 + g + 16 <= nchan) {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(src));
                v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
            } else {
                for (int j = 0; j < 16; ++j)
                    if (c0 + g + j < nchan) v[j >> 2] |= (uint32_t)src[j] << (8 * (j & 3));
            }
        }
        uint32_t *dst = reinterpret_cast<uint32_t *>(&tile[r][g]);
        dst[0] = v[0]; dst[1] = v[1]; dst[2] = v[2]; dst[3] = v[3];
    }
    __syncthreads();
    const int cc = threadIdx.x >> 2;
    const int tg = (threadIdx.x & 3) * 16;
    if (c0 + cc < nchan) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            w[q] = (uint32_t)tile[tg + 4 * q + 0][cc] | ((uint32_t)tile[tg + 4 * q + 1][cc] << 8) |
                   ((uint32_t)tile[tg + 4 * q + 2][cc] << 16) | ((uint32_t)tile[tg + 4 * q + 3][cc] << 24);
        }
        *reinterpret_cast<uint4 *>(xt + (int64_t)(c0 + cc) * pitch + t0 + tg) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// ---- TMA (bulk async copy) and mbarrier helpers (inline PTX, sm_90+) ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Test hook of the bounded waits (sp_debug_staging_fault): the number of
// SM cycles after which a staging wait gives up (~2^31, about a second, by
// default), and extra bytes that every CTA's first chunk expects beyond
// those its bulk copies bring (0 by default), so that a test can make the
// waits run out with every access in bounds.
__device__ long long g_wait_limit = 1LL << 31;
__device__ uint32_t g_fault_extra_bytes = 0;

// Bounded wait: gives up after g_wait_limit SM cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    const long long limit = *(volatile long long *)&g_wait_limit;
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}
// 1-D bulk copy global -> shared, completion counted on `bar` (bytes and
// both addresses 16-byte multiples).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Summation: for four channels a..d of a chunk and one trial DM, each thread
// loads one aligned word per channel (4 consecutive samples, from the copy
// that matches the channel's delay modulo 4), transposes the 4x4 bytes with
// byte permutes so that word j holds sample j of the four channels, and adds
// each word into sample j's int32 accumulator with one 4-way byte dot
// product (dp4a against 0x01010101): four channel adds per instruction.
__device__ __forceinline__ void add_quad(uint32_t wa, uint32_t wb, uint32_t wc, uint32_t wd, int32_t *acc) {
    const uint32_t t0 = __byte_perm(wa, wb, 0x5140), t1 = __byte_perm(wa, wb, 0x7362);
    const uint32_t t2 = __byte_perm(wc, wd, 0x5140), t3 = __byte_perm(wc, wd, 0x7362);
    acc[0] = (int32_t)__dp4a(__byte_perm(t0, t2, 0x5410), 0x01010101u, (uint32_t)acc[0]);
    acc[1] = (int32_t)__dp4a(__byte_perm(t0, t2, 0x7632), 0x01010101u, (uint32_t)acc[1]);
    acc[2] = (int32_t)__dp4a(__byte_perm(t1, t3, 0x5410), 0x01010101u, (uint32_t)acc[2]);
    acc[3] = (int32_t)__dp4a(__byte_perm(t1, t3, 0x7632), 0x01010101u, (uint32_t)acc[3]);
}

// Packed 8-DM sums: for one channel's word w (samples t..t+3 in bytes 0..3)
// the raw word is added to S and its odd bytes, moved into the low byte of
// each 16-bit lane, to H.  After n <= 257 channels every 16-bit lane of H
// holds an exact sum (samples t+1 and t+3), and S - (H << 8) holds samples
// t and t+2 in its 16-bit lanes: the carries out of the even bytes of S are
// exactly the odd-byte sums that H removes.  Two channels per call, so that
// each sum is one 3-input add.
__device__ __forceinline__ void add_packed(uint32_t wa, uint32_t wb, uint32_t &S, uint32_t &H) {
    S = S + wa + wb;
    H = H + __byte_perm(wa, 0u, 0x4341) + __byte_perm(wb, 0u, 0x4341);
}

// Shared-memory layout (bytes), for a shape with CH channels per chunk and
// DT trial DMs per tile:
//   [0, 8*NS)                 one mbarrier per raw slot
//   [32, 40)                  work item of a persistent CTA
//   [64, 64 + NS*CH*16)       geometry of the chunk in each raw slot
//   [512, 512 + NS*CH*DT*4)   offset table of the chunk in each raw slot
//   then raw[NS][raw_max]     raw channel rows as copied from global memory
//   then copies[2][copies_max] per channel four copies of stride R:
//                             copy r, word j = staged bytes [4j + r, 4j + r + 4)
//
// Chunks are numbered across all tiles a CTA processes (seq0 + k), so that
// a persistent CTA keeps using its mbarriers: chunk g lives in raw slot
// g % NS and completes phase (g / NS) & 1 of that slot's barrier.
//
// Iteration k: warp (k+2) % CH issues chunk k+2; every warp sums chunk k from copies
// buffer k & 1, then waits for chunk k+1's bytes and expands its channel of
// it into copies buffer (k+1) & 1; barrier.  A raw slot is refilled two
// barriers after its chunk was expanded; a copies buffer one barrier after
// its chunk was summed.
//
// A shape has NDT = 4 or 8 trial DMs per thread (DT = NDT*CH per tile).
// With 4, a thread keeps 4 DMs x SPT int32 sums.  With 8, a tile of more than
// 4*CH DMs keeps per DM and 4-sample word two packed 16-bit-lane partials
// (add_packed) -- the same registers as 4 DMs of int32 sums -- and adds
// them to the output every kDedispPackedChannels channels; a smaller tile of
// that shape runs with 4 DMs per thread.  Eight DMs per thread halve the
// copy expansion, the offset-table traffic and the barriers per add.
template <int CH, int SPT, int NDT>
struct Shape {
    static constexpr int DT = NDT * CH;
    static constexpr int T = 32 * SPT;
    static constexpr int NQ = SPT / 4;  // 4-sample words per thread per row
    static constexpr int NS = kDedispRawSlots;
    static constexpr int HDR = dedisp_header_bytes(CH, DT);
    static constexpr int GROUP = kDedispTileGroupDms / DT;  // DM tiles per raster group
    static constexpr int FLUSH = kDedispPackedChannels / CH;  // chunks per packed flush
    static_assert(NDT == 4 || NDT == 8, "offsets are read as int4 per 4 DMs");
    static_assert(kDedispPackedChannels % CH == 0 && kDedispPackedChannels <= 257, "16-bit lanes");
    static_assert(SPT % 4 == 0 && T <= kDedispMaxTimeTile, "time tile");
    static_assert(CH <= kDedispMaxChanChunk && CH % 4 == 0, "the issuing warp's lanes copy one channel each; quads");
    static_assert(8 * NS <= kDedispItemOffset && kDedispItemOffset + 8 <= kDedispGeoOffset,
                  "mbarriers, work item and geometry ring overlap");
    static_assert(kDedispGeoOffset + NS * CH * 16 <= kDedispOffTabOffset, "geometry ring overlaps the offsets");
    static_assert(HDR % 128 == 0, "raw slots start 128-byte aligned");
};

// Maps the id of a (DM tile, time tile) pair of one beam to the pair.
// Groups of G DM tiles sweep all time tiles, so the CTAs resident at one
// time share an input window that fits in L2 (DM-tile-fastest order would
// make them span the whole dispersion sweep).
__device__ __forceinline__ void raster(int64_t id, int ntiles, int64_t ntime, int G, int &tile, int64_t &tq) {
    const int64_t per_group = (int64_t)G * ntime;
    const int group = (int)(id / per_group);
    const int64_t r = id - group * per_group;
    const int width = min(G, ntiles - group * G);
    tile = group * G + (int)(r % width);
    tq = r / width;
}

// One (DM tile, time tile) of one beam, with DT = the shape's table stride
// and PACKED = 8 DMs per thread; SPLIT (with PACKED) = the warps split the
// time tile in two halves, so that CH/2 warps of 8 DMs cover a tile of at
// most 4*CH DMs with the packed sums.  Returns false (uniformly across the CTA)
// if a staging wait ran out; copies still in flight are waited for (with
// the same bound) before it returns.
template <int CH, int SPT, int DT, bool PACKED, bool SPLIT = false>
__device__ __forceinline__ bool dedisp_tile_body(uint8_t *smem, uint32_t seq0, const uint8_t *__restrict__ xt,
                                                 int64_t pitch, int32_t nchan, int32_t nchunks, int d_first,
                                                 int d_cnt, int64_t t0, const int4 *__restrict__ geo_g,
                                                 const int32_t *__restrict__ off_g, int32_t copies_max,
                                                 int32_t raw_max, int64_t n_out, int32_t *__restrict__ out) {
    using S = Shape<CH, SPT, DT / CH>;
    constexpr int NDT = PACKED ? 8 : 4, NS = S::NS, HDR = S::HDR, FLUSH = S::FLUSH;
    static_assert(!SPLIT || (PACKED && CH % 2 == 0 && S::NQ % 2 == 0), "time split: packed body, even halves");
    // 4-sample words per lane and row of this warp's share of the time tile
    constexpr int NQ = SPLIT ? S::NQ / 2 : S::NQ;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);                       // [NS]
    int4 *geo_s = reinterpret_cast<int4 *>(smem + kDedispGeoOffset);           // [NS][CH]
    int32_t *offt_s = reinterpret_cast<int32_t *>(smem + kDedispOffTabOffset);  // [NS][CH*DT]
    uint8_t *raw_s = smem + HDR;                                                // [NS][raw_max]
    uint8_t *cop_s = raw_s + NS * raw_max;                                      // [2][copies_max]

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    // DM group and time half of this warp (one half without SPLIT)
    const int dg = SPLIT ? warp % (CH / 2) : warp;
    const int th = SPLIT ? warp / (CH / 2) : 0;
    const bool warp_active = dg * NDT < d_cnt;
    const int4 zero4 = make_int4(0, 0, 0, 0);

    auto slot_of = [&](int kk) { return (int)((seq0 + (uint32_t)kk) % NS); };
    auto parity_of = [&](int kk) { return ((seq0 + (uint32_t)kk) / NS) & 1u; };
    auto issue = [&](int kk, int4 g) {  // by one warp: chunk kk into its raw slot
        const int sl = slot_of(kk);
        const int nc = min(CH, nchan - kk * CH);
        uint32_t bytes = (lane < nc) ? (uint32_t)g.y + 16u : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
        if (lane < CH) geo_s[sl * CH + lane] = (lane < nc) ? g : zero4;
        fence_proxy_async();
        if (lane == 0)
            mbar_arrive_expect_tx(&mbar[sl], bytes + (uint32_t)(CH * DT * 4) + (kk == 0 ? g_fault_extra_bytes : 0u));
        __syncwarp();
        if (lane < nc)
            bulk_g2s(raw_s + sl * raw_max + g.w, xt + (int64_t)(kk * CH + lane) * pitch + t0 + g.x,
                     (uint32_t)g.y + 16u, &mbar[sl]);
        if (lane == CH) bulk_g2s(offt_s + sl * CH * DT, off_g + (int64_t)kk * CH * DT, CH * DT * 4, &mbar[sl]);
    };
    auto load_geo = [&](int kk) -> int4 {
        return (kk < nchunks && lane < CH && kk * CH + lane < nchan) ? __ldg(geo_g + (int64_t)kk * CH + lane)
                                                                      : zero4;
    };
    // Four shifted copies of this warp's channel of chunk kk, from its raw
    // slot into copies buffer kk & 1.
    auto build = [&](int kk) {
        const int sl = slot_of(kk);
        if (kk * CH + warp >= nchan) return;
        const int4 g = geo_s[sl * CH + warp];
        const int32_t R = g.y, Sd = g.y;
        const uint8_t *src = raw_s + sl * raw_max + g.w;
        uint8_t *row = cop_s + (kk & 1) * copies_max + g.z;
        const int nseg = R / 16;
        for (int q0 = 0; q0 < nseg; q0 += 32) {
            const int q = q0 + lane;
            const bool act = q < nseg;
            uint4 a = make_uint4(0u, 0u, 0u, 0u);
            if (act) a = *reinterpret_cast<const uint4 *>(src + 16 * q);
            uint32_t e = __shfl_down_sync(0xffffffffu, a.x, 1);
            if (act && (lane == 31 || q + 1 >= nseg)) e = *reinterpret_cast<const uint32_t *>(src + 16 * q + 16);
            if (act) {
                *reinterpret_cast<uint4 *>(row + 16 * q) = a;
                *reinterpret_cast<uint4 *>(row + Sd + 16 * q) =
                    make_uint4(__byte_perm(a.x, a.y, 0x4321), __byte_perm(a.y, a.z, 0x4321),
                               __byte_perm(a.z, a.w, 0x4321), __byte_perm(a.w, e, 0x4321));
                *reinterpret_cast<uint4 *>(row + 2 * Sd + 16 * q) =
                    make_uint4(__byte_perm(a.x, a.y, 0x5432), __byte_perm(a.y, a.z, 0x5432),
                               __byte_perm(a.z, a.w, 0x5432), __byte_perm(a.w, e, 0x5432));
                *reinterpret_cast<uint4 *>(row + 3 * Sd + 16 * q) =
                    make_uint4(__byte_perm(a.x, a.y, 0x6543), __byte_perm(a.y, a.z, 0x6543),
                               __byte_perm(a.z, a.w, 0x6543), __byte_perm(a.w, e, 0x6543));
            }
        }
    };
    // Warp 0 issues chunks 0 and 1; chunk j >= 2 is issued by warp j % CH,
    // so that the issuing work (and the wait at the next barrier for the
    // warp doing it) rotates over the warps.  Each warp holds the geometry of
    // the next chunk it will issue, loaded CH chunks ahead.
    const int first_mine = warp >= 2 ? warp : warp + CH;
    int4 g_mine = load_geo(first_mine);
    if (warp == 0) {
        const int4 g0 = load_geo(0), g1 = load_geo(1);
        issue(0, g0);
        if (nchunks > 1) issue(1, g1);
    }
    __syncthreads();
    // A wait that runs out sets `failed`.  Later iterations then issue and
    // sum nothing; they wait again (bounded) for the chunk that timed out and
    // then for every chunk already issued, so that no copy lands in shared
    // memory after the CTA has left.  A second timeout gives up waiting.
    int last_issued = min(nchunks, 2) - 1;
    int pending = 0;  // next chunk to wait for
    bool failed = false;
    {
        const bool ok = mbar_wait_bounded(&mbar[slot_of(0)], parity_of(0));
        if (ok) {
            build(0);
            pending = 1;
        }
        failed = __syncthreads_or(!ok);
    }

    // 4 DMs: int32 sums acc[i][4q + j] of sample t0 + 128q + 4*lane + j.
    // 8 DMs: packed partials pk[i][q] = {S, H} of the same samples.
    constexpr int NACC = PACKED ? 1 : NDT;
    constexpr int NPK = PACKED ? NDT : 1;
    int32_t acc[NACC][SPT];
    uint32_t pk[NPK][NQ][2];
#pragma unroll
    for (int i = 0; i < NACC; ++i)
#pragma unroll
        for (int j = 0; j < SPT; ++j) acc[i][j] = 0;
#pragma unroll
    for (int i = 0; i < NPK; ++i)
#pragma unroll
        for (int q = 0; q < NQ; ++q) pk[i][q][0] = pk[i][q][1] = 0u;
    const bool vec = (n_out & 3) == 0;

    // Adds the packed partials to the output (stores them on the first
    // flush) and clears them.
    auto flush = [&](bool first) {
#pragma unroll
        for (int i = 0; i < NPK; ++i) {
            const int dl = dg * NDT + i;
            if (dl >= d_cnt) continue;
            int32_t *orow = out + (int64_t)(d_first + dl) * n_out;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const uint32_t H = pk[i][q][1], L = pk[i][q][0] - (H << 8);
                const int32_t v0 = (int32_t)(L & 0xFFFFu), v1 = (int32_t)(H & 0xFFFFu);
                const int32_t v2 = (int32_t)(L >> 16), v3 = (int32_t)(H >> 16);
                pk[i][q][0] = pk[i][q][1] = 0u;
                const int64_t t = t0 + 128 * NQ * th + 128 * q + 4 * lane;
                if (vec && t + 3 < n_out) {
                    int4 *dst = reinterpret_cast<int4 *>(orow + t);
                    int4 cur = first ? zero4 : *dst;
                    cur.x += v0;
                    cur.y += v1;
                    cur.z += v2;
                    cur.w += v3;
                    *dst = cur;
                } else {
                    const int32_t v[4] = {v0, v1, v2, v3};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (t + j < n_out) orow[t + j] = (first ? 0 : orow[t + j]) + v[j];
                }
            }
        }
    };

    for (int k = 0; k < nchunks; ++k) {
        const int b = k & 1;
        const int nc = min(CH, nchan - k * CH);
        if (!failed && k + 2 < nchunks) {
            last_issued = k + 2;
            if (warp == (k + 2) % CH) {
                issue(k + 2, g_mine);
                g_mine = load_geo(k + 2 + CH);
            }
        }
        if (warp_active && !failed) {
            const uint8_t *sb = cop_s + b * copies_max + 128 * NQ * th + lane * 4;
            const int32_t *ot = offt_s + slot_of(k) * CH * DT + dg * NDT;
            if constexpr (PACKED) {
                if (nc == CH) {
#pragma unroll
                    for (int cp = 0; cp < CH / 2; ++cp) {
                        const int4 x0 = *reinterpret_cast<const int4 *>(ot + (2 * cp) * DT);
                        const int4 x1 = *reinterpret_cast<const int4 *>(ot + (2 * cp) * DT + 4);
                        const int4 y0 = *reinterpret_cast<const int4 *>(ot + (2 * cp + 1) * DT);
                        const int4 y1 = *reinterpret_cast<const int4 *>(ot + (2 * cp + 1) * DT + 4);
                        const int32_t oa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
                        const int32_t ob[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
                        for (int i = 0; i < NDT; ++i) {
#pragma unroll
                            for (int q = 0; q < NQ; ++q) {
                                const uint32_t wa = *reinterpret_cast<const uint32_t *>(sb + oa[i] + 128 * q);
                                const uint32_t wb = *reinterpret_cast<const uint32_t *>(sb + ob[i] + 128 * q);
                                add_packed(wa, wb, pk[i][q][0], pk[i][q][1]);
                            }
                        }
                    }
                } else {
                    for (int c = 0; c < nc; ++c) {
                        const int4 x0 = *reinterpret_cast<const int4 *>(ot + c * DT);
                        const int4 x1 = *reinterpret_cast<const int4 *>(ot + c * DT + 4);
                        const int32_t oa[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                        for (int i = 0; i < NDT; ++i) {
#pragma unroll
                            for (int q = 0; q < NQ; ++q) {
                                const uint32_t w = *reinterpret_cast<const uint32_t *>(sb + oa[i] + 128 * q);
                                add_packed(w, 0u, pk[i][q][0], pk[i][q][1]);
                            }
                        }
                    }
                }
            } else {
                if (nc == CH) {
#pragma unroll
                    for (int qd = 0; qd < CH / 4; ++qd) {
                        const int4 o0 = *reinterpret_cast<const int4 *>(ot + (4 * qd + 0) * DT);
                        const int4 o1 = *reinterpret_cast<const int4 *>(ot + (4 * qd + 1) * DT);
                        const int4 o2 = *reinterpret_cast<const int4 *>(ot + (4 * qd + 2) * DT);
                        const int4 o3 = *reinterpret_cast<const int4 *>(ot + (4 * qd + 3) * DT);
                        const int32_t a0[4] = {o0.x, o0.y, o0.z, o0.w}, a1[4] = {o1.x, o1.y, o1.z, o1.w};
                        const int32_t a2[4] = {o2.x, o2.y, o2.z, o2.w}, a3[4] = {o3.x, o3.y, o3.z, o3.w};
#pragma unroll
                        for (int i = 0; i < NDT; ++i) {
#pragma unroll
                            for (int q = 0; q < NQ; ++q) {
                                const uint32_t wa = *reinterpret_cast<const uint32_t *>(sb + a0[i] + 128 * q);
                                const uint32_t wb = *reinterpret_cast<const uint32_t *>(sb + a1[i] + 128 * q);
                                const uint32_t wc = *reinterpret_cast<const uint32_t *>(sb + a2[i] + 128 * q);
                                const uint32_t wd = *reinterpret_cast<const uint32_t *>(sb + a3[i] + 128 * q);
                                add_quad(wa, wb, wc, wd, &acc[i][4 * q]);
                            }
                        }
                    }
                } else {
                    for (int c = 0; c < nc; ++c) {
                        const int4 oc = *reinterpret_cast<const int4 *>(ot + c * DT);
                        const int32_t ac[4] = {oc.x, oc.y, oc.z, oc.w};
#pragma unroll
                        for (int i = 0; i < NDT; ++i) {
#pragma unroll
                            for (int q = 0; q < NQ; ++q) {
                                const uint32_t w = *reinterpret_cast<const uint32_t *>(sb + ac[i] + 128 * q);
                                add_quad(w, 0u, 0u, 0u, &acc[i][4 * q]);
                            }
                        }
                    }
                }
            }
            if constexpr (PACKED) {
                if ((k + 1) % FLUSH == 0 || k + 1 == nchunks) flush(k < FLUSH);
            }
        }
        bool ok = true;
        if (pending <= last_issued) {
            ok = mbar_wait_bounded(&mbar[slot_of(pending)], parity_of(pending));
            if (ok) {
                if (!failed) build(pending);
                ++pending;
            } else if (failed) {
                pending = last_issued + 1;
            }
        }
        failed = __syncthreads_or(failed || !ok);
    }
    if (failed) return false;

    if constexpr (!PACKED) {
#pragma unroll
        for (int i = 0; i < NDT; ++i) {
            const int dl = dg * NDT + i;
            if (dl >= d_cnt) continue;
            int32_t *orow = out + (int64_t)(d_first + dl) * n_out;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const int64_t t = t0 + 128 * NQ * th + 128 * q + 4 * lane;
                if (vec && t + 3 < n_out) {
                    *reinterpret_cast<int4 *>(orow + t) =
                        make_int4(acc[i][4 * q], acc[i][4 * q + 1], acc[i][4 * q + 2], acc[i][4 * q + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (t + j < n_out) orow[t + j] = acc[i][4 * q + j];
                }
            }
        }
    }
    return true;
}

// One tile of a shape with NDT DMs per thread: tiles of more than 4*CH DMs
// take the packed 8-DM body, the others the packed body with the time tile
// split between two halves of the warps (same tables); shapes with 4 DMs
// per thread take the 4-DM body.
template <int CH, int SPT, int NDT>
__device__ __forceinline__ bool dedisp_tile(uint8_t *smem, uint32_t seq0, const uint8_t *__restrict__ xt,
                                            int64_t pitch, int32_t nchan, int32_t nchunks, int d_first, int d_cnt,
                                            int64_t t0, const int4 *__restrict__ geo_g,
                                            const int32_t *__restrict__ off_g, int32_t copies_max,
                                            int32_t raw_max, int64_t n_out, int32_t *__restrict__ out) {
    constexpr int DT = NDT * CH;
    if constexpr (NDT == 8) {
        if (d_cnt > 4 * CH)
            return dedisp_tile_body<CH, SPT, DT, true>(smem, seq0, xt, pitch, nchan, nchunks, d_first, d_cnt, t0,
                                                       geo_g, off_g, copies_max, raw_max, n_out, out);
        return dedisp_tile_body<CH, SPT, DT, true, true>(smem, seq0, xt, pitch, nchan, nchunks, d_first, d_cnt, t0,
                                                         geo_g, off_g, copies_max, raw_max, n_out, out);
    } else {
        return dedisp_tile_body<CH, SPT, DT, false>(smem, seq0, xt, pitch, nchan, nchunks, d_first, d_cnt, t0,
                                                    geo_g, off_g, copies_max, raw_max, n_out, out);
    }
}

__device__ __forceinline__ void init_barriers(uint8_t *smem) {
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);
    if (threadIdx.x < kDedispRawSlots) mbar_init(&mbar[threadIdx.x], 1);
    if (threadIdx.x == 0) fence_mbar_init();
    __syncthreads();
}

// One beam: grid = (DM tiles, time tiles), one (DM tile, time tile) per CTA
// in raster order.
template <int CH, int SPT, int NDT>
__global__ void __launch_bounds__(CH * 32, (CH == 8 ? 2 : 3))
dedisperse_kernel(const uint8_t *__restrict__ xt, int64_t pitch, int32_t nchan, int32_t nchunks,
                  const int32_t *__restrict__ tile_first, const int32_t *__restrict__ tile_count,
                  const int4 *__restrict__ chunk_geo, const int32_t *__restrict__ chunk_off, int32_t copies_max,
                  int32_t raw_max, int64_t n_out, int32_t *__restrict__ out, int32_t *__restrict__ status) {
    using S = Shape<CH, SPT, NDT>;
    extern __shared__ __align__(128) uint8_t smem[];
    int tile;
    int64_t tq;
    raster((int64_t)blockIdx.y * gridDim.x + blockIdx.x, (int)gridDim.x, (int64_t)gridDim.y, S::GROUP, tile, tq);
    init_barriers(smem);
    const bool ok = dedisp_tile<CH, SPT, NDT>(smem, 0u, xt, pitch, nchan, nchunks, tile_first[tile], tile_count[tile],
                                         tq * S::T, chunk_geo + (int64_t)tile * nchunks * CH,
                                         chunk_off + (int64_t)tile * nchunks * CH * S::DT, copies_max, raw_max,
                                         n_out, out);
    if (!ok && threadIdx.x == 0) atomicOr(status, SP_STATUS_STAGING_TIMEOUT);
}

// Last beam whose first item is <= item.
__device__ __forceinline__ int beam_of(const int64_t *__restrict__ item_begin, int32_t nbeams, int64_t item) {
    int lo = 0, hi = nbeams - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(item_begin + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Many beams in one launch, one item per CTA (item = blockIdx.x): the grid
// kernel's body after a lookup of the item's beam.  CTAs retire, so the
// block scheduler can interleave other kernels' CTAs (a search, a
// classifier) between them.  Items are (beam, DM tile, time tile), numbered
// beam by beam and, within a beam, in the raster order of the grid kernel;
// beams may differ in length, DM list and channel count but share the kernel
// shape.
template <int CH, int SPT, int NDT>
__global__ void __launch_bounds__(CH * 32, (CH == 8 ? 2 : 3))
dedisperse_items_kernel(const BatchBeamDev *__restrict__ beams, const int64_t *__restrict__ item_begin,
                        int32_t nbeams, int64_t nitems, int32_t copies_max, int32_t raw_max,
                        int32_t *__restrict__ status) {
    using S = Shape<CH, SPT, NDT>;
    extern __shared__ __align__(128) uint8_t smem[];
    const int64_t item = blockIdx.x;
    if (item >= nitems) return;
    const int b = beam_of(item_begin, nbeams, item);
    const BatchBeamDev bm = beams[b];
    int tile;
    int64_t tq;
    raster(item - __ldg(item_begin + b), bm.ntiles, (int64_t)bm.ntime, S::GROUP, tile, tq);
    init_barriers(smem);
    const bool ok = dedisp_tile<CH, SPT, NDT>(smem, 0u, bm.xt, bm.pitch, bm.nchan, bm.nchunks, __ldg(bm.tile_first + tile),
                                         __ldg(bm.tile_count + tile), tq * S::T,
                                         bm.geo + (int64_t)tile * bm.nchunks * CH,
                                         bm.off + (int64_t)tile * bm.nchunks * CH * S::DT, copies_max, raw_max,
                                         bm.n_out, bm.out);
    if (!ok && threadIdx.x == 0) atomicOr(status, SP_STATUS_STAGING_TIMEOUT);
}

// The same items from a persistent grid: each CTA takes items from a work
// queue (one atomic per item) until it is empty; its mbarrier phases carry
// over from item to item.  (counter == nullptr: one item per CTA, as the
// items kernel, in this kernel's loop.)
template <int CH, int SPT, int NDT>
__global__ void __launch_bounds__(CH * 32, (CH == 8 ? 2 : 3))
dedisperse_batch_kernel(const BatchBeamDev *__restrict__ beams, const int64_t *__restrict__ item_begin,
                        int32_t nbeams, int64_t nitems, unsigned long long *__restrict__ counter,
                        int32_t copies_max, int32_t raw_max, int32_t *__restrict__ status) {
    using S = Shape<CH, SPT, NDT>;
    extern __shared__ __align__(128) uint8_t smem[];
    long long *s_item = reinterpret_cast<long long *>(smem + kDedispItemOffset);
    init_barriers(smem);
    uint32_t seq = 0;
    for (int pass = 0;; ++pass) {
        if (counter) {
            if (threadIdx.x == 0) *s_item = (long long)atomicAdd(counter, 1ull);
        } else if (threadIdx.x == 0) {
            *s_item = pass == 0 ? (long long)blockIdx.x : (long long)nitems;
        }
        __syncthreads();
        const int64_t item = *s_item;  // thread 0 rewrites it only after the tile's barriers
        if (item >= nitems) break;
        const int lo = beam_of(item_begin, nbeams, item);
        const BatchBeamDev &bm = beams[lo];
        const int32_t nchunks = bm.nchunks;
        int tile;
        int64_t tq;
        raster(item - __ldg(item_begin + lo), bm.ntiles, (int64_t)bm.ntime, S::GROUP, tile, tq);
        const bool ok = dedisp_tile<CH, SPT, NDT>(smem, seq, bm.xt, bm.pitch, bm.nchan, nchunks, __ldg(bm.tile_first + tile),
                                             __ldg(bm.tile_count + tile), tq * S::T,
                                             bm.geo + (int64_t)tile * nchunks * CH,
                                             bm.off + (int64_t)tile * nchunks * CH * S::DT, copies_max, raw_max,
                                             bm.n_out, bm.out);
        if (!ok) {
            if (threadIdx.x == 0) atomicOr(status, SP_STATUS_STAGING_TIMEOUT);
            return;
        }
        seq += (uint32_t)nchunks;
    }
}

using GridKernel = void (*)(const uint8_t *, int64_t, int32_t, int32_t, const int32_t *, const int32_t *,
                            const int4 *, const int32_t *, int32_t, int32_t, int64_t, int32_t *, int32_t *);
using BatchKernel = void (*)(const BatchBeamDev *, const int64_t *, int32_t, int64_t, unsigned long long *, int32_t,
                             int32_t, int32_t *);
using ItemsKernel = void (*)(const BatchBeamDev *, const int64_t *, int32_t, int64_t, int32_t, int32_t, int32_t *);
struct ShapeKernels {
    GridKernel grid;
    BatchKernel batch;
    ItemsKernel items;
    int threads;
    int time_tile;
};
template <int CH, int SPT, int NDT>
constexpr ShapeKernels shape_kernels() {
    return {dedisperse_kernel<CH, SPT, NDT>, dedisperse_batch_kernel<CH, SPT, NDT>,
            dedisperse_items_kernel<CH, SPT, NDT>, CH * 32, Shape<CH, SPT, NDT>::T};
}
template <int I, int CH, int SPT, int NDT>
constexpr bool shape_is() {
    return kDedispShapeCh[I] == CH && kDedispShapeSpt[I] == SPT && kDedispShapeNdt[I] == NDT;
}
static_assert(kDedispNumShapes == 4 && shape_is<0, 8, 16, 8>() && shape_is<1, 8, 16, 4>() &&
                  shape_is<2, 8, 8, 4>() && shape_is<3, 4, 16, 4>(),
              "compiled shapes match the shape table");
const ShapeKernels kShapes[kDedispNumShapes] = {shape_kernels<8, 16, 8>(), shape_kernels<8, 16, 4>(),
                                                shape_kernels<8, 8, 4>(), shape_kernels<4, 16, 4>()};

constexpr int kMaxDev = 64;
std::mutex g_cfg_lock;
int g_cfg_smem[kMaxDev][kDedispNumShapes] = {};  // configured dynamic smem per (device, shape)

int configure_shape(int shape, int smem_bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SP_ECUDA;
    if (dev < 0 || dev >= kMaxDev || shape < 0 || shape >= kDedispNumShapes) return SP_ELIMIT;
    std::lock_guard<std::mutex> guard(g_cfg_lock);
    if (g_cfg_smem[dev][shape] >= smem_bytes) return SP_OK;
    if (cudaFuncSetAttribute(kShapes[shape].grid, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(kShapes[shape].batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(kShapes[shape].items, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes) !=
            cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    g_cfg_smem[dev][shape] = smem_bytes;
    return SP_OK;
}

}  // namespace

int set_staging_fault(uint32_t extra_bytes, long long wait_limit) {
    if (cudaMemcpyToSymbol(g_fault_extra_bytes, &extra_bytes, sizeof extra_bytes) != cudaSuccess ||
        cudaMemcpyToSymbol(g_wait_limit, &wait_limit, sizeof wait_limit) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    return SP_OK;
}

int launch_stage_input(const uint8_t *d_in, int64_t n_in, int32_t nchan, uint8_t *d_staged, int64_t pitch,
                       cudaStream_t stream, int64_t row0, int64_t ring_rows) {
    if (ring_rows <= 0) ring_rows = n_in;
    if (row0 < 0 || row0 >= ring_rows || n_in > ring_rows) return SP_EINVAL;
    const dim3 grid((unsigned)(pitch / kStTime), (unsigned)((nchan + kStChan - 1) / kStChan));
    stage_input_kernel<<<grid, 256, 0, stream>>>(d_in, n_in, nchan, d_staged, pitch, row0, ring_rows);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int64_t dedisp_time_tiles(const sp_plan *plan, int64_t n_out) {
    return (n_out + plan->time_tile - 1) / plan->time_tile;
}

int dedisp_configure(const sp_plan *plan) { return configure_shape(plan->shape, plan->smem_bytes); }

int launch_dedisperse(const sp_plan *plan, const uint8_t *d_xt, int64_t pitch, int64_t n_out, int32_t *d_out,
                      cudaStream_t stream, int32_t *status) {
    int rc = dedisp_configure(plan);
    if (rc) return rc;
    const ShapeKernels &k = kShapes[plan->shape];
    const dim3 grid((unsigned)plan->ntiles, (unsigned)dedisp_time_tiles(plan, n_out));
    k.grid<<<grid, k.threads, plan->smem_bytes, stream>>>(d_xt, pitch, plan->nchan, plan->nchunks,
                                                          plan->d_tile_first, plan->d_tile_count,
                                                          plan->d_chunk_geo, plan->d_chunk_off, plan->copies_max,
                                                          plan->raw_max, n_out, d_out,
                                                          status ? status : plan->d_status);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

// Persistent grid: as many CTAs as fit on the device at once.
int batch_grid(BatchLaunch &b) {
    if (b.shape < 0 || b.shape >= kDedispNumShapes) return SP_EINVAL;
    int rc = configure_shape(b.shape, b.smem_bytes);
    if (rc) return rc;
    const ShapeKernels &k = kShapes[b.shape];
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.batch, k.threads, b.smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    if (per_sm < 1) return SP_ELIMIT;
    b.grid = nsm * per_sm;
    return SP_OK;
}

int launch_dedisperse_batch(const BatchLaunch &b, cudaStream_t stream, bool persistent) {
    if (b.shape < 0 || b.shape >= kDedispNumShapes || b.grid < 1) return SP_EINVAL;
    const ShapeKernels &k = kShapes[b.shape];
    int64_t grid = std::max<int64_t>(b.nitems, 1);
    if (persistent) {
        if (cudaMemsetAsync(b.d_counter, 0, sizeof(unsigned long long), stream) != cudaSuccess) return SP_ECUDA;
        grid = std::min<int64_t>(b.grid, grid);
    } else if (grid > INT32_MAX) {
        return SP_ELIMIT;
    }
    if (persistent)
        k.batch<<<(unsigned)grid, k.threads, b.smem_bytes, stream>>>(b.d_beams, b.d_item_begin, b.nbeams, b.nitems,
                                                                     b.d_counter, b.copies_max, b.raw_max, b.d_status);
    else
        k.items<<<(unsigned)grid, k.threads, b.smem_bytes, stream>>>(b.d_beams, b.d_item_begin, b.nbeams, b.nitems,
                                                                     b.copies_max, b.raw_max, b.d_status);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

}  // namespace sp
