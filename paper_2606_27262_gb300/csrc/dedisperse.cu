// dedisperse.cu -- brute-force incoherent dedispersion on sm_103a
// (arXiv 2606.27262, Sec. 3.1.1: shift every channel by its Eq.-1 delay and
// sum, for every trial DM; the result is the DM transform).
//
//   out[d][t] = sum_c in[t + delay[d][c]][c]
//
// Two kernels:
//   stage_input_kernel  time-major [n_in][nchan] -> channel-major
//                       [nchan][pitch] (zero padded), so that one channel's
//                       time series is contiguous.
//   dedisperse_kernel   one CTA = up to 32 consecutive trial DMs (a "DM tile"
//                       from the plan) x 512 output samples.  Channels go in
//                       chunks of 8: per channel the CTA stages the window of
//                       input samples the tile's delays reach (512 + delay
//                       spread + alignment slack).  Warp 0 fetches chunk k+2
//                       with bulk asynchronous copies (TMA) into a ring of
//                       three raw slots while the CTA sums chunk k, so every
//                       fetch has two chunks of work to land in; each warp
//                       expands one channel of chunk k+1 into four copies
//                       shifted by 0..3 bytes (double-buffered), so that any
//                       4 consecutive samples are one aligned 32-bit load.
//                       One barrier per chunk.  One staged byte serves up to
//                       32 DMs.
//
// Arithmetic: the sum is a pure integer add of bytes (no tensor-core
// contraction exists here).  Each thread owns 4 DMs x 16 samples.  For every
// group of four channels it loads one word (4 consecutive samples) per
// channel, transposes the 4x4 bytes with byte permutes, and adds each
// 4-channel word into an int32 accumulator with one 4-way byte dot product:
// four channel adds per instruction, exact (every sum is at most 255*nchan).
#include "sp_internal.h"

namespace sp {
namespace {

constexpr int kStTime = 64;
constexpr int kStChan = 64;

// 64 samples x 64 channels per CTA through shared memory.  Positions of the
// output at and past n_in (up to the pitch) are written as zeros.
__global__ void __launch_bounds__(256) stage_input_kernel(const uint8_t *__restrict__ in, int64_t n_in,
                                                          int32_t nchan, uint8_t *__restrict__ xt,
                                                          int64_t pitch) {
    __shared__ __align__(16) uint8_t tile[kStTime][kStChan + 4];
    const int64_t t0 = (int64_t)blockIdx.x * kStTime;
    const int c0 = blockIdx.y * kStChan;
    {
        const int r = threadIdx.x >> 2;
        const int g = (threadIdx.x & 3) * 16;
        const int64_t t = t0 + r;
        uint32_t v[4] = {0u, 0u, 0u, 0u};
        if (t < n_in) {
            const uint8_t *src = in + t * nchan + c0 + g;
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
// Bounded wait: gives up after ~2^31 SM cycles (about a second).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) return false;
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

// Shared-memory layout (bytes):
//   [0, 8*NS)                 one mbarrier per raw slot
//   [64, 64 + NS*CH*16)       geometry of the chunk in each raw slot
//   [512, 512 + NS*CH*DT*4)   offset table of the chunk in each raw slot
//   then raw[NS][raw_max]     raw channel rows as copied from global memory
//   then copies[2][copies_max] per channel four copies of stride R:
//                             copy r, word j = staged bytes [4j + r, 4j + r + 4)
//
// Iteration k: warp 0 issues chunk k+2 into raw slot (k+2) % NS; every warp
// sums chunk k from copies buffer k & 1, then waits for chunk k+1's bytes and
// expands its channel of it into copies buffer (k+1) & 1; barrier.  A raw
// slot is refilled two barriers after its chunk was expanded; a copies
// buffer one barrier after its chunk was summed.
template <int NDT, int NWARP, int CH>
__global__ void __launch_bounds__(NWARP * 32, 2)
dedisperse_kernel(const uint8_t *__restrict__ xt, int64_t pitch, int32_t nchan, int32_t nchunks,
                  const int32_t *__restrict__ tile_first, const int32_t *__restrict__ tile_count,
                  const int4 *__restrict__ chunk_geo, const int32_t *__restrict__ chunk_off, int32_t copies_max,
                  int32_t raw_max, int64_t n_out, int32_t *__restrict__ out, int32_t *__restrict__ status) {
    static_assert(NDT == 4, "offset table is read as int4 per thread");
    constexpr int DT = NDT * NWARP;
    constexpr int T = kDedispTimeTile;
    constexpr int NS = kDedispRawSlots;
    static_assert(T == 32 * 16, "a warp spans the time tile: 32 lanes x 16 samples");
    static_assert(CH <= 31 && NWARP == CH && CH % 4 == 0, "warp 0 lanes issue one channel each; one warp per channel");
    static_assert(DT == kDedispDmTile && CH == kDedispChanChunk, "layout shared with the plan");
    static_assert(8 * NS <= kDedispGeoOffset, "mbarriers overlap the geometry ring");
    static_assert(kDedispGeoOffset + NS * CH * 16 <= kDedispOffTabOffset, "geometry ring overlaps the offsets");

    extern __shared__ __align__(128) uint8_t smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);                       // [NS]
    int4 *geo_s = reinterpret_cast<int4 *>(smem + kDedispGeoOffset);           // [NS][CH]
    int32_t *offt_s = reinterpret_cast<int32_t *>(smem + kDedispOffTabOffset);  // [NS][CH*DT]
    uint8_t *raw_s = smem + kDedispHeaderBytes;                                 // [NS][raw_max]
    uint8_t *cop_s = raw_s + NS * raw_max;                                      // [2][copies_max]

    // Raster: groups of kDedispTileGroup DM tiles sweep all time tiles, so
    // the CTAs resident at one time share an input window that fits in L2
    // (DM-tile-fastest order would make them span the whole sweep).
    int tile;
    int64_t t0;
    {
        const int ntiles = gridDim.x, ntime = gridDim.y;
        const int64_t id = (int64_t)blockIdx.y * ntiles + blockIdx.x;
        const int64_t per_group = (int64_t)kDedispTileGroup * ntime;
        const int group = (int)(id / per_group);
        const int64_t r = id - group * per_group;
        const int width = min(kDedispTileGroup, ntiles - group * kDedispTileGroup);
        tile = group * kDedispTileGroup + (int)(r % width);
        t0 = (r / width) * T;
    }
    const int d_first = tile_first[tile];
    const int d_cnt = tile_count[tile];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const bool warp_active = warp * NDT < d_cnt;
    const int4 *geo_g = chunk_geo + (int64_t)tile * nchunks * CH;
    const int32_t *off_g = chunk_off + (int64_t)tile * nchunks * CH * DT;
    const int4 zero4 = make_int4(0, 0, 0, 0);

    if (threadIdx.x < NS) mbar_init(&mbar[threadIdx.x], 1);
    if (threadIdx.x == 0) fence_mbar_init();
    __syncthreads();

    auto issue = [&](int kk, int4 g) {  // warp 0; chunk kk into raw slot kk % NS
        const int sl = kk % NS;
        const int nc = min(CH, nchan - kk * CH);
        uint32_t bytes = (lane < nc) ? (uint32_t)g.y + 16u : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
        if (lane < CH) geo_s[sl * CH + lane] = (lane < nc) ? g : zero4;
        fence_proxy_async();
        if (lane == 0) mbar_arrive_expect_tx(&mbar[sl], bytes + (uint32_t)(CH * DT * 4));
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
    // Four shifted copies of this warp's channel of chunk kk, from raw slot
    // kk % NS into copies buffer kk & 1.
    auto build = [&](int kk) {
        const int sl = kk % NS;
        if (kk * CH + warp >= nchan) return;
        const int4 g = geo_s[sl * CH + warp];
        const int32_t R = g.y, S = g.y;
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
                *reinterpret_cast<uint4 *>(row + S + 16 * q) =
                    make_uint4(__byte_perm(a.x, a.y, 0x4321), __byte_perm(a.y, a.z, 0x4321),
                               __byte_perm(a.z, a.w, 0x4321), __byte_perm(a.w, e, 0x4321));
                *reinterpret_cast<uint4 *>(row + 2 * S + 16 * q) =
                    make_uint4(__byte_perm(a.x, a.y, 0x5432), __byte_perm(a.y, a.z, 0x5432),
                               __byte_perm(a.z, a.w, 0x5432), __byte_perm(a.w, e, 0x5432));
                *reinterpret_cast<uint4 *>(row + 3 * S + 16 * q) =
                    make_uint4(__byte_perm(a.x, a.y, 0x6543), __byte_perm(a.y, a.z, 0x6543),
                               __byte_perm(a.z, a.w, 0x6543), __byte_perm(a.w, e, 0x6543));
            }
        }
    };

    int4 g_next = zero4;  // warp 0: geometry of the next chunk to issue
    if (warp == 0) {
        const int4 g0 = load_geo(0), g1 = load_geo(1);
        g_next = load_geo(2);
        issue(0, g0);
        if (nchunks > 1) issue(1, g1);
    }
    __syncthreads();
    {
        const bool ok = mbar_wait_bounded(&mbar[0], 0u);
        if (ok) build(0);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(status, SP_STATUS_STAGING_TIMEOUT);
            return;
        }
    }

    int32_t acc[NDT][16];
#pragma unroll
    for (int i = 0; i < NDT; ++i)
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[i][j] = 0;

    for (int k = 0; k < nchunks; ++k) {
        const int b = k & 1;
        const int nc = min(CH, nchan - k * CH);
        if (warp == 0 && k + 2 < nchunks) {
            issue(k + 2, g_next);
            g_next = load_geo(k + 3);
        }
        if (warp_active) {
            const uint8_t *sb = cop_s + b * copies_max + lane * 4;
            const int32_t *ot = offt_s + (k % NS) * CH * DT + warp * NDT;
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
                        for (int q = 0; q < 4; ++q) {
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
                        for (int q = 0; q < 4; ++q) {
                            const uint32_t w = *reinterpret_cast<const uint32_t *>(sb + ac[i] + 128 * q);
                            add_quad(w, 0u, 0u, 0u, &acc[i][4 * q]);
                        }
                    }
                }
            }
        }
        bool ok = true;
        if (k + 1 < nchunks) {
            ok = mbar_wait_bounded(&mbar[(k + 1) % NS], (uint32_t)((k + 1) / NS) & 1u);
            if (ok) build(k + 1);
        }
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) atomicOr(status, SP_STATUS_STAGING_TIMEOUT);
            return;
        }
    }

    const bool vec = (n_out & 3) == 0;
#pragma unroll
    for (int i = 0; i < NDT; ++i) {
        const int dl = warp * NDT + i;
        if (dl >= d_cnt) continue;
        int32_t *orow = out + (int64_t)(d_first + dl) * n_out;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t t = t0 + 128 * q + 4 * lane;
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

using DedispKernel = void (*)(const uint8_t *, int64_t, int32_t, int32_t, const int32_t *, const int32_t *,
                              const int4 *, const int32_t *, int32_t, int32_t, int64_t, int32_t *, int32_t *);
constexpr DedispKernel kDedisp = dedisperse_kernel<kDedispDmPerThread, kDedispWarps, kDedispChanChunk>;



}  // namespace

int launch_stage_input(const uint8_t *d_in, int64_t n_in, int32_t nchan, uint8_t *d_staged, int64_t pitch,
                       cudaStream_t stream) {
    const dim3 grid((unsigned)(pitch / kStTime), (unsigned)((nchan + kStChan - 1) / kStChan));
    stage_input_kernel<<<grid, 256, 0, stream>>>(d_in, n_in, nchan, d_staged, pitch);
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int launch_dedisperse(const sp_plan *plan, const uint8_t *d_xt, int64_t pitch, int64_t n_out, int32_t *d_out,
                      cudaStream_t stream) {
    static int configured_smem[64] = {0};
    const int dev = plan->device < 64 ? plan->device : 63;
    if (configured_smem[dev] < plan->smem_bytes) {
        if (cudaFuncSetAttribute(kDedisp, cudaFuncAttributeMaxDynamicSharedMemorySize, plan->smem_bytes) !=
            cudaSuccess)
            return SP_ECUDA;
        configured_smem[dev] = plan->smem_bytes;
    }
    const int64_t ntime = (n_out + kDedispTimeTile - 1) / kDedispTimeTile;
    const dim3 grid((unsigned)plan->ntiles, (unsigned)ntime);
    kDedisp<<<grid, kDedispWarps * 32, plan->smem_bytes, stream>>>(
        d_xt, pitch, plan->nchan, plan->nchunks, plan->d_tile_first, plan->d_tile_count, plan->d_chunk_geo,
        plan->d_chunk_off, plan->copies_max, plan->raw_max, n_out, d_out, plan->d_status);
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

}  // namespace sp
