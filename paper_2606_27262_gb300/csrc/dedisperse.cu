// dedisperse.cu -- brute-force incoherent dedispersion on sm_103a
// (arXiv 2606.27262, Sec. 3.1.1: shift every channel by its Eq.-1 delay and
// sum, for every trial DM; the result is the DM transform).
//
//   out[d][t] = sum_c in[t + delay[d][c]][c]
//
// Two kernels:
//   transpose_u8_kernel  time-major [n_in][nchan] -> channel-major
//                        [nchan][pitch] (zero padded), so that one channel's
//                        time series is contiguous.
//   dedisperse_kernel    one CTA = 32 consecutive trial DMs (a "DM tile" from
//                        the plan) x 512 output samples.  For each chunk of
//                        16 channels it stages, per channel, the window of
//                        input samples that the tile's 32 delays reach
//                        (512 + delay spread + alignment slack) into shared
//                        memory as four copies shifted by 0..3 bytes, so that
//                        any 4 consecutive samples are one aligned 32-bit
//                        load.  One staged byte then serves up to 32 DMs.
//
// Arithmetic: the sum is a pure integer add of bytes (no tensor-core
// contraction exists here).  Each thread owns 4 DMs x 16 samples.  A loaded
// word (4 consecutive samples of one channel) is split into two words of two
// 16-bit lanes (even samples: AND 0x00FF00FF; odd samples: byte permute), and
// two channels are added per 3-input integer add, i.e. four byte-adds per
// instruction.  16-bit lanes hold at most 257 byte sums exactly, so every
// 256 channels the lanes are widened into 32-bit accumulators.  The result
// is exact and bit-identical to the definition.
#include <cstdio>

#include "sp_internal.h"

namespace sp {
namespace {

constexpr int kTrTime = 64;
constexpr int kTrChan = 64;

// 64 samples x 64 channels per CTA through shared memory.  Rows of the
// output beyond n_in (up to the pitch) are written as zeros.
__global__ void __launch_bounds__(256) transpose_u8_kernel(const uint8_t *__restrict__ in,
                                                           int64_t n_in, int32_t nchan,
                                                           uint8_t *__restrict__ xt,
                                                           int64_t pitch) {
    __shared__ __align__(16) uint8_t tile[kTrTime][kTrChan + 4];
    const int64_t t0 = (int64_t)blockIdx.x * kTrTime;
    const int c0 = blockIdx.y * kTrChan;
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
    {
        const int cc = threadIdx.x >> 2;
        const int tg = (threadIdx.x & 3) * 16;
        if (c0 + cc < nchan) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                w[q] = (uint32_t)tile[tg + 4 * q + 0][cc] | ((uint32_t)tile[tg + 4 * q + 1][cc] << 8) |
                       ((uint32_t)tile[tg + 4 * q + 2][cc] << 16) | ((uint32_t)tile[tg + 4 * q + 3][cc] << 24);
            }
            *reinterpret_cast<uint4 *>(xt + (int64_t)(c0 + cc) * pitch + t0 + tg) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Smem layout of one channel chunk: offset table [CH][DT] int32, then for
// each channel of the chunk four shifted copies of R_c bytes each.  Copy r,
// word j = staged bytes [4j + r, 4j + r + 4).
template <int NDT, int NWARP, int CH>
__global__ void __launch_bounds__(NWARP * 32, 2)
dedisperse_kernel(const uint8_t *__restrict__ xt, int64_t pitch, const int32_t *__restrict__ delays,
                  int32_t nchan, const int32_t *__restrict__ tile_first,
                  const int32_t *__restrict__ tile_count, const int32_t *__restrict__ tile_dlo,
                  const int32_t *__restrict__ tile_span, int64_t n_out, int32_t *__restrict__ out) {
    static_assert(NDT == 4, "offset table is read as int4 per thread");
    constexpr int DT = NDT * NWARP;
    constexpr int T = kDedispTimeTile;
    constexpr int NTHR = NWARP * 32;
    constexpr int THR_PER_CH = NTHR / CH;
    static_assert(T == 32 * 16, "a warp spans the time tile: 32 lanes x 16 samples");
    constexpr int kFlushChunks = 256 / CH;

    extern __shared__ __align__(16) uint8_t smem[];
    int32_t *offtab = reinterpret_cast<int32_t *>(smem);
    uint8_t *stage = smem + CH * DT * 4;
    __shared__ int64_t s_base[CH];
    __shared__ int32_t s_R[CH];
    __shared__ int32_t s_off[CH];

    const int tile = blockIdx.x;
    const int64_t t0 = (int64_t)blockIdx.y * T;
    const int d_first = tile_first[tile];
    const int d_cnt = tile_count[tile];
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const bool warp_active = warp * NDT < d_cnt;

    uint32_t acc16[NDT][4][2];
    int32_t acc32[NDT][16];
#pragma unroll
    for (int i = 0; i < NDT; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc16[i][k][0] = acc16[i][k][1] = 0u;
#pragma unroll
        for (int j = 0; j < 16; ++j) acc32[i][j] = 0;
    }

    int chunks_since_flush = 0;
    for (int c0 = 0; c0 < nchan; c0 += CH) {
        const int nc = min(CH, nchan - c0);
        if (threadIdx.x < CH) {
            const int c = threadIdx.x;
            int32_t R = 0;
            int64_t base = 0;
            if (c < nc) {
                const int64_t idx = (int64_t)tile * nchan + c0 + c;
                base = (t0 + tile_dlo[idx]) & ~int64_t(15);
                R = dedisp_row_bytes(tile_span[idx]);
            }
            s_base[c] = base;
            s_R[c] = R;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t acc = 0;
            for (int c = 0; c < CH; ++c) {
                s_off[c] = acc;
                acc += 4 * s_R[c];
            }
        }
        __syncthreads();
        // Offset of each (channel, DM) in the staged copies; DM slots past
        // the tile's count reuse the last valid DM (their sums are dropped).
        for (int i = threadIdx.x; i < CH * DT; i += NTHR) {
            const int c = i / DT;
            const int dl = i - c * DT;
            int32_t off = 0;
            if (c < nc) {
                const int dd = min(dl, d_cnt - 1);
                const int32_t dly = __ldg(delays + (int64_t)(d_first + dd) * nchan + c0 + c);
                const int32_t shift = (int32_t)(t0 + dly - s_base[c]);
                off = s_off[c] + (shift & 3) * s_R[c] + (shift & ~3);
            }
            offtab[i] = off;
        }
        // Stage: THR_PER_CH threads per channel, 16 input bytes per step.
        {
            const int c = threadIdx.x / THR_PER_CH;
            const int j = threadIdx.x - c * THR_PER_CH;
            if (c < nc) {
                const int32_t R = s_R[c];
                const uint8_t *src = xt + (int64_t)(c0 + c) * pitch + s_base[c];
                uint8_t *dst = stage + s_off[c];
                for (int q = j; q < R / 16; q += THR_PER_CH) {
                    const uint4 a = __ldg(reinterpret_cast<const uint4 *>(src + 16 * q));
                    const uint32_t e = __ldg(reinterpret_cast<const uint32_t *>(src + 16 * q + 16));
                    *reinterpret_cast<uint4 *>(dst + 16 * q) = a;
                    *reinterpret_cast<uint4 *>(dst + R + 16 * q) =
                        make_uint4(__byte_perm(a.x, a.y, 0x4321), __byte_perm(a.y, a.z, 0x4321),
                                   __byte_perm(a.z, a.w, 0x4321), __byte_perm(a.w, e, 0x4321));
                    *reinterpret_cast<uint4 *>(dst + 2 * R + 16 * q) =
                        make_uint4(__byte_perm(a.x, a.y, 0x5432), __byte_perm(a.y, a.z, 0x5432),
                                   __byte_perm(a.z, a.w, 0x5432), __byte_perm(a.w, e, 0x5432));
                    *reinterpret_cast<uint4 *>(dst + 3 * R + 16 * q) =
                        make_uint4(__byte_perm(a.x, a.y, 0x6543), __byte_perm(a.y, a.z, 0x6543),
                                   __byte_perm(a.z, a.w, 0x6543), __byte_perm(a.w, e, 0x6543));
                }
            }
        }
        __syncthreads();

        if (warp_active) {
            const uint8_t *sb = stage + lane * 4;
            const int32_t *ot = offtab + warp * NDT;
            int c = 0;
            for (; c + 1 < nc; c += 2) {
                const int4 oa = *reinterpret_cast<const int4 *>(ot + c * DT);
                const int4 ob = *reinterpret_cast<const int4 *>(ot + (c + 1) * DT);
                const int32_t oas[4] = {oa.x, oa.y, oa.z, oa.w};
                const int32_t obs[4] = {ob.x, ob.y, ob.z, ob.w};
#pragma unroll
                for (int i = 0; i < NDT; ++i) {
                    const uint8_t *pa = sb + oas[i];
                    const uint8_t *pb = sb + obs[i];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t wa = *reinterpret_cast<const uint32_t *>(pa + 128 * k);
                        const uint32_t wb = *reinterpret_cast<const uint32_t *>(pb + 128 * k);
                        acc16[i][k][0] += (wa & 0x00FF00FFu) + (wb & 0x00FF00FFu);
                        acc16[i][k][1] += __byte_perm(wa, 0u, 0x4341) + __byte_perm(wb, 0u, 0x4341);
                    }
                }
            }
            if (c < nc) {
                const int4 oa = *reinterpret_cast<const int4 *>(ot + c * DT);
                const int32_t oas[4] = {oa.x, oa.y, oa.z, oa.w};
#pragma unroll
                for (int i = 0; i < NDT; ++i) {
                    const uint8_t *pa = sb + oas[i];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t wa = *reinterpret_cast<const uint32_t *>(pa + 128 * k);
                        acc16[i][k][0] += wa & 0x00FF00FFu;
                        acc16[i][k][1] += __byte_perm(wa, 0u, 0x4341);
                    }
                }
            }
        }
        __syncthreads();

        if (++chunks_since_flush == kFlushChunks || c0 + CH >= nchan) {
            chunks_since_flush = 0;
#pragma unroll
            for (int i = 0; i < NDT; ++i) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t e = acc16[i][k][0], o = acc16[i][k][1];
                    acc32[i][4 * k + 0] += (int32_t)(e & 0xFFFFu);
                    acc32[i][4 * k + 2] += (int32_t)(e >> 16);
                    acc32[i][4 * k + 1] += (int32_t)(o & 0xFFFFu);
                    acc32[i][4 * k + 3] += (int32_t)(o >> 16);
                    acc16[i][k][0] = acc16[i][k][1] = 0u;
                }
            }
        }
    }

    const bool vec = (n_out & 3) == 0;
#pragma unroll
    for (int i = 0; i < NDT; ++i) {
        const int dl = warp * NDT + i;
        if (dl >= d_cnt) continue;
        int32_t *row = out + (int64_t)(d_first + dl) * n_out;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t t = t0 + 128 * k + 4 * lane;
            if (vec && t + 3 < n_out) {
                *reinterpret_cast<int4 *>(row + t) =
                    make_int4(acc32[i][4 * k], acc32[i][4 * k + 1], acc32[i][4 * k + 2], acc32[i][4 * k + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (t + j < n_out) row[t + j] = acc32[i][4 * k + j];
            }
        }
    }
}

using DedispKernel = void (*)(const uint8_t *, int64_t, const int32_t *, int32_t, const int32_t *,
                              const int32_t *, const int32_t *, const int32_t *, int64_t, int32_t *);
constexpr DedispKernel kDedisp = dedisperse_kernel<kDedispDmPerThread, kDedispWarps, kDedispChanChunk>;

}  // namespace

int launch_transpose(const uint8_t *d_in, int64_t n_in, int32_t nchan, uint8_t *d_xt, int64_t pitch,
                     cudaStream_t stream) {
    const dim3 grid((unsigned)(pitch / kTrTime), (unsigned)((nchan + kTrChan - 1) / kTrChan));
    transpose_u8_kernel<<<grid, 256, 0, stream>>>(d_in, n_in, nchan, d_xt, pitch);
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int launch_dedisperse(const sp_plan *plan, const uint8_t *d_xt, int64_t pitch, int64_t n_out,
                      int32_t *d_out, cudaStream_t stream) {
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
        d_xt, pitch, plan->d_delays, plan->nchan, plan->d_tile_first, plan->d_tile_count, plan->d_tile_dlo,
        plan->d_tile_span, n_out, d_out);
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

}  // namespace sp
