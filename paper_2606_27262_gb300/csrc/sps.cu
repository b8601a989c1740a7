// sps.cu -- boxcar matched-filter single-pulse search on sm_103a
// (arXiv 2606.27262, Sec. 3.1.2: boxcar templates of several trial widths as
// differences of a running cumulative sum, S/N against per-block statistics,
// a threshold, and a 3x3 peak filter in the DM-time plane).
//
// Kernels:
//   sps_stats_kernel   one CTA per (row, normalisation block): exact int64
//                      sum and sum of squares (16-byte loads), the 128-bit
//                      variance term, and per-width float coefficients of
//                      the S/N affine map.
//   sps_boxcar_kernel  one CTA per 14 rows x 256 samples (+1 halo row and
//                      sample on each side).  Stages prefix sums of the rows
//                      in shared memory (warp-shuffle scans), evaluates every
//                      width for every (row, sample), keeps the best, then
//                      applies the threshold and the 3x3 rule from the staged
//                      best-S/N tile and appends candidates with one atomic
//                      per warp.  A template switch writes the best-S/N map
//                      instead of candidates.
//
// S/N arithmetic.  For block b of row d with count n, sum Sx, sum of squares
// Sxx, let m0 = floor(Sx/n) and f = Sx/n - m0.  For a window sum S of width w
//   snr = (n*S - w*Sx) / (sqrt(w)*sqrt(n*Sxx - Sx^2))
//       = ((S - w*m0) - w*f) * inv_w,   inv_w = n / (sqrt(w)*sqrt(V)).
// x = S - w*m0 is an exact integer; only its conversion to float and one
// fused multiply-add round.  x is formed from 32-bit prefix sums with
// wrap-around arithmetic: the result is exact whenever |x| < 2^31, which the
// kernel proves per CTA from the staged values (|x| <= w * max|v - m0|);
// 8-bit beams of up to 8192 channels always qualify.  A CTA that cannot
// prove it evaluates the same formula in 64-bit integers instead.
#include <cmath>
#include <mutex>

#include "sp_internal.h"

namespace sp {
namespace {

struct WidthList {
    int32_t w[SP_MAX_WIDTHS];
    int32_t nw;
};

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) sps_stats_kernel(const int32_t *__restrict__ dmt, int64_t n_out,
                                                        int64_t norm_block, int64_t nblk, WidthList wl,
                                                        int32_t *__restrict__ m0_out,
                                                        float2 *__restrict__ coef_out) {
    __shared__ int64_t red1[8], red2[8];
    const int64_t b = blockIdx.x;
    const int64_t d = blockIdx.y;
    const int64_t lo = (nblk == 1) ? 0 : b * norm_block;
    const int64_t hi = (b == nblk - 1) ? n_out : (b + 1) * norm_block;
    const int32_t *row = dmt + d * n_out;
    int64_t s1 = 0, s2 = 0;
    // Scalar head up to a 16-byte boundary, 16-byte body, scalar tail.
    const int64_t head = min(hi, lo + (int64_t)((4 - (((uintptr_t)(row + lo) >> 2) & 3)) & 3));
    const int64_t nvec = (hi - head) / 4;
    for (int64_t t = lo + threadIdx.x; t < head; t += 256) {
        const int64_t x = __ldg(row + t);
        s1 += x;
        s2 += x * x;
    }
    const int4 *vrow = reinterpret_cast<const int4 *>(row + head);
    for (int64_t i = threadIdx.x; i < nvec; i += 256) {
        const int4 q = __ldg(vrow + i);
        const int64_t a = q.x, bb = q.y, c = q.z, e = q.w;
        s1 += a + bb + c + e;
        s2 += a * a + bb * bb + c * c + e * e;
    }
    for (int64_t t = head + 4 * nvec + threadIdx.x; t < hi; t += 256) {
        const int64_t x = __ldg(row + t);
        s1 += x;
        s2 += x * x;
    }
    s1 = warp_sum_i64(s1);
    s2 = warp_sum_i64(s2);
    if ((threadIdx.x & 31) == 0) {
        red1[threadIdx.x >> 5] = s1;
        red2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t S1 = 0, S2 = 0;
        for (int i = 0; i < 8; ++i) {
            S1 += red1[i];
            S2 += red2[i];
        }
        const int64_t n = hi - lo;
        int64_t m0 = S1 / n;
        if (S1 - m0 * n < 0) --m0;  // floor for negative sums
        const double frac = (double)(S1 - m0 * n) / (double)n;
        const __int128 var_n2 = (__int128)n * S2 - (__int128)S1 * S1;
        const double inv_sigma = var_n2 > 0 ? (double)n / sqrt((double)var_n2) : 0.0;
        const int64_t idx = d * nblk + b;
        m0_out[idx] = (int32_t)m0;
        for (int k = 0; k < wl.nw; ++k) {
            const double w = (double)wl.w[k];
            const double inv = inv_sigma / sqrt(w);
            coef_out[idx * wl.nw + k] = make_float2((float)inv, (float)(w * frac * inv));
        }
    }
}

constexpr int kBxT = 256;                 // output samples per CTA
constexpr int kBxRows = 16;               // staged rows: 14 interior + 2 halo
constexpr int kBxIn = kBxRows - 2;
constexpr int kBxTT = kBxT + 2;           // staged samples incl. halo
constexpr int kBxPerLane = (kBxTT + 31) / 32;

// Best S/N over the widths at staged sample ti of one row, from prefix sums
// P (uint32 wrap-around or int64).  cw[k] = w_k * m0 in the same type.
// Windows must end by staged index fit_end (exclusive).
template <typename PT>
__device__ __forceinline__ void best_over_widths(const PT *Pr, int ti, int fit_end, const WidthList &wl,
                                                 const PT *cw, const float2 *cf, float &best, int &kb) {
    const PT p0 = Pr[ti];
#pragma unroll
    for (int k = 0; k < SP_MAX_WIDTHS; ++k) {
        if (k >= wl.nw) break;
        const int w = wl.w[k];
        if (ti + w > fit_end) break;  // widths increase: no later one fits either
        const PT xs = Pr[ti + w] - p0 - cw[k];
        float xf;
        if constexpr (sizeof(PT) == 4)
            xf = (float)(int32_t)xs;  // exact value of x: |x| < 2^31 was checked
        else
            xf = (float)(int64_t)xs;
        const float s = fmaf(xf, cf[k].x, -cf[k].y);
        if (s > best) {
            best = s;
            kb = k;
        }
    }
}

// Phase 1 for one row: P[i] = sum_{j<i} v(tbase + j) for i in [0, LP], with
// staged indices outside [i_lo, i_hi) read as zero; also the min/max of the
// staged values.
template <typename PT>
__device__ __forceinline__ void prefix_row(const int32_t *__restrict__ row, int64_t tbase, int LP, int i_lo,
                                           int i_hi, PT *Pr, int32_t &vmin, int32_t &vmax) {
    const int lane = threadIdx.x & 31;
    if (lane == 0) Pr[0] = 0;
    PT carry = 0;
    for (int base = 0; base < LP; base += 32) {
        const int i = base + lane;
        int32_t x = 0;
        if (i >= i_lo && i < i_hi) {
            x = __ldg(row + (tbase + i));
            vmin = min(vmin, x);
            vmax = max(vmax, x);
        }
        PT v = (PT)x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const PT u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (i < LP) Pr[i + 1] = carry + v;
        carry += __shfl_sync(0xffffffffu, v, 31);
    }
}

// Phase 2 for one row: best S/N and width of every staged sample.
template <typename PT>
__device__ __forceinline__ void score_row(const PT *Pr, int d, int64_t tbase, int i_lo, int i_hi, int fit_end,
                                          const WidthList &wl, int64_t norm_block, int64_t nblk,
                                          const int32_t *__restrict__ m0s, const float2 *__restrict__ coefs,
                                          float *snr_row, int8_t *k_row) {
    const int lane = threadIdx.x & 31;
    const int ti0 = lane * kBxPerLane;
    int next_edge = -1;  // staged index where the next normalisation block starts
    PT cw[SP_MAX_WIDTHS];
    float2 cf[SP_MAX_WIDTHS];
#pragma unroll
    for (int k = 0; k < SP_MAX_WIDTHS; ++k) {
        cw[k] = 0;
        cf[k] = make_float2(0.f, 0.f);
    }
    for (int j = 0; j < kBxPerLane; ++j) {
        const int ti = ti0 + j;
        if (ti >= kBxTT) break;
        float best = -INFINITY;
        int kb = -1;
        if (ti >= i_lo && ti < i_hi) {
            if (ti >= next_edge) {
                const int64_t t = tbase + ti;
                int64_t b = (norm_block > 0) ? t / norm_block : 0;
                if (b > nblk - 1) b = nblk - 1;
                const int64_t edge = (b == nblk - 1) ? INT64_MAX : (b + 1) * norm_block;
                next_edge = (int)min(edge - tbase, (int64_t)INT32_MAX);
                const int64_t idx = (int64_t)d * nblk + b;
                const PT m0 = (PT)(int64_t)__ldg(m0s + idx);
#pragma unroll
                for (int k = 0; k < SP_MAX_WIDTHS; ++k) {
                    if (k < wl.nw) {
                        cw[k] = (PT)wl.w[k] * m0;
                        cf[k] = __ldg(coefs + idx * wl.nw + k);
                    }
                }
            }
            best_over_widths<PT>(Pr, ti, fit_end, wl, cw, cf, best, kb);
        }
        snr_row[ti] = best;
        k_row[ti] = (int8_t)kb;
    }
}

template <bool MAP>
__global__ void __launch_bounds__(256, 2)
sps_boxcar_kernel(const int32_t *__restrict__ dmt, int32_t ndm, int64_t n_out, WidthList wl, int32_t maxw,
                  float thr, int64_t norm_block, int64_t nblk, const int32_t *__restrict__ m0s,
                  const float2 *__restrict__ coefs, sp_cand *__restrict__ cands, int64_t cap,
                  unsigned long long *__restrict__ count, float *__restrict__ map_best,
                  int8_t *__restrict__ map_k) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int LP = kBxTT + maxw;  // prefix entries 0..LP
    float *snr_s = reinterpret_cast<float *>(smem + (size_t)kBxRows * (LP + 1) * 8);
    int8_t *k_s = reinterpret_cast<int8_t *>(snr_s + kBxRows * kBxTT);
    uint32_t *P32 = reinterpret_cast<uint32_t *>(smem);
    int64_t *P64 = reinterpret_cast<int64_t *>(smem);

    const int64_t t0 = (int64_t)blockIdx.x * kBxT;
    const int64_t tbase = t0 - 1;
    const int d0 = blockIdx.y * kBxIn;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Staged index i is sample tbase + i; samples exist for i in [i_lo, i_hi).
    const int i_lo = tbase < 0 ? (int)(-tbase) : 0;
    const int i_hi = (int)min((int64_t)LP, n_out - tbase);
    const int fit_end = (int)min(n_out - tbase, (int64_t)INT32_MAX);  // windows end by this index

    // Phase 1 in 32-bit wrap-around prefix sums, tracking the value range.
    // x = S - w*m0 is exact if maxw * max|v - m0| < 2^31 for every block
    // whose windows start in this tile; otherwise redo it in 64 bits.
    bool wide = false;
    for (int rr = 2 * warp; rr < 2 * warp + 2; ++rr) {
        const int d = d0 - 1 + rr;
        if (d < 0 || d >= ndm) continue;
        const int32_t *row = dmt + (int64_t)d * n_out;
        int32_t vmin = INT32_MAX, vmax = INT32_MIN;
        prefix_row<uint32_t>(row, tbase, LP, i_lo, i_hi, P32 + (size_t)rr * (LP + 1), vmin, vmax);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
            vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        }
        if (vmin > vmax) continue;
        const int64_t ts = tbase + i_lo, te = tbase + min(i_hi, kBxTT) - 1;
        int64_t bs = (norm_block > 0) ? ts / norm_block : 0, be = (norm_block > 0) ? te / norm_block : 0;
        bs = min(bs, nblk - 1);
        be = min(be, nblk - 1);
        for (int64_t b = bs + lane; b <= be; b += 32) {
            const int64_t m0 = __ldg(m0s + (int64_t)d * nblk + b);
            const int64_t dev = max((int64_t)vmax - m0, m0 - (int64_t)vmin);
            if (dev * maxw > (int64_t)INT32_MAX) wide = true;
        }
    }
    wide = __syncthreads_or(wide);
    if (wide) {
        for (int rr = 2 * warp; rr < 2 * warp + 2; ++rr) {
            const int d = d0 - 1 + rr;
            if (d < 0 || d >= ndm) continue;
            int32_t vmin = 0, vmax = 0;
            prefix_row<int64_t>(dmt + (int64_t)d * n_out, tbase, LP, i_lo, i_hi, P64 + (size_t)rr * (LP + 1),
                                vmin, vmax);
        }
    }
    __syncthreads();

    // Phase 2: best S/N over the widths for every staged (row, sample).
    for (int rr = 2 * warp; rr < 2 * warp + 2; ++rr) {
        const int d = d0 - 1 + rr;
        if (d < 0 || d >= ndm) {
            for (int ti = lane; ti < kBxTT; ti += 32) snr_s[rr * kBxTT + ti] = -INFINITY;
            continue;
        }
        if (wide)
            score_row<int64_t>(P64 + (size_t)rr * (LP + 1), d, tbase, i_lo, i_hi, fit_end, wl, norm_block, nblk,
                               m0s, coefs, snr_s + rr * kBxTT, k_s + rr * kBxTT);
        else
            score_row<uint32_t>(P32 + (size_t)rr * (LP + 1), d, tbase, i_lo, i_hi, fit_end, wl, norm_block,
                                nblk, m0s, coefs, snr_s + rr * kBxTT, k_s + rr * kBxTT);
    }
    __syncthreads();

    // Phase 3: interior points -- map output, or threshold + 3x3 + append.
    const int rows_in = min(kBxIn, ndm - d0);
    const int t_in = (int)min((int64_t)kBxT, n_out - t0);
    for (int idx = threadIdx.x; idx < kBxIn * kBxT; idx += 256) {
        const int r = idx / kBxT;
        const int tt = idx % kBxT;
        const int rr = 1 + r;
        const int ti = 1 + tt;
        const bool inr = r < rows_in && tt < t_in;
        const float v = snr_s[rr * kBxTT + ti];
        if (MAP) {
            if (inr) {
                const int64_t o = (int64_t)(d0 + r) * n_out + t0 + tt;
                map_best[o] = v;
                map_k[o] = k_s[rr * kBxTT + ti];
            }
        } else {
            bool cand = inr && v >= thr;
            if (cand) {
                const float *up = snr_s + (rr - 1) * kBxTT + ti;
                const float *mid = snr_s + rr * kBxTT + ti;
                const float *dn = snr_s + (rr + 1) * kBxTT + ti;
                cand = v > up[-1] && v > up[0] && v > up[1] && v > mid[-1] && v >= mid[1] && v >= dn[-1] &&
                       v >= dn[0] && v >= dn[1];
            }
            const unsigned mask = __ballot_sync(0xffffffffu, cand);
            if (mask) {
                const int leader = __ffs(mask) - 1;
                unsigned long long base = 0;
                if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (cand) {
                    const unsigned long long pos = base + __popc(mask & ((1u << lane) - 1u));
                    if ((int64_t)pos < cap) {
                        sp_cand c;
                        c.dm_idx = d0 + r;
                        c.t = (int32_t)(t0 + tt);
                        c.width_idx = k_s[rr * kBxTT + ti];
                        c.snr = v;
                        cands[pos] = c;
                    }
                }
            }
        }
    }
}

size_t boxcar_smem(int maxw) {
    return (size_t)kBxRows * (kBxTT + maxw + 1) * 8 + (size_t)kBxRows * kBxTT * 4 + (size_t)kBxRows * kBxTT;
}

}  // namespace

int64_t sps_nblocks(int64_t n_out, int64_t norm_block) {
    if (norm_block <= 0 || norm_block >= n_out) return 1;
    const int64_t nb = n_out / norm_block;
    return nb < 1 ? 1 : nb;
}

int64_t sps_workspace_bytes(int32_t ndm, int64_t n_out, int32_t nw, int64_t norm_block) {
    const int64_t nblk = sps_nblocks(n_out, norm_block);
    return align256((int64_t)ndm * nblk * 4) + align256((int64_t)ndm * nblk * nw * 8);
}

namespace {
std::mutex g_sps_lock;
size_t g_sps_smem[64][2] = {};  // configured boxcar shared memory per (device, kernel)

int configure_boxcar(bool map, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    if (dev < 0 || dev >= 64) return SP_ELIMIT;
    std::lock_guard<std::mutex> guard(g_sps_lock);
    if (g_sps_smem[dev][map] >= smem) return SP_OK;
    const cudaError_t e = map ? cudaFuncSetAttribute(sps_boxcar_kernel<true>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                              : cudaFuncSetAttribute(sps_boxcar_kernel<false>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    g_sps_smem[dev][map] = smem;
    return SP_OK;
}
}  // namespace

int sps_configure(int32_t maxw) {
    const size_t smem = boxcar_smem(maxw);
    int rc = configure_boxcar(false, smem);
    if (!rc) rc = configure_boxcar(true, smem);
    return rc;
}

int launch_sps(const SpsArgs &a, cudaStream_t stream) {
    WidthList wl;
    for (int k = 0; k < SP_MAX_WIDTHS; ++k) wl.w[k] = k < a.nw ? a.widths[k] : 0;
    wl.nw = a.nw;
    const int maxw = a.widths[a.nw - 1];
    int32_t *m0s = reinterpret_cast<int32_t *>(a.work);
    float2 *coefs = reinterpret_cast<float2 *>(reinterpret_cast<uint8_t *>(a.work) +
                                               align256((int64_t)a.ndm * a.nblk * 4));
    const size_t smem = boxcar_smem(maxw);
    const bool map = a.map_best != nullptr;
    int rc = configure_boxcar(map, smem);
    if (rc) return rc;
    sps_stats_kernel<<<dim3((unsigned)a.nblk, (unsigned)a.ndm), 256, 0, stream>>>(a.dmt, a.n_out, a.norm_block,
                                                                                a.nblk, wl, m0s, coefs);
    if (cudaGetLastError() != cudaSuccess) return SP_ECUDA;

    const dim3 grid((unsigned)((a.n_out + kBxT - 1) / kBxT), (unsigned)((a.ndm + kBxIn - 1) / kBxIn));
    if (map) {
        sps_boxcar_kernel<true><<<grid, 256, smem, stream>>>(a.dmt, a.ndm, a.n_out, wl, maxw, a.threshold,
                                                             a.norm_block, a.nblk, m0s, coefs, nullptr, 0,
                                                             nullptr, a.map_best, a.map_wbest);
    } else {
        if (cudaMemsetAsync(a.count, 0, sizeof(int64_t), stream) != cudaSuccess) return SP_ECUDA;
        sps_boxcar_kernel<false><<<grid, 256, smem, stream>>>(
            a.dmt, a.ndm, a.n_out, wl, maxw, a.threshold, a.norm_block, a.nblk, m0s, coefs, a.cands, a.cap,
            reinterpret_cast<unsigned long long *>(a.count), nullptr, nullptr);
    }
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

}  // namespace sp
