// sps.cu -- boxcar matched-filter single-pulse search on sm_103a
// (arXiv 2606.27262, Sec. 3.1.2: boxcar templates of several trial widths as
// differences of a running cumulative sum, S/N against per-block statistics,
// a threshold, and a 3x3 peak filter in the DM-time plane).
//
// Kernels:
//   sps_stats_kernel   one CTA per (row, normalisation block): exact sum
//                      (64-bit) and sum of squares (128-bit: int32 values
//                      near 2^31 square to 2^62 each), 16-byte loads.
//   sps_coef_kernel    one thread per (row, block): m0, the 128-bit
//                      variance term, the per-width float coefficients of the
//                      S/N affine map and the candidate pre-filter constants.
//   sps_stream_kernel  candidate search for power-of-two widths: one CTA per
//                      14 rows (+1 halo row on each side) and a segment of
//                      chunks of 256 samples, walked with a two-chunk ring of
//                      prefix sums per row; an integer pre-filter per point
//                      and width, the exact S/N where it passes, the
//                      threshold and the 3x3 peak filter, one atomic per warp
//                      for the candidate append.  Chunks it cannot prove
//                      exact in 32-bit float-convertible arithmetic, and the
//                      beam's last chunk(s), are listed for the tile kernel.
//   sps_boxcar_kernel  the tile kernel: one CTA per 14 rows x 256 samples
//                      (+1 halo row and sample on each side).  Stages prefix
//                      sums of the rows in shared memory (warp-shuffle scans),
//                      evaluates every width for every (row, sample), keeps
//                      the best, then applies the threshold and the 3x3 rule
//                      from the staged best-S/N tile.  A template switch
//                      writes the best-S/N map instead of candidates.  Runs
//                      as a grid (best-S/N map, width lists the streamed
//                      kernel does not take) or over a tile list
//                      (sps_boxcar_listed_kernel).
//   sps_boxcar_wide_kernel  the tile kernel in 64-bit prefix arithmetic over
//                      the tiles the 32-bit passes listed.
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

using u128 = unsigned __int128;

__device__ __forceinline__ u128 warp_sum_u128(u128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t lo = __shfl_xor_sync(0xffffffffu, (uint64_t)v, o);
        const uint64_t hi = __shfl_xor_sync(0xffffffffu, (uint64_t)(v >> 64), o);
        v += ((u128)hi << 64) | lo;
    }
    return v;
}

// x*x of an int32 is at most 2^62, so two squares add without overflow in
// 64 bits before they join the 128-bit sum.
__device__ __forceinline__ uint64_t sq2(int32_t a, int32_t b) {
    return (uint64_t)((int64_t)a * a) + (uint64_t)((int64_t)b * b);
}

// Block sums: one CTA per (row, block) streams the block once (16-byte
// loads, four in flight per thread) and writes its count's sum Sx (int64)
// and sum of squares Sxx (128-bit, as two 64-bit words).
struct BlockSums {
    int64_t s1;
    uint64_t s2_lo, s2_hi;
};

__global__ void __launch_bounds__(256) sps_stats_kernel(const int32_t *__restrict__ dmt, int64_t n_out,
                                                        int64_t norm_block, int64_t nblk,
                                                        BlockSums *__restrict__ sums) {
    __shared__ int64_t red1[8];
    __shared__ u128 red2[8];
    const int64_t b = blockIdx.x;
    const int64_t d = blockIdx.y;
    const int64_t lo = (nblk == 1) ? 0 : b * norm_block;
    const int64_t hi = (b == nblk - 1) ? n_out : (b + 1) * norm_block;
    const int32_t *row = dmt + d * n_out;
    int64_t s1 = 0;
    u128 s2 = 0;
    // Scalar head up to a 16-byte boundary, 16-byte body, scalar tail.
    const int64_t head = min(hi, lo + (int64_t)((4 - (((uintptr_t)(row + lo) >> 2) & 3)) & 3));
    const int64_t nvec = (hi - head) / 4;
    for (int64_t t = lo + threadIdx.x; t < head; t += 256) {
        const int32_t x = __ldg(row + t);
        s1 += x;
        s2 += sq2(x, 0);
    }
    const int4 *vrow = reinterpret_cast<const int4 *>(row + head);
#pragma unroll 4
    for (int64_t i = threadIdx.x; i < nvec; i += 256) {  // four 16-byte loads in flight per thread
        const int4 q = __ldg(vrow + i);
        s1 += (int64_t)q.x + q.y + (int64_t)q.z + q.w;
        s2 += sq2(q.x, q.y);
        s2 += sq2(q.z, q.w);
    }
    for (int64_t t = head + 4 * nvec + threadIdx.x; t < hi; t += 256) {
        const int32_t x = __ldg(row + t);
        s1 += x;
        s2 += sq2(x, 0);
    }
    s1 = warp_sum_i64(s1);
    s2 = warp_sum_u128(s2);
    if ((threadIdx.x & 31) == 0) {
        red1[threadIdx.x >> 5] = s1;
        red2[threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t S1 = 0;
        u128 S2 = 0;
        for (int i = 0; i < 8; ++i) {
            S1 += red1[i];
            S2 += red2[i];
        }
        BlockSums o;
        o.s1 = S1;
        o.s2_lo = (uint64_t)S2;
        o.s2_hi = (uint64_t)(S2 >> 64);
        sums[d * nblk + b] = o;
    }
}

// sqrt(w) and 1/sqrt(w) of each width, in double (computed on the host).
struct WidthRoots {
    double sw[SP_MAX_WIDTHS], rsw[SP_MAX_WIDTHS];
};

// Pre-filter bound of the streamed candidate search: an integer X such that
// every window with x = S - w*m0 < X has an S/N below thr in the search's
// float arithmetic (snr = fmaf((float)x, cx, -cy), one rounding), also after
// the search clears the low four mantissa bits of a negative S/N (which
// raises it by less than 2^-19 of its size): thr is lowered by 2^-15 of its
// size (and 2^-100), multiplied by rcx, a reciprocal of cx to within 2^-23
// relative (so the quotient is within 1/2 of (t + cy)/cx where that is below
// 2^23 in magnitude), rounded down and lowered by two more.  Clamped to
// [-2^30, 2^30]: -2^30 lets every window through, 2^30 none (the search's |x|
// stays below 2^22, so an error in a bound beyond 2^23 decides nothing).
__device__ int32_t prefilter_bound(float thr, float cx, float cy, double rcx) {
    constexpr double kLim = 1073741824.0;
    if (thr != thr) return (int32_t)kLim;                      // NaN: nothing reaches it
    if (isinf(thr)) return thr > 0.0f ? (int32_t)kLim : -(int32_t)kLim;
    if (!(cx > 0.0f)) return thr <= 0.0f ? -(int32_t)kLim : (int32_t)kLim;  // zero variance: snr = 0
    const double t = (double)thr - fabs((double)thr) * 0x1p-15 - 0x1p-100;
    const double x = floor((t + (double)cy) * rcx) - 2.0;
    if (!(x > -kLim)) return -(int32_t)kLim;
    if (x >= kLim) return (int32_t)kLim;
    return (int32_t)x;
}

// Per (row, block), one thread each: m0 = floor(Sx/n), f = Sx/n - m0, the
// per-width float coefficients of the S/N affine map (inv = n/(sqrt(w)
// sqrt(V)), bias = w f inv) and the pre-filter constants w*m0 + X (32-bit
// wrap-around: the search subtracts them from a window's prefix difference
// to get x - X exactly).  The double arithmetic runs here, spread over
// threads, not at the end of every reduction CTA.
__global__ void __launch_bounds__(256) sps_coef_kernel(const BlockSums *__restrict__ sums, int64_t nrb,
                                                       int64_t n_out, int64_t norm_block, int64_t nblk,
                                                       WidthList wl, WidthRoots wr, float thr,
                                                       int32_t *__restrict__ m0_out, float2 *__restrict__ coef_out,
                                                       uint32_t *__restrict__ cthr_out) {
    const int64_t idx = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (idx >= nrb) return;
    const int64_t b = idx % nblk;
    const int64_t lo = (nblk == 1) ? 0 : b * norm_block;
    const int64_t hi = (b == nblk - 1) ? n_out : (b + 1) * norm_block;
    const int64_t n = hi - lo;
    const BlockSums sm = sums[idx];
    const int64_t S1 = sm.s1;
    const u128 S2 = ((u128)sm.s2_hi << 64) | sm.s2_lo;
    int64_t m0 = S1 / n;
    if (S1 - m0 * n < 0) --m0;  // floor for negative sums
    const double rn = 1.0 / (double)n;
    const double frac = (double)(S1 - m0 * n) * rn;
    // n <= 2^31 and S2 <= n * 2^62: the product stays below 2^124.
    const __int128 var_n2 = (__int128)n * (__int128)S2 - (__int128)S1 * S1;
    const double sq = var_n2 > 0 ? sqrt((double)var_n2) : 0.0;
    const double inv_sigma = var_n2 > 0 ? (double)n / sq : 0.0;
    const double sig_n = sq * rn;
    m0_out[idx] = (int32_t)m0;
    for (int k = 0; k < wl.nw; ++k) {
        const double w = (double)wl.w[k];
        const double inv = inv_sigma * wr.rsw[k];
        const float cx = (float)inv, cy = (float)(w * frac * inv);
        coef_out[idx * wl.nw + k] = make_float2(cx, cy);
        cthr_out[idx * wl.nw + k] =
            (uint32_t)wl.w[k] * (uint32_t)m0 + (uint32_t)prefilter_bound(thr, cx, cy, wr.sw[k] * sig_n);
    }
}

constexpr int kBxT = 256;                 // interior output samples per CTA
constexpr int kBxRows = 16;               // staged rows: 14 interior + 2 halo
constexpr int kBxIn = kBxRows - 2;
constexpr int kBxPts = kBxT + 2;          // scored points per row: samples t0-1 .. t0+256
constexpr int kBxOrg = 4;                 // staged index 0 = sample t0 - 4 (16-byte aligned rows)
constexpr int kBxFirst = kBxOrg - 1;      // staged index of point 0 (sample t0 - 1)
constexpr int kBxPass = 8;                // points per thread and pass (16 threads per row)

// Entries of the inclusive prefix Q of one staged row: point i's windows
// [i, i + w) need Q[i + w - 1] - Q[i - 1], up to i = kBxFirst + kBxPts - 1.
__host__ __device__ inline int boxcar_nq(int maxw) { return ((kBxFirst + kBxPts + maxw - 1 + 15) / 16) * 16; }

template <typename PT>
__host__ __device__ inline size_t boxcar_smem_t(int maxw) {
    return (size_t)kBxRows * boxcar_nq(maxw) * sizeof(PT) + (size_t)kBxRows * kBxPts * 4 + (size_t)kBxRows * kBxPts;
}

// Phase 1 for the two rows of one warp: Q[i] = sum_{j <= i} v(s0 + j) for
// the staged indices i < nq of each row, values outside [0, n_out) (and
// rows that are absent: row == nullptr) read as 0; also the min and max of
// each row's values.  Chunks of 512 entries: 16 values per lane (four
// 16-byte loads when rows are 16-byte aligned), both rows' loads issued
// before either is scanned, an in-register scan, then a warp scan of the
// lane totals; a last chunk of at most 16 entries is scanned by the 16
// lanes of a half-warp per row.
__device__ __forceinline__ void load_run16(const int32_t *__restrict__ row, int64_t t, int64_t n_out, bool vec,
                                           bool active, int32_t (&v)[16], int32_t &vmin, int32_t &vmax) {
    if (row && active && vec && t >= 0 && t + 16 <= n_out) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int4 x = __ldg(reinterpret_cast<const int4 *>(row + t) + q);
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            vmin = min(vmin, v[e]);
            vmax = max(vmax, v[e]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            v[e] = 0;
            if (row && active && t + e >= 0 && t + e < n_out) {
                v[e] = __ldg(row + t + e);
                vmin = min(vmin, v[e]);
                vmax = max(vmax, v[e]);
            }
        }
    }
}

template <typename PT>
__device__ __forceinline__ void scan_run16(const int32_t (&v)[16], bool active, int base, PT *Q, PT &carry) {
    const int lane = threadIdx.x & 31;
    PT r[16];
    PT acc = 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        acc += (PT)v[e];
        r[e] = acc;
    }
    PT incl = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const PT u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    const PT off = carry + incl - acc;
    if (active) {
#pragma unroll
        for (int e = 0; e < 16; ++e) Q[base + e] = off + r[e];
    }
    carry += __shfl_sync(0xffffffffu, incl, 31);
}

template <typename PT>
__device__ __forceinline__ void prefix_rows2(const int32_t *__restrict__ rowA, const int32_t *__restrict__ rowB,
                                             int64_t s0, int64_t n_out, bool vec, int nq, PT *QA, PT *QB,
                                             int32_t &minA, int32_t &maxA, int32_t &minB, int32_t &maxB) {
    const int lane = threadIdx.x & 31;
    PT carryA = 0, carryB = 0;
    for (int base0 = 0; base0 < nq; base0 += 512) {
        if (nq - base0 <= 16) {  // last short chunk: lanes 0-15 row A, 16-31 row B
            const bool isA = lane < 16;
            const int e = lane & 15;
            const int32_t *row = isA ? rowA : rowB;
            const int64_t t = s0 + base0 + e;
            const bool in = row != nullptr && e < nq - base0;
            int32_t x = 0;
            if (in && t >= 0 && t < n_out) {
                x = __ldg(row + t);
                if (isA) {
                    minA = min(minA, x);
                    maxA = max(maxA, x);
                } else {
                    minB = min(minB, x);
                    maxB = max(maxB, x);
                }
            }
            PT incl = (PT)x;
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
                const PT u = __shfl_up_sync(0xffffffffu, incl, o, 16);
                if (e >= o) incl += u;
            }
            if (in) (isA ? QA : QB)[base0 + e] = (isA ? carryA : carryB) + incl;
            break;
        }
        const int base = base0 + lane * 16;
        const bool active = base < nq;
        const int64_t t = s0 + base;
        int32_t vA[16], vB[16];
        load_run16(rowA, t, n_out, vec, active, vA, minA, maxA);
        load_run16(rowB, t, n_out, vec, active, vB, minB, maxB);
        if (rowA) scan_run16<PT>(vA, active, base, QA, carryA);
        if (rowB) scan_run16<PT>(vB, active, base, QB, carryB);
    }
}

// Normalisation block of sample t >= 0 (32-bit division when both fit).
__device__ __forceinline__ int64_t block_of(int64_t t, int64_t norm_block, int64_t nblk) {
    int64_t b;
    if (norm_block <= 0)
        b = 0;
    else if (t <= INT32_MAX && norm_block <= INT32_MAX)
        b = (int64_t)((uint32_t)t / (uint32_t)norm_block);
    else
        b = t / norm_block;
    return b > nblk - 1 ? nblk - 1 : b;
}

// Phase 2 for the points p = p0 + 16 j, j < NP (those with p < kBxPts), of
// one staged row: best S/N over the widths and its width index.
// `interior`: every point of the tile is a sample of the beam; `tile_block`:
// the one normalisation block of all of them, or -1.
// MAGIC (32-bit pass, every |S - w*m0| of the tile below 2^22): the
// integer converts to float by adding the bit pattern of 1.5*2^23 and
// subtracting that float (exact below 2^22), and on the check-free path the
// best width is kept with one float max: the width code 15 - k sits in the
// low 4 mantissa bits of the S/N (on equal upper bits the smaller width
// wins), cleared again when the point is stored.  The S/N keeps 19 bits:
// within 2^-19 relative of the value the exact compare would keep.
constexpr uint32_t kMagicBits = 0x4B400000u;   // bit pattern of 12582912.0f = 1.5 * 2^23
constexpr float kMagicValue = 12582912.0f;

template <typename PT, int NP, bool MAGIC>
__device__ __forceinline__ void score_points(const PT *Q, int d, int64_t s0, int64_t n_out, int fit_end, int p0,
                                             bool interior, int64_t tile_block, const WidthList &wl,
                                             int64_t norm_block, int64_t nblk, const int32_t *__restrict__ m0s,
                                             const float2 *__restrict__ coefs, float *snr_row, int8_t *k_row) {
    float best[NP];
    int kb[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        best[j] = -INFINITY;
        kb[j] = -1;
    }
    // valid points: p < kBxPts and sample t in [0, n_out)
    int jlo = NP, jhi = -1;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int p = p0 + 16 * j;
        const int64_t t = s0 + kBxFirst + p;
        if (p < kBxPts && (interior || (t >= 0 && t < n_out))) {
            jlo = min(jlo, j);
            jhi = max(jhi, j);
        }
    }
    if (jhi >= 0) {
        const int64_t t_lo = s0 + kBxFirst + p0 + 16 * jlo, t_hi = s0 + kBxFirst + p0 + 16 * jhi;
        const int64_t b_lo = tile_block >= 0 ? tile_block : block_of(t_lo, norm_block, nblk);
        const int64_t b_hi = tile_block >= 0 ? tile_block : block_of(t_hi, norm_block, nblk);
        const int64_t row_blk = (int64_t)d * nblk;
        const int i_last = kBxFirst + p0 + 16 * jhi;
        if (b_lo == b_hi && jlo == 0 && jhi == NP - 1 && i_last + wl.w[wl.nw - 1] <= fit_end) {
            // every point valid, every window inside the beam, one block
            const PT m0 = (PT)(int64_t)__ldg(m0s + row_blk + b_lo);
            const float2 *cfs = coefs + (row_blk + b_lo) * wl.nw;
            PT q0[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) q0[j] = Q[kBxFirst + p0 + 16 * j - 1];
            if constexpr (MAGIC) {
                for (int k = 0; k < wl.nw; ++k) {
                    const int w = wl.w[k];
                    const uint32_t mc = kMagicBits - (uint32_t)w * (uint32_t)m0;
                    const float2 cf = __ldg(cfs + k);
                    const PT *Qw = Q + kBxFirst + p0 + w - 1;
                    const uint32_t code = 15u - (uint32_t)k;
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        const uint32_t xs = (uint32_t)Qw[16 * j] - (uint32_t)q0[j] + mc;
                        const float sv = fmaf(__uint_as_float(xs) - kMagicValue, cf.x, -cf.y);
                        best[j] = fmaxf(best[j], __uint_as_float((__float_as_uint(sv) & ~15u) | code));
                    }
                }
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const uint32_t bits = __float_as_uint(best[j]);
                    kb[j] = 15 - (int)(bits & 15u);
                    best[j] = __uint_as_float(bits & ~15u);
                }
            } else {
                for (int k = 0; k < wl.nw; ++k) {
                    const int w = wl.w[k];
                    const PT cw = (PT)w * m0;
                    const float2 cf = __ldg(cfs + k);
                    const PT *Qw = Q + kBxFirst + p0 + w - 1;
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        const PT xs = Qw[16 * j] - q0[j] - cw;
                        const float xf = sizeof(PT) == 4 ? (float)(int32_t)xs : (float)(int64_t)xs;
                        const float sv = fmaf(xf, cf.x, -cf.y);
                        if (sv > best[j]) {
                            best[j] = sv;
                            kb[j] = k;
                        }
                    }
                }
            }
        } else if (b_lo == b_hi) {  // one normalisation block: coefficients once per width
            const PT m0 = (PT)(int64_t)__ldg(m0s + row_blk + b_lo);
            for (int k = 0; k < wl.nw; ++k) {
                const int w = wl.w[k];
                const PT cw = (PT)w * m0;
                const float2 cf = __ldg(coefs + (row_blk + b_lo) * wl.nw + k);
                bool any = false;
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const int i = kBxFirst + p0 + 16 * j;
                    if (j < jlo || j > jhi || i + w > fit_end) continue;
                    any = true;
                    const PT xs = Q[i + w - 1] - Q[i - 1] - cw;
                    const float xf = sizeof(PT) == 4 ? (float)(int32_t)xs : (float)(int64_t)xs;
                    const float sv = fmaf(xf, cf.x, -cf.y);
                    if (sv > best[j]) {
                        best[j] = sv;
                        kb[j] = k;
                    }
                }
                if (!any) break;  // widths increase: no later one fits either
            }
        } else {  // points in several blocks
            for (int k = 0; k < wl.nw; ++k) {
                const int w = wl.w[k];
                bool any = false;
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    const int i = kBxFirst + p0 + 16 * j;
                    if (j < jlo || j > jhi || i + w > fit_end) continue;
                    any = true;
                    const int64_t b = block_of(s0 + i, norm_block, nblk);
                    const PT cw = (PT)w * (PT)(int64_t)__ldg(m0s + row_blk + b);
                    const float2 cf = __ldg(coefs + (row_blk + b) * wl.nw + k);
                    const PT xs = Q[i + w - 1] - Q[i - 1] - cw;
                    const float xf = sizeof(PT) == 4 ? (float)(int32_t)xs : (float)(int64_t)xs;
                    const float sv = fmaf(xf, cf.x, -cf.y);
                    if (sv > best[j]) {
                        best[j] = sv;
                        kb[j] = k;
                    }
                }
                if (!any) break;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        const int p = p0 + 16 * j;
        if (p < kBxPts) {
            snr_row[p] = best[j];
            k_row[p] = (int8_t)kb[j];
        }
    }
}

struct BoxcarArgs {
    const int32_t *dmt;
    int32_t ndm;
    int64_t n_out;
    WidthList wl;
    int32_t maxw;
    float thr;
    int64_t norm_block, nblk;
    const int32_t *m0s;
    const float2 *coefs;
    sp_cand *cands;
    int64_t cap;
    unsigned long long *count;
    float *map_best;
    int8_t *map_k;
    int *wide_count;  // tiles the 32-bit pass could not prove exact
    int2 *wide_list;
    bool vec;         // rows 16-byte aligned: 16-byte loads
    // Streamed search: chunks [0, n_fast) of every row group, pre-filter
    // constants w*m0 + X per (row, block, width), and the tiles it leaves
    // to the tile kernel.
    int32_t n_fast;
    const uint32_t *cthr;
    int *slow_count;
    int2 *slow_list;
};

// One tile (14 rows x 256 samples + halo).  PT = uint32: prefix sums in
// 32-bit wrap-around arithmetic; returns false (uniformly) without writing
// anything when a window sum might not fit in 32 bits.  PT = int64: always
// exact.
template <typename PT, bool MAP>
__device__ __forceinline__ bool boxcar_tile(const BoxcarArgs &a, int tx, int ty, uint8_t *smem) {
    const int nq = boxcar_nq(a.maxw);
    PT *Qs = reinterpret_cast<PT *>(smem);
    float *snr_s = reinterpret_cast<float *>(smem + (size_t)kBxRows * nq * sizeof(PT));
    int8_t *k_s = reinterpret_cast<int8_t *>(snr_s + kBxRows * kBxPts);
    const int64_t t0 = (int64_t)tx * kBxT;
    const int64_t s0 = t0 - kBxOrg;
    const int d0 = ty * kBxIn;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool vec = a.vec;
    const int fit_end = (int)min(a.n_out - s0, (int64_t)INT32_MAX);
    // The tile's scored samples [ts, te] inside the beam and their blocks.
    const int64_t ts = max(s0 + kBxFirst, (int64_t)0), te = min(s0 + kBxFirst + kBxPts, a.n_out) - 1;
    const bool interior = s0 + kBxFirst >= 0 && s0 + kBxFirst + kBxPts <= a.n_out;
    const int64_t bs = ts <= te ? block_of(ts, a.norm_block, a.nblk) : 0;
    const int64_t be = ts <= te ? block_of(te, a.norm_block, a.nblk) : -1;
    const int64_t tile_block = bs == be ? bs : -1;

    bool wide = false, big = sizeof(PT) != 4;
    {
        const int dA = d0 - 1 + 2 * warp, dB = dA + 1;
        const bool okA = dA >= 0 && dA < a.ndm, okB = dB >= 0 && dB < a.ndm;
        int32_t mn[2] = {INT32_MAX, INT32_MAX}, mx[2] = {INT32_MIN, INT32_MIN};
        prefix_rows2<PT>(okA ? a.dmt + (int64_t)dA * a.n_out : nullptr, okB ? a.dmt + (int64_t)dB * a.n_out : nullptr,
                         s0, a.n_out, vec, nq, Qs + (size_t)(2 * warp) * nq, Qs + (size_t)(2 * warp + 1) * nq, mn[0],
                         mx[0], mn[1], mx[1]);
        if (sizeof(PT) == 4) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int d = dA + h;
                int32_t vmin = mn[h], vmax = mx[h];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vmin = min(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
                    vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
                }
                if ((h ? okB : okA) && vmin <= vmax && ts <= te) {
                    for (int64_t b = bs + lane; b <= be; b += 32) {
                        const int64_t m0 = __ldg(a.m0s + (int64_t)d * a.nblk + b);
                        const int64_t dev = max((int64_t)vmax - m0, m0 - (int64_t)vmin);
                        if (dev * a.maxw > (int64_t)INT32_MAX) wide = true;
                        if (dev * a.maxw >= (int64_t)(1 << 22)) big = true;
                    }
                }
            }
        }
    }
    if (__syncthreads_or(wide)) return false;
    const bool magic = !__syncthreads_or(big);

    {
        const int rr = threadIdx.x >> 4, l = threadIdx.x & 15;
        const int d = d0 - 1 + rr;
        float *srow = snr_s + rr * kBxPts;
        int8_t *krow = k_s + rr * kBxPts;
        if (d < 0 || d >= a.ndm) {
            for (int p = l; p < kBxPts; p += 16) {
                srow[p] = -INFINITY;
                krow[p] = -1;
            }
        } else {
            const PT *Q = Qs + (size_t)rr * nq;
            // points l + 16 j: two passes of eight over p < 256
            if (sizeof(PT) == 4 && magic) {
                score_points<PT, kBxPass, true>(Q, d, s0, a.n_out, fit_end, l, interior, tile_block, a.wl,
                                                a.norm_block, a.nblk, a.m0s, a.coefs, srow, krow);
                score_points<PT, kBxPass, true>(Q, d, s0, a.n_out, fit_end, l + 16 * kBxPass, interior, tile_block,
                                                a.wl, a.norm_block, a.nblk, a.m0s, a.coefs, srow, krow);
            } else {
                score_points<PT, kBxPass, false>(Q, d, s0, a.n_out, fit_end, l, interior, tile_block, a.wl,
                                                 a.norm_block, a.nblk, a.m0s, a.coefs, srow, krow);
                score_points<PT, kBxPass, false>(Q, d, s0, a.n_out, fit_end, l + 16 * kBxPass, interior, tile_block,
                                                 a.wl, a.norm_block, a.nblk, a.m0s, a.coefs, srow, krow);
            }
        }
        // The last two points (256, 257) of all 16 rows: one warp, one point
        // per lane, instead of two threads in each row's half-warp.
        static_assert(kBxPts - 32 * kBxPass == 2 && kBxRows * 2 == 32, "one tail point per lane of one warp");
        if (threadIdx.x < 32) {
            const int tr = threadIdx.x >> 1, tp = 32 * kBxPass + (threadIdx.x & 1);
            const int td = d0 - 1 + tr;
            float *tsrow = snr_s + tr * kBxPts;
            int8_t *tkrow = k_s + tr * kBxPts;
            if (td < 0 || td >= a.ndm) {
                tsrow[tp] = -INFINITY;
                tkrow[tp] = -1;
            } else if (sizeof(PT) == 4 && magic) {
                score_points<PT, 1, true>(Qs + (size_t)tr * nq, td, s0, a.n_out, fit_end, tp, interior, tile_block,
                                          a.wl, a.norm_block, a.nblk, a.m0s, a.coefs, tsrow, tkrow);
            } else {
                score_points<PT, 1, false>(Qs + (size_t)tr * nq, td, s0, a.n_out, fit_end, tp, interior, tile_block,
                                           a.wl, a.norm_block, a.nblk, a.m0s, a.coefs, tsrow, tkrow);
            }
        }
    }
    __syncthreads();

    // Phase 3: interior points -- map output, or threshold + 3x3 + append.
    const int rows_in = min(kBxIn, a.ndm - d0);
    const int t_in = (int)min((int64_t)kBxT, a.n_out - t0);
    for (int idx = threadIdx.x; idx < kBxIn * kBxT; idx += blockDim.x) {
        const int r = idx / kBxT;
        const int tt = idx % kBxT;
        const int rr = 1 + r;
        const int ti = 1 + tt;
        const bool inr = r < rows_in && tt < t_in;
        const float v = snr_s[rr * kBxPts + ti];
        if (MAP) {
            if (inr) {
                const int64_t o = (int64_t)(d0 + r) * a.n_out + t0 + tt;
                a.map_best[o] = v;
                a.map_k[o] = k_s[rr * kBxPts + ti];
            }
        } else {
            bool cand = inr && v >= a.thr;
            if (cand) {
                const float *up = snr_s + (rr - 1) * kBxPts + ti;
                const float *mid = snr_s + rr * kBxPts + ti;
                const float *dn = snr_s + (rr + 1) * kBxPts + ti;
                cand = v > up[-1] && v > up[0] && v > up[1] && v > mid[-1] && v >= mid[1] && v >= dn[-1] &&
                       v >= dn[0] && v >= dn[1];
            }
            const unsigned mask = __ballot_sync(0xffffffffu, cand);
            if (mask) {
                const int leader = __ffs(mask) - 1;
                unsigned long long basec = 0;
                if (lane == leader) basec = atomicAdd(a.count, (unsigned long long)__popc(mask));
                basec = __shfl_sync(0xffffffffu, basec, leader);
                if (cand) {
                    const unsigned long long pos = basec + __popc(mask & ((1u << lane) - 1u));
                    if ((int64_t)pos < a.cap) {
                        sp_cand c;
                        c.dm_idx = d0 + r;
                        c.t = (int32_t)(t0 + tt);
                        c.width_idx = k_s[rr * kBxPts + ti];
                        c.snr = v;
                        a.cands[pos] = c;
                    }
                }
            }
        }
    }
    return true;
}

// Fast pass: every tile in 32-bit prefix arithmetic; a tile that cannot
// prove its window sums exact is listed for the 64-bit pass.
template <bool MAP>
__global__ void __launch_bounds__(256, 4) sps_boxcar_kernel(BoxcarArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    if (!boxcar_tile<uint32_t, MAP>(a, blockIdx.x, blockIdx.y, smem) && threadIdx.x == 0) {
        const int slot = atomicAdd(a.wide_count, 1);
        a.wide_list[slot] = make_int2(blockIdx.x, blockIdx.y);
    }
}

// The tiles the streamed search listed (the beam's last chunk(s) of every
// row group and the chunks it could not prove exact in 2^22), in the 32-bit
// tile kernel (persistent grid); a tile it cannot prove exact goes on to the
// 64-bit pass.
__global__ void __launch_bounds__(256, 4) sps_boxcar_listed_kernel(BoxcarArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int n = *a.slow_count;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int2 tile = a.slow_list[i];
        if (!boxcar_tile<uint32_t, false>(a, tile.x, tile.y, smem) && threadIdx.x == 0) {
            const int slot = atomicAdd(a.wide_count, 1);
            a.wide_list[slot] = tile;
        }
        __syncthreads();
    }
}

// Exact pass over the listed tiles, 64-bit prefix sums (persistent grid).
template <bool MAP>
__global__ void __launch_bounds__(256, 1) sps_boxcar_wide_kernel(BoxcarArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int n = *a.wide_count;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int2 tile = a.wide_list[i];
        boxcar_tile<int64_t, MAP>(a, tile.x, tile.y, smem);
        __syncthreads();
    }
}

// Streamed candidate search (3x3 peaks).  One CTA per 14 DM rows (+1 halo
// row on each side) and a segment of kStSeg chunks of 256 samples, walked
// chunk by chunk.  Per staged row the CTA keeps the exclusive prefix sums
// R[t] = sum_{s < t} v(s) of two consecutive chunks in a ring of 512 entries
// (R[t] at t mod 512; the sums start at the segment's first sample, which
// cancels in every difference), so each sample is loaded and scanned once.
// The window sum of point t and width w is R[t + w] - R[t].
//
// Pre-filter: with C_w = w*m0 + X_w (X_w from prefilter_bound, per row,
// block and width), max_w (R[t + w] - R[t] - C_w) < 0 shows that no width of
// point t reaches the threshold; its S/N is recorded as -inf, which leaves
// every 3x3 decision as it was (a candidate is at or above the threshold, so
// it is above a neighbour that is below it, whatever that neighbour's
// value).  A point that passes gets the exact S/N of the tile kernel's
// check-free path.  A chunk whose window sums are not proven below 2^22 in
// magnitude (per row: w_max * max|v - m0| over the samples t0-1 .. t0+511,
// against the blocks of t0-1, t0 and t0+256) is listed for the tile kernel.
// Used when the widths are 1, 2, 4, ..., 2^(nw-1) <= 256, rows are 16-byte
// aligned, blocks are a multiple of 256 samples (or one block), for the
// chunks c < n_out/256 - 1 (chunk c+1 lies inside the beam).
constexpr int kStRing = 512;
constexpr int kStSS = 264;  // staged S/N row stride: sample t0+p at index 4+p, p in [-1, 256]
constexpr int kStSeg = 16;  // chunks per CTA

__host__ __device__ inline size_t stream_smem() {
    return (size_t)kBxRows * kStRing * 4 + (size_t)kBxRows * kStSS * 4 + (size_t)kBxRows * kStSS +
           (size_t)kBxRows * 16 * 4;
}

__device__ __forceinline__ uint4 lds128(const uint32_t *p) { return *reinterpret_cast<const uint4 *>(p); }

// Chunk k of one staged row, by the 16 threads of a half-warp: thread l
// holds the samples 256k + 64m + 4l + e (m, e < 4), 16-byte loads that are
// contiguous across the half-warp.  A row that is absent (row == nullptr)
// reads as zeros.
__device__ __forceinline__ void stream_load(const int32_t *__restrict__ row, int64_t k, int l, int4 (&q)[4]) {
    if (row) {
        const int4 *src = reinterpret_cast<const int4 *>(row + k * 256 + 4 * l);
#pragma unroll
        for (int m = 0; m < 4; ++m) q[m] = __ldg(src + 16 * m);
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) q[m] = make_int4(0, 0, 0, 0);
    }
}

// The exclusive prefix of the loaded chunk k into ring slot k & 1,
// continuing `carry` (16-byte stores, contiguous across the half-warp), and
// the chunk's min and max.
__device__ __forceinline__ void stream_scan(const int4 (&q)[4], int64_t k, uint32_t *ring, int l, uint32_t &carry,
                                            int32_t &vmin, int32_t &vmax) {
    uint32_t g[4], incl[4];
    int32_t mn = INT32_MAX, mx = INT32_MIN;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        g[m] = (uint32_t)q[m].x + (uint32_t)q[m].y + (uint32_t)q[m].z + (uint32_t)q[m].w;
        incl[m] = g[m];
        mn = min(min(mn, min(q[m].x, q[m].y)), min(q[m].z, q[m].w));
        mx = max(max(mx, max(q[m].x, q[m].y)), max(q[m].z, q[m].w));
    }
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl[m], o, 16);
            if (l >= o) incl[m] += u;
        }
    }
    uint32_t base = carry;
    uint32_t *dst = ring + (int)(k & 1) * 256 + 4 * l;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const uint32_t tot = __shfl_sync(0xffffffffu, incl[m], 15, 16);
        uint4 o;
        o.x = base + incl[m] - g[m];
        o.y = o.x + (uint32_t)q[m].x;
        o.z = o.y + (uint32_t)q[m].y;
        o.w = o.z + (uint32_t)q[m].z;
        *reinterpret_cast<uint4 *>(dst + 64 * m) = o;
        base += tot;
    }
    carry = base;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o, 16));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o, 16));
    }
    vmin = mn;
    vmax = mx;
}

// Chunk c's magic-range proof for one staged row, by three lanes of the
// row's half-warp (lane j checks the block of sample t0 - 1, t0 or t0 + 256):
// false when some window sum S - w*m0 of the chunk's points (t0-1 .. t0+256)
// may reach 2^22 in magnitude.  [vmin, vmax] covers the samples t0 .. t0+511;
// a window is at most w_max * max|v - m0|, and lim = (2^22 - 1) / w_max.
__device__ __forceinline__ bool stream_proof(const BoxcarArgs &a, const int32_t *__restrict__ row, int64_t d,
                                             int64_t c, int j, int32_t vmin, int32_t vmax, int64_t lim) {
    const int64_t t0 = c * 256;
    if (j > 2 || (j == 0 && t0 == 0)) return true;
    const int64_t t = j == 0 ? t0 - 1 : (j == 1 ? t0 : t0 + 256);
    int64_t lo = vmin, hi = vmax;
    if (t0 > 0) {
        const int64_t v = __ldg(row + t0 - 1);
        lo = min(lo, v);
        hi = max(hi, v);
    }
    const int64_t m0 = __ldg(a.m0s + d * a.nblk + block_of(t, a.norm_block, a.nblk));
    return hi - m0 <= lim && m0 - lo <= lim;
}

// Exact S/N of one point over all widths (the tile kernel's check-free
// formula): Rw(k) = R[t + 2^k], Rt = R[t].  Returns the S/N and sets kbest.
template <typename RW>
__device__ __forceinline__ float stream_exact(RW Rw, uint32_t Rt, int nw, int32_t m0, const float2 *__restrict__ cf,
                                              int &kbest) {
    float best = -INFINITY;
#pragma unroll 1
    for (int k = 0; k < nw; ++k) {  // rare path: kept rolled, so it takes no registers from the hot loop
        const uint32_t w = 1u << k;
        const uint32_t xs = Rw(k) - Rt + (kMagicBits - w * (uint32_t)m0);
        const float2 c = __ldg(cf + k);
        const float sv = fmaf(__uint_as_float(xs) - kMagicValue, c.x, -c.y);
        best = fmaxf(best, __uint_as_float((__float_as_uint(sv) & ~15u) | (15u - (uint32_t)k)));
    }
    const uint32_t bits = __float_as_uint(best);
    kbest = 15 - (int)(bits & 15u);
    return __uint_as_float(bits & ~15u);
}

// Pre-filter of four consecutive points (ring index i0, 16-byte aligned):
// a[e] = max_k (R[t_e + 2^k] - R[t_e] - C_k) as a 32-bit signed value.  NW
// widths when NW > 0, else nw (at most 9).
template <int NW>
__device__ __forceinline__ void stream_prefilter4(const uint32_t *ring, int i0, int nw, const uint32_t *cw,
                                                  uint4 &B, int32_t (&a)[4]) {
    const int n = NW > 0 ? NW : nw;
    B = lds128(ring + i0);
    const uint4 N = lds128(ring + ((i0 + 4) & (kStRing - 1)));
    a[0] = (int32_t)(B.y - B.x - cw[0]);
    a[1] = (int32_t)(B.z - B.y - cw[0]);
    a[2] = (int32_t)(B.w - B.z - cw[0]);
    a[3] = (int32_t)(N.x - B.w - cw[0]);
    if (n > 1) {
        a[0] = max(a[0], (int32_t)(B.z - B.x - cw[1]));
        a[1] = max(a[1], (int32_t)(B.w - B.y - cw[1]));
        a[2] = max(a[2], (int32_t)(N.x - B.z - cw[1]));
        a[3] = max(a[3], (int32_t)(N.y - B.w - cw[1]));
    }
    if (n > 2) {
        a[0] = max(a[0], (int32_t)(N.x - B.x - cw[2]));
        a[1] = max(a[1], (int32_t)(N.y - B.y - cw[2]));
        a[2] = max(a[2], (int32_t)(N.z - B.z - cw[2]));
        a[3] = max(a[3], (int32_t)(N.w - B.w - cw[2]));
    }
#pragma unroll
    for (int k = 3; k < 9; ++k) {
        if (k < n) {
            const uint4 V = lds128(ring + ((i0 + (1 << k)) & (kStRing - 1)));
            a[0] = max(a[0], (int32_t)(V.x - B.x - cw[k]));
            a[1] = max(a[1], (int32_t)(V.y - B.y - cw[k]));
            a[2] = max(a[2], (int32_t)(V.z - B.z - cw[k]));
            a[3] = max(a[3], (int32_t)(V.w - B.w - cw[k]));
        }
    }
}

// Halo point of chunk c (t0 - 1 or t0 + 256) of staged row hr: its S/N, or
// -inf where the pre-filter shows that no width reaches the threshold or the
// point lies before the beam.
__device__ __forceinline__ float stream_halo(const BoxcarArgs &a, const uint32_t *ring_all, int d0, int hr,
                                             bool right, int64_t t0, int nw) {
    const int64_t hd = (int64_t)d0 - 1 + hr;
    const int64_t t = right ? t0 + 256 : t0 - 1;
    if (t < 0) return -INFINITY;
    const int t0m = (int)(t0 & (kStRing - 1));
    const int32_t *hrow = a.dmt + hd * a.n_out;
    const uint32_t *hring = ring_all + hr * kStRing;
    const uint32_t Rt = right ? hring[(t0m + 256) & (kStRing - 1)] : hring[t0m] - (uint32_t)__ldg(hrow + t0 - 1);
    // R[t0 + 512] = R[t0 + 511] + v(t0 + 511)
    const uint32_t Rend = right ? hring[(t0m + 511) & (kStRing - 1)] + (uint32_t)__ldg(hrow + t0 + 511) : 0u;
    auto Rw = [&](int k) -> uint32_t {
        const int64_t j = t + (1 << k);
        return j <= t0 + 511 ? hring[(int)(j & (kStRing - 1))] : Rend;
    };
    const int64_t rb = hd * a.nblk + block_of(t, a.norm_block, a.nblk);
    const uint32_t *C = a.cthr + rb * nw;
    int32_t acc = INT32_MIN;
    for (int k = 0; k < nw; ++k) acc = max(acc, (int32_t)(Rw(k) - Rt - __ldg(C + k)));
    if (acc < 0) return -INFINITY;
    int kb;
    return stream_exact(Rw, Rt, nw, __ldg(a.m0s + rb), a.coefs + rb * nw, kb);
}

template <int NW>
__global__ void __launch_bounds__(256, 4) sps_stream_kernel(BoxcarArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *ring_all = reinterpret_cast<uint32_t *>(smem);
    float *snr_s = reinterpret_cast<float *>(smem + (size_t)kBxRows * kStRing * 4);
    int8_t *k_s = reinterpret_cast<int8_t *>(snr_s + kBxRows * kStSS);
    uint32_t *cw_all = reinterpret_cast<uint32_t *>(k_s + kBxRows * kStSS);  // [16][16] pre-filter constants
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = tid >> 4, l = tid & 15;  // staged row of this half-warp, lane in it
    const int ty = blockIdx.y;
    const int d0 = ty * kBxIn;
    const int64_t dr = (int64_t)d0 - 1 + r;
    const bool present = dr >= 0 && dr < a.ndm;
    const int32_t *row = present ? a.dmt + dr * a.n_out : nullptr;
    uint32_t *ring = ring_all + r * kStRing;
    uint32_t *cw = cw_all + r * 16;
    const int nw = NW > 0 ? NW : a.wl.nw;
    const int64_t lim = ((1 << 22) - 1) / a.maxw;
    const int cs = (int)blockIdx.x * kStSeg;
    const int ce = min(cs + kStSeg, a.n_fast);
    if (!present)
        for (int p = l; p < kStSS; p += 16) snr_s[r * kStSS + p] = -INFINITY;
    // The beam's last chunk(s) go to the tile kernel's list.
    const int n_tail = (int)((a.n_out + kBxT - 1) / kBxT) - a.n_fast;
    if (blockIdx.x == gridDim.x - 1 && tid < n_tail) {
        const int slot = atomicAdd(a.slow_count, 1);
        a.slow_list[slot] = make_int2(a.n_fast + tid, ty);
    }

    uint32_t carry = 0;
    int32_t mnA, mxA, mnB, mxB;  // chunks c and c+1
    int4 q[4];
    stream_load(row, cs, l, q);
    stream_scan(q, cs, ring, l, carry, mnA, mxA);
    stream_load(row, cs + 1, l, q);
    stream_scan(q, cs + 1, ring, l, carry, mnB, mxB);
    bool slow =
        __syncthreads_or(present && !stream_proof(a, row, dr, cs, l, min(mnA, mnB), max(mxA, mxB), lim));

    for (int c = cs; c < ce; ++c) {
        const int64_t t0 = (int64_t)c * 256;
        const int t0m = (int)(t0 & (kStRing - 1));
        bool any = false;
        if (!slow) {  // uniform across the CTA
            // the row's pre-filter constants, staged by its own half-warp; the
            // whole warp meets at the __syncwarp
            const int64_t rb = present ? dr * a.nblk + block_of(t0, a.norm_block, a.nblk) : 0;
            if (present && l < nw) cw[l] = __ldg(a.cthr + rb * nw + l);
            __syncwarp();
            if (present) {
                // main points t0 + 64m + 4l + e of this row
                float *srow = snr_s + r * kStSS + 4;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int p = 64 * m + 4 * l;
                    uint4 B;
                    int32_t acc[4];
                    stream_prefilter4<NW>(ring, t0m + p, nw, cw, B, acc);
                    float4 o = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
                    if ((acc[0] & acc[1] & acc[2] & acc[3]) >= 0) {  // some point passes
                        any = true;
                        const int32_t m0 = __ldg(a.m0s + rb);
                        const float2 *cf = a.coefs + rb * nw;
                        const uint32_t Bv[4] = {B.x, B.y, B.z, B.w};
                        float ov[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            ov[e] = -INFINITY;
                            if (acc[e] >= 0) {
                                const int i = t0m + p + e;
                                int kb;
                                ov[e] = stream_exact([&](int k) { return ring[(i + (1 << k)) & (kStRing - 1)]; }, Bv[e],
                                                     nw, m0, cf, kb);
                                k_s[r * kStSS + 4 + p + e] = (int8_t)kb;
                            }
                        }
                        o = make_float4(ov[0], ov[1], ov[2], ov[3]);
                    }
                    *reinterpret_cast<float4 *>(srow + p) = o;
                }
            }
        } else if (tid == 0) {
            const int slot = atomicAdd(a.slow_count, 1);
            a.slow_list[slot] = make_int2(c, ty);
        }
        any = __syncthreads_or(any);
        if (any) {
            // Halo points t0-1 and t0+256 of all 16 rows (one warp, a point
            // per lane): needed only where a point passed.
            if (warp == 0) {
                const int hr = lane >> 1;
                const int64_t hd = (int64_t)d0 - 1 + hr;
                if (hd >= 0 && hd < a.ndm) {
                    const bool right = lane & 1;
                    snr_s[hr * kStSS + 4 + (right ? 256 : -1)] = stream_halo(a, ring_all, d0, hr, right, t0, nw);
                }
            }
            __syncthreads();
            // interior points: threshold, 3x3 rule, append
            for (int idx = tid; idx < kBxIn * 256; idx += 256) {
                const int rr = 1 + (idx >> 8), p = idx & 255;
                const int d = d0 + rr - 1;
                const float *mid = snr_s + rr * kStSS + 4 + p;
                const float v = *mid;
                bool cand = d < a.ndm && v >= a.thr;
                if (cand) {
                    const float *up = mid - kStSS, *dn = mid + kStSS;
                    cand = v > up[-1] && v > up[0] && v > up[1] && v > mid[-1] && v >= mid[1] && v >= dn[-1] &&
                           v >= dn[0] && v >= dn[1];
                }
                const unsigned mask = __ballot_sync(0xffffffffu, cand);
                if (mask) {
                    const int leader = __ffs(mask) - 1;
                    unsigned long long basec = 0;
                    if (lane == leader) basec = atomicAdd(a.count, (unsigned long long)__popc(mask));
                    basec = __shfl_sync(0xffffffffu, basec, leader);
                    if (cand) {
                        const unsigned long long pos = basec + __popc(mask & ((1u << lane) - 1u));
                        if ((int64_t)pos < a.cap) {
                            sp_cand cd;
                            cd.dm_idx = d;
                            cd.t = (int32_t)(t0 + p);
                            cd.width_idx = k_s[rr * kStSS + 4 + p];
                            cd.snr = v;
                            a.cands[pos] = cd;
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (c + 2 <= ce) {  // chunk c+1 is scored next: bring in chunk c+2
            mnA = mnB;
            mxA = mxB;
            stream_load(row, c + 2, l, q);
            stream_scan(q, c + 2, ring, l, carry, mnB, mxB);
            slow = __syncthreads_or(present &&
                                    !stream_proof(a, row, dr, c + 1, l, min(mnA, mnB), max(mxA, mxB), lim));
        }
    }
}

// Peak filter with a (2R+1) x (2R+1) window (Sec. 3.1.2: the paper's
// second stencil is 11 x 11, R = 5) over a best-S/N map the boxcar kernel
// wrote: one CTA per 32 rows x 256 samples, staged with an R-wide halo (-inf
// outside the map); a point at or above the threshold is kept when it is
// above every neighbour that precedes it in (row, t) order and not below any
// that follows (the same tie rule as the 3 x 3 filter); kept points are
// appended with one atomic per warp.
constexpr int kPkRows = 32;
constexpr int kPkT = 256;

__host__ __device__ inline size_t peaks_smem(int radius) {
    return (size_t)(kPkRows + 2 * radius) * (kPkT + 2 * radius) * sizeof(float);
}

__global__ void __launch_bounds__(256) sps_peaks_window_kernel(const float *__restrict__ best,
                                                               const int8_t *__restrict__ wbest, int32_t ndm,
                                                               int64_t n_out, int radius, float thr,
                                                               sp_cand *__restrict__ cands, int64_t cap,
                                                               unsigned long long *__restrict__ count) {
    extern __shared__ __align__(16) float tile[];
    const int W = kPkT + 2 * radius;
    const int H = kPkRows + 2 * radius;
    const int64_t t0 = (int64_t)blockIdx.x * kPkT;
    const int d0 = blockIdx.y * kPkRows;
    for (int i = threadIdx.x; i < H * W; i += blockDim.x) {
        const int rr = i / W, cc = i - rr * W;
        const int d = d0 - radius + rr;
        const int64_t t = t0 - radius + cc;
        tile[i] = (d >= 0 && d < ndm && t >= 0 && t < n_out) ? __ldg(best + (int64_t)d * n_out + t) : -INFINITY;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kPkRows * kPkT; i += blockDim.x) {
        const int r = i / kPkT, c = i - r * kPkT;
        const int d = d0 + r;
        const int64_t t = t0 + c;
        const float v = tile[(r + radius) * W + c + radius];
        bool keep = d < ndm && t < n_out && v >= thr;
        for (int dr = -radius; dr <= radius && keep; ++dr) {
            const float *row = tile + (r + radius + dr) * W + c + radius;
            for (int dc = -radius; dc <= radius; ++dc) {
                if (dr == 0 && dc == 0) continue;
                const float u = row[dc];
                const bool before = dr < 0 || (dr == 0 && dc < 0);
                if (before ? !(v > u) : !(v >= u)) {
                    keep = false;
                    break;
                }
            }
        }
        const unsigned mask = __ballot_sync(0xffffffffu, keep);
        if (mask) {
            const int leader = __ffs(mask) - 1;
            unsigned long long basec = 0;
            if (lane == leader) basec = atomicAdd(count, (unsigned long long)__popc(mask));
            basec = __shfl_sync(0xffffffffu, basec, leader);
            if (keep) {
                const unsigned long long pos = basec + __popc(mask & ((1u << lane) - 1u));
                if ((int64_t)pos < cap) {
                    sp_cand cd;
                    cd.dm_idx = d;
                    cd.t = (int32_t)t;
                    cd.width_idx = __ldg(wbest + (int64_t)d * n_out + t);
                    cd.snr = v;
                    cands[pos] = cd;
                }
            }
        }
    }
}

size_t boxcar_smem(int maxw) { return boxcar_smem_t<uint32_t>(maxw); }
size_t boxcar_wide_smem(int maxw) { return boxcar_smem_t<int64_t>(maxw); }

int64_t boxcar_tiles(int32_t ndm, int64_t n_out) {
    return ((n_out + kBxT - 1) / kBxT) * (((int64_t)ndm + kBxIn - 1) / kBxIn);
}

}  // namespace

int64_t sps_nblocks(int64_t n_out, int64_t norm_block) {
    if (norm_block <= 0 || norm_block >= n_out) return 1;
    const int64_t nb = n_out / norm_block;
    return nb < 1 ? 1 : nb;
}

// Workspace: per-(row, block) m0, per-(row, block, width) coefficients and
// pre-filter constants, two counters, the tiles the streamed search leaves
// to the tile kernel and the tiles left to the 64-bit pass (one entry per
// tile each), and the per-(row, block) sums.
int64_t sps_workspace_bytes(int32_t ndm, int64_t n_out, int32_t nw, int64_t norm_block) {
    const int64_t nblk = sps_nblocks(n_out, norm_block);
    return align256((int64_t)ndm * nblk * 4) + align256((int64_t)ndm * nblk * nw * 8) +
           align256((int64_t)ndm * nblk * nw * 4) + 256 + 2 * align256(boxcar_tiles(ndm, n_out) * 8) +
           align256((int64_t)ndm * nblk * (int64_t)sizeof(BlockSums));
}

namespace {
std::mutex g_sps_lock;
size_t g_sps_smem[64][7] = {};  // configured boxcar shared memory per (device, kernel)

template <typename K>
int configure_kernel(K kernel, int slot, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    if (dev < 0 || dev >= 64) return SP_ELIMIT;
    std::lock_guard<std::mutex> guard(g_sps_lock);
    if (g_sps_smem[dev][slot] >= smem) return SP_OK;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    g_sps_smem[dev][slot] = smem;
    return SP_OK;
}

int configure_boxcar(bool map, int maxw) {
    int rc = map ? configure_kernel(sps_boxcar_kernel<true>, 0, boxcar_smem(maxw))
                 : configure_kernel(sps_boxcar_kernel<false>, 1, boxcar_smem(maxw));
    if (!rc)
        rc = map ? configure_kernel(sps_boxcar_wide_kernel<true>, 2, boxcar_wide_smem(maxw))
                 : configure_kernel(sps_boxcar_wide_kernel<false>, 3, boxcar_wide_smem(maxw));
    if (!rc && !map) rc = configure_kernel(sps_boxcar_listed_kernel, 4, boxcar_smem(maxw));
    if (!rc && !map) rc = configure_kernel(sps_stream_kernel<0>, 5, stream_smem());
    if (!rc && !map) rc = configure_kernel(sps_stream_kernel<9>, 6, stream_smem());
    return rc;
}
}  // namespace

int sps_configure(int32_t maxw) {
    int rc = configure_boxcar(false, maxw);
    if (!rc) rc = configure_boxcar(true, maxw);
    return rc;
}

int launch_sps(const SpsArgs &a, cudaStream_t stream) {
    WidthList wl;
    for (int k = 0; k < SP_MAX_WIDTHS; ++k) wl.w[k] = k < a.nw ? a.widths[k] : 0;
    wl.nw = a.nw;
    const int maxw = a.widths[a.nw - 1];
    uint8_t *w8 = reinterpret_cast<uint8_t *>(a.work);
    int32_t *m0s = reinterpret_cast<int32_t *>(w8);
    w8 += align256((int64_t)a.ndm * a.nblk * 4);
    float2 *coefs = reinterpret_cast<float2 *>(w8);
    w8 += align256((int64_t)a.ndm * a.nblk * a.nw * 8);
    uint32_t *cthr = reinterpret_cast<uint32_t *>(w8);
    w8 += align256((int64_t)a.ndm * a.nblk * a.nw * 4);
    int *wide_count = reinterpret_cast<int *>(w8);
    int *slow_count = wide_count + 1;
    const int64_t ntiles = boxcar_tiles(a.ndm, a.n_out);
    int2 *wide_list = reinterpret_cast<int2 *>(w8 + 256);
    int2 *slow_list = reinterpret_cast<int2 *>(w8 + 256 + align256(ntiles * 8));
    BlockSums *sums = reinterpret_cast<BlockSums *>(w8 + 256 + 2 * align256(ntiles * 8));
    const bool map = a.map_best != nullptr;
    int rc = configure_boxcar(map, maxw);
    if (rc) return rc;
    WidthRoots wr;
    for (int k = 0; k < SP_MAX_WIDTHS; ++k) {
        const double w = k < a.nw ? (double)a.widths[k] : 1.0;
        wr.sw[k] = std::sqrt(w);
        wr.rsw[k] = 1.0 / std::sqrt(w);
    }
    const int64_t nrb = (int64_t)a.ndm * a.nblk;
    sps_stats_kernel<<<dim3((unsigned)a.nblk, (unsigned)a.ndm), 256, 0, stream>>>(a.dmt, a.n_out, a.norm_block,
                                                                                a.nblk, sums);
    sps_coef_kernel<<<(unsigned)((nrb + 255) / 256), 256, 0, stream>>>(sums, nrb, a.n_out, a.norm_block, a.nblk, wl,
                                                                      wr, a.threshold, m0s, coefs, cthr);
    note_launch(2);
    if (cudaGetLastError() != cudaSuccess) return SP_ECUDA;
    if (cudaMemsetAsync(wide_count, 0, 2 * sizeof(int), stream) != cudaSuccess) return SP_ECUDA;
    if (!map && cudaMemsetAsync(a.count, 0, sizeof(int64_t), stream) != cudaSuccess) return SP_ECUDA;

    BoxcarArgs b;
    b.dmt = a.dmt;
    b.ndm = a.ndm;
    b.n_out = a.n_out;
    b.wl = wl;
    b.maxw = maxw;
    b.thr = a.threshold;
    b.norm_block = a.norm_block;
    b.nblk = a.nblk;
    b.m0s = m0s;
    b.coefs = coefs;
    b.cands = a.cands;
    b.cap = a.cap;
    b.count = reinterpret_cast<unsigned long long *>(a.count);
    b.map_best = a.map_best;
    b.map_k = a.map_wbest;
    b.wide_count = wide_count;
    b.wide_list = wide_list;
    b.vec = (a.n_out & 3) == 0 && (reinterpret_cast<uintptr_t>(a.dmt) & 15) == 0;
    b.n_fast = 0;
    b.cthr = cthr;
    b.slow_count = slow_count;
    b.slow_list = slow_list;
    const int64_t ntx = (a.n_out + kBxT - 1) / kBxT;
    const unsigned ngroups = (unsigned)((a.ndm + kBxIn - 1) / kBxIn);
    int nsm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    if (map) {
        sps_boxcar_kernel<true><<<dim3((unsigned)ntx, ngroups), 256, boxcar_smem(maxw), stream>>>(b);
        sps_boxcar_wide_kernel<true><<<nsm, 256, boxcar_wide_smem(maxw), stream>>>(b);
        note_launch(2);
        return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
    }
    // Streamed search over the chunks it can take, the tile kernel over the
    // tiles it lists (the beam's last chunk(s) and the chunks it cannot prove
    // exact), then the 64-bit pass.
    bool pow2 = maxw <= 256;
    for (int k = 0; k < a.nw; ++k) pow2 = pow2 && a.widths[k] == (1 << k);
    const int64_t n_fast = a.n_out / kBxT - 1;
    if (pow2 && b.vec && (a.nblk == 1 || a.norm_block % kBxT == 0) && n_fast >= 1 && n_fast <= INT32_MAX) {
        b.n_fast = (int32_t)n_fast;
        const dim3 sgrid((unsigned)((n_fast + kStSeg - 1) / kStSeg), ngroups);
        if (a.nw == 9)  // widths 1..256
            sps_stream_kernel<9><<<sgrid, 256, stream_smem(), stream>>>(b);
        else
            sps_stream_kernel<0><<<sgrid, 256, stream_smem(), stream>>>(b);
        sps_boxcar_listed_kernel<<<nsm * 4, 256, boxcar_smem(maxw), stream>>>(b);
        note_launch(2);
    } else {
        sps_boxcar_kernel<false><<<dim3((unsigned)ntx, ngroups), 256, boxcar_smem(maxw), stream>>>(b);
        note_launch();
    }
    sps_boxcar_wide_kernel<false><<<nsm, 256, boxcar_wide_smem(maxw), stream>>>(b);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

int64_t sps_window_workspace_bytes(int32_t ndm, int64_t n_out, int32_t nw, int64_t norm_block, int32_t radius) {
    const int64_t base = sps_workspace_bytes(ndm, n_out, nw, norm_block);
    if (radius <= 1) return base;
    return base + align256((int64_t)ndm * n_out * 4) + align256((int64_t)ndm * n_out);
}

// Radius 1: the fused 3 x 3 search.  Radius 2..kMaxPeakRadius: the best-S/N
// map into the workspace's tail, then the windowed peak filter.
int launch_sps_window(SpsArgs a, int32_t radius, cudaStream_t stream) {
    if (radius <= 1) return launch_sps(a, stream);
    uint8_t *tail = reinterpret_cast<uint8_t *>(a.work) + sps_workspace_bytes(a.ndm, a.n_out, a.nw, a.norm_block);
    float *map = reinterpret_cast<float *>(tail);
    int8_t *wmap = reinterpret_cast<int8_t *>(tail + align256((int64_t)a.ndm * a.n_out * 4));
    sp_cand *cands = a.cands;
    const int64_t cap = a.cap;
    int64_t *count = a.count;
    const float thr = a.threshold;
    a.cands = nullptr;
    a.count = nullptr;
    a.cap = 0;
    a.map_best = map;
    a.map_wbest = wmap;
    int rc = launch_sps(a, stream);
    if (rc) return rc;
    static std::mutex lock;
    static size_t configured[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return SP_ECUDA;
    }
    const size_t smem = peaks_smem(radius);
    {
        std::lock_guard<std::mutex> guard(lock);
        if (configured[dev] < smem) {
            if (cudaFuncSetAttribute(sps_peaks_window_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess) {
                cudaGetLastError();
                return SP_ECUDA;
            }
            configured[dev] = smem;
        }
    }
    if (cudaMemsetAsync(count, 0, sizeof(int64_t), stream) != cudaSuccess) return SP_ECUDA;
    const dim3 grid((unsigned)((a.n_out + kPkT - 1) / kPkT), (unsigned)((a.ndm + kPkRows - 1) / kPkRows));
    sps_peaks_window_kernel<<<grid, 256, smem, stream>>>(map, wmap, a.ndm, a.n_out, radius, thr, cands, cap,
                                                         reinterpret_cast<unsigned long long *>(count));
    note_launch();
    return cudaGetLastError() == cudaSuccess ? SP_OK : SP_ECUDA;
}

}  // namespace sp
