/*
 * oracle.c -- plain, slow, obviously-correct CPU statement of the SPOTLIGHT
 * search hot path (dedispersion + boxcar single-pulse search + 3x3 peaks).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA library is
 * checked against.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may load it.  It shares no code, header or constant table with
 * the CUDA library: every formula below is written out again from the paper.
 *
 * Every function follows one passage of arXiv 2606.27262:
 *   oracle_delays      -- Sec. 3.1.1, Eq. 1 (cold-plasma delay, reference =
 *                         highest frequency), rounded half-up to samples.
 *   oracle_dedisperse  -- Sec. 3.1.1, brute-force incoherent dedispersion:
 *                         shift every channel by its delay and sum -> the
 *                         "DM transform" (one time series per trial DM).
 *   oracle_moments     -- Sec. 3.1.2 normalisation: per-row, per-block count,
 *                         sum (exact, 64-bit) and sum of squares (exact,
 *                         128-bit: a block of int32 values near 2^31 has a
 *                         sum of squares far beyond 2^63).
 *   oracle_boxcar_snr  -- Sec. 3.1.2 matched filter: boxcar of width w as a
 *                         difference of the running cumulative sum, S/N =
 *                         (S - w*mean) / (sigma*sqrt(w)).
 *   oracle_best        -- Sec. 3.1.2: multiple trial widths, keep the best.
 *   oracle_peaks       -- Sec. 3.1.2 peak filtering with a 3x3 window in the
 *                         DM-time plane, threshold in units of sigma.
 *   oracle_peaks_window -- the same filter with a (2r+1) x (2r+1) window; the
 *                         paper's second stencil is 11 x 11 (r = 5).
 *
 * Readings where the paper is silent (all stated, none hidden):
 *   - channel 0 is the highest frequency (the band is flipped so that the
 *     highest frequency comes first, Sec. 2); f_top = freqs[0].
 *   - delay = floor(x + 0.5) with x = K*DM*(1/f^2 - 1/f_top^2)/tsamp, evaluated
 *     in IEEE double left to right, built with -ffp-contract=off.
 *   - output sample t of trial DM d sums in[t + delay[d][c]][c] over channels;
 *     n_in >= n_out + max delay (the overlap-read of Sec. 3.1).
 *   - normalisation blocks: nblk = max(1, n_out / L); block b covers
 *     [b*L, (b+1)*L), the last one also takes the remainder.  Population
 *     variance (divide by n).  A row/block with zero variance gives S/N 0.
 *   - boxcar window [t, t+w) never crosses n_out; it uses the block of t.
 *   - best width: maximum S/N over widths, smallest width on ties.
 *   - 3x3 peak: keep (d,t) if best(d,t) >= threshold and best(d,t) is strictly
 *     greater than each in-range neighbour that comes before it in (d,t)
 *     lexicographic order and greater-or-equal to each neighbour after it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t dm_idx;
    int32_t t;
    int32_t width_idx;
    int32_t pad_;
    double snr;
} oracle_cand;

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Eq. 1: delay of channel c at trial DM d, in samples, rounded half up.
 * Returns 0, or -1 on invalid input (non-positive sizes/tsamp, a negative
 * DM, a non-positive or non-decreasing-in-index frequency). */
int oracle_delays(const double *freqs_mhz, int32_t nchan, double tsamp_s,
                  const double *dms, int32_t ndm, double kdm, int32_t *delays)
{
    if (nchan <= 0 || ndm <= 0 || !(tsamp_s > 0.0))
        return -1;
    for (int32_t c = 0; c < nchan; ++c) {
        if (!(freqs_mhz[c] > 0.0))
            return -1;
        if (c > 0 && !(freqs_mhz[c] < freqs_mhz[c - 1]))
            return -1;
    }
    for (int32_t d = 0; d < ndm; ++d)
        if (!(dms[d] >= 0.0))
            return -1;

    const double ftop = freqs_mhz[0];
    for (int32_t d = 0; d < ndm; ++d) {
        for (int32_t c = 0; c < nchan; ++c) {
            const double f = freqs_mhz[c];
            const double x = kdm * dms[d] * (1.0 / (f * f) - 1.0 / (ftop * ftop)) / tsamp_s;
            delays[(int64_t)d * nchan + c] = (int32_t)floor(x + 0.5);
        }
    }
    return 0;
}

/* Brute-force dedispersion, the definition:
 *   out[r][t] = sum_{c < nchan} in[(t + delays[r][c]) * nchan + c]
 * for t in [0, n_out).  `in` is time-major [n_in][nchan] uint8.  Returns -1
 * if some read would fall outside [0, n_in). */
int oracle_dedisperse(const uint8_t *in, int64_t n_in, int32_t nchan,
                      const int32_t *delays, int32_t nrows, int64_t n_out,
                      int32_t *out)
{
    for (int64_t i = 0; i < (int64_t)nrows * nchan; ++i)
        if (delays[i] < 0 || delays[i] + n_out > n_in)
            return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t r = 0; r < nrows; ++r) {
        const int32_t *dl = delays + (int64_t)r * nchan;
        int32_t *row = out + (int64_t)r * n_out;
        for (int64_t t = 0; t < n_out; ++t) {
            int32_t acc = 0;
            for (int32_t c = 0; c < nchan; ++c)
                acc += in[(t + dl[c]) * (int64_t)nchan + c];
            row[t] = acc;
        }
    }
    return 0;
}

int64_t oracle_nblocks(int64_t n_out, int64_t norm_block)
{
    if (norm_block <= 0 || norm_block >= n_out)
        return 1;
    int64_t nb = n_out / norm_block;
    return nb < 1 ? 1 : nb;
}

static int64_t block_start(int64_t b, int64_t norm_block, int64_t nblk)
{
    return nblk == 1 ? 0 : b * norm_block;
}

static int64_t block_end(int64_t b, int64_t norm_block, int64_t nblk, int64_t n_out)
{
    return (b == nblk - 1) ? n_out : (b + 1) * norm_block;
}

/* Per row r and block b: count, sum and sum of squares of the DM-transform
 * samples in the block.  Arrays are [nrows][nblk].  The sum of squares is
 * formed in 128 bits and returned as its high (signed) and low (unsigned)
 * 64-bit halves. */
static void block_moments(const int32_t *row, int64_t lo, int64_t hi, int64_t *s1_out, __int128 *s2_out)
{
    int64_t s1 = 0;
    __int128 s2 = 0;
    for (int64_t t = lo; t < hi; ++t) {
        s1 += row[t];
        s2 += (__int128)((int64_t)row[t] * row[t]);
    }
    *s1_out = s1;
    *s2_out = s2;
}

int oracle_moments(const int32_t *dmt, int32_t nrows, int64_t n_out,
                   int64_t norm_block, int64_t *cnt, int64_t *sx, int64_t *sxx_hi, uint64_t *sxx_lo)
{
    if (nrows <= 0 || n_out <= 0)
        return -1;
    const int64_t nblk = oracle_nblocks(n_out, norm_block);
    for (int32_t r = 0; r < nrows; ++r) {
        const int32_t *row = dmt + (int64_t)r * n_out;
        for (int64_t b = 0; b < nblk; ++b) {
            const int64_t lo = block_start(b, norm_block, nblk);
            const int64_t hi = block_end(b, norm_block, nblk, n_out);
            int64_t s1;
            __int128 s2;
            block_moments(row, lo, hi, &s1, &s2);
            cnt[(int64_t)r * nblk + b] = hi - lo;
            sx[(int64_t)r * nblk + b] = s1;
            sxx_hi[(int64_t)r * nblk + b] = (int64_t)(s2 >> 64);
            sxx_lo[(int64_t)r * nblk + b] = (uint64_t)s2;
        }
    }
    return 0;
}

/* Boxcar S/N for every row r, width index k and start t:
 *   snr[r][k][t] = (n*S - w*Sx) / (sqrt(w) * sqrt(n*Sxx - Sx^2))
 * with S = C[t+w] - C[t] (C = running cumulative sum of the row), and n, Sx,
 * Sxx the moments of the block containing t.  NaN where t + w > n_out.  The
 * variance term is formed exactly in 128-bit integers before the square
 * root.  Widths must be >= 1. */
int oracle_boxcar_snr(const int32_t *dmt, int32_t nrows, int64_t n_out,
                      const int32_t *widths, int32_t nw, int64_t norm_block,
                      double *snr)
{
    if (nrows <= 0 || n_out <= 0 || nw <= 0)
        return -1;
    for (int32_t k = 0; k < nw; ++k)
        if (widths[k] < 1)
            return -1;
    const int64_t nblk = oracle_nblocks(n_out, norm_block);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * nblk * nrows);
    int64_t *sx = (int64_t *)malloc(sizeof(int64_t) * nblk * nrows);
    __int128 *sxx = (__int128 *)malloc(sizeof(__int128) * nblk * nrows);
    if (!cnt || !sx || !sxx) {
        free(cnt); free(sx); free(sxx);
        return -2;
    }
    for (int32_t r = 0; r < nrows; ++r)
        for (int64_t b = 0; b < nblk; ++b) {
            const int64_t lo = block_start(b, norm_block, nblk);
            const int64_t hi = block_end(b, norm_block, nblk, n_out);
            cnt[(int64_t)r * nblk + b] = hi - lo;
            block_moments(dmt + (int64_t)r * n_out, lo, hi, &sx[(int64_t)r * nblk + b],
                          &sxx[(int64_t)r * nblk + b]);
        }

    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t r = 0; r < nrows; ++r) {
        const int32_t *row = dmt + (int64_t)r * n_out;
        int64_t *cum = (int64_t *)malloc(sizeof(int64_t) * (n_out + 1));
        if (!cum) {
            rc = -2;
            continue;
        }
        cum[0] = 0;
        for (int64_t t = 0; t < n_out; ++t)
            cum[t + 1] = cum[t] + row[t];
        for (int32_t k = 0; k < nw; ++k) {
            const int64_t w = widths[k];
            double *out = snr + ((int64_t)r * nw + k) * n_out;
            for (int64_t t = 0; t < n_out; ++t) {
                if (t + w > n_out) {
                    out[t] = NAN;
                    continue;
                }
                int64_t b = t / (norm_block > 0 ? norm_block : n_out);
                if (b > nblk - 1)
                    b = nblk - 1;
                const int64_t n = cnt[(int64_t)r * nblk + b];
                const int64_t s1 = sx[(int64_t)r * nblk + b];
                const __int128 s2 = sxx[(int64_t)r * nblk + b];
                const __int128 var_n2 = (__int128)n * s2 - (__int128)s1 * s1;
                const int64_t S = cum[t + w] - cum[t];
                const __int128 num = (__int128)n * S - (__int128)w * s1;
                if (var_n2 <= 0) {
                    out[t] = 0.0;
                    continue;
                }
                out[t] = (double)num / (sqrt((double)w) * sqrt((double)var_n2));
            }
        }
        free(cum);
    }
    free(cnt); free(sx); free(sxx);
    return rc;
}

/* Best S/N over the trial widths for every (r, t): best[r][t] and the index
 * of the width that reached it (smallest index on ties).  Where no width
 * fits (t + widths[k] > n_out for all k) best = -inf and wbest = -1. */
int oracle_best(const int32_t *dmt, int32_t nrows, int64_t n_out,
                const int32_t *widths, int32_t nw, int64_t norm_block,
                double *best, int32_t *wbest)
{
    for (int32_t r = 0; r < nrows; ++r) {
        double *snr = (double *)malloc(sizeof(double) * nw * n_out);
        if (!snr)
            return -2;
        int rc = oracle_boxcar_snr(dmt + (int64_t)r * n_out, 1, n_out, widths, nw,
                                   norm_block, snr);
        if (rc) {
            free(snr);
            return rc;
        }
        for (int64_t t = 0; t < n_out; ++t) {
            double b = -INFINITY;
            int32_t kb = -1;
            for (int32_t k = 0; k < nw; ++k) {
                const double v = snr[(int64_t)k * n_out + t];
                if (isnan(v))
                    continue;
                if (kb < 0 || v > b) {
                    b = v;
                    kb = k;
                }
            }
            best[(int64_t)r * n_out + t] = b;
            wbest[(int64_t)r * n_out + t] = kb;
        }
        free(snr);
    }
    return 0;
}

/* 3x3 peak filter + threshold over a best-S/N map of nrows consecutive trial
 * DMs whose first row is DM index row0.  Candidates are emitted only for rows
 * in [emit_lo, emit_hi) (indices into the map); the other rows act only as
 * neighbours.  Rows outside the map are treated as out of range.  Output is
 * in (dm_idx, t) order; returns the total count (which may exceed cap: only
 * the first cap are written). */
int64_t oracle_peaks(const double *best, const int32_t *wbest, int32_t nrows,
                     int64_t n_out, double thr, int32_t row0, int32_t emit_lo,
                     int32_t emit_hi, oracle_cand *out, int64_t cap)
{
    int64_t count = 0;
    for (int32_t r = emit_lo; r < emit_hi; ++r) {
        for (int64_t t = 0; t < n_out; ++t) {
            const double v = best[(int64_t)r * n_out + t];
            if (!(v >= thr))
                continue;
            int keep = 1;
            for (int32_t dr = -1; dr <= 1 && keep; ++dr) {
                for (int64_t dt = -1; dt <= 1; ++dt) {
                    if (dr == 0 && dt == 0)
                        continue;
                    const int32_t rr = r + dr;
                    const int64_t tt = t + dt;
                    if (rr < 0 || rr >= nrows || tt < 0 || tt >= n_out)
                        continue;
                    const double u = best[(int64_t)rr * n_out + tt];
                    const int before = (dr < 0) || (dr == 0 && dt < 0);
                    if (before ? !(v > u) : !(v >= u)) {
                        keep = 0;
                        break;
                    }
                }
            }
            if (!keep)
                continue;
            if (count < cap) {
                out[count].dm_idx = row0 + r;
                out[count].t = (int32_t)t;
                out[count].width_idx = wbest[(int64_t)r * n_out + t];
                out[count].pad_ = 0;
                out[count].snr = v;
            }
            ++count;
        }
    }
    return count;
}

/* Peak filter with a (2*radius+1) x (2*radius+1) window in the DM-time plane
 * (Sec. 3.1.2: a window slides over the candidates and only the highest S/N
 * of each window survives; the paper's stencils are 3 x 3 and 11 x 11) plus
 * the threshold, over a whole best-S/N map.  (r, t) is kept when best >= thr
 * and, for every in-range neighbour (r', t') of the window, best(r, t) >
 * best(r', t') if (r', t') comes before (r, t) in (row, t) order and >=
 * otherwise.  Output in (row, t) order; returns the total count (which may
 * exceed cap: only the first cap are written). */
int64_t oracle_peaks_window(const double *best, const int32_t *wbest, int32_t nrows,
                            int64_t n_out, double thr, int32_t radius,
                            oracle_cand *out, int64_t cap)
{
    if (radius < 1)
        return -1;
    int64_t count = 0;
    for (int32_t r = 0; r < nrows; ++r) {
        for (int64_t t = 0; t < n_out; ++t) {
            const double v = best[(int64_t)r * n_out + t];
            if (!(v >= thr))
                continue;
            int keep = 1;
            for (int32_t dr = -radius; dr <= radius && keep; ++dr) {
                for (int64_t dt = -radius; dt <= radius; ++dt) {
                    if (dr == 0 && dt == 0)
                        continue;
                    const int32_t rr = r + dr;
                    const int64_t tt = t + dt;
                    if (rr < 0 || rr >= nrows || tt < 0 || tt >= n_out)
                        continue;
                    const double u = best[(int64_t)rr * n_out + tt];
                    const int before = (dr < 0) || (dr == 0 && dt < 0);
                    if (before ? !(v > u) : !(v >= u)) {
                        keep = 0;
                        break;
                    }
                }
            }
            if (!keep)
                continue;
            if (count < cap) {
                out[count].dm_idx = r;
                out[count].t = (int32_t)t;
                out[count].width_idx = wbest[(int64_t)r * n_out + t];
                out[count].pad_ = 0;
                out[count].snr = v;
            }
            ++count;
        }
    }
    return count;
}
