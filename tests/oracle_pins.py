"""Pins of the CPU oracle against facts fixed outside it.

Each ``pin_*`` function takes a loaded oracle library handle and raises
AssertionError on disagreement, so that tests/test_oracle_pins.py can run them
against the real oracle and tests/test_oracle_mutants.py can run them against
deliberately broken builds of it (every mutant must trip at least one pin).

What pins what (arXiv 2606.27262):
* Eq. 1 delays: exact rational arithmetic on the same binary64 inputs, round
  half up; the maximum sweeps of the two single-beam workloads.
* Brute-force dedispersion (Sec. 3.1.1): a pure-Python loop on tiny random
  inputs; DM 0 equals the channel sum (numpy); a constant input; the
  Appendix A S/N-loss law (Eq. A1-A3) for a pulse dedispersed at a wrong DM.
* Boxcar S/N (Sec. 3.1.2): width 1 equals numpy's standardisation; an
  impulse row has a closed form for every width and window position; block
  boundaries; zero variance; white noise has unit variance at every width.
* Best width and 3x3 peaks (Sec. 3.1.2): a pure-Python brute force of the
  tie rule on small maps with planted ties.
* Whole path: an injected burst is recovered at its true DM and width.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
from scipy.special import erf

import oracle
import synth


# ---------------------------------------------------------------- delays --
def _exact_delays(freqs, tsamp, dms, kdm=oracle.KDM):
    """floor(x + 1/2) of the exact rational value of Eq. 1 on the binary64
    inputs, and the distance of x from the nearest half-integer."""
    F = [Fraction(float(f)) for f in freqs]
    ftop2 = 1 / (F[0] * F[0])
    A = [1 / (f * f) - ftop2 for f in F]
    K = Fraction(float(kdm)) / Fraction(float(tsamp))
    out = np.empty((len(dms), len(freqs)), np.int64)
    tie = np.zeros(out.shape, bool)
    for i, dm in enumerate(dms):
        kd = K * Fraction(float(dm))
        for j, a in enumerate(A):
            x = kd * a
            k = math.floor(x + Fraction(1, 2))
            out[i, j] = k
            frac = x - math.floor(x)
            tie[i, j] = abs(float(frac) - 0.5) < 1e-9
    return out, tie


def pin_delays_exact(lib):
    wl = synth.config1()
    got = oracle.delays(wl.freqs, wl.tsamp, wl.dms, lib=lib)
    want, tie = _exact_delays(wl.freqs, wl.tsamp, wl.dms)
    bad = (got != want) & ~tie
    assert not bad.any(), f"config-1 delays differ from exact rational at {np.argwhere(bad)[:5]}"
    assert int(got.max()) == 11163, got.max()
    wl2 = synth.config2()
    chans = np.r_[np.arange(0, 4096, 97), 4095]
    dsel = np.r_[np.arange(0, wl2.dms.size, 7), wl2.dms.size - 1]
    got2 = oracle.delays(wl2.freqs, wl2.tsamp, wl2.dms, lib=lib)
    want2, tie2 = _exact_delays(wl2.freqs[chans], wl2.tsamp, wl2.dms[dsel])
    sub = got2[np.ix_(dsel, chans)]
    bad2 = (sub != want2) & ~tie2
    assert not bad2.any(), "config-2 delays differ from exact rational"
    assert int(got2.max()) == 44995, got2.max()


def pin_delays_structure(lib):
    """DM 0 and the top channel have zero delay; delays grow with DM and with
    decreasing frequency (Eq. 1)."""
    f = synth.band_freqs(64)
    dms = np.array([0.0, 10.0, 100.0, 1000.0])
    d = oracle.delays(f, synth.TSAMP, dms, lib=lib)
    assert (d[0] == 0).all()
    assert (d[:, 0] == 0).all()
    assert (np.diff(d, axis=0) >= 0).all() and (np.diff(d, axis=1) >= 0).all()
    assert d[-1, -1] > d[-2, -1] > d[1, -1] > 0


# ------------------------------------------------------------ dedisperse --
def _py_dedisperse(x, delays, n_out):
    out = []
    for row in delays:
        r = []
        for t in range(n_out):
            s = 0
            for c in range(x.shape[1]):
                s += int(x[t + int(row[c]), c])
            r.append(s)
        out.append(r)
    return np.array(out, dtype=np.int64)


def pin_dedisperse_bruteforce(lib):
    rng = np.random.default_rng(7)
    for nchan, ndm, n_out in [(1, 1, 5), (3, 4, 17), (8, 6, 40), (5, 2, 64)]:
        delays = np.sort(rng.integers(0, 12, size=(ndm, nchan)), axis=1).astype(np.int32)
        delays[:, 0] = 0
        n_in = n_out + int(delays.max())
        x = rng.integers(0, 256, size=(n_in, nchan)).astype(np.uint8)
        got = oracle.dedisperse(x, delays, n_out, lib=lib)
        want = _py_dedisperse(x, delays, n_out)
        assert np.array_equal(got, want), (nchan, ndm, n_out)


def pin_dm0_channel_sum(lib):
    rng = np.random.default_rng(11)
    f = synth.band_freqs(32)
    dms = np.array([0.0, 50.0])
    d = oracle.delays(f, synth.TSAMP, dms, lib=lib)
    n_out = 300
    x = rng.integers(0, 256, size=(n_out + int(d.max()), 32)).astype(np.uint8)
    got = oracle.dedisperse(x, d, n_out, lib=lib)
    assert np.array_equal(got[0], x[:n_out].astype(np.int64).sum(axis=1))
    c = np.full_like(x, 201)
    assert (oracle.dedisperse(c, d, n_out, lib=lib) == 201 * 32).all()


def pin_smearing_appendix_a(lib):
    """S(dDM)/S = (sqrt(pi)/2) erf(zeta)/zeta with zeta = 6.91e-3 dDM
    dnu_MHz / (W_ms nu_GHz^3) (Appendix A), within 15% for zeta <= 2 on the
    Band-3 layout (the law assumes a narrow band; 300-500 MHz is not)."""
    nchan = 2048
    freqs = synth.band_freqs(nchan)
    dm0, W = 300.0, 16.0
    sig = W / (2 * math.sqrt(2 * math.log(2)))
    wms = W * synth.TSAMP * 1e3
    for ddm in [0.25, 0.5, 1.0, 2.0]:
        dms = np.array([dm0, dm0 + ddm])
        d = oracle.delays(freqs, synth.TSAMP, dms, lib=lib)
        n_out = 2048
        n_in = n_out + int(d.max()) + 4
        cen = 1000 + synth.fractional_delay(freqs, dm0)
        s = np.arange(n_in)[:, None]
        x = np.rint(200 * np.exp(-0.5 * ((s - cen[None, :]) / sig) ** 2)).astype(np.uint8)
        dmt = oracle.dedisperse(x, d, n_out, lib=lib).astype(np.float64)
        ratio = dmt[1].max() / dmt[0].max()
        zeta = 6.91e-3 * ddm * synth.BANDWIDTH / (wms * 0.4 ** 3)
        pred = math.sqrt(math.pi) / 2 / zeta * erf(zeta)
        assert abs(ratio / pred - 1) < 0.15, (ddm, zeta, ratio, pred)
        assert int(np.argmax(dmt[0])) in (999, 1000, 1001)


# ------------------------------------------------------------ boxcar S/N --
def pin_snr_width1_standardisation(lib):
    rng = np.random.default_rng(3)
    row = rng.integers(-1000, 100000, size=(2, 777)).astype(np.int32)
    snr = oracle.boxcar_snr(row, [1], 0, lib=lib)[:, 0, :]
    x = row.astype(np.float64)
    want = (x - x.mean(axis=1, keepdims=True)) / x.std(axis=1, keepdims=True)
    assert np.allclose(snr, want, rtol=1e-12, atol=1e-12)


def pin_snr_impulse_closed_form(lib):
    """A row of zeros with one impulse h at t*: mean h/n, variance h^2(n-1)/n^2,
    so a window [t, t+w) holding the impulse has S/N (n-w)/sqrt(w(n-1)) and
    one without it -sqrt(w/(n-1))."""
    n, ts, h = 200, 77, 5000
    row = np.zeros((1, n), np.int32)
    row[0, ts] = h
    widths = [1, 2, 3, 8, 16]
    snr = oracle.boxcar_snr(row, widths, 0, lib=lib)[0]
    for k, w in enumerate(widths):
        for t in range(n):
            if t + w > n:
                assert math.isnan(snr[k, t])
                continue
            inside = t <= ts < t + w
            want = (n - w) / math.sqrt(w * (n - 1)) if inside else -math.sqrt(w / (n - 1))
            assert abs(snr[k, t] - want) < 1e-12 * max(1, abs(want)), (w, t, snr[k, t], want)


def pin_snr_blocks(lib):
    """Two normalisation blocks (L=100, n=250 -> blocks [0,100), [100,250))
    with different levels: each block is standardised with its own moments,
    and a window that starts in block 0 uses block 0 even if it crosses."""
    rng = np.random.default_rng(5)
    row = np.concatenate([rng.integers(0, 50, 100), 1000 + rng.integers(0, 500, 150)]).astype(np.int32)[None]
    assert oracle.nblocks(250, 100, lib=lib) == 2
    s1 = oracle.boxcar_snr(row, [1, 4], 100, lib=lib)[0]
    x = row[0].astype(np.float64)
    a, b = x[:100], x[100:]
    assert np.allclose(s1[0, :100], (a - a.mean()) / a.std(), rtol=1e-12)
    assert np.allclose(s1[0, 100:], (b - b.mean()) / b.std(), rtol=1e-12)
    t = 98  # window [98, 102) crosses into block 1 but uses block 0
    want = (x[t:t + 4].sum() - 4 * a.mean()) / (a.std() * 2.0)
    assert abs(s1[1, t] - want) < 1e-10 * abs(want)
    cnt, sx, sxx = oracle.moments(row, 100, lib=lib)
    assert cnt.tolist() == [[100, 150]]
    assert sx[0, 1] == int(b.sum()) and sxx[0, 0] == int((a * a).sum())


def pin_snr_large_values(lib):
    """Values near +-2^30 over 4096-sample blocks: the sum of squares
    (~2^72) exceeds 64 bits.  The moments must equal Python's exact integer
    sums and the width-1 S/N must equal numpy's standardisation; a 64-bit sum
    of squares wraps and fails both."""
    rng = np.random.default_rng(11)
    row = (rng.choice([-1, 1], 8192) * (2 ** 30 + rng.integers(0, 2 ** 20, 8192))).astype(np.int32)[None]
    cnt, sx, sxx = oracle.moments(row, 4096, lib=lib)
    for b in range(2):
        seg = [int(v) for v in row[0, 4096 * b:4096 * (b + 1)]]
        assert cnt[0, b] == 4096 and sx[0, b] == sum(seg)
        assert sxx[0, b] == sum(v * v for v in seg) and sxx[0, b] > 2 ** 63
    s = oracle.boxcar_snr(row, [1], 4096, lib=lib)[0, 0]
    x = row[0].astype(np.float64)
    for b in range(2):
        seg = x[4096 * b:4096 * (b + 1)]
        assert np.allclose(s[4096 * b:4096 * (b + 1)], (seg - seg.mean()) / seg.std(), rtol=1e-9, atol=1e-9)


def pin_snr_zero_variance(lib):
    row = np.full((1, 64), 12345, np.int32)
    s = oracle.boxcar_snr(row, [1, 2, 4], 0, lib=lib)[0]
    assert np.all(s[~np.isnan(s)] == 0.0)
    b, k = oracle.best(row, [1, 2, 4], 0, lib=lib)
    assert (k[0, :61] == 0).all() and (b[0, :61] == 0).all()


def pin_snr_white_noise(lib):
    """On white noise every width gives S/N with mean 0 and variance 1 (up to
    sampling error; overlapping windows correlate, so the error bar is wide)."""
    rng = np.random.default_rng(9)
    n = 1 << 16
    row = np.rint(rng.normal(5e5, 1000.0, size=(1, n))).astype(np.int32)
    widths = [1, 4, 32, 256]
    s = oracle.boxcar_snr(row, widths, 0, lib=lib)[0]
    for k, w in enumerate(widths):
        v = s[k][~np.isnan(s[k])]
        neff = v.size / w
        assert abs(v.mean()) < 5 / math.sqrt(neff), (w, v.mean())
        assert abs(v.var() - 1) < 5 * math.sqrt(2 / neff), (w, v.var())


# --------------------------------------------------------- best + peaks --
def _py_best(snr):
    nw, n = snr.shape
    best, kb = np.full(n, -np.inf), np.full(n, -1, np.int32)
    for t in range(n):
        for k in range(nw):
            v = snr[k, t]
            if math.isnan(v):
                continue
            if kb[t] < 0 or v > best[t]:
                best[t], kb[t] = v, k
    return best, kb


def _py_peaks(best, thr):
    nd, n = best.shape
    out = []
    for d in range(nd):
        for t in range(n):
            v = best[d, t]
            if not v >= thr:
                continue
            ok = True
            for dd in (-1, 0, 1):
                for dt in (-1, 0, 1):
                    if (dd, dt) == (0, 0):
                        continue
                    e, u = d + dd, t + dt
                    if not (0 <= e < nd and 0 <= u < n):
                        continue
                    earlier = (e, u) < (d, t)
                    if (earlier and not v > best[e, u]) or (not earlier and not v >= best[e, u]):
                        ok = False
            if ok:
                out.append((d, t))
    return out


def pin_best_and_peaks_bruteforce(lib):
    rng = np.random.default_rng(13)
    dmt = rng.integers(0, 30, size=(9, 60)).astype(np.int32)
    dmt[4, 20:23] = 200                       # plateau -> width ties/peaks
    dmt[2, 40] = 150
    dmt[3, 40] = 150                          # equal neighbours across DM
    widths = [1, 2, 3, 5]
    snr = oracle.boxcar_snr(dmt, widths, 0, lib=lib)
    b, k = oracle.best(dmt, widths, 0, lib=lib)
    for d in range(dmt.shape[0]):
        pb, pk = _py_best(snr[d])
        assert np.array_equal(pk, k[d]) and np.array_equal(pb, b[d])
    for thr in (-1e9, 0.5, 2.0):
        c, n = oracle.peaks(b, k, thr, lib=lib)
        want = _py_peaks(b, thr)
        assert n == len(want)
        assert [(int(a), int(t)) for a, t in zip(c["dm_idx"], c["t"])] == want
    # planted exact ties in a hand-made map
    m = np.zeros((3, 8))
    m[1, 1] = m[1, 2] = 9.0                   # equal in time: the earlier wins
    m[0, 4] = m[1, 4] = 4.0                   # equal across DM: the earlier wins
    m[2, 7] = 1.0                             # exactly at the threshold: kept
    kk = np.zeros(m.shape, np.int32)
    c, n = oracle.peaks(m, kk, 1.0, lib=lib)
    got = [(int(a), int(t)) for a, t in zip(c["dm_idx"], c["t"])]
    assert got == _py_peaks(m, 1.0) == [(0, 4), (1, 1), (2, 7)], got


def _py_window_peaks(best, thr, radius):
    """Brute force of the sliding-window rule: a point survives its
    (2r+1)^2 window when it is at least the threshold, strictly above every
    in-range point of the window that comes before it in (row, t) order and
    not below any that comes after."""
    nd, n = best.shape
    out = []
    for d in range(nd):
        for t in range(n):
            v = best[d, t]
            if not v >= thr:
                continue
            window = [(e, u) for e in range(max(0, d - radius), min(nd, d + radius + 1))
                      for u in range(max(0, t - radius), min(n, t + radius + 1)) if (e, u) != (d, t)]
            if all((v > best[e, u]) if (e, u) < (d, t) else (v >= best[e, u]) for e, u in window):
                out.append((d, t))
    return out


def pin_peaks_window_bruteforce(lib):
    """The (2r+1)^2 peak filter (Sec. 3.1.2's 3x3 and 11x11 stencils):
    equal to the brute force on random maps with many exact ties for r = 2
    and 5, equal to the 3x3 filter for r = 1, and on a hand-made row an
    11x11 window keeps only the higher of two peaks 4 samples apart while
    3x3 keeps both."""
    rng = np.random.default_rng(17)
    for radius in (1, 2, 5):
        b = np.round(rng.normal(0, 1.5, size=(14, 45)) * 2) / 2  # half-unit grid: many ties
        b[rng.random(b.shape) < 0.05] = -np.inf
        kk = np.zeros(b.shape, np.int32)
        c, n = oracle.peaks_window(b, kk, 0.5, radius, lib=lib)
        want = _py_window_peaks(b, 0.5, radius)
        assert n == len(want) and [(int(a), int(t)) for a, t in zip(c["dm_idx"], c["t"])] == want, radius
        if radius == 1:
            c3, n3 = oracle.peaks(b, kk, 0.5, lib=lib)
            assert [(int(a), int(t)) for a, t in zip(c3["dm_idx"], c3["t"])] == want
    m = np.zeros((3, 16))
    m[1, 4], m[1, 8] = 5.0, 6.0
    kk = np.zeros(m.shape, np.int32)
    got3 = [(int(a), int(t)) for a, t in zip(*(lambda c: (c["dm_idx"], c["t"]))(oracle.peaks_window(m, kk, 1.0, 1,
                                                                                                   lib=lib)[0]))]
    got11 = [(int(a), int(t)) for a, t in zip(*(lambda c: (c["dm_idx"], c["t"]))(oracle.peaks_window(m, kk, 1.0, 5,
                                                                                                    lib=lib)[0]))]
    assert got3 == [(1, 4), (1, 8)] and got11 == [(1, 8)], (got3, got11)


# ------------------------------------------------------------ whole path --
def pin_burst_recovered(lib):
    """A strong Gaussian burst at an on-grid DM in config-1 noise is found at
    exactly its DM, at its arrival sample, with a width near its FWHM."""
    wl = synth.config1()
    d = oracle.delays(wl.freqs, wl.tsamp, wl.dms, lib=lib)
    n_in = wl.n_out + int(d.max())
    b = synth.Burst(t0=3000, dm=250.0, fwhm=8.0, snr=40.0)
    x = synth.make_beam(77, wl.nchan, n_in, wl.freqs, [b], widths=wl.widths)
    rows = np.arange(240, 261)
    dmt = oracle.dedisperse(x, d[rows], wl.n_out, lib=lib)
    best, kb = oracle.best(dmt, wl.widths, wl.norm_block, lib=lib)
    i, t = np.unravel_index(np.argmax(best), best.shape)
    assert wl.dms[rows[i]] == 250.0, wl.dms[rows[i]]
    w = int(wl.widths[kb[i, t]])
    assert w in (4, 8, 16), w
    assert t <= 3000 < t + w or abs(int(t) - 3000) <= w, (t, w)
    assert 0.75 * 40 <= best[i, t] <= 1.25 * 40, best[i, t]


ALL_PINS = [
    pin_delays_exact, pin_delays_structure, pin_dedisperse_bruteforce, pin_dm0_channel_sum,
    pin_smearing_appendix_a, pin_snr_width1_standardisation, pin_snr_impulse_closed_form,
    pin_snr_blocks, pin_snr_large_values, pin_snr_zero_variance, pin_snr_white_noise, pin_best_and_peaks_bruteforce,
    pin_peaks_window_bruteforce,
    pin_burst_recovered,
]
