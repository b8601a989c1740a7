"""Seeded radio-frequency interference for 8-bit filterbank beams (test and
bench inputs of the candidate classifier, arXiv 2606.27262 Sec. 3.2.2: the
classifier separates astrophysical bursts from RFI among the candidates the
search and the sifter keep).

Three kinds, added (in 8-bit units above the noise mean) to the beams that
``synth.make_beam_torch`` draws, before rounding and clipping:

* ``narrowband``: a block of 4-16 adjacent channels switching on in pulses
  of 32-256 samples throughout a span (a persistent narrowband emitter);
  seen by the search at every DM, since a single channel is not dispersed.
* ``impulse``: every channel for 1-4 samples (a broadband impulse at DM 0);
  after the DM >= 10 cut of the sifter it is seen smeared at low DMs.
* ``tone``: 2-8 adjacent channels whose centre drifts across the band at a
  constant rate while the tone switches on and off with a period of 50-500
  samples; a drift towards lower frequencies mimics part of a dispersion
  sweep.

Nothing here computes a delay table, a dedispersed sum or an S/N.
"""
from __future__ import annotations

import dataclasses

import numpy as np

KINDS = ("narrowband", "impulse", "tone")


@dataclasses.dataclass
class Rfi:
    kind: str
    t0: int            # first sample
    dur: int           # samples
    amp: float         # 8-bit units above the noise mean
    c0: int = 0        # first channel (narrowband, tone)
    nch: int = 0       # channels (narrowband, tone)
    period: float = 0  # samples: pulse spacing (narrowband), on/off period (tone)
    duty: float = 1.0  # fraction of each period that is on
    drift: float = 0.0  # channels per sample (tone)


def draw_rfi(rng: np.random.Generator, n: int, n_in: int, nchan: int, kinds=None) -> list[Rfi]:
    """n events with uniform random kinds (or the given list of kinds) over
    samples [0, n_in) of an nchan-channel beam."""
    out = []
    ks = [KINDS[int(i)] for i in rng.integers(0, len(KINDS), n)] if kinds is None else list(kinds)
    for k in ks:
        if k == "narrowband":
            nch = int(rng.integers(4, 17))
            dur = int(rng.integers(n_in // 8, n_in // 2 + 1))
            out.append(Rfi(k, int(rng.integers(0, n_in - dur + 1)), dur, float(rng.uniform(50.0, 110.0)),
                           c0=int(rng.integers(0, nchan - nch + 1)), nch=nch,
                           period=float(rng.uniform(400.0, 2000.0)), duty=float(rng.uniform(0.05, 0.3))))
        elif k == "impulse":
            dur = int(rng.integers(1, 5))
            out.append(Rfi(k, int(rng.integers(0, n_in - dur + 1)), dur, float(rng.uniform(25.0, 90.0))))
        elif k == "tone":
            nch = int(rng.integers(2, 9))
            dur = int(rng.integers(2000, 8001))
            rate = float(rng.uniform(0.2, 2.0)) * nchan / 4096.0
            out.append(Rfi(k, int(rng.integers(0, max(1, n_in - dur))), dur, float(rng.uniform(60.0, 120.0)),
                           c0=int(rng.integers(0, nchan // 2)), nch=nch, period=float(rng.uniform(50.0, 500.0)),
                           duty=float(rng.uniform(0.3, 0.7)), drift=rate))
        else:
            raise ValueError(f"unknown RFI kind {k}")
    return out


def rfi_signal(events: list[Rfi], n_in: int, nchan: int):
    """Sparse additive signal (rows, cols, values) of the events, for
    ``synth.make_beam_torch(..., extra=...)``."""
    rows, cols, vals = [], [], []
    for e in events:
        t = np.arange(e.t0, min(n_in, e.t0 + e.dur), dtype=np.int64)
        if e.kind == "impulse":
            r = np.repeat(t, nchan)
            c = np.tile(np.arange(nchan, dtype=np.int64), t.size)
        elif e.kind == "narrowband":
            on = ((t - e.t0) % max(1.0, e.period)) < e.duty * e.period
            t = t[on]
            r = np.repeat(t, e.nch)
            c = np.tile(np.arange(e.c0, e.c0 + e.nch, dtype=np.int64), t.size)
        else:  # tone: centre channel drifts towards higher channel numbers (lower frequencies)
            on = ((t - e.t0) % max(1.0, e.period)) < e.duty * e.period
            t = t[on]
            centre = np.floor(e.c0 + e.drift * (t - e.t0)).astype(np.int64)
            r = np.repeat(t, e.nch)
            c = (centre[:, None] + np.arange(e.nch, dtype=np.int64)[None, :]).reshape(-1)
            keep = (c >= 0) & (c < nchan)
            r, c = r[keep], c[keep]
        rows.append(r)
        cols.append(c)
        vals.append(np.full(r.size, e.amp, np.float64))
    if not rows:
        z = np.zeros(0, np.int64)
        return z, z, np.zeros(0)
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)


def pipeline_beam(seed: int, out, freqs, n_out: int, widths, nbursts: int = 4, dm_lo: float = 50.0,
                  dm_hi: float = 1950.0, fwhm_lo: float = 1.0, fwhm_hi: float = 64.0, snr_lo: float = 6.0,
                  snr_hi: float = 50.0, nrfi_lo: int = 3, nrfi_hi: int = 6):
    """A beam for training and judging the classifier on the search's own
    candidates: fills ``out`` (uint8 CUDA tensor [n_in][nchan], n_in >=
    n_out + the sweep of dm_hi) with noise, ``nbursts`` dispersed bursts
    arriving in [64, n_out) and 3-6 RFI events anywhere in the input.
    Returns the bursts (amplitudes filled in)."""
    from . import draw_bursts, make_beam_torch
    rng = np.random.default_rng((seed, 7))
    bursts = draw_bursts(rng, nbursts, n_out, dm_lo, dm_hi, fwhm_lo, fwhm_hi, snr_lo, snr_hi)
    n_in, nchan = int(out.shape[0]), int(out.shape[1])
    events = draw_rfi(rng, int(rng.integers(nrfi_lo, nrfi_hi + 1)), n_in, nchan)
    make_beam_torch(seed, out, freqs, bursts, widths=widths, extra=rfi_signal(events, n_in, nchan))
    return bursts
