"""Seeded synthetic inputs for the SPOTLIGHT search hot path.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle's tests.  It holds the *inputs* only -- frequency axes, trial-DM lists,
boxcar widths and 8-bit filterbank beams with injected dispersed bursts -- and
none of the search arithmetic (no integer delay tables, no shift-and-sum, no
boxcar S/N).  Forward-modelling a dispersed burst needs the cold-plasma law
(arXiv 2606.27262 Sec. 3.1.1, Eq. 1); here it is applied as a fractional,
unrounded arrival time per channel, the physics of the sky, not the search.

Workload shapes follow the paper's Band-3 setup (300-500 MHz, 4096 channels,
1.31072 ms sampling, DM up to 2000 pc cm^-3; Sec. 2, Sec. 3.1.1):

* ``config1``: 256 ch, 8192 searched samples, DM 0..500 step 1, 3 bursts.
* ``config2``: 4096 ch, 131072 searched samples, DM 0..2000 on a
  0.1/0.2/0.5/1.0 step schedule, 20 bursts.

Noise is N(128, 16^2) rounded and clipped to [0, 255]; an optional
per-channel gain multiplies noise and signal alike.  Random numbers come from
NumPy's PCG64: noise from ``default_rng(seed)``, burst parameters from
``default_rng((seed, 1))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

TSAMP = 1.31072e-3          # s, Sec. 2
F_TOP = 500.0               # MHz, Band 3 top edge; channel 0
BANDWIDTH = 200.0           # MHz, Band 3
KDM_PHYS = 4.148808e3       # MHz^2 pc^-1 cm^3 s, Eq. 1 (rounded)
NOISE_MEAN = 128.0
NOISE_STD = 16.0


def band_freqs(nchan: int, f_top: float = F_TOP, bandwidth: float = BANDWIDTH) -> np.ndarray:
    """Channel frequencies in MHz, highest first: f_c = f_top - c*bw/nchan."""
    c = np.arange(nchan, dtype=np.float64)
    return f_top - c * (bandwidth / nchan)


def dm_range(lo: float, hi: float, step: float, include_hi: bool = False) -> np.ndarray:
    """DM_k = lo + k*step for lo + k*step < hi (k integer, no accumulation)."""
    n = int(math.floor((hi - lo) / step + 1e-9))
    k = np.arange(n, dtype=np.float64)
    v = lo + k * step
    v = v[v < hi - 1e-12]
    if include_hi:
        v = np.append(v, hi)
    return v


def dm_schedule(ranges, final: float | None = None) -> np.ndarray:
    """Concatenate half-open [lo, hi) sub-ranges with their own steps and
    optionally a final DM value (the plan layout of Sec. 3.1.1)."""
    parts = [dm_range(lo, hi, step) for lo, hi, step in ranges]
    if final is not None:
        parts.append(np.array([final], dtype=np.float64))
    return np.concatenate(parts)


def dm_plan_config1() -> np.ndarray:
    """0..500 pc cm^-3 in steps of 1 (501 trials)."""
    return np.arange(0, 501, dtype=np.float64)


def dm_plan_config2() -> np.ndarray:
    """0..2000 pc cm^-3: 0.1 over [0,250), 0.2 over [250,500), 0.5 over
    [500,1000), 1.0 over [1000,2000), then 2000 itself (5751 trials)."""
    return dm_schedule([(0.0, 250.0, 0.1), (250.0, 500.0, 0.2),
                        (500.0, 1000.0, 0.5), (1000.0, 2000.0, 1.0)], final=2000.0)


def dm_plan_upto(max_dm: float) -> np.ndarray:
    """The config-2 step schedule cut at ``max_dm`` (inclusive)."""
    full = dm_plan_config2()
    return full[full <= max_dm + 1e-9]


def widths_pow2(max_width: int) -> np.ndarray:
    """1, 2, 4, ... up to max_width."""
    out = [1]
    while out[-1] * 2 <= max_width:
        out.append(out[-1] * 2)
    return np.array(out, dtype=np.int32)


@dataclasses.dataclass
class Burst:
    t0: int            # arrival sample at the top channel (= searched sample index)
    dm: float          # pc cm^-3
    fwhm: float        # samples
    snr: float         # target best-boxcar S/N
    amp: float = 0.0   # per-channel peak amplitude in 8-bit units (before gain)


def fractional_delay(freqs_mhz: np.ndarray, dm: float, tsamp: float = TSAMP) -> np.ndarray:
    """Unrounded arrival-time offset (samples) of each channel w.r.t. the top
    channel for a burst at ``dm`` -- the forward model of Eq. 1."""
    f = np.asarray(freqs_mhz, dtype=np.float64)
    return KDM_PHYS * dm * (1.0 / (f * f) - 1.0 / (f[0] * f[0])) / tsamp


def _gauss_sigma(fwhm: float) -> float:
    return fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def burst_amplitude(snr: float, fwhm: float, widths, gains: np.ndarray) -> float:
    """Per-channel amplitude giving an ideal best-boxcar S/N of ``snr`` for a
    Gaussian pulse of this FWHM centred on a sample, summed over channels with
    the given gains, against white noise of std NOISE_STD*gain per channel."""
    sig = _gauss_sigma(fwhm)
    half = int(math.ceil(6 * sig)) + max(int(w) for w in widths) + 2
    s = np.arange(-half, half + 1, dtype=np.float64)
    g = np.exp(-0.5 * (s / sig) ** 2)
    csum = np.concatenate([[0.0], np.cumsum(g)])
    best = 0.0
    for w in widths:
        w = int(w)
        if w > g.size:
            continue
        win = csum[w:] - csum[:-w]
        best = max(best, float(win.max()) / math.sqrt(w))
    gsum = float(np.sum(gains))
    gnorm = float(np.sqrt(np.sum(gains * gains)))
    return snr * NOISE_STD * gnorm / (gsum * best)


def draw_bursts(rng: np.random.Generator, nbursts: int, n_out: int, dm_lo: float, dm_hi: float,
                fwhm_lo: float, fwhm_hi: float, snr_lo: float, snr_hi: float) -> list[Burst]:
    """Burst parameters: DM ~ U(dm_lo, dm_hi), FWHM ~ U(fwhm_lo, fwhm_hi),
    S/N ~ U(snr_lo, snr_hi); arrival samples at least 4*max FWHM + 64 apart
    and inside [64, n_out - 64 - 4*fwhm_hi]."""
    gap = int(4 * fwhm_hi + 64)
    lo, hi = 64, int(n_out - 64 - 4 * fwhm_hi)
    if nbursts == 0:
        return []
    if hi - lo < (nbursts - 1) * gap:
        raise ValueError("searched span too short for the requested bursts")
    # Distinct sorted slots with the required spacing: draw offsets in a
    # shrunken span and re-expand by the gap.
    span = hi - lo - (nbursts - 1) * gap
    offs = np.sort(rng.integers(0, span + 1, size=nbursts))
    t0s = lo + offs + np.arange(nbursts) * gap
    dms = rng.uniform(dm_lo, dm_hi, size=nbursts)
    fwhms = rng.uniform(fwhm_lo, fwhm_hi, size=nbursts)
    snrs = rng.uniform(snr_lo, snr_hi, size=nbursts)
    return [Burst(int(t), float(d), float(f), float(s)) for t, d, f, s in zip(t0s, dms, fwhms, snrs)]


def _burst_signal(bursts: list[Burst], freqs: np.ndarray, n_in: int, widths, g: np.ndarray, tsamp: float):
    """Sparse signal of the bursts: (rows, cols, values) sorted by row, for
    a band of samples around each channel's arrival time.  Fills in each
    burst's amplitude from its target S/N."""
    nchan = freqs.size
    sig_rows, sig_cols, sig_vals = [], [], []
    for b in bursts:
        b.amp = burst_amplitude(b.snr, b.fwhm, widths, g)
        sig = _gauss_sigma(b.fwhm)
        half = int(math.ceil(6 * sig)) + 1
        centre = b.t0 + fractional_delay(freqs, b.dm, tsamp)            # [nchan]
        base = np.floor(centre).astype(np.int64)
        k = np.arange(-half, half + 2, dtype=np.int64)
        rows = base[:, None] + k[None, :]                                # [nchan][K]
        vals = b.amp * np.exp(-0.5 * ((rows - centre[:, None]) / sig) ** 2)
        cols = np.broadcast_to(np.arange(nchan)[:, None], rows.shape)
        ok = (rows >= 0) & (rows < n_in)
        sig_rows.append(rows[ok]); sig_cols.append(cols[ok]); sig_vals.append(vals[ok])
    if sig_rows:
        sr = np.concatenate(sig_rows); sc = np.concatenate(sig_cols); sv = np.concatenate(sig_vals)
        order = np.argsort(sr, kind="stable")
        return sr[order], sc[order], sv[order]
    z = np.zeros(0, np.int64)
    return z, z, np.zeros(0)


def make_beam(seed: int, nchan: int, n_in: int, freqs: np.ndarray, bursts: list[Burst] | None = None,
              widths=(1,), gains: np.ndarray | None = None, tsamp: float = TSAMP,
              chunk_rows: int = 8192) -> np.ndarray:
    """uint8 filterbank [n_in][nchan] (time-major, channel 0 = highest
    frequency): x = clip(round(g_c * (128 + 16 z + signal)), 0, 255).  Burst
    amplitudes are filled in (``Burst.amp``) from their target S/N."""
    rng = np.random.default_rng(seed)
    freqs = np.asarray(freqs, dtype=np.float64)
    g = np.ones(nchan, np.float64) if gains is None else np.asarray(gains, np.float64)
    sr, sc, sv = _burst_signal(list(bursts or []), freqs, n_in, widths, g, tsamp)

    out = np.empty((n_in, nchan), dtype=np.uint8)
    gf = g.astype(np.float32)
    for r0 in range(0, n_in, chunk_rows):
        r1 = min(n_in, r0 + chunk_rows)
        z = rng.standard_normal(size=(r1 - r0, nchan), dtype=np.float32)
        v = z * np.float32(NOISE_STD) + np.float32(NOISE_MEAN)
        lo, hi = np.searchsorted(sr, r0), np.searchsorted(sr, r1)
        if hi > lo:
            np.add.at(v, (sr[lo:hi] - r0, sc[lo:hi]), sv[lo:hi].astype(np.float32))
        if gains is not None:
            v *= gf[None, :]
        np.rint(v, out=v)
        np.clip(v, 0, 255, out=v)
        out[r0:r1] = v.astype(np.uint8)
    return out


def make_beam_torch(seed: int, out, freqs: np.ndarray, bursts: list[Burst] | None = None, widths=(1,),
                    gains: np.ndarray | None = None, tsamp: float = TSAMP, chunk_rows: int = 16384,
                    extra=None):
    """The noise model of ``make_beam`` drawn on a torch device (for beams
    too large to draw on the host in reasonable time): fills ``out``, a
    uint8 tensor [n_in][nchan], in place.  Same distribution and burst
    model; a different random stream (torch's generator, seeded by
    ``seed``).  ``extra``: another sparse signal (rows, cols, values), e.g.
    RFI from ``synth.rfi.rfi_signal``, added before the gain and rounding."""
    import torch
    n_in, nchan = int(out.shape[0]), int(out.shape[1])
    dev = out.device
    freqs = np.asarray(freqs, dtype=np.float64)
    g = np.ones(nchan, np.float64) if gains is None else np.asarray(gains, np.float64)
    sr, sc, sv = _burst_signal(list(bursts or []), freqs, n_in, widths, g, tsamp)
    if extra is not None and len(extra[0]):
        sr, sc, sv = (np.concatenate([sr, extra[0]]), np.concatenate([sc, extra[1]]),
                      np.concatenate([sv, extra[2]]))
        order = np.argsort(sr, kind="stable")
        sr, sc, sv = sr[order], sc[order], sv[order]
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    gt = torch.as_tensor(g.astype(np.float32), device=dev)
    for r0 in range(0, n_in, chunk_rows):
        r1 = min(n_in, r0 + chunk_rows)
        v = torch.randn((r1 - r0, nchan), generator=gen, device=dev, dtype=torch.float32)
        v.mul_(NOISE_STD).add_(NOISE_MEAN)
        lo, hi = np.searchsorted(sr, r0), np.searchsorted(sr, r1)
        if hi > lo:
            idx = (torch.as_tensor(sr[lo:hi] - r0, device=dev), torch.as_tensor(sc[lo:hi], device=dev))
            v.index_put_(idx, torch.as_tensor(sv[lo:hi].astype(np.float32), device=dev), accumulate=True)
        if gains is not None:
            v.mul_(gt[None, :])
        v.round_().clamp_(0, 255)
        out[r0:r1].copy_(v.to(torch.uint8))
    return out


@dataclasses.dataclass
class Workload:
    name: str
    nchan: int
    n_out: int
    freqs: np.ndarray
    dms: np.ndarray
    widths: np.ndarray
    threshold: float
    norm_block: int
    seed: int
    nbursts: int
    dm_lo: float
    dm_hi: float
    fwhm_lo: float = 1.0
    fwhm_hi: float = 16.0
    snr_lo: float = 8.0
    snr_hi: float = 30.0
    tsamp: float = TSAMP


def config1() -> Workload:
    """Single beam, plain method: 256 ch, 8192 samples, 501 DMs, widths 1..32."""
    return Workload("single beam 256ch x 8192 samples, DM 0-500 step 1 (501 trials), widths 1-32",
                    256, 8192, band_freqs(256), dm_plan_config1(), widths_pow2(32), 6.0, 8192,
                    1001, 3, 50.0, 450.0)


def config2() -> Workload:
    """Single beam at full size: 4096 ch, 131072 samples, 5751 DMs, widths 1..256."""
    return Workload("single beam 4096ch x 131072 samples, DM 0-2000 step schedule (5751 trials), widths 1-256",
                    4096, 131072, band_freqs(4096), dm_plan_config2(), widths_pow2(256), 6.0, 8192,
                    1002, 20, 50.0, 1950.0)


def make_workload_beam(wl: Workload, n_in: int, seed: int | None = None):
    """Filterbank + bursts for a workload, ``n_in`` = n_out + max delay."""
    s = wl.seed if seed is None else seed
    brng = np.random.default_rng((s, 1))
    bursts = draw_bursts(brng, wl.nbursts, wl.n_out, wl.dm_lo, wl.dm_hi, wl.fwhm_lo,
                         wl.fwhm_hi, wl.snr_lo, wl.snr_hi)
    data = make_beam(s, wl.nchan, n_in, wl.freqs, bursts, widths=wl.widths, tsamp=wl.tsamp)
    return data, bursts


@dataclasses.dataclass
class BatchWorkload:
    """Many beams of uneven length and DM range searched as one batch."""
    name: str
    nchan: int
    freqs: np.ndarray
    plan_dms: list            # DM list per plan
    beam_plan: np.ndarray     # int32 [nbeams] plan index
    n_out: np.ndarray         # int64 [nbeams]
    widths: np.ndarray
    threshold: float
    norm_block: int
    seed: int
    nbursts: int              # per beam
    fwhm_lo: float = 1.0
    fwhm_hi: float = 16.0
    snr_lo: float = 8.0
    snr_hi: float = 30.0
    tsamp: float = TSAMP

    @property
    def nbeams(self) -> int:
        return int(self.n_out.size)

    def beam_seed(self, b: int) -> int:
        return int(np.random.SeedSequence((self.seed, int(b))).generate_state(1)[0])

    def gains(self, b: int) -> np.ndarray:
        """Bandpass gain of beam b: U(0.5, 1.5) per channel."""
        return np.random.default_rng((self.seed, int(b), 2)).uniform(0.5, 1.5, self.nchan)

    def bursts(self, b: int) -> list[Burst]:
        """Bursts of beam b: DM U(50, max DM - 50) of its plan, FWHM, S/N and
        spacing as in the single-beam workloads."""
        brng = np.random.default_rng((self.seed, int(b), 1))
        hi = float(self.plan_dms[int(self.beam_plan[b])][-1]) - 50.0
        return draw_bursts(brng, self.nbursts, int(self.n_out[b]), 50.0, hi, self.fwhm_lo, self.fwhm_hi,
                           self.snr_lo, self.snr_hi)


def config3(nbeams: int = 128, n_lo: int = 16384, n_hi: int = 131072, nchan: int = 4096,
            max_dms=(500.0, 1000.0, 2000.0)) -> BatchWorkload:
    """Batched: 128 beams of 4096 ch, lengths U{16384..131072}, max DM per
    beam from {500, 1000, 2000} (the config-2 step schedule cut there),
    per-channel gains U(0.5, 1.5), 4 bursts per beam, widths 1..256."""
    rng = np.random.default_rng(1003)
    n_out = rng.integers(n_lo, n_hi + 1, size=nbeams).astype(np.int64)
    beam_plan = rng.integers(0, len(max_dms), size=nbeams).astype(np.int32)
    plan_dms = [dm_plan_upto(m) for m in max_dms]
    return BatchWorkload(f"{nbeams} beams x {nchan}ch, n_out U{{{n_lo}..{n_hi}}}, max DM in "
                         f"{{{', '.join(str(int(m)) for m in max_dms)}}}, gains U(0.5,1.5), widths 1-256",
                         nchan, band_freqs(nchan), plan_dms, beam_plan, n_out, widths_pow2(256), 6.0, 8192,
                         1003, 4)


def burst_signal(freqs: np.ndarray, n_in: int, bursts: list[Burst], widths=(1,), gains: np.ndarray | None = None,
                 tsamp: float = TSAMP) -> np.ndarray:
    """The bursts of ``make_beam`` alone, as a dense float32 [n_in][nchan]
    signal in the units of the 8-bit samples (before gain and quantisation):
    the input of an injection into already-quantised data."""
    freqs = np.asarray(freqs, dtype=np.float64)
    g = np.ones(freqs.size, np.float64) if gains is None else np.asarray(gains, np.float64)
    sr, sc, sv = _burst_signal(list(bursts), freqs, n_in, widths, g, tsamp)
    out = np.zeros((n_in, freqs.size), np.float32)
    np.add.at(out, (sr, sc), sv.astype(np.float32))
    return out
