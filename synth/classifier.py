"""Seeded synthetic candidates for the classifier (test and bench inputs).

Each example is a subband dynamic spectrum sub[256][t_in] as the feature
extractor sees it after dedispersion at the candidate DM within each subband:
unit-variance Gaussian noise per (subband, time bin) plus one of

* an astrophysical burst (label 1): a Gaussian pulse (FWHM 1-16 bins,
  log-uniform) whose residual dispersion sweep across the band is within
  +-12 bins (the candidate DM is near the true DM), with a random smooth
  spectral envelope, band-limited to 25-100 % of the band in 30 % of the
  bursts, scaled to a target band-summed boxcar S/N;
* RFI or noise (label 0), one of: persistent narrowband channels (1-12
  subbands with a constant or slowly modulated offset), a broadband impulse
  seen through the wrong DM (flat spectrum, residual sweep -30 to -128 bins,
  as a DM-0 impulse dedispersed at a positive DM), a periodic tone drifting
  across a block of subbands, or pure noise.

Residual sweeps follow Eq. 1 across the subband centre frequencies.  The
draws come from a numpy Generator; the arrays are built with torch on the
given device.  Nothing here computes a feature or a network output.
"""
from __future__ import annotations

import numpy as np

NSUB = 256


def sweep_fraction(freqs_mhz, nsub: int = NSUB) -> np.ndarray:
    """(f_s^-2 - f_top^-2) / (f_last^-2 - f_top^-2) per subband centre."""
    f = np.asarray(freqs_mhz, np.float64).reshape(nsub, -1).mean(axis=1)
    g = 1.0 / (f * f)
    return (g - g[0]) / (g[-1] - g[0])


def _boxcar_gain(fwhm: float) -> float:
    """max over widths 1..64 of (sum of a unit-peak Gaussian over the best
    window) / sqrt(width)."""
    sig = fwhm / 2.3548200450309493
    half = int(np.ceil(6 * sig)) + 66
    t = np.arange(-half, half + 1, dtype=np.float64)
    g = np.exp(-0.5 * (t / sig) ** 2)
    c = np.concatenate([[0.0], np.cumsum(g)])
    best = 0.0
    w = 1
    while w <= 64:
        best = max(best, float((c[w:] - c[:-w]).max()) / np.sqrt(w))
        w *= 2
    return best


def classifier_batch(rng: np.random.Generator, n: int, freqs_mhz, device="cuda", t_in: int = 512,
                     p_burst: float = 0.5, snr_lo: float = 6.0, snr_hi: float = 50.0, kinds=None):
    """(sub float32 tensor [n][256][t_in], labels float32 [n], meta dict of
    per-example arrays: kind (0 burst, 1 narrowband, 2 impulse, 3 tone,
    4 noise) and snr)."""
    import torch
    frac = torch.as_tensor(sweep_fraction(freqs_mhz), dtype=torch.float32, device=device)  # [S]
    S, T = NSUB, t_in
    if kinds is None:
        kinds = np.where(rng.random(n) < p_burst, 0, rng.integers(1, 5, n))
    kinds = np.asarray(kinds)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(rng.integers(0, 2**62)))
    sub = torch.randn((n, S, T), generator=gen, device=device, dtype=torch.float32)
    tt = torch.arange(T, device=device, dtype=torch.float32)
    ss = torch.arange(S, device=device, dtype=torch.float32)
    snr = np.zeros(n)

    def pulses(idx, t_c, sweep, fwhm, amp_s):
        # amp_s [m][S] peak amplitude per subband; arrival t_c + sweep * frac
        t_c = torch.as_tensor(t_c, dtype=torch.float32, device=device)
        sweep = torch.as_tensor(sweep, dtype=torch.float32, device=device)
        sig = torch.as_tensor(np.asarray(fwhm) / 2.3548200450309493, dtype=torch.float32, device=device)
        arr = t_c[:, None] + sweep[:, None] * frac[None, :]                     # [m][S]
        prof = torch.exp(-0.5 * ((tt[None, None, :] - arr[:, :, None]) / sig[:, None, None]) ** 2)
        sub[idx] += prof * torch.as_tensor(amp_s, dtype=torch.float32, device=device)[:, :, None]

    # bursts
    b = np.flatnonzero(kinds == 0)
    if b.size:
        m = b.size
        fwhm = np.exp(rng.uniform(0.0, np.log(16.0), m))
        snr[b] = rng.uniform(snr_lo, snr_hi, m)
        k = rng.uniform(0.5, 3.0, m)
        ph = rng.uniform(0, 2 * np.pi, m)
        s_axis = np.arange(S) / S
        env = np.maximum(0.0, 1.0 + 0.6 * np.sin(2 * np.pi * k[:, None] * s_axis[None, :] + ph[:, None]))
        lim = rng.random(m) < 0.3
        for i in np.flatnonzero(lim):
            width = int(rng.integers(S // 4, S + 1))
            lo = int(rng.integers(0, S - width + 1))
            mask = np.zeros(S)
            mask[lo:lo + width] = 1.0
            env[i] *= mask
        env = np.where(env.sum(axis=1, keepdims=True) > 0, env, 1.0)
        gain = np.array([_boxcar_gain(f) for f in fwhm])
        # band sum has noise sqrt(S) per bin
        amp = snr[b] * np.sqrt(S) / (env.sum(axis=1) * gain)
        pulses(b, T / 2 + rng.uniform(-3, 3, m), rng.uniform(-12, 12, m), fwhm, amp[:, None] * env)
    # narrowband persistent channels
    a = np.flatnonzero(kinds == 1)
    for i in a:
        nb = int(rng.integers(1, 13))
        chans = rng.choice(S, nb, replace=False)
        lvl = rng.uniform(1.0, 6.0, nb)
        per = rng.uniform(8.0, 200.0)
        mod = 1.0 + 0.5 * torch.sin(2 * np.pi * tt / per + float(rng.uniform(0, 2 * np.pi)))
        sub[i, torch.as_tensor(chans, device=device)] += torch.as_tensor(lvl, dtype=torch.float32,
                                                                        device=device)[:, None] * mod[None, :]
    # broadband impulses through the wrong DM
    c = np.flatnonzero(kinds == 2)
    if c.size:
        m = c.size
        fwhm = rng.uniform(1.0, 3.0, m)
        snr[c] = rng.uniform(10.0, snr_hi, m)
        amp = snr[c] * np.sqrt(S) / (S * np.array([_boxcar_gain(f) for f in fwhm]))
        pulses(c, T / 2 + rng.uniform(-3, 3, m), -rng.uniform(30, 128, m), fwhm, np.repeat(amp[:, None], S, 1))
    # drifting periodic tones
    d = np.flatnonzero(kinds == 3)
    for i in d:
        width = int(rng.integers(10, 61))
        lo = int(rng.integers(0, S - width + 1))
        per = rng.uniform(3.0, 40.0)
        drift = rng.uniform(-0.05, 0.05)
        amp = rng.uniform(0.5, 2.0)
        band = ss[lo:lo + width]
        sub[i, lo:lo + width] += amp * torch.sin(2 * np.pi * (tt[None, :] / per + drift * band[:, None]))
    labels = (kinds == 0).astype(np.float32)
    return sub, labels, {"kind": kinds, "snr": snr}
