"""Pins of the classifier's oracle (oracle/cnn.py; arXiv 2606.27262,
Sec. 3.2.2 classification, and the candidate features of Sec. 3.2.1-3.2.2).

Every pin takes the oracle module as its argument so that the mutation tests
can run the same pins against copies of the oracle with planted mistakes.
Each pin checks the oracle against something other than itself: scipy's
2-D correlation, central finite differences, closed forms worked out by hand
(Adam's first step, the fused probability, standardised impulse and step
images), a shift table computed by hand from Eq. 1, or the rounding rules of
bfloat16.  None of them calls the CUDA library."""
from __future__ import annotations

import math

import numpy as np

import synth


# ------------------------------------------------------------- network --
def pin_conv_matches_scipy_correlate(m):
    """A 3x3, stride-2, zero-padded convolution is scipy's 'same' 2-D
    correlation sampled at every second row and column, plus the bias."""
    try:
        from scipy import signal
    except ImportError:  # the GPU machine has scipy; without it this pin is vacuous
        return
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 12, 10, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    z = m.conv(x, w, b)
    assert z.shape == (2, 6, 5, 4)
    for n in range(2):
        for o in range(4):
            ref = sum(signal.correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same") for c in range(3))
            assert np.allclose(z[n, :, :, o], ref[::2, ::2] + b[o], atol=1e-12)


def he_params(m, rng):
    """He-normal convolution weights, small biases and heads (flat order)."""
    parts = []
    for _ in range(2):
        for ci, co in zip(m.CIN, m.COUT):
            parts += [rng.normal(0, np.sqrt(2 / (9 * ci)), co * 9 * ci), rng.normal(0, 0.05, co)]
        parts += [rng.normal(0, 1 / 16, m.FEAT), rng.normal(0, 0.1, 1)]
    return np.concatenate(parts)


def small_problem(m, rng, n=3, h=32):
    p = he_params(m, rng)
    ft = rng.normal(size=(n, h, h))
    dmt = rng.normal(size=(n, h, h))
    y = np.array([1.0, 0.0, 1.0][:n])
    return p, ft, dmt, y


def pin_gradients_match_finite_differences(m):
    """Every analytic gradient the oracle returns (a sample of 60 parameters
    plus both heads and the first weight of each branch) equals the central
    finite difference of its loss."""
    rng = np.random.default_rng(1)
    p, ft, dmt, y = small_problem(m, rng)
    _, loss, g = m.forward_backward(p, ft, dmt, y, round_bf16=False)
    idx = rng.choice(p.size, 60, replace=False)
    nb = m.num_params_branch()
    idx = np.unique(np.concatenate([idx, [nb - 1, 2 * nb - 1, nb - 2, 0, nb]]))
    h = 1e-6
    rel = []
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp = m.forward_backward(p + e, ft, dmt, y, round_bf16=False)[1]
        lm = m.forward_backward(p - e, ft, dmt, y, round_bf16=False)[1]
        fd = (lp - lm) / (2 * h)
        rel.append(abs(fd - g[i]) / max(abs(fd), abs(g[i]), 1e-9))
    rel = np.array(rel)
    assert np.median(rel) < 1e-5 and np.mean(rel < 1e-3) >= 0.95, rel.max()
    assert np.isfinite(loss) and loss > 0


def pin_fused_probability_and_loss_closed_form(m):
    """p = sigmoid(l_ft) * sigmoid(l_dmt) (FETCH's fusion of the two
    branches); the loss is the mean binary cross-entropy of p.  With all
    weights zero each logit is its head bias."""
    rng = np.random.default_rng(2)
    p, ft, dmt, y = small_problem(m, rng)
    prob = m.forward_backward(p, ft, dmt, None, round_bf16=False)
    _, loss, _ = m.forward_backward(p, ft, dmt, y, round_bf16=False)
    assert ((prob > 0) & (prob < 1)).all()
    assert np.isclose(loss, np.mean(-(y * np.log(prob) + (1 - y) * np.log(1 - prob))))
    z = np.zeros_like(p)
    nb = m.num_params_branch()
    z[nb - 1], z[2 * nb - 1] = 0.3, -1.1
    pz = m.forward_backward(z, ft, dmt, None, round_bf16=False)
    assert np.allclose(pz, 1 / (1 + np.exp(-0.3)) / (1 + np.exp(1.1)))
    # Zero convolution weights and positive biases: every layer outputs its
    # ReLU'd bias everywhere, so on 64 x 64 images the last 2 x 2 map is
    # constant and global average pooling gives relu(b5) itself (a sum would
    # give four times it): logit = head_w . relu(b5) + head_b per branch.
    z = np.zeros_like(p)
    nb = m.num_params_branch()
    heads = []
    for br in range(2):
        k = br * nb
        for ci, co in zip(m.CIN, m.COUT):
            k += co * 9 * ci
            z[k:k + co] = rng.uniform(0.1, 0.5, co)
            k += co
        b5 = z[k - m.COUT[-1]:k]
        z[k:k + m.FEAT] = rng.normal(0, 0.05, m.FEAT)
        z[k + m.FEAT] = 0.2 - br
        heads.append(float(z[k:k + m.FEAT] @ b5) + 0.2 - br)
    img = rng.normal(size=(2, 64, 64))
    pz = m.forward_backward(z, img, img, None, round_bf16=False)
    assert np.allclose(pz, 1 / (1 + np.exp(-heads[0])) / (1 + np.exp(-heads[1])), rtol=1e-12)


def pin_adam_first_step_closed_form(m):
    """From zero moments Adam's first step is w - lr * g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    w, g = rng.normal(size=50), rng.normal(size=50)
    w1, mo, v = m.adam(w, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8))
    assert np.allclose(mo, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # second step with the same gradient: bias-corrected moments are still g, g^2
    w2, _, _ = m.adam(w1, g, mo, v, 2, 1e-3)
    assert np.allclose(w2, w1 - 1e-3 * g / (np.abs(g) + 1e-8))
    # a gradient far below eps: the step is lr * g / (|g| + eps), eps outside
    # the square root (1e-9 / 1.1e-8 of lr, not 1e-9 / 1e-4)
    w3, _, _ = m.adam(np.zeros(1), np.array([1e-9]), np.zeros(1), np.zeros(1), 1, 1.0)
    assert abs(w3[0] + 1e-9 / 1.1e-8) < 1e-12, w3


def pin_bf16_rounding(m):
    """bfloat16 keeps 8 significant bits, rounding to nearest with ties to
    even."""
    assert m.bf16(1 + 2 ** -8) == 1.0  # a tie between 1 and 1 + 2^-7: even is 1
    assert m.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6  # a tie between 1 + 2^-7 and 1 + 2^-6
    assert m.bf16(1 + 2 ** -8 + 2 ** -12) == 1 + 2 ** -7  # above the tie
    assert m.bf16(-2.5) == -2.5
    x = np.random.default_rng(4).normal(size=1000)
    assert (np.abs(m.bf16(x) - x) <= np.abs(x) * 2 ** -8).all()


# ------------------------------------------------------------ features --
# Eight channels whose four two-channel subbands have mean frequencies 1,
# 0.5, 0.25 and 0.125 (arbitrary units, exact in binary): 1/f^2 = 1, 4, 16,
# 64, so Eq. 1's residual delay across the band is in proportion to
# (1/f^2 - 1) / 63 = 0, 1/21, 5/21, 1 for the four subbands.
HAND_FREQS = np.array([1.125, 0.875, 0.625, 0.375, 0.3125, 0.1875, 0.15625, 0.09375])
# Three rows sweeping -44.5, 0 and +44.5 bins across the band:
#   subband 1: 44.5/21 = 2.119 -> 2;  subband 2: 44.5*5/21 = 10.595 -> 11;
#   subband 3: 44.5, an exact half, rounded away from zero -> 45 (rounding
#   half up would give -44 on the first row, ties-to-even 44 on both).
# Taking each subband's first channel instead of its mean gives 10, not 11.
HAND_SHIFTS = np.array([[0, -2, -11, -45], [0, 0, 0, 0], [0, 2, 11, 45]])


def pin_dmt_shifts_hand_table(m):
    got = m.dmt_shifts(HAND_FREQS, 4, 44.5, rows=3)
    assert np.array_equal(got, HAND_SHIFTS), got


def pin_dmt_shifts_band_structure(m):
    """On the 4096-channel band: no shift in the top subband, the bottom
    subband sweeps the full +-max_sweep, rows are mirror images, and the
    residual delay grows monotonically down the band (Eq. 1)."""
    got = m.dmt_shifts(synth.band_freqs(4096), 256, 128)
    assert got.shape == (256, 256)
    assert (got[:, 0] == 0).all() and got[0, -1] == -128 and got[-1, -1] == 128
    assert np.array_equal(got[::-1], -got)
    assert (np.diff(got[-1]) >= 0).all() and (np.diff(got[0]) <= 0).all()


def _impulse_sub(t, background=7.0, amp=5.0, k=1, col=7):
    """Four subbands x t bins of a constant plus one impulse at subband k,
    crop column col (the crop starts at (t - 256) // 2)."""
    sub = np.full((1, 4, t), background)
    sub[0, k, (t - 256) // 2 + col] += amp
    return sub


def pin_features_impulse_closed_form(m):
    """A constant plus one impulse.  An image of M values of which K are
    raised by the same amount standardises (zero mean, population variance
    1 over the whole image) to sqrt((M-K)/K) at the raised values and
    -sqrt(K/(M-K)) elsewhere.  Frequency-time image: 4 x 256 values, the
    impulse alone at crop column 7 of subband 1 (M = 1024, K = 1).  DM-time
    image with the hand shift table: row j sums subband k at column
    u + shift[j][k], so the impulse lands at column 7 - shift[j][1] of every
    row (M = 768, K = 3) over a constant background of 4 x 7."""
    t = 346  # crop [45, 301): every read shifted by up to +-45 stays inside
    ft, dmt = m.features(_impulse_sub(t), HAND_SHIFTS)
    assert ft.shape == (1, 4, 256) and dmt.shape == (1, 3, 256)
    want_ft = np.full((4, 256), -math.sqrt(1 / 1023))
    want_ft[1, 7] = math.sqrt(1023)
    assert np.allclose(ft[0], want_ft, rtol=1e-12, atol=1e-12)
    want_dmt = np.full((3, 256), -math.sqrt(3 / 765))
    for j in range(3):
        want_dmt[j, 7 - HAND_SHIFTS[j, 1]] = math.sqrt(765 / 3)
    assert np.allclose(dmt[0], want_dmt, rtol=1e-12, atol=1e-12)


def pin_features_dmt_sums_subbands(m):
    """Two equal impulses, in subbands 0 and 2, with the second 11 bins
    later: DM-time row 2 (shifts 0 and 11) adds them into one value 2a at
    column 7, rows 0 and 1 see them apart (columns 7 and 18 + 11 = 29 in row
    0, 7 and 18 in row 1).  Relative to the background the image holds four
    values a, one 2a and 763 zeros; its standardised values follow from the
    mean 6a/768 and the population variance 8a^2/768 - (6a/768)^2."""
    t = 346
    u0 = (t - 256) // 2
    a = 2.0
    sub = np.full((1, 4, t), 1.5)
    sub[0, 0, u0 + 7] += a
    sub[0, 2, u0 + 18] += a
    _, dmt = m.features(sub, HAND_SHIFTS)
    mean = 6 * a / 768
    sd = math.sqrt(8 * a * a / 768 - mean * mean)
    raw = np.zeros((3, 256))
    raw[0, 7] = raw[0, 29] = a
    raw[1, 7] = raw[1, 18] = a
    raw[2, 7] = 2 * a
    assert np.allclose(dmt[0], (raw - mean) / sd, rtol=1e-12, atol=1e-12)


def pin_features_step_and_crop(m):
    """A two-level step at crop column 128 (values 0 before, 3 from there on)
    standardises to exactly -1 and +1, half and half; the crop is the centre
    256 bins, starting at (t - 256) // 2 (a crop shifted by one bin leaves
    127 or 129 raised columns and values other than +-1)."""
    for t in (300, 301):
        u0 = (t - 256) // 2
        sub = np.zeros((2, 4, t))
        sub[:, :, u0 + 128:] = 3.0
        ft, _ = m.features(sub, np.zeros((1, 4), np.int64))
        want = np.concatenate([-np.ones(128), np.ones(128)])
        for n in range(2):
            for s in range(4):
                assert np.allclose(ft[n, s], want, rtol=0, atol=1e-12), (t, n, s)


def pin_features_zero_sigma(m):
    """An image with no variance (a constant subband spectrum) is all zeros,
    and one example's statistics do not leak into another's."""
    sub = np.stack([np.full((4, 346), 2.5), _impulse_sub(346)[0]])
    ft, dmt = m.features(sub, HAND_SHIFTS)
    assert np.array_equal(ft[0], np.zeros((4, 256))) and np.array_equal(dmt[0], np.zeros((3, 256)))
    assert np.isclose(ft[1].max(), math.sqrt(1023))


def pin_features_align_a_swept_pulse(m):
    """A pulse swept by +40 bins across the band (per subband in proportion
    to Eq. 1's f^-2 - f_top^-2) is straightened by the DM-time row whose
    sweep is nearest +40 and lands at its arrival column."""
    f = synth.band_freqs(4096)
    sh = m.dmt_shifts(f, 256, 128)
    frac = (1 / f.reshape(256, -1).mean(1) ** 2 - 1 / f[:16].mean() ** 2)
    frac = frac / frac[-1]
    sub = np.zeros((1, 256, 512))
    sweep = 40.0
    for s in range(256):
        sub[0, s, 128 + 30 + int(round(sweep * frac[s]))] = 1.0
    ft, dmt = m.features(sub, sh)
    j, u = np.unravel_index(np.argmax(dmt[0]), dmt[0].shape)
    assert u == 30 and abs(128 * (2 * j / 255 - 1) - sweep) <= 1.0


ALL_CNN_PINS = [
    pin_conv_matches_scipy_correlate, pin_gradients_match_finite_differences,
    pin_fused_probability_and_loss_closed_form, pin_adam_first_step_closed_form, pin_bf16_rounding,
    pin_dmt_shifts_hand_table, pin_dmt_shifts_band_structure, pin_features_impulse_closed_form,
    pin_features_dmt_sums_subbands, pin_features_step_and_crop, pin_features_zero_sigma, pin_features_align_a_swept_pulse,
]
