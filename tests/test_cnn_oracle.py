"""The classifier's oracle (arXiv 2606.27262, Sec. 3.2.2) pinned to
independent facts: the convolution equals scipy's 2-D correlation sampled
at stride 2; gradients equal central finite differences of the loss; Adam's
first step has its closed form; the subband shift table follows Eq. 1 and is
what the library's host code computes.  No GPU needed."""
import numpy as np
import pytest

import paper_2606_27262_gb300 as sp
import synth
from oracle import cnn as ocnn
from paper_2606_27262_gb300 import build as spbuild


@pytest.fixture(scope="module", autouse=True)
def _built():
    spbuild.build()


def test_conv_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 12, 10, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    z = ocnn.conv(x, w, b)
    assert z.shape == (2, 6, 5, 4)
    for n in range(2):
        for o in range(4):
            ref = sum(signal.correlate2d(x[n, :, :, c], w[o, :, :, c], mode="same") for c in range(3))
            assert np.allclose(z[n, :, :, o], ref[::2, ::2] + b[o], atol=1e-12)


def he_params(rng):
    """He-normal convolution weights, small biases and heads (flat order)."""
    parts = []
    for _ in range(2):
        for ci, co in zip(ocnn.CIN, ocnn.COUT):
            parts += [rng.normal(0, np.sqrt(2 / (9 * ci)), co * 9 * ci), rng.normal(0, 0.05, co)]
        parts += [rng.normal(0, 1 / 16, ocnn.FEAT), rng.normal(0, 0.1, 1)]
    return np.concatenate(parts)


def _small_problem(rng, n=3, h=32):
    p = he_params(rng)
    ft = rng.normal(size=(n, h, h))
    dmt = rng.normal(size=(n, h, h))
    y = np.array([1.0, 0.0, 1.0][:n])
    return p, ft, dmt, y


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p, ft, dmt, y = _small_problem(rng)
    _, loss, g = ocnn.forward_backward(p, ft, dmt, y, round_bf16=False)
    idx = rng.choice(p.size, 60, replace=False)
    # include every head parameter and the first layer of each branch
    nb = ocnn.num_params_branch()
    idx = np.unique(np.concatenate([idx, [nb - 1, 2 * nb - 1, nb - 2, 0, nb]]))
    h = 1e-6
    rel = []
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        lp = ocnn.forward_backward(p + e, ft, dmt, y, round_bf16=False)[1]
        lm = ocnn.forward_backward(p - e, ft, dmt, y, round_bf16=False)[1]
        fd = (lp - lm) / (2 * h)
        rel.append(abs(fd - g[i]) / max(abs(fd), abs(g[i]), 1e-9))
    rel = np.array(rel)
    assert np.median(rel) < 1e-5 and np.mean(rel < 1e-3) >= 0.95, rel.max()
    assert np.isfinite(loss) and loss > 0


def test_fused_probability_and_loss_closed_form():
    rng = np.random.default_rng(2)
    p, ft, dmt, y = _small_problem(rng)
    prob = ocnn.forward_backward(p, ft, dmt, None, round_bf16=False)
    _, loss, _ = ocnn.forward_backward(p, ft, dmt, y, round_bf16=False)
    assert ((prob > 0) & (prob < 1)).all()
    assert np.isclose(loss, np.mean(-(y * np.log(prob) + (1 - y) * np.log(1 - prob))))
    # zero weights: each branch logit is its head bias -> p = s(b1) s(b2)
    z = np.zeros_like(p)
    nb = ocnn.num_params_branch()
    z[nb - 1], z[2 * nb - 1] = 0.3, -1.1
    pz = ocnn.forward_backward(z, ft, dmt, None, round_bf16=False)
    assert np.allclose(pz, 1 / (1 + np.exp(-0.3)) / (1 + np.exp(1.1)))


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    w, g = rng.normal(size=50), rng.normal(size=50)
    w1, m, v = ocnn.adam(w, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties go to even (1)
    assert ocnn.bf16(1 + 2 ** -8) == 1.0
    assert ocnn.bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6
    assert ocnn.bf16(-2.5) == -2.5
    x = np.random.default_rng(4).normal(size=1000)
    assert (np.abs(ocnn.bf16(x) - x) <= np.abs(x) * 2 ** -8).all()


def test_dmt_shift_table_library_equals_oracle():
    f = synth.band_freqs(4096)
    got = sp.dmt_shifts(f, 256, 128)
    want = ocnn.dmt_shifts(f, 256, 128)
    assert np.array_equal(got, want)
    assert (got[:, 0] == 0).all() and got[0, -1] == -128 and got[-1, -1] == 128
    assert np.array_equal(got[::-1], -got)  # rows are symmetric sweeps
    # the residual delay of Eq. 1 grows monotonically down the band
    assert (np.diff(got[-1]) >= 0).all()


def test_feature_oracle_aligns_a_swept_pulse():
    f = synth.band_freqs(4096)
    sh = ocnn.dmt_shifts(f, 256, 128)
    frac = (1 / f.reshape(256, -1).mean(1) ** 2 - 1 / f[:16].mean() ** 2)
    frac = frac / frac[-1]
    sub = np.zeros((1, 256, 512))
    sweep = 40.0
    for s in range(256):
        sub[0, s, 128 + 30 + int(round(sweep * frac[s]))] = 1.0  # crop starts at (512 - 256) / 2
    ft, dmt = ocnn.features(sub, sh)
    j, u = np.unravel_index(np.argmax(dmt[0]), dmt[0].shape)
    assert u == 30 and abs(128 * (2 * j / 255 - 1) - sweep) <= 1.0
