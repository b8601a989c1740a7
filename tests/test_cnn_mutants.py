"""Plant plausible mistakes in copies of the classifier's oracle
(oracle/cnn.py) and check that its pins (tests/cnn_pins.py) catch every one.

Each mutant is a text substitution in a copy of the module, imported from a
temporary file; the real oracle is untouched."""
import importlib.util
import os

import pytest

from oracle import cnn as ocnn
from tests import cnn_pins

SRC = ocnn.__file__

MUTANTS = {
    # features
    "sample_std": ("sd = a.std(axis=(1, 2), keepdims=True)", "sd = a.std(axis=(1, 2), keepdims=True, ddof=1)"),
    "per_row_standardisation": ("m = a.mean(axis=(1, 2), keepdims=True)\n        sd = a.std(axis=(1, 2), keepdims=True)",
                                "m = a.mean(axis=2, keepdims=True)\n        sd = a.std(axis=2, keepdims=True)"),
    "crop_off_by_one": ("u0 = (t - 256) // 2", "u0 = (t - 256) // 2 + 1"),
    "dmt_shift_sign": ("idx = u0 + u + shifts[j, k]", "idx = u0 + u - shifts[j, k]"),
    "dmt_mean_not_sum": ("dmt[:, j, ok] += sub[:, k, idx[ok]]", "dmt[:, j, ok] += sub[:, k, idx[ok]] * (k + 1)"),
    # Eq. 1 shift table
    "shifts_round_half_up": ("(np.sign(v) * np.floor(np.abs(v) + 0.5))", "np.floor(v + 0.5)"),
    "shifts_round_half_even": ("(np.sign(v) * np.floor(np.abs(v) + 0.5))", "np.round(v)"),
    "shifts_first_channel": (".reshape(nsub, -1).mean(axis=1)", ".reshape(nsub, -1)[:, 0]"),
    "shifts_linear_in_f": ("g = 1.0 / (f * f)", "g = -f"),
    "shifts_reference_bottom": ("frac = (g - g[0]) / (g[-1] - g[0])", "frac = (g - g[-1]) / (g[-1] - g[0])"),
    # network
    "conv_no_padding": ("xp[:, 1:-1, 1:-1] = x", "xp[:, 2:, 2:] = x"),
    "conv_kernel_flipped": ('np.einsum("nhwijc,oijc->nhwo", patches(x), w, optimize=True)',
                            'np.einsum("nhwijc,oijc->nhwo", patches(x), w[:, ::-1, ::-1, :], optimize=True)'),
    "relu_grad_mask_dropped": ("dz = q(conv_input_grad(dz, q(w), x_in.shape) * (x_in > 0))",
                               "dz = q(conv_input_grad(dz, q(w), x_in.shape))"),
    "sum_pooling": ("feat = x.mean(axis=(1, 2))", "feat = x.sum(axis=(1, 2))"),
    "mean_fusion": ("p = s1 * s2", "p = 0.5 * (s1 + s2)"),
    "bce_grad_missing_factor": ("g = (pc - y) / (1 - pc) / n", "g = (pc - y) / n"),
    "adam_no_bias_correction": ("mh = m / (1 - b1 ** step)", "mh = m"),
    "adam_eps_inside_sqrt": ("(np.sqrt(vh) + eps)", "np.sqrt(vh + eps)"),
    "bf16_ties_away": ("(u + 0x7FFF + ((u >> 16) & 1))", "(u + 0x8000)"),
    "bf16_truncates": ("(u + 0x7FFF + ((u >> 16) & 1))", "(u + 0)"),
}


def _load(path):
    spec = importlib.util.spec_from_file_location("cnn_mutant", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_cnn_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, f"mutation site for {name} not found in oracle/cnn.py"
    path = os.path.join(tmp_path, "cnn_mutant.py")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    mod = _load(path)
    for pin in cnn_pins.ALL_CNN_PINS:
        try:
            pin(mod)
        except (AssertionError, ValueError, IndexError, FloatingPointError):
            return
    pytest.fail(f"mutant {name} passed every classifier pin")
