"""Plant plausible mistakes in copies of the oracle and check that the pins
catch every one (a pin that cannot fail pins nothing).

Each mutant is a text substitution in oracle/oracle.c, compiled to a temporary
shared library; the real oracle is untouched."""
import os

import pytest

import oracle
from tests import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "round_truncates": ("(int32_t)floor(x + 0.5)", "(int32_t)floor(x)"),
    "reference_is_lowest_freq": ("1.0 / (ftop * ftop)",
                                 "1.0 / (freqs_mhz[nchan - 1] * freqs_mhz[nchan - 1])"),
    "square_dropped": ("(1.0 / (f * f) - 1.0 / (ftop * ftop))", "(1.0 / f - 1.0 / ftop)"),
    "channel_order_reversed": ("acc += in[(t + dl[c]) * (int64_t)nchan + c];",
                               "acc += in[(t + dl[nchan - 1 - c]) * (int64_t)nchan + c];"),
    "first_row_delays_for_all": ("const int32_t *dl = delays + (int64_t)r * nchan;",
                                 "const int32_t *dl = delays;"),
    "boxcar_drops_first": ("const int64_t S = cum[t + w] - cum[t];",
                           "const int64_t S = cum[t + w] - cum[t + 1];"),
    "sigma_times_w": ("(sqrt((double)w) * sqrt((double)var_n2))", "((double)w * sqrt((double)var_n2))"),
    "mean_term_dropped": ("(__int128)n * S - (__int128)w * s1", "(__int128)n * S - (__int128)s1"),
    "block_of_window_end": ("int64_t b = t / (norm_block > 0 ? norm_block : n_out);",
                            "int64_t b = (t + w - 1) / (norm_block > 0 ? norm_block : n_out);"),
    "sum_of_squares_64bit": ("s2 += (__int128)((int64_t)row[t] * row[t]);",
                             "s2 = (int64_t)((uint64_t)s2 + (uint64_t)((int64_t)row[t] * row[t]));"),
    "sample_variance": ("(__int128)n * s2 - (__int128)s1 * s1",
                        "((__int128)n * s2 - (__int128)s1 * s1) * n / (n > 1 ? n - 1 : 1)"),
    "widest_on_ties": ("if (kb < 0 || v > b) {", "if (kb < 0 || v >= b) {"),
    "tie_rule_reversed": ("if (before ? !(v > u) : !(v >= u)) {", "if (before ? !(v >= u) : !(v > u)) {"),
    "threshold_strict": ("if (!(v >= thr))", "if (!(v > thr))"),
    "window_radius_ignored": ("for (int32_t dr = -radius; dr <= radius && keep; ++dr) {",
                              "for (int32_t dr = -1; dr <= 1 && keep; ++dr) {"),
    "no_dm_neighbours": ("for (int32_t dr = -1; dr <= 1 && keep; ++dr) {",
                         "for (int32_t dr = 0; dr <= 0 && keep; ++dr) {"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert old in src, f"mutation site for {name} not found in oracle.c"
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    lib = oracle.load(oracle.compile_library(str(mpath), str(tmp_path / "libmutant.so")))
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, ValueError):
            failed.append(pin.__name__)
            break
    assert failed, f"mutant {name} passed every pin"
