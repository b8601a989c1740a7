"""The classifier's oracle (arXiv 2606.27262, Sec. 3.2.2) against its pins
(tests/cnn_pins.py: scipy's correlation, finite differences, closed forms,
a hand-computed Eq.-1 shift table, hand-standardised images), and the
library's host shift table against the oracle's.  No GPU needed."""
import numpy as np
import pytest

import paper_2606_27262_gb300 as sp
import synth
from oracle import cnn as ocnn
from paper_2606_27262_gb300 import build as spbuild
from tests import cnn_pins


@pytest.mark.parametrize("pin", cnn_pins.ALL_CNN_PINS, ids=lambda f: f.__name__)
def test_cnn_oracle_pin(pin):
    pin(ocnn)


def test_dmt_shift_table_library_equals_oracle():
    spbuild.build()
    f = synth.band_freqs(4096)
    got = sp.dmt_shifts(f, 256, 128)
    want = ocnn.dmt_shifts(f, 256, 128)
    assert np.array_equal(got, want)
    assert (got[:, 0] == 0).all() and got[0, -1] == -128 and got[-1, -1] == 128
    assert np.array_equal(got[::-1], -got)  # rows are symmetric sweeps
    # the residual delay of Eq. 1 grows monotonically down the band
    assert (np.diff(got[-1]) >= 0).all()
