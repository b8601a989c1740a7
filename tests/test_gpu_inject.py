"""GPU parity of the quantised-data injector (arXiv 2606.27262, Appendix B)
against its oracle, and an injected dispersed burst recovered by the search
(the validation use of Sec. 4)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_27262_gb300 as sp
import synth
from oracle import inject as oi
from paper_2606_27262_gb300 import build as spbuild
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    spbuild.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("bits,mu,sigma,level,smax,n", [
    (8, 127.5, 16.0, 1 / 16, 40.0, 2000),      # round(128 + 16 z) data
    (8, 0.0, 1.0, 0.030765, 2.0, 1500),        # Appendix B's 8-bit level setting
    (2, 0.0, 1.0, 0.8, 3.0, 20000),
    (1, 0.5, 1.3, 1.0, 4.0, 20000),
])
def test_inject_parity(bits, mu, sigma, level, smax, n):
    rng = np.random.default_rng(bits * 100 + n)
    vals = rng.integers(0, 2 ** bits, n).astype(np.uint8)
    vals[:4] = [0, 2 ** bits - 1, 0, 1 if bits > 1 else 0]
    sig = rng.uniform(0, smax, n).astype(np.float32)
    sig[::7] = 0.0
    d = torch.from_numpy(vals).cuda()
    sp.inject_quantised(d, torch.from_numpy(sig).cuda(), bits, mu, sigma, level)
    got = d.cpu().numpy().astype(np.int64)
    want, gap = oi.inject(vals, sig, bits, mu, sigma, level)
    diff = got != want
    assert not (diff & (gap > 1e-12)).any(), np.flatnonzero(diff & (gap > 1e-12))[:5]
    assert diff.sum() <= max(2, n // 1000)
    assert (got >= vals).all()


def test_injected_burst_is_recovered():
    """A dispersed burst injected into quantised noise (mu 127.5, sigma 16,
    level 1/16 for data drawn as round(128 + 16 z)) is found by the search at
    its DM, time and S/N, as when the same burst is added before quantising."""
    wl = synth.config1()
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms)
    n_in = wl.n_out + plan.max_delay
    noise = synth.make_beam(77, wl.nchan, n_in, wl.freqs)
    burst = synth.Burst(t0=3000, dm=251.3, fwhm=4.0, snr=20.0)
    sig = synth.burst_signal(wl.freqs, n_in, [burst], widths=wl.widths)
    d = torch.from_numpy(noise).cuda()
    sp.inject_quantised(d, torch.from_numpy(sig).cuda(), 8, 127.5, 16.0, 1 / 16)
    x = d.cpu().numpy()
    assert (x >= noise).all() and (x > noise).sum() > 0
    dmt = gu.dev_dedisperse(plan, x)
    g, _ = gu.dev_candidates(dmt, wl.widths, wl.threshold, wl.norm_block)
    near = g[(np.abs(wl.dms[g["dm_idx"]] - burst.dm) <= 2) & (np.abs(g["t"] - burst.t0) <= 16)]
    assert near.size > 0
    snr = float(near["snr"].max())
    assert abs(snr - burst.snr) <= 0.25 * burst.snr, snr
    # the oracle's search of the injected beam agrees
    _, ob, _, oc, _ = oracle.search(x, oracle.delays(wl.freqs, wl.tsamp, wl.dms), wl.n_out, wl.widths,
                                    wl.threshold, wl.norm_block)
    gu.check_candidates(g, oc, ob, wl.threshold)
