"""The dedispersion kernel's bounded waits run out on purpose, with every
access in bounds (failure detection without a GPU fault): the test hook
makes every CTA's first staging barrier expect 16 bytes more than its bulk
copies bring and bounds each wait at 20000 SM cycles.  The kernels must
return, flag SP_STATUS_STAGING_TIMEOUT in the plan's status word (a
batched launch in the batch's word; a streaming batch returns each of its
gulps with SP_ETIMEOUT and no candidates), and leave the device usable: with
the hook cleared the same calls are bit-exact against the oracle again."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_27262_gb300 as sp
import synth
from paper_2606_27262_gb300 import build as spbuild
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

DEFAULT_LIMIT = 1 << 31


@pytest.fixture(scope="module", autouse=True)
def _built():
    spbuild.build()
    assert torch.cuda.is_available()
    yield
    sp.debug_staging_fault(0, DEFAULT_LIMIT)


@pytest.mark.parametrize("shape", range(sp.SP_DEDISP_NUM_SHAPES))
def test_timeout_is_flagged_and_device_recovers(shape):
    rng = np.random.default_rng(70 + shape)
    f = synth.band_freqs(64)
    dms = np.arange(0, 90, dtype=np.float64) * 1.5
    plan = sp.Plan(f, synth.TSAMP, dms, shape=shape)
    n_out = 2048
    x = rng.integers(0, 256, size=(n_out + plan.max_delay, 64), dtype=np.uint8)
    want = oracle.dedisperse(x, oracle.delays(f, synth.TSAMP, dms), n_out)
    assert plan.status() == 0
    sp.debug_staging_fault(16, 20000)
    try:
        gu.dev_dedisperse(plan, x)
        torch.cuda.synchronize()
    finally:
        sp.debug_staging_fault(0, DEFAULT_LIMIT)
    assert plan.status(clear=True) & sp.SP_STATUS_STAGING_TIMEOUT
    assert plan.status() == 0
    got = gu.dev_dedisperse(plan, x).cpu().numpy()
    assert np.array_equal(got, want)
    assert plan.status() == 0


def test_timeout_in_a_streaming_batch_voids_its_gulps():
    rng = np.random.default_rng(77)
    nchan, gulp = 64, 1000
    f = synth.band_freqs(nchan)
    dms = np.arange(0, 40, dtype=np.float64)
    plan = sp.Plan(f, synth.TSAMP, dms)
    s = sp.Stream(plan, 2, gulp, [1, 2, 4], 6.0, 0, 1024, 1 << 30, max_batch=2)
    hist = torch.from_numpy(rng.integers(0, 256, size=(plan.max_delay, nchan), dtype=np.uint8)).pin_memory()
    g = torch.from_numpy(rng.integers(0, 256, size=(gulp, nchan), dtype=np.uint8)).pin_memory()
    for b in range(2):
        s.history(b, hist)
    sp.debug_staging_fault(16, 20000)
    try:
        s.push(0, g)
        s.push(1, g)
        res = s.drain()
    finally:
        sp.debug_staging_fault(0, DEFAULT_LIMIT)
    assert len(res) == 2
    for r in res:
        info = r[0]
        assert info.status == sp.SP_ETIMEOUT and info.count == 0
    # the stream goes on: later gulps search normally
    s.push(0, g)
    s.push(1, g)
    res = s.drain()
    assert len(res) == 2 and all(r[0].status == sp.SP_OK for r in res)
    s.close()
