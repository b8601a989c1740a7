"""Every row of the full-size single-beam DM plan (4096 channels over
300-500 MHz, DM 0-2000 in the 0.1/0.2/0.5/1.0 step schedule: 5751 trials,
180+ DM tiles, three step boundaries) against the oracle, at a shorter
searched length (8192 samples, so that the oracle finishes in about a minute
on the host cores): the DM transform bit for bit for every compiled kernel
shape and for one batched launch; the best-S/N map of every row within 1e-4;
the candidate set of every row modulo near-ties.  (arXiv 2606.27262,
Sec. 3.1.1 and Sec. 3.1.2.)"""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_27262_gb300 as sp
import synth
from paper_2606_27262_gb300 import build as spbuild
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

N_OUT = 8192
N_OUT_SHORT = 3001  # a second, ragged beam in the batched launch: a prefix of the first


@pytest.fixture(scope="module")
def full_plan_case():
    spbuild.build()
    assert torch.cuda.is_available()
    wl = synth.config2()
    d = oracle.delays(wl.freqs, wl.tsamp, wl.dms)
    n_in = N_OUT + int(d.max())
    bursts = [synth.Burst(t0=1500, dm=180.0, fwhm=4.0, snr=25.0), synth.Burst(t0=5200, dm=1230.0, fwhm=8.0, snr=30.0)]
    x = synth.make_beam(2002, wl.nchan, n_in, wl.freqs, bursts, widths=wl.widths)
    want = oracle.dedisperse(x, d, N_OUT)
    return wl, x, want


@pytest.mark.parametrize("shape", range(sp.SP_DEDISP_NUM_SHAPES))
def test_every_row_bitexact(full_plan_case, shape):
    wl, x, want = full_plan_case
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms, shape=shape)
    assert plan.ndm == 5751 and plan.max_delay == 44995
    assert plan.ntiles >= 5751 // sp.shape_info(shape)[0]
    got = gu.dev_dedisperse(plan, x).cpu().numpy()
    bad = np.argwhere((got != want).any(axis=1)).ravel()
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:10]}"
    assert plan.status() == 0


def test_every_row_bitexact_batched(full_plan_case):
    wl, x, want = full_plan_case
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms)
    beams = []
    for n_out in (N_OUT, N_OUT_SHORT):
        n_in = n_out + plan.max_delay
        staged = sp.staged_buffer(wl.nchan, n_in)
        sp.stage_input(torch.from_numpy(np.ascontiguousarray(x[:n_in])).cuda(), staged)
        out = torch.full((plan.ndm, n_out), -1, dtype=torch.int32, device="cuda")
        beams.append((plan, staged, n_in, out))
    work = torch.empty(sp.dedisperse_batch_workspace_bytes(len(beams)), dtype=torch.uint8, device="cuda")
    sp.dedisperse_batch(beams, work)
    torch.cuda.synchronize()
    assert np.array_equal(beams[0][3].cpu().numpy(), want)
    assert np.array_equal(beams[1][3].cpu().numpy(), want[:, :N_OUT_SHORT])
    assert plan.status() == 0


def test_every_row_search(full_plan_case):
    """Best S/N and width of every (DM, t) and the candidates of every row,
    so that every DM tile and every step boundary of the plan meets the
    oracle's search."""
    wl, x, want = full_plan_case
    dmt = torch.from_numpy(want).cuda()
    gb, gk = gu.dev_best_map(dmt, wl.widths, wl.norm_block)
    ob, ok = oracle.best(want, wl.widths, wl.norm_block)
    ninf_g, ninf_o = np.isneginf(gb), np.isneginf(ob)
    assert np.array_equal(ninf_g, ninf_o)
    fin = ~ninf_o
    err = np.abs(gb[fin].astype(np.float64) - ob[fin])
    assert (err <= gu.SNR_RTOL * np.maximum(np.abs(ob[fin]), 0.1)).all(), err.max()
    # where the widths differ, the GPU's width must tie with the oracle's best
    rows = np.unique(np.argwhere(fin & (gk != ok))[:, 0])
    for r in rows:
        snr = oracle.boxcar_snr(want[r:r + 1], wl.widths, wl.norm_block)[0]
        ts = np.argwhere(fin[r] & (gk[r] != ok[r])).ravel()
        alt = snr[gk[r, ts], ts]
        assert (alt >= ob[r, ts] - gu.SNR_RTOL * np.maximum(np.abs(ob[r, ts]), 0.1)).all()
    g, gn = gu.dev_candidates(dmt, wl.widths, wl.threshold, wl.norm_block, cap=1 << 22)
    o, on = oracle.peaks(ob, ok, wl.threshold, cap=1 << 22)
    assert gn == g.size and on == o.size and gn > 0
    gu.check_candidates(g, o, ob, wl.threshold)
    # the two injected bursts are found near their DM and arrival time
    for dm, t0 in ((180.0, 1500), (1230.0, 5200)):
        near = g[(np.abs(wl.dms[g["dm_idx"]] - dm) <= 5) & (np.abs(g["t"] - t0) <= 64)]
        assert near.size > 0, (dm, t0)
