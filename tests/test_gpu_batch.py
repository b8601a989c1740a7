"""GPU parity of the batched path: the dedispersion kernel shapes, the
autotuner, many beams in one persistent launch, and the grouped batch step
(sp_batch_*) against the CPU oracle.

Every beam of a batch is an independent search (arXiv 2606.27262, Sec. 2 and
3.1), so each beam's result is held to the single-beam bars: DM transforms
bit-exact, S/N within 1e-4, candidate sets equal up to near-ties."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_27262_gb300 as sp
import synth
from paper_2606_27262_gb300 import build as spbuild
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    spbuild.build()
    assert torch.cuda.is_available()


SMALL = [
    # nchan, ndm, n_out, dm kind
    (1, 5, 37, "random"),
    (17, 65, 1000, "grid"),
    (64, 40, 513, "random"),
    (256, 100, 2049, "grid"),
    (100, 31, 4103, "random"),
    (48, 1, 1, "grid"),
]


def _dms(kind, ndm, rng):
    if kind == "grid":
        return np.arange(ndm, dtype=np.float64) * 0.7
    d = rng.uniform(0, 2000, ndm)
    d[0] = 0.0
    if ndm > 3:
        d[2] = d[1]
    return d


@pytest.mark.parametrize("shape", range(sp.SP_DEDISP_NUM_SHAPES))
@pytest.mark.parametrize("nchan,ndm,n_out,kind", SMALL)
def test_shapes_bitexact(shape, nchan, ndm, n_out, kind):
    rng = np.random.default_rng(nchan * 1000 + ndm + 7)
    f = synth.band_freqs(nchan)
    dms = _dms(kind, ndm, rng)
    plan = sp.Plan(f, synth.TSAMP, dms, shape=shape)
    dt, tt, cc = sp.shape_info(shape)
    assert plan.shape == shape and plan.ntiles >= (ndm + dt - 1) // dt
    n_in = n_out + plan.max_delay
    x = rng.integers(0, 256, size=(n_in, nchan), dtype=np.uint8)
    got = gu.dev_dedisperse(plan, x).cpu().numpy()
    assert np.array_equal(got, oracle.dedisperse(x, oracle.delays(f, synth.TSAMP, dms), n_out))
    assert plan.status() == 0


def test_autotune_choice_and_cache():
    f = synth.band_freqs(256)
    dms = np.arange(300, dtype=np.float64) * 1.0
    best, ms = sp.autotune_dedisperse(f, synth.TSAMP, dms, n_out_sample=4096, reps=2)
    assert 0 <= best < sp.SP_DEDISP_NUM_SHAPES
    assert np.isfinite(ms).all() and (ms > 0).all() and ms[best] == ms.min()
    best2, ms2 = sp.autotune_dedisperse(f, synth.TSAMP, dms, n_out_sample=4096, reps=2)
    assert best2 == best and np.array_equal(ms, ms2)  # cached
    plan = sp.Plan(f, synth.TSAMP, dms, shape=sp.SP_SHAPE_AUTO)
    assert 0 <= plan.shape < sp.SP_DEDISP_NUM_SHAPES
    rng = np.random.default_rng(5)
    x = rng.integers(0, 256, size=(1500 + plan.max_delay, 256), dtype=np.uint8)
    got = gu.dev_dedisperse(plan, x).cpu().numpy()
    assert np.array_equal(got, oracle.dedisperse(x, oracle.delays(f, synth.TSAMP, dms), 1500))


@pytest.mark.parametrize("shape", range(sp.SP_DEDISP_NUM_SHAPES))
def test_dedisperse_batch_bitexact(shape):
    """Beams with different channel counts, DM lists and lengths in one
    persistent launch; each equals the oracle."""
    rng = np.random.default_rng(40 + shape)
    specs = [(64, np.arange(50) * 0.9, 3000), (33, rng.uniform(0, 900, 70), 1537), (256, np.arange(120) * 0.5, 700),
             (16, np.arange(9) * 3.0, 1), (128, np.arange(40) * 2.5, 5003)]
    beams, refs, keep = [], [], []
    for nchan, dms, n_out in specs:
        f = synth.band_freqs(nchan)
        plan = sp.Plan(f, synth.TSAMP, dms, shape=shape)
        n_in = n_out + plan.max_delay
        x = rng.integers(0, 256, size=(n_in, nchan), dtype=np.uint8)
        staged = sp.staged_buffer(nchan, n_in)
        sp.stage_input(torch.from_numpy(x).cuda(), staged)
        out = torch.full((plan.ndm, n_out), -1, dtype=torch.int32, device="cuda")
        beams.append((plan, staged, n_in, out))
        refs.append(oracle.dedisperse(x, oracle.delays(f, synth.TSAMP, dms), n_out))
        keep.append(plan)
    work = torch.empty(sp.dedisperse_batch_workspace_bytes(len(beams)), dtype=torch.uint8, device="cuda")
    sp.dedisperse_batch(beams, work)
    torch.cuda.synchronize()
    for (plan, _, _, out), ref in zip(beams, refs):
        assert np.array_equal(out.cpu().numpy(), ref)
    assert keep[0].status() == 0


def test_dedisperse_batch_errors():
    f = synth.band_freqs(32)
    p0 = sp.Plan(f, synth.TSAMP, np.arange(10.0), shape=0)
    p1 = sp.Plan(f, synth.TSAMP, np.arange(10.0), shape=1)
    n_in = 100 + p0.max_delay
    st = sp.staged_buffer(32, n_in)
    out = torch.empty((10, 100), dtype=torch.int32, device="cuda")
    work = torch.empty(sp.dedisperse_batch_workspace_bytes(2), dtype=torch.uint8, device="cuda")
    with pytest.raises(sp.SpotlightError) as e:  # mixed shapes
        sp.dedisperse_batch([(p0, st, n_in, out), (p1, st, n_in, out)], work)
    assert e.value.code == sp.SP_EINVAL
    bad = torch.empty((10, 99), dtype=torch.int32, device="cuda")
    with pytest.raises(sp.SpotlightError) as e:  # n_out != n_in - max_delay
        sp.dedisperse_batch([(p0, st, n_in, bad)], work)
    assert e.value.code == sp.SP_ESHAPE
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(sp.SpotlightError) as e:
        sp.dedisperse_batch([(p0, st, n_in, out)], small)
    assert e.value.code == sp.SP_EWORKSPACE


def _small_batch(shape=0, budget=None):
    """Six beams over three DM plans, uneven lengths, per-channel gains and
    bursts; a DM-transform budget that forces several groups."""
    nchan = 128
    f = synth.band_freqs(nchan)
    plan_dms = [np.arange(0, 150.0, 1.0), np.arange(0, 300.0, 2.0), np.arange(0, 400.0, 0.8)]
    plans = [sp.Plan(f, synth.TSAMP, d, shape=shape) for d in plan_dms]
    beam_plan = np.array([2, 0, 1, 2, 1, 0], np.int32)
    n_out = np.array([9000, 4100, 12000, 3000, 8192, 16500], np.int64)
    widths = synth.widths_pow2(64)
    if budget is None:
        budget = int(plans[2].ndm * 9000 * 4 + 1)  # about one large beam per group
    batch = sp.Batch(plans, beam_plan, n_out, widths, 6.0, 4096, 1 << 16, budget)
    data, bursts = [], []
    for b in range(beam_plan.size):
        rng = np.random.default_rng((77, b))
        p = plans[beam_plan[b]]
        n_in = int(n_out[b]) + p.max_delay
        bl = synth.draw_bursts(rng, 2, int(n_out[b]), 30.0, float(plan_dms[beam_plan[b]][-1]) - 30, 2, 12, 12, 30)
        x = synth.make_beam((77, b, 9), nchan, n_in, f, bl, widths=widths,
                            gains=np.random.default_rng((77, b, 2)).uniform(0.5, 1.5, nchan))
        batch.input_tensor(b, nchan).copy_(torch.from_numpy(x))
        data.append(x)
        bursts.append(bl)
    torch.cuda.synchronize()
    return batch, plans, plan_dms, f, widths, data, bursts


def _oracle_beam(x, f, dms, n_out, widths, thr, L):
    dmt = oracle.dedisperse(x, oracle.delays(f, synth.TSAMP, dms), n_out)
    ob, ok = oracle.best(dmt, widths, L)
    o, _ = oracle.peaks(ob, ok, thr)
    return dmt, ob, o


def test_batch_grouped_matches_oracle_and_per_beam():
    batch, plans, plan_dms, f, widths, data, bursts = _small_batch()
    assert batch.ngroups >= 3
    batch.run(sp.SP_BATCH_GROUPED)
    grouped = [batch.results(b) for b in range(batch.nbeams)]
    for b in range(batch.nbeams):
        dms = plan_dms[batch.beam_plan[b]]
        dmt, ob, o = _oracle_beam(data[b], f, dms, int(batch.n_out[b]), widths, 6.0, 4096)
        gu.check_candidates(grouped[b], o, ob, 6.0)
        # every injected burst is found near its DM and time
        for bu in bursts[b]:
            g = grouped[b]
            assert ((np.abs(dms[g["dm_idx"]] - bu.dm) <= 5) & (np.abs(g["t"] - bu.t0) <= 64)).any(), (b, bu)
    # DM transforms of the last two groups are still held: bit-exact
    last = [b for b in range(batch.nbeams) if _held(batch, b)]
    assert last
    for b in last:
        dms = plan_dms[batch.beam_plan[b]]
        want = oracle.dedisperse(data[b], oracle.delays(f, synth.TSAMP, dms), int(batch.n_out[b]))
        assert np.array_equal(batch.dmt_tensor(b, dms.size).cpu().numpy(), want)
    # per-beam launches and one CTA per item: identical candidate lists
    for mode in (sp.SP_BATCH_PER_BEAM, sp.SP_BATCH_GROUPED_GRID):
        batch.run(mode)
        for b in range(batch.nbeams):
            assert np.array_equal(batch.results(b), grouped[b])
    assert batch.status() == 0


def _held(batch, b):
    try:
        batch.dmt_ptr(b)
        return True
    except sp.SpotlightError:
        return False


@pytest.mark.parametrize("mode", [sp.SP_BATCH_GROUPED, sp.SP_BATCH_GROUPED_GRID, sp.SP_BATCH_PER_BEAM])
def test_batch_graph_replay(mode):
    """Graph replays give the eager results; the launch counter sees the
    eager run's kernels once per replay and none at capture (per beam:
    staging, block sums, block coefficients, streamed boxcar, the tile
    kernel over the tiles it lists, 64-bit boxcar pass; dedispersion once per
    group, or once per beam with per-beam launches)."""
    batch, plans, plan_dms, f, widths, data, bursts = _small_batch(shape=1)
    s = torch.cuda.Stream()
    per_step = 7 * batch.nbeams if mode == sp.SP_BATCH_PER_BEAM else 6 * batch.nbeams + batch.ngroups
    with torch.cuda.stream(s):
        lc = sp.launch_count()
        batch.run(mode, stream=s)
        assert sp.launch_count() - lc == per_step
        eager = [batch.results(b, stream=s) for b in range(batch.nbeams)]
        lc = sp.launch_count()
        batch.capture(mode, stream=s)
        assert sp.launch_count() == lc
        for _ in range(2):
            lc = sp.launch_count()
            batch.launch(stream=s)
            assert sp.launch_count() - lc == per_step
            for b in range(batch.nbeams):
                assert np.array_equal(batch.results(b, stream=s), eager[b])
    for b in range(batch.nbeams):
        dms = plan_dms[batch.beam_plan[b]]
        _, ob, o = _oracle_beam(data[b], f, dms, int(batch.n_out[b]), widths, 6.0, 4096)
        gu.check_candidates(eager[b], o, ob, 6.0)


@pytest.mark.parametrize("one_group", [True, False])
def test_batch_run_host(one_group):
    """End to end from host memory (inputs copied group by group on the
    batch's copy stream): the device inputs are cleared first, and every
    beam's candidates equal the device-resident run's."""
    batch, plans, plan_dms, f, widths, data, bursts = _small_batch(budget=(1 << 40) if one_group else None)
    assert (batch.ngroups == 1) == one_group
    batch.run(sp.SP_BATCH_GROUPED)
    dev = [batch.results(b) for b in range(batch.nbeams)]
    for b in range(batch.nbeams):
        batch.input_tensor(b, data[b].shape[1]).zero_()
    torch.cuda.synchronize()
    cap = 1 << 16
    hc = np.zeros((batch.nbeams * cap, 4), np.int32)
    pinned = [torch.from_numpy(x).pin_memory() for x in data]
    counts = batch.run_host(pinned, hc)
    for b in range(batch.nbeams):
        got = sp.cands_to_numpy(hc[b * cap:(b + 1) * cap], int(counts[b]))
        assert np.array_equal(got, dev[b])
        if _held(batch, b):
            dms = plan_dms[batch.beam_plan[b]]
            want = oracle.dedisperse(data[b], oracle.delays(f, synth.TSAMP, dms), int(batch.n_out[b]))
            assert np.array_equal(batch.dmt_tensor(b, dms.size).cpu().numpy(), want)


def test_batch_create_errors():
    f = synth.band_freqs(32)
    p0 = sp.Plan(f, synth.TSAMP, np.arange(10.0), shape=0)
    p1 = sp.Plan(f, synth.TSAMP, np.arange(10.0), shape=2)
    w = [1, 2, 4]
    for args, code in [(([p0, p1], [0, 1], [100, 100]), sp.SP_EINVAL),   # mixed shapes
                       (([p0], [1], [100]), sp.SP_EINVAL),               # plan index out of range
                       (([p0], [0], [0]), sp.SP_EINVAL)]:                # empty beam
        with pytest.raises(sp.SpotlightError) as e:
            sp.Batch(*args, w, 6.0, 64, 16, 1 << 20)
        assert e.value.code == code


# ------------------------------------------------- config 3 at full size --
CFG3_CHECK_BEAMS = 3  # one beam of each DM plan


@pytest.fixture(scope="module")
def config3_run():
    bw = synth.config3()
    best, ms = sp.autotune_dedisperse(bw.freqs, bw.tsamp, bw.plan_dms[-1])
    plans = [sp.Plan(bw.freqs, bw.tsamp, d, shape=best) for d in bw.plan_dms]
    batch = sp.Batch(plans, bw.beam_plan, bw.n_out, bw.widths, bw.threshold, bw.norm_block, 1 << 20, 24 << 30)
    for b in range(bw.nbeams):
        synth.make_beam_torch(bw.beam_seed(b), batch.input_tensor(b, bw.nchan), bw.freqs, bw.bursts(b),
                              widths=bw.widths, gains=bw.gains(b))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    batch.capture(sp.SP_BATCH_GROUPED, stream=s)
    batch.launch(stream=s)
    torch.cuda.synchronize()
    yield bw, plans, batch
    batch.close()
    torch.cuda.empty_cache()


def _sample_beams(bw, batch):
    out = []
    for p in range(len(bw.plan_dms)):
        cand = [b for b in range(bw.nbeams) if bw.beam_plan[b] == p and _held(batch, b)]
        if not cand:
            cand = [b for b in range(bw.nbeams) if bw.beam_plan[b] == p]
        out.append(cand[-1])
    return out


def test_config3_sampled_parity(config3_run):
    """Sampled DM rows of one beam per plan: DM transform rows bit-exact
    (where the arena still holds the beam) and candidates equal to the
    oracle's on those rows."""
    bw, plans, batch = config3_run
    assert batch.status() == 0
    for b in _sample_beams(bw, batch):
        dms = bw.plan_dms[bw.beam_plan[b]]
        n_out = int(bw.n_out[b])
        x = batch.input_tensor(b, bw.nchan).cpu().numpy()
        g = batch.results(b)
        for lo in (0, dms.size // 2, dms.size - 3):
            rows = np.arange(lo, lo + 3)
            dmt_o = oracle.dedisperse(x, oracle.delays(bw.freqs, bw.tsamp, dms[rows]), n_out)
            if _held(batch, b):
                got = batch.dmt_tensor(b, dms.size)[lo:lo + 3].cpu().numpy()
                assert np.array_equal(got, dmt_o)
            ob, ok = oracle.best(dmt_o, bw.widths, bw.norm_block)
            emit_lo = 0 if lo == 0 else 1
            emit_hi = 3 if rows[-1] == dms.size - 1 else 2
            o, _ = oracle.peaks(ob, ok, bw.threshold, row0=int(lo), emit_lo=emit_lo, emit_hi=emit_hi)
            sel = (g["dm_idx"] >= lo + emit_lo) & (g["dm_idx"] < lo + emit_hi)
            gs = g[sel].copy()
            gs["dm_idx"] -= lo
            o = o.copy()
            o["dm_idx"] -= lo
            gu.check_candidates(gs, o, ob, bw.threshold)


def _halfstep_smear(freqs, dms, dm, tsamp):
    """Samples of residual sweep across the band at half the local trial
    spacing around dm (Eq. 1 with the DM error of the nearest trial)."""
    k = int(np.clip(np.searchsorted(dms, dm), 1, dms.size - 1))
    half = 0.5 * (dms[k] - dms[k - 1])
    return synth.KDM_PHYS * half * (1.0 / freqs[-1] ** 2 - 1.0 / freqs[0] ** 2) / tsamp


def test_config3_burst_recall(config3_run):
    """Injected bursts (S/N 8-30 at their exact DM) are found near their DM
    and time.  Narrow bursts whose sweep error at half a trial step exceeds
    their width lose S/N between trials (Appendix A); recall must be >= 99 %
    over the bursts the trial grid resolves and is reported over all."""
    bw, plans, batch = config3_run
    found = total = found_res = total_res = 0
    for b in range(bw.nbeams):
        dms = bw.plan_dms[bw.beam_plan[b]]
        g = batch.results(b)
        for bu in bw.bursts(b):
            near = (np.abs(dms[g["dm_idx"]] - bu.dm) <= max(5.0, 0.02 * bu.dm)) & (np.abs(g["t"] - bu.t0) <= 64)
            hit = bool(near.any())
            total += 1
            found += hit
            if _halfstep_smear(bw.freqs, dms, bu.dm, bw.tsamp) <= bu.fwhm:
                total_res += 1
                found_res += hit
    print(f"config-3 recall: {found}/{total} all bursts, {found_res}/{total_res} resolved by the trial grid")
    assert total == 4 * bw.nbeams and total_res >= total // 4
    assert found_res >= 0.99 * total_res, (found_res, total_res)
