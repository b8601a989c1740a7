"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars: delay tables and DM transforms bit-exact; best S/N within 1e-4
relative; best width a maximiser within that tolerance; candidate sets equal
up to near-ties at the threshold or between neighbours (arXiv 2606.27262,
Sec. 3.1.1-3.1.2).  Inputs are seeded synthetic beams (synth)."""
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


# ------------------------------------------------------------- delays ---
@pytest.mark.parametrize("cfg", [synth.config1, synth.config2])
def test_plan_delays_bitexact(cfg):
    wl = cfg()
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms)
    want = oracle.delays(wl.freqs, wl.tsamp, wl.dms)
    assert np.array_equal(plan.delays(), want)
    assert plan.max_delay == int(want.max())


# --------------------------------------------------------- dedisperse ---
SMALL = [
    # nchan, ndm, n_out, dm kind
    (1, 5, 37, "random"),
    (3, 7, 100, "random"),
    (16, 33, 512, "grid"),
    (17, 65, 1000, "grid"),
    (64, 40, 513, "random"),
    (256, 100, 2049, "grid"),
    (100, 31, 4103, "random"),
    (48, 1, 1, "grid"),
    (33, 70, 1537, "grid"),
]


def _dms(kind, ndm, rng):
    if kind == "grid":
        return np.arange(ndm, dtype=np.float64) * 0.7
    d = rng.uniform(0, 2000, ndm)
    d[0] = 0.0
    if ndm > 3:
        d[2] = d[1]  # a duplicate trial
    return d


@pytest.mark.parametrize("nchan,ndm,n_out,kind", SMALL)
def test_dedisperse_small_bitexact(nchan, ndm, n_out, kind):
    rng = np.random.default_rng(nchan * 1000 + ndm)
    f = synth.band_freqs(nchan)
    dms = _dms(kind, ndm, rng)
    plan = sp.Plan(f, synth.TSAMP, dms)
    n_in = n_out + plan.max_delay
    x = rng.integers(0, 256, size=(n_in, nchan), dtype=np.uint8)
    got = gu.dev_dedisperse(plan, x).cpu().numpy()
    want = oracle.dedisperse(x, oracle.delays(f, synth.TSAMP, dms), n_out)
    assert np.array_equal(got, want)


def test_dedisperse_saturated_input():
    """All-255 input over 4096 channels: the largest sums (1,044,480) exercise
    the 16-bit lane widening every 256 channels."""
    f = synth.band_freqs(4096)
    dms = np.arange(40, dtype=np.float64) * 0.5
    plan = sp.Plan(f, synth.TSAMP, dms)
    n_out = 1000
    x = np.full((n_out + plan.max_delay, 4096), 255, np.uint8)
    got = gu.dev_dedisperse(plan, x).cpu().numpy()
    assert (got == 255 * 4096).all()


def test_dedisperse_config1_bitexact():
    """Also counts the kernels: sp_dedisperse launches two (staging,
    dedispersion), sp_single_pulse_search five here (block sums, block
    coefficients, streamed boxcar with peaks, the tile kernel over the tiles
    it lists, 64-bit boxcar pass)."""
    wl = synth.config1()
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms)
    x, _ = synth.make_workload_beam(wl, wl.n_out + plan.max_delay)
    lc = sp.launch_count()
    dmt = gu.dev_dedisperse(plan, x)
    assert sp.launch_count() - lc == 2
    got = dmt.cpu().numpy()
    want = oracle.dedisperse(x, oracle.delays(wl.freqs, wl.tsamp, wl.dms), wl.n_out)
    assert np.array_equal(got, want)
    lc = sp.launch_count()
    gu.dev_candidates(dmt, wl.widths, wl.threshold, wl.norm_block)
    assert sp.launch_count() - lc == 5


def test_shape_errors():
    f = synth.band_freqs(16)
    plan = sp.Plan(f, synth.TSAMP, np.arange(8.0))
    x = torch.zeros((100 + plan.max_delay, 16), dtype=torch.uint8, device="cuda")
    out = torch.empty((8, 99), dtype=torch.int32, device="cuda")
    work = torch.empty(sp.dedisperse_workspace_bytes(plan, x.shape[0]), dtype=torch.uint8, device="cuda")
    with pytest.raises(sp.SpotlightError) as e:
        sp.dedisperse(plan, x, out, work)
    assert e.value.code == sp.SP_ESHAPE
    out = torch.empty((8, 100), dtype=torch.int32, device="cuda")
    with pytest.raises(sp.SpotlightError) as e:
        sp.dedisperse(plan, x, out, work[:100])
    assert e.value.code == sp.SP_EWORKSPACE


# ------------------------------------------------------------ S/N map ---
SPS_CASES = [
    # ndm, n_out, widths, norm_block, value kind
    (7, 1000, [1, 2, 4, 8], 0, "noise"),
    (30, 5000, [1, 2, 4, 8, 16, 32], 1024, "noise"),      # 4 blocks + remainder
    (15, 777, [1, 3, 5, 17, 100], 200, "signed"),           # odd widths, negative values
    (3, 300, [2, 64, 256, 1024], 0, "noise"),               # width longer than most windows
    (20, 513, [1], 0, "flat"),                              # zero variance
    (1, 1, [1], 0, "noise"),
    (29, 2600, list(range(1, 17)), 500, "noise"),           # 16 widths
    (10, 1000, [1, 4, 64, 256], 300, "huge"),               # |window sums| >= 2^31: 64-bit path
    (6, 9000, [1, 2, 8, 32], 4096, "near_int32_max"),       # sums of squares beyond 2^63
]


def _dmt_values(kind, ndm, n_out, rng):
    if kind == "noise":
        return np.rint(rng.normal(5.2e5, 1024.0, size=(ndm, n_out))).astype(np.int32)
    if kind == "signed":
        return rng.integers(-50000, 50000, size=(ndm, n_out)).astype(np.int32)
    if kind == "huge":
        return rng.integers(-10_000_000, 10_000_000, size=(ndm, n_out)).astype(np.int32)
    if kind == "near_int32_max":
        sign = rng.choice([-1, 1], size=(ndm, n_out))
        return (sign * (2 ** 30 + rng.integers(0, 2 ** 29, size=(ndm, n_out)))).astype(np.int32)
    return np.full((ndm, n_out), 777, np.int32)


@pytest.mark.parametrize("ndm,n_out,widths,L,kind", SPS_CASES)
def test_best_map_parity(ndm, n_out, widths, L, kind):
    rng = np.random.default_rng(ndm + n_out)
    dmt = _dmt_values(kind, ndm, n_out, rng)
    if kind == "noise" and n_out > 100:
        dmt[ndm // 2, n_out // 3: n_out // 3 + 9] += 9000  # a pulse
    gb, gk = gu.dev_best_map(torch.from_numpy(dmt).cuda(), widths, L)
    ob, ok = oracle.best(dmt, widths, L)
    gu.check_best_map(gb, gk, ob, ok, oracle.boxcar_snr(dmt, widths, L))


@pytest.mark.parametrize("ndm,n_out,widths,L,kind", SPS_CASES)
def test_candidates_parity(ndm, n_out, widths, L, kind):
    rng = np.random.default_rng(ndm + n_out + 1)
    dmt = _dmt_values(kind, ndm, n_out, rng)
    for thr in (3.0, 0.0):
        g, gn = gu.dev_candidates(torch.from_numpy(dmt).cuda(), widths, thr, L)
        ob, ok = oracle.best(dmt, widths, L)
        o, on = oracle.peaks(ob, ok, thr)
        assert gn == g.size
        gu.check_candidates(g, o, ob, thr)


@pytest.mark.parametrize("radius", [2, 5])
@pytest.mark.parametrize("ndm,n_out,widths,L,kind", [SPS_CASES[1], SPS_CASES[2], SPS_CASES[6]])
def test_window_peaks_parity(ndm, n_out, widths, L, kind, radius):
    """The (2r+1)^2 peak filter (the paper's 11 x 11 stencil is r = 5)
    against the oracle's, and r = 1 equal to the fused 3 x 3 search."""
    rng = np.random.default_rng(ndm + n_out + 3)
    dmt = torch.from_numpy(_dmt_values(kind, ndm, n_out, rng)).cuda()
    ob, ok = oracle.best(dmt.cpu().numpy(), widths, L)
    for thr in (3.0, 0.0):
        work = torch.empty(sp.sps_window_workspace_bytes(ndm, n_out, len(widths), L, radius), dtype=torch.uint8,
                           device="cuda")
        cands = torch.zeros((1 << 20, 4), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        sp.single_pulse_search_window(dmt, widths, thr, L, radius, work, cands, cnt)
        torch.cuda.synchronize()
        n = int(cnt.item())
        g = sp.cands_to_numpy(cands.cpu().numpy(), n)
        o, on = oracle.peaks_window(ob, ok, thr, radius)
        assert n == g.size
        gu.check_candidates(g, o, ob, thr, radius=radius)
        g3, _ = gu.dev_candidates(dmt, widths, thr, L)
        assert g.size <= g3.size  # a wider window keeps a subset of the 3 x 3 peaks (up to near-ties)
        w1 = torch.empty(sp.sps_window_workspace_bytes(ndm, n_out, len(widths), L, 1), dtype=torch.uint8,
                         device="cuda")
        sp.single_pulse_search_window(dmt, widths, thr, L, 1, w1, cands, cnt)
        torch.cuda.synchronize()
        assert np.array_equal(sp.cands_to_numpy(cands.cpu().numpy(), int(cnt.item())), g3)


def test_candidate_overflow():
    rng = np.random.default_rng(5)
    dmt = rng.integers(0, 1000, size=(40, 4000)).astype(np.int32)
    full, n = gu.dev_candidates(torch.from_numpy(dmt).cuda(), [1, 2], -1e9, 0)
    assert n > 100
    part, n2 = gu.dev_candidates(torch.from_numpy(dmt).cuda(), [1, 2], -1e9, 0, cap=100)
    assert n2 == n and part.size == 100
    fs = {(int(a), int(b)) for a, b in zip(full["dm_idx"], full["t"])}
    assert all((int(a), int(b)) in fs for a, b in zip(part["dm_idx"], part["t"]))


# ------------------------------------------------------ whole workload ---
def test_config1_search_parity_and_recovery():
    wl = synth.config1()
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms)
    x, bursts = synth.make_workload_beam(wl, wl.n_out + plan.max_delay)
    dmt = gu.dev_dedisperse(plan, x)
    dmt_o = oracle.dedisperse(x, oracle.delays(wl.freqs, wl.tsamp, wl.dms), wl.n_out)
    assert np.array_equal(dmt.cpu().numpy(), dmt_o)
    gb, gk = gu.dev_best_map(dmt, wl.widths, wl.norm_block)
    ob, ok = oracle.best(dmt_o, wl.widths, wl.norm_block)
    gu.check_best_map(gb, gk, ob, ok, oracle.boxcar_snr(dmt_o, wl.widths, wl.norm_block))
    g, gn = gu.dev_candidates(dmt, wl.widths, wl.threshold, wl.norm_block)
    o, on = oracle.peaks(ob, ok, wl.threshold)
    assert gu.check_candidates(g, o, ob, wl.threshold) >= 1
    # a burst the oracle detects (a candidate near its DM and time) is detected on the GPU too
    hits = 0
    for b in bursts:
        ng = np.sum((np.abs(wl.dms[g["dm_idx"]] - b.dm) <= 3) & (np.abs(g["t"] - b.t0) <= 32))
        no = np.sum((np.abs(wl.dms[o["dm_idx"]] - b.dm) <= 3) & (np.abs(o["t"] - b.t0) <= 32))
        assert (ng > 0) == (no > 0), (b, ng, no)
        hits += ng > 0
    assert hits >= 2


def test_searcher_run_host_matches_device_path():
    wl = synth.config1()
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms)
    x, _ = synth.make_workload_beam(wl, wl.n_out + plan.max_delay)
    s = sp.Searcher(plan, wl.n_out, wl.widths, wl.threshold, wl.norm_block, 1 << 16)
    h_in = torch.from_numpy(x).pin_memory()
    hc = np.zeros((1 << 16, 4), np.int32)
    n = s.run_host(h_in, hc)
    got = sp.cands_to_numpy(hc, n)
    dmt = gu.dev_dedisperse(plan, x)
    want, wn = gu.dev_candidates(dmt, wl.widths, wl.threshold, wl.norm_block)
    assert n == wn and np.array_equal(got, want)
    # device-resident run gives the same list
    d_in = torch.from_numpy(x).cuda()
    dc = torch.zeros((1 << 16, 4), dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    s.run(d_in, dc, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == n
    assert np.array_equal(sp.cands_to_numpy(dc.cpu().numpy(), n), want)


def test_searcher_pipelined_host_runs_match_run_host():
    """submit_host/collect on three different beams in a row (two in flight)
    gives each beam the result run_host gives it; a third submit with two
    uncollected beams and a collect with none queued are refused."""
    wl = synth.config1()
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms)
    n_in = wl.n_out + plan.max_delay
    s = sp.Searcher(plan, wl.n_out, wl.widths, wl.threshold, wl.norm_block, 1 << 16)
    beams = [torch.from_numpy(synth.make_workload_beam(wl, n_in, seed=seed)[0]).pin_memory() for seed in (5, 6, 7)]
    want = []
    for b in beams:
        hc = np.zeros((1 << 16, 4), np.int32)
        n = s.run_host(b, hc)
        want.append(sp.cands_to_numpy(hc, n))
    got = []
    s.submit_host(beams[0])
    s.submit_host(beams[1])
    with pytest.raises(sp.SpotlightError):
        s.submit_host(beams[2])
    for k in range(3):
        hc = np.zeros((1 << 16, 4), np.int32)
        n = s.collect(hc)
        got.append(sp.cands_to_numpy(hc, n))
        if k == 0:
            s.submit_host(beams[2])
    with pytest.raises(sp.SpotlightError):
        s.collect(np.zeros((4, 4), np.int32))
    for g, w in zip(got, want):
        assert g.size > 0 and np.array_equal(g, w)
    # a smaller caller capacity: five of the candidates, and the full count
    s.submit_host(beams[0])
    hc = np.zeros((5, 4), np.int32)
    assert s.collect(hc) == want[0].size
    full = {(int(a), int(b)) for a, b in zip(want[0]["dm_idx"], want[0]["t"])}
    part = sp.cands_to_numpy(hc, 5)
    assert part.size == 5 and all((int(a), int(b)) in full for a, b in zip(part["dm_idx"], part["t"]))


@pytest.fixture(scope="module")
def config2_run():
    wl = synth.config2()
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms)
    x, bursts = synth.make_workload_beam(wl, wl.n_out + plan.max_delay)
    dmt = gu.dev_dedisperse(plan, x)
    yield wl, plan, x, bursts, dmt
    del dmt
    torch.cuda.empty_cache()


# Sampled rows: tile edges, step-schedule edges, the two ends.
CFG2_ROWS = [0, 1, 31, 32, 33, 2499, 2500, 2501, 3750, 4750, 5749, 5750]


def test_config2_dedisperse_sampled_rows(config2_run):
    wl, plan, x, bursts, dmt = config2_run
    rows = np.array(CFG2_ROWS)
    want = oracle.dedisperse(x, oracle.delays(wl.freqs, wl.tsamp, wl.dms[rows]), wl.n_out)
    got = dmt[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.array_equal(got, want)
    # properties over every row: DM 0 row is the channel sum, all sums in range
    assert np.array_equal(dmt[0].cpu().numpy(), x[: wl.n_out].astype(np.int64).sum(axis=1))
    assert int(dmt.min()) >= 0 and int(dmt.max()) <= 255 * wl.nchan


def test_config2_search_sampled(config2_run):
    wl, plan, x, bursts, dmt = config2_run
    g, gn = gu.dev_candidates(dmt, wl.widths, wl.threshold, wl.norm_block, cap=1 << 22)
    assert gn == g.size
    for lo in (0, 2499, 5748):  # check rows lo+1 .. lo+1 (needs neighbours lo, lo+2)
        rows = np.arange(lo, min(lo + 3, plan.ndm))
        dmt_o = oracle.dedisperse(x, oracle.delays(wl.freqs, wl.tsamp, wl.dms[rows]), wl.n_out)
        ob, ok = oracle.best(dmt_o, wl.widths, wl.norm_block)
        emit_lo = 0 if lo == 0 else 1
        emit_hi = rows.size if rows[-1] == plan.ndm - 1 else rows.size - 1
        o, _ = oracle.peaks(ob, ok, wl.threshold, row0=int(rows[0]), emit_lo=emit_lo, emit_hi=emit_hi)
        sel = (g["dm_idx"] >= rows[0] + emit_lo) & (g["dm_idx"] < rows[0] + emit_hi)
        gsub = g[sel].copy()
        gsub["dm_idx"] -= rows[0]
        o = o.copy()
        o["dm_idx"] -= rows[0]
        gu.check_candidates(gsub, o, ob, wl.threshold)
        gb, gk = gu.dev_best_map(dmt[int(rows[0]):int(rows[-1]) + 1].contiguous(), wl.widths, wl.norm_block)
        gu.check_best_map(gb, gk, ob, ok, oracle.boxcar_snr(dmt_o, wl.widths, wl.norm_block))
    # injected bursts are detected near their DM and arrival time (narrow
    # bursts between coarse high-DM trials lose S/N to smearing, Appendix A)
    found = 0
    for b in bursts:
        near = g[(np.abs(wl.dms[g["dm_idx"]] - b.dm) <= 5) & (np.abs(g["t"] - b.t0) <= 64)]
        found += near.size > 0
    assert found >= len(bursts) // 2, (found, len(bursts))


def test_staged_entry_points():
    """stage_input + dedisperse_staged equals dedisperse; the staged form is
    the zero-padded channel-major input; the probe reports a sane rate; the
    plan's device status stays clear."""
    rng = np.random.default_rng(21)
    f = synth.band_freqs(80)
    dms = np.arange(70, dtype=np.float64) * 1.3
    plan = sp.Plan(f, synth.TSAMP, dms)
    n_out = 3001
    n_in = n_out + plan.max_delay
    x = rng.integers(0, 256, size=(n_in, 80), dtype=np.uint8)
    ref = gu.dev_dedisperse(plan, x)
    d_in = torch.from_numpy(x).cuda()
    xt = sp.staged_buffer(80, n_in)
    sp.stage_input(d_in, xt)
    out = torch.empty_like(ref)
    sp.dedisperse_staged(plan, xt, n_in, out)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    pitch = sp.staged_pitch(n_in)
    xs = xt.cpu().numpy()[: 80 * pitch].reshape(80, pitch)
    assert np.array_equal(xs[:, :n_in], x.T) and not xs[:, n_in:].any()
    rate, nsm = sp.probe_iadd3_rate(256)
    assert nsm >= 100 and 16 <= rate <= 160
    assert plan.status() == 0


def test_config2_sift(config2_run):
    """Sifting the GPU's config-2 candidates (Sec. 3.2.1): the library's
    sifter equals the oracle sifter on the same list, and the injected
    bursts the search found at S/N >= 12 keep a cluster peak nearby."""
    from oracle import sift as osift
    wl, plan, x, bursts, dmt = config2_run
    g, gn = gu.dev_candidates(dmt, wl.widths, wl.threshold, wl.norm_block, cap=1 << 22)
    got, glab = sp.sift(g, wl.dms, wl.widths, wl.tsamp, labels=True)
    want, wlab = osift.sift(g, wl.dms, wl.widths, wl.tsamp)
    assert np.array_equal(glab, wlab) and np.array_equal(got, want)
    assert 0 < got.size < g.size
    for b in bursts:
        seen = g[(np.abs(wl.dms[g["dm_idx"]] - b.dm) <= 5) & (np.abs(g["t"] - b.t0) <= 64) & (g["snr"] >= 12)]
        if seen.size >= 5:
            near = (np.abs(wl.dms[got["dm_idx"]] - b.dm) <= 10) & (np.abs(got["t"] - b.t0) <= 400)
            assert near.any(), b
