"""GPU parity of the streaming search (sp_stream_*): every gulp's result
equals the oracle's search of its window, and is the same whether the gulp
was searched alone or batched with other beams' gulps (arXiv 2606.27262,
Sec. 2-3.1: beams arrive as continuous streams read in blocks that overlap
by the largest dispersion sweep)."""
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


def _streams(nchan, dms, gulp, ngulps, nbeams, seed):
    """Per beam: the whole stream (history + gulps) with two bursts, split
    into the history block and the gulps (pinned host buffers)."""
    f = synth.band_freqs(nchan)
    dmax = int(oracle.delays(f, synth.TSAMP, dms).max())
    out = []
    for b in range(nbeams):
        rng = np.random.default_rng((seed, b))
        n_total = dmax + ngulps * gulp
        bursts = synth.draw_bursts(rng, 2, ngulps * gulp, 10.0, float(dms[-1]) - 10.0, 2, 10, 12, 30)
        x = synth.make_beam((seed, b, 5), nchan, n_total, f, bursts, widths=(1, 2, 4, 8, 16, 32))
        hist = torch.from_numpy(np.ascontiguousarray(x[:dmax])).pin_memory()
        gulps = [torch.from_numpy(np.ascontiguousarray(x[dmax + k * gulp:dmax + (k + 1) * gulp])).pin_memory()
                 for k in range(ngulps)]
        out.append((x, hist, gulps, bursts))
    return f, dmax, out


def _run(stream, beams, order):
    """Histories, then gulps pushed in `order` (list of (beam, k)); returns
    {(beam, seq): (result, candidates)}."""
    for b, (_, hist, _, _) in beams.items():
        stream.history(b, hist)
    res = {}
    for b, k in order:
        seq = stream.push(b, beams[b][2][k])
        assert seq == k
        for r, c in stream.poll():
            res[(r.beam, r.seq)] = (r, c)
    for r, c in stream.drain():
        res[(r.beam, r.seq)] = (r, c)
    return res


WIDTHS = (1, 2, 4, 8, 16, 32)


def _check_oracle(res, beams, f, dms, gulp, dmax):
    delays = oracle.delays(f, synth.TSAMP, dms)
    for (b, k), (r, c) in res.items():
        x = beams[b][0]
        win = x[k * gulp:k * gulp + gulp + dmax]
        dmt = oracle.dedisperse(win, delays, gulp)
        ob, ok = oracle.best(dmt, WIDTHS, 8192)
        o, _ = oracle.peaks(ob, ok, 6.0)
        assert r.t0 == k * gulp and r.t_done >= r.t_push > 0 and r.status == sp.SP_OK
        assert r.count == c.size
        gu.check_candidates(c, o, ob, 6.0)


@pytest.mark.parametrize("flags,max_batch", [(0, 3), (sp.SP_STREAM_PER_GULP | sp.SP_STREAM_ONE_STREAM, 1),
                                             (sp.SP_STREAM_PER_GULP, 2)])
def test_stream_parity_and_alone_vs_mix(flags, max_batch):
    nchan, gulp, ngulps, nbeams = 64, 1500, 6, 4
    dms = np.arange(0, 120.0, 1.0)
    f, dmax, data = _streams(nchan, dms, gulp, ngulps, nbeams, 31)
    plan = sp.Plan(f, synth.TSAMP, dms)
    beams = dict(enumerate(data))
    order = [(b, k) for k in range(ngulps) for b in range(nbeams)]
    s = sp.Stream(plan, nbeams, gulp, WIDTHS, 6.0, 8192, 4096, 64 << 20, max_batch=max_batch, flags=flags)
    assert s.slots >= 1 and s.n_in == gulp + dmax
    mix = _run(s, beams, order)
    assert len(mix) == nbeams * ngulps
    _check_oracle(mix, beams, f, dms, gulp, dmax)
    s.close()
    # beam 2 alone on a fresh stream: identical results
    alone_s = sp.Stream(plan, nbeams, gulp, WIDTHS, 6.0, 8192, 4096, 64 << 20, max_batch=max_batch, flags=flags)
    alone = _run(alone_s, {2: beams[2]}, [(2, k) for k in range(ngulps)])
    for k in range(ngulps):
        ra, ca = alone[(2, k)]
        rm, cm = mix[(2, k)]
        assert ra.count == rm.count and np.array_equal(ca, cm)
    alone_s.close()
    # each burst is found in the gulp that searches its arrival time
    for b in range(nbeams):
        for bu in beams[b][3]:
            k = bu.t0 // gulp
            _, c = mix[(b, k)]
            near = (np.abs(dms[c["dm_idx"]] - bu.dm) <= 5) & (np.abs(c["t"] + k * gulp - bu.t0) <= 64)
            assert near.any(), (b, bu)


def test_stream_one_slot_budget_and_errors():
    nchan, gulp, ngulps, nbeams = 32, 1000, 3, 3
    dms = np.arange(0, 60.0, 2.0)
    f, dmax, data = _streams(nchan, dms, gulp, ngulps, nbeams, 41)
    plan = sp.Plan(f, synth.TSAMP, dms)
    beams = dict(enumerate(data))
    # A budget that holds the rings and exactly one slot.
    probe = sp.Stream(plan, nbeams, gulp, WIDTHS, 6.0, 8192, 1024, 1 << 30, max_batch=4)
    per_slot = (probe.device_bytes - _ring_bytes(probe, nchan, nbeams)) // probe.slots
    probe.close()
    s = sp.Stream(plan, nbeams, gulp, WIDTHS, 6.0, 8192, 1024, _ring_bytes_plan(plan, gulp, nbeams) + per_slot + 8192,
                  max_batch=4)
    assert s.slots == 1
    with pytest.raises(sp.SpotlightError) as e:
        s.push(0, beams[0][2][0])  # no history yet
    assert e.value.code == sp.SP_EINVAL
    res = _run(s, beams, [(b, k) for k in range(ngulps) for b in range(nbeams)])
    assert len(res) == nbeams * ngulps
    _check_oracle(res, beams, f, dms, gulp, dmax)
    s.history(1, beams[1][1])
    s.push(1, beams[1][2][0])
    with pytest.raises(sp.SpotlightError) as e:
        s.history(1, beams[1][1])  # gulp pending or in flight
    assert e.value.code == sp.SP_EINVAL
    s.drain()
    with pytest.raises(sp.SpotlightError) as e:
        sp.Stream(plan, nbeams, gulp, WIDTHS, 6.0, 8192, 1024, 1024, max_batch=4)  # rings do not fit
    assert e.value.code == sp.SP_ENOMEM
    s.close()


def _ring_bytes(stream, nchan, nbeams):
    return nbeams * ((stream.n_in * nchan + 255) // 256 * 256)


def _ring_bytes_plan(plan, gulp, nbeams):
    n_in = gulp + plan.max_delay
    return nbeams * ((n_in * plan.nchan + 255) // 256 * 256)


def test_stream_full_band_gulps():
    """4096 channels, the 0-500 trial plan, 6104-sample (8.0 s) gulps: every
    gulp of several beams equals the oracle, batched in the mix."""
    nchan, gulp, ngulps, nbeams = 4096, 6104, 2, 3
    dms = synth.dm_plan_config1()
    f, dmax, data = _streams(nchan, dms, gulp, ngulps, nbeams, 51)
    plan = sp.Plan(f, synth.TSAMP, dms)
    assert dmax == plan.max_delay
    beams = dict(enumerate(data))
    s = sp.Stream(plan, nbeams, gulp, WIDTHS, 6.0, 8192, 1 << 14, 8 << 30, max_batch=4)
    res = _run(s, beams, [(b, k) for k in range(ngulps) for b in range(nbeams)])
    _check_oracle(res, beams, f, dms, gulp, dmax)
    assert plan.status() == 0
    s.close()


@pytest.mark.parametrize("with_classifier", [False, True])
def test_stream_sift_and_classify_in_the_stream(with_classifier):
    """A sifter (and classifier) attached to the stream (Sec. 3.2 per
    searched block): each gulp's kept peaks equal sp_sift of the gulp's own
    candidates, and each probability equals the standalone chain -- stage
    the window, sp_cnn_extract, sp_cnn_features, sp_cnn_forward -- on the
    same window; the forward batches of 4 inside the stream split 8 peaks."""
    nchan, gulp, ngulps, nbeams = 256, 1500, 5, 3
    dms = np.arange(0, 120.0, 1.0)
    f, dmax, data = _streams(nchan, dms, gulp, ngulps, nbeams, 57)
    plan = sp.Plan(f, synth.TSAMP, dms)
    beams = dict(enumerate(data))
    clf = sp.Classifier(max_batch=4, seed=3) if with_classifier else None
    s = sp.Stream(plan, nbeams, gulp, WIDTHS, 6.0, 8192, 4096, 1 << 32, max_batch=3)
    s.attach(clf, t_in=512, kept_cap=8, min_points=2, snr_min=8.0)
    with pytest.raises(sp.SpotlightError):
        s.attach(clf)  # once only
    for b, (_, hist, _, _) in beams.items():
        s.history(b, hist)
    res = {}
    for k in range(ngulps):
        for b in range(nbeams):
            s.push(b, beams[b][2][k])
            for r, c, kept, prob in s.poll_sifted(with_cands=True):
                res[(r.beam, r.seq)] = (r, c, kept, prob)
    for r, c, kept, prob in s.drain(with_cands=True, sifted=True):
        res[(r.beam, r.seq)] = (r, c, kept, prob)
    assert len(res) == nbeams * ngulps
    with pytest.raises(sp.SpotlightError):
        s.attach(clf)  # not after a push
    t_in, classified = 512, 0
    shift = torch.from_numpy(sp.dmt_shifts(f, 256, (t_in - 256) // 2)).cuda()
    for (b, k), (r, c, kept, prob) in sorted(res.items()):
        assert r.status == sp.SP_OK and r.count == c.size
        assert r.t_done >= r.t_search >= r.t_push > 0
        want = sp.sift(c, dms, WIDTHS, synth.TSAMP, min_points=2, snr_min=8.0)
        assert r.kept == want.size
        assert np.array_equal(kept, want[:8])
        if not with_classifier:
            assert np.all(prob == -1.0) and r.accepted == kept.size
            continue
        if kept.size == 0:
            assert r.accepted == 0
            continue
        classified += 1
        x = beams[b][0]
        win = torch.from_numpy(np.ascontiguousarray(x[k * gulp:k * gulp + gulp + dmax])).cuda()
        staged = sp.staged_buffer(nchan, win.shape[0])
        sp.stage_input(win, staged)
        d_c = torch.from_numpy(np.ascontiguousarray(kept).view(np.int32).reshape(-1, 4)).cuda()
        sub = sp.cnn_extract(plan, staged, win.shape[0], d_c, WIDTHS, t_in=t_in)
        n = kept.size
        ft = torch.empty((n, 256, 256), dtype=torch.bfloat16, device="cuda")
        img = torch.empty_like(ft)
        sp.cnn_features(sub, shift, ft, img)
        p = torch.empty(n, dtype=torch.float32, device="cuda")
        for i in range(0, n, 4):
            j = min(n, i + 4)
            clf.forward(ft[i:j].contiguous(), img[i:j].contiguous(), p[i:j])
        p = p.cpu().numpy()
        assert np.array_equal(prob, p), (b, k, prob, p)
        assert r.accepted == int((p >= 0.5).sum())
    if with_classifier:
        assert classified >= nbeams  # every beam's bursts reach the classifier
    s.close()
