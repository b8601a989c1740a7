"""The candidate classifier trained and judged on the search's own
candidates (arXiv 2606.27262, Sec. 3.2.1 sifting, Sec. 3.2.2 classification).

4096-channel beams (300-500 MHz, 1.31072 ms, 16384 searched samples, the
5751-trial plan to DM 2000) carry injected bursts (DM 50-1950, FWHM 1-64
samples, S/N 6-50) and synthetic RFI drawn into the 8-bit filterbank itself:
persistent narrowband channels, broadband DM-0 impulses and drifting
periodic tones.  Every beam goes through the library's search, the host
sifter (DBSCAN, S/N >= 10, DM >= 10), cutouts of the kept peaks and their
images; a kept peak is a burst when it lies on an injection.  The network is
pre-trained on synthetic subband spectra and then trained on the kept peaks
of one set of beams, by the library's own forward, backward and Adam
kernels, and judged on another set: every burst injected at S/N >= 8 that
the sifter keeps must be accepted (recall >= 0.99 relative to the sifter,
which judges it), and the classifier must pass fewer of the sifter's
non-burst peaks (RFI and noise) than the sifter alone does."""
import numpy as np
import pytest
import torch

import paper_2606_27262_gb300 as sp
import synth
from paper_2606_27262_gb300 import build as spbuild
from paper_2606_27262_gb300 import learning
from synth import classifier as scls
from synth import rfi

pytestmark = pytest.mark.gpu

N_OUT = 16384
FREQS = synth.band_freqs(4096)
WIDTHS = synth.widths_pow2(256)
TRAIN_BEAMS = 160
TEST_BEAMS = 48


def beam_truths(seed):
    rng = np.random.default_rng((seed, 7))
    bursts = synth.draw_bursts(rng, 4, N_OUT, 50.0, 1950.0, 1.0, 64.0, 6.0, 50.0)
    events = rfi.draw_rfi(rng, int(rng.integers(3, 7)), N_OUT + 44995, 4096)
    return bursts, events


def make_beam(seed, out):
    bursts, events = beam_truths(seed)
    synth.make_beam_torch(seed, out, FREQS, bursts, widths=WIDTHS,
                          extra=rfi.rfi_signal(events, out.shape[0], out.shape[1]))
    return [learning.Truth(b.t0, b.dm, b.fwhm, b.snr) for b in bursts]


def harvest(h, seeds, beam):
    fts, dms, labs, peaks, truths_all, n_cands = [], [], [], [], [], 0
    for s in seeds:
        truths = make_beam(s, beam)
        ft, dm_img, lab, kept, which, n = h.run(beam, truths)
        fts.append(ft)
        dms.append(dm_img)
        labs.append(lab)
        peaks.append((kept, which))
        truths_all.append(truths)
        n_cands += n
    return torch.cat(fts), torch.cat(dms), np.concatenate(labs), peaks, truths_all, n_cands


@pytest.fixture(scope="module")
def pipeline():
    spbuild.build()
    assert torch.cuda.is_available()
    plan = sp.Plan(FREQS, synth.TSAMP, synth.dm_plan_config2())
    h = learning.Harvester(plan, N_OUT, WIDTHS, 6.0, 8192)
    beam = torch.empty((N_OUT + plan.max_delay, 4096), dtype=torch.uint8, device="cuda")
    train_set = harvest(h, range(TRAIN_BEAMS), beam)
    test_set = harvest(h, range(10_000, 10_000 + TEST_BEAMS), beam)
    clf = sp.Classifier(max_batch=64, seed=21)
    rng = np.random.default_rng(8)

    def sample(n):
        sub, labels, _ = scls.classifier_batch(rng, n, FREQS, t_in=512, p_burst=0.6)
        return sub, labels
    pre = learning.train(clf, learning.subband_batches(sample, FREQS, 64), 2000)
    ft, dm_img, lab = train_set[0], train_set[1], train_set[2]
    post = learning.train(clf, learning.pool_batches(ft, dm_img, lab, rng, 64), 1500, lr=1e-3)
    yield plan, clf, train_set, test_set, pre + post
    clf.close()


def test_training_set_has_both_classes(pipeline):
    _, _, train_set, _, losses = pipeline
    lab = train_set[2]
    print(f"pipeline training set: {lab.size} kept peaks from {TRAIN_BEAMS} beams "
          f"({int(lab.sum())} on bursts) out of {train_set[5]} search candidates")
    assert lab.sum() >= 100 and (lab == 0).sum() >= 100
    assert losses[-1] < losses[0]


def test_classifier_on_pipeline_candidates(pipeline):
    plan, clf, _, test_set, _ = pipeline
    ft, dm_img, lab, peaks, truths_all, n_cands = test_set
    p = learning.classify(clf, ft, dm_img)
    # per beam: bursts the sifter kept (some peak on them) and whether the
    # classifier accepted one of those peaks
    kept_bursts = accepted_bursts = 0
    off = 0
    for (kept, which), truths in zip(peaks, truths_all):
        pb = p[off:off + kept.size]
        off += kept.size
        for i, tr in enumerate(truths):
            on = which == i
            if tr.snr < 8.0 or not on.any():
                continue
            kept_bursts += 1
            accepted_bursts += bool((pb[on] >= 0.5).any())
    noise = lab == 0
    fp_sifter = int(noise.sum())
    fp_clf = int((p[noise] >= 0.5).sum())
    recall = accepted_bursts / max(kept_bursts, 1)
    injected = sum(1 for tr in truths_all for t in tr if t.snr >= 8.0)
    print(f"pipeline candidates of {TEST_BEAMS} held-out beams: {n_cands} found, {lab.size} kept by the sifter; "
          f"bursts S/N >= 8: {injected} injected, {kept_bursts} kept, {accepted_bursts} accepted "
          f"(recall {recall:.4f}); non-burst peaks passed: sifter alone {fp_sifter}, with the classifier {fp_clf}")
    assert kept_bursts >= 0.8 * injected
    assert recall >= 0.99
    assert fp_clf < fp_sifter
