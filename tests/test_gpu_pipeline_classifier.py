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


def make_beam(seed, out):
    bursts = rfi.pipeline_beam(seed, out, FREQS, N_OUT, WIDTHS)
    return [learning.Truth(b.t0, b.dm, b.fwhm, b.snr) for b in bursts]


@pytest.fixture(scope="module")
def pipeline():
    spbuild.build()
    assert torch.cuda.is_available()
    plan = sp.Plan(FREQS, synth.TSAMP, synth.dm_plan_config2())
    h = learning.Harvester(plan, N_OUT, WIDTHS, 6.0, 8192)
    beam = torch.empty((N_OUT + plan.max_delay, 4096), dtype=torch.uint8, device="cuda")
    train_set = learning.harvest_beams(h, make_beam, range(TRAIN_BEAMS), beam)
    test_set = learning.harvest_beams(h, make_beam, range(10_000, 10_000 + TEST_BEAMS), beam)
    clf = sp.Classifier(max_batch=64, seed=21)
    rng = np.random.default_rng(8)

    def sample(n):
        sub, labels, _ = scls.classifier_batch(rng, n, FREQS, t_in=512, p_burst=0.6)
        return sub, labels
    pre = learning.train(clf, learning.subband_batches(sample, FREQS, 64), 2000)
    post = learning.train(clf, learning.pool_batches(train_set.ft, train_set.dm_img, train_set.labels, rng, 64),
                          1500, lr=1e-3)
    yield plan, clf, train_set, test_set, pre + post
    clf.close()


def test_training_set_has_both_classes(pipeline):
    _, _, train_set, _, losses = pipeline
    lab = train_set.labels
    print(f"pipeline training set: {lab.size} kept peaks from {TRAIN_BEAMS} beams "
          f"({int(lab.sum())} on bursts) out of {train_set.candidates} search candidates")
    assert lab.sum() >= 100 and (lab == 0).sum() >= 100
    assert losses[-1] < losses[0]


def test_classifier_on_pipeline_candidates(pipeline):
    plan, clf, _, test_set, _ = pipeline
    p = learning.classify(clf, test_set.ft, test_set.dm_img)
    j = learning.assess(p, test_set)
    print(f"pipeline candidates of {TEST_BEAMS} held-out beams: {j['candidates']} found, {j['kept_peaks']} kept "
          f"by the sifter; bursts S/N >= 8: {j['injected']} injected, {j['kept']} kept, {j['accepted']} accepted "
          f"(recall {j['recall']:.4f}); non-burst peaks passed: sifter alone {j['fp_sifter']}, "
          f"with the classifier {j['fp_classifier']}")
    assert j["kept"] >= 0.8 * j["injected"]
    assert j["recall"] >= 0.99
    assert j["fp_classifier"] < j["fp_sifter"]
