"""Training data and training loop of the candidate classifier (arXiv
2606.27262, Sec. 3.2: candidates of the search are clustered by the sifter,
their kept peaks are cut from the data and scored by a convolutional
classifier trained on labelled examples).

Everything that computes runs in the library's kernels through this
package's bindings: staging, dedispersion, the search, cutouts of the kept
peaks, their images, and the classifier's forward, backward and Adam steps.
The sifter runs on the host inside the library.  This module only arranges
the calls, holds the buffers they share, and labels each kept peak by the
injection it lies on (a burst of known arrival time, DM and width), so that
the network can be trained and judged on the search's own candidates.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import (CAND_DTYPE, Classifier, Plan, cnn_extract, cnn_features, dedisperse_staged, dmt_shifts, library,
               sift, single_pulse_search, sps_workspace_bytes, stage_input, staged_buffer)

CUT = 256  # image side of the classifier (frequency-time and DM-time)


@dataclasses.dataclass
class Truth:
    """An injected burst: arrival sample at the top channel, DM, FWHM in
    samples and its target S/N."""
    t0: int
    dm: float
    fwhm: float
    snr: float


def match_peaks(peaks: np.ndarray, dms: np.ndarray, widths, truths: list[Truth]) -> np.ndarray:
    """Index of the injected burst each kept peak lies on, or -1.  A peak
    (boxcar [t, t + w) at trial DM d) lies on a burst when the window reaches
    the burst's arrival within twice its FWHM plus 8 samples and the DM is
    within 3 % + 3 pc cm^-3 of the burst's."""
    out = np.full(peaks.size, -1, np.int64)
    if not truths or peaks.size == 0:
        return out
    t = peaks["t"].astype(np.int64)
    w = np.asarray(widths, np.int64)[peaks["width_idx"]]
    d = np.asarray(dms, np.float64)[peaks["dm_idx"]]
    best = np.full(peaks.size, np.inf)
    for i, b in enumerate(truths):
        slack = 2.0 * b.fwhm + 8.0
        ok = (t <= b.t0 + slack) & (t + w >= b.t0 - slack) & (np.abs(d - b.dm) <= 0.03 * b.dm + 3.0)
        dist = np.abs(d - b.dm)
        take = ok & (dist < best)
        out[take] = i
        best[take] = dist[take]
    return out


class Harvester:
    """Runs the search, the sifter and the feature extraction on device
    beams of one plan and length, keeping the kept peaks' images (bf16
    [n][256][256] frequency-time and DM-time CUDA tensors) with their labels
    (1 on an injected burst, else 0)."""

    def __init__(self, plan: Plan, n_out: int, widths, threshold: float, norm_block: int, t_in: int = 512,
                 max_sweep: int = 128, cand_cap: int = 1 << 21, device="cuda"):
        import torch
        self.plan, self.n_out, self.n_in = plan, int(n_out), int(n_out) + plan.max_delay
        self.widths = np.asarray(widths, np.int32)
        self.threshold, self.norm_block, self.t_in = float(threshold), int(norm_block), int(t_in)
        self.dms = plan.dms
        self.staged = staged_buffer(plan.nchan, self.n_in, device)
        self.dmt = torch.empty((plan.ndm, self.n_out), dtype=torch.int32, device=device)
        self.sw = torch.empty(sps_workspace_bytes(plan.ndm, self.n_out, self.widths.size, self.norm_block),
                              dtype=torch.uint8, device=device)
        self.cands = torch.empty((cand_cap, 4), dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.shift = torch.from_numpy(dmt_shifts(plan.freqs, CUT, max_sweep)).to(device)
        self.device = device

    def run(self, beam, truths: list[Truth]):
        """beam: uint8 CUDA tensor [n_in][nchan].  Returns (ft, dmt images,
        labels float32 [n], kept peaks (CAND_DTYPE), burst index per peak,
        candidates the search found)."""
        import torch
        stage_input(beam, self.staged)
        dedisperse_staged(self.plan, self.staged, self.n_in, self.dmt)
        single_pulse_search(self.dmt, self.widths, self.threshold, self.norm_block, self.sw, self.cands, self.count)
        n = min(int(self.count.item()), self.cands.shape[0])
        rec = np.ascontiguousarray(self.cands[:n].cpu().numpy()).view(CAND_DTYPE).reshape(-1)
        kept = sift(np.sort(rec, order=["dm_idx", "t"]), self.dms, self.widths, self.plan.tsamp)
        which = match_peaks(kept, self.dms, self.widths, truths)
        labels = (which >= 0).astype(np.float32)
        if kept.size == 0:
            empty = torch.empty((0, CUT, CUT), dtype=torch.bfloat16, device=self.device)
            return empty, empty.clone(), labels, kept, which, n
        d_k = torch.from_numpy(np.ascontiguousarray(kept).view(np.int32).reshape(-1, 4)).to(self.device)
        sub = cnn_extract(self.plan, self.staged, self.n_in, d_k, self.widths, t_in=self.t_in)
        ft = torch.empty((kept.size, CUT, CUT), dtype=torch.bfloat16, device=self.device)
        dm_img = torch.empty_like(ft)
        cnn_features(sub, self.shift, ft, dm_img)
        return ft, dm_img, labels, kept, which, n


def classify(clf: Classifier, ft, dm_img):
    """Probabilities (numpy float32 [n]) of images in batches of the
    network's size."""
    import torch
    n = int(ft.shape[0])
    p = torch.empty(max(n, 1), dtype=torch.float32, device=ft.device)
    for i in range(0, n, clf.max_batch):
        j = min(n, i + clf.max_batch)
        clf.forward(ft[i:j].contiguous(), dm_img[i:j].contiguous(), p[i:j])
    return p[:n].cpu().numpy()


def train(clf: Classifier, batch_fn, steps: int, lr: float = 2e-3, loss_every: int = 50):
    """Adam with a cosine learning-rate schedule over ``steps`` batches from
    batch_fn(step) -> (ft, dm_img, labels CUDA tensors).  Returns the losses
    sampled every ``loss_every`` steps."""
    losses = []
    for k in range(steps):
        ft, dm_img, labels = batch_fn(k)
        rate = lr * 0.5 * (1.0 + np.cos(np.pi * k / steps))
        loss = clf.train_step(ft, dm_img, labels, rate, want_loss=(k % loss_every == 0))
        if loss is not None:
            losses.append(loss)
    return losses


def subband_batches(sample_fn, freqs, batch: int, max_sweep: int = 128, device="cuda"):
    """batch_fn for ``train`` from sample_fn(batch) -> (subband spectra
    float32 CUDA tensor [batch][256][t_in], labels numpy [batch]): the
    images are made by the library's feature kernel."""
    import torch
    shift = torch.from_numpy(dmt_shifts(freqs, CUT, max_sweep)).to(device)
    ft = torch.empty((batch, CUT, CUT), dtype=torch.bfloat16, device=device)
    dm_img = torch.empty_like(ft)
    work = torch.empty(int(library().sp_cnn_features_workspace_bytes(batch)), dtype=torch.uint8, device=device)

    def fn(_k):
        sub, labels = sample_fn(batch)
        cnn_features(sub, shift, ft, dm_img, work)
        return ft, dm_img, torch.from_numpy(np.asarray(labels, np.float32)).to(device)
    return fn


def pool_batches(ft, dm_img, labels: np.ndarray, rng, batch: int, p_pos: float = 0.5):
    """batch_fn drawing from a pool of harvested examples, positives and
    negatives in proportion p_pos (with replacement)."""
    import torch
    pos, neg = np.flatnonzero(labels > 0.5), np.flatnonzero(labels <= 0.5)
    lab_d = torch.from_numpy(labels.astype(np.float32)).to(ft.device)

    def fn(_k):
        npos = int(rng.binomial(batch, p_pos)) if pos.size and neg.size else (batch if pos.size else 0)
        idx = np.concatenate([rng.choice(pos, npos), rng.choice(neg, batch - npos)]) if neg.size else \
            rng.choice(pos, batch)
        it = torch.from_numpy(idx).to(ft.device)
        return ft.index_select(0, it).contiguous(), dm_img.index_select(0, it).contiguous(), lab_d.index_select(0, it)
    return fn


@dataclasses.dataclass
class Harvest:
    """Kept peaks of many beams: images, labels, and per beam the peaks,
    the burst each lies on (-1: none) and the injected bursts."""
    ft: object
    dm_img: object
    labels: np.ndarray
    beams: list
    candidates: int


def harvest_beams(h: Harvester, make_beam, seeds, beam) -> Harvest:
    """Runs ``h`` on the beam make_beam(seed, beam) -> truths writes into the
    device tensor ``beam`` for every seed."""
    import torch
    fts, dms, labs, beams, n_cands = [], [], [], [], 0
    for s in seeds:
        truths = make_beam(s, beam)
        ft, dm_img, lab, kept, which, n = h.run(beam, truths)
        fts.append(ft)
        dms.append(dm_img)
        labs.append(lab)
        beams.append((kept, which, truths))
        n_cands += n
    return Harvest(torch.cat(fts), torch.cat(dms), np.concatenate(labs), beams, n_cands)


def assess(p: np.ndarray, hv: Harvest, snr_min: float = 8.0, p_min: float = 0.5) -> dict:
    """Recall and false positives of probabilities p (one per kept peak of
    ``hv``): a burst injected at S/N >= snr_min counts as kept when the
    sifter kept a peak on it, and as accepted when one of those peaks has
    p >= p_min; non-burst peaks are the sifter's false positives."""
    kept_b = acc_b = injected = 0
    off = 0
    for kept, which, truths in hv.beams:
        pb = p[off:off + kept.size]
        off += kept.size
        for i, tr in enumerate(truths):
            if tr.snr < snr_min:
                continue
            injected += 1
            on = which == i
            if on.any():
                kept_b += 1
                acc_b += bool((pb[on] >= p_min).any())
    noise = hv.labels == 0
    return {"injected": injected, "kept": kept_b, "accepted": acc_b, "recall": acc_b / max(kept_b, 1),
            "fp_sifter": int(noise.sum()), "fp_classifier": int((p[noise] >= p_min).sum()),
            "kept_peaks": int(hv.labels.size), "candidates": int(hv.candidates)}
