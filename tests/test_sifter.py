"""Candidate sifter (arXiv 2606.27262, Sec. 3.2.1): the oracle pinned to an
independent DBSCAN (scikit-learn) and to hand-made cases, and the library's
host sifter (sp_sift) against the oracle.  No GPU needed."""
import numpy as np
import pytest

import oracle
import paper_2606_27262_gb300 as sp
import synth
from oracle import sift as osift
from paper_2606_27262_gb300 import build as spbuild


@pytest.fixture(scope="module", autouse=True)
def _built():
    spbuild.build()


def _cands(dm_idx, t, snr, width_idx=None):
    c = np.zeros(len(dm_idx), sp.CAND_DTYPE)
    c["dm_idx"], c["t"], c["snr"] = dm_idx, t, snr
    c["width_idx"] = 0 if width_idx is None else width_idx
    return c


def _random_cloud(rng, ncl=6, per=30, noise=80, ndm=400, nt=20000):
    dm, t = [], []
    for _ in range(ncl):
        d0, t0 = rng.integers(0, ndm), rng.integers(0, nt)
        dm += list(np.clip(d0 + rng.integers(-4, 5, per), 0, ndm - 1))
        t += list(np.clip(t0 + rng.integers(-200, 201, per), 0, nt - 1))
    dm += list(rng.integers(0, ndm, noise))
    t += list(rng.integers(0, nt, noise))
    snr = rng.uniform(6, 40, len(dm)).astype(np.float32)
    return _cands(np.array(dm), np.array(t), snr, rng.integers(0, 6, len(dm)))


def test_oracle_dbscan_matches_sklearn():
    cluster = pytest.importorskip("sklearn.cluster")
    rng = np.random.default_rng(3)
    for trial in range(8):
        n = int(rng.integers(20, 400))
        x = np.concatenate([rng.normal(rng.uniform(0, 20), 0.3, n // 2), rng.uniform(0, 20, n - n // 2)])
        y = np.concatenate([rng.normal(rng.uniform(0, 20), 0.3, n // 2), rng.uniform(0, 20, n - n // 2)])
        eps, mp = float(rng.uniform(0.2, 0.8)), int(rng.integers(2, 8))
        lab, core = osift.dbscan(x, y, eps, mp)
        ref = cluster.DBSCAN(eps=eps, min_samples=mp).fit(np.stack([x, y], 1))
        rcore = np.zeros(n, bool)
        rcore[ref.core_sample_indices_] = True
        assert np.array_equal(core, rcore)
        assert np.array_equal(lab == -1, ref.labels_ == -1)  # noise is unique
        # partition of the core points is unique up to renaming
        pairs = {(a, b) for a, b in zip(lab[core], ref.labels_[core])}
        assert len(pairs) == len({a for a, _ in pairs}) == len({b for _, b in pairs})
        # border points sit within eps of a core point of their cluster
        for i in np.flatnonzero((lab >= 0) & ~core):
            near = ((x - x[i]) ** 2 + (y - y[i]) ** 2 <= eps * eps) & core & (lab == lab[i])
            assert near.any()


def test_oracle_sift_rules():
    dms = np.arange(0, 100, 0.1)
    widths = [1, 2, 4, 8, 16, 32, 64, 128]
    ts = 1e-3
    # 4 points within eps: noise; 5: one cluster, its highest S/N is kept
    c4 = _cands([400, 400, 401, 401], [1000, 1010, 1000, 1010], [20, 30, 25, 22])
    assert osift.sift(c4, dms, widths, ts)[0].size == 0
    c5 = _cands([400, 400, 401, 401, 400], [1000, 1010, 1000, 1010, 1005], [20, 30, 25, 22, 29])
    kept, lab = osift.sift(c5, dms, widths, ts)
    assert kept.size == 1 and kept["snr"][0] == 30 and (lab == 0).all()
    # neighbours need distance <= eps: DM 0.6 apart breaks the cluster
    far = c5.copy(); far["dm_idx"][[2, 3]] = 406
    assert osift.sift(far, dms, widths, ts)[0].size == 0
    # thresholds: S/N below 10, DM below 10, width above 100 ms
    lo = c5.copy(); lo["snr"] = [9, 9.5, 9.9, 8, 7]
    assert osift.sift(lo, dms, widths, ts)[0].size == 0
    low_dm = c5.copy(); low_dm["dm_idx"] -= 310  # DM 9.0 - 9.1
    assert osift.sift(low_dm, dms, widths, ts)[0].size == 0
    wide = c5.copy(); wide["width_idx"] = 7  # 128 ms
    assert osift.sift(wide, dms, widths, ts)[0].size == 0
    assert osift.sift(wide, dms, widths, ts, width_max_s=0.2)[0].size == 1
    # two clusters far apart in time (> eps seconds): two peaks
    two = np.concatenate([c5, _cands([400, 400, 401, 401, 400], [5000, 5010, 5000, 5010, 5005],
                                     [11, 12, 13, 14, 15])])
    kept, _ = osift.sift(two, dms, widths, ts)
    assert list(kept["t"]) == [1010, 5005] and list(kept["snr"]) == [30, 15]


def test_library_sift_matches_oracle_random():
    rng = np.random.default_rng(11)
    dms = synth.dm_plan_config2()[:400]
    widths = synth.widths_pow2(32)
    for trial in range(10):
        c = _random_cloud(rng, ncl=int(rng.integers(1, 10)), per=int(rng.integers(3, 60)))
        if trial % 3 == 0:
            c["snr"] = np.round(c["snr"])  # ties
        rng.shuffle(c)
        for tsamp, eps in [(synth.TSAMP, 0.5), (1e-4, 0.05), (synth.TSAMP, 1.5)]:
            want, wl = osift.sift(c, dms, widths, tsamp, eps=eps, snr_min=8.0, dm_min=1.0)
            got, gl = sp.sift(c, dms, widths, tsamp, labels=True, eps=eps, snr_min=8.0, dm_min=1.0)
            assert np.array_equal(gl, wl)
            assert np.array_equal(got, want)


def test_library_sift_on_oracle_search():
    """Config 1 candidates from the oracle's own search: the library sifter
    equals the oracle sifter, and every injected burst of S/N >= 10 keeps a
    peak near its DM and arrival time."""
    wl = synth.config1()
    d = oracle.delays(wl.freqs, wl.tsamp, wl.dms)
    x, bursts = synth.make_workload_beam(wl, wl.n_out + int(d.max()))
    *_, found, _ = oracle.search(x, d, wl.n_out, wl.widths, wl.threshold, wl.norm_block)
    cands = np.zeros(found.size, sp.CAND_DTYPE)
    for f in ("dm_idx", "t", "width_idx", "snr"):
        cands[f] = found[f]
    want, wlab = osift.sift(cands, wl.dms, wl.widths, wl.tsamp)
    got, glab = sp.sift(cands, wl.dms, wl.widths, wl.tsamp, labels=True)
    assert np.array_equal(glab, wlab) and np.array_equal(got, want)
    assert got.size < cands.size
    for b in bursts:
        if b.snr >= 12:
            near = (np.abs(wl.dms[got["dm_idx"]] - b.dm) <= 10) & (np.abs(got["t"] - b.t0) <= 64)
            assert near.any(), b


def test_library_sift_errors_and_overflow():
    dms = np.arange(10.0, 60.0)
    c = _cands([1, 1, 1, 1, 1], [100, 101, 102, 103, 104], [20, 21, 22, 23, 24])
    assert sp.sift(c, dms, [1, 2], 1e-3).size == 1
    bad = c.copy(); bad["dm_idx"][0] = 99
    with pytest.raises(sp.SpotlightError) as e:
        sp.sift(bad, dms, [1, 2], 1e-3)
    assert e.value.code == sp.SP_EINVAL
    assert sp.sift(c[:0], dms, [1, 2], 1e-3).size == 0
