"""Streamed candidate search (Sec. 3.1.2: boxcar S/N from a running
cumulative sum, threshold, 3x3 peak filter) against the oracle.

The library takes the streamed kernel for power-of-two width lists up to 256,
16-byte-aligned rows and blocks that are a multiple of 256 samples (or one
block); it walks segments of 16 chunks of 256 samples, keeps a two-chunk ring
of prefix sums per row, puts every point through an integer pre-filter and
leaves the beam's last chunk and any chunk it cannot prove exact in 2^22 to
the tile kernel (and on to the 64-bit pass).  These cases cross chunk and
segment boundaries, the DM edges, block edges, listed tiles of both kinds and
thresholds at which every point passes the pre-filter."""
import numpy as np
import pytest
import torch

import oracle
import paper_2606_27262_gb300 as sp
from paper_2606_27262_gb300 import build as spbuild
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

SEG = 16 * 256  # samples per segment of the streamed kernel


@pytest.fixture(scope="module", autouse=True)
def _built():
    spbuild.build()
    assert torch.cuda.is_available()


def _noise(rng, ndm, n_out):
    return np.rint(rng.normal(5.2e5, 1024.0, size=(ndm, n_out))).astype(np.int32)


def _plant_pulses(dmt, rng, times):
    ndm = dmt.shape[0]
    for t in times:
        d = int(rng.integers(0, ndm))
        w = int(rng.choice([1, 3, 8, 40]))
        for dd in (-1, 0, 1):
            if 0 <= d + dd < ndm:
                dmt[d + dd, t: t + w] += int(9000 if dd == 0 else 4000)


def _search(dmt_np, widths, thr, L):
    launches = sp.launch_count()
    g, n = gu.dev_candidates(torch.from_numpy(dmt_np).cuda(), widths, thr, L)
    return g, n, sp.launch_count() - launches


def _check(dmt, widths, L, thrs, streamed=True):
    ob, ok = oracle.best(dmt, widths, L)
    found = 0
    for thr in thrs:
        g, n, kernels = _search(dmt, widths, thr, L)
        # sums, coefficients, streamed search, tile kernel over the tiles it
        # lists, 64-bit pass -- against sums, coefficients, tile kernel, 64-bit
        # pass
        assert kernels == (5 if streamed else 4)
        o, _ = oracle.peaks(ob, ok, thr)
        assert n == g.size
        found += gu.check_candidates(g, o, ob, thr)
    return found


BOUNDARY_TIMES = [0, 1, 255, 256, 511, SEG - 1, SEG, SEG + 1, 2 * SEG - 1, 2 * SEG, 2 * SEG + 255]


@pytest.mark.parametrize("ndm", [1, 13, 14, 15, 29])
def test_stream_segments_and_dm_edges(ndm):
    """Three segments (16 + 16 + 1 chunks) and the beam's tail chunk; pulses on
    chunk and segment boundaries; row groups with 1 to 14 rows."""
    rng = np.random.default_rng(100 + ndm)
    n_out = 2 * SEG + 512 + 100  # n_out / 256 = 34 chunks: 33 streamed
    dmt = _noise(rng, ndm, n_out)
    _plant_pulses(dmt, rng, BOUNDARY_TIMES)
    assert _check(dmt, sp_widths(256), 0, (6.0, 3.0)) > 0


def sp_widths(maxw):
    return [1 << k for k in range(maxw.bit_length()) if (1 << k) <= maxw]


@pytest.mark.parametrize("L", [256, 1024, 3 * 256 * 5])
def test_stream_blocks(L):
    """Blocks of 256, 1024 and 3840 samples (the last takes the remainder):
    halo points of a chunk use their own block's statistics; a step in the
    mean between blocks."""
    rng = np.random.default_rng(L)
    ndm, n_out = 20, 2 * SEG + 3000
    dmt = _noise(rng, ndm, n_out)
    dmt[:, n_out // 2:] += 3000  # a level step
    _plant_pulses(dmt, rng, [L - 1, L, 2 * L - 3, 2 * L, n_out // 2 - 2, n_out // 2])
    _check(dmt, sp_widths(32), L, (5.0, 0.0))


def test_stream_single_chunk_beams():
    """n_out of 512 and 700: one streamed chunk, the rest in the tile kernel."""
    rng = np.random.default_rng(7)
    for n_out in (512, 700):
        dmt = _noise(rng, 16, n_out)
        _plant_pulses(dmt, rng, [0, 255, 256, 300])
        _check(dmt, sp_widths(256), 0, (6.0, 2.0))


def test_stream_listed_tiles():
    """Chunks whose window sums exceed 2^22 (listed for the 32-bit tile
    kernel) and 2^31 (passed on to the 64-bit pass) among streamed ones."""
    rng = np.random.default_rng(11)
    ndm, n_out = 30, SEG + 2048
    dmt = _noise(rng, ndm, n_out)
    dmt[3, 1000:1010] += 1_000_000            # dev * 256 > 2^22: 32-bit tile kernel
    dmt[17, 5000:5300] += 9_000_000           # dev * 256 > 2^31: 64-bit pass
    dmt[25, SEG - 6:SEG + 4] -= 2_000_000     # across a segment boundary
    _plant_pulses(dmt, rng, [300, 2000, 7000])
    _check(dmt, sp_widths(256), 0, (6.0, 1.0))


@pytest.mark.parametrize("thr", [-1e30, -2.5, 0.0])
def test_stream_low_thresholds(thr):
    """Thresholds at or below zero: every point, or most, passes the
    pre-filter and the peak filter decides alone."""
    rng = np.random.default_rng(5)
    dmt = _noise(rng, 17, 1300)
    _check(dmt, sp_widths(64), 512, (thr,))


def test_stream_zero_variance_rows():
    """Flat rows (S/N 0 everywhere) beside noisy ones."""
    rng = np.random.default_rng(9)
    dmt = _noise(rng, 12, 2048)
    dmt[2:5] = 777
    _check(dmt, sp_widths(16), 0, (0.0, 3.0))


def test_non_pow2_widths_use_the_tile_kernel():
    rng = np.random.default_rng(13)
    dmt = _noise(rng, 9, 2048)
    _check(dmt, [1, 3, 5, 17], 0, (3.0,), streamed=False)
    _check(dmt, sp_widths(512), 0, (3.0,), streamed=False)  # widths past 256
    _check(dmt, sp_widths(32), 1000, (3.0,), streamed=False)  # blocks not a multiple of 256


def test_stream_threshold_at_exact_values():
    """Thresholds set exactly to S/N values the library computes: a 3x3 peak
    whose best S/N equals the threshold is a candidate (v >= thr), so the
    pre-filter's bound must let every such window through.  The values come
    from the best-S/N map, whose tile kernel evaluates the same expression as
    the streamed kernel's exact path on these noise rows."""
    rng = np.random.default_rng(21)
    ndm, n_out = 20, 3 * 256 + 40
    dmt = _noise(rng, ndm, n_out)
    _plant_pulses(dmt, rng, [100, 300, 520])
    gb, _ = gu.dev_best_map(torch.from_numpy(dmt).cuda(), sp_widths(256), 0)
    fin = np.where(np.isfinite(gb), gb, -np.inf)
    pad = np.pad(fin, 1, constant_values=-np.inf)
    # strict 3x3 maxima (no ties) in the streamed chunks (t < 512)
    nb = np.stack([pad[1 + a: 1 + a + ndm, 1 + b: 1 + b + n_out] for a in (-1, 0, 1) for b in (-1, 0, 1)
                   if a or b])
    peak = (fin > nb.max(axis=0)) & np.isfinite(fin)
    peak[:, 512:] = False
    d_idx, t_idx = np.nonzero(peak)
    order = np.argsort(-fin[d_idx, t_idx])
    picks = [(int(d_idx[i]), int(t_idx[i])) for i in order[:: max(1, order.size // 12)][:12]]
    assert len(picks) >= 6
    for d, t in picks:
        thr = float(gb[d, t])
        g, n, kernels = _search(dmt, sp_widths(256), thr, 0)
        assert kernels == 5
        found = {(int(a), int(b)): float(v) for a, b, v in zip(g["dm_idx"], g["t"], g["snr"])}
        assert (d, t) in found, (d, t, thr)
        assert found[(d, t)] == np.float32(thr)
        assert all(v >= np.float32(thr) for v in found.values())
