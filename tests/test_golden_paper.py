"""The sampling constants of the synthetic workloads against the arithmetic
the paper prints (tests/golden/paper_arithmetic.json)."""
import json
import os

import synth

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_arithmetic.json")))


def test_sampling_and_ring_arithmetic():
    assert synth.TSAMP == G["tsamp_s"]["value"]
    blk = G["telring_block_s"]
    assert abs(blk["samples"] * synth.TSAMP - blk["value"]) < 1e-12
    assert abs(G["telring_total_s"]["blocks"] * blk["value"] - G["telring_total_s"]["value"]) < 1e-12
    fb = G["frbring_block_s"]
    assert abs(fb["telring_blocks"] * blk["value"] - fb["value"]) < 1e-12
    assert abs(G["frbring_total_s"]["blocks"] * fb["value"] - G["frbring_total_s"]["value"]) < 1e-9
    assert abs(G["read_segment_s"]["blocks"] * fb["value"] - G["read_segment_s"]["value"]) < 1e-9
    rb = G["frbring_bytes"]
    samples = round(G["frbring_total_s"]["value"] / synth.TSAMP)
    assert samples == 307200
    assert rb["beams"] * rb["nchan"] * samples == rb["value_gib"] * 2 ** 30


def test_band3_axis():
    f = synth.band_freqs(4096)
    assert f[0] == 500.0 and abs(f[-1] - (500.0 - 4095 * 200.0 / 4096)) < 1e-12
    assert (f[1:] < f[:-1]).all()
    assert synth.dm_plan_config1().size == 501
    d2 = synth.dm_plan_config2()
    assert d2.size == 5751 and d2[0] == 0.0 and d2[-1] == 2000.0 and (d2[1:] > d2[:-1]).all()
