"""bench.py's multi-rank helpers on CPU with the gloo backend (world size 2):
the slowest rank's time wins, every rank searches its own beam, and the
JSON-line helpers need no GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, lr = bench.dist_env()
    bench.dist_init(w, "gloo")
    bench.barrier(w)
    m = bench.reduce_max(10.0 * (r + 1), w)
    seed = bench.beam_seed(1002, r)
    q.put((r, m, seed))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_distinct_beams():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [m for _, m, _ in res] == [20.0, 20.0]
    assert len({s for _, _, s in res}) == world


def test_single_rank_helpers():
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)
    wl = bench.workload(4096)
    assert wl.n_out == 4096 and wl.nchan == 4096
    assert bench.workload().n_out == 131072


def test_profiled_traffic_guard(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "PROFILE_JSON", str(tmp_path / "p.json"))
    assert bench.profiled_traffic(131072) is None
    (tmp_path / "p.json").write_text('{"kernel_source_sha256_16": "stale", "n_out": 131072, '
                                     '"dram_bytes_per_launch_full_config": 5}')
    assert bench.profiled_traffic(131072) is None
    h = bench.kernel_source_hash()
    (tmp_path / "p.json").write_text('{"kernel_source_sha256_16": "%s", "n_out": 131072, '
                                     '"dram_bytes_per_launch_full_config": 5}' % h)
    assert bench.profiled_traffic(131072) == 5.0
    assert bench.profiled_traffic(16384) is None  # another workload length


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the CPU oracle on the host cores) prints
    one JSON line with the contract's keys; small workload, one step."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--n-out", "16384",
                          "--steps", "1", "--warmup", "0", "--cpu-stride", "256"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # a step is the sampled work: its time is what ran, the extrapolation is stated
    assert line["extrapolated"] is True and 0 < line["trial_fraction"] < 1
    assert abs(line["full_beam_s_extrapolated"] * line["trial_fraction"] - line["ms_per_step"] / 1e3) < 1e-6
    beam_s = 16384 * 1.31072e-3
    assert abs(line["value"] - beam_s * line["trial_fraction"] / (line["ms_per_step"] / 1e3)) < 1e-9 * line["value"]
