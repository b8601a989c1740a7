#!/usr/bin/env python3
"""Benchmark of the SPOTLIGHT search hot path on GB300 (arXiv 2606.27262,
Sec. 3.1): real-time beams per GPU for one full-size beam per step.

Workload (one step = one beam through the whole path): 4096 channels over
300-500 MHz, 1.31072 ms sampling, 131072 searched samples (+44995 overlap),
5751 trial DMs on the 0.1/0.2/0.5/1.0 step schedule to 2000 pc cm^-3, boxcar
widths 1..256, threshold 6 sigma, normalisation blocks of 8192 samples.  The
input (721 MB) and the DM transform (3.0 GB) are larger than the 129 MB L2,
so no L2 flush is needed between steps.

  value   real-time beams = ranks * (131072 * 1.31072 ms) / device time per step
          (input staging + dedispersion + block statistics + boxcar/peaks + the 64-bit
          boxcar pass over tiles the 32-bit pass could not prove exact), inputs
          resident in HBM.
  e2e     the same metric through the searcher's host API: every step copies
          its pinned host input in and its candidates out; beams go back to
          back (sp_searcher_submit_host / sp_searcher_collect, two in flight,
          so each input copy overlaps the previous beam's search), with the
          one-beam-at-a-time sp_searcher_run_host figure beside it.
  roofline  dedispersion kernel alone: channel x DM x sample adds per launch
          over its CUDA-event time, against the integer-add issue rate
          (SMs x measured 32-bit add lanes per SM per clock x max SM clock).

`--impl reference` times the CPU oracle (test infrastructure) on a bounded
sample of the same workload on the host cores.

Multi-GPU (torchrun): every rank searches its own beam (replicas, weak
scaling, no collective on the data path); the timed region is bracketed by
barriers and the slowest rank's time is reported.

`--workload batched` measures the multi-beam step instead: 128 beams of
4096 channels with lengths U{16384..131072} and max DM from {500, 1000,
2000} (bandpass gains U(0.5, 1.5)), dedispersed in grouped launches (one
CTA per work item) with the autotuned kernel shape and searched on a second stream,
the whole step replayed as one CUDA graph; value = seconds of data searched
per second, next to the same work as per-beam launches (also a graph).

`--workload stream` measures the streaming server: 256 beams of 4096
channels arriving as 8.0 s gulps (6104 samples) overlapped by the DM-2000
sweep (5751 trials), device rings and slots admitted by an HBM budget,
continuous batching, each gulp's candidates sifted on the host and the kept
peaks scored by the classifier inside the stream.  The classifier is first
trained in the run by the library's own kernels (synthetic subband spectra,
then the kept peaks of beams with injected bursts and RFI).  value =
sustained real-time beams (gulps finished per second at saturation x 8.0 s),
next to the same stream without sifter and classifier and to per-gulp
launches on one stream with the plain sifter; the chain's recall on bursts
injected into streamed beams; the p50/p99 latency of real-time arrivals at
90 % of the sustained rate through the whole chain against the 8.0 s
deadline.

`--workload classifier` measures the candidate classifier: training steps
(features + forward + backward + Adam, batch 64) and inference (features +
forward, batch 256) on device-resident synthetic candidate spectra, with the
algorithmic tensor-core rate (convolution FLOPs of the step over its time)
against the measured bf16 GEMM peak.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "real-time beams per GB300; dedispersion G(chan·DM·samp)/s vs roofline"
MAX_SM_MHZ = 2070.0  # GB300 maximum SM clock
PROFILE_JSON = os.path.join(ROOT, "profiles", "dedisperse_config2_traffic.json")
DEDISP_SRC = os.path.join(ROOT, "paper_2606_27262_gb300", "csrc", "dedisperse.cu")


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--cpu-stride", type=int, default=64,
                   help="CPU baseline samples every n-th trial DM")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--n-out", type=int, default=None,
                   help="searched samples per beam (default: the full 131072); smaller values are for "
                        "profiler captures only")
    p.add_argument("--workload", choices=["single", "batched", "stream", "classifier"], default="single")
    p.add_argument("--shape", type=int, default=None,
                   help="single workload: dedispersion kernel shape (default: the library's default plan)")
    p.add_argument("--stream-beams", type=int, default=256, help="stream workload: beams")
    p.add_argument("--stream-periods", type=float, default=3.0,
                   help="stream workload: gulp periods of real-time arrivals for the latency figures")
    p.add_argument("--stream-train-beams", type=int, default=96,
                   help="stream workload: beams with bursts and RFI whose kept peaks train the classifier")
    p.add_argument("--stream-recall-beams", type=int, default=32,
                   help="stream workload: streamed beams carrying injected bursts for the chain's recall")
    p.add_argument("--stream-plan", choices=["dm2000", "dm500"], default="dm2000",
                   help="stream workload: the 5751-trial plan to DM 2000 or the 501-trial plan to DM 500")
    p.add_argument("--beams", type=int, default=128, help="batched workload: number of beams")
    p.add_argument("--dmt-budget-gb", type=float, default=24.0,
                   help="batched workload: DM-transform bytes per group arena (GB)")
    p.add_argument("--no-per-beam", action="store_true", help="batched workload: skip the comparisons")
    p.add_argument("--cls-infer-only", action="store_true",
                   help="classifier workload: skip the training phase (for profiling the inference step)")
    p.add_argument("--batch-mode", choices=["persistent", "grid"], default="grid",
                   help="batched workload: dedispersion launch style of the timed step (grid: one CTA per "
                        "work item; persistent: a resident grid draining a work queue)")
    return p.parse_args(argv)


# ------------------------------------------------------------ distributed --
def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def dist_init(world: int, backend: str):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x: float, world: int, device="cpu") -> float:
    """Maximum of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def beam_seed(base: int, rank: int) -> int:
    """Each rank searches a different synthetic beam."""
    return base + 1000 * rank


# ---------------------------------------------------------------- clocks --
class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = sorted({name for r in rows for name, v in zip(self.REASONS, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# -------------------------------------------------------------- workload --
def workload(n_out=None):
    import dataclasses

    import synth
    wl = synth.config2()
    if n_out is not None and n_out != wl.n_out:
        wl = dataclasses.replace(wl, n_out=int(n_out), name=wl.name.replace("131072", str(int(n_out))))
    return wl


def kernel_source_hash() -> str:
    return hashlib.sha256(open(DEDISP_SRC, "rb").read()).hexdigest()[:16]


def profiled_traffic(n_out: int):
    """DRAM bytes per launch of the dedispersion kernel from the committed ncu
    summary of the full single-beam workload, or None when the kernel source
    changed since the capture or another length is being measured."""
    try:
        prof = json.load(open(PROFILE_JSON))
    except (OSError, ValueError):
        return None
    if prof.get("kernel_source_sha256_16") != kernel_source_hash() or int(n_out) != int(prof.get("n_out", -1)):
        return None
    return float(prof["dram_bytes_per_launch_full_config"])


def profiled_instructions_per_add():
    """Lane instructions the dedispersion kernel issues per channel x DM x
    sample add (smsp__inst_executed x 32 / adds of one ncu capture, committed
    with the traffic summary), or None when the kernel source changed since."""
    try:
        prof = json.load(open(PROFILE_JSON))
    except (OSError, ValueError):
        return None
    if prof.get("kernel_source_sha256_16") != kernel_source_hash() or "lane_instructions_per_add" not in prof:
        return None
    return float(prof["lane_instructions_per_add"])


def issue_roofline(adds_tps: float, nsm: int):
    """The dedispersion kernel against the SMs' instruction-issue rate (four
    schedulers x 32 lanes per SM per clock at the maximum SM clock): lane
    instructions per add (from the committed ncu capture) x adds per second."""
    ipa = profiled_instructions_per_add()
    if ipa is None:
        return None
    peak = nsm * 128 * MAX_SM_MHZ * 1e6 / 1e12
    return {"lane_instructions_per_add": ipa, "achieved": adds_tps * ipa, "peak": peak,
            "unit": "T lane-instructions/s", "frac": adds_tps * ipa / peak,
            "peak_basis": f"{nsm} SMs x 4 schedulers x 32 lanes x {MAX_SM_MHZ:.0f} MHz"}


def cpu_oracle_sample(wl, plan_delays, x, stride: int):
    """Time the oracle on every `stride`-th trial DM (full length, all
    channels): dedispersion + best-width S/N.  Returns (seconds for the full
    workload extrapolated by trial count, sample description, threads)."""
    import numpy as np

    import oracle
    rows = np.arange(0, plan_delays.shape[0], stride)
    t = time.perf_counter()
    dmt = oracle.dedisperse(x, plan_delays[rows], wl.n_out)
    oracle.best(dmt, wl.widths, wl.norm_block)
    dt = time.perf_counter() - t
    full = dt * plan_delays.shape[0] / rows.size
    desc = (f"oracle dedispersion + boxcar S/N on every {stride}th trial DM ({rows.size} of "
            f"{plan_delays.shape[0]}) x {wl.n_out} samples x {wl.nchan} ch, {dt:.1f} s, "
            f"scaled by trial count")
    return full, desc, oracle.num_threads()


def config_dict(wl, plan_ndm, max_delay):
    return {
        "workload": wl.name,
        "nchan": wl.nchan, "n_out": wl.n_out, "n_in": wl.n_out + max_delay, "ndm": plan_ndm,
        "widths": [int(w) for w in wl.widths], "threshold": wl.threshold, "norm_block": wl.norm_block,
        "tsamp_s": wl.tsamp, "l2": "inputs larger than L2 (721 MB filterbank, 3.0 GB DM transform), no flush",
    }


# ------------------------------------------------------------------ ours --
def run_ours(args):
    import numpy as np
    import torch

    import paper_2606_27262_gb300 as sp
    import synth
    from paper_2606_27262_gb300 import build as spbuild

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    spbuild.build()
    wl = workload(args.n_out)
    plan = sp.Plan(wl.freqs, wl.tsamp, wl.dms) if args.shape is None else \
        sp.Plan(wl.freqs, wl.tsamp, wl.dms, shape=args.shape)
    n_in = wl.n_out + plan.max_delay
    x, _ = synth.make_workload_beam(wl, n_in, seed=beam_seed(wl.seed, rank))

    d_in = torch.from_numpy(x).to(dev)
    xt = sp.staged_buffer(wl.nchan, n_in, dev)
    dmt = torch.empty((plan.ndm, wl.n_out), dtype=torch.int32, device=dev)
    sw = torch.empty(sp.sps_workspace_bytes(plan.ndm, wl.n_out, len(wl.widths), wl.norm_block),
                     dtype=torch.uint8, device=dev)
    cap = 1 << 22
    cands = torch.empty((cap, 4), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        sp.stage_input(d_in, xt, stream)
        if ev is not None:
            ev[1].record(stream)
        sp.dedisperse_staged(plan, xt, n_in, dmt, stream)
        if ev is not None:
            ev[2].record(stream)
        sp.single_pulse_search(dmt, wl.widths, wl.threshold, wl.norm_block, sw, cands, cnt, stream)
        if ev is not None:
            ev[3].record(stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize(dev)
    lanes, nsm = sp.probe_iadd3_rate()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(dev)
    lc0 = sp.launch_count()
    t_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t_end.record(stream)
    launches = sp.launch_count() - lc0
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    elapsed = reduce_max(t_start.elapsed_time(t_end), world, dev)
    ms_step = elapsed / args.steps
    tr_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    dd_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    sps_ms = statistics.mean(e[2].elapsed_time(e[3]) for e in evs)
    ncand = int(cnt.item())
    beam_s = wl.n_out * wl.tsamp
    value = world * beam_s / (ms_step / 1e3)
    adds = float(wl.nchan) * plan.ndm * wl.n_out
    achieved = adds / (dd_ms / 1e3) / 1e12
    peak = nsm * lanes * MAX_SM_MHZ * 1e6 / 1e12

    e2e = None
    if not args.no_e2e:
        del xt
        s = sp.Searcher(plan, wl.n_out, wl.widths, wl.threshold, wl.norm_block, cap)
        h_in = torch.from_numpy(x).pin_memory()
        hc = np.empty((cap, 4), np.int32)
        s.run_host(h_in, hc)
        s.submit_host(h_in)  # first submit allocates the second slot
        s.collect(hc)
        # one beam at a time: copy in, search, results out, then the next
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            s.run_host(h_in, hc)
        serial_s = reduce_max(time.perf_counter() - t0, world, dev) / args.steps
        # beams back to back: each beam's input copy overlaps the search of
        # the beam before it; every step still copies its whole input in and
        # its candidates out
        barrier(world)
        t0 = time.perf_counter()
        n_found = 0
        s.submit_host(h_in)
        for k in range(args.steps):
            if k + 1 < args.steps:
                s.submit_host(h_in)
            n_found = s.collect(hc)
        e2e_s = reduce_max(time.perf_counter() - t0, world, dev) / args.steps
        barrier(world)
        e2e = {"value": world * beam_s / e2e_s, "unit": "beams", "ms_per_step": e2e_s * 1e3,
               "h2d_bytes_per_step": int(x.nbytes), "d2h_bytes_per_step": 8 + 16 * min(n_found, cap),
               "api": "sp_searcher_submit_host + sp_searcher_collect (two beams in flight)",
               "serial": {"value": world * beam_s / serial_s, "ms_per_step": serial_s * 1e3,
                          "api": "sp_searcher_run_host (one beam at a time)"}}
        s.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        full_s, desc, cores = cpu_oracle_sample(wl, plan.delays(), x, args.cpu_stride)
        cpu = {"value": beam_s / full_s, "unit": "beams", "cores": cores, "kind": "oracle", "sample": desc}

    line = {
        "metric": METRIC, "value": value, "unit": "beams", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded noise + injected dispersed bursts)",
        "config": config_dict(wl, plan.ndm, plan.max_delay) | {"parallelism": f"replicas x{world}"},
        "gchan_dm_samp_per_s": adds / (ms_step / 1e3) / 1e9,
        "stage_ms": {"stage_input": tr_ms, "dedisperse": dd_ms, "single_pulse_search": sps_ms},
        "candidates_per_beam": ncand,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tadd/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(wl.n_out),
                     "kernel": "dedisperse_kernel",
                     "kernel_shape": dict(zip(("dm_tile", "time_tile", "chan_chunk"), sp.shape_info(plan.shape)))
                     | {"shape": plan.shape, "dm_tiles": plan.ntiles},
                     "issue": issue_roofline(achieved, nsm),
                     "peak_basis": f"{nsm} SMs x {lanes:.1f} measured 32-bit add lanes/SM/clk x "
                                   f"{MAX_SM_MHZ:.0f} MHz"},
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clk, "gpu_launches": launches,
        # staging, dedispersion, block sums, block coefficients, streamed
        # boxcar/peaks, tile kernel over the listed tiles, 64-bit pass
        "kernels_per_step": launches / args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- batched --
def host_mem_available() -> int:
    """MemAvailable of /proc/meminfo in bytes (0 if unreadable)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except (OSError, ValueError, IndexError):
        pass
    return 0


def batched_e2e(args, batch, bw, data_s, stream, world, dev):
    """The batched step end to end through sp_batch_run_host: every beam
    copied from page-locked host memory, the grouped step, counts and
    candidates back to the host.  The host copies of the beams are made once
    (outside the timed region) from the device inputs, in one page-locked
    buffer (torch's pinned allocator rounds it up to a power of two)."""
    import numpy as np
    import torch
    sizes = [batch.input_tensor(b, bw.nchan).numel() for b in range(bw.nbeams)]
    total = int(sum(sizes))
    pinned = 1 << (total - 1).bit_length()
    avail = host_mem_available()
    if avail < 2 * pinned:
        return {"value": None, "unit": "beams",
                "unavailable": f"host memory: {avail / 1e9:.0f} GB available, {2 * pinned / 1e9:.0f} GB wanted "
                               f"to page-lock a copy of the {total / 1e9:.1f} GB of beams"}
    host = torch.empty(total, dtype=torch.uint8, pin_memory=True)
    views, off = [], 0
    for b, n in enumerate(sizes):
        v = host[off:off + n]
        v.copy_(batch.input_tensor(b, bw.nchan).reshape(-1))
        views.append(v)
        off += n
    cap_pb = 8192
    hc = np.zeros((bw.nbeams * cap_pb, 4), np.int32)
    counts = batch.run_host(views, hc, stream)  # warm-up
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        counts = batch.run_host(views, hc, stream)
    dt = reduce_max(time.perf_counter() - t0, world, dev) / args.steps
    barrier(world)
    del views, host
    return {"value": world * data_s / dt, "unit": "beams", "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": total,
            "d2h_bytes_per_step": int(8 * bw.nbeams + 16 * np.minimum(counts, cap_pb).sum()),
            "api": "sp_batch_run_host (grouped step, one CTA per work item; beams in page-locked host memory)"}


def run_batched(args):
    import numpy as np
    import torch

    import paper_2606_27262_gb300 as sp
    import synth
    from paper_2606_27262_gb300 import build as spbuild

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    spbuild.build()
    bw = synth.config3(nbeams=args.beams)
    stream = torch.cuda.Stream(device=dev)  # graph capture needs a stream other than the legacy default
    best, tune_ms = sp.autotune_dedisperse(bw.freqs, bw.tsamp, bw.plan_dms[-1], stream=stream)
    plans = [sp.Plan(bw.freqs, bw.tsamp, d, shape=best) for d in bw.plan_dms]
    cap = 1 << 19
    batch = sp.Batch(plans, bw.beam_plan, bw.n_out, bw.widths, bw.threshold, bw.norm_block, cap,
                     int(args.dmt_budget_gb * (1 << 30)))
    for b in range(bw.nbeams):
        synth.make_beam_torch(bw.beam_seed(b) + 7919 * rank, batch.input_tensor(b, bw.nchan), bw.freqs,
                              bw.bursts(b), widths=bw.widths, gains=bw.gains(b))
    torch.cuda.synchronize(dev)
    ndms = np.array([plans[p].ndm for p in bw.beam_plan], np.float64)
    adds = float(np.sum(ndms * bw.n_out.astype(np.float64))) * bw.nchan
    data_s = float(np.sum(bw.n_out)) * bw.tsamp

    # Dedispersion kernel time inside a grouped step (events around each
    # group's persistent launch on the launching stream), for the roofline.
    batch.run({"persistent": sp.SP_BATCH_GROUPED, "grid": sp.SP_BATCH_GROUPED_GRID}[args.batch_mode]
              | sp.SP_BATCH_TIMED, stream)
    torch.cuda.synchronize(dev)
    group_ms = batch.group_ms()
    lanes, nsm = sp.probe_iadd3_rate()

    def timed_graph(mode, steps, warmup):
        batch.capture(mode, stream)
        for _ in range(max(warmup, 0)):
            batch.launch(stream)
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        barrier(world)
        torch.cuda.synchronize(dev)
        lc0 = sp.launch_count()
        ev[0].record(stream)
        for k in range(steps):
            batch.launch(stream)
            ev[k + 1].record(stream)
        torch.cuda.synchronize(dev)
        timed_graph.launches = sp.launch_count() - lc0
        barrier(world)
        return reduce_max(ev[0].elapsed_time(ev[-1]), world, dev) / steps

    main_mode = {"persistent": sp.SP_BATCH_GROUPED, "grid": sp.SP_BATCH_GROUPED_GRID}[args.batch_mode]
    per_beam, other = None, None
    if not args.no_per_beam:
        pb_ms = timed_graph(sp.SP_BATCH_PER_BEAM, max(1, args.steps // 2), 1)
        per_beam = {"value": world * data_s / (pb_ms / 1e3), "unit": "beams", "ms_per_step": pb_ms,
                    "launches": "per beam: stage, dedisperse (grid kernel), statistics, boxcar; one stream; "
                                "captured as one CUDA graph"}
        alt = sp.SP_BATCH_GROUPED_GRID if main_mode == sp.SP_BATCH_GROUPED else sp.SP_BATCH_GROUPED
        alt_ms = timed_graph(alt, max(1, args.steps // 2), 1)
        other = {"mode": "grid" if alt == sp.SP_BATCH_GROUPED_GRID else "persistent",
                 "value": world * data_s / (alt_ms / 1e3), "ms_per_step": alt_ms}
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ms_step = timed_graph(main_mode, args.steps, args.warmup)
    launches = timed_graph.launches
    clk = clocks.stop()
    counts = [batch.count(b, stream) for b in range(bw.nbeams)]
    value = world * data_s / (ms_step / 1e3)
    dd_ms = float(np.sum(group_ms))
    achieved = adds / (dd_ms / 1e3) / 1e12
    peak = nsm * lanes * MAX_SM_MHZ * 1e6 / 1e12

    e2e = None if args.no_e2e else batched_e2e(args, batch, bw, data_s, stream, world, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t_cpu, work = 0.0, 0.0
        stride = 4 * args.cpu_stride
        for p in range(len(bw.plan_dms)):
            b = int(np.flatnonzero(bw.beam_plan == p)[0])
            x = batch.input_tensor(b, bw.nchan).cpu().numpy()
            rows = np.arange(0, bw.plan_dms[p].size, stride)
            t0 = time.perf_counter()
            dmt = oracle.dedisperse(x, oracle.delays(bw.freqs, bw.tsamp, bw.plan_dms[p][rows]), int(bw.n_out[b]))
            oracle.best(dmt, bw.widths, bw.norm_block)
            t_cpu += time.perf_counter() - t0
            work += float(rows.size) * int(bw.n_out[b]) * bw.nchan
        full_s = t_cpu * adds / work
        cpu = {"value": data_s / full_s, "unit": "beams", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"oracle dedispersion + boxcar S/N on every {stride}th trial DM of one beam per DM "
                         f"plan (full length), {t_cpu:.1f} s, scaled by channel x DM x sample count"}

    ngroups = batch.ngroups
    line = {
        "metric": METRIC, "value": value, "unit": "beams", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded noise drawn on the device, per-channel gains, injected dispersed bursts)",
        "config": {"workload": bw.name, "nbeams": bw.nbeams, "data_seconds": data_s,
                   "shape": dict(zip(("dm_tile", "time_tile", "chan_chunk"), sp.shape_info(best))),
                   "autotune_ms": [float(v) for v in tune_ms], "groups": ngroups,
                   "dmt_budget_bytes": int(args.dmt_budget_gb * (1 << 30)), "device_bytes": batch.device_bytes,
                   "graph": True, "widths": [int(w) for w in bw.widths], "threshold": bw.threshold,
                   "norm_block": bw.norm_block,
                   "l2": "inputs larger than L2 (0.1-0.7 GB per beam, 52 GB per batch), no flush",
                   "parallelism": f"replicas x{world}"},
        "gchan_dm_samp_per_s": adds / (ms_step / 1e3) / 1e9,
        "batch_mode": args.batch_mode, "other_batch_mode": other,
        "per_beam": per_beam,
        "speedup_vs_per_beam": (per_beam["ms_per_step"] / ms_step) if per_beam else None,
        "candidates": int(sum(counts)),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tadd/s", "frac": achieved / peak,
                     "traffic": None,
                     "kernel": "dedisperse_items_kernel" if args.batch_mode == "grid" else "dedisperse_batch_kernel",
                     "kernel_ms_per_step": dd_ms,
                     "peak_basis": f"{nsm} SMs x {lanes:.1f} measured 32-bit add lanes/SM/clk x "
                                   f"{MAX_SM_MHZ:.0f} MHz"},
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
        "gpu_launches": launches,  # per beam: staging, statistics, boxcar, 64-bit pass; per group: dedispersion
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------- stream --
def train_pipeline_classifier(plan, freqs, widths, dev, seed: int, nbeams: int):
    """The classifier trained by the library's kernels: 2000 steps of 64
    synthetic subband spectra (60 % bursts), then 1500 steps of 64 kept peaks
    (half on bursts) of ``nbeams`` 16384-sample beams with 4 injected bursts
    (DM 50-1950, FWHM 1-64 samples, S/N 6-50) and 3-6 RFI events each, found
    by this plan's search and the sifter.  Returns (classifier, info)."""
    import numpy as np
    import torch

    import paper_2606_27262_gb300 as sp
    from paper_2606_27262_gb300 import learning
    from synth import classifier as scls
    from synth import rfi
    n_out = 16384
    h = learning.Harvester(plan, n_out, widths, 6.0, 8192, device=dev)
    beam = torch.empty((n_out + plan.max_delay, plan.nchan), dtype=torch.uint8, device=dev)

    def make(sd, out):
        return [learning.Truth(b.t0, b.dm, b.fwhm, b.snr) for b in rfi.pipeline_beam(sd, out, freqs, n_out, widths)]
    hv = learning.harvest_beams(h, make, range(seed, seed + nbeams), beam)
    del h, beam
    clf = sp.Classifier(max_batch=64, seed=seed)
    rng = np.random.default_rng(seed)

    def sample(n):
        sub, labels, _ = scls.classifier_batch(rng, n, freqs, device=dev, t_in=512, p_burst=0.6)
        return sub, labels
    pre = learning.train(clf, learning.subband_batches(sample, freqs, 64, device=dev), 2000)
    post = learning.train(clf, learning.pool_batches(hv.ft, hv.dm_img, hv.labels, rng, 64), 1500, lr=1e-3)
    info = {"synthetic_steps": 2000, "pipeline_steps": 1500, "batch": 64, "pipeline_beams": nbeams,
            "pipeline_kept_peaks": int(hv.labels.size), "pipeline_burst_peaks": int(hv.labels.sum()),
            "loss_first": pre[0], "loss_last": post[-1]}
    return clf, info


def stream_recall(plan, clf, freqs, widths, gulp: int, cap: int, kept_cap: int, t_in: int, dev, seed: int,
                  nbeams: int):
    """Streams ``nbeams`` beams whose first max_delay samples (the history
    that the first searched windows cover) hold one dispersed burst per
    gulp-long window (S/N 8-30, FWHM 1-16 samples, DM 50-1000 with the sweep
    inside the history) and 4 RFI events, through search, sifter and the
    classifier; the pushed gulps are noise.  A burst counts as kept when the
    sifter keeps a peak on it and as accepted when the classifier accepts one
    of those peaks."""
    import numpy as np
    import torch

    import paper_2606_27262_gb300 as sp
    import synth
    from paper_2606_27262_gb300 import learning
    from synth import rfi
    nchan, D = plan.nchan, plan.max_delay
    rounds = D // gulp
    per_dm = float(synth.fractional_delay(freqs, 1.0)[-1])
    # RFI makes 10^4-10^5 candidates per gulp: a capacity that holds all of
    # them, so that the sifter sees every candidate of every window
    cap = 1 << 20
    s = sp.Stream(plan, nbeams, gulp, widths, 6.0, 8192, cap, 24 * (1 << 30) + nbeams * (gulp + D) * nchan,
                  max_batch=16)
    s.attach(clf, t_in=t_in, kept_cap=kept_cap)
    hist_d = torch.empty((D, nchan), dtype=torch.uint8, device=dev)
    truths = []
    for b in range(nbeams):
        rng = np.random.default_rng((seed, b))
        bursts = []
        for k in range(rounds):
            t0 = k * gulp + int(rng.integers(64, gulp - 64))
            fwhm = float(rng.uniform(1.0, 16.0))
            dm_hi = min(1000.0, (D - t0 - 8 * fwhm - 64) / per_dm)
            if dm_hi < 60.0:
                break
            bursts.append(synth.Burst(t0, float(rng.uniform(50.0, dm_hi)), fwhm, float(rng.uniform(8.0, 30.0))))
        events = rfi.draw_rfi(rng, 4, D, nchan)
        synth.make_beam_torch(seed * 1000 + b, hist_d, freqs, bursts, widths=widths,
                              extra=rfi.rfi_signal(events, D, nchan))
        s.history(b, np.ascontiguousarray(hist_d.cpu().numpy()))
        truths.append(bursts)
    noise = [torch.from_numpy(synth.make_beam((seed, 50 + i), nchan, gulp, freqs)).pin_memory() for i in range(4)]
    for k in range(rounds):
        for b in range(nbeams):
            s.push(b, noise[(b + k) % len(noise)])
    res = s.drain(with_cands=False, sifted=True)
    s.close()
    kept_b = acc_b = injected = fp_sifter = fp_clf = overflow = cand_overflow = n_cands = 0
    for info, _, kept, prob in res:
        k = int(info.seq)
        n_cands += int(info.count)
        cand_overflow += int(info.count) > cap
        win = [learning.Truth(bb.t0 - k * gulp, bb.dm, bb.fwhm, bb.snr) for bb in truths[int(info.beam)]
               if k * gulp <= bb.t0 < (k + 1) * gulp]
        which = learning.match_peaks(kept, plan.dms, widths, win)
        overflow += int(info.kept) > kept_cap
        for i in range(len(win)):
            injected += 1
            on = which == i
            if on.any():
                kept_b += 1
                acc_b += bool((prob[on] >= 0.5).any())
        fp_sifter += int((which < 0).sum())
        fp_clf += int(((which < 0) & (prob >= 0.5)).sum())
    return {"beams": nbeams, "gulps": len(res), "bursts_injected": injected, "bursts_kept_by_sifter": kept_b,
            "bursts_accepted": acc_b, "recall_vs_sifter": acc_b / max(kept_b, 1),
            "recall_vs_injected": acc_b / max(injected, 1), "snr_range": [8.0, 30.0],
            "non_burst_peaks_sifter": fp_sifter, "non_burst_peaks_accepted": fp_clf,
            "candidates": n_cands, "gulps_over_candidate_cap": cand_overflow, "gulps_over_kept_cap": overflow}


def run_stream(args):
    import numpy as np
    import torch

    import paper_2606_27262_gb300 as sp
    import synth
    from paper_2606_27262_gb300 import build as spbuild

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist_init(world, "nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    spbuild.build()
    nchan, gulp, nbeams = 4096, 6104, args.stream_beams
    freqs = synth.band_freqs(nchan)
    dms = synth.dm_plan_config2() if args.stream_plan == "dm2000" else synth.dm_plan_config1()
    widths = synth.widths_pow2(256)
    plan = sp.Plan(freqs, synth.TSAMP, dms)
    period = gulp * synth.TSAMP
    cap = 4096
    # Host data: one history block and a pool of distinct gulps (pinned),
    # gulp k of beam b = pool[(3 b + k) % len(pool)].  Each pool gulp holds a
    # burst whose whole sweep fits inside it (DM <= 200: under 4600 samples
    # over the band), so that reused gulps stay physically consistent.
    rng_seed = 1005 + 7919 * rank
    sweep = int(np.ceil(synth.fractional_delay(freqs, 200.0)[-1]))
    pool = []
    for i in range(8):
        bursts = synth.draw_bursts(np.random.default_rng((rng_seed, i, 1)), 1, gulp - sweep, 20.0, 200.0,
                                   1.0, 16.0, 8.0, 30.0)
        x = synth.make_beam((rng_seed, i), nchan, gulp, freqs, bursts, widths=widths)
        pool.append(torch.from_numpy(x).pin_memory())
    # The shared history (the first max_delay samples, which the first
    # searched windows cover) holds one burst per gulp-long segment whose
    # sweep fits inside it (DM <= 1000, and lower late in the history), so
    # that every gulp searched in a short run has a burst for the sifter
    # and the classifier.
    hrng = np.random.default_rng((rng_seed, 98))
    per_dm = float(synth.fractional_delay(freqs, 1.0)[-1])
    hb = []
    for j in range(plan.max_delay // gulp):
        t0 = j * gulp + int(hrng.integers(64, gulp - 128))
        dm_hi = min(1000.0, (plan.max_delay - t0 - 256) / per_dm)
        if dm_hi < 60.0:
            break
        hb.append(synth.Burst(t0, float(hrng.uniform(50.0, dm_hi)), float(hrng.uniform(2.0, 16.0)),
                              float(hrng.uniform(15.0, 30.0))))
    hist = torch.from_numpy(synth.make_beam((rng_seed, 99), nchan, plan.max_delay, freqs, hb,
                                            widths=widths)).pin_memory()
    budget = int(args.dmt_budget_gb * (1 << 30)) + nbeams * (gulp + plan.max_delay) * nchan
    adds_per_gulp = float(nchan) * plan.ndm * gulp

    # The classifier of the full chain, trained here by the library's own
    # kernels: synthetic subband spectra first, then the kept peaks of beams
    # with injected bursts and RFI searched by this plan.
    t_in, kept_cap = 512, 64
    t_train = time.perf_counter()
    clf, train_info = train_pipeline_classifier(plan, freqs, widths, dev, 3005 + 101 * rank,
                                                args.stream_train_beams)
    train_info["seconds"] = time.perf_counter() - t_train

    def make_stream(flags, max_batch, stage):
        s = sp.Stream(plan, nbeams, gulp, widths, 6.0, 8192, cap, budget, max_batch=max_batch, flags=flags)
        if stage is not None:
            s.attach(clf if stage == "classify" else None, t_in=t_in, kept_cap=kept_cap)
        for b in range(nbeams):
            s.history(b, hist)
        return s

    def saturated(flags, max_batch, stage, rounds=2):
        s = make_stream(flags, max_batch, stage)
        k = 0
        tally = [0, 0, 0]  # candidates, kept, accepted

        def poll(wait=False):
            res = (s.drain(with_cands=False, sifted=True) if wait else s.poll_sifted()) if stage is not None \
                else (s.drain(with_cands=False) if wait else s.poll(with_cands=False))
            for r in res:
                tally[0] += int(r[0].count)
                tally[1] += int(r[0].kept)
                tally[2] += int(r[0].accepted)

        def one_round():
            nonlocal k
            for b in range(nbeams):
                s.push(b, pool[(3 * b + k) % len(pool)])
                poll()
            k += 1
        one_round()
        poll(wait=True)  # warm-up round
        tally[:] = [0, 0, 0]
        barrier(world)
        lc0 = sp.launch_count()
        t0 = time.perf_counter()
        for _ in range(rounds):
            one_round()
        poll(wait=True)
        dt = reduce_max(time.perf_counter() - t0, world, dev)
        info = {"slots": s.slots, "device_bytes": s.device_bytes, "candidates": tally[0], "kept": tally[1],
                "accepted": tally[2], "launches": sp.launch_count() - lc0}
        s.close()
        return rounds * nbeams / dt, dt, info

    rate_b, dt_b, info_b = saturated(0, 16, "classify")
    rate_s, dt_s, info_s = saturated(0, 16, None)
    rate_p, dt_p, info_p = saturated(sp.SP_STREAM_PER_GULP | sp.SP_STREAM_ONE_STREAM, 1, "sift")
    rate_q, dt_q, info_q = saturated(sp.SP_STREAM_PER_GULP | sp.SP_STREAM_ONE_STREAM, 1, None)

    # Recall of the whole chain (search, sifter, classifier) on bursts
    # injected into the streamed beams themselves.
    # (every kept peak of a gulp scored: RFI leaves up to a few hundred)
    recall = stream_recall(plan, clf, freqs, widths, gulp, cap, sp.SP_CNN_MAX_BATCH, t_in, dev, 2007 + 31 * rank,
                           args.stream_recall_beams)

    # Real-time arrivals near saturation: as many beams as 90 % of the
    # sustained rate above serves (fewer if their rings do not fit the
    # device), every beam pushing a gulp each period, beams staggered evenly
    # over the period; the full chain attached.
    ring_bytes = (gulp + plan.max_delay) * nchan
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info(dev)
    fit = int((free - 40 * (1 << 30)) // ring_bytes)
    nb_rt = max(1, min(int(0.9 * rate_b * period), fit))
    s = sp.Stream(plan, nb_rt, gulp, widths, 6.0, 8192, cap,
                  int(args.dmt_budget_gb * (1 << 30)) + nb_rt * ring_bytes, max_batch=16)
    s.attach(clf, t_in=t_in, kept_cap=kept_cap)
    for b in range(nb_rt):
        s.history(b, hist)
    lat, lat_search, cand_total, kept_total = [], [], 0, 0
    nper = max(1, int(round(args.stream_periods)))
    arrivals = sorted((k * period + b * period / nb_rt, b, k) for k in range(nper) for b in range(nb_rt))
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    t_start = sp.stream_now() + 0.05
    def record(res):
        nonlocal cand_total, kept_total
        for r, _, _, _ in res:
            lat.append(r.t_done - r.t_push)
            lat_search.append(r.t_search - r.t_push)
            cand_total += int(r.count)
            kept_total += int(r.kept)
    for ta, b, k in arrivals:
        while sp.stream_now() < t_start + ta:
            record(s.poll_sifted())
            time.sleep(0.0005)
        s.push(b, pool[(3 * b + k) % len(pool)])
    record(s.drain(with_cands=False, sifted=True))
    clk = clocks.stop()
    s.close()
    clf.close()
    lat, lat_search = np.array(lat), np.array(lat_search)
    lines = {
        "metric": METRIC, "value": world * rate_b * period, "unit": "beams", "n_gpus": world,
        "steps": 2 * nbeams, "warmup": nbeams, "ms_per_step": 1e3 / rate_b, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (pool of 8 seeded noise gulps with injected bursts, pinned host memory)",
        "config": {"workload": f"streaming: {nbeams} beams x {nchan}ch, {gulp}-sample gulps ({period:.2f} s) "
                               f"overlapped by the DM-{int(dms[-1])} sweep ({plan.ndm} trials, "
                               f"{plan.max_delay} samples), widths 1-256",
                   "gulp": gulp, "n_in": gulp + plan.max_delay, "ndm": plan.ndm, "max_batch": 16,
                   "hbm_budget_bytes": budget, "slots": info_b["slots"], "device_bytes": info_b["device_bytes"],
                   "step": "one gulp through search, sifter and classifier (value = gulps finished per second "
                           "at saturation x gulp duration)",
                   "chain": f"batched dedispersion (one CTA per work item while a classifier is attached), "
                            f"search on a high-priority stream, host DBSCAN sifter (Sec. 3.2.1 defaults), "
                            f"classifier on the kept peaks of each finished batch on a high-priority stream "
                            f"(t_in {t_in}, up to {kept_cap} per gulp, weights trained in this run)",
                   "l2": "rings and windows larger than L2, no flush", "parallelism": f"replicas x{world}"},
        "sifted": {"candidates": info_b["candidates"], "kept": info_b["kept"], "classified": info_b["kept"],
                   "gulps": 2 * nbeams},
        "search_only": {"value": world * rate_s * period, "unit": "beams", "ms_per_gulp": 1e3 / rate_s,
                        "candidates": info_s["candidates"], "launches": "batched, no sifter or classifier attached"},
        "per_gulp": {"value": world * rate_p * period, "unit": "beams", "ms_per_gulp": 1e3 / rate_p,
                     "candidates": info_p["candidates"], "kept": info_p["kept"],
                     "launches": "each gulp: copy, stage, dedisperse (grid kernel), search, plain sifter; "
                                 "one stream"},
        "per_gulp_search_only": {"value": world * rate_q * period, "unit": "beams", "ms_per_gulp": 1e3 / rate_q,
                                 "launches": "as per_gulp, without the sifter"},
        "speedup_vs_per_gulp": rate_b / rate_p,
        "classifier_training": train_info,
        "recall": recall,
        "latency": {"beams": nb_rt, "load_vs_sustained": nb_rt / (rate_b * period), "periods": nper,
                    "gulps": int(lat.size), "deadline_s": period,
                    "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "max_s": float(lat.max()), "met_deadline": bool(lat.max() < period),
                    "search_p50_s": float(np.percentile(lat_search, 50)),
                    "search_p99_s": float(np.percentile(lat_search, 99)),
                    "candidates": cand_total, "kept": kept_total},
        "roofline": {"bound": "alu", "achieved": adds_per_gulp * rate_b / 1e12, "unit": "Tadd/s",
                     "kernel": "whole streaming chain at saturation (copies, staging, dedispersion, search, sifter, "
                               "classifier)",
                     "peak": None, "frac": None, "traffic": None},
        "e2e": {"value": world * rate_b * period, "unit": "beams", "h2d_bytes_per_step": gulp * nchan,
                "d2h_bytes_per_step": 8 + 16 * cap + 4 * kept_cap,
                "api": "sp_stream_push / sp_stream_poll_sifted from pinned host gulps"},
        "cpu_baseline": None, "clocks": clk,
        "gpu_launches": info_b["launches"],
    }
    lanes, nsm = sp.probe_iadd3_rate()
    peak = nsm * lanes * MAX_SM_MHZ * 1e6 / 1e12
    lines["roofline"]["peak"] = peak
    lines["roofline"]["frac"] = lines["roofline"]["achieved"] / peak
    if rank == 0:
        print(json.dumps(lines), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------- classifier --
CNN_LAYERS = [(1, 16, 256), (16, 32, 128), (32, 64, 64), (64, 128, 32), (128, 256, 16)]  # cin, cout, h_in


def cnn_flops_per_example(train: bool) -> float:
    """Algorithmic multiply-add FLOPs of the two 5-layer branches (3x3
    convolutions, stride 2): forward, plus weight and input gradients."""
    fwd = dx = 0.0
    for i, (ci, co, h) in enumerate(CNN_LAYERS):
        f = 2.0 * (h // 2) ** 2 * co * 9 * ci
        fwd += f
        if i > 0:
            dx += f
    per_branch = fwd + (fwd + dx if train else 0.0)
    return 2 * per_branch


def run_classifier(args):
    import numpy as np
    import torch

    import paper_2606_27262_gb300 as sp
    import synth
    from paper_2606_27262_gb300 import build as spbuild
    from synth import classifier as scls

    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    spbuild.build()
    freqs = synth.band_freqs(4096)
    shift = torch.from_numpy(sp.dmt_shifts(freqs, 256, 128)).to(dev)
    rng = np.random.default_rng(1004 + rank)
    bt, bi = 64, 256
    pool = [scls.classifier_batch(rng, bt, freqs, device=dev, p_burst=0.6) for _ in range(8)]
    clf = sp.Classifier(max_batch=bi, seed=11)
    ft = torch.empty((bi, 256, 256), dtype=torch.bfloat16, device=dev)
    dmt = torch.empty_like(ft)
    work = torch.empty(int(sp.library().sp_cnn_features_workspace_bytes(bi)), dtype=torch.uint8, device=dev)
    labels = [torch.from_numpy(lab).to(dev) for _, lab, _ in pool]
    stream = torch.cuda.current_stream(dev)

    def train_step(k):
        sub = pool[k % len(pool)][0]
        sp.cnn_features(sub, shift, ft[:bt], dmt[:bt], work)
        clf.train_step(ft[:bt], dmt[:bt], labels[k % len(pool)], 1e-3)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    steps, train_ms = 0, None
    if not args.cls_infer_only:
        for k in range(max(args.warmup, 3)):
            train_step(k)
        torch.cuda.synchronize(dev)
        steps = max(args.steps, 1) * 40
        clocks.start()
        e0.record(stream)
        for k in range(steps):
            train_step(k)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        train_ms = e0.elapsed_time(e1) / steps
    else:
        clocks.start()
    # inference: features + forward on batches of 256 candidates
    big = scls.classifier_batch(rng, bi, freqs, device=dev)[0]
    prob = torch.empty(bi, device=dev)
    for _ in range(3):
        sp.cnn_features(big, shift, ft, dmt, work)
        clf.forward(ft, dmt, prob)
    torch.cuda.synchronize(dev)
    reps = max(args.steps, 1) * 10
    lc0 = sp.launch_count()
    e0.record(stream)
    for _ in range(reps):
        sp.cnn_features(big, shift, ft, dmt, work)
        clf.forward(ft, dmt, prob)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    launches = sp.launch_count() - lc0
    infer_ms = e0.elapsed_time(e1) / reps
    clk = clocks.stop()
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops", 1900.0)
    tr_tflops = cnn_flops_per_example(True) * bt / (train_ms / 1e3) / 1e12 if train_ms else None
    in_tflops = cnn_flops_per_example(False) * bi / (infer_ms / 1e3) / 1e12
    line = {
        "metric": "classifier candidates per second (inference) and training examples per second",
        "value": bi / (infer_ms / 1e3), "unit": "candidates/s", "n_gpus": 1, "steps": reps, "warmup": 3,
        "ms_per_step": infer_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic candidate spectra (bursts, narrowband and broadband RFI, tones, noise)",
        "config": {"workload": "classifier: two 5-layer 3x3 stride-2 CNNs on 256x256 frequency-time and DM-time "
                               "images, 0.79 M parameters", "batch_infer": bi, "batch_train": bt,
                   "params": int(sp.library().sp_cnn_num_params())},
        "training": {"examples_per_s": bt / (train_ms / 1e3), "ms_per_step": train_ms, "steps": steps,
                     "tflops": tr_tflops} if train_ms else None,
        "roofline": {"bound": "tensor", "achieved": in_tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": in_tflops / peak, "traffic": None,
                     "kernel": "inference step (features, first layer, im2col + tcgen05 GEMMs, pooling/head), "
                               "algorithmic convolution FLOPs over the step time",
                     "peak_basis": "measured bf16 GEMM burst (MEASURED_PEAKS.json)"},
        "e2e": None, "cpu_baseline": None, "clocks": clk, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- reference --
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    import synth
    wl = workload(args.n_out)
    delays = oracle.delays(wl.freqs, wl.tsamp, wl.dms)
    n_in = wl.n_out + int(delays.max())
    x, _ = synth.make_workload_beam(wl, n_in)
    beam_s = wl.n_out * wl.tsamp
    for _ in range(max(args.warmup, 0)):
        cpu_oracle_sample(wl, delays, x, args.cpu_stride * 4)
    # A step is the bounded sample itself (every stride-th trial DM of the
    # beam, full length): ms_per_step is the time it took, and the value
    # scales the sampled share of the beam's data to real-time beams.
    times, desc, cores = [], "", oracle.num_threads()
    ndm = delays.shape[0]
    frac = np.arange(0, ndm, args.cpu_stride).size / ndm
    for _ in range(args.steps):
        full_s, desc, cores = cpu_oracle_sample(wl, delays, x, args.cpu_stride)
        times.append(full_s * frac)
    sample_s = statistics.mean(times)
    value = beam_s * frac / sample_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "beams", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sample_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": config_dict(wl, ndm, int(delays.max())) | {"parallelism": "host cores"},
        "step": f"one sampled step: every {args.cpu_stride}th trial DM ({round(frac * ndm)} of {ndm}) of one beam "
                f"at full length; value = the sampled share of the beam's {beam_s:.1f} s of data per second",
        "extrapolated": True, "trial_fraction": frac, "full_beam_s_extrapolated": sample_s / frac,
        "cpu_baseline": {"value": value, "unit": "beams", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "beams", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "stream":
        run_stream(args)
    elif args.workload == "classifier":
        run_classifier(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
