"""Helpers for the GPU tests: device buffers through torch, calls through the
C ABI (paper_2606_27262_gb300), and comparisons against the oracle."""
from __future__ import annotations

import math

import numpy as np
import torch

import paper_2606_27262_gb300 as sp

# S/N agreement bar between the float32 GPU path and the float64 oracle.
SNR_RTOL = 1e-4


def dev_dedisperse(plan: sp.Plan, data: np.ndarray) -> torch.Tensor:
    d_in = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    n_out = data.shape[0] - plan.max_delay
    out = torch.empty((plan.ndm, n_out), dtype=torch.int32, device="cuda")
    work = torch.empty(sp.dedisperse_workspace_bytes(plan, data.shape[0]), dtype=torch.uint8, device="cuda")
    sp.dedisperse(plan, d_in, out, work)
    torch.cuda.synchronize()
    return out


def sps_work(ndm, n_out, nw, norm_block):
    return torch.empty(sp.sps_workspace_bytes(ndm, n_out, nw, norm_block), dtype=torch.uint8, device="cuda")


def dev_best_map(dmt: torch.Tensor, widths, norm_block: int):
    ndm, n_out = dmt.shape
    best = torch.empty((ndm, n_out), dtype=torch.float32, device="cuda")
    wb = torch.empty((ndm, n_out), dtype=torch.int8, device="cuda")
    sp.best_snr_map(dmt, widths, norm_block, sps_work(ndm, n_out, len(widths), norm_block), best, wb)
    torch.cuda.synchronize()
    return best.cpu().numpy(), wb.cpu().numpy().astype(np.int32)


def dev_candidates(dmt: torch.Tensor, widths, thr: float, norm_block: int, cap: int = 1 << 20):
    ndm, n_out = dmt.shape
    cands = torch.zeros((cap, 4), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    sp.single_pulse_search(dmt, widths, thr, norm_block, sps_work(ndm, n_out, len(widths), norm_block), cands,
                           count)
    torch.cuda.synchronize()
    n = int(count.item())
    return sp.cands_to_numpy(cands.cpu().numpy(), n), n


def check_best_map(gb, gk, ob, ok, osnr=None):
    """GPU best map (float32) vs oracle (float64): same -inf pattern, finite
    values within SNR_RTOL (absolute floor 1e-5 for values near 0), and the
    GPU's width is a maximiser of the oracle's S/N up to that tolerance."""
    ninf_g, ninf_o = np.isneginf(gb), np.isneginf(ob)
    assert np.array_equal(ninf_g, ninf_o)
    fin = ~ninf_o
    err = np.abs(gb[fin].astype(np.float64) - ob[fin])
    tol = SNR_RTOL * np.maximum(np.abs(ob[fin]), 0.1)
    bad = err > tol
    assert not bad.any(), f"{bad.sum()} S/N values off; worst {err.max()}"
    same = gk[fin] == ok[fin]
    if osnr is not None and not same.all():
        # A different width is fine only where the two widths tie within tolerance.
        idx = np.argwhere(fin & (gk != ok))
        for d, t in idx:
            alt = osnr[d, gk[d, t], t]
            assert alt >= ob[d, t] - SNR_RTOL * max(abs(ob[d, t]), 0.1), (d, t, alt, ob[d, t])
    else:
        assert same.all(), f"{(~same).sum()} width indices differ"


def check_candidates(g, o, ob, thr: float, radius: int = 1):
    """Candidate sets equal except where a decision sits within SNR_RTOL of
    a threshold or of a neighbour's value in the (2 radius + 1)^2 peak
    window (G8: near-ties are don't-care)."""
    gs = {(int(a), int(b)) for a, b in zip(g["dm_idx"], g["t"])}
    os_ = {(int(a), int(b)) for a, b in zip(o["dm_idx"], o["t"])}
    ndm, n_out = ob.shape

    def near_tie(d, t):
        v = ob[d, t]
        if abs(v - thr) <= SNR_RTOL * max(abs(thr), 1):
            return True
        for dd in range(-radius, radius + 1):
            for dt in range(-radius, radius + 1):
                e, u = d + dd, t + dt
                if (dd or dt) and 0 <= e < ndm and 0 <= u < n_out and math.isfinite(ob[e, u]):
                    if abs(ob[e, u] - v) <= SNR_RTOL * max(abs(v), 1):
                        return True
        return False

    diff = [p for p in gs ^ os_ if not near_tie(*p)]
    assert not diff, f"{len(diff)} candidates differ, e.g. {diff[:5]}"
    common = gs & os_
    gm = {(int(a), int(b)): (float(s), int(k)) for a, b, s, k in zip(g["dm_idx"], g["t"], g["snr"], g["width_idx"])}
    om = {(int(a), int(b)): (float(s), int(k)) for a, b, s, k in zip(o["dm_idx"], o["t"], o["snr"], o["width_idx"])}
    for p in common:
        assert abs(gm[p][0] - om[p][0]) <= SNR_RTOL * max(abs(om[p][0]), 0.1), (p, gm[p], om[p])
    return len(common)
