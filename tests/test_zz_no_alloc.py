"""The allocation-free single-pulse search against the workspace version.

sp_single_pulse_search_noalloc serves callers that cannot allocate device
memory while searching (a real-time loop whose memory budget was fixed at
start-up, a host whose device memory belongs to its own pool allocator, a
plug-in barred from cudaMalloc): its block statistics live in a 16 MiB
library-owned device array instead of a caller workspace.  This file is
collected last so that a run stopping at its first failure has run every
other test before it; it also passes on its own in a fresh process.

Two calls in a row on different inputs must each match the workspace entry
point and the CPU oracle (candidate sets equal up to near-ties, S/N within
1e-4), showing that the shared array's leftover contents from the first call
do not leak into the second.  The rejection of requests beyond the array's
size is a host-side check and is tested without a GPU in test_capi_host.py."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2606_27262_gb300 as sp
from paper_2606_27262_gb300 import build as spbuild
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    spbuild.build()
    assert torch.cuda.is_available()


def _noalloc_via_cabi(dmt, widths, thr, norm_block, cap=1 << 18):
    lib = sp.library()
    w = np.ascontiguousarray(widths, dtype=np.int32)
    cands = torch.zeros((cap, 4), dtype=torch.int32, device="cuda")
    count = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.sp_single_pulse_search_noalloc(dmt.data_ptr(), dmt.shape[0], dmt.shape[1], w.ctypes.data, w.size,
                                            ctypes.c_float(thr), norm_block, cands.data_ptr(), cap,
                                            count.data_ptr(), stream)
    assert rc == sp.SP_OK, lib.sp_strerror(rc)
    torch.cuda.synchronize()
    n = int(count.item())
    return sp.cands_to_numpy(cands.cpu().numpy(), n), n


def test_noalloc_matches_workspace_entry_point_twice():
    rng = np.random.default_rng(2024)
    widths = [1, 2, 4, 8, 16, 32]
    cases = [
        (np.rint(rng.normal(5.2e5, 1024.0, size=(300, 9000))).astype(np.int32), 4.0, 2048),
        (np.rint(rng.normal(1.0e5, 300.0, size=(170, 5000))).astype(np.int32), 3.5, 0),
    ]
    cases[0][0][150, 4000:4010] += 20000
    for dmt_np, thr, L in cases:  # two calls in a row, different inputs and blocks
        dmt = torch.from_numpy(dmt_np).cuda()
        got, gn = _noalloc_via_cabi(dmt, widths, thr, L)
        want, wn = gu.dev_candidates(dmt, widths, thr, L, cap=1 << 18)
        assert gn == got.size and wn == want.size and gn > 0
        ob = gu.dev_best_map(dmt, widths, L)[0].astype(np.float64)
        gu.check_candidates(got, want, ob, thr)
        # and directly against the oracle's search of the same rows
        orb, ork = oracle.best(dmt_np, widths, L)
        oc, on = oracle.peaks(orb, ork, thr, cap=1 << 18)
        assert on == oc.size
        gu.check_candidates(got, oc, orb, thr)

