"""CPU-only checks of the C ABI: the library builds, loads and exports every
function include/spotlight.h declares; host-side argument checking; the
host delay table equals the oracle's bit for bit (Eq. 1)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2606_27262_gb300 as sp
import synth
from paper_2606_27262_gb300 import build as spbuild

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")


@pytest.fixture(scope="module")
def lib():
    spbuild.build()
    return sp.library()


def declared_functions():
    text = "".join(open(os.path.join(INCLUDE, h)).read() for h in sorted(os.listdir(INCLUDE)) if h.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sp_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(sp.SIGNATURES), set(names) ^ set(sp.SIGNATURES)


def test_strerror(lib):
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8, -99):
        assert isinstance(lib.sp_strerror(code), bytes)
    assert lib.sp_strerror(sp.SP_ETIMEOUT).startswith(b"a bounded wait")
    assert lib.sp_strerror(-2).startswith(b"inconsistent")


def test_workspace_sizes(lib):
    # m0 per (row, block); coefficients and pre-filter constants per (row, block, width); two counters;
    # the tile lists of the streamed search and of the 64-bit pass (32 x 36 tiles each); 24-byte sums
    # per (row, block)
    assert lib.sp_sps_workspace_bytes(501, 8192, 6, 8192) == 2048 + 24064 + 12032 + 256 + 2 * 9216 + 12032
    assert lib.sp_sps_workspace_bytes(0, 10, 1, 0) == -1
    # classifier features: both raw fp32 images per candidate and 8 blocks x 4 fp32 sums per candidate
    assert lib.sp_cnn_features_workspace_bytes(3) == 2 * 786432 + 512
    assert lib.sp_cnn_features_workspace_bytes(0) == -1


def test_argument_checks_need_no_gpu(lib):
    f = synth.band_freqs(8)
    d = np.array([0.0, 10.0])
    h = ctypes.c_void_p()
    bad_f = f[::-1].copy()  # increasing: the band must be flipped highest-first
    assert lib.sp_plan_create(bad_f.ctypes.data, 8, 1e-3, d.ctypes.data, 2, ctypes.byref(h)) == sp.SP_EINVAL
    neg = np.array([-1.0])
    assert lib.sp_plan_create(f.ctypes.data, 8, 1e-3, neg.ctypes.data, 1, ctypes.byref(h)) == sp.SP_EINVAL
    assert lib.sp_plan_create(f.ctypes.data, 8, 0.0, d.ctypes.data, 2, ctypes.byref(h)) == sp.SP_EINVAL
    w = np.array([1, 2, 2], np.int32)  # not strictly increasing
    assert lib.sp_single_pulse_search(1, 4, 100, w.ctypes.data, 3, 6.0, 0, 256, 1 << 20, 256, 10, 256, 0) \
        == sp.SP_EINVAL
    wbig = np.array([1, 2048], np.int32)
    assert lib.sp_best_snr_map(1, 4, 100, wbig.ctypes.data, 2, 0, 256, 1 << 20, 256, 256, 0) == sp.SP_ELIMIT
    w1 = np.array([1], np.int32)
    assert lib.sp_single_pulse_search(1, 4, 100, w1.ctypes.data, 1, 6.0, 0, 256, 10, 256, 10, 256, 0) \
        == sp.SP_EWORKSPACE


@pytest.mark.parametrize("cfg", [synth.config1, synth.config2])
def test_host_delays_equal_oracle(lib, cfg):
    wl = cfg()
    got, md = sp.compute_delays(wl.freqs, wl.tsamp, wl.dms)
    want = oracle.delays(wl.freqs, wl.tsamp, wl.dms)
    assert np.array_equal(got, want)
    assert md == int(want.max())


def test_host_delays_odd_plans(lib):
    rng = np.random.default_rng(4)
    for nchan in (1, 3, 100):
        f = np.sort(rng.uniform(100, 1500, nchan))[::-1].copy()
        if np.unique(f).size != nchan:
            continue
        dms = rng.uniform(0, 3000, 37)  # unsorted
        got, md = sp.compute_delays(f, 6.4e-5, dms)
        assert np.array_equal(got, oracle.delays(f, 6.4e-5, dms))


def test_shape_table_and_batch_argument_checks(lib):
    """Kernel shapes are reported without a GPU; the batch and autotuner
    entry points reject bad arguments before touching a device."""
    dt, tt, cc = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    seen = set()
    for s in range(sp.SP_DEDISP_NUM_SHAPES):
        assert lib.sp_dedisp_shape_info(s, ctypes.byref(dt), ctypes.byref(tt), ctypes.byref(cc)) == sp.SP_OK
        assert dt.value in (4 * cc.value, 8 * cc.value) and tt.value % 128 == 0 and cc.value % 4 == 0
        seen.add((dt.value, tt.value, cc.value))
    assert len(seen) == sp.SP_DEDISP_NUM_SHAPES
    assert (64, 512, 8) in seen and (32, 512, 8) in seen
    assert lib.sp_dedisp_shape_info(sp.SP_DEDISP_NUM_SHAPES, None, None, None) == sp.SP_EINVAL
    assert lib.sp_dedisp_shape_info(-1, None, None, None) == sp.SP_EINVAL
    f = synth.band_freqs(8)
    d = np.array([0.0, 10.0])
    ms = np.zeros(sp.SP_DEDISP_NUM_SHAPES, np.float32)
    best = ctypes.c_int32()
    assert lib.sp_autotune_dedisperse(None, 8, 1e-3, d.ctypes.data, 2, 100, 1, ms.ctypes.data, ctypes.byref(best),
                                      None) == sp.SP_EINVAL
    assert lib.sp_autotune_dedisperse(f.ctypes.data, 8, 1e-3, d.ctypes.data, 2, 0, 1, ms.ctypes.data,
                                      ctypes.byref(best), None) == sp.SP_EINVAL
    h = ctypes.c_void_p()
    assert lib.sp_plan_create_shaped(f.ctypes.data, 8, 1e-3, d.ctypes.data, 2, 7, ctypes.byref(h)) == sp.SP_EINVAL
    assert lib.sp_dedisperse_batch_workspace_bytes(0) == -1
    assert lib.sp_dedisperse_batch_workspace_bytes(3) % 256 == 0
    assert lib.sp_dedisperse_batch(None, 1, None, 0, None) == sp.SP_EINVAL
    w = np.array([1, 2, 4], np.int32)
    bp = np.zeros(1, np.int32)
    bn = np.full(1, 100, np.int64)
    assert lib.sp_batch_create(None, 1, bp.ctypes.data, bn.ctypes.data, 1, w.ctypes.data, 3, 6.0, 0, 10, 1 << 20,
                               ctypes.byref(h)) == sp.SP_EINVAL
    assert lib.sp_batch_create(None, 0, None, None, 0, w.ctypes.data, 3, 6.0, 0, 10, 1 << 20, None) == sp.SP_EINVAL
    for fn, args in [("sp_batch_destroy", [None]), ("sp_batch_info", [None, None, None]),
                     ("sp_batch_input", [None, 0, None, None]), ("sp_batch_run", [None, 0, None]),
                     ("sp_batch_capture", [None, 0, None]), ("sp_batch_launch", [None, None]),
                     ("sp_batch_results", [None, 0, None, 0, None, None]), ("sp_batch_dmt", [None, 0, None]),
                     ("sp_batch_run_host", [None, None, None, 0, None, None]),
                     ("sp_batch_status", [None, None, 0]), ("sp_batch_group_ms", [None, None])]:
        assert getattr(lib, fn)(*args) == sp.SP_EINVAL, fn


def test_stream_argument_checks(lib):
    """The streaming entry points reject bad arguments before any device
    work; the clock is monotonic."""
    w = np.array([1, 2, 4], np.int32)
    h = ctypes.c_void_p()
    assert lib.sp_stream_create(None, 4, 100, w.ctypes.data, 3, 6.0, 0, 16, 1 << 30, 4, 0, ctypes.byref(h)) \
        == sp.SP_EINVAL
    assert lib.sp_stream_create(None, 4, 100, w.ctypes.data, 3, 6.0, 0, 16, 1 << 30, 4, 0, None) == sp.SP_EINVAL
    for fn, args in [("sp_stream_destroy", [None]), ("sp_stream_info", [None, None, None, None]),
                     ("sp_stream_history", [None, 0, None]), ("sp_stream_push", [None, 0, None, None]),
                     ("sp_stream_poll", [None, 0, None, None, 0, None]),
                     ("sp_stream_pending", [None, None, None, None]),
                     ("sp_stream_attach", [None, None, None, 512, 64]),
                     ("sp_stream_poll_sifted", [None, 0, None, None, None, None, 0, None])]:
        assert getattr(lib, fn)(*args) == sp.SP_EINVAL, fn
    t0 = lib.sp_stream_now()
    t1 = lib.sp_stream_now()
    assert t1 >= t0 > 0


def test_launch_counter_needs_no_device(lib):
    """The launch counter is host state, readable without a GPU; a call
    rejected by its argument checks launches nothing."""
    c0 = sp.launch_count()
    assert c0 >= 0
    assert lib.sp_single_pulse_search(None, 0, 0, None, 0, 6.0, 0, None, 0, None, 0, None, None) == sp.SP_EINVAL
    assert sp.launch_count() == c0


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_staging_tables_sound_for_every_workload(lib, shape):
    """Every bulk copy, shifted copy and shared load the dedispersion kernel
    makes with a plan's tables stays aligned and in bounds (host-only check),
    and the kernel's shared memory fits a GB300 SM: configs 1 and 2, the
    three DM plans of config 3 at both ends of its length range, and random
    unsorted DM lists with duplicates over ragged channel counts."""
    cases = []
    c1, c2 = synth.config1(), synth.config2()
    cases.append((c1.freqs, c1.tsamp, c1.dms, c1.n_out))
    cases.append((c2.freqs, c2.tsamp, c2.dms, c2.n_out))
    f4k = synth.band_freqs(4096)
    for dm_max in (500.0, 1000.0, 2000.0):
        dms = synth.dm_plan_upto(dm_max)
        for n_out in (16384, 131072):
            cases.append((f4k, synth.TSAMP, dms, n_out))
    rng = np.random.default_rng(5)
    for nchan in (1, 7, 64, 100, 256):
        dms = rng.choice(np.arange(0, 800.0, 0.5), size=int(rng.integers(1, 300)))
        cases.append((synth.band_freqs(nchan), synth.TSAMP, dms, int(rng.integers(1, 5000))))
    for freqs, tsamp, dms, n_out in cases:
        rep = sp.plan_check_tables(freqs, tsamp, dms, shape, n_out)
        assert rep["violations"] == 0, rep
        assert rep["smem_bytes"] <= 227 * 1024, rep
    with pytest.raises(sp.SpotlightError):
        sp.plan_check_tables(c1.freqs, c1.tsamp, c1.dms, 7, 100)  # no such shape


def test_noalloc_rejects_requests_beyond_its_scratch(lib):
    """The allocation-free search refuses, before any CUDA call, a request
    whose block statistics exceed its fixed 16 MiB array.  No device buffer
    is involved: the DM transform pointer is never dereferenced, and the
    candidate count is NULL so that even a regressed size check would stop
    at the argument check instead of launching anything."""
    huge_rows, n_out, L = 65535, 4096 * 64, 64  # statistics for 65535 rows x 4096 blocks
    assert sp.sps_workspace_bytes(huge_rows, n_out, 2, L) > sp.SP_NOALLOC_SCRATCH_BYTES
    w = np.array([1, 2], np.int32)
    fake = ctypes.c_void_p(16)
    rc = lib.sp_single_pulse_search_noalloc(fake, huge_rows, n_out, w.ctypes.data, 2, ctypes.c_float(6.0), L,
                                            None, 0, None, None)
    assert rc == sp.SP_ELIMIT
    # within the limit the same NULL count is an argument error, still without a GPU
    small = sp.sps_workspace_bytes(8, 1024, 2, 0)
    assert 0 < small <= sp.SP_NOALLOC_SCRATCH_BYTES
