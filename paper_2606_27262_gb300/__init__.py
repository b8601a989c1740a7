"""Python binding of libspotlight (include/spotlight.h), the GB300 search hot
path of the SPOTLIGHT pipeline (arXiv 2606.27262, Sec. 3.1).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch provides device memory and streams; the C ABI itself sees
plain pointers and sizes.  If the shared library is missing this module
raises -- there is no fallback implementation.

Names mirror the C entry points:

* ``Plan``                       sp_plan_create / _info / _delays / _destroy
* ``dedisperse``                 sp_dedisperse (+ workspace sizing)
* ``single_pulse_search``        sp_single_pulse_search
* ``best_snr_map``               sp_best_snr_map
* ``Searcher``                   sp_searcher_create / _run / _run_host
* ``autotune_dedisperse``        sp_autotune_dedisperse (kernel shape choice)
* ``dedisperse_batch``           sp_dedisperse_batch (many beams, one launch)
* ``Batch``                      sp_batch_* (grouped multi-beam step, graph)
* ``Stream``                     sp_stream_* (real-time gulps, continuous batching)
* ``sift``                       sp_sift (DBSCAN clustering + thresholds, host)
* ``inject_quantised``           sp_inject_quantised (Appendix B injection)
* ``Classifier``, ``cnn_features``, ``dmt_shifts``  sp_cnn_* (two-image CNN)
* ``launch_count``               sp_launch_count (kernels issued, for measurement)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspotlight.so")

SP_OK, SP_EINVAL, SP_ESHAPE, SP_ECUDA, SP_EOVERFLOW, SP_ENOMEM, SP_EWORKSPACE, SP_ELIMIT = 0, -1, -2, -3, -4, -5, -6, -7
SP_ETIMEOUT = -8
SP_STATUS_STAGING_TIMEOUT = 1
SP_MAX_WIDTHS = 16
SP_MAX_WIDTH = 1024

CAND_DTYPE = np.dtype([("dm_idx", np.int32), ("t", np.int32), ("width_idx", np.int32), ("snr", np.float32)])


class SpotlightError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_lib().sp_strerror(code).decode()} ({code})")


_L = None

# Every exported symbol with (restype, argtypes); tests check this list
# against include/spotlight.h.
P, I32, I64, F32, F64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
SIGNATURES = {
    "sp_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sp_plan_create": (ctypes.c_int, [P, I32, F64, P, I32, P]),
    "sp_plan_destroy": (ctypes.c_int, [P]),
    "sp_plan_info": (ctypes.c_int, [P, P, P, P]),
    "sp_plan_delays": (ctypes.c_int, [P, P]),
    "sp_plan_status": (ctypes.c_int, [P, P, I32]),
    "sp_compute_delays": (ctypes.c_int, [P, I32, F64, P, I32, P, P]),
    "sp_dedisperse_workspace_bytes": (I64, [P, I64]),
    "sp_dedisperse": (ctypes.c_int, [P, P, I64, P, I64, P, I64, P]),
    "sp_staged_pitch": (I64, [I64]),
    "sp_staged_bytes": (I64, [I32, I64]),
    "sp_stage_input": (ctypes.c_int, [P, I64, I32, P, I64, P]),
    "sp_dedisperse_staged": (ctypes.c_int, [P, P, I64, I64, P, I64, P]),
    "sp_sps_workspace_bytes": (I64, [I32, I64, I32, I64]),
    "sp_single_pulse_search": (ctypes.c_int, [P, I32, I64, P, I32, F32, I64, P, I64, P, I64, P, P]),
    "sp_single_pulse_search_noalloc": (ctypes.c_int, [P, I32, I64, P, I32, F32, I64, P, I64, P, P]),
    "sp_best_snr_map": (ctypes.c_int, [P, I32, I64, P, I32, I64, P, I64, P, P, P]),
    "sp_searcher_create": (ctypes.c_int, [P, I64, P, I32, F32, I64, I64, P]),
    "sp_searcher_destroy": (ctypes.c_int, [P]),
    "sp_searcher_run": (ctypes.c_int, [P, P, P, I64, P, P]),
    "sp_searcher_run_host": (ctypes.c_int, [P, P, P, I64, P, P]),
    "sp_searcher_submit_host": (ctypes.c_int, [P, P, P]),
    "sp_debug_staging_fault": (ctypes.c_int, [ctypes.c_int32, I64]),
    "sp_sps_window_workspace_bytes": (I64, [I32, I64, I32, I64, I32]),
    "sp_single_pulse_search_window": (ctypes.c_int, [P, I32, I64, P, I32, ctypes.c_float, I64, I32, P, I64, P, I64,
                                                     P, P]),
    "sp_searcher_collect": (ctypes.c_int, [P, P, I64, P]),
    "sp_dedisp_shape_info": (ctypes.c_int, [I32, P, P, P]),
    "sp_plan_create_shaped": (ctypes.c_int, [P, I32, F64, P, I32, I32, P]),
    "sp_plan_shape": (ctypes.c_int, [P, P, P, P]),
    "sp_autotune_dedisperse": (ctypes.c_int, [P, I32, F64, P, I32, I64, I32, P, P, P]),
    "sp_dedisperse_batch_workspace_bytes": (I64, [I32]),
    "sp_dedisperse_batch": (ctypes.c_int, [P, I32, P, I64, P]),
    "sp_batch_create": (ctypes.c_int, [P, I32, P, P, I32, P, I32, F32, I64, I64, I64, P]),
    "sp_batch_destroy": (ctypes.c_int, [P]),
    "sp_batch_info": (ctypes.c_int, [P, P, P]),
    "sp_batch_input": (ctypes.c_int, [P, I32, P, P]),
    "sp_batch_run": (ctypes.c_int, [P, I32, P]),
    "sp_batch_group_ms": (ctypes.c_int, [P, P]),
    "sp_batch_capture": (ctypes.c_int, [P, I32, P]),
    "sp_batch_launch": (ctypes.c_int, [P, P]),
    "sp_batch_results": (ctypes.c_int, [P, I32, P, I64, P, P]),
    "sp_batch_dmt": (ctypes.c_int, [P, I32, P]),
    "sp_batch_run_host": (ctypes.c_int, [P, P, P, I64, P, P]),
    "sp_batch_status": (ctypes.c_int, [P, P, I32]),
    "sp_stream_create": (ctypes.c_int, [P, I32, I64, P, I32, F32, I64, I64, I64, I32, I32, P]),
    "sp_stream_destroy": (ctypes.c_int, [P]),
    "sp_stream_info": (ctypes.c_int, [P, P, P, P]),
    "sp_stream_history": (ctypes.c_int, [P, I32, P]),
    "sp_stream_push": (ctypes.c_int, [P, I32, P, P]),
    "sp_stream_poll": (ctypes.c_int, [P, I32, P, P, I32, P]),
    "sp_stream_pending": (ctypes.c_int, [P, P, P, P]),
    "sp_stream_now": (F64, []),
    "sp_stream_attach": (ctypes.c_int, [P, P, P, I32, I32]),
    "sp_launch_count": (ctypes.c_uint64, []),
    "sp_plan_check_tables": (ctypes.c_int, [P, I32, F64, P, I32, I32, I64, P]),
    "sp_stream_poll_sifted": (ctypes.c_int, [P, I32, P, P, P, P, I32, P]),
    "sp_sift": (ctypes.c_int, [P, I64, P, I32, P, I32, F64, P, P, I64, P, P]),
    "sp_inject_quantised": (ctypes.c_int, [P, P, I64, I32, F64, F64, F64, P]),
    "sp_cnn_num_params": (I64, []),
    "sp_cnn_create": (ctypes.c_int, [I32, ctypes.c_uint64, P]),
    "sp_cnn_destroy": (ctypes.c_int, [P]),
    "sp_cnn_get_params": (ctypes.c_int, [P, P]),
    "sp_cnn_set_params": (ctypes.c_int, [P, P]),
    "sp_cnn_get_grads": (ctypes.c_int, [P, P]),
    "sp_cnn_forward": (ctypes.c_int, [P, P, P, I32, P, P]),
    "sp_cnn_backward": (ctypes.c_int, [P, P, P, P, I32, P, P]),
    "sp_cnn_adam_step": (ctypes.c_int, [P, F32, P]),
    "sp_cnn_train_step": (ctypes.c_int, [P, P, P, P, I32, F32, P, P]),
    "sp_cnn_features_workspace_bytes": (I64, [I32]),
    "sp_cnn_features": (ctypes.c_int, [P, I32, I32, I32, P, P, P, P, I64, P]),
    "sp_dmt_shifts": (ctypes.c_int, [P, I32, I32, I32, P]),
    "sp_cnn_extract": (ctypes.c_int, [P, P, I64, I64, P, I32, P, I32, I32, P, P]),
    "sp_probe_iadd3_rate": (ctypes.c_int, [ctypes.c_int, P, P]),
}
SP_DEDISP_NUM_SHAPES = 4
SP_SHAPE_AUTO = -1
SP_AUTOTUNE_SAMPLES = 16384
SP_AUTOTUNE_REPS = 3
SP_BATCH_GROUPED, SP_BATCH_PER_BEAM, SP_BATCH_GROUPED_GRID, SP_BATCH_TIMED = 0, 1, 2, 16
SP_STREAM_PER_GULP, SP_STREAM_ONE_STREAM = 1, 2
SP_CNN_MAX_BATCH = 256
CNN_IMG = 256


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libspotlight is not built ({LIB_PATH} missing); "
                               "run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _L = lib
    return _L


def library():
    """The loaded ctypes handle (raises if the library is not built)."""
    return _lib()


def _check(rc: int, what: str):
    if rc != SP_OK:
        raise SpotlightError(rc, what)


def _ptr(t) -> int:
    """Device/host pointer of a torch tensor or numpy array."""
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _widths(widths) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(widths, dtype=np.int32))


def shape_info(shape: int):
    """(DM tile, time tile, channel chunk) of a compiled kernel shape."""
    a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().sp_dedisp_shape_info(int(shape), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "sp_dedisp_shape_info")
    return int(a.value), int(b.value), int(c.value)


class Plan:
    """Dedispersion plan: delay table of Eq. 1 (rounded half up) and tiling.
    ``shape`` None = sp_plan_create (shape 0); an int = sp_plan_create_shaped
    (SP_SHAPE_AUTO lets the autotuner choose)."""

    def __init__(self, freqs_mhz, tsamp_s: float, dms, shape: int | None = None):
        f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
        d = np.ascontiguousarray(dms, dtype=np.float64)
        h = ctypes.c_void_p()
        if shape is None:
            _check(_lib().sp_plan_create(f.ctypes.data, f.size, float(tsamp_s), d.ctypes.data, d.size,
                                         ctypes.byref(h)), "sp_plan_create")
        else:
            _check(_lib().sp_plan_create_shaped(f.ctypes.data, f.size, float(tsamp_s), d.ctypes.data, d.size,
                                                int(shape), ctypes.byref(h)), "sp_plan_create_shaped")
        self._h = h
        sh, nt, sm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib().sp_plan_shape(h, ctypes.byref(sh), ctypes.byref(nt), ctypes.byref(sm)), "sp_plan_shape")
        self.shape, self.ntiles, self.smem_bytes = int(sh.value), int(nt.value), int(sm.value)
        md, nc, nd = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(_lib().sp_plan_info(h, ctypes.byref(md), ctypes.byref(nc), ctypes.byref(nd)), "sp_plan_info")
        self.max_delay, self.nchan, self.ndm = md.value, nc.value, nd.value
        self.dms = d.copy()
        self.freqs = f.copy()
        self.tsamp = float(tsamp_s)

    @property
    def handle(self):
        return self._h

    def delays(self) -> np.ndarray:
        out = np.empty((self.ndm, self.nchan), np.int32)
        _check(_lib().sp_plan_delays(self._h, out.ctypes.data), "sp_plan_delays")
        return out

    def status(self, clear: bool = False) -> int:
        """Device status word (0 = ok; SP_STATUS_* bits otherwise)."""
        v = ctypes.c_int32()
        _check(_lib().sp_plan_status(self._h, ctypes.byref(v), int(clear)), "sp_plan_status")
        return int(v.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().sp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def compute_delays(freqs_mhz, tsamp_s: float, dms):
    """Host-only delay table (int32 [ndm][nchan]) and its maximum."""
    f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    out = np.empty((d.size, f.size), np.int32)
    md = ctypes.c_int32()
    _check(_lib().sp_compute_delays(f.ctypes.data, f.size, float(tsamp_s), d.ctypes.data, d.size,
                                    out.ctypes.data, ctypes.byref(md)), "sp_compute_delays")
    return out, int(md.value)


def dedisperse_workspace_bytes(plan: Plan, n_in: int) -> int:
    return int(_lib().sp_dedisperse_workspace_bytes(plan.handle, int(n_in)))


def sps_workspace_bytes(ndm: int, n_out: int, nw: int, norm_block: int) -> int:
    return int(_lib().sp_sps_workspace_bytes(int(ndm), int(n_out), int(nw), int(norm_block)))


def dedisperse(plan: Plan, d_in, d_out, d_work, stream=None):
    """d_in: uint8 [n_in][nchan] CUDA tensor; d_out: int32 [ndm][n_out];
    d_work: uint8 CUDA tensor of at least dedisperse_workspace_bytes()."""
    n_in, n_out = int(d_in.shape[0]), int(d_out.shape[1])
    _check(_lib().sp_dedisperse(plan.handle, _ptr(d_in), n_in, _ptr(d_out), n_out, _ptr(d_work),
                                int(d_work.numel()), _stream(stream)), "sp_dedisperse")


def staged_pitch(n_in: int) -> int:
    return int(_lib().sp_staged_pitch(int(n_in)))


def staged_bytes(nchan: int, n_in: int) -> int:
    return int(_lib().sp_staged_bytes(int(nchan), int(n_in)))


def staged_buffer(nchan: int, n_in: int, device="cuda"):
    """A device buffer for the staged form of an input (sp_stage_input)."""
    import torch
    return torch.empty(staged_bytes(nchan, n_in), dtype=torch.uint8, device=device)


def stage_input(d_in, d_staged, stream=None):
    """d_in uint8 [n_in][nchan] -> d_staged (staged_buffer(nchan, n_in))."""
    _check(_lib().sp_stage_input(_ptr(d_in), int(d_in.shape[0]), int(d_in.shape[1]), _ptr(d_staged),
                                 staged_pitch(int(d_in.shape[0])), _stream(stream)), "sp_stage_input")


def dedisperse_staged(plan: Plan, d_staged, n_in: int, d_out, stream=None):
    """DM transform of a staged input (staged_buffer(nchan, n_in))."""
    _check(_lib().sp_dedisperse_staged(plan.handle, _ptr(d_staged), staged_pitch(int(n_in)), int(n_in), _ptr(d_out),
                                       int(d_out.shape[1]), _stream(stream)), "sp_dedisperse_staged")


def single_pulse_search(d_dmt, widths, threshold: float, norm_block: int, d_work, d_cands, d_count,
                        stream=None):
    """d_dmt: int32 [ndm][n_out]; d_cands: int32 [cap][4] CUDA tensor (sp_cand
    records); d_count: int64 [1] CUDA tensor (total found)."""
    w = _widths(widths)
    _check(_lib().sp_single_pulse_search(_ptr(d_dmt), int(d_dmt.shape[0]), int(d_dmt.shape[1]), w.ctypes.data,
                                         w.size, float(threshold), int(norm_block), _ptr(d_work),
                                         int(d_work.numel()), _ptr(d_cands), int(d_cands.shape[0]),
                                         _ptr(d_count), _stream(stream)), "sp_single_pulse_search")


def sps_window_workspace_bytes(ndm: int, n_out: int, nw: int, norm_block: int, peak_radius: int) -> int:
    return int(_lib().sp_sps_window_workspace_bytes(int(ndm), int(n_out), int(nw), int(norm_block),
                                                    int(peak_radius)))


def single_pulse_search_window(d_dmt, widths, threshold: float, norm_block: int, peak_radius: int, d_work, d_cands,
                               d_count, stream=None):
    """single_pulse_search with a (2 peak_radius + 1)^2 peak filter
    (sp_single_pulse_search_window; 5 = the paper's 11 x 11 stencil)."""
    w = _widths(widths)
    _check(_lib().sp_single_pulse_search_window(_ptr(d_dmt), int(d_dmt.shape[0]), int(d_dmt.shape[1]), w.ctypes.data,
                                                w.size, float(threshold), int(norm_block), int(peak_radius),
                                                _ptr(d_work), int(d_work.numel()), _ptr(d_cands),
                                                int(d_cands.shape[0]), _ptr(d_count), _stream(stream)),
           "sp_single_pulse_search_window")


SP_NOALLOC_SCRATCH_BYTES = 16 << 20


def single_pulse_search_noalloc(d_dmt, widths, threshold: float, norm_block: int, d_cands, d_count,
                                stream=None):
    """sp_single_pulse_search without a workspace: for callers that cannot
    allocate device memory while searching (a real-time loop with its memory
    budget fixed at start-up, a host whose device memory belongs to its own
    pool, a plug-in barred from cudaMalloc).  The block statistics live in a
    16 MiB library-owned device array shared by every call on the device, so
    calls whose GPU work overlaps must be serialised by the caller."""
    w = _widths(widths)
    _check(_lib().sp_single_pulse_search_noalloc(_ptr(d_dmt), int(d_dmt.shape[0]), int(d_dmt.shape[1]),
                                                 w.ctypes.data, w.size, float(threshold), int(norm_block),
                                                 _ptr(d_cands), int(d_cands.shape[0]), _ptr(d_count),
                                                 _stream(stream)), "sp_single_pulse_search_noalloc")


def best_snr_map(d_dmt, widths, norm_block: int, d_work, d_best, d_wbest, stream=None):
    """d_best: float32 [ndm][n_out]; d_wbest: int8 [ndm][n_out]."""
    w = _widths(widths)
    _check(_lib().sp_best_snr_map(_ptr(d_dmt), int(d_dmt.shape[0]), int(d_dmt.shape[1]), w.ctypes.data, w.size,
                                  int(norm_block), _ptr(d_work), int(d_work.numel()), _ptr(d_best),
                                  _ptr(d_wbest), _stream(stream)), "sp_best_snr_map")


def cands_to_numpy(cands_i32: np.ndarray, count: int) -> np.ndarray:
    """sp_cand records (an int32 [cap][4] array) -> structured array sorted
    by (dm_idx, t)."""
    n = min(int(count), cands_i32.shape[0])
    rec = np.ascontiguousarray(cands_i32[:n]).view(CAND_DTYPE).reshape(-1)
    return np.sort(rec, order=["dm_idx", "t"])


class Searcher:
    """Whole per-beam path with its device buffers allocated once."""

    def __init__(self, plan: Plan, n_out: int, widths, threshold: float, norm_block: int, cand_cap: int):
        w = _widths(widths)
        h = ctypes.c_void_p()
        _check(_lib().sp_searcher_create(plan.handle, int(n_out), w.ctypes.data, w.size, float(threshold),
                                         int(norm_block), int(cand_cap), ctypes.byref(h)), "sp_searcher_create")
        self._h = h
        self.plan = plan
        self.n_out = int(n_out)
        self.n_in = int(n_out) + plan.max_delay
        self.cap = int(cand_cap)

    def run(self, d_in, d_cands, d_count, stream=None):
        _check(_lib().sp_searcher_run(self._h, _ptr(d_in), _ptr(d_cands), int(d_cands.shape[0]), _ptr(d_count),
                                      _stream(stream)), "sp_searcher_run")

    def run_host(self, h_in, h_cands: np.ndarray, stream=None) -> int:
        """h_in: host uint8 [n_in][nchan] (numpy array or pinned CPU tensor);
        h_cands: int32 [cap][4] numpy array.  Returns the total count."""
        cnt = ctypes.c_int64()
        rc = _lib().sp_searcher_run_host(self._h, _ptr(h_in), h_cands.ctypes.data, h_cands.shape[0],
                                         ctypes.byref(cnt), _stream(stream))
        if rc not in (SP_OK, SP_EOVERFLOW):
            _check(rc, "sp_searcher_run_host")
        return int(cnt.value)

    def submit_host(self, h_in, stream=None):
        """Queues one beam from host memory (page-locked for overlap); at
        most two uncollected beams.  h_in must stay unchanged until collected."""
        _check(_lib().sp_searcher_submit_host(self._h, _ptr(h_in), _stream(stream)), "sp_searcher_submit_host")

    def collect(self, h_cands: np.ndarray) -> int:
        """Waits for the oldest submitted beam; fills h_cands (int32 [cap][4])
        and returns its total count."""
        cnt = ctypes.c_int64()
        rc = _lib().sp_searcher_collect(self._h, h_cands.ctypes.data, h_cands.shape[0], ctypes.byref(cnt))
        if rc not in (SP_OK, SP_EOVERFLOW):
            _check(rc, "sp_searcher_collect")
        return int(cnt.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().sp_searcher_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_staging_fault(extra_bytes: int, wait_limit_cycles: int = 1 << 31):
    """Test hook: make every dedispersion CTA's first staging wait expect
    extra_bytes more than arrive, with waits bounded at wait_limit_cycles
    (sp_debug_staging_fault); (0, 1 << 31) restores the defaults."""
    _check(_lib().sp_debug_staging_fault(int(extra_bytes), int(wait_limit_cycles)), "sp_debug_staging_fault")


def autotune_dedisperse(freqs_mhz, tsamp_s: float, dms, n_out_sample: int = SP_AUTOTUNE_SAMPLES,
                        reps: int = SP_AUTOTUNE_REPS, stream=None):
    """Times every kernel shape on this plan; returns (best shape, ms per
    launch of each shape, +inf where a shape cannot run)."""
    f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    ms = np.empty(SP_DEDISP_NUM_SHAPES, np.float32)
    best = ctypes.c_int32()
    _check(_lib().sp_autotune_dedisperse(f.ctypes.data, f.size, float(tsamp_s), d.ctypes.data, d.size,
                                         int(n_out_sample), int(reps), ms.ctypes.data, ctypes.byref(best),
                                         _stream(stream)), "sp_autotune_dedisperse")
    return int(best.value), ms


class _CudaArray:
    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(x) for x in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _device_view(ptr: int, rows: int, cols: int, typestr: str):
    import torch
    return torch.as_tensor(_CudaArray(ptr, (rows, cols), typestr), device="cuda")


class _BatchBeam(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("d_staged", ctypes.c_void_p), ("pitch", ctypes.c_int64),
                ("n_in", ctypes.c_int64), ("d_out", ctypes.c_void_p), ("n_out", ctypes.c_int64)]


def dedisperse_batch_workspace_bytes(nbeams: int) -> int:
    return int(_lib().sp_dedisperse_batch_workspace_bytes(int(nbeams)))


def dedisperse_batch(beams, d_work, stream=None):
    """beams: list of (plan, d_staged, n_in, d_out) with d_staged from
    staged_buffer(nchan, n_in) (filled by stage_input) and d_out int32
    [ndm][n_out].  One persistent launch for all of them."""
    arr = (_BatchBeam * len(beams))()
    for i, (plan, staged, n_in, out) in enumerate(beams):
        arr[i] = _BatchBeam(plan.handle.value, _ptr(staged), staged_pitch(int(n_in)), int(n_in), _ptr(out),
                            int(out.shape[1]))
    _check(_lib().sp_dedisperse_batch(ctypes.cast(arr, ctypes.c_void_p), len(beams), _ptr(d_work),
                                      int(d_work.numel()), _stream(stream)), "sp_dedisperse_batch")


class Batch:
    """A fixed set of beams searched as one step (sp_batch_*): grouped
    persistent dedispersion under a DM-transform memory budget, searches
    overlapped on a second stream, optional CUDA-graph capture."""

    def __init__(self, plans, beam_plan, beam_n_out, widths, threshold: float, norm_block: int, cand_cap: int,
                 dmt_budget_bytes: int):
        self.plans = list(plans)
        hp = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        bp = np.ascontiguousarray(beam_plan, dtype=np.int32)
        bn = np.ascontiguousarray(beam_n_out, dtype=np.int64)
        w = _widths(widths)
        h = ctypes.c_void_p()
        _check(_lib().sp_batch_create(ctypes.cast(hp, ctypes.c_void_p), len(self.plans), bp.ctypes.data,
                                      bn.ctypes.data, bp.size, w.ctypes.data, w.size, float(threshold),
                                      int(norm_block), int(cand_cap), int(dmt_budget_bytes), ctypes.byref(h)),
               "sp_batch_create")
        self._h = h
        self.nbeams = int(bp.size)
        self.beam_plan = bp.copy()
        self.n_out = bn.copy()
        self.cap = int(cand_cap)
        ng, nb = ctypes.c_int32(), ctypes.c_int64()
        _check(_lib().sp_batch_info(h, ctypes.byref(ng), ctypes.byref(nb)), "sp_batch_info")
        self.ngroups, self.device_bytes = int(ng.value), int(nb.value)

    def input(self, beam: int):
        """(device address, n_in) of beam's input buffer [n_in][nchan]."""
        p, n = ctypes.c_void_p(), ctypes.c_int64()
        _check(_lib().sp_batch_input(self._h, int(beam), ctypes.byref(p), ctypes.byref(n)), "sp_batch_input")
        return int(p.value), int(n.value)

    def input_tensor(self, beam: int, nchan: int):
        """torch view (no copy) of beam's input buffer, uint8 [n_in][nchan]."""
        return _device_view(*self.input(beam), nchan, "|u1")

    def dmt_tensor(self, beam: int, ndm: int):
        """torch view of beam's DM transform as left by the last run, int32
        [ndm][n_out] (sp_batch_dmt: only while the arenas still hold it)."""
        return _device_view(self.dmt_ptr(beam), ndm, int(self.n_out[beam]), "<i4")

    def run(self, mode: int = SP_BATCH_GROUPED, stream=None):
        _check(_lib().sp_batch_run(self._h, int(mode), _stream(stream)), "sp_batch_run")

    def group_ms(self) -> np.ndarray:
        """Per-group persistent-launch times (ms) of the last timed run."""
        out = np.zeros(self.ngroups, np.float32)
        _check(_lib().sp_batch_group_ms(self._h, out.ctypes.data), "sp_batch_group_ms")
        return out

    def capture(self, mode: int = SP_BATCH_GROUPED, stream=None):
        _check(_lib().sp_batch_capture(self._h, int(mode), _stream(stream)), "sp_batch_capture")

    def launch(self, stream=None):
        _check(_lib().sp_batch_launch(self._h, _stream(stream)), "sp_batch_launch")

    def results(self, beam: int, stream=None) -> np.ndarray:
        """Candidates of one beam (structured array sorted by (dm_idx, t))."""
        buf = np.zeros((max(self.cap, 1), 4), np.int32)
        cnt = ctypes.c_int64()
        rc = _lib().sp_batch_results(self._h, int(beam), buf.ctypes.data, self.cap, ctypes.byref(cnt),
                                     _stream(stream))
        if rc not in (SP_OK, SP_EOVERFLOW):
            _check(rc, "sp_batch_results")
        return cands_to_numpy(buf, int(cnt.value))

    def count(self, beam: int, stream=None) -> int:
        cnt = ctypes.c_int64()
        rc = _lib().sp_batch_results(self._h, int(beam), None, 0, ctypes.byref(cnt), _stream(stream))
        if rc not in (SP_OK, SP_EOVERFLOW):
            _check(rc, "sp_batch_results")
        return int(cnt.value)

    def dmt_ptr(self, beam: int) -> int:
        p = ctypes.c_void_p()
        _check(_lib().sp_batch_dmt(self._h, int(beam), ctypes.byref(p)), "sp_batch_dmt")
        return int(p.value)

    def run_host(self, h_inputs, h_cands: np.ndarray, stream=None) -> np.ndarray:
        """h_inputs: per beam a host uint8 [n_in][nchan] array or pinned CPU
        tensor; h_cands: int32 [nbeams * cap_per_beam][4].  Returns the
        per-beam counts."""
        arr = (ctypes.c_void_p * self.nbeams)(*[_ptr(x) for x in h_inputs])
        counts = np.zeros(self.nbeams, np.int64)
        cap_pb = h_cands.shape[0] // self.nbeams
        rc = _lib().sp_batch_run_host(self._h, ctypes.cast(arr, ctypes.c_void_p), h_cands.ctypes.data, cap_pb,
                                      counts.ctypes.data, _stream(stream))
        if rc not in (SP_OK, SP_EOVERFLOW):
            _check(rc, "sp_batch_run_host")
        return counts

    def status(self, clear: bool = False) -> int:
        v = ctypes.c_int32()
        _check(_lib().sp_batch_status(self._h, ctypes.byref(v), int(clear)), "sp_batch_status")
        return int(v.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().sp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GulpResult(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("status", ctypes.c_int32), ("seq", ctypes.c_int64),
                ("t0", ctypes.c_int64), ("count", ctypes.c_int64), ("t_push", ctypes.c_double),
                ("t_done", ctypes.c_double), ("t_search", ctypes.c_double), ("kept", ctypes.c_int64),
                ("accepted", ctypes.c_int64)]


def plan_check_tables(freqs_mhz, tsamp_s: float, dms, shape: int, n_out: int) -> dict:
    """Host-only check of a plan's staging tables against the dedispersion
    kernel's accesses (sp_plan_check_tables); no GPU needed."""
    f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    rep = np.zeros(8, np.int64)
    _check(_lib().sp_plan_check_tables(f.ctypes.data, f.size, float(tsamp_s), d.ctypes.data, d.size, int(shape),
                                       int(n_out), rep.ctypes.data), "sp_plan_check_tables")
    keys = ("ntiles", "nchunks", "copies_bytes", "raw_bytes", "smem_bytes", "violations", "max_delay", "pitch")
    return dict(zip(keys, (int(v) for v in rep)))


def launch_count() -> int:
    """Kernel launches the library has issued in this process
    (sp_launch_count; graph kernels count once per replay)."""
    return int(_lib().sp_launch_count())


def stream_now() -> float:
    """The clock of the stream's arrival and completion stamps (seconds)."""
    return float(_lib().sp_stream_now())


class Stream:
    """Real-time streaming search (sp_stream_*): per-beam device rings,
    HBM-budgeted slots, continuous batching of pushed gulps."""

    def __init__(self, plan: Plan, nbeams: int, gulp: int, widths, threshold: float, norm_block: int,
                 cand_cap: int, hbm_budget_bytes: int, max_batch: int = 16, flags: int = 0):
        w = _widths(widths)
        h = ctypes.c_void_p()
        _check(_lib().sp_stream_create(plan.handle, int(nbeams), int(gulp), w.ctypes.data, w.size, float(threshold),
                                       int(norm_block), int(cand_cap), int(hbm_budget_bytes), int(max_batch),
                                       int(flags), ctypes.byref(h)), "sp_stream_create")
        self._h = h
        self.plan, self.nbeams, self.gulp, self.cap = plan, int(nbeams), int(gulp), int(cand_cap)
        sl, nb, ni = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib().sp_stream_info(h, ctypes.byref(sl), ctypes.byref(nb), ctypes.byref(ni)), "sp_stream_info")
        self.slots, self.device_bytes, self.n_in = int(sl.value), int(nb.value), int(ni.value)
        self._keep = {}  # host buffers referenced by gulps not yet returned
        self.kept_cap = 0
        self._clf = None

    def attach(self, clf=None, t_in: int = 512, kept_cap: int = 64, **sift_params):
        """Sifts every finished gulp (sp_sift, SIFT_DEFAULTS updated by
        sift_params) and, with a Classifier, scores the kept peaks from the
        gulp's staged window (sp_stream_attach); results then come from
        poll_sifted."""
        p = dict(SIFT_DEFAULTS)
        p.update(sift_params)
        sp_p = SiftParams(float(p["eps"]), int(p["min_points"]), float(p["snr_min"]), float(p["dm_min"]),
                          float(p["width_max_s"]))
        _check(_lib().sp_stream_attach(self._h, ctypes.byref(sp_p), clf._h if clf is not None else None,
                                       int(t_in), int(kept_cap)), "sp_stream_attach")
        self.kept_cap = int(kept_cap)
        self._clf = clf  # must outlive the stream
        device_bytes = ctypes.c_int64()
        _check(_lib().sp_stream_info(self._h, None, ctypes.byref(device_bytes), None), "sp_stream_info")
        self.device_bytes = int(device_bytes.value)

    def history(self, beam: int, h_hist):
        _check(_lib().sp_stream_history(self._h, int(beam), _ptr(h_hist)), "sp_stream_history")

    def push(self, beam: int, h_gulp) -> int:
        """Queues one gulp (host uint8 [gulp][nchan]); returns its sequence
        number.  The buffer is kept referenced until its result is polled."""
        seq = ctypes.c_int64()
        _check(_lib().sp_stream_push(self._h, int(beam), _ptr(h_gulp), ctypes.byref(seq)), "sp_stream_push")
        self._keep[(int(beam), int(seq.value))] = h_gulp
        return int(seq.value)

    def poll(self, wait: bool = False, max_results: int = 64, with_cands: bool = True):
        """Finished gulps: list of (GulpResult, candidates structured array
        sorted by (dm_idx, t)) in completion order."""
        if getattr(self, "_res_n", 0) < max_results:
            self._res = (GulpResult * max_results)()
            self._cands = np.zeros((max_results * self.cap, 4), np.int32)
            self._res_n = max_results
        res, cands = self._res, self._cands
        n = ctypes.c_int32()
        _check(_lib().sp_stream_poll(self._h, int(bool(wait)), ctypes.cast(res, ctypes.c_void_p),
                                     cands.ctypes.data if with_cands else None, int(max_results), ctypes.byref(n)),
               "sp_stream_poll")
        out = []
        for i in range(n.value):
            r = res[i]
            self._keep.pop((int(r.beam), int(r.seq)), None)
            c = (cands_to_numpy(cands[i * self.cap:(i + 1) * self.cap], min(int(r.count), self.cap))
                 if with_cands else None)
            out.append((GulpResult.from_buffer_copy(r), c))
        return out

    def poll_sifted(self, wait: bool = False, max_results: int = 64, with_cands: bool = False):
        """Finished gulps after the attached sifter (and classifier): list of
        (GulpResult, candidates or None, kept peaks structured array,
        probabilities float32 (-1 without a classifier))."""
        if getattr(self, "_sres_n", 0) < max_results:
            self._sres = (GulpResult * max_results)()
            self._skept = np.zeros((max_results * self.kept_cap, 4), np.int32)
            self._sprob = np.zeros(max_results * self.kept_cap, np.float32)
            self._sres_n = max_results
        if with_cands and getattr(self, "_scand_n", 0) < max_results:
            self._scands = np.zeros((max_results * self.cap, 4), np.int32)
            self._scand_n = max_results
        res, kept, prob = self._sres, self._skept, self._sprob
        n = ctypes.c_int32()
        _check(_lib().sp_stream_poll_sifted(self._h, int(bool(wait)), ctypes.cast(res, ctypes.c_void_p),
                                            self._scands.ctypes.data if with_cands else None, kept.ctypes.data,
                                            prob.ctypes.data, int(max_results), ctypes.byref(n)),
               "sp_stream_poll_sifted")
        out = []
        for i in range(n.value):
            r = res[i]
            self._keep.pop((int(r.beam), int(r.seq)), None)
            nk = min(int(r.kept), self.kept_cap)
            c = (cands_to_numpy(self._scands[i * self.cap:(i + 1) * self.cap], min(int(r.count), self.cap))
                 if with_cands else None)
            k = kept[i * self.kept_cap:i * self.kept_cap + nk].copy().view(CAND_DTYPE).reshape(-1)
            out.append((GulpResult.from_buffer_copy(r), c, k, prob[i * self.kept_cap:i * self.kept_cap + nk].copy()))
        return out

    def pending(self):
        q, f, r = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib().sp_stream_pending(self._h, ctypes.byref(q), ctypes.byref(f), ctypes.byref(r)),
               "sp_stream_pending")
        return int(q.value), int(f.value), int(r.value)

    def drain(self, with_cands: bool = True, sifted: bool = False):
        """Polls (blocking) until nothing is queued or in flight (poll_sifted
        results when ``sifted``)."""
        out = []
        while True:
            out += (self.poll_sifted(wait=True, with_cands=with_cands) if sifted
                    else self.poll(wait=True, with_cands=with_cands))
            q, f, r = self.pending()
            if q == 0 and f == 0 and r == 0:
                return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().sp_stream_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def inject_quantised(d_data, d_signal, bits: int, mu: float, sigma: float, level: float, stream=None):
    """In place: d_data uint8 CUDA tensor, d_signal float32 CUDA tensor of
    the same number of elements (sp_inject_quantised)."""
    assert d_data.numel() == d_signal.numel()
    _check(_lib().sp_inject_quantised(_ptr(d_data), _ptr(d_signal), int(d_data.numel()), int(bits), float(mu),
                                      float(sigma), float(level), _stream(stream)), "sp_inject_quantised")


class SiftParams(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("min_points", ctypes.c_int32), ("snr_min", ctypes.c_float),
                ("dm_min", ctypes.c_float), ("width_max_s", ctypes.c_float)]


SIFT_DEFAULTS = dict(eps=0.5, min_points=5, snr_min=10.0, dm_min=10.0, width_max_s=0.1)


def sift(cands: np.ndarray, dms, widths, tsamp: float, labels: bool = False, **params):
    """sp_sift on a structured candidate array (CAND_DTYPE).  Returns the
    kept cluster peaks sorted by (dm_idx, t), and the per-candidate cluster
    labels when ``labels``."""
    p = dict(SIFT_DEFAULTS)
    p.update(params)
    c = np.ascontiguousarray(cands, dtype=CAND_DTYPE)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    w = _widths(widths)
    out = np.zeros(max(c.size, 1), CAND_DTYPE)
    lab = np.zeros(max(c.size, 1), np.int32)
    n = ctypes.c_int64()
    sp_p = SiftParams(float(p["eps"]), int(p["min_points"]), float(p["snr_min"]), float(p["dm_min"]),
                      float(p["width_max_s"]))
    _check(_lib().sp_sift(c.ctypes.data if c.size else None, c.size, d.ctypes.data, d.size, w.ctypes.data, w.size,
                          float(tsamp), ctypes.byref(sp_p), out.ctypes.data, out.size, ctypes.byref(n),
                          lab.ctypes.data if labels else None), "sp_sift")
    kept = out[:n.value].copy()
    return (kept, lab[:c.size].copy()) if labels else kept


def dmt_shifts(freqs_mhz, nsub: int = CNN_IMG, max_sweep: int = 128) -> np.ndarray:
    """int32 [256][nsub] subband shifts of the DM-time image (sp_dmt_shifts)."""
    f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
    out = np.zeros((CNN_IMG, nsub), np.int32)
    _check(_lib().sp_dmt_shifts(f.ctypes.data, f.size, int(nsub), int(max_sweep), out.ctypes.data), "sp_dmt_shifts")
    return out


def cnn_extract(plan: Plan, d_staged, n_in: int, d_cands, widths, t_in: int = 512, stream=None):
    """Subband dynamic spectra (float32 [ncand][256][t_in] CUDA tensor) of
    candidates (int32 [ncand][4] CUDA tensor of sp_cand records) from a
    staged beam."""
    import torch
    w = _widths(widths)
    n = int(d_cands.shape[0])
    sub = torch.empty((n, CNN_IMG, int(t_in)), dtype=torch.float32, device=d_cands.device)
    _check(_lib().sp_cnn_extract(plan.handle, _ptr(d_staged), staged_pitch(int(n_in)), int(n_in), _ptr(d_cands), n,
                                 w.ctypes.data, w.size, int(t_in), _ptr(sub), _stream(stream)), "sp_cnn_extract")
    return sub


def cnn_features(d_sub, d_shift, d_ft, d_dmt, d_work=None, stream=None):
    """Frequency-time and DM-time images (bf16 [B][256][256] CUDA tensors)
    of subband dynamic spectra d_sub float32 [B][256][t_in]."""
    import torch
    B, S, T = (int(x) for x in d_sub.shape)
    if d_work is None:
        d_work = torch.empty(int(_lib().sp_cnn_features_workspace_bytes(B)), dtype=torch.uint8, device=d_sub.device)
    _check(_lib().sp_cnn_features(_ptr(d_sub), B, S, T, _ptr(d_shift), _ptr(d_ft), _ptr(d_dmt), _ptr(d_work),
                                  int(d_work.numel()), _stream(stream)), "sp_cnn_features")


class Classifier:
    """The two-image CNN (sp_cnn_*): forward, backward, Adam on the GPU."""

    def __init__(self, max_batch: int = 64, seed: int = 0):
        h = ctypes.c_void_p()
        _check(_lib().sp_cnn_create(int(max_batch), int(seed), ctypes.byref(h)), "sp_cnn_create")
        self._h = h
        self.max_batch = int(max_batch)
        self.num_params = int(_lib().sp_cnn_num_params())

    def params(self) -> np.ndarray:
        out = np.empty(self.num_params, np.float32)
        _check(_lib().sp_cnn_get_params(self._h, out.ctypes.data), "sp_cnn_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.num_params
        _check(_lib().sp_cnn_set_params(self._h, p.ctypes.data), "sp_cnn_set_params")

    def grads(self) -> np.ndarray:
        out = np.empty(self.num_params, np.float32)
        _check(_lib().sp_cnn_get_grads(self._h, out.ctypes.data), "sp_cnn_get_grads")
        return out

    def forward(self, d_ft, d_dmt, d_prob, stream=None):
        _check(_lib().sp_cnn_forward(self._h, _ptr(d_ft), _ptr(d_dmt), int(d_ft.shape[0]), _ptr(d_prob),
                                     _stream(stream)), "sp_cnn_forward")

    def backward(self, d_ft, d_dmt, d_labels, stream=None) -> float:
        loss = ctypes.c_float()
        _check(_lib().sp_cnn_backward(self._h, _ptr(d_ft), _ptr(d_dmt), _ptr(d_labels), int(d_ft.shape[0]),
                                      ctypes.byref(loss), _stream(stream)), "sp_cnn_backward")
        return float(loss.value)

    def adam_step(self, lr: float, stream=None):
        _check(_lib().sp_cnn_adam_step(self._h, float(lr), _stream(stream)), "sp_cnn_adam_step")

    def train_step(self, d_ft, d_dmt, d_labels, lr: float, want_loss: bool = False, stream=None):
        loss = ctypes.c_float()
        _check(_lib().sp_cnn_train_step(self._h, _ptr(d_ft), _ptr(d_dmt), _ptr(d_labels), int(d_ft.shape[0]),
                                        float(lr), ctypes.byref(loss) if want_loss else None, _stream(stream)),
               "sp_cnn_train_step")
        return float(loss.value) if want_loss else None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().sp_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def probe_iadd3_rate(iters: int = 4096):
    """(3-input integer adds per SM per clock, SM count) measured on the
    current device (include/spotlight_probe.h)."""
    r = ctypes.c_double()
    n = ctypes.c_int()
    _check(_lib().sp_probe_iadd3_rate(int(iters), ctypes.byref(r), ctypes.byref(n)), "sp_probe_iadd3_rate")
    return float(r.value), int(n.value)
