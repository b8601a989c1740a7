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
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspotlight.so")

SP_OK, SP_EINVAL, SP_ESHAPE, SP_ECUDA, SP_EOVERFLOW, SP_ENOMEM, SP_EWORKSPACE, SP_ELIMIT = 0, -1, -2, -3, -4, -5, -6, -7
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
    "sp_probe_iadd3_rate": (ctypes.c_int, [ctypes.c_int, P, P]),
}


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


class Plan:
    """Dedispersion plan: delay table of Eq. 1 (rounded half up) and tiling."""

    def __init__(self, freqs_mhz, tsamp_s: float, dms):
        f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
        d = np.ascontiguousarray(dms, dtype=np.float64)
        h = ctypes.c_void_p()
        _check(_lib().sp_plan_create(f.ctypes.data, f.size, float(tsamp_s), d.ctypes.data, d.size,
                                     ctypes.byref(h)), "sp_plan_create")
        self._h = h
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

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib().sp_searcher_destroy(self._h)
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
