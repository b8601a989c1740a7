"""CPU oracle for the SPOTLIGHT search hot path (test infrastructure only).

This package is the slow, plainly written reference that the CUDA library is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product path never does.  It
shares no code with the CUDA library (``paper_2606_27262_gb300``): the C file
``oracle.c`` restates each formula of arXiv 2606.27262 on its own:

* ``delays``        Sec. 3.1.1, Eq. 1, rounded half up to whole samples.
* ``dedisperse``    Sec. 3.1.1, brute-force shift-and-sum (the DM transform).
* ``moments``       Sec. 3.1.2, per-block count / sum / sum of squares.
* ``boxcar_snr``    Sec. 3.1.2, boxcar matched filter via the cumulative sum.
* ``best``          Sec. 3.1.2, best S/N over the trial widths.
* ``peaks``         Sec. 3.1.2, 3x3 peak filter in the DM-time plane + threshold.
* ``peaks_window``  Sec. 3.1.2, the same with a (2r+1) x (2r+1) window (11 x 11: r = 5).
* ``sift.sift``     Sec. 3.2.1, DBSCAN clustering, cluster peaks, thresholds (numpy).

The shared library is compiled from ``oracle.c`` with gcc on first use
(``-O2 -ffp-contract=off -fopenmp``) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

# Dispersion constant used by the delay reading (MHz^2 pc^-1 cm^3 s).  Eq. 1
# quotes 4.1488064239e3; the search workloads fix the rounded 4.148808e3.
KDM = 4.148808e3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
CFLAGS = ["-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11"]

_lock = threading.Lock()
_lib = None


class Cand(ctypes.Structure):
    _fields_ = [("dm_idx", ctypes.c_int32), ("t", ctypes.c_int32),
                ("width_idx", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("snr", ctypes.c_double)]


CAND_DTYPE = np.dtype([("dm_idx", np.int32), ("t", np.int32), ("width_idx", np.int32),
                       ("pad_", np.int32), ("snr", np.float64)])


def compile_library(src: str = _SRC, out: str = _LIB_PATH, extra_flags=()) -> str:
    """Compile ``src`` into the shared library ``out`` with gcc."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, *extra_flags, src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_delays.argtypes = [P, i32, f64, P, i32, f64, P]
    lib.oracle_delays.restype = ctypes.c_int
    lib.oracle_dedisperse.argtypes = [P, i64, i32, P, i32, i64, P]
    lib.oracle_dedisperse.restype = ctypes.c_int
    lib.oracle_nblocks.argtypes = [i64, i64]
    lib.oracle_nblocks.restype = i64
    lib.oracle_moments.argtypes = [P, i32, i64, i64, P, P, P, P]
    lib.oracle_moments.restype = ctypes.c_int
    lib.oracle_boxcar_snr.argtypes = [P, i32, i64, P, i32, i64, P]
    lib.oracle_boxcar_snr.restype = ctypes.c_int
    lib.oracle_best.argtypes = [P, i32, i64, P, i32, i64, P, P]
    lib.oracle_best.restype = ctypes.c_int
    lib.oracle_peaks.argtypes = [P, P, i32, i64, f64, i32, i32, i32, P, i64]
    lib.oracle_peaks.restype = i64
    lib.oracle_peaks_window.argtypes = [P, P, i32, i64, f64, i32, P, i64]
    lib.oracle_peaks_window.restype = i64
    return lib


def load(path: str | None = None):
    """Load (compiling first if needed) the oracle library; ``path`` loads a
    specific build instead (used by the mutation tests)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if (not os.path.exists(_LIB_PATH)
                    or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
                compile_library()
            _lib = _bind(ctypes.CDLL(_LIB_PATH))
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads(lib=None) -> int:
    return int((lib or load()).oracle_num_threads())


def delays(freqs_mhz, tsamp_s, dms, kdm: float = KDM, lib=None) -> np.ndarray:
    """int32 [ndm][nchan] delays in samples (Eq. 1, rounded half up)."""
    lib = lib or load()
    f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    out = np.empty((d.size, f.size), dtype=np.int32)
    rc = lib.oracle_delays(_p(f), f.size, float(tsamp_s), _p(d), d.size, float(kdm), _p(out))
    if rc != 0:
        raise ValueError("oracle_delays: invalid plan inputs")
    return out


def dedisperse(data: np.ndarray, delay_rows: np.ndarray, n_out: int, lib=None) -> np.ndarray:
    """int32 [nrows][n_out] DM transform of uint8 ``data`` [n_in][nchan]."""
    lib = lib or load()
    x = np.ascontiguousarray(data, dtype=np.uint8)
    dl = np.ascontiguousarray(delay_rows, dtype=np.int32)
    if dl.ndim != 2 or dl.shape[1] != x.shape[1]:
        raise ValueError("delay rows must be [nrows][nchan]")
    out = np.empty((dl.shape[0], int(n_out)), dtype=np.int32)
    rc = lib.oracle_dedisperse(_p(x), x.shape[0], x.shape[1], _p(dl), dl.shape[0], int(n_out), _p(out))
    if rc != 0:
        raise ValueError("oracle_dedisperse: a delayed read falls outside the input")
    return out


def nblocks(n_out: int, norm_block: int, lib=None) -> int:
    return int((lib or load()).oracle_nblocks(int(n_out), int(norm_block)))


def moments(dmt: np.ndarray, norm_block: int, lib=None):
    """(count, sum, sum of squares) [nrows][nblk]: count and sum int64, the
    sum of squares exact Python integers (object array; it is formed in 128
    bits because it can exceed 2^63)."""
    lib = lib or load()
    a = np.ascontiguousarray(dmt, dtype=np.int32)
    nb = nblocks(a.shape[1], norm_block, lib)
    cnt = np.empty((a.shape[0], nb), np.int64)
    sx = np.empty_like(cnt)
    hi = np.empty_like(cnt)
    lo = np.empty((a.shape[0], nb), np.uint64)
    rc = lib.oracle_moments(_p(a), a.shape[0], a.shape[1], int(norm_block), _p(cnt), _p(sx), _p(hi), _p(lo))
    if rc != 0:
        raise ValueError("oracle_moments failed")
    sxx = np.empty((a.shape[0], nb), dtype=object)
    for idx in np.ndindex(sxx.shape):
        sxx[idx] = (int(hi[idx]) << 64) + int(lo[idx])
    return cnt, sx, sxx


def boxcar_snr(dmt: np.ndarray, widths, norm_block: int, lib=None) -> np.ndarray:
    """float64 [nrows][nw][n_out] boxcar S/N (NaN where the window overruns)."""
    lib = lib or load()
    a = np.ascontiguousarray(dmt, dtype=np.int32)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    out = np.empty((a.shape[0], w.size, a.shape[1]), np.float64)
    rc = lib.oracle_boxcar_snr(_p(a), a.shape[0], a.shape[1], _p(w), w.size, int(norm_block), _p(out))
    if rc != 0:
        raise ValueError("oracle_boxcar_snr failed")
    return out


def best(dmt: np.ndarray, widths, norm_block: int, lib=None):
    """(best S/N float64 [nrows][n_out], best width index int32 [nrows][n_out])."""
    lib = lib or load()
    a = np.ascontiguousarray(dmt, dtype=np.int32)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    b = np.empty(a.shape, np.float64)
    k = np.empty(a.shape, np.int32)
    rc = lib.oracle_best(_p(a), a.shape[0], a.shape[1], _p(w), w.size, int(norm_block), _p(b), _p(k))
    if rc != 0:
        raise ValueError("oracle_best failed")
    return b, k


def peaks(best_map: np.ndarray, wbest: np.ndarray, thr: float, row0: int = 0,
          emit_lo: int = 0, emit_hi: int | None = None, cap: int = 1 << 20, lib=None):
    """Candidates (structured array: dm_idx, t, width_idx, snr) in (dm, t) order
    and the total count found (may exceed ``cap``)."""
    lib = lib or load()
    b = np.ascontiguousarray(best_map, dtype=np.float64)
    k = np.ascontiguousarray(wbest, dtype=np.int32)
    if emit_hi is None:
        emit_hi = b.shape[0]
    out = np.zeros(int(cap), dtype=CAND_DTYPE)
    n = lib.oracle_peaks(_p(b), _p(k), b.shape[0], b.shape[1], float(thr), int(row0),
                         int(emit_lo), int(emit_hi), _p(out), int(cap))
    return out[: min(n, cap)].copy(), int(n)


def peaks_window(best_map: np.ndarray, wbest: np.ndarray, thr: float, radius: int, cap: int = 1 << 20,
                 lib=None):
    """Candidates of a (2 radius + 1)^2 peak filter over the whole map, in
    (dm, t) order, and the total count (may exceed ``cap``)."""
    lib = lib or load()
    b = np.ascontiguousarray(best_map, dtype=np.float64)
    k = np.ascontiguousarray(wbest, dtype=np.int32)
    out = np.zeros(int(cap), dtype=CAND_DTYPE)
    n = lib.oracle_peaks_window(_p(b), _p(k), b.shape[0], b.shape[1], float(thr), int(radius), _p(out), int(cap))
    if n < 0:
        raise ValueError("oracle_peaks_window: radius must be >= 1")
    return out[: min(n, cap)].copy(), int(n)


def search(data: np.ndarray, delay_rows: np.ndarray, n_out: int, widths, thr: float,
           norm_block: int, lib=None):
    """Whole hot path on the CPU: DM transform, best S/N map, candidates."""
    dmt = dedisperse(data, delay_rows, n_out, lib)
    b, k = best(dmt, widths, norm_block, lib)
    cands, n = peaks(b, k, thr, lib=lib)
    return dmt, b, k, cands, n
