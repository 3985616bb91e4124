"""CPU oracle for the stable record sort -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The GPU
sorter never calls it and shares no code with it.

``oracle.c`` holds the plain LSD counting sort (Sec. 1 of the paper); this
module compiles it with gcc on first use and wraps it with ctypes.  Records are
numpy ``uint64`` arrays of shape ``(n, rec_bytes // 8)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``oracle/_build/liboracle.so`` (plain -O2 C)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-Wall", "-Wextra", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.c_void_p
            lib.oracle_sort.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_counting_pass.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint32,
                                                 ctypes.c_uint32, ctypes.c_uint32]
            lib.oracle_segmented_counting_pass.argtypes = [u8p, u8p, ctypes.c_uint32, ctypes.c_uint32,
                                                           ctypes.c_uint32, u8p, ctypes.c_uint64]
            lib.oracle_histogram.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, u8p]
            lib.oracle_sort_segments.argtypes = [u8p, u8p, u8p, ctypes.c_uint64, ctypes.c_uint32,
                                                 ctypes.c_uint32, ctypes.c_uint32]
            for f in (lib.oracle_sort, lib.oracle_counting_pass, lib.oracle_segmented_counting_pass,
                      lib.oracle_histogram, lib.oracle_sort_segments):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _recs(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.uint64 or a.ndim != 2:
        raise TypeError("records must be a (n, rec_bytes/8) uint64 array")
    return a


def sort(recs: np.ndarray, key_bytes: int, threads: int = 1) -> np.ndarray:
    """Stable sort of the records by their key (returns a new array)."""
    recs = _recs(recs)
    out = np.empty_like(recs)
    rc = _load().oracle_sort(_ptr(recs), _ptr(out), recs.shape[0], recs.shape[1] * 8, key_bytes, threads)
    if rc:
        raise ValueError(f"oracle_sort failed with code {rc}")
    return out


def counting_pass(recs: np.ndarray, key_bytes: int, digit: int) -> np.ndarray:
    """One stable counting pass on digit ``digit`` (0 = least significant byte of the key)."""
    recs = _recs(recs)
    out = np.empty_like(recs)
    rc = _load().oracle_counting_pass(_ptr(recs), _ptr(out), recs.shape[0], recs.shape[1] * 8,
                                      key_bytes, digit)
    if rc:
        raise ValueError(f"oracle_counting_pass failed with code {rc}")
    return out


def segmented_counting_pass(recs: np.ndarray, key_bytes: int, digit: int,
                            offsets: np.ndarray) -> np.ndarray:
    recs = _recs(recs)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    out = recs.copy()
    rc = _load().oracle_segmented_counting_pass(_ptr(recs), _ptr(out), recs.shape[1] * 8, key_bytes,
                                                digit, _ptr(offsets), offsets.size - 1)
    if rc:
        raise ValueError(f"oracle_segmented_counting_pass failed with code {rc}")
    return out


def histogram(recs: np.ndarray, key_bytes: int, digit: int) -> np.ndarray:
    recs = _recs(recs)
    h = np.zeros(256, dtype=np.uint64)
    rc = _load().oracle_histogram(_ptr(recs), recs.shape[0], recs.shape[1] * 8, key_bytes, digit, _ptr(h))
    if rc:
        raise ValueError(f"oracle_histogram failed with code {rc}")
    return h


def sort_segments(recs: np.ndarray, key_bytes: int, offsets: np.ndarray, threads: int = 1) -> np.ndarray:
    """Sort every segment [offsets[s], offsets[s+1]) on its own."""
    recs = _recs(recs)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    out = recs.copy()
    rc = _load().oracle_sort_segments(_ptr(recs), _ptr(out), _ptr(offsets), offsets.size - 1,
                                      recs.shape[1] * 8, key_bytes, threads)
    if rc:
        raise ValueError(f"oracle_sort_segments failed with code {rc}")
    return out


def usable_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1
