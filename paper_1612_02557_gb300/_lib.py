"""ctypes binding of ``libraduls.so`` (argument marshalling only).

Buffers may be given as torch CUDA tensors (any dtype; their bytes are the
records) or as raw integer device addresses.  ``stream`` may be a
``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None for the
current torch stream of the tensors' device (the legacy default stream when
no tensor is given).
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

STATUS = {
    0: "RADULS_OK",
    1: "RADULS_ERR_INVALID_ARG",
    2: "RADULS_ERR_MISALIGNED",
    3: "RADULS_ERR_UNSUPPORTED",
    4: "RADULS_ERR_CUDA",
    5: "RADULS_ERR_OOM",
    6: "RADULS_ERR_TIMEOUT",
    7: "RADULS_ERR_INTERNAL",
}


class RaduLSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where} failed: {STATUS.get(code, code)}")


KERNEL_CLASSES = ["setup", "hist", "plan", "scatter", "copy", "block", "learned", "batched", "bucket"]
N_KERNEL_CLASSES = len(KERNEL_CLASSES)


class Stats(ctypes.Structure):
    _fields_ = [
        ("grid_passes", ctypes.c_uint32),
        ("levels", ctypes.c_uint32),
        ("hist_bytes_read", ctypes.c_uint64),
        ("scatter_bytes", ctypes.c_uint64),
        ("block_bytes", ctypes.c_uint64),
        ("block_items", ctypes.c_uint64),
        ("skipped_digits", ctypes.c_uint64),
        ("learned_used", ctypes.c_uint32),
        ("learned_fell_back", ctypes.c_uint32),
        ("learned_ratio", ctypes.c_float),
        ("gpu_launches", ctypes.c_uint32),
        ("bucket_items", ctypes.c_uint64),
        ("bucket_bytes", ctypes.c_uint64),
        ("kernel_ms", ctypes.c_float * N_KERNEL_CLASSES),
        ("kernel_launches", ctypes.c_uint32 * N_KERNEL_CLASSES),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("kernel_ms", "kernel_launches")}
        d["kernel_ms"] = {KERNEL_CLASSES[i]: float(self.kernel_ms[i]) for i in range(N_KERNEL_CLASSES)}
        d["kernel_launches"] = {KERNEL_CLASSES[i]: int(self.kernel_launches[i]) for i in range(N_KERNEL_CLASSES)}
        return d




class Opts(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_uint32),
        ("learned_log2_buckets", ctypes.c_uint32),
        ("fallback_ratio", ctypes.c_float),
        ("train_steps", ctypes.c_uint32),
        ("stats", ctypes.POINTER(Stats)),
    ]


MODES = {"auto": 0, "plain": 1, "learned": 2}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def build_library(force: bool = False, verbose: bool = False) -> str:
    return _build.build(force=force, verbose=verbose)


def load():
    """Load libraduls.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1612_02557_gb300.build_library() "
                               "(the sorter has no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
        sigs = {
            "raduls_sort": [vp, vp, u64, u32, u32, vp],
            "raduls_sort_ex": [vp, vp, u64, u32, u32, ctypes.POINTER(Opts), vp],
            "raduls_sort_batched": [vp, vp, vp, u32, u32, u32, vp],
            "raduls_sort_indexed": [vp, vp, u64, u32, u32, vp],
            "raduls_unique_counts": [vp, u64, u32, u32, vp, vp, vp, vp],
            "raduls_sort_host": [vp, vp, u64, u32, u32, ctypes.POINTER(Opts), vp],
            "raduls_autotune": [vp, vp, u64, u32, u32, vp, u32, vp, vp],
            "raduls_autotune_reset": [],
            "raduls_histogram": [vp, u64, u32, u32, u32, vp, vp],
            "raduls_histogram_static": [vp, u64, u32, u32, u32, vp, vp],
            "raduls_distribution_pass": [vp, vp, u64, u32, u32, u32, vp],
            "raduls_stream_status": [vp],
            "raduls_debug_inject": [u32, u64],
            "raduls_set_wait_limit_ns": [u64],
        }
        sigs.update({
            "raduls_model_fit": [ctypes.POINTER(ctypes.c_void_p), vp, u64, u32, u32, u32, u32, vp],
            "raduls_model_train": [vp, u32, u32, vp],
            "raduls_model_loss_grad": [vp, u32, ctypes.POINTER(ctypes.c_double), vp, vp],
            "raduls_model_buckets": [vp, vp, u64, vp, vp],
            "raduls_model_sizes": [vp, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32)],
            "raduls_model_copy_out": [vp, vp, vp, vp, vp, vp, vp],
        })
        for name, args in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.raduls_model_free.argtypes = [vp]
        lib.raduls_model_free.restype = None
        lib.raduls_status_string.argtypes = [ctypes.c_int]
        lib.raduls_status_string.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _addr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    dp = getattr(x, "data_ptr", None)
    if dp is None:
        raise TypeError(f"expected a CUDA tensor or a device address, got {type(x)}")
    if not x.is_cuda:
        raise ValueError("buffers must live on a CUDA device")
    if not x.is_contiguous():
        raise ValueError("buffers must be contiguous")
    return int(dp())


def _nbytes(x) -> int | None:
    if isinstance(x, int) or x is None:
        return None
    return x.numel() * x.element_size()


def _stream(stream, *tensors) -> int:
    if stream is None:
        for t in tensors:
            if t is not None and not isinstance(t, int):
                import torch
                return int(torch.cuda.current_stream(t.device).cuda_stream)
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _check_size(x, need: int, name: str):
    nb = _nbytes(x)
    if nb is not None and nb < need:
        raise ValueError(f"{name} holds {nb} bytes, needs {need}")


def _raise(rc: int, where: str):
    if rc != 0:
        raise RaduLSError(rc, where)


def raduls_sort(in_, tmp, n_recs: int, rec_bytes: int, key_bytes: int, stream=None) -> None:
    _check_size(in_, n_recs * rec_bytes, "in")
    _check_size(tmp, n_recs * rec_bytes, "tmp")
    rc = load().raduls_sort(_addr(in_), _addr(tmp), n_recs, rec_bytes, key_bytes, _stream(stream, in_, tmp))
    _raise(rc, "raduls_sort")


def raduls_sort_ex(in_, tmp, n_recs: int, rec_bytes: int, key_bytes: int, mode: str = "auto",
                   learned_log2_buckets: int = 0, fallback_ratio: float = 0.0, train_steps: int = 0,
                   stats: bool = False, stream=None) -> dict | None:
    _check_size(in_, n_recs * rec_bytes, "in")
    _check_size(tmp, n_recs * rec_bytes, "tmp")
    st = Stats()
    o = Opts(MODES[mode], learned_log2_buckets, fallback_ratio, train_steps,
             ctypes.pointer(st) if stats else None)
    rc = load().raduls_sort_ex(_addr(in_), _addr(tmp), n_recs, rec_bytes, key_bytes, ctypes.byref(o),
                               _stream(stream, in_, tmp))
    _raise(rc, "raduls_sort_ex")
    return st.as_dict() if stats else None


def _host_addr(x, writable: bool) -> tuple[int, int]:
    """(address, bytes) of a host buffer: a CPU torch tensor or a numpy array."""
    if hasattr(x, "data_ptr"):
        if x.is_cuda:
            raise ValueError("raduls_sort_host takes host buffers")
        if not x.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return int(x.data_ptr()), int(x.numel() * x.element_size())
    iface = getattr(x, "__array_interface__", None)
    if iface is None:
        raise TypeError(f"expected a CPU tensor or a numpy array, got {type(x)}")
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("buffers must be contiguous")
    if writable and iface["data"][1]:
        raise ValueError("the output buffer must be writable")
    return int(iface["data"][0]), int(x.nbytes)


def raduls_sort_host(h_in, h_out, n_recs: int, rec_bytes: int, key_bytes: int, mode: str = "auto",
                     learned_log2_buckets: int = 0, fallback_ratio: float = 0.0, train_steps: int = 0,
                     stats: bool = False, stream=None) -> dict | None:
    """Sort host records end to end (copy in, sort, copy out) through the C
    ABI; h_out may be h_in.  Ordered on `stream` (default: the current CUDA
    stream): synchronise before reading h_out."""
    a_in, nb_in = _host_addr(h_in, False)
    a_out, nb_out = _host_addr(h_out, True)
    need = n_recs * rec_bytes
    if nb_in < need or nb_out < need:
        raise ValueError(f"host buffers hold {nb_in} and {nb_out} bytes, need {need}")
    st = Stats()
    o = Opts(MODES[mode], learned_log2_buckets, fallback_ratio, train_steps,
             ctypes.pointer(st) if stats else None)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    rc = load().raduls_sort_host(a_in, a_out, n_recs, rec_bytes, key_bytes, ctypes.byref(o), _stream(stream))
    _raise(rc, "raduls_sort_host")
    return st.as_dict() if stats else None


def raduls_sort_batched(in_, tmp, seg_offsets, n_segs: int, rec_bytes: int, key_bytes: int, stream=None) -> None:
    rc = load().raduls_sort_batched(_addr(in_), _addr(tmp), _addr(seg_offsets), n_segs, rec_bytes, key_bytes,
                                    _stream(stream, in_, tmp))
    _raise(rc, "raduls_sort_batched")


def raduls_sort_indexed(in_, tmp, n_recs: int, rec_bytes: int, key_bytes: int, stream=None) -> None:
    """Sort through (key, index) pairs, then one gather of whole records."""
    rc = load().raduls_sort_indexed(_addr(in_), _addr(tmp), n_recs, rec_bytes, key_bytes, _stream(stream, in_, tmp))
    _raise(rc, "raduls_sort_indexed")


def raduls_unique_counts(in_, n_recs: int, rec_bytes: int, key_bytes: int, keys_out, counts_out, n_unique_out,
                         stream=None) -> None:
    """Distinct keys of sorted records with their counts (device outputs)."""
    rc = load().raduls_unique_counts(_addr(in_), n_recs, rec_bytes, key_bytes, _addr(keys_out), _addr(counts_out),
                                     _addr(n_unique_out), _stream(stream, in_))
    _raise(rc, "raduls_unique_counts")


class Tuning(ctypes.Structure):
    _fields_ = [
        ("scatter_variant", ctypes.c_int32),
        ("scatter_tile", ctypes.c_uint32),
        ("block_cap", ctypes.c_uint32),
        ("bucket_max", ctypes.c_uint32),
        ("best_ms", ctypes.c_float),
        ("candidates", ctypes.c_uint32),
        ("digit_bits", ctypes.c_uint32),
        ("leaf", ctypes.c_uint32),
        ("bin_sort", ctypes.c_uint32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def raduls_autotune(in_, tmp, n_recs: int, rec_bytes: int, key_bytes: int, seg_offsets=None, n_segs: int = 0,
                    stream=None) -> dict:
    """Tune launch shapes and size-class thresholds on seeded records written
    into in_ (in_ and tmp are scratch); returns the chosen settings."""
    _check_size(in_, n_recs * rec_bytes, "in")
    _check_size(tmp, n_recs * rec_bytes, "tmp")
    t = Tuning()
    rc = load().raduls_autotune(_addr(in_), _addr(tmp), n_recs, rec_bytes, key_bytes,
                                _addr(seg_offsets) if seg_offsets is not None else None, n_segs,
                                ctypes.byref(t), _stream(stream, in_, tmp))
    _raise(rc, "raduls_autotune")
    return t.as_dict()


def raduls_autotune_reset() -> None:
    _raise(load().raduls_autotune_reset(), "raduls_autotune_reset")


def raduls_histogram(in_, n_recs: int, rec_bytes: int, key_bytes: int, digit: int, hist_out, stream=None) -> None:
    _check_size(in_, n_recs * rec_bytes, "in")
    _check_size(hist_out, 256 * 8, "hist_out")
    rc = load().raduls_histogram(_addr(in_), n_recs, rec_bytes, key_bytes, digit, _addr(hist_out),
                                 _stream(stream, in_))
    _raise(rc, "raduls_histogram")


def raduls_histogram_static(in_, n_recs: int, rec_bytes: int, key_bytes: int, digit: int, hist_out,
                            stream=None) -> None:
    """raduls_histogram() without any allocation (fixed 1 MiB scratch inside the library)."""
    _check_size(in_, n_recs * rec_bytes, "in")
    _check_size(hist_out, 256 * 8, "hist_out")
    rc = load().raduls_histogram_static(_addr(in_), n_recs, rec_bytes, key_bytes, digit, _addr(hist_out),
                                        _stream(stream, in_))
    _raise(rc, "raduls_histogram_static")


def raduls_distribution_pass(in_, out, n_recs: int, rec_bytes: int, key_bytes: int, digit: int,
                             stream=None) -> None:
    _check_size(in_, n_recs * rec_bytes, "in")
    _check_size(out, n_recs * rec_bytes, "out")
    rc = load().raduls_distribution_pass(_addr(in_), _addr(out), n_recs, rec_bytes, key_bytes, digit,
                                         _stream(stream, in_, out))
    _raise(rc, "raduls_distribution_pass")


def raduls_stream_status(stream=None) -> int:
    return int(load().raduls_stream_status(_stream(stream)))


def raduls_status_string(code: int) -> str:
    return load().raduls_status_string(code).decode()


def raduls_debug_inject(kind: int, tile: int = 0) -> None:
    _raise(load().raduls_debug_inject(kind, tile), "raduls_debug_inject")


def raduls_set_wait_limit_ns(ns: int) -> None:
    _raise(load().raduls_set_wait_limit_ns(ns), "raduls_set_wait_limit_ns")


class RaduLSModel:
    """Handle of a learned partition model fitted on the GPU (raduls_model_*)."""

    SEG_DTYPE = [("base", "<u8"), ("x0", "<f4"), ("inv_w", "<f4"), ("koff", "<u4"), ("m", "<u4"),
                 ("poff", "<u4"), ("sh", "<u4")]

    def __init__(self, in_, n_recs: int, rec_bytes: int, key_bytes: int, log2_buckets: int = 16,
                 train_steps: int = 16, stream=None):
        self._lib = load()
        self._h = ctypes.c_void_p()
        rc = self._lib.raduls_model_fit(ctypes.byref(self._h), _addr(in_), n_recs, rec_bytes, key_bytes,
                                        log2_buckets, train_steps, _stream(stream, in_))
        _raise(rc, "raduls_model_fit")
        np_, ns, lb = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _raise(self._lib.raduls_model_sizes(self._h, ctypes.byref(np_), ctypes.byref(ns), ctypes.byref(lb)),
               "raduls_model_sizes")
        self.n_params, self.n_sample, self.log2_buckets = np_.value, ns.value, lb.value

    def train(self, stage: int, steps: int, stream=None) -> None:
        _raise(self._lib.raduls_model_train(self._h, stage, steps, _stream(stream)), "raduls_model_train")

    def loss_grad(self, stage: int, grad_out, stream=None) -> float:
        loss = ctypes.c_double()
        _raise(self._lib.raduls_model_loss_grad(self._h, stage, ctypes.byref(loss), _addr(grad_out),
                                                _stream(stream, grad_out)), "raduls_model_loss_grad")
        return loss.value

    def buckets(self, keys, out, stream=None) -> None:
        n = keys.numel() if hasattr(keys, "numel") else 0
        _raise(self._lib.raduls_model_buckets(self._h, _addr(keys), n, _addr(out), _stream(stream, keys)),
               "raduls_model_buckets")

    def copy_out(self) -> dict:
        import numpy as np
        root = np.zeros(256, dtype=np.uint64)
        seg = np.zeros((2, 256), dtype=self.SEG_DTYPE)
        theta = np.zeros(self.n_params, dtype=np.float32)
        heights = np.zeros(self.n_params, dtype=np.float32)
        sample = np.zeros(self.n_sample, dtype=np.uint64)
        _raise(self._lib.raduls_model_copy_out(self._h, root.ctypes.data, seg.ctypes.data, theta.ctypes.data,
                                               heights.ctypes.data, sample.ctypes.data, None),
               "raduls_model_copy_out")
        return {"root": root, "seg": seg, "theta": theta, "heights": heights, "sample": sample}

    def close(self) -> None:
        if self._h:
            self._lib.raduls_model_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
