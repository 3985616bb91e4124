"""GB300-native stable MSD radix sort of fixed-size records (RADULS method).

Thin Python binding of the C ABI declared in ``include/raduls.h``: every
function here only marshals arguments and calls ``libraduls.so``; all the
sorting runs in the library's CUDA kernels.  PyTorch is used for device
memory and streams only.  There is no CPU fallback: when the library is not
built, every call raises.
"""
from __future__ import annotations

from ._lib import (RaduLSError, RaduLSModel, STATUS, build_library, library_path, load, raduls_autotune,
                   raduls_autotune_reset, raduls_debug_inject, raduls_distribution_pass, raduls_histogram,
                   raduls_histogram_static, raduls_set_wait_limit_ns, raduls_sort, raduls_sort_batched, raduls_sort_ex,
                   raduls_sort_host, raduls_sort_indexed, raduls_status_string, raduls_stream_status,
                   raduls_unique_counts)

__all__ = [
    "RaduLSError",
    "RaduLSModel",
    "STATUS",
    "build_library",
    "library_path",
    "load",
    "raduls_sort",
    "raduls_sort_ex",
    "raduls_sort_batched",
    "raduls_sort_host",
    "raduls_sort_indexed",
    "raduls_unique_counts",
    "raduls_autotune",
    "raduls_autotune_reset",
    "raduls_histogram",
    "raduls_histogram_static",
    "raduls_distribution_pass",
    "raduls_stream_status",
    "raduls_status_string",
    "raduls_debug_inject",
    "raduls_set_wait_limit_ns",
]
