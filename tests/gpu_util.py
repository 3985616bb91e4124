"""Helpers of the GPU tests: move record arrays between numpy and torch."""
from __future__ import annotations

import numpy as np


def lib():
    import paper_1612_02557_gb300 as p
    p.build_library()
    p.load()
    return p


def to_dev(recs: np.ndarray):
    import torch
    flat = np.ascontiguousarray(recs).view(np.uint8).reshape(-1)
    t = torch.empty(max(flat.size, 16), dtype=torch.uint8, device="cuda")
    if flat.size:
        t[: flat.size].copy_(torch.from_numpy(flat))
    return t


def from_dev(t, n: int, rw: int) -> np.ndarray:
    a = t[: n * rw * 8].cpu().numpy().view(np.uint64)
    return a.reshape(n, rw).copy()


def scratch(n: int, rw: int):
    import torch
    return torch.empty(max(n * rw * 8, 16), dtype=torch.uint8, device="cuda")


def gpu_sort(recs: np.ndarray, key_bytes: int, **kw) -> np.ndarray:
    p = lib()
    n, rw = recs.shape
    d = to_dev(recs)
    t = scratch(n, rw)
    if kw:
        p.raduls_sort_ex(d, t, n, rw * 8, key_bytes, **kw)
    else:
        p.raduls_sort(d, t, n, rw * 8, key_bytes)
    st = p.raduls_stream_status()
    assert st == 0, f"device status {st} ({p.raduls_status_string(st)})"
    return from_dev(d, n, rw)
