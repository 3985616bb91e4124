"""Parity at the full workload sizes, in the launch configuration bench.py
times (raduls_autotune first, then the workload's modes), checked through
properties that hold at any size and fix the output uniquely:

  * ordered: consecutive records are in key order (unsigned, word 0 first),
    and records with equal keys are in input order (every workload's payload
    carries the record's input index);
  * a permutation of the input: every output record is, word for word, the
    input record its index names, and every index appears exactly once (for
    the batched workload: inside its own array).

An ordered permutation with equal keys in input order is exactly the stable
sort, so these checks are the oracle's definition applied record by record.
"""
from __future__ import annotations

import numpy as np
import pytest

import datagen
from gpu_util import lib

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

CHUNK = 1 << 26  # rows per checking step (bounds the temporaries)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


def _check(out, pristine, kw: int, iw: int, offsets=None):
    """out, pristine: (n, rw) int64 CUDA tensors; kw key words; index in word iw."""
    import torch
    n = out.shape[0]
    dev = out.device
    sign = -(1 << 63)
    seen = torch.zeros(n, dtype=torch.bool, device=dev)
    if offsets is not None:
        offs = torch.from_numpy(offsets.astype(np.int64)).to(dev)
    for a in range(0, n, CHUNK):
        b = min(n, a + CHUNK)
        blk = out[a:b]
        idx = blk[:, iw]
        assert bool(((idx >= 0) & (idx < n)).all()), "index out of range"
        seen[idx] = True
        assert bool((pristine[idx] == blk).all()), f"records {a}..{b} are not the input records they name"
        if offsets is not None:
            pos = torch.arange(a, b, device=dev)
            s_pos = torch.searchsorted(offs, pos, right=True) - 1
            s_idx = torch.searchsorted(offs, idx.contiguous(), right=True) - 1
            assert bool((s_pos == s_idx).all()), "a record left its array"
        # order between row i and row i+1 for i in [a, min(b, n-1))
        e = min(b + 1, n)
        x = out[a:e - 1]
        y = out[a + 1:e]
        lt = torch.zeros(x.shape[0], dtype=torch.bool, device=dev)
        eq = torch.ones(x.shape[0], dtype=torch.bool, device=dev)
        for w in range(kw):
            xw, yw = x[:, w] ^ sign, y[:, w] ^ sign
            lt |= eq & (xw < yw)
            eq &= xw == yw
        ok = lt | (eq & (x[:, iw] < y[:, iw]))
        if offsets is not None:
            brk = offs[1:-1] - 1  # last position of each array but the final one
            brk = brk[(brk >= a) & (brk < e - 1)] - a
            ok[brk] = True
        assert bool(ok.all()), f"order broken in rows {a}..{e}"
    assert bool(seen.all()), "some input index is missing from the output"


def _run(torch, p, host: np.ndarray, kw: int, iw: int, modes, offsets=None):
    rw = host.shape[1]
    n = host.shape[0]
    pristine = torch.from_numpy(host.view(np.int64)).cuda()
    d = torch.empty_like(pristine)
    t = torch.empty_like(pristine)
    if offsets is None:
        p.raduls_autotune(d, t, n, rw * 8, kw * 8)
    else:
        d_off = torch.from_numpy(offsets.view(np.int64)).cuda()
        p.raduls_autotune(d, t, n, rw * 8, kw * 8, d_off, offsets.size - 1)
    torch.cuda.synchronize()
    for mode in modes:
        d.copy_(pristine)
        if mode == "batched":
            p.raduls_sort_batched(d, t, d_off, offsets.size - 1, rw * 8, kw * 8)
        else:
            p.raduls_sort_ex(d, t, n, rw * 8, kw * 8, mode=mode)
        assert p.raduls_stream_status() == 0
        _check(d, pristine, kw, iw, offsets)
    p.raduls_autotune_reset()


def test_uniform16_full():
    """2^31 x 16 B uniform keys, payload = index (generated on the device; the
    bench's workload has the same law)."""
    import torch
    p = lib()
    n = 1 << 31
    g = torch.Generator(device="cuda")
    g.manual_seed(0x52414455)
    pristine = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    pristine[:, 0] = torch.randint(-2**63, 2**63 - 1, (n,), dtype=torch.int64, device="cuda", generator=g)
    pristine[:, 1] = torch.arange(n, dtype=torch.int64, device="cuda")
    d = torch.empty_like(pristine)
    t = torch.empty_like(pristine)
    p.raduls_autotune(d, t, n, 16, 8)
    d.copy_(pristine)
    p.raduls_sort_ex(d, t, n, 16, 8, mode="plain")
    assert p.raduls_stream_status() == 0
    _check(d, pristine, 1, 1)
    p.raduls_autotune_reset()


def test_skewed16_full_learned_and_plain():
    import torch
    _run(torch, lib(), datagen.skewed16(), 1, 1, ("learned", "plain"))


def test_widekey32_full_learned_and_plain():
    import torch
    _run(torch, lib(), datagen.widekey32(), 2, 2, ("learned", "plain"))


def test_batched16_full():
    import torch
    recs, offsets = datagen.batched16()
    _run(torch, lib(), recs, 1, 1, ("batched",), offsets)
