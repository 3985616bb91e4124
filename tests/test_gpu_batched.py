"""GPU parity of the batched (segmented) sort: every array equals the oracle's
sort of that array on its own; records never cross arrays."""
from __future__ import annotations

import numpy as np
import pytest

import datagen
from gpu_util import from_dev, lib, scratch, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


def _run(recs, offsets, key_bytes, repeat=1):
    import torch
    p = lib()
    n, rw = recs.shape
    d_off = torch.from_numpy(offsets.astype(np.uint64).view(np.int64)).cuda()
    t = scratch(n, rw)
    out = None
    for _ in range(repeat):
        d = to_dev(recs)
        p.raduls_sort_batched(d, t, d_off, offsets.size - 1, rw * 8, key_bytes)
        st = p.raduls_stream_status()
        assert st == 0, f"device status {st}"
        got = from_dev(d, n, rw)
        assert out is None or np.array_equal(out, got)
        out = got
    return out


def _check(oracle_mod, recs, offsets, key_bytes, repeat=1):
    got = _run(recs, offsets, key_bytes, repeat)
    np.testing.assert_array_equal(got, oracle_mod.sort_segments(recs, key_bytes, offsets, threads=8))


def test_workload_sizes_mixed(oracle_mod):
    """1500 arrays, sizes log-uniform on [16, 42324], odd arrays with a fixed top half-key."""
    sizes = datagen.batched_sizes(1500)
    recs, offs = datagen.batched16(sizes=sizes)
    _check(oracle_mod, recs, offs, 8, repeat=2)   # the second call replays the captured graph


def test_every_size_class_and_edges(oracle_mod):
    rng = np.random.default_rng(3)
    sizes = np.array([0, 1, 2, 0, 3, 31, 32, 33, 255, 256, 257, 1000, 4095, 4096, 4097, 8191, 9000,
                      70000, 0, 1, 5, 300001, 2, 2, 2] + list(rng.integers(0, 300, size=600)), dtype=np.int64)
    recs, offs = datagen.batched16(sizes=sizes)
    _check(oracle_mod, recs, offs, 8)


def test_many_tiny_arrays(oracle_mod):
    sizes = np.random.default_rng(4).integers(0, 8, size=20000)
    recs, offs = datagen.batched16(sizes=sizes)
    _check(oracle_mod, recs, offs, 8)


def test_wide_records_and_keys(oracle_mod):
    for rec_bytes, key_bytes in ((32, 16), (24, 8), (8, 8)):
        sizes = np.random.default_rng(rec_bytes).integers(0, 6000, size=120)
        n = int(sizes.sum())
        recs = datagen.random_records(n, rec_bytes, key_bytes, rec_bytes, alphabet=None)
        if rec_bytes == 32:
            recs[:, 0] &= np.uint64(0xFF)          # heavy duplicates in the top word
        offs = np.zeros(sizes.size + 1, dtype=np.uint64)
        np.cumsum(sizes, out=offs[1:])
        _check(oracle_mod, recs, offs, key_bytes)


def test_bad_offsets_are_reported_and_nothing_moves():
    import torch
    p = lib()
    recs = datagen.random_records(1000, 16, 8, 1)
    offs = np.array([0, 600, 300, 1000], dtype=np.uint64)   # decreasing
    d = to_dev(recs)
    t = scratch(1000, 2)
    d_off = torch.from_numpy(offs.view(np.int64)).cuda()
    p.raduls_sort_batched(d, t, d_off, 3, 16, 8)
    assert p.raduls_stream_status() == 1
    np.testing.assert_array_equal(from_dev(d, 1000, 2), recs)


def test_pushed_sub_bins_and_heavy_groups(oracle_mod):
    """Mid-size arrays whose two top varying digits leave groups too large for
    code ranks take the stable split; their sub-bins bigger than one on-chip
    group are pushed back to the persistent kernel's queue and sorted by
    whichever CTA takes them."""
    rng = np.random.default_rng(21)
    sizes = np.array([30000, 500, 25000, 4097, 12, 30001, 40960, 100, 20000], dtype=np.int64)
    recs, offs = datagen.batched16(sizes=sizes)
    k = recs[:, 0].copy()
    for a in range(sizes.size):
        lo, hi = int(offs[a]), int(offs[a + 1])
        if hi - lo < 10000:
            continue
        m = hi - lo
        low = rng.integers(0, 1 << 48, size=m, dtype=np.uint64)
        byte6 = np.where(rng.random(m) < 0.6, 0, rng.integers(1, 256, size=m)).astype(np.uint64)
        k[lo:hi] = (np.uint64(0x11) << np.uint64(56)) | (byte6 << np.uint64(48)) | low
        if a % 2:  # a few exact duplicates as well
            k[lo:lo + 3000] = k[lo]
    recs[:, 0] = k
    _check(oracle_mod, recs, offs, 8, repeat=2)


def test_wide_sizes_reading_prefix(oracle_mod):
    """The second batched reading (sizes log-uniform on [16, 2^20]): its first
    150 arrays, many of them far above the mid-size class."""
    sizes = datagen.batched_sizes_wide()[:150]
    recs, offs = datagen.batched16w(sizes=sizes)
    _check(oracle_mod, recs, offs, 8)


def _heavy_mid_arrays(count=6, size=40_000, seed=5):
    """Mid-size arrays whose keys take only two top-byte values and few values
    below them: their code groups are too big, so the persistent kernel splits
    them stably and pushes the sub-bins back onto its queue."""
    rng = np.random.default_rng(seed)
    recs = np.empty((count * size, 2), dtype=np.uint64)
    recs[:, 0] = (rng.integers(0, 2, count * size).astype(np.uint64) << np.uint64(56)) | \
        rng.integers(0, 1 << 40, count * size, dtype=np.uint64)
    recs[:, 1] = np.arange(count * size, dtype=np.uint64)
    offs = np.arange(count + 1, dtype=np.uint64) * np.uint64(size)
    return recs, offs


def test_queue_wait_timeout_is_reported_and_context_survives(oracle_mod):
    """A host-side switch withholds the ready flag of the first item the
    persistent kernel pushes back: the CTA that takes its queue slot waits for
    it, the bounded wait runs out, the call reports RADULS_ERR_TIMEOUT, and the
    next batched call on the same context is correct."""
    import torch
    p = lib()
    recs, offs = _heavy_mid_arrays()
    n = recs.shape[0]
    d_off = torch.from_numpy(offs.view(np.int64)).cuda()
    t = scratch(n, 2)
    p.raduls_set_wait_limit_ns(200_000_000)
    try:
        p.raduls_debug_inject(2, 0)
        d = to_dev(recs)
        p.raduls_sort_batched(d, t, d_off, offs.size - 1, 16, 8)
        assert p.raduls_stream_status() == 6
        assert p.raduls_stream_status() == 0
    finally:
        p.raduls_debug_inject(0, 0)
        p.raduls_set_wait_limit_ns(2_000_000_000)
    d = to_dev(recs)
    p.raduls_sort_batched(d, t, d_off, offs.size - 1, 16, 8)
    assert p.raduls_stream_status() == 0
    np.testing.assert_array_equal(from_dev(d, n, 2), oracle_mod.sort_segments(recs, 8, offs, threads=8))
