"""GPU parity of the key-index sort with one gather (wide records) and of the
distinct keys with counts of sorted records, against the CPU oracle: the
oracle's sort for the first, and for the second the oracle's sorted records
with their runs of equal keys counted on the CPU."""
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


@pytest.mark.parametrize("rec_bytes,key_bytes", [(40, 8), (64, 8), (64, 16), (256, 16), (256, 32), (24, 8), (8, 8)])
@pytest.mark.parametrize("n", [0, 1, 2, 4097, 300_001])
def test_indexed_sort_matches_oracle(oracle_mod, rec_bytes, key_bytes, n):
    if n > 100_000 and rec_bytes == 256 and key_bytes == 32:
        pytest.skip("large case on the other shapes")
    p = lib()
    for alphabet in (None, 3):
        recs = datagen.random_records(n, rec_bytes, key_bytes, n + rec_bytes + key_bytes, alphabet=alphabet)
        d = to_dev(recs)
        t = scratch(n, rec_bytes // 8)
        p.raduls_sort_indexed(d, t, n, rec_bytes, key_bytes)
        assert p.raduls_stream_status() == 0
        np.testing.assert_array_equal(from_dev(d, n, rec_bytes // 8), oracle_mod.sort(recs, key_bytes, threads=8),
                                      err_msg=f"n={n} shape={rec_bytes},{key_bytes} alphabet={alphabet}")


def _runs(keys: np.ndarray):
    """Runs of equal adjacent key rows: (distinct keys, lengths), by a plain loop over boundaries."""
    if keys.shape[0] == 0:
        return keys[:0], np.zeros(0, dtype=np.uint64)
    change = np.any(keys[1:] != keys[:-1], axis=1)
    starts = np.concatenate([[0], np.flatnonzero(change) + 1])
    ends = np.concatenate([starts[1:], [keys.shape[0]]])
    return keys[starts], (ends - starts).astype(np.uint64)


@pytest.mark.parametrize("rec_bytes,key_bytes", [(16, 8), (32, 16), (8, 8), (40, 32)])
@pytest.mark.parametrize("n", [0, 1, 2, 5000, 4096 * 3 + 17, 1_000_003])
def test_unique_counts_of_sorted_records(oracle_mod, rec_bytes, key_bytes, n):
    import torch
    p = lib()
    recs = datagen.random_records(n, rec_bytes, key_bytes, n + 7, alphabet=4)
    srt = oracle_mod.sort(recs, key_bytes, threads=8)
    kw = key_bytes // 8
    d = to_dev(srt)
    keys = torch.zeros(max(n, 1) * kw, dtype=torch.int64, device="cuda")
    counts = torch.zeros(max(n, 1), dtype=torch.int64, device="cuda")
    nu = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    p.raduls_unique_counts(d, n, rec_bytes, key_bytes, keys, counts, nu)
    assert p.raduls_stream_status() == 0
    want_keys, want_counts = _runs(srt[:, :kw])
    m = int(nu.item())
    assert m == want_keys.shape[0]
    np.testing.assert_array_equal(keys[: m * kw].cpu().numpy().view(np.uint64).reshape(m, kw), want_keys)
    np.testing.assert_array_equal(counts[:m].cpu().numpy().view(np.uint64), want_counts)
    assert int(want_counts.sum()) == n


def test_sort_then_count_kmers(oracle_mod):
    """The counting use: 16-byte keys with heavy repeats (k-mer-like), sorted
    on the GPU, then counted: every distinct key once, counts summing to n."""
    import torch
    p = lib()
    n = 2_000_000
    rng = np.random.default_rng(3)
    pool = rng.integers(0, 1 << 63, size=(50_000, 2), dtype=np.uint64)
    recs = np.empty((n, 2), dtype=np.uint64)
    recs[:] = pool[rng.zipf(1.3, size=n) % pool.shape[0]]
    d = to_dev(recs)
    t = scratch(n, 2)
    p.raduls_sort(d, t, n, 16, 16)
    keys = torch.zeros(n * 2, dtype=torch.int64, device="cuda")
    counts = torch.zeros(n, dtype=torch.int64, device="cuda")
    nu = torch.zeros(1, dtype=torch.int64, device="cuda")
    p.raduls_unique_counts(d, n, 16, 16, keys, counts, nu)
    assert p.raduls_stream_status() == 0
    want_keys, want_counts = _runs(oracle_mod.sort(recs, 16, threads=8))
    m = int(nu.item())
    assert m == want_keys.shape[0] == np.unique(recs, axis=0).shape[0]
    np.testing.assert_array_equal(counts[:m].cpu().numpy().view(np.uint64), want_counts)
