"""Independent checks of a sorted record array (test helpers).

Nothing here shares code with the oracle or with the GPU sorter.  The checks
follow the definition of the sort directly:

* ``brute_force_sort``: Python's own ``sorted`` (guaranteed stable) on the key
  tuple (word 0, word 1, ...) of each record -- the lexicographic order of
  little-endian u64 words, word 0 most significant;
* ``is_sorted``: every adjacent pair of keys is non-decreasing;
* ``multiset_hash``: an order-independent hash of whole records (sum and xor
  of a 64-bit mix of each record), equal for permutations of the same records;
* ``stable_by_payload``: with payload word = input index, equal keys must
  carry increasing payloads.
"""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1


def brute_force_sort(recs: np.ndarray, key_bytes: int) -> np.ndarray:
    kw = key_bytes // 8
    rows = [tuple(int(x) for x in recs[i, :kw]) for i in range(recs.shape[0])]
    order = sorted(range(len(rows)), key=lambda i: rows[i])
    return recs[np.asarray(order, dtype=np.int64)] if order else recs.copy()


def lexsort_sort(recs: np.ndarray, key_bytes: int) -> np.ndarray:
    """numpy lexsort on (index, word W-1, ..., word 0): primary key is word 0,
    the input index breaks ties, so the order is the unique stable one."""
    kw = key_bytes // 8
    n = recs.shape[0]
    keys = [np.arange(n)] + [recs[:, j] for j in range(kw - 1, -1, -1)]
    return recs[np.lexsort(keys)]


def _mix(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def multiset_hash(recs: np.ndarray) -> tuple[int, int]:
    """Order-independent hash of the records: (sum, xor) of per-record mixes."""
    if recs.shape[0] == 0:
        return (0, 0)
    with np.errstate(over="ignore"):
        h = np.zeros(recs.shape[0], dtype=np.uint64)
        for j in range(recs.shape[1]):
            h = _mix(h ^ recs[:, j] ^ np.uint64((j * 0x632BE59BD9B4E019) & M64))
        s = int(np.sum(h, dtype=np.uint64))
        x = int(np.bitwise_xor.reduce(h))
    return (s, x)


def key_cmp_adjacent(recs: np.ndarray, key_bytes: int) -> np.ndarray:
    """For i in [0, n-1): -1/0/+1 comparing key(i) with key(i+1) lexicographically."""
    kw = key_bytes // 8
    n = recs.shape[0]
    res = np.zeros(max(n - 1, 0), dtype=np.int8)
    undecided = np.ones(max(n - 1, 0), dtype=bool)
    for j in range(kw):
        a = recs[:-1, j]
        b = recs[1:, j]
        lt = undecided & (a < b)
        gt = undecided & (a > b)
        res[lt] = -1
        res[gt] = 1
        undecided &= ~(lt | gt)
    return res


def is_sorted(recs: np.ndarray, key_bytes: int) -> bool:
    return bool(np.all(key_cmp_adjacent(recs, key_bytes) <= 0))


def stable_by_payload(recs: np.ndarray, key_bytes: int, payload_word: int | None = None) -> bool:
    kw = key_bytes // 8
    pw = kw if payload_word is None else payload_word
    c = key_cmp_adjacent(recs, key_bytes)
    eq = c == 0
    return bool(np.all(recs[:-1, pw][eq] < recs[1:, pw][eq]))


def check_sorted_output(inp: np.ndarray, out: np.ndarray, key_bytes: int, payload_index: bool) -> None:
    assert out.shape == inp.shape
    assert is_sorted(out, key_bytes), "output not ordered by key"
    assert multiset_hash(out) == multiset_hash(inp), "output is not a permutation of the input records"
    if payload_index:
        assert stable_by_payload(out, key_bytes), "equal keys lost their input order"
