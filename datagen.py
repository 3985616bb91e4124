"""Seeded synthetic record generators for the sorter's workloads.

This module only draws random inputs. It holds none of the sort's arithmetic
(no digit extraction, no ordering, no counting), and both the CPU oracle tests
and the GPU tests/bench draw their inputs from it.

Record model (Sec. 4 of the paper: 16-byte records made of an 8-byte key and
8 bytes of data; 8..32-byte records; 16-byte k-mer keys): a record is
``rec_bytes`` bytes, ``rec_bytes % 8 == 0``; the key is the first
``key_bytes`` bytes, read as ``key_bytes // 8`` little-endian u64 words, word 0
most significant.  Records are returned as a C-contiguous ``uint64`` array of
shape ``(n, rec_bytes // 8)``.

Random streams: every workload uses numpy ``Generator(PCG64(seed))``.  Large
arrays are drawn in fixed chunks of ``CHUNK`` records, chunk ``c`` coming from
``PCG64(seed).jumped(c)``.  For the uniform workloads (and the batched one's
records) each chunk's draws are sequential, so the first ``m`` records do not
depend on ``n``: small inputs are prefixes of the full-size ones.  The
mixtures (``skewed16``, ``widekey32``) draw each chunk's components in
batches whose size depends on how much of the chunk is filled, so a smaller
input is a draw of the same law and seed, not a prefix.

Workloads (sizes are the full ones; tests pass a smaller ``n``):

* ``uniform8``   -- 2^20 records of 8 B, key uniform over all 64-bit values.
* ``uniform16``  -- 2^31 records of 16 B: uniform u64 key, payload = index.
* ``skewed16``   -- 2^30 records of 16 B: per record one of three components
  (probabilities 0.5/0.3/0.2): Zipf(1.1) rank over 2^32 ranks mapped through a
  seeded bijective 64-bit mix; round(Exp(mean 1e12)); 2^63 + round(N(0, 2^40)).
  Payload = index.
* ``batched16``  -- 200,000 arrays of 16 B records, sizes log-uniform on
  [16, U] with U chosen so the expected total is 2^30; keys uniform; every odd
  array has its top 32 key bits fixed to mix(seed, array) >> 32.  Payload =
  index within the whole buffer.
* ``batched16w`` -- the second batched reading: arrays with sizes log-uniform
  on [16, 2^20], drawn until 2^30 records (about 11,400 arrays); keys as in
  ``batched16``.
* ``uniform64``  -- 2^27 records of 64 B: uniform u64 key, payload = index and
  six uniform words (wide records, for the key-index sort).
* ``widekey32``  -- 2^28 records of 32 B: key word 0 is one of 2^20 seeded
  distinct values drawn with Zipf(1.0) frequencies, key word 1 uniform;
  payload = (index, mix(seed, index)).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CHUNK = 1 << 24
MASK64 = (1 << 64) - 1

SEEDS = {
    "uniform8": 0x52414455_00000001,
    "uniform16": 0x52414455_00000002,
    "skewed16": 0x52414455_00000003,
    "batched16": 0x52414455_00000004,
    "widekey32": 0x52414455_00000005,
    "batched16w": 0x52414455_00000006,
    "uniform64": 0x52414455_00000007,
}

FULL_N = {
    "uniform8": 1 << 20,
    "uniform16": 1 << 31,
    "skewed16": 1 << 30,
    "batched16": 1 << 30,   # expected total; the array count is what is fixed
    "widekey32": 1 << 28,
    "uniform64": 1 << 27,
}

REC_BYTES = {"uniform8": 8, "uniform16": 16, "skewed16": 16, "batched16": 16, "widekey32": 32, "uniform64": 64}
KEY_BYTES = {"uniform8": 8, "uniform16": 8, "skewed16": 8, "batched16": 8, "widekey32": 16, "uniform64": 8}

BATCHED_N_ARRAYS = 200_000
BATCHED_MIN = 16


def mix64(x: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) of ``x ^ seed``.

    A bijection on 64-bit integers; used to turn ranks into scattered keys
    and to fill hash payloads.  Pure input scrambling, not sort arithmetic.
    """
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) ^ np.uint64(seed & MASK64)
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def _chunk_rng(seed: int, c: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed).jumped(c))


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _chunked(n: int, seed: int, fill, out: np.ndarray) -> np.ndarray:
    """Run ``fill(rng, lo, hi, out)`` over the fixed chunks, in threads."""
    nchunks = (n + CHUNK - 1) // CHUNK

    def job(c):
        lo = c * CHUNK
        hi = min(n, lo + CHUNK)
        fill(_chunk_rng(seed, c), lo, hi, out)

    if nchunks <= 1:
        for c in range(nchunks):
            job(c)
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(job, range(nchunks)))
    return out


def uniform8(n: int | None = None, seed: int | None = None) -> np.ndarray:
    n = FULL_N["uniform8"] if n is None else n
    seed = SEEDS["uniform8"] if seed is None else seed
    out = np.empty((n, 1), dtype=np.uint64)

    def fill(rng, lo, hi, o):
        o[lo:hi, 0] = rng.bit_generator.random_raw(hi - lo)

    return _chunked(n, seed, fill, out)


def uniform16(n: int | None = None, seed: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    n = FULL_N["uniform16"] if n is None else n
    seed = SEEDS["uniform16"] if seed is None else seed
    if out is None:
        out = np.empty((n, 2), dtype=np.uint64)

    def fill(rng, lo, hi, o):
        o[lo:hi, 0] = rng.bit_generator.random_raw(hi - lo)
        o[lo:hi, 1] = np.arange(lo, hi, dtype=np.uint64)

    return _chunked(n, seed, fill, out)


def uniform64(n: int | None = None, seed: int | None = None) -> np.ndarray:
    """Wide records: 64 B each, a uniform u64 key, the index, then six
    uniform payload words."""
    n = FULL_N["uniform64"] if n is None else n
    seed = SEEDS["uniform64"] if seed is None else seed
    out = np.empty((n, 8), dtype=np.uint64)

    def fill(rng, lo, hi, o):
        o[lo:hi, 0] = rng.bit_generator.random_raw(hi - lo)
        o[lo:hi, 1] = np.arange(lo, hi, dtype=np.uint64)
        o[lo:hi, 2:] = rng.bit_generator.random_raw((hi - lo) * 6).reshape(hi - lo, 6)

    return _chunked(n, seed, fill, out)


ZIPF_S3 = 1.1
ZIPF_RANKS3 = 1 << 32
EXP_MEAN3 = 1e12
NORM_SIGMA3 = float(1 << 40)


def skewed16(n: int | None = None, seed: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """Three-component skewed mixture (Zipf / exponential / normal)."""
    n = FULL_N["skewed16"] if n is None else n
    seed = SEEDS["skewed16"] if seed is None else seed
    if out is None:
        out = np.empty((n, 2), dtype=np.uint64)

    def fill(rng, lo, hi, o):
        m = hi - lo
        comp = rng.choice(3, size=m, p=[0.5, 0.3, 0.2])
        keys = np.empty(m, dtype=np.uint64)
        iz = np.flatnonzero(comp == 0)
        ranks = rng.zipf(ZIPF_S3, size=iz.size).astype(np.uint64)
        bad = ranks > ZIPF_RANKS3
        while bad.any():                       # rejection of ranks beyond 2^32
            ranks[bad] = rng.zipf(ZIPF_S3, size=int(bad.sum())).astype(np.uint64)
            bad = ranks > ZIPF_RANKS3
        keys[iz] = mix64(ranks, seed)
        ie = np.flatnonzero(comp == 1)
        keys[ie] = np.rint(rng.exponential(EXP_MEAN3, size=ie.size)).astype(np.uint64)
        inn = np.flatnonzero(comp == 2)
        dev = np.rint(rng.normal(0.0, NORM_SIGMA3, size=inn.size)).astype(np.int64)
        dev = np.clip(dev, -(1 << 63), (1 << 63) - 1)
        keys[inn] = (dev.view(np.uint64) + np.uint64(1 << 63))  # 2^63 + dev, wraps as int math
        o[lo:hi, 0] = keys
        o[lo:hi, 1] = np.arange(lo, hi, dtype=np.uint64)

    return _chunked(n, seed, fill, out)


def batched_upper(total: float = float(1 << 30), n_arrays: int = BATCHED_N_ARRAYS,
                  lo: float = BATCHED_MIN) -> float:
    """Upper size U of the log-uniform [lo, U] law whose mean times n_arrays is ``total``.

    Mean of a log-uniform variable on [a, b] is (b - a) / ln(b / a); solved by bisection.
    """
    target = total / n_arrays
    a, b = lo * 1.0001, 1e9
    for _ in range(200):
        mid = math.sqrt(a * b)
        mean = (mid - lo) / math.log(mid / lo)
        if mean < target:
            a = mid
        else:
            b = mid
    return math.sqrt(a * b)


def batched_sizes(n_arrays: int = BATCHED_N_ARRAYS, seed: int | None = None,
                  upper: float | None = None) -> np.ndarray:
    seed = SEEDS["batched16"] if seed is None else seed
    upper = batched_upper() if upper is None else upper
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5A5A))
    u = rng.uniform(math.log(BATCHED_MIN), math.log(upper), size=n_arrays)
    return np.floor(np.exp(u)).astype(np.int64)


def batched16(n_arrays: int = BATCHED_N_ARRAYS, seed: int | None = None,
              upper: float | None = None, sizes: np.ndarray | None = None):
    """Returns (records (n, 2) uint64, offsets (n_arrays + 1,) uint64)."""
    seed = SEEDS["batched16"] if seed is None else seed
    if sizes is None:
        sizes = batched_sizes(n_arrays, seed, upper)
    sizes = np.asarray(sizes, dtype=np.int64)
    offsets = np.zeros(sizes.size + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    n = int(offsets[-1])
    out = uniform16(n, seed)
    # fix the top 32 bits of the key for every odd array
    odd = np.arange(1, sizes.size, 2)
    top = (mix64(odd.astype(np.uint64), seed) >> np.uint64(32)) << np.uint64(32)
    lo32 = np.uint64(0xFFFFFFFF)
    for a, t in zip(odd.tolist(), top.tolist()):
        k = out[int(offsets[a]):int(offsets[a + 1]), 0]
        np.bitwise_and(k, lo32, out=k)
        np.bitwise_or(k, np.uint64(t), out=k)
    return out, offsets


BATCHED_WIDE_MAX = 1 << 20
BATCHED_WIDE_TOTAL = 1 << 30


def batched_sizes_wide(seed: int | None = None, total: int = BATCHED_WIDE_TOTAL) -> np.ndarray:
    """Array sizes of the second batched reading: log-uniform on [16, 2^20],
    drawn until their sum first reaches `total` (2^30 records: about 11,400
    arrays, the biggest ones far above the mid-size class)."""
    seed = SEEDS["batched16w"] if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5A5A))
    out, acc = [], 0
    while acc < total:
        u = rng.uniform(math.log(BATCHED_MIN), math.log(BATCHED_WIDE_MAX), size=1024)
        sz = np.floor(np.exp(u)).astype(np.int64)
        cs = acc + np.cumsum(sz)
        k = int(np.searchsorted(cs, total, side="left"))
        if k < sz.size:
            out.append(sz[: k + 1])
            acc = int(cs[k])
            break
        out.append(sz)
        acc = int(cs[-1])
    return np.concatenate(out)


def batched16w(sizes: np.ndarray | None = None, seed: int | None = None):
    """The second batched reading (sizes from batched_sizes_wide), keys drawn
    as in batched16.  Returns (records, offsets)."""
    seed = SEEDS["batched16w"] if seed is None else seed
    if sizes is None:
        sizes = batched_sizes_wide(seed)
    return batched16(seed=seed, sizes=sizes)


ZIPF_S5 = 1.0
DISTINCT5 = 1 << 20


def widekey32(n: int | None = None, seed: int | None = None, out: np.ndarray | None = None) -> np.ndarray:
    """32-byte records, 16-byte key: Zipf(1.0) over 2^20 distinct high words, uniform low word."""
    n = FULL_N["widekey32"] if n is None else n
    seed = SEEDS["widekey32"] if seed is None else seed
    if out is None:
        out = np.empty((n, 4), dtype=np.uint64)
    values = mix64(np.arange(DISTINCT5, dtype=np.uint64), seed ^ 0xC0FFEE)
    h = np.cumsum(1.0 / np.arange(1, DISTINCT5 + 1, dtype=np.float64) ** ZIPF_S5)
    cdf = h / h[-1]

    def fill(rng, lo, hi, o):
        m = hi - lo
        u = rng.random(m)
        rank = np.minimum(np.searchsorted(cdf, u, side="right"), DISTINCT5 - 1)
        o[lo:hi, 0] = values[rank]
        o[lo:hi, 1] = rng.bit_generator.random_raw(m)
        idx = np.arange(lo, hi, dtype=np.uint64)
        o[lo:hi, 2] = idx
        o[lo:hi, 3] = mix64(idx, seed)

    return _chunked(n, seed, fill, out)


def random_records(n: int, rec_bytes: int, key_bytes: int, seed: int,
                   alphabet: int | None = None, payload_index: bool = True) -> np.ndarray:
    """Generic test records: key words uniform (or drawn from a small alphabet of
    byte values to force many duplicates); the first payload word is the index."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rec_bytes // 8
    kw = key_bytes // 8
    out = np.empty((n, w), dtype=np.uint64)
    if alphabet is None:
        out[:, :] = rng.bit_generator.random_raw(n * w).reshape(n, w) if n * w else 0
    else:
        b = rng.integers(0, alphabet, size=(n, w * 8), dtype=np.uint8)
        out[:, :] = b.view(np.uint64).reshape(n, w) if n else 0
        out[:, kw:] = rng.bit_generator.random_raw(n * (w - kw)).reshape(n, w - kw) if n * (w - kw) else 0
    if payload_index and w > kw:
        out[:, kw] = np.arange(n, dtype=np.uint64)
    return out


WORKLOADS = {
    "uniform8": uniform8,
    "uniform16": uniform16,
    "skewed16": skewed16,
    "widekey32": widekey32,
    "uniform64": uniform64,
}
