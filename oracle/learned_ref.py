"""CPU fp64 reference of the learned partitioner -- TEST INFRASTRUCTURE ONLY.

The paper has no learned model; this is the reference for the GPU's
monotone two-level piecewise-linear CDF model used for the first scatter on
skewed keys (the GPU kernels share no code with it).  Everything here is
plain numpy in float64, written from the model's definition:

* Root (level 1): the exact histogram R_j of the top byte j of key word 0
  over all records (the first MSD pass's digit histogram, Sec. 1 / Fig. 1),
  with exclusive prefix C_j.
* Leaf (level 2), one per root segment j: two piecewise-linear stages
  u = f2(f1(key)); each stage maps its input through knots (x_i, h_i),
  i = 0..m_j-1.  Stage 1's input is the key's low 56 bits in units of its
  knot spacing, g = (low - base_j) / 2^sh_j (stage1_coords), with knots at
  g = 0, 1, ..., m-1: the GPU model puts them 2^sh_j apart from the
  segment's first sample.  Stage 2's input is f1's output in [0, 1] with
  uniform knots.  knots_from_segments writes the knot positions out.  (The
  generic functions below also accept t = fp32(word0 mod 2^56) * 2^-56 as
  the default input, for synthetic knot layouts.)  The heights are h_0 = 0
  and h_i = sum_{l<i} softplus(theta_l) / sum_l softplus(theta_l), so h is
  non-decreasing and ends at 1 by construction.
* u(t) = 0 for t < x_0, 1 for t >= x_{m-1}, otherwise with i the last knot
  index in [0, m-2] with x_i <= t and lam = (t - x_i) / (x_{i+1} - x_i):
  u = h_i + (h_{i+1} - h_i) * lam.
* Training loss on a sorted sample of S keys: the mean over samples of
  (u_s - F_s)^2 with F_s = (r_s + 0.5) / s_j, r_s the sample's rank inside
  its segment and s_j the segment's sample count; u_s is f1(t_s) when stage 1
  is trained alone and f2(f1(t_s)) for stage 2.
* Analytic gradient: with sigma the logistic function and T_j the segment's
  softplus sum, d u / d theta_l = sigma(theta_l) / T_j * ([l < i] + lam [l == i] - u).

* The bucket map (bucket_of_model) and the warm start (warm_heights) follow
  the GPU model's definition; the map emulates its fp32 steps exactly, since
  an fp32 result decides an integer there.

The pins in tests/test_learned_ref.py check this reference against central
finite differences of its own forward pass, closed-form special cases,
exactly rounded fp32 arithmetic and planted mistakes.
"""
from __future__ import annotations

import numpy as np

T_SCALE = 2.0 ** -56


def softplus(x):
    x = np.asarray(x, dtype=np.float64)
    return np.where(x > 30, x, np.log1p(np.exp(np.minimum(x, 30))))


def sigmoid(x):
    x = np.asarray(x, dtype=np.float64)
    return 1.0 / (1.0 + np.exp(-x))


def split_keys(keys: np.ndarray):
    """(segment j, in-segment coordinate t) of u64 key words.

    The model defines t = fp32(key mod 2^56) * 2^-56: the 56-bit remainder is
    rounded to single precision (round to nearest), then scaled exactly.
    """
    keys = np.asarray(keys, dtype=np.uint64)
    j = (keys >> np.uint64(56)).astype(np.int64)
    t = (keys & np.uint64((1 << 56) - 1)).astype(np.float32).astype(np.float64) * T_SCALE
    return j, t


LOW56 = (1 << 56) - 1


def stage1_coords(keys: np.ndarray, seg) -> np.ndarray:
    """Stage-1 input of each key: g = (low - base_j) / 2^sh_j in float64, with
    low = key mod 2^56 and j its top byte (exact integer difference; -1 below
    the segment's first knot, where the stage's output is 0)."""
    out = np.zeros(len(keys))
    for idx, k in enumerate(np.asarray(keys, dtype=np.uint64).tolist()):
        j = k >> 56
        low, base, sh = k & LOW56, int(seg["base"][j]), int(seg["sh"][j])
        out[idx] = -1.0 if low < base else float(low - base) / float(1 << sh)
    return out


def knots_from_segments(seg, stage: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Explicit knot arrays of one stage of the GPU model, given per segment as
    (base, x0, inv_w, first knot, knots, first parameter, sh): returns
    (knot_off relative to the stage, knot_x, parameter offsets).  Stage 0
    (the first) has its knots at 0, 1, ..., m-1 of the stage1_coords scale;
    stage 1 at x0 + i / inv_w."""
    m = np.asarray(seg["m"], dtype=np.int64)
    off = np.zeros(257, dtype=np.int64)
    off[1:] = np.cumsum(m)
    xs = np.zeros(int(off[-1]))
    for j in range(256):
        i = np.arange(m[j])
        if stage == 0:
            xs[off[j]:off[j + 1]] = i
        else:
            xs[off[j]:off[j + 1]] = float(seg["x0"][j]) + i / float(seg["inv_w"][j])
    return off, xs, np.asarray(seg["poff"], dtype=np.int64)


def heights(theta_seg: np.ndarray) -> np.ndarray:
    """Knot heights of one segment from its m-1 parameters."""
    sp = softplus(theta_seg)
    total = sp.sum()
    h = np.zeros(theta_seg.size + 1)
    h[1:] = np.cumsum(sp) / total
    h[-1] = 1.0
    return h


def leaf_u(t: float, x: np.ndarray, h: np.ndarray):
    """(u, i, lam) of one coordinate; i = -1 outside the knot range."""
    m = x.size
    if t < x[0]:
        return 0.0, -1, 0.0
    if t >= x[m - 1]:
        return 1.0, -1, 0.0
    i = int(np.searchsorted(x[: m - 1], t, side="right") - 1)
    lam = (t - x[i]) / (x[i + 1] - x[i])
    return h[i] + (h[i + 1] - h[i]) * lam, i, lam


def _seg_layout(sample_sorted, knot_off, poff, coords):
    j_all, t_all = split_keys(sample_sorted)
    x_all = t_all if coords is None else np.asarray(coords, dtype=np.float64)
    if poff is None:
        poff = np.asarray(knot_off[:256], dtype=np.int64) - np.arange(256)
    seg_count = np.bincount(j_all, minlength=256)
    seg_start = np.concatenate([[0], np.cumsum(seg_count)])
    return x_all, poff, seg_count, seg_start


def loss_and_grad(sample_sorted: np.ndarray, knot_off: np.ndarray, knot_x: np.ndarray, theta: np.ndarray,
                  poff=None, coords=None):
    """Loss and its analytic gradient w.r.t. theta for one piecewise-linear stage.

    sample_sorted: u64 key words, ascending.  knot_off[j]..knot_off[j+1] are
    segment j's knots in knot_x; segment j's m_j - 1 parameters start at
    theta[poff[j]] (default knot_off[j] - j).  coords: the stage's input per
    sample (default t; the second stage of a leaf takes the first stage's
    output); inside a segment they must be non-decreasing.
    """
    x_all, poff, seg_count, seg_start = _seg_layout(sample_sorted, knot_off, poff, coords)
    S = sample_sorted.size
    grad = np.zeros_like(theta, dtype=np.float64)
    loss = 0.0
    for j in range(256):
        a, b = int(knot_off[j]), int(knot_off[j + 1])
        m = b - a
        pa = int(poff[j])
        th = np.asarray(theta[pa: pa + m - 1], dtype=np.float64)
        x = np.asarray(knot_x[a:b], dtype=np.float64)
        sj = int(seg_count[j])
        if sj == 0:
            continue
        h = heights(th)
        sp_total = softplus(th).sum()
        sg = sigmoid(th)
        for r in range(sj):
            s = seg_start[j] + r
            u, i, lam = leaf_u(x_all[s], x, h)
            F = (r + 0.5) / sj
            e = u - F
            loss += e * e
            if i < 0:
                continue
            ind = (np.arange(m - 1) < i).astype(np.float64)
            ind[i] += lam
            grad[pa: pa + m - 1] += 2.0 * e * sg / sp_total * (ind - u)
    return loss / S, grad / S


def loss_only(sample_sorted, knot_off, knot_x, theta, poff=None, coords=None) -> float:
    x_all, poff, seg_count, seg_start = _seg_layout(sample_sorted, knot_off, poff, coords)
    S = sample_sorted.size
    loss = 0.0
    for j in range(256):
        a, b = int(knot_off[j]), int(knot_off[j + 1])
        m = b - a
        pa = int(poff[j])
        sj = int(seg_count[j])
        if sj == 0:
            continue
        h = heights(np.asarray(theta[pa: pa + m - 1], dtype=np.float64))
        x = np.asarray(knot_x[a:b], dtype=np.float64)
        for r in range(sj):
            u, _, _ = leaf_u(x_all[seg_start[j] + r], x, h)
            loss += (u - (r + 0.5) / sj) ** 2
    return loss / S


def stage_output(sample_sorted, knot_off, knot_x, theta, poff=None, coords=None) -> np.ndarray:
    """Output of one stage for every sample (the next stage's input)."""
    x_all, poff, seg_count, seg_start = _seg_layout(sample_sorted, knot_off, poff, coords)
    j_all, _ = split_keys(sample_sorted)
    out = np.zeros(sample_sorted.size)
    for j in range(256):
        if seg_count[j] == 0:
            continue
        a, b = int(knot_off[j]), int(knot_off[j + 1])
        pa = int(poff[j])
        h = heights(np.asarray(theta[pa: pa + b - a - 1], dtype=np.float64))
        x = np.asarray(knot_x[a:b], dtype=np.float64)
        for s in range(int(seg_start[j]), int(seg_start[j + 1])):
            out[s], _, _ = leaf_u(x_all[s], x, h)
    return out


# ---------------------------------------------------------------- bucket map
#
# The GPU model decides each key's bucket (an integer) with fp32 arithmetic,
# so the reference takes that decision in the same precision: every fp32 step
# of the map is emulated exactly (IEEE binary32, round to nearest even), and
# the final position and bucket are exact integers.  The steps, in order:
#   stage 1: low = key mod 2^56; below base_j -> 0; interval i = (low - base_j)
#            >> sh_j, past the last knot -> 1; lam = rn32(remainder) * 2^-sh_j;
#            u1 = min(max(fma32(h[i+1] - h[i], lam, h[i]), h[i]), h[i+1]);
#   stage 2: g = (u1 - x0) * inv_w (fp32); g <= 0 -> 0; g >= m-1 -> 1;
#            i = min(trunc(g), m-2), lam = g - i, then the same interpolation;
#   root:    uq = floor(u * 2^64) (2^64 - 1 when u >= 1),
#            q = min(floor(uq * R_j / 2^64), R_j - 1), p = C_j + q,
#            b = min(floor(p * B / n), B - 1).
# The heights h are the model's fp32 knot heights (its parameters as the GPU
# holds them); how they follow from theta is checked separately.

def f32(x: float) -> float:
    """Round a double to the nearest binary32 value (ties to even)."""
    return float(np.float32(x))


def _round_exact_to_f32(v) -> float:
    """Round an exact rational (fractions.Fraction) to binary32, ties to even."""
    from fractions import Fraction
    d = float(v)                                   # correctly rounded to binary64
    f = np.float32(d)
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    best = None
    for c in cands:
        if not np.isfinite(c):
            continue
        dist = abs(Fraction(float(c)) - v)
        odd = int(np.array(c, dtype=np.float32).view(np.uint32)) & 1
        key = (dist, odd)
        if best is None or key < best[0]:
            best = (key, float(c))
    return best[1]


def fma32(a: float, b: float, c: float) -> float:
    """fp32 fused multiply-add: a*b + c rounded once to binary32."""
    from fractions import Fraction
    return _round_exact_to_f32(Fraction(a) * Fraction(b) + Fraction(c))


def u64_to_f32(x: int) -> float:
    """Unsigned integer to binary32, round to nearest, ties to even."""
    x = int(x)
    nb = x.bit_length()
    if nb <= 24:
        return float(x)
    sh = nb - 24
    q, r = x >> sh, x & ((1 << sh) - 1)
    half = 1 << (sh - 1)
    if r > half or (r == half and (q & 1)):
        q += 1
    return float(q << sh)


def _interp32(h: np.ndarray, koff: int, i: int, lam: float) -> float:
    h0, h1 = float(h[koff + i]), float(h[koff + i + 1])
    v = fma32(f32(h1 - h0), lam, h0)
    return min(max(v, h0), h1)


def stage1_f32(key: int, seg0, h: np.ndarray) -> float:
    """Stage 1 of the key's segment, as the GPU evaluates it (fp32)."""
    j = key >> 56
    low = key & LOW56
    base, sh, m, koff = int(seg0["base"][j]), int(seg0["sh"][j]), int(seg0["m"][j]), int(seg0["koff"][j])
    if low < base:
        return 0.0
    off = low - base
    i = off >> sh
    if i >= m - 1:
        return 1.0
    lam = f32(u64_to_f32(off & ((1 << sh) - 1)) * 2.0 ** -sh)
    return _interp32(h, koff, i, lam)


def stage2_f32(x: float, j: int, seg1, h: np.ndarray) -> float:
    """Stage 2 of segment j at the stage-1 output x (fp32)."""
    m, koff = int(seg1["m"][j]), int(seg1["koff"][j])
    x0, inv_w = float(seg1["x0"][j]), float(seg1["inv_w"][j])
    g = f32(f32(x - x0) * inv_w)
    if not g > 0.0:
        return 0.0
    if g >= float(m - 1):
        return 1.0
    i = min(int(g), m - 2)
    lam = f32(g - float(i))
    return _interp32(h, koff, i, lam)


def bucket_of_model(keys, root_counts, seg, h, n: int, log2_buckets: int) -> np.ndarray:
    """Bucket of every key word under a fitted model (see the steps above).

    root_counts: R_j, 256 u64; seg: the two stages' segment tables (fields
    base, x0, inv_w, koff, m, sh); h: the fp32 knot heights."""
    R = [int(r) for r in np.asarray(root_counts, dtype=np.uint64)]
    C = [0] * 257
    for j in range(256):
        C[j + 1] = C[j] + R[j]
    B = 1 << log2_buckets
    out = np.zeros(len(keys), dtype=np.int64)
    for idx, k in enumerate(np.asarray(keys, dtype=np.uint64).tolist()):
        j = k >> 56
        u = stage2_f32(stage1_f32(k, seg[0], h), j, seg[1], h)
        r = R[j]
        uq = (1 << 64) - 1 if u >= 1.0 else int(np.floor(u * 2.0 ** 64))
        q = (uq * r) >> 64
        if q >= r:
            q = r - 1 if r else 0
        out[idx] = min(((C[j] + q) * B) // n, B - 1)
    return out


def warm_heights(sample_sorted: np.ndarray, seg, stage: int, h_stage1=None) -> np.ndarray:
    """Warm-start knot heights of one stage, in float64: at every knot the
    fraction of the segment's sample whose stage input lies at or below the
    knot, with each interval's increment floored at 1e-6 / (m - 1) (so the
    heights stay strictly representable by softplus parameters) and the
    result renormalised to end at 1.  Stage 0's input is the key's low 56 bits
    against knots base + i * 2^sh; stage 1's is the stage-1 output (computed
    with h_stage1, the model's fp32 heights) against knots x0 + i / inv_w.
    Returns a dict j -> heights of segment j (non-empty segments only)."""
    keys = np.asarray(sample_sorted, dtype=np.uint64)
    tops = (keys >> np.uint64(56)).astype(np.int64)
    out = {}
    sg = seg[stage]
    for j in range(256):
        sel = np.flatnonzero(tops == j)
        if sel.size == 0:
            continue
        m = int(sg["m"][j])
        if stage == 0:
            low = [int(k) & LOW56 for k in keys[sel].tolist()]
            base, sh = int(sg["base"][j]), int(sg["sh"][j])
            xs = [base + (i << sh) for i in range(m)]
        else:
            low = [stage1_f32(int(k), seg[0], h_stage1) for k in keys[sel].tolist()]
            x0, inv_w = float(sg["x0"][j]), float(sg["inv_w"][j])
            xs = [f32(x0 + f32(float(i) / inv_w)) for i in range(m)]
        low = np.sort(np.asarray(low, dtype=object))
        cdf = np.zeros(m)
        for i in range(1, m - 1):
            cdf[i] = sum(1 for v in low if v <= xs[i]) / sel.size
        cdf[m - 1] = 1.0
        inc = np.maximum(np.diff(cdf), 1e-6 / (m - 1))
        hj = np.zeros(m)
        hj[1:] = np.cumsum(inc) / inc.sum()
        hj[-1] = 1.0
        out[j] = hj
    return out
