"""Pins of the CPU fp64 reference of the learned partitioner.

The analytic gradient is checked against central finite differences of the
forward loss (independent of the gradient formula), the loss against
closed-form cases, the bucket map against monotonicity, and a planted mistake
in a copy of the gradient formula must be caught by the finite-difference
check.
"""
from __future__ import annotations

import numpy as np

from oracle import learned_ref as L


def _problem(seed=0, segs=(0, 3, 200), per_seg=(40, 7, 25), knots=(5, 2, 4)):
    rng = np.random.default_rng(seed)
    keys = []
    knot_off = np.zeros(257, dtype=np.int64)
    m_of = np.full(256, 2, dtype=np.int64)
    for s, cnt, m in zip(segs, per_seg, knots):
        t = rng.beta(0.7, 2.5, size=cnt)            # skewed inside the segment
        low = np.floor(t * 2.0 ** 56).astype(np.uint64)
        keys.append((np.uint64(s) << np.uint64(56)) | low)
        m_of[s] = m
    keys = np.sort(np.concatenate(keys))
    knot_off[1:] = np.cumsum(m_of)
    knot_x = np.zeros(int(knot_off[-1]))
    j_all, t_all = L.split_keys(keys)
    for j in range(256):
        a, b = int(knot_off[j]), int(knot_off[j + 1])
        tj = t_all[j_all == j]
        if tj.size == 0:
            knot_x[a:b] = np.linspace(0.0, 1.0, b - a)
        else:
            q = np.linspace(0, tj.size - 1, b - a).round().astype(int)
            knot_x[a:b] = np.sort(tj)[q]
    theta = rng.normal(0.3, 0.8, size=int(knot_off[-1]) - 256)
    return keys, knot_off, knot_x, theta


def _fd_grad(fn, theta, eps=1e-6):
    g = np.zeros_like(theta)
    for k in range(theta.size):
        tp = theta.copy()
        tm = theta.copy()
        tp[k] += eps
        tm[k] -= eps
        g[k] = (fn(tp) - fn(tm)) / (2 * eps)
    return g


def test_gradient_matches_finite_differences():
    for seed in range(3):
        keys, ko, kx, th = _problem(seed)
        loss, g = L.loss_and_grad(keys, ko, kx, th)
        fd = _fd_grad(lambda t: L.loss_only(keys, ko, kx, t), th)
        assert abs(loss - L.loss_only(keys, ko, kx, th)) < 1e-14
        np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-9)
        assert np.abs(g).max() > 1e-6          # the check is not vacuous


def test_planted_gradient_mistake_is_caught():
    """A copy of the gradient with the '- u' term dropped must fail the FD check."""
    keys, ko, kx, th = _problem(1)

    def wrong_grad(theta):
        j_all, t_all = L.split_keys(keys)
        S = keys.size
        cnt = np.bincount(j_all, minlength=256)
        start = np.concatenate([[0], np.cumsum(cnt)])
        grad = np.zeros_like(theta)
        for j in range(256):
            a, b = int(ko[j]), int(ko[j + 1])
            m = b - a
            pa = a - j
            if cnt[j] == 0:
                continue
            h = L.heights(theta[pa: pa + m - 1])
            tot = L.softplus(theta[pa: pa + m - 1]).sum()
            sg = L.sigmoid(theta[pa: pa + m - 1])
            for r in range(int(cnt[j])):
                u, i, lam = L.leaf_u(t_all[start[j] + r], kx[a:b], h)
                if i < 0:
                    continue
                ind = (np.arange(m - 1) < i).astype(float)
                ind[i] += lam
                grad[pa: pa + m - 1] += 2 * (u - (r + 0.5) / cnt[j]) * sg / tot * ind   # '- u' dropped
        return grad / S

    fd = _fd_grad(lambda t: L.loss_only(keys, ko, kx, t), th)
    assert not np.allclose(wrong_grad(th), fd, rtol=1e-4, atol=1e-8)


def test_two_knot_segment_is_the_identity_and_has_no_gradient():
    """m = 2 with knots {0, 1}: u(t) = t; a sample at the exact mid-quantiles has zero loss."""
    s = 17
    ranks = np.arange(s)
    t = (ranks + 0.5) / s
    keys = (np.uint64(9) << np.uint64(56)) | np.floor(t * 2.0 ** 56).astype(np.uint64)
    ko = np.zeros(257, dtype=np.int64)
    ko[1:] = np.cumsum(np.full(256, 2))
    kx = np.tile([0.0, 1.0], 256)
    th = np.zeros(256)
    loss, g = L.loss_and_grad(keys, ko, kx, th)
    assert loss < 1e-13          # only t's single-precision rounding remains
    assert np.all(g == 0)


def test_heights_are_monotone_and_normalised():
    rng = np.random.default_rng(5)
    for m in (2, 3, 9):
        h = L.heights(rng.normal(0, 5, size=m - 1))
        assert h[0] == 0.0 and h[-1] == 1.0
        assert np.all(np.diff(h) >= 0)


SEG = [("base", "<u8"), ("x0", "<f4"), ("inv_w", "<f4"), ("koff", "<u4"), ("m", "<u4"), ("poff", "<u4"),
       ("sh", "<u4")]


def _model(segs):
    """Model tables from {j: (base, sh, stage-1 heights, stage-2 heights)}; other
    segments get two knots at heights 0 and 1 in both stages."""
    seg = np.zeros((2, 256), dtype=SEG)
    h = []
    for stage in range(2):
        for j in range(256):
            base, sh, h1, h2 = segs.get(j, (0, 56, [0.0, 1.0], [0.0, 1.0]))
            hs = h1 if stage == 0 else h2
            seg[stage]["koff"][j] = len(h)
            seg[stage]["m"][j] = len(hs)
            if stage == 0:
                seg[0]["base"][j], seg[0]["sh"][j] = base, sh
            else:
                seg[1]["inv_w"][j] = float(len(hs) - 1)
            h.extend(hs)
    return seg, np.asarray(h, dtype=np.float32)


def test_u64_to_f32_rounds_to_nearest_even():
    assert L.u64_to_f32((1 << 24) + 1) == float(1 << 24)          # tie -> even (down)
    assert L.u64_to_f32((1 << 24) + 3) == float((1 << 24) + 4)    # tie -> even (up)
    assert L.u64_to_f32((1 << 24) + 2) == float((1 << 24) + 2)    # exact
    rng = np.random.default_rng(1)
    for bits in (20, 25, 33, 40, 56, 63):
        for x in rng.integers(0, 1 << bits, size=200, dtype=np.uint64).tolist():
            f = L.u64_to_f32(x)
            # f is a binary32 value and no binary32 value lies closer to x
            assert float(np.float32(f)) == f
            lo = float(np.nextafter(np.float32(f), np.float32(0)))
            hi = float(np.nextafter(np.float32(f), np.float32(np.inf)))
            assert abs(f - x) <= abs(lo - x) and abs(f - x) <= abs(hi - x)


def test_fma32_rounds_once():
    # a*b + c exactly representable in binary64: one rounding to binary32
    rng = np.random.default_rng(2)
    a = rng.random(300).astype(np.float32)
    b = rng.random(300).astype(np.float32)
    c = rng.random(300).astype(np.float32)
    for x, y, z in zip(a.tolist(), b.tolist(), c.tolist()):
        p = x * y                                   # exact: 24 x 24 bits
        s = p + z
        if (s - p) == z and (s - z) == p:          # the binary64 sum is exact
            assert L.fma32(x, y, z) == float(np.float32(s))
    # a case where rounding twice (binary64, then binary32) lands on a tie and
    # goes the wrong way: a*b = 2^-24 + r 2^-71 with 0 < r < 2^17, c = 1
    q = (1 << 24) - 1
    while True:
        pa = -(-(1 << 47) // q)
        r = pa * q - (1 << 47)
        if pa < (1 << 24) and 0 < r < (1 << 17):
            break
        q -= 1
    x, y = pa * 2.0 ** -36, q * 2.0 ** -35
    assert float(np.float32(x)) == x and float(np.float32(y)) == y
    assert float(np.float32(x * y + 1.0)) == 1.0                  # double rounding: tie to even
    assert L.fma32(x, y, 1.0) == 1.0 + 2.0 ** -23                 # one rounding: above the tie


def test_bucket_map_linear_leaf_is_the_rank_interpolation():
    """Two knots at heights 0, 1 in both stages with a 2^56 knot spacing: the
    leaf is u = fp32(low) / 2^56, so for lows with at most 24 significant bits
    the bucket is floor((C_j + floor(low R_j / 2^56)) B / n)."""
    seg, h = _model({})
    root = np.zeros(256, dtype=np.uint64)
    root[[3, 9, 200]] = [1000, 3000, 6000]
    n, log2b = 10_000, 12
    rng = np.random.default_rng(3)
    keys, want = [], []
    C = np.concatenate([[0], np.cumsum(root.astype(np.int64))])
    for j in (3, 9, 200):
        for low in rng.integers(0, 1 << 24, size=60).tolist():
            low <<= 32
            keys.append((j << 56) | low)
            want.append(((int(C[j]) + (low * int(root[j])) // (1 << 56)) << log2b) // n)
    got = L.bucket_of_model(np.asarray(keys, dtype=np.uint64), root, seg, h, n, log2b)
    np.testing.assert_array_equal(got, want)


def test_bucket_map_knots_ends_and_order():
    """A three-knot stage 1 (heights 0, 0.25, 1, knots 2^40 apart from base
    2^44): keys below the base land at the segment's first position, keys
    past the last knot at its last, the middle knot at a quarter, and the map
    is monotone over random and boundary keys."""
    j = 7
    base, sh = 1 << 44, 40
    seg, h = _model({j: (base, sh, [0.0, 0.25, 1.0], [0.0, 1.0])})
    root = np.zeros(256, dtype=np.uint64)
    root[j] = 1 << 20
    root[8] = 1 << 20
    n, log2b = 1 << 21, 12
    B = 1 << log2b
    k = lambda low: (j << 56) | low
    b = L.bucket_of_model(np.asarray([k(0), k(base - 1), k(base), k(base + (1 << sh)),
                                      k(base + (2 << sh)), k((1 << 56) - 1)], dtype=np.uint64),
                          root, seg, h, n, log2b)
    assert b[0] == 0 and b[1] == 0 and b[2] == 0
    assert b[3] == (((1 << 20) // 4) * B) // n                  # the middle knot: a quarter of the segment
    assert b[4] == b[5] == (((1 << 20) - 1) * B) // n            # past the last knot: the segment's end
    rng = np.random.default_rng(4)
    lows = np.sort(rng.integers(0, 1 << 56, size=400, dtype=np.uint64))
    probes = np.concatenate([np.uint64(j << 56) | lows, np.asarray([8 << 56], dtype=np.uint64)])
    bb = L.bucket_of_model(probes, root, seg, h, n, log2b)
    assert np.all(np.diff(bb) >= 0) and bb.min() >= 0 and bb.max() < B
    assert bb[-1] == ((1 << 20) * B) // n                      # segment 8 starts after segment 7's records


def test_bucket_map_pins_catch_planted_mistakes(monkeypatch):
    """A knot interval off by one, or a dropped segment offset C_j, fails the
    pins above."""
    good = L.stage1_f32

    def off_by_one(key, seg0, h):
        j = key >> 56
        low = key & L.LOW56
        base, sh, m, koff = int(seg0["base"][j]), int(seg0["sh"][j]), int(seg0["m"][j]), int(seg0["koff"][j])
        if low < base:
            return 0.0
        i = ((low - base) >> sh) + 1
        if i >= m - 1:
            return 1.0
        lam = L.f32(L.u64_to_f32((low - base) & ((1 << sh) - 1)) * 2.0 ** -sh)
        return L._interp32(h, koff, i, lam)

    monkeypatch.setattr(L, "stage1_f32", off_by_one)
    import pytest as _pt
    with _pt.raises(AssertionError):
        test_bucket_map_knots_ends_and_order()
    monkeypatch.setattr(L, "stage1_f32", good)
    real = L.bucket_of_model

    def no_offset(keys, root_counts, seg, h, n, log2_buckets):
        r = np.asarray(root_counts, dtype=np.uint64).copy()
        out = []
        for key in np.asarray(keys, dtype=np.uint64).tolist():
            only = np.zeros(256, dtype=np.uint64)
            only[key >> 56] = r[key >> 56]               # C_j = 0: the segment's offset dropped
            out.append(real(np.asarray([key], dtype=np.uint64), only, seg, h, n, log2_buckets)[0])
        return np.asarray(out)

    monkeypatch.setattr(L, "bucket_of_model", no_offset)
    with _pt.raises(AssertionError):
        test_bucket_map_linear_leaf_is_the_rank_interpolation()


def test_second_stage_gradient_matches_finite_differences():
    """Stage 2 takes stage 1's output as its input coordinate."""
    keys, ko, kx, th = _problem(4)
    coords = L.stage_output(keys, ko, kx, th)
    ko2 = ko.copy()
    kx2 = np.concatenate([np.linspace(0.0, 1.0, int(ko[j + 1] - ko[j])) for j in range(256)])
    th2 = np.random.default_rng(9).normal(0.2, 0.7, size=th.size)
    _, g = L.loss_and_grad(keys, ko2, kx2, th2, coords=coords)
    fd = _fd_grad(lambda t: L.loss_only(keys, ko2, kx2, t, coords=coords), th2)
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-9)
    assert np.abs(g).max() > 1e-6


def test_gradient_descent_reduces_loss():
    keys, ko, kx, th = _problem(3)
    l0, _ = L.loss_and_grad(keys, ko, kx, th)
    t = th.copy()
    for _ in range(50):
        _, g = L.loss_and_grad(keys, ko, kx, t)
        t -= 2.0 * g
    l1, _ = L.loss_and_grad(keys, ko, kx, t)
    assert l1 < 0.5 * l0


def test_stage1_coordinate_resolves_the_top_of_a_segment():
    """Keys a few units apart just below 2^63 (the top of segment 0x7F) get
    distinct, exactly spaced stage-1 coordinates: the integer offset keeps
    the last bit, where fp32(key mod 2^56) * 2^-56 would merge 2^32 keys."""
    seg = np.zeros(256, dtype=[("base", "<u8"), ("sh", "<u4")])
    seg["base"][0x7F] = (1 << 56) - (1 << 20)
    seg["sh"][0x7F] = 4
    keys = np.array([(1 << 63) - 1 - 3 * k for k in range(5)][::-1], dtype=np.uint64)
    g = L.stage1_coords(keys, seg)
    assert np.all(np.diff(g) == 3.0 / 16.0)
    assert g[-1] == ((1 << 20) - 1) / 16.0
    _, t = L.split_keys(keys)
    assert np.unique(t).size == 1          # the fp32 coordinate cannot tell them apart
    below = np.array([(0x7F << 56) | 5], dtype=np.uint64)
    assert L.stage1_coords(below, seg)[0] == -1.0

