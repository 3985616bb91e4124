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


def test_bucket_map_is_monotone_and_in_range():
    keys, ko, kx, th = _problem(2)
    n = 10_000
    root = np.zeros(256, dtype=np.int64)
    root[[0, 3, 200]] = [6000, 1000, 3000]
    probes = np.sort(np.concatenate([
        keys,
        keys + np.uint64(1),
        keys - np.uint64(1),
        np.array([0, 2 ** 64 - 1, (3 << 56), (3 << 56) - 1, (200 << 56) + 5], dtype=np.uint64),
    ]))
    # keep probes whose segment has records (the map is defined for present segments)
    j, _ = L.split_keys(probes)
    probes = probes[root[j] > 0]
    b = L.bucket_of(probes, root, n, 12, ko, kx, th)
    assert np.all(np.diff(b) >= 0)
    assert b.min() >= 0 and b.max() < (1 << 12)


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

