"""The bench's roofline object from per-class figures (pure host arithmetic):
the dominant class, achieved GB/s and fraction of the peak, the per-launch
DRAM traffic scaled from the ncu figure per record, and the per-class table."""
from __future__ import annotations

import pytest

import bench


def _uniform16_like(steps=2):
    # two steps of 2^31 x 16 B: two distribution launches and one mid-size launch per step
    n, rec = 1 << 31, 16
    kernel_ms = {"scatter": 50.0 * steps, "bucket": 52.5 * steps, "hist": 9.3 * steps, "block": 0.01 * steps}
    cls_bytes = {"scatter": 2 * 2 * n * rec * steps, "bucket": 2 * n * rec * steps, "hist": 2 * n * rec * steps,
                 "block": 0}
    cls_launches = {"scatter": 2 * steps, "bucket": steps, "hist": 2 * steps, "block": steps}
    return n, rec, kernel_ms, cls_bytes, cls_launches


def test_dominant_class_and_fraction():
    n, rec, kms, cb, cl = _uniform16_like()
    r = bench.roofline_of(kms, cb, cl, 2, rec, 6809.3, "measured", 0, 224.0, 1)
    assert r["kernel"] == bench.CLASS_KERNEL["bucket"]              # 52.5 ms per step beats 50.0
    algo = 2 * n * rec                                               # one launch: read + write every record
    assert r["algorithmic_bytes_per_launch"] == algo
    assert r["launch_ms_avg"] == pytest.approx(52.5)
    assert r["achieved"] == pytest.approx(algo / 52.5e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6809.3)
    assert r["traffic"] == pytest.approx(bench.DRAM_BYTES_PER_RECORD["bucket"] * n)
    assert set(r["per_kernel"]) == {"scatter", "bucket", "hist", "block"}
    assert r["per_kernel"]["block"]["gbs"] == 0.0                     # launched, moved nothing
    assert r["per_kernel"]["scatter"]["launches_per_step"] == 2
    assert r["per_kernel"]["scatter"]["gbs"] == pytest.approx(2 * algo / 50e-3 / 1e9)
    assert r["kernel_ms_per_step"]["bucket"] == pytest.approx(52.5)


def test_whole_sort_rate_is_per_rank():
    n, rec, kms, cb, cl = _uniform16_like(steps=1)
    total = 5 * n * rec
    r1 = bench.roofline_of(kms, cb, cl, 1, rec, 6809.3, "measured", total, 112.0, 1)
    r2 = bench.roofline_of(kms, cb, cl, 1, rec, 6809.3, "measured", 2 * total, 112.0, 2)
    assert r1["whole_sort_gbs"] == pytest.approx(total / 0.112 / 1e9)
    assert r2["whole_sort_gbs"] == pytest.approx(r1["whole_sort_gbs"])


def test_no_timings_gives_no_rate():
    r = bench.roofline_of({}, {c: 0 for c in bench.CLASS_BYTES}, {c: 0 for c in bench.CLASS_BYTES}, 1, 16,
                          6809.3, "fallback", 0, 0.0, 1)
    assert r["achieved"] is None and r["frac"] is None and r["traffic"] is None
    assert r["per_kernel"] == {}
