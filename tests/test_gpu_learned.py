"""GPU tests of the learned first partition.

* the training kernels' loss and gradient against the CPU fp64 reference
  (oracle/learned_ref.py) on the model's own parameters and sample;
* the bucket map is monotone in the key (exhaustive boundary probes);
* sorts in learned mode, and with the learned partition forced to fall back,
  equal the oracle bit for bit;
* the bucket map, the knot heights and the warm start against the CPU
  reference, exactly for the map (its fp32 steps taken in fp32 on both sides);
* what training gains: the trained model's max/ideal bucket ratio against the
  untrained (linear-leaf) model's, the training loss, and the bytes moved
  against the plain MSD sort on the skewed workload.
"""
from __future__ import annotations

import numpy as np
import pytest

import datagen
from gpu_util import from_dev, gpu_sort, lib, scratch, to_dev
from oracle import learned_ref as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib()


def _model(recs, key_bytes, log2b=12, steps=0):
    p = lib()
    d = to_dev(recs)
    return p.RaduLSModel(d, recs.shape[0], recs.shape[1] * 8, key_bytes, log2_buckets=log2b, train_steps=steps), d


@pytest.mark.parametrize("steps", [0, 5])
def test_gradient_matches_cpu_fp64_reference(steps):
    """Both stages: loss and gradient of the GPU training kernels against the
    CPU fp64 reference on the model's own parameters and sample."""
    import torch
    recs = datagen.skewed16(1 << 14)
    m, _ = _model(recs, 8, 12, steps)
    out = m.copy_out()
    theta = out["theta"].astype(np.float64)
    ko1, kx1, po1 = L.knots_from_segments(out["seg"][0], 0)
    ko2, kx2, po2 = L.knots_from_segments(out["seg"][1], 1)
    coords1 = L.stage1_coords(out["sample"], out["seg"][0])
    coords2 = L.stage_output(out["sample"], ko1, kx1, theta, po1, coords=coords1)
    for stage, (ko, kx, po, coords) in enumerate(((ko1, kx1, po1, coords1), (ko2, kx2, po2, coords2))):
        grad = torch.zeros(m.n_params, dtype=torch.float32, device="cuda")
        loss = m.loss_grad(stage, grad)
        ref_loss, g_ref = L.loss_and_grad(out["sample"], ko, kx, theta, po, coords)
        sel = np.concatenate([np.arange(po[j], po[j] + ko[j + 1] - ko[j] - 1) for j in range(256)])
        g_gpu = grad.cpu().numpy().astype(np.float64)[sel]
        g_ref = g_ref[sel]
        # fp32 arithmetic on the GPU (t, the knot coordinate, lam, stage-1 output) against fp64
        assert abs(loss - ref_loss) <= 1e-4 * abs(ref_loss) + 1e-9, (stage, loss, ref_loss)
        scale = np.abs(g_ref).max()
        assert scale > 0
        np.testing.assert_allclose(g_gpu, g_ref, rtol=2e-3, atol=2e-4 * scale, err_msg=f"stage {stage}")
    m.close()


def test_bucket_map_is_monotone():
    import torch
    recs = datagen.skewed16(1 << 18)
    m, _ = _model(recs, 8, 14, 30)
    out = m.copy_out()
    root = out["root"]
    keys = np.sort(recs[:, 0])
    segs = np.flatnonzero(root > 0).astype(np.uint64)
    probes = np.concatenate([
        keys, keys + np.uint64(1), keys - np.uint64(1),
        segs << np.uint64(56), (segs << np.uint64(56)) | np.uint64((1 << 56) - 1),
        np.array([0, 2 ** 64 - 1], dtype=np.uint64),
    ])
    probes = np.unique(probes)
    dk = torch.from_numpy(probes.view(np.int64)).cuda()
    db = torch.zeros(probes.size, dtype=torch.int32, device="cuda")
    m.buckets(dk, db)
    b = db.cpu().numpy().astype(np.int64)
    assert np.all(np.diff(b) >= 0), "bucket order differs from key order"
    assert b.min() >= 0 and b.max() < (1 << 14)
    m.close()


def _probe_keys(out, recs, rng, n_sample=4000, n_knots=3000):
    """Keys that exercise every branch of the map: sample keys, every stage-1
    knot of a random subset (and one key either side), segment ends."""
    seg0 = out["seg"][0]
    keys = [rng.choice(recs[:, 0], size=n_sample, replace=False)]
    knots = []
    for j in np.flatnonzero(out["root"] > 0).tolist():
        base, sh, m = int(seg0["base"][j]), int(seg0["sh"][j]), int(seg0["m"][j])
        for i in range(m):
            x = base + (i << sh)
            if x <= L.LOW56:
                for d in (-1, 0, 1):
                    if 0 <= x + d <= L.LOW56:
                        knots.append((j << 56) | (x + d))
        knots += [j << 56, (j << 56) | L.LOW56]
    knots = np.asarray(knots, dtype=np.uint64)
    if knots.size > n_knots:
        knots = rng.choice(knots, size=n_knots, replace=False)
    return np.unique(np.concatenate(keys + [knots]))


@pytest.mark.parametrize("name,log2b,steps", [("skewed16", 14, 30), ("widekey32", 12, 16), ("skewed16", 16, 0)])
def test_bucket_map_equals_reference(name, log2b, steps):
    """raduls_model_buckets against the reference map, bucket for bucket: the
    same model (root counts, segment tables, fp32 heights), the map's fp32
    steps taken in fp32 on both sides, the integer steps exact."""
    import torch
    recs = datagen.WORKLOADS[name](1 << 18)
    kb = datagen.KEY_BYTES[name]
    m, _ = _model(recs, kb, log2b, steps)
    out = m.copy_out()
    n = recs.shape[0]
    probes = _probe_keys(out, recs, np.random.default_rng(log2b))
    dk = torch.from_numpy(probes.view(np.int64).copy()).cuda()
    db = torch.zeros(probes.size, dtype=torch.int32, device="cuda")
    m.buckets(dk, db)
    got = db.cpu().numpy().astype(np.int64)
    want = L.bucket_of_model(probes, out["root"], out["seg"], out["heights"], n, log2b)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{bad.size} of {probes.size} buckets differ, first key {probes[bad[0]]:#x}: " \
                          f"GPU {got[bad[0]]}, reference {want[bad[0]]}"
    m.close()


def test_heights_follow_theta():
    """The GPU's fp32 knot heights against the fp64 normalised cumulative
    softplus of its own parameters, segment by segment, both stages."""
    recs = datagen.skewed16(1 << 16)
    m, _ = _model(recs, 8, 12, 8)
    out = m.copy_out()
    for stage in range(2):
        sg = out["seg"][stage]
        for j in np.flatnonzero(sg["m"] > 1).tolist():
            k, mm, pofs = int(sg["koff"][j]), int(sg["m"][j]), int(sg["poff"][j])
            ref = L.heights(out["theta"][pofs:pofs + mm - 1].astype(np.float64))
            np.testing.assert_allclose(out["heights"][k:k + mm], ref, rtol=0, atol=2e-5,
                                       err_msg=f"stage {stage} segment {j}")
    m.close()


def test_warm_start_is_the_sample_cdf_at_the_knots():
    """Warm start only (no Adam steps): every stage's knot heights equal the
    fraction of the segment's sample at or below each knot (increments
    floored at 1e-6 / (m - 1)), computed on the CPU from the model's sample
    and knots; stage 2's input is the reference stage-1 output."""
    recs = datagen.skewed16(1 << 15)
    m, _ = _model(recs, 8, 12, 0x80000000)
    out = m.copy_out()
    for stage in range(2):
        ref = L.warm_heights(out["sample"], out["seg"], stage, out["heights"])
        sg = out["seg"][stage]
        for j, hj in ref.items():
            k, mm = int(sg["koff"][j]), int(sg["m"][j])
            np.testing.assert_allclose(out["heights"][k:k + mm], hj, rtol=0, atol=1e-4,
                                       err_msg=f"stage {stage} segment {j}")
    m.close()


@pytest.mark.parametrize("name,kb", [("skewed16", 8), ("widekey32", 16)])
def test_balance_ratio_matches_reference(name, kb):
    """The learned partition's balance check against a reference computed apart
    from it: the same model (warm start only, so the fit is deterministic) and
    its key sample; the heavy keys are the sample's runs of at least S / B
    equal keys; the buckets of the other sample keys come from
    raduls_model_buckets (pinned to the reference map above); the ratio is the
    largest bucket load over S / B."""
    import torch
    p = lib()
    n = 1 << 21
    recs = datagen.WORKLOADS[name](n)
    rw = recs.shape[1]
    d = to_dev(recs)
    m = p.RaduLSModel(d, n, rw * 8, kb, log2_buckets=10, train_steps=0x80000000)
    sample = m.copy_out()["sample"]
    S = sample.size
    thr = max(2, S >> 10)
    starts = np.concatenate([[0], np.flatnonzero(sample[1:] != sample[:-1]) + 1])
    runs = np.diff(np.concatenate([starts, [S]]))
    heavy = sample[starts[runs >= thr]]
    light = sample[~np.isin(sample, heavy)]
    keys = torch.from_numpy(light.view(np.int64).copy()).cuda()
    b = torch.zeros(light.size, dtype=torch.int32, device="cuda")
    m.buckets(keys, b)
    load = np.bincount(b.cpu().numpy().astype(np.int64), minlength=1024)
    ratio_ref = np.float32(load.max() / (S / 1024))
    t = scratch(n, rw)
    d2 = to_dev(recs)
    st = p.raduls_sort_ex(d2, t, n, rw * 8, kb, mode="learned", learned_log2_buckets=10, train_steps=0x80000000,
                          fallback_ratio=1e9, stats=True)
    assert p.raduls_stream_status() == 0
    assert st["learned_used"] == 1 and st["learned_fell_back"] == 0
    print(f"{name}: ratio {st['learned_ratio']:.3f} (reference {ratio_ref:.3f}), {heavy.size} heavy keys")
    assert np.float32(st["learned_ratio"]) == ratio_ref
    m.close()


def test_one_key_buckets_need_no_more_passes(oracle_mod):
    """Buckets holding a single key value are finished by the learned pass:
    with 20 distinct keys in 2^21 records, nothing is left for another
    distribution pass after it, and the output is the oracle's."""
    p = lib()
    n = 1 << 21
    rng = np.random.default_rng(9)
    vals = np.sort(rng.integers(0, 1 << 63, size=20, dtype=np.uint64))
    recs = np.empty((n, 2), dtype=np.uint64)
    recs[:, 0] = vals[rng.integers(0, 20, n)]
    recs[:, 1] = np.arange(n, dtype=np.uint64)
    d = to_dev(recs)
    t = scratch(n, 2)
    st = p.raduls_sort_ex(d, t, n, 16, 8, mode="learned", fallback_ratio=1e9, stats=True)
    assert p.raduls_stream_status() == 0
    assert st["learned_used"] == 1
    assert st["grid_passes"] == 1 and st["block_items"] == 0 and st["bucket_items"] == 0
    np.testing.assert_array_equal(from_dev(d, n, 2), oracle_mod.sort(recs, 8, threads=8))


@pytest.mark.parametrize("name,n", [("skewed16", 1 << 22), ("widekey32", 1 << 21), ("uniform16", 1 << 21)])
def test_learned_sort_matches_oracle(oracle_mod, name, n):
    recs = datagen.WORKLOADS[name](n)
    kb = datagen.KEY_BYTES[name]
    p = lib()
    d = to_dev(recs)
    t = scratch(n, recs.shape[1])
    st = p.raduls_sort_ex(d, t, n, recs.shape[1] * 8, kb, mode="learned", stats=True)
    assert p.raduls_stream_status() == 0
    assert st["learned_used"] == 1
    np.testing.assert_array_equal(from_dev(d, n, recs.shape[1]), oracle_mod.sort(recs, kb, threads=8))


def test_forced_fallback_gives_the_same_bytes(oracle_mod):
    recs = datagen.skewed16(1 << 21)
    n = recs.shape[0]
    p = lib()
    d = to_dev(recs)
    t = scratch(n, 2)
    st = p.raduls_sort_ex(d, t, n, 16, 8, mode="learned", fallback_ratio=1e-6, stats=True)
    assert p.raduls_stream_status() == 0
    assert st["learned_used"] == 1 and st["learned_fell_back"] == 1
    np.testing.assert_array_equal(from_dev(d, n, 2), oracle_mod.sort(recs, 8, threads=8))


def test_auto_mode_keeps_the_plain_passes(oracle_mod):
    """AUTO takes the plain passes on every input (the learned first partition
    runs only when asked for), and the output is the oracle's."""
    p = lib()
    for name in ("uniform16", "skewed16"):
        recs = datagen.WORKLOADS[name](1 << 20)
        d = to_dev(recs)
        t = scratch(recs.shape[0], 2)
        st = p.raduls_sort_ex(d, t, recs.shape[0], 16, 8, mode="auto", stats=True)
        assert st["learned_used"] == 0, name
        np.testing.assert_array_equal(from_dev(d, recs.shape[0], 2), oracle_mod.sort(recs, 8, threads=8))


def _bucket_ratio(m, keys_dev, log2b):
    import torch
    n = keys_dev.numel()
    b = torch.zeros(n, dtype=torch.int32, device="cuda")
    m.buckets(keys_dev, b)
    cnt = torch.bincount(b.long(), minlength=1 << log2b)
    return float(cnt.max().item()) / (n / (1 << log2b))


def test_training_gain_over_untrained_and_plain():
    """What the fitted network gains over the method without it: its leaves
    balance the buckets far better than the untrained (linear) leaves, and
    the learned sort moves fewer bytes than the plain MSD sort on the skewed
    workload.  The fit is the warm start (the sample's CDF at the knots)
    followed by Adam steps on the mean squared CDF error: the steps must lower
    that training loss; they are not required to improve the bucket balance,
    which is not what they minimise (the measured ratios are printed)."""
    import torch
    p = lib()
    n = 1 << 23
    recs = datagen.skewed16(n)
    # the ratio counts every bucket here, so compare models on the distinct
    # keys (Zipf heavy hitters cannot be split by any key map)
    d = to_dev(recs)
    keys = torch.from_numpy(recs[:, 0].view(np.int64).copy()).cuda()
    distinct = torch.unique(keys)
    untrained = p.RaduLSModel(d, n, 16, 8, log2_buckets=12, train_steps=0)
    warm = p.RaduLSModel(d, n, 16, 8, log2_buckets=12, train_steps=0x80000000)
    trained = p.RaduLSModel(d, n, 16, 8, log2_buckets=12, train_steps=16)
    r_untrained = _bucket_ratio(untrained, distinct, 12)
    r_warm = _bucket_ratio(warm, distinct, 12)
    r_trained = _bucket_ratio(trained, distinct, 12)
    g = torch.zeros(max(warm.n_params, trained.n_params), dtype=torch.float32, device="cuda")
    loss = {name: mdl.loss_grad(1, g) for name, mdl in (("untrained", untrained), ("warm", warm),
                                                       ("trained", trained))}
    print(f"max/ideal over distinct keys: untrained {r_untrained:.2f}, warm start {r_warm:.2f}, "
          f"trained {r_trained:.2f}; leaf loss {loss}")
    assert r_trained < r_untrained / 10
    assert r_warm < r_untrained / 10
    assert loss["warm"] < loss["untrained"] / 2   # the fitted CDF is far closer than the linear leaves
    assert loss["trained"] <= loss["warm"]        # Adam lowers the objective it descends
    warm.close()
    t = scratch(n, 2)
    st_plain = p.raduls_sort_ex(d, t, n, 16, 8, mode="plain", stats=True)
    d2 = to_dev(recs)
    st_learn = p.raduls_sort_ex(d2, t, n, 16, 8, mode="learned", stats=True)
    moved = lambda s: s["hist_bytes_read"] + s["scatter_bytes"] + s["block_bytes"] + s["bucket_bytes"]
    print(f"bytes moved: plain {moved(st_plain) / 2**20:.0f} MiB in {st_plain['grid_passes']} passes, "
          f"learned {moved(st_learn) / 2**20:.0f} MiB in {st_learn['grid_passes']} passes, "
          f"ratio {st_learn['learned_ratio']:.2f}")
    assert st_learn["learned_fell_back"] == 0
    assert moved(st_learn) < moved(st_plain)
    assert np.array_equal(from_dev(d, n, 2), from_dev(d2, n, 2))
    untrained.close()
    trained.close()
