"""Benchmark of the GB300 stable MSD radix sorter (one JSON line on rank 0).

A "step" sorts one batch of synthetic records end to end through the C ABI
(histograms, distribution passes, on-chip bin sorts).  The default workload
is 2^31 records of 16 bytes (uniform u64 key + u64 index payload).  Before
each timed step the input is restored from a pristine device copy (untimed);
the 32 GiB input is far larger than the 129 MB L2, so no step starts warm.

Reported next to records/s:
  * roofline -- the dominant kernel (the class with the most device time per
    step): algorithmic bytes per launch (read + write of every record it
    moves) over its launch time measured live with CUDA events recorded by the
    library on the launching stream, against the measured HBM copy bandwidth;
    every class's figure is listed under roofline.per_kernel;
  * cpu_baseline -- the CPU oracle (LSD counting sort) on a bounded sample of
    the same workload on this host's cores;
  * e2e -- the same metric through the library's host entry point
    (raduls_sort_host: records in pinned host memory, the host->device copy,
    the sort and the device->host copy of the sorted records all inside the
    timed region; batched calls copy with torch around raduls_sort_batched).

``--impl reference`` times the CPU oracle instead (the only reference there
is for this method) on bounded samples of the same workload.
Multi-GPU (torchrun): every rank sorts its own array (replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen  # noqa: E402

METRIC = "sorted records/s and % HBM peak at 1 GB300; plain vs learned/batched, bit-exact"


def job_time_ms(local_ms: float, dist=None, device: str = "cuda") -> float:
    """Whole-job time of a timed region: the slowest rank's own time (every
    rank timed the same steps between barriers)."""
    if dist is None:
        return local_ms
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(records_per_rank: int, world: int, steps: int, job_ms: float) -> float:
    """Whole-job throughput: the records every rank sorted over the job time."""
    return records_per_rank * world * steps / (job_ms / 1e3)


UNIT = "records/s"

WORKLOADS = {
    "uniform16": dict(desc="2^31 records x 16 B (u64 key uniform over 2^64 + u64 index payload), plain MSD sort",
                      n=1 << 31, rec=16, key=8, mode="plain"),
    "uniform8": dict(desc="2^20 records x 8 B (u64 key only, uniform), plain MSD sort", n=1 << 20, rec=8, key=8,
                     mode="plain"),
    "skewed16": dict(desc="2^30 records x 16 B, Zipf(1.1)/exponential/normal key mixture; learned first "
                          "partition (plain MSD timed alongside)", n=1 << 30, rec=16, key=8, mode="learned"),
    "widekey32": dict(desc="2^28 records x 32 B, 16-byte key (Zipf(1.0) high word over 2^20 values, uniform low "
                           "word); learned first partition (plain MSD timed alongside)", n=1 << 28, rec=32, key=16,
                      mode="learned"),
    "batched16": dict(desc="200,000 arrays of 16 B records, sizes log-uniform on [16, 42324] (expected total "
                           "2^30), odd arrays with a fixed top half-key; one batched call (a per-array plain loop "
                           "on a prefix of the arrays timed alongside)", n=0, rec=16, key=8, mode="batched"),
    "batched16w": dict(desc="about 11,400 arrays of 16 B records, sizes log-uniform on [16, 2^20] drawn until 2^30 "
                            "records, odd arrays with a fixed top half-key; one batched call (a per-array plain loop "
                            "timed alongside)", n=0, rec=16, key=8, mode="batched"),
    "uniform64": dict(desc="2^27 records x 64 B (u64 key uniform, index, six payload words); key-index sort with one "
                           "gather (the direct record sort timed alongside)", n=1 << 27, rec=64, key=8,
                      mode="indexed"),
}

# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per record
# moved, per kernel class, from one capture of the current kernels on uniform
# 16-byte records.  A class missing here has no capture of its current code.
DRAM_BYTES_PER_RECORD = {
    # wscatter_kernel, a 2^27-record sort split 10 bits (variant 11) then 9 bits (variant 9)
    "scatter": (2.605462e9 + 2.451761e9 + 2.291758e9 + 2.199927e9) / 2 / 2 ** 27,
    # bin_sort_kernel, 2^27 records in ~2,048-record bins
    "block": (2.151157e9 + 2.090265e9) / 2 ** 27,
    # bucket_kernel, 10^7 records in 256 mid-size bins
    "bucket": (565.243136e6 + 414.964992e6) / 1e7,
}
# stats field holding each class's algorithmic bytes (read + write of every record it moves)
CLASS_BYTES = {"scatter": "scatter_bytes", "bucket": "bucket_bytes", "block": "block_bytes",
               "hist": "hist_bytes_read"}
CLASS_KERNEL = {"scatter": "wscatter_kernel (MSD distribution pass of big bins)",
                "bucket": "bucket_kernel (mid-size bins, one CTA each)",
                "block": "bin_sort_kernel (streamed on-chip sort of small bins; block_sort_kernel takes what it leaves)",
                "hist": "whist_kernel (chunk histograms chained by look-back)"}


def roofline_of(kernel_ms: dict, cls_bytes: dict, cls_launches: dict, steps: int, rec: int, hbm_peak: float,
                peak_kind: str, total_bytes: int, tot_ms: float, world: int) -> dict:
    """The JSON line's roofline object from the library's per-class figures
    summed over the timed steps: per class, algorithmic bytes (read + write
    of every record it moves) over its CUDA-event time; the dominant class
    (most time per step) is the roofline's kernel, its `traffic` the ncu DRAM
    bytes per record moved (DRAM_BYTES_PER_RECORD) times the records a launch
    moves."""
    per_kernel = {}
    for c in CLASS_BYTES:
        ms = kernel_ms.get(c, 0.0)
        if ms > 0 and cls_launches.get(c, 0) > 0:
            gbs = cls_bytes[c] / (ms / 1e3) / 1e9
            per_kernel[c] = {"ms_per_step": ms / steps, "launches_per_step": cls_launches[c] / steps,
                             "gbs": gbs, "frac": gbs / hbm_peak}
    dom = max(per_kernel, key=lambda c: per_kernel[c]["ms_per_step"]) if per_kernel else "scatter"
    dom_ms, dom_launches, dom_bytes = kernel_ms.get(dom, 0.0), cls_launches.get(dom, 0), cls_bytes.get(dom, 0)
    achieved = (dom_bytes / (dom_ms / 1e3)) / 1e9 if dom_ms > 0 else None
    traffic = None
    if dom in DRAM_BYTES_PER_RECORD and dom_launches and dom != "hist":
        traffic = DRAM_BYTES_PER_RECORD[dom] * (dom_bytes / (2 * rec)) / dom_launches
    whole = total_bytes / (tot_ms / 1e3) / 1e9 / world if tot_ms else None
    return {
        "bound": "hbm", "kernel": CLASS_KERNEL[dom],
        "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
        "frac": (achieved / hbm_peak) if achieved else None,
        "traffic": traffic, "peak_kind": f"{peak_kind} copy bandwidth",
        "algorithmic_bytes_per_launch": dom_bytes / max(dom_launches, 1),
        "launch_ms_avg": dom_ms / max(dom_launches, 1),
        "per_kernel": per_kernel,
        "whole_sort_gbs": whole,
        "whole_sort_frac": whole / hbm_peak if whole else None,
        "kernel_ms_per_step": {k: v / steps for k, v in kernel_ms.items() if v > 0},
    }



def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def make_input(name: str, n: int):
    """Pinned host records of the workload (uint64, (n, rec/8)), and the array
    offsets for the batched workload (else None)."""
    import torch
    w = WORKLOADS[name]
    rw = w["rec"] // 8
    offsets = None
    if name == "batched16":
        recs, offsets = datagen.batched16()
        n = recs.shape[0]
    host = torch.empty((n, rw), dtype=torch.int64, pin_memory=True)
    arr = host.numpy().view(np.uint64)
    if name == "batched16":
        arr[:] = recs
        del recs
    elif name == "uniform8":
        arr[:] = datagen.uniform8(n)
    else:
        getattr(datagen, name)(n, out=arr)
    return host, offsets


def _prefix(name: str, m: int):
    """About m leading records of the workload, and for the batched workload
    the offsets of the whole arrays they hold (else None)."""
    if name == "batched16":
        sizes = datagen.batched_sizes()
        cut = int(np.searchsorted(np.cumsum(sizes), m)) + 1
        return datagen.batched16(sizes=sizes[:cut])
    return getattr(datagen, name)(m), None


def _oracle_run(oracle, recs, offs, key, cores):
    if offs is None:
        oracle.sort(recs, key, threads=cores)
    else:
        oracle.sort_segments(recs, key, offs, threads=cores)


def cpu_baseline(name: str, budget_s: float = 15.0) -> dict:
    """The oracle, as it stands, on a bounded sample of the workload (a prefix
    for the uniform and batched workloads, a smaller draw of the same law for
    the mixtures; whole records sorted by the LSD counting sort; for the
    batched workload the sample's arrays sorted one by one)."""
    import oracle
    w = WORKLOADS[name]
    cores = oracle.usable_cores()
    m = min(1 << 22, w["n"] or (1 << 22))  # never more than the workload itself
    recs, offs = _prefix(name, m)
    t0 = time.perf_counter()
    _oracle_run(oracle, recs, offs, w["key"], cores)
    dt = time.perf_counter() - t0
    target = int(m * budget_s / max(dt, 1e-3))
    m2 = max(m, min(1 << 28, w["n"] or (1 << 30), 1 << int(np.log2(max(target, 1)))))
    if m2 > m:
        recs, offs = _prefix(name, m2)
        t0 = time.perf_counter()
        _oracle_run(oracle, recs, offs, w["key"], cores)
        dt = time.perf_counter() - t0
    m = recs.shape[0]
    what = (f"first {m} records of the {name} workload" if name in ("uniform8", "uniform16", "batched16")
            else f"{m} records drawn from the {name} workload's law and seed")
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what} ({w['rec']} B records), one LSD oracle sort with {cores} threads, {dt:.2f} s"}


def run_reference(args, rank: int, world: int) -> None:
    """--impl reference: the CPU oracle timed on bounded samples of the workload."""
    if rank != 0:
        return
    import oracle
    w = WORKLOADS[args.workload]
    cores = oracle.usable_cores()
    m = args.ref_records or (1 << 24)
    recs, offs = _prefix(args.workload, m)
    m = recs.shape[0]
    for _ in range(args.warmup):
        _oracle_run(oracle, recs, offs, w["key"], cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _oracle_run(oracle, recs, offs, w["key"], cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = m * args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "n_records": m, "rec_bytes": w["rec"],
                   "key_bytes": w["key"], "sample": "bounded prefix of the workload, sorted on the host"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {m} records of {args.workload}, LSD oracle, {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def check_sorted_gpu(recs, pristine_keys=None) -> bool:
    """Order + stability check on the device (payload = input index)."""
    import torch
    k = recs[:, 0] ^ (-(1 << 63))
    ok = bool(((k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (recs[1:, 1] > recs[:-1, 1]))).all())
    if pristine_keys is not None:
        ok = ok and bool((pristine_keys[recs[:, 1]] == recs[:, 0]).all())
    return ok


def _timed(fn, stream):
    """Device time (ms) of fn() with CUDA events on `stream`."""
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def _moved(st) -> int:
    return st["hist_bytes_read"] + st["scatter_bytes"] + st["block_bytes"] + st["bucket_bytes"]


def compare_workload(name: str, pkg, steps: int, warmup: int, hbm_peak: float, peak_kind: str) -> dict:
    """One comparison of the metric's second half on a full-size workload:
    the learned (skewed16, widekey32) or batched (batched16) form against the
    plain MSD sort of the same input, each timed with CUDA events, the input
    restored from a pristine device copy before every step (untimed), the
    forms run alternately, and their outputs compared byte for byte."""
    import torch
    w = WORKLOADS[name]
    rec, key, mode = w["rec"], w["key"], w["mode"]
    offsets = None
    if name == "batched16":
        host, offsets = datagen.batched16()
    elif name == "batched16w":
        host, offsets = datagen.batched16w()
    else:
        host = getattr(datagen, name)(w["n"])
    n = host.shape[0]
    pristine = torch.from_numpy(host.view(np.int64)).cuda()
    del host
    recs = torch.empty_like(pristine)
    tmp = torch.empty_like(pristine)
    stream = torch.cuda.current_stream()
    d_off = torch.from_numpy(offsets.view(np.int64)).cuda() if offsets is not None else None
    n_segs = offsets.size - 1 if offsets is not None else 0
    if mode == "batched":
        tuning = pkg.raduls_autotune(recs, tmp, n, rec, key, d_off, n_segs)
    else:
        tuning = pkg.raduls_autotune(recs, tmp, n, rec, key)
    torch.cuda.synchronize()

    def form():
        if mode == "batched":
            pkg.raduls_sort_batched(recs, tmp, d_off, n_segs, rec, key)
            return None
        if mode == "indexed":
            pkg.raduls_sort_indexed(recs, tmp, n, rec, key)
            return None
        return pkg.raduls_sort_ex(recs, tmp, n, rec, key, mode="learned", stats=True)

    def plain():
        if mode == "batched":
            # the plain path on every array, one raduls_sort_ex call each
            for a in range(n_segs):
                s0, s1 = int(offsets[a]), int(offsets[a + 1])
                if s1 - s0 > 1:
                    pkg.raduls_sort_ex(recs[s0:s1], tmp[s0:s1], s1 - s0, rec, key, mode="plain")
            return None
        return pkg.raduls_sort_ex(recs, tmp, n, rec, key, mode="plain", stats=True)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    for _ in range(warmup):
        recs.copy_(pristine)
        form()
        recs.copy_(pristine)
        if mode != "batched":
            plain()
    torch.cuda.synchronize()
    if pkg.raduls_stream_status() != 0:
        raise SystemExit(f"device status during the {name} warm-up")
    f_ms, p_ms, f_st, p_st = [], [], None, None
    for i in range(steps):
        recs.copy_(pristine)
        ms, f_st = _timed(form, stream)
        f_ms.append(ms)
        if mode != "batched":      # alternate the two forms
            recs.copy_(pristine)
            ms, p_st = _timed(plain, stream)
            p_ms.append(ms)
    # the form's output, then (for the batched form, whose per-array loop is
    # long, once) the plain output last, left in recs
    recs.copy_(pristine)
    form()
    f_out = recs.clone()
    recs.copy_(pristine)
    if mode == "batched":
        ms, p_st = _timed(plain, stream)
        p_ms.append(ms)
    else:
        plain()
    clocks = sampler.stop()
    if pkg.raduls_stream_status() != 0:
        raise SystemExit(f"device status during the {name} timed steps")
    identical = bool(torch.equal(f_out, recs))
    ordered = None
    if rec == 16 and key == 8 and mode != "batched":
        ordered = check_sorted_gpu(recs.view(n, 2), pristine.view(n, 2)[:, 0])
    fm, pm = sum(f_ms) / len(f_ms), sum(p_ms) / len(p_ms)
    out = {
        "desc": w["desc"], "n_records": n, "rec_bytes": rec, "key_bytes": key,
        "form": mode, "ms_per_step": fm, "records_per_s": n / (fm / 1e3),
        "ms_steps": [round(x, 2) for x in f_ms],
        "plain_ms_per_step": pm, "plain_records_per_s": n / (pm / 1e3),
        "plain_ms_steps": [round(x, 2) for x in p_ms],
        "speedup_over_plain": pm / fm,
        "identical_output": identical,
        "clocks": clocks, "tuning": tuning,
    }
    if ordered is not None:
        out["stable_order_checked"] = ordered
    if mode == "batched":
        out["n_arrays"] = n_segs
        out["plain_form"] = f"every one of the {n_segs} arrays sorted by its own raduls_sort_ex call (plain mode)"
    elif mode == "indexed":
        out["plain_form"] = "the same input sorted record by record by raduls_sort_ex in plain mode"
    else:
        out["plain_form"] = "the same input sorted by raduls_sort_ex in plain mode"
        out["learned_used"] = f_st["learned_used"]
        out["learned_fell_back"] = f_st["learned_fell_back"]
        out["max_over_ideal_bucket"] = f_st["learned_ratio"]
        out["bytes_moved"] = _moved(f_st)
        out["plain_bytes_moved"] = _moved(p_st)
        for tag, st in (("roofline", f_st), ("plain_roofline", p_st)):
            cls_b = {c: st[f] for c, f in CLASS_BYTES.items()}
            cls_l = {c: st["kernel_launches"][c] for c in CLASS_BYTES}
            rf = roofline_of(st["kernel_ms"], cls_b, cls_l, 1, rec, hbm_peak, peak_kind, _moved(st),
                             sum(st["kernel_ms"].values()), 1)
            rf["traffic"] = None       # no ncu capture of this workload's launches
            out[tag] = rf
    del pristine, recs, tmp, d_off
    torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uniform16", choices=sorted(WORKLOADS))
    ap.add_argument("--records", type=int, default=0, help="override the workload's record count")
    ap.add_argument("--ref-records", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=15.0)
    ap.add_argument("--no-tune", action="store_true", help="skip raduls_autotune before the warm-up")
    ap.add_argument("--compare", default="skewed16,widekey32,batched16,batched16w,uniform64",
                    help="workloads timed against the plain sort after the headline (N = 1 only; '' = none)")
    ap.add_argument("--compare-steps", type=int, default=3)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    # the CPU baseline runs before any GPU work (rank 0, N = 1 only), in a
    # spawned child process: its multi-GB arrays are returned to the system
    # when the child exits instead of fragmenting this process's heap, where
    # the pinned host buffers of the end-to-end measurement are allocated
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(1) as pool:
            cpu = pool.apply(cpu_baseline, (args.workload, args.cpu_budget_s))

    import torch
    import paper_1612_02557_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build_library()
    pkg.load()

    w = WORKLOADS[args.workload]
    mode = w["mode"]
    rec, key = w["rec"], w["key"]
    rw = rec // 8
    host_in, offsets = make_input(args.workload, args.records or w["n"])
    n = host_in.shape[0]
    pristine = host_in.to("cuda", non_blocking=False)
    recs = torch.empty_like(pristine)
    tmp = torch.empty_like(pristine)
    d_off = None
    if offsets is not None:
        d_off = torch.from_numpy(offsets.view(np.int64)).cuda()
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    def one_sort(stats=False, how=None):
        how = how or mode
        if how == "batched":
            pkg.raduls_sort_batched(recs, tmp, d_off, offsets.size - 1, rec, key)
            return None
        return pkg.raduls_sort_ex(recs, tmp, n, rec, key, mode=how, stats=stats)

    # launch shapes and size-class thresholds tuned on seeded records of the
    # same size and layout (untimed; recs and tmp serve as its scratch)
    tuning = None
    if not args.no_tune:
        if mode == "batched":
            tuning = pkg.raduls_autotune(recs, tmp, n, rec, key, d_off, offsets.size - 1)
        else:
            tuning = pkg.raduls_autotune(recs, tmp, n, rec, key)
        torch.cuda.synchronize()

    # the clock sampler starts before the warm-up: nvidia-smi's start-up
    # (driver queries) then falls outside the timed steps, which it still covers
    sampler = ClockSampler(local)
    sampler.start()

    # warm-up (untimed), first one checked
    for i in range(args.warmup):
        recs.copy_(pristine)
        one_sort()
        if i == 0:
            torch.cuda.synchronize()
            st = pkg.raduls_stream_status()
            if st != 0:
                raise SystemExit(f"device status {st} during warm-up")
            if rec == 16 and key == 8 and mode != "batched":
                assert check_sorted_gpu(recs, pristine[:, 0]), "warm-up sort output is not the stable order"

    hbm_peak, peak_kind = peaks()
    step_ms = []
    cls_bytes = {c: 0 for c in CLASS_BYTES}
    cls_launches = {c: 0 for c in CLASS_BYTES}
    launches = 0
    total_bytes = 0
    kernel_ms = {}
    learned_info = None
    for _ in range(args.steps):
        recs.copy_(pristine)                      # restore the input (untimed)
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = one_sort(stats=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        step_ms.append(ev0.elapsed_time(ev1))
        if st is None:
            continue
        for c, field in CLASS_BYTES.items():
            cls_bytes[c] += st[field]
            cls_launches[c] += st["kernel_launches"][c]
        launches += st["gpu_launches"]
        total_bytes += st["hist_bytes_read"] + st["scatter_bytes"] + st["block_bytes"] + st["bucket_bytes"]
        for k, v in st["kernel_ms"].items():
            kernel_ms[k] = kernel_ms.get(k, 0.0) + v
        if st.get("learned_used"):
            learned_info = {"learned_used": st["learned_used"], "fell_back": st["learned_fell_back"],
                            "max_over_ideal_bucket": st["learned_ratio"]}
    clocks = sampler.stop()
    if pkg.raduls_stream_status() != 0:
        raise SystemExit("device-side error during the timed steps")

    tot_ms = job_time_ms(sum(step_ms), dist)
    value = job_rate(n, world, args.steps, tot_ms)

    # the same input through the plain path (learned workloads) or a per-array
    # plain loop over a prefix of the arrays (batched workload), for comparison
    comparison = None
    if mode == "learned":
        cms = []
        for _ in range(max(2, args.steps // 2)):
            recs.copy_(pristine)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cst = one_sort(stats=True, how="plain")
            e1.record(stream)
            torch.cuda.synchronize()
            cms.append(e0.elapsed_time(e1))
        comparison = {"plain_records_per_s": n * len(cms) / (sum(cms) / 1e3),
                      "plain_ms_per_step": sum(cms) / len(cms),
                      "plain_bytes_moved": (cst["hist_bytes_read"] + cst["scatter_bytes"] + cst["block_bytes"]
                                            + cst["bucket_bytes"]),
                      "learned_bytes_moved": total_bytes // max(args.steps, 1),
                      "learned_speedup": (sum(cms) / len(cms)) / (tot_ms / args.steps)}
    elif mode == "batched":
        k_arrays = min(2000, offsets.size - 1)
        lo, hi = int(offsets[0]), int(offsets[k_arrays])
        recs.copy_(pristine)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for a in range(k_arrays):
            s0, s1 = int(offsets[a]), int(offsets[a + 1])
            if s1 - s0 > 1:
                pkg.raduls_sort_ex(recs[s0:s1], tmp[s0:s1], s1 - s0, rec, key, mode="plain")
        e1.record(stream)
        torch.cuda.synchronize()
        loop_ms = e0.elapsed_time(e1)
        comparison = {"per_array_plain_loop_records_per_s": (hi - lo) / (loop_ms / 1e3),
                      "loop_sample": f"first {k_arrays} arrays ({hi - lo} records) sorted one plain raduls_sort_ex "
                                     "call each",
                      "batched_speedup": ((hi - lo) / (loop_ms / 1e3)) and value / ((hi - lo) / (loop_ms / 1e3))}

    # end to end: pinned host records -> device -> sort -> device -> pinned host,
    # in place (no second host buffer: the unsorted records are put back from
    # the device's pristine copy before every step, untimed)
    e2e = None
    if args.e2e_steps > 0:
        e2e_ms = []

        def e2e_step():
            if mode == "batched":
                recs.copy_(host_in, non_blocking=True)
                one_sort()
                host_in.copy_(recs, non_blocking=True)
            else:
                # the library's host entry point: copy in, sort, copy out
                pkg.raduls_sort_host(host_in, host_in, n, rec, key, mode=mode, stream=stream)

        def restore_host():
            host_in.copy_(pristine)
            torch.cuda.synchronize()

        # one untimed call first: the library allocates its device copy of the
        # records on the first host-entry call, as the timed loop's warm-up
        restore_host()
        e2e_step()
        torch.cuda.synchronize()
        for _ in range(args.e2e_steps):
            restore_host()
            barrier()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            e2e_step()
            ev1.record(stream)
            torch.cuda.synchronize()
            barrier()
            e2e_ms.append(ev0.elapsed_time(ev1))
        if rec == 16 and key == 8 and mode != "batched":
            # the last end-to-end result, checked on the device like the warm-up's
            recs.copy_(host_in)
            assert check_sorted_gpu(recs, pristine[:, 0]), "end-to-end output is not the stable order"
        et = job_time_ms(sum(e2e_ms), dist)
        e2e = {"value": job_rate(n, world, args.e2e_steps, et), "unit": UNIT,
               "h2d_bytes_per_step": n * rec, "d2h_bytes_per_step": n * rec,
               "ms_per_step": et / args.e2e_steps, "ms_steps": [round(x, 2) for x in e2e_ms]}

    roofline = roofline_of(kernel_ms, cls_bytes, cls_launches, args.steps, rec, hbm_peak, peak_kind, total_bytes,
                           tot_ms, world)

    # learned / batched forms against the plain sort, on their own full-size
    # workloads (one GPU only: the headline's buffers are released first)
    comparisons = None
    names = [x for x in args.compare.split(",") if x and x != args.workload]
    if world == 1 and names:
        del pristine, recs, tmp, host_in
        torch.cuda.empty_cache()
        comparisons = {}
        for nm in names:
            comparisons[nm] = compare_workload(nm, pkg, max(1, args.compare_steps), 2, hbm_peak, peak_kind)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "ms_steps": [round(x, 2) for x in step_ms],
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": w["desc"], "n_records": n, "rec_bytes": rec,
                   "key_bytes": key, "mode": mode,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "input 32 GiB-class, far larger than L2; restored from a pristine device copy before each step",
                   "tuning": tuning},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if comparison is not None:
        line["comparison"] = comparison
    if comparisons is not None:
        line["comparisons"] = comparisons
    if learned_info is not None:
        line["learned"] = learned_info
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
