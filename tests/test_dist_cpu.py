"""Multi-rank host logic of bench.py on CPU: two gloo ranks (world size 2),
each timing a different region, agree on the whole-job time (the slower
rank's) and on the whole-job rate.  The GPU path is replicas only (every rank
sorts its own array, no data-path collective), so this reduction is the only
cross-rank step."""
from __future__ import annotations

import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str) -> None:
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        local = [120.0, 95.5][rank]
        job = bench.job_time_ms(local, dist, device="cpu")
        rate = bench.job_rate(1000, world, 4, job)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{job} {rate}")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_job_time_and_rate(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    pytest.importorskip("torch.distributed")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    vals = [tuple(map(float, open(tmp_path / f"r{r}.txt").read().split())) for r in range(2)]
    assert vals[0] == vals[1]
    job, rate = vals[0]
    assert job == 120.0                       # the slower rank sets the job time
    assert rate == pytest.approx(1000 * 2 * 4 / 0.120)


def test_single_rank_is_its_own_job():
    import bench
    assert bench.job_time_ms(42.0, None) == 42.0
    assert bench.job_rate(10, 1, 2, 1000.0) == pytest.approx(20.0)
