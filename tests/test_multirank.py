"""The N > 1 path of the benchmark on CPU: two gloo ranks (replicas, weak
scaling).  The whole-job rate is units per rank x ranks over the slowest
rank's time, identical on every rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [40.0, 25.0][rank]
    rate, ms = bench.whole_job_rate(1000, ms_local, world)
    out[rank] = (rate, ms, bench.rank_max(float(rank), world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_whole_job_rate():
    import torch.multiprocessing as mp
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:  # no fork of a process that may run threads
        out = man.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
        res = dict(out)
    for rank in (0, 1):
        rate, ms, mx = res[rank]
        assert ms == 40.0                      # the slowest rank's time on every rank
        assert abs(rate - 2 * 1000 / 0.040) < 1e-6
        assert mx == 1.0


def test_single_rank_rate():
    import bench
    rate, ms = bench.whole_job_rate(500, 10.0, 1)
    assert ms == 10.0 and abs(rate - 50000.0) < 1e-9
