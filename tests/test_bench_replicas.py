"""The replica path of bench.py (--gpus N under torchrun): the job time is the
maximum over ranks and the value counts every replica's atoms.  Two gloo ranks
on the CPU; no GPU is touched."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    # rank r took (r + 1) ms for the device-timed steps and 10 (r + 1) ms end to end
    got = bench.max_over_ranks([rank + 1.0, 10.0 * (rank + 1)], dist, "cpu")
    q.put((rank, got))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == [2.0, 20.0] and res[1] == [2.0, 20.0]
    sys.path.insert(0, ROOT)
    import bench
    # two replicas of 4,000,000 atoms, 100 substeps per step, 20 steps in 2 s
    assert bench.job_value(2, 4_000_000, 100, 20, 2000.0) == pytest.approx(8.0e9)
    assert bench.job_value(1, 4_000_000, 100, 20, 2000.0) == pytest.approx(4.0e9)
