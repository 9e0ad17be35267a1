"""The multi-GPU path of bench.py is replicas only: every rank contracts its own
batch and the job's time is the slowest rank's.  Two gloo ranks on the CPU
check the cross-rank aggregation, the whole-job rate and that the replicas'
inputs differ (no GPU, no collective on the data path)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    from paper_1908_08553_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, _ = bench._dist()
        t_local = 1.0 + 0.25 * rank                  # rank 1 is the slow replica
        t_max = bench.max_over_ranks(t_local, got_ws, device="cpu")
        rate = bench.job_rate(got_ws, 256, 20, t_max)
        first = inputs.random_lattice(8, 8, 2, inputs.lattice_seed(bench.replica_seed(got_rank), 0))[:8]
        out.put((got_rank, got_ws, t_max, rate, first.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[2] == pytest.approx(1.25) for r in res)          # every rank sees the slowest time
    assert all(r[3] == pytest.approx(2 * 256 * 20 / 1.25) for r in res)
    assert not np.allclose(res[0][4], res[1][4])                  # replicas contract different lattices


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(1, 256, 20, 2.0) == 2560.0
