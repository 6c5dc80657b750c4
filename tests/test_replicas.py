"""Replica bookkeeping on CPU: two gloo ranks agree on the slowest rank's
time and on the whole-job rate (no GPU, no collective on the data path)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2605_27147_gb300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = replicas.rank_info()
        my_ms = 10.0 + 7.5 * r                     # rank 1 is the slow one
        job_ms = replicas.max_over_ranks(my_ms, dist)
        rate = replicas.job_rate(1_000_000, w, job_ms)
        out.put((r, w, lr, job_ms, rate, replicas.replica_seed(3, r)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_job_time_and_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 and r[2] == r[0] for r in res)
    assert all(r[3] == 17.5 for r in res)                          # the slowest rank's time
    assert all(abs(r[4] - 2_000_000 / 0.0175) < 1e-6 for r in res)  # units of both ranks / job time
    assert res[0][5] != res[1][5]                                  # replicas may sort different data


def test_single_rank_needs_no_process_group():
    assert replicas.max_over_ranks(4.25) == 4.25
    assert replicas.job_rate(3, 1, 1000.0) == 3.0
    with pytest.raises(ValueError):
        replicas.job_rate(3, 1, 0.0)
