"""The benchmark's N > 1 path on the CPU: two gloo ranks, each with its own
shard of independent stacks, no data-path collective, whole-job rate from the
slowest rank's time."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2111_13667_gb300 import dist as D
from paper_2111_13667_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, wsz, local = D.env()
        w = W.dispersive(S=8, L=3, n_lambda=4, n_theta=2, shard=r)
        D.barrier()
        rate, ms = D.aggregate_rate(units_per_rank=w.evals, ms_per_rank=10.0 * (r + 1), world=wsz)
        out[rank] = (r, wsz, local, rate, ms, float(w.d.sum()), float(w.table.real.sum()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    evals = W.dispersive(S=8, L=3, n_lambda=4, n_theta=2).evals
    for rank, (r, wsz, local, rate, ms, dsum, tsum) in res.items():
        assert (r, wsz, local) == (rank, 2, rank)
        assert ms == 20.0  # the slowest rank's time, seen by every rank
        assert rate == pytest.approx(evals * 2 / 20e-3)
    # shards hold different stacks over the same material table; shard 0 is the 1-GPU workload
    assert res[0][5] != res[1][5] and res[0][6] == res[1][6]
    assert res[0][5] == pytest.approx(float(W.dispersive(S=8, L=3, n_lambda=4, n_theta=2).d.sum()))


def test_single_process_helpers_without_process_group():
    assert D.max_over_ranks(3.5) == 3.5
    rate, ms = D.aggregate_rate(100, 2.0, 1)
    assert ms == 2.0 and rate == pytest.approx(100 / 2e-3)
