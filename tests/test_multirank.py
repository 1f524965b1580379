"""The multi-rank path of bench.py on CPU: two gloo ranks (weak scaling, one
batch of instances per rank, no data-path collective) check the instance
slices, the max-over-ranks timing and the whole-job rate, and each rank
contracts its own slice with the oracle (ranks are independent problems)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from oracle import dmtree  # noqa: E402

PER_RANK = 2
SIZE = 4


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = bench.rank_slice(rank, PER_RANK)
        ws = bench.make_instances(first, count, SIZE)
        logz = [dmtree.partitioned_contract_rows(w, 16)["logz"] for w in ws]
        slowest = bench.max_over_ranks(1.0 + rank, world)
        rate = bench.whole_job_rate(PER_RANK, world, 3, slowest)
        gathered = [None] * world
        dist.all_gather_object(gathered, (first, count, logz, slowest, rate))
        if rank == 0:
            out.put(gathered)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    firsts = sorted(g[0] for g in got)
    assert firsts == [0, PER_RANK]                      # disjoint slices covering 0..2B-1
    assert all(g[1] == PER_RANK for g in got)
    assert all(g[3] == 2.0 for g in got)                # max over ranks on every rank
    assert all(g[4] == PER_RANK * world * 3 / 2.0 for g in got)
    # every rank's results equal a single-process contraction of the same instances
    ws = bench.make_instances(0, PER_RANK * world, SIZE)
    ref = [dmtree.partitioned_contract_rows(w, 16)["logz"] for w in ws]
    mine = [x for g in sorted(got) for x in g[2]]
    np.testing.assert_allclose(mine, ref, rtol=0, atol=0)
