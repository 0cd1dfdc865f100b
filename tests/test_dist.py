"""Multi-rank path of bench.py on CPU (gloo, world size 2).

The RIR path shards by room with no exchange step: each rank builds its own
batch (its own seed), works alone, and only the timing is reduced (maximum
over ranks).  These tests run the same helpers bench.py uses under torchrun,
with the gloo backend and 127.0.0.1 rendezvous, without a GPU.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_2104_13347_gb300 import workloads as wl
    local_ms = 10.0 + 5.0 * rank
    bench.barrier(ws)
    got = bench.max_over_ranks(local_ms, ws)
    rooms = wl.room_batch(3, seed=bench.rank_seed(rank))
    out.put((rank, got, float(rooms[0]["dims"][0]), bench.rank_seed(rank)))
    dist.destroy_process_group()


def test_two_ranks_max_time_and_disjoint_batches():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]   # max over ranks on every rank
    assert res[0][3] != res[1][3]                # distinct seeds
    assert res[0][2] != res[1][2]                # so distinct rooms


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
