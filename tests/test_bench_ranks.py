"""bench.py's multi-rank host logic on the CPU: two gloo ranks (127.0.0.1) read their rank from
the launcher's environment and agree on the largest of their timings, the figure the benchmark
divides the work of all ranks by.  The GPU arm runs the same helper over NCCL, one rank per
GPU; the timed work itself is an independent replica per rank (no collective on the data path).
"""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, timings, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE="2")
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    r, lr, ws = bench.dist_info()
    dist.init_process_group("gloo", rank=r, world_size=ws)
    try:
        dist.barrier()
        got = bench.max_over_ranks(torch, timings[r], torch.device("cpu"), ws)
        dist.barrier()
        q.put((r, lr, ws, got))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("timings", [(3.0, 5.0), (7.25, 0.5)])
def test_two_gloo_ranks_take_the_slowest_rank(timings):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, timings, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r, lr, ws) for r, lr, ws, _ in out] == [(0, 0, 2), (1, 1, 2)]
    assert all(got == max(timings) for *_, got in out)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import torch
    import bench
    assert bench.max_over_ranks(torch, 4.5, torch.device("cpu"), 1) == 4.5
