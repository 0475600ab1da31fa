"""The multi-process path of bench.py on CPU: two gloo ranks (one per
process, rendezvous on 127.0.0.1) reduce their step times and units the way
replicas on separate GPUs do under torchrun, and the reference arm runs on
rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, result_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r took 10 + 2 r ms for 100 (r + 1) units
        value, ms = bench.whole_job(10.0 + 2.0 * rank, 100.0 * (rank + 1), ws, dist)
        # the reference arm returns at once on every rank but 0
        if rank != 0:
            bench.run_reference(None)
        result_q.put((rank, value, ms))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_units():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=120)
    assert all(pr.exitcode == 0 for pr in procs), [pr.exitcode for pr in procs]
    res = sorted(q.get(timeout=10) for _ in range(ws))
    for _, value, ms in res:
        assert ms == 12.0  # the slowest rank's time
        assert value == pytest.approx(300.0 / 12e-3)  # all ranks' units over it


def test_single_process_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.whole_job(4.0, 8.0, 1)
    assert ms == 4.0 and value == pytest.approx(2000.0)
