"""The N-GPU bench path runs independent replicas (no data-path collective).  Its only
cross-rank step, the max-over-ranks job time and the whole-job rate, is checked here with
two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_total = [1.5, 2.25][rank]            # seconds spent by this replica
    slowest = bench._max_over_ranks(local_total, "cpu")
    q.put((rank, slowest, bench.aggregate_rate(world, 10, 8, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_on_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in out:
        assert slowest == 2.25
        assert rate == pytest.approx(2 * 10 * 8 / 2.25)


def test_single_rank_rate():
    assert bench.aggregate_rate(1, 20, 1, 0.05) == pytest.approx(400.0)
