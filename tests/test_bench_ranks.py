"""The multi-rank path of the benchmark on CPU: two gloo ranks (replicas,
no data-path collective) agree on the slowest rank's time, and the job's
throughput counts every replica."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    b = _bench()
    dist.barrier()
    t = b.max_over_ranks(1.0 + 0.5 * rank, world, device="cpu")
    out.put((rank, t, b.job_throughput(world, 1000, 10, t)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [1.5, 1.5]
    assert all(abs(r[2] - 2 * 1000 * 3 * 10 / 1.5) < 1e-9 for r in res)


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(3.25, 1) == 3.25
    assert b.job_throughput(1, 8, 2, 0.5) == 96.0
