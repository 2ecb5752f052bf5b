"""The N > 1 path of bench.py: replicas only (no collective on the data path;
the sweep is not sharded), with the slowest rank's time taken by an all-reduce
MAX.  Run here as two gloo ranks on the CPU."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    b = _bench()
    r, w, local = b.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    local_ms = 100.0 + 50.0 * rank            # rank 1 is the slower replica
    ms, value = b.replica_timing(local_ms, 10, 1.0e9, w, dist, "cpu")
    out.put((r, w, local, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_the_whole_job_rate():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, local, ms, value) in enumerate(results):
        assert (rank, world, local) == (r, 2, r)
        assert ms == pytest.approx(15.0)                 # max(100, 150) ms / 10 steps
        assert value == pytest.approx(2 * 1.0e9 / 15.0e-3)


def test_single_process_needs_no_process_group():
    b = _bench()
    ms, value = b.replica_timing(50.0, 5, 2.0e9, 1, None, "cpu")
    assert ms == 10.0 and value == pytest.approx(2.0e9 / 10.0e-3)
