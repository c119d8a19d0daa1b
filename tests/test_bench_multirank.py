"""Host-side logic of bench.py's multi-process form (one replica per GPU,
launched by torch.distributed.run): rank environment, the max-over-ranks
timing and the whole-job value, run as two gloo processes on the CPU."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, times, out):
    import torch.distributed as dist

    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    bench = load_bench()
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    ms = bench.max_over_ranks(times[rank], w, "cpu")
    out.put((rank, r, w, local, ms, bench.job_value(1000.0, w, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    times = [12.0, 30.0]
    procs = [ctx.Process(target=rank_main, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, r, w, local, ms, value in res:
        assert (r, w, local) == (rank, 2, rank)
        assert ms == 30.0                       # every rank sees the maximum
        assert value == pytest.approx(2 * 1000.0 / 0.030)


def test_single_process_defaults():
    bench = load_bench()
    saved = {k: os.environ.pop(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_env() == (0, 1, 0)
        assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
        assert bench.job_value(2097152, 1, 51.4) == pytest.approx(2097152 / 0.0514)
    finally:
        os.environ.update(saved)
