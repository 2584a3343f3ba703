"""The N>1 path of bench.py on CPU: two gloo ranks (replicas, no data-path collective)
check the barrier, the max-over-ranks time and the whole-job throughput (units of all
ranks over the slowest rank's time), and that the reference arm does its work on rank 0
only."""
import importlib.util
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _load_bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    bench = _load_bench()
    r, w, l = bench.dist_init(None)
    assert (r, w, l) == (rank, world, rank)
    bench.barrier(w)
    # rank r processed (r + 1) * 100 units in (r + 1) * 0.5 s
    el = bench.max_over_ranks((rank + 1) * 0.5, w)
    thr = bench.job_throughput((rank + 1) * 100, el, w)
    q.put((rank, el, thr))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=5) for _ in range(world))
    for rank, el, thr in out:
        assert el == pytest.approx(1.0)                 # the slowest rank
        assert thr == pytest.approx(300.0 / 1.0)        # 100 + 200 units over 1 s


def test_single_rank_helpers_do_not_touch_distributed():
    bench = _load_bench()
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_throughput(10, 2.0, 1) == 5.0
