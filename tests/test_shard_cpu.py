"""Host logic of the ordinate-sharded sweep on CPU: the shard ranges, and the fixed-order
sum of partial moments across two gloo ranks (bitwise equal on both ranks and to the
ordered sum computed in one process)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2608_19150_b300 import shard, synth


@pytest.mark.parametrize("n,dim,parts", [(32, 2, 1), (32, 2, 3), (16, 3, 4), (20, 2, 7), (8, 3, 8)])
def test_ordinate_shards_cover_all_ordinates_in_whole_outer_values(n, dim, parts):
    r = shard.ordinate_shards(n, dim, parts)
    inner = n ** (dim - 1)
    assert r[0][0] == 0 and r[-1][1] == n ** dim
    for (a, b), (c, _) in zip(r, r[1:]):
        assert b == c
    sizes = [(b - a) // inner for a, b in r]
    assert all((b - a) % inner == 0 and a % inner == 0 for a, b in r)
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        shard.ordinate_shards(n, dim, n + 1)


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _partials(world, shape):
    u = synth.splitmix64_uniform(5, world * int(np.prod(shape))).reshape((world,) + shape)
    return (u - 0.5) * 10.0 ** np.arange(shape[-1])      # mixed magnitudes: order matters


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = torch.from_numpy(_partials(world, (64, 4))[rank])
    tot = shard.sum_fixed_order(p)
    q.put((rank, tot.numpy()))
    dist.destroy_process_group()


def test_fixed_order_sum_across_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=5) for _ in range(world))
    parts = _partials(world, (64, 4))
    expect = parts[0].copy()
    for k in range(1, world):
        expect += parts[k]
    np.testing.assert_array_equal(res[0], res[1])
    np.testing.assert_array_equal(res[0], expect)


def test_sum_without_a_group_is_the_partial_itself():
    p = torch.arange(6, dtype=torch.float64)
    assert torch.equal(shard.sum_fixed_order(p), p)
