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


class _ToyShard:
    """A stand-in for a solver shard with the same three calls, for the host control flow:
    ordinates j in [jb, je) of a relaxation problem f_j <- (f_j^k + a M_j(U)) / (1 + a),
    M_j(U) = (U_n + c v_j U_m) / J at every node (linear; it keeps the mass and feeds the
    momentum back, so the loop converges geometrically, rate a c sum v^2 / (J (1 + a))),
    U = (sum_j f_j, sum_j v_j f_j, sum_j v_j^2 f_j / 2) per node, v_j = j - (J - 1) / 2."""

    def __init__(self, jb, je, J=8, nnode=5, a=3.0, c=0.12):
        self.jb, self.je, self.J, self.a, self.c = jb, je, J, a, c
        g = synth.splitmix64_uniform(11, J * nnode).reshape(J, nnode)
        self.fk = torch.from_numpy(0.5 + g[jb:je]).to(torch.float64)
        self.f = self.fk.clone()
        self.v = torch.arange(jb, je, dtype=torch.float64) - (J - 1) / 2
        self.nnode = nnode

    def new_moments(self):
        return torch.empty((self.nnode, 3), dtype=torch.float64)

    def partial(self, U):
        U[:, 0] = self.f.sum(0)
        U[:, 1] = (self.v[:, None] * self.f).sum(0)
        U[:, 2] = (0.5 * self.v[:, None] ** 2 * self.f).sum(0)

    def sweep(self, U):
        M = (U[:, 0][None, :] + self.c * self.v[:, None] * U[:, 1][None, :]) / self.J
        self.f = (self.fk + self.a * M) / (1 + self.a)

    def commit(self):
        self.fk = self.f.clone()


def _sharded_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    (jb, je), = [r for k, r in enumerate(shard.ordinate_shards(8, 1, world)) if k == rank]
    part = _ToyShard(jb, je)
    its = [shard.picard_sharded([part], shard.sum_fixed_order, 1, 1e-12, 200) for _ in range(3)]
    q.put((rank, its, part.f.numpy()))
    dist.destroy_process_group()


def test_sharded_picard_across_two_gloo_ranks_matches_one_process():
    """picard_sharded with the ordinates split over two gloo ranks takes the same number of
    iterations on both ranks as one process holding every ordinate, and each rank's
    ordinates end where the single-process run puts them (up to summation order)."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_sharded_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = {r: (its, f) for r, its, f in (q.get(timeout=5) for _ in range(world))}
    whole = _ToyShard(0, 8)
    its_ref = [shard.picard_sharded([whole], lambda U: U, 1, 1e-12, 200) for _ in range(3)]
    assert res[0][0] == res[1][0] == its_ref
    assert min(its_ref) > 10
    for r, (a, b) in enumerate(shard.ordinate_shards(8, 1, world)):
        np.testing.assert_allclose(res[r][1], whole.f.numpy()[a:b], rtol=1e-14, atol=0)


def test_sharded_picard_in_one_process_with_two_parts():
    parts = [_ToyShard(0, 4), _ToyShard(4, 8)]
    whole = _ToyShard(0, 8)
    assert (shard.picard_sharded(parts, lambda U: U, 1, 1e-12, 200)
            == shard.picard_sharded([whole], lambda U: U, 1, 1e-12, 200))
    np.testing.assert_allclose(torch.cat([p.f for p in parts]).numpy(), whole.f.numpy(), rtol=1e-14)
    with pytest.raises(RuntimeError):
        shard.picard_sharded([_ToyShard(0, 8)], lambda U: U, 1, 1e-30, 3)
