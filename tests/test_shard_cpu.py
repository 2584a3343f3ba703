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


def _dirk3():
    """The L-stable three-stage DIRK of App. A (gamma the root of 6x^3 - 18x^2 + 9x - 1 near
    0.4358665; stiffly accurate)."""
    g = float(next(r.real for r in np.roots([6.0, -18.0, 9.0, -1.0]) if abs(r.imag) < 1e-12 and 0.43 < r.real < 0.44))
    b1, b2 = -1.5 * g * g + 4.0 * g - 0.25, 1.5 * g * g - 5.0 * g + 1.25
    return np.array([[g, 0, 0], [(1 - g) / 2, g, 0], [b1, b2, g]]), np.array([b1, b2, g])


class _ToyShard:
    """A stand-in for a solver part with the same calls, for the host control flow (test
    code): ordinates j in [jb, je) of a transport-free relaxation df_j/dt = nu (M_j(U) - f_j)
    with a linear M_j(U) = (U_n + c v_j U_m) / J at every node, advanced by DIRK3 stages
    (stage s solves (nu + 1/(dt A_ss)) f = q^(s) + nu M(U) by the Picard loop, which converges
    geometrically because M feeds the momentum back), U = (sum_j f_j, sum_j v_j f_j,
    sum_j v_j^2 f_j / 2) per node, v_j = j - (J - 1) / 2."""

    def __init__(self, jb, je, J=8, nnode=5, nu=4.0, dt=0.5, c=0.12):
        self.jb, self.je, self.J, self.nu, self.dt, self.c = jb, je, J, nu, dt, c
        g = synth.splitmix64_uniform(11, J * nnode).reshape(J, nnode)
        self.f = torch.from_numpy(0.5 + g[jb:je]).to(torch.float64)
        self.v = torch.arange(jb, je, dtype=torch.float64) - (J - 1) / 2
        self.nnode = nnode
        self.A, self.b = _dirk3()
        self.F = [None] * 3

    def new_moments(self):
        return torch.empty((self.nnode, 3), dtype=torch.float64)

    def partial(self, U):
        U[:, 0] = self.f.sum(0)
        U[:, 1] = (self.v[:, None] * self.f).sum(0)
        U[:, 2] = (0.5 * self.v[:, None] ** 2 * self.f).sum(0)

    def sum_partials(self, stack):
        tot = stack[0].clone()
        for x in stack[1:]:
            tot += x
        return tot

    def measure(self, Un, Uo):
        n = torch.linalg.vector_norm
        d = Un - Uo
        return float(max(n(d[:, 0]) / n(Uo[:, 0]), n(d[:, 1]) / max(n(Uo[:, 1]), n(Uo[:, 0])),
                         n(d[:, 2]) / n(Uo[:, 2])))

    def step_begin(self):
        self.fk = self.f.clone()
        return 3, 1e-12

    def stage_begin(self, s):
        a = self.A[s, s]
        acc = self.fk.clone()
        for r in range(s):
            acc += self.dt * self.A[s, r] * self.F[r]
        self.q = acc / (self.dt * a)
        self.nus = self.nu + 1.0 / (self.dt * a)

    def sweep(self, U):
        M = (U[:, 0][None, :] + self.c * self.v[:, None] * U[:, 1][None, :]) / self.J
        self.f = (self.q + self.nu * M) / self.nus

    def stage_end(self, s):
        self.F[s] = self.f / (self.dt * self.A[s, s]) - self.q

    def step_end(self):
        pass          # stiffly accurate: f^{k+1} is the last stage's value


def _sharded_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    (jb, je), = [r for k, r in enumerate(shard.ordinate_shards(8, 1, world)) if k == rank]
    part = _ToyShard(jb, je)
    its = shard.sharded_steps([part], 3, l_max=200)
    q.put((rank, its, part.f.numpy()))
    dist.destroy_process_group()


def test_sharded_dirk3_steps_across_two_gloo_ranks_match_one_process():
    """sharded_steps with the ordinates split over two gloo ranks (DIRK3 stages, the partial
    moments gathered and added in rank order) takes the same Picard iterations in every
    stage on both ranks as one process holding every ordinate, and each rank's ordinates
    end where the single-process run puts them (up to summation order)."""
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
    its_ref = shard.sharded_steps([whole], 3, l_max=200)
    assert res[0][0] == res[1][0] == its_ref
    assert len(its_ref) == 3 and all(len(s) == 3 for s in its_ref) and min(min(s) for s in its_ref) > 5
    for r, (a, b) in enumerate(shard.ordinate_shards(8, 1, world)):
        np.testing.assert_allclose(res[r][1], whole.f.numpy()[a:b], rtol=1e-14, atol=0)


def test_sharded_steps_in_one_process_with_two_parts():
    parts = [_ToyShard(0, 4), _ToyShard(4, 8)]
    whole = _ToyShard(0, 8)
    assert shard.sharded_steps(parts, 2, l_max=200) == shard.sharded_steps([whole], 2, l_max=200)
    np.testing.assert_allclose(torch.cat([p.f for p in parts]).numpy(), whole.f.numpy(), rtol=1e-14)
    with pytest.raises(RuntimeError):
        shard.sharded_steps([_ToyShard(0, 8)], 1, l_max=3)


def test_toy_dirk3_step_equals_the_stability_function_when_m_is_fixed():
    """With c = 0 the toy's M(U) is the density over J, which the relaxation conserves, so a
    step is f^1 - M = R(-nu dt) (f^0 - M) with R of the DIRK3 tableau: the toy's stage
    bookkeeping (the control flow under test) is the method's."""
    t = _ToyShard(0, 8, c=0.0)
    f0 = t.f.clone()
    M = f0.sum(0, keepdim=True) / t.J
    shard.sharded_steps([t], 1, l_max=200)
    A, b = _dirk3()
    z = -t.nu * t.dt
    R = 1.0 + z * b @ np.linalg.solve(np.eye(3) - z * A, np.ones(3))
    np.testing.assert_allclose(t.f.numpy(), (M + R * (f0 - M)).numpy(), rtol=1e-12)
