"""The sharded single-cloud evaluation's host logic (paper_1912_04197_gb300/shard.py) on
CPU ranks: two gloo ranks, each with an engine whose force evaluation is the FP64 oracle
(the walk of Sec. 2.1, kernel 5, restricted to the rank's Morton range of bodies).  Each
body's oracle force does not depend on which other bodies are evaluated with it, so the
task split, the all-gather of padded ranges and the scatter back to the caller's order
must reproduce the single-rank oracle run exactly: positions, velocities and
accelerations after a few leapfrog (and semi-implicit Euler) steps, bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

N_BODIES, STEPS, DT, THETA, EPS = 3001, 4, 1e-3, 0.5, 5e-3


class OracleEngine:
    """The engine interface of shard.py over the oracle (host tensors, FP64)."""

    def __init__(self, leaf_max, order):
        self.leaf_max, self.order = leaf_max, order
        self.tree, self.perm, self.n = None, None, 0

    def build(self, pos, mass):
        import oracle
        self.tree = oracle.Tree(pos.numpy(), mass.numpy(), leaf_max=self.leaf_max, order=self.order)
        self.perm = self.tree.order_arrays()[1]
        self.n = len(self.perm)

    def walk_tasks(self):
        return (self.n + 31) // 32

    def task_bodies(self, first, count):
        if count == 0:
            return 0, 0
        return 32 * first, min(32 * (first + count), self.n) - 32 * first

    def forces_range(self, theta, eps, first, count, out):
        b0, nb = self.task_bodies(first, count)
        if nb:
            a = self.tree.forces(theta, eps, targets=self.perm[b0:b0 + nb])[0]
            out[:nb] = torch.from_numpy(a)

    def scatter_sorted(self, first_body, src, dst):
        dst[torch.from_numpy(self.perm[first_body:first_body + src.shape[0]])] = src

    def kick_drift(self, pos, vel, acc, h, dt):
        vel.copy_(vel + acc * h)              # the oracle's roundings: product, then sum
        pos.copy_(pos + vel * dt)

    def kick(self, vel, acc, h):
        vel.copy_(vel + acc * h)

    def empty(self, rows, like):
        return torch.empty((rows, 3), dtype=torch.float64)


def _inputs():
    from paper_1912_04197_gb300 import inputs
    return inputs.rubble_pile(N_BODIES, seed=12)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1912_04197_gb300 import shard
        pos, vel, m = _inputs()
        comm = shard.TorchComm()
        res = {}
        for scheme in (0, 1):
            eng = OracleEngine(leaf_max=8, order=2)
            P, V, M = torch.tensor(pos), torch.tensor(vel), torch.tensor(m)
            A = torch.tensor(oracle.tree_forces(pos, m, THETA, EPS, leaf_max=8, order=2))
            # one sharded force evaluation equals the oracle's forces of all bodies
            eng.build(P, M)
            A1 = torch.zeros_like(P)
            shard.sharded_forces(eng, comm, THETA, EPS, A1)
            shard.sharded_leapfrog(eng, comm, P, V, M, A, DT, STEPS, THETA, EPS, scheme=scheme)
            res[scheme] = (A1.numpy(), P.numpy(), V.numpy(), A.numpy())
        out[rank] = res
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_plan_is_contiguous_and_balanced():
    from paper_1912_04197_gb300 import shard
    for ntasks in (0, 1, 7, 32768):
        for world in (1, 2, 3, 8):
            p = shard.plan(ntasks, world)
            assert len(p) == world and p[0][0] == 0
            assert all(p[r][0] + p[r][1] == p[r + 1][0] for r in range(world - 1))
            assert p[-1][0] + p[-1][1] == ntasks
            assert max(c for _, c in p) - min(c for _, c in p) <= 1


def test_local_comm_equals_single_rank_oracle():
    # one process, three ranks emulated: ranges computed one after another, no collective
    import oracle
    from paper_1912_04197_gb300 import shard
    pos, vel, m = _inputs()
    eng = OracleEngine(leaf_max=8, order=2)
    eng.build(torch.tensor(pos), torch.tensor(m))
    A = torch.zeros((N_BODIES, 3), dtype=torch.float64)
    shard.sharded_forces(eng, shard.LocalComm(3), THETA, EPS, A)
    ref = oracle.tree_forces(pos, m, THETA, EPS, leaf_max=8, order=2)
    assert np.array_equal(A.numpy(), ref)


def test_two_gloo_ranks_reproduce_the_single_rank_oracle_run():
    import oracle
    world = 2
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    pos, vel, m = _inputs()
    a0 = oracle.tree_forces(pos, m, THETA, EPS, leaf_max=8, order=2)
    for scheme in (0, 1):
        op, ov, oa = oracle.step(pos, vel, m, a0, DT, STEPS, scheme=scheme, theta=THETA, eps=EPS,
                                 leaf_max=8, order=2)
        for rank in range(world):
            A1, P, V, A = res[rank][scheme]
            assert np.array_equal(A1, a0)
            assert np.array_equal(P, op) and np.array_equal(V, ov) and np.array_equal(A, oa)


def test_partition_clouds_balances_cost():
    import math
    from paper_1912_04197_gb300 import inputs, shard
    off, _, _, _ = inputs.ensemble(nclouds=256, seed=100)
    sizes = np.diff(off)
    cost = sizes * np.log(sizes)
    for world in (1, 2, 3, 8):
        parts = shard.partition_clouds(sizes, world)
        assert parts[0][0] == 0 and parts[-1][1] == len(sizes)
        assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
        loads = [cost[a:b].sum() for a, b in parts]
        # every rank is within one (largest) cloud of its equal share
        assert max(abs(l - cost.sum() / world) for l in loads) <= cost.max()
    two = shard.partition_clouds([10, 10], 4)          # more ranks than clouds: empty ranges
    assert sorted(b - a for a, b in two) == [0, 0, 1, 1]
    with pytest.raises(ValueError):
        shard.partition_clouds([5], 0)
    assert math.isclose(sum(b - a for a, b in shard.partition_clouds(sizes, 5)), len(sizes))
