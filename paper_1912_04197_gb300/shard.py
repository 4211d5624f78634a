"""Sharded evaluation of one cloud over several processes, one GPU each.

The walk of Sec. 2.1 (kernel 5) computes each body's force from the tree alone, so the
bodies can be split between devices without changing any result:

  * every rank holds all N positions and builds the same tree (the build is
    deterministic, so the trees are identical bit for bit);
  * the tree's walk tasks (up to 32 Morton-consecutive bodies of one cloud each) are cut
    into contiguous ranges, one per rank (`plan`), and each rank walks its own range
    (`gravity_forces_range`, rows in sorted order);
  * one all-gather per force evaluation hands every rank all ranges' rows, which
    `gravity_scatter_sorted` puts back in the caller's order;
  * the integrator's O(N) kick-drift and kick run on every rank over all bodies
    (replicated, identical), so every rank ends each step with the same positions and
    velocities as a single-device leapfrog_step, bit for bit.

The exchange is expressed through a small communicator object: `TorchComm` wraps a
torch.distributed process group (NCCL on GPUs; gloo for host tensors), `LocalComm` runs
every rank's range in one process (a test of the decomposition on one device).  The
engine object supplies the library calls (`GpuEngine` on a gravity Context); the
orchestration below does only bookkeeping: the arithmetic runs in the engine.
"""
from __future__ import annotations

import torch


def plan(ntasks: int, world: int) -> list[tuple[int, int]]:
    """Contiguous task ranges (first, count) of `world` ranks, counts differing by <= 1."""
    if world < 1:
        raise ValueError("world must be >= 1")
    return [(ntasks * r // world, ntasks * (r + 1) // world - ntasks * r // world)
            for r in range(world)]


class LocalComm:
    """All ranks' ranges computed in this process (no collective)."""

    def __init__(self, world: int):
        self.rank, self.world = 0, int(world)

    def gather_parts(self, make_part):
        return [make_part(r) for r in range(self.world)]


class TorchComm:
    """One rank of a torch.distributed process group: computes its own range and
    all-gathers the padded parts (dist.all_gather: NCCL or gloo)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def gather_parts(self, make_part):
        part = make_part(self.rank)
        out = [torch.empty_like(part) for _ in range(self.world)]
        self.dist.all_gather(out, part, group=self.group)
        return out


class GpuEngine:
    """The library calls of one rank's context (see gravity.py / gravity.h)."""

    def __init__(self, ctx, params):
        from . import gravity
        self.g, self.ctx, self.params = gravity, ctx, params

    def build(self, pos, mass):
        self.g.gravity_tree_build(self.ctx, pos, mass, self.params)

    def walk_tasks(self) -> int:
        return self.g.gravity_walk_tasks(self.ctx)

    def task_bodies(self, first: int, count: int) -> tuple[int, int]:
        return self.g.gravity_task_bodies(self.ctx, first, count)

    def forces_range(self, theta, eps, first, count, out):
        if count > 0:
            self.g.gravity_forces_range(self.ctx, theta, eps, first, count, out)

    def scatter_sorted(self, first_body, src, dst):
        if src.shape[0] > 0:
            self.g.gravity_scatter_sorted(self.ctx, first_body, src, dst)

    def kick_drift(self, pos, vel, acc, h, dt):
        self.g.gravity_kick_drift(self.ctx, pos, vel, acc, h, dt)

    def kick(self, vel, acc, h):
        self.g.gravity_kick(self.ctx, vel, acc, h)

    def empty(self, rows, like):
        return torch.empty((rows, 3), dtype=torch.float64, device=like.device)


def sharded_forces(engine, comm, theta: float, eps: float, acc: torch.Tensor) -> torch.Tensor:
    """Accelerations of every body (caller order, into acc) from the tree the engine built
    last: this rank walks its task range, the ranges are all-gathered and scattered back."""
    ranges = plan(engine.walk_tasks(), comm.world)
    bodies = [engine.task_bodies(f, c) for f, c in ranges]
    rows = max(1, max(nb for _, nb in bodies))

    def make_part(r):
        part = engine.empty(rows, acc)
        part.zero_()
        f, c = ranges[r]
        engine.forces_range(theta, eps, f, c, part)
        return part

    parts = comm.gather_parts(make_part)
    for (b0, nb), part in zip(bodies, parts):
        engine.scatter_sorted(b0, part[:nb], acc)
    return acc


def sharded_leapfrog(engine, comm, pos, vel, mass, acc, dt: float, nsteps: int, theta: float,
                     eps: float, scheme: int = 0):
    """nsteps steps of the KDK leapfrog (scheme 0) or semi-implicit Euler (scheme 1) of
    Sec. 2.3 with sharded force evaluations; acc holds a(x) on entry and on exit, as for
    leapfrog_step.  Every rank updates all bodies, so pos / vel / acc stay identical on
    every rank."""
    kdk = scheme == 0
    h = 0.5 * dt if kdk else dt
    for _ in range(int(nsteps)):
        engine.kick_drift(pos, vel, acc, h, dt)
        engine.build(pos, mass)
        sharded_forces(engine, comm, theta, eps, acc)
        if kdk:
            engine.kick(vel, acc, h)
    return pos, vel, acc


def partition_clouds(sizes, world: int) -> list[tuple[int, int]]:
    """Independent clouds over `world` ranks: contiguous cloud ranges [k0, k1) per rank with
    about equal cost, the cost of a cloud of N_k bodies taken as N_k log N_k (the tree walk's
    work; the build is O(N_k)).  A cut falls at the cloud boundary nearest to each rank's
    share of the total; clouds are never split, so no exchange is needed."""
    import math
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = [float(n) * math.log(max(float(n), 2.0)) for n in sizes]
    total = sum(cost)
    cuts, acc, k = [0], 0.0, 0
    for r in range(1, world):
        target = total * r / world
        while k < len(cost) and acc + cost[k] <= target:
            acc += cost[k]
            k += 1
        if k < len(cost) and (target - acc) > (acc + cost[k] - target):
            acc += cost[k]                     # the nearer boundary is after this cloud
            k += 1
        cuts.append(max(k, cuts[-1]))
    cuts.append(len(cost))
    return [(cuts[r], cuts[r + 1]) for r in range(world)]
