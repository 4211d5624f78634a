"""Range walks (gravity_forces_range) and the sharded single-cloud stepping on one GPU.

The walk computes each body's force from the tree alone (Sec. 2.1, kernel 5), so walking
the tree's tasks in G contiguous ranges and putting the rows back in the caller's order
(gravity_scatter_sorted) must give exactly what one gravity_forces launch gives, bit for
bit: at sizes where the walk splits its tasks between two warps, between 64 and where it
does not, with one cloud and with several.  The sharded leapfrog (shard.py, every rank's range
computed in this process) must equal leapfrog_step bit for bit."""
import numpy as np
import pytest
import torch

from paper_1912_04197_gb300 import inputs, shard

pytestmark = pytest.mark.gpu


def _setup(g, kind, order, leaf):
    ctx = g.Context(0)
    if kind == "clouds":
        off, pos, vel, m = inputs.ensemble(nclouds=9, seed=3, nmin=200, nmax=20000)
        g.gravity_set_clouds(ctx, off)
    elif kind == "small":
        pos, vel, m = inputs.rubble_pile(5000, seed=4)           # few tasks: split walk
    elif kind == "tiny":
        pos, vel, m = inputs.rubble_pile(2000, seed=6)           # 63 tasks: 64 parts each
    else:
        pos, vel, m = inputs.clumpy_plummer(200_000, seed=5, nclusters=8)
        vel = np.zeros_like(pos)
    P = torch.tensor(pos, device="cuda")
    V = torch.tensor(vel, device="cuda")
    M = torch.tensor(m, device="cuda")
    return ctx, P, V, M, g.params(order=order, leaf_max=leaf)


@pytest.mark.parametrize("kind,order,leaf", [("clumpy", 2, 16), ("clumpy", 0, 1),
                                             ("small", 2, 16), ("clouds", 2, 16),
                                             ("tiny", 2, 16), ("tiny", 0, 1)])
@pytest.mark.parametrize("world", [2, 3, 7])
def test_range_walks_equal_the_full_walk(gpu, kind, order, leaf, world):
    ctx, P, _, M, p = _setup(gpu, kind, order, leaf)
    gpu.gravity_tree_build(ctx, P, M, p)
    full = torch.empty_like(P)
    gpu.gravity_forces(ctx, 0.5, 1e-3, full)
    got = torch.full_like(P, float("nan"))
    ntasks = gpu.gravity_walk_tasks(ctx)
    covered = 0
    for first, count in shard.plan(ntasks, world):
        b0, nb = gpu.gravity_task_bodies(ctx, first, count)
        assert b0 == covered
        covered += nb
        part = torch.full((max(nb, 1), 3), float("nan"), dtype=torch.float64, device="cuda")
        gpu.gravity_forces_range(ctx, 0.5, 1e-3, first, count, part)
        gpu.gravity_scatter_sorted(ctx, b0, part[:nb], got)
    gpu.gravity_sync(ctx)
    assert covered == P.shape[0]
    assert torch.equal(got, full)


def test_range_arguments(gpu):
    ctx, P, _, M, p = _setup(gpu, "small", 0, 1)
    with pytest.raises(gpu.GravityError) as e:
        gpu.gravity_walk_tasks(ctx)
    assert e.value.code == gpu.GRAVITY_E_NOTREE
    gpu.gravity_tree_build(ctx, P, M, p)
    nt = gpu.gravity_walk_tasks(ctx)
    assert nt == (P.shape[0] + 31) // 32
    assert gpu.gravity_task_bodies(ctx, nt - 1, 1) == (32 * (nt - 1), P.shape[0] - 32 * (nt - 1))
    for bad in ((-1, 1), (0, nt + 1), (nt, 1)):
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_task_bodies(ctx, *bad)
        assert e.value.code == gpu.GRAVITY_E_ARG


@pytest.mark.parametrize("kind,scheme", [("clumpy", 0), ("small", 0), ("clouds", 0),
                                         ("tiny", 0), ("clumpy", 1)])
def test_sharded_leapfrog_equals_leapfrog_step(gpu, kind, scheme):
    out = []
    for sharded in (False, True):
        ctx, P, V, M, p = _setup(gpu, kind, 2, 16)
        p.scheme = scheme
        A = torch.empty_like(P)
        gpu.gravity_tree_build(ctx, P, M, p)
        gpu.gravity_forces(ctx, 0.5, 1e-3, A)
        if sharded:
            eng = shard.GpuEngine(ctx, p)
            shard.sharded_leapfrog(eng, shard.LocalComm(3), P, V, M, A, 1e-3, 5, 0.5, 1e-3,
                                   scheme=scheme)
        else:
            gpu.leapfrog_step(ctx, P, V, M, A, 1e-3, 5, 0.5, 1e-3, p)
        gpu.gravity_sync(ctx)
        out.append((P.cpu(), V.cpu(), A.cpu()))
    for x, y in zip(*out):
        assert torch.equal(x, y)
