"""Parity at the full sizes of the benchmarked workloads, in the launch configuration the
benchmark times (default walk shape, default stream), on outputs the oracle computes one
by one.

  * clumpy aggregate, 1,048,576 bodies (the headline workload), theta 0.5, quadrupole,
    leaf 16: root cube, keys, order, topology, node mass and COM bit-exact against the
    oracle's tree of all bodies; forces and decision counts of 65,536 seeded bodies
    against the oracle's walk for them (16,384 bodies at theta 0.3, 0.7, 0.9, with the
    FP64 accumulator, and for the monopole at leaf 1 and 16); the direct sum of 4096
    seeded bodies against the oracle's;
  * ensemble of 256 clouds (4.4 M bodies): six clouds, each against an oracle tree of
    that cloud alone, on up to 512 seeded bodies per cloud;
  * rubble pile, 100,000 bodies: one leapfrog step against the oracle's, and 100 steps
    (the whole run) against properties that hold at any size (momentum, energy);
  * uniform sphere, 65,536 bodies: the vector-Jacobian product of every body.

Tolerances are those of the smaller parity tests, on every sampled body: forces within
1e-6 of sum |t| and within 1e-5 relative unless cancelled more than tenfold (direct sum:
1e-6 relative), with the figures recorded per case; VJP 5e-6 of the magnitude sum."""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_04197_gb300 import inputs
from util import check_parity, oracle_node_order, preorder_from_oracle, preorder_from_topo

pytestmark = pytest.mark.gpu

N_HEAD = 1_048_576


@pytest.fixture(scope="module")
def head():
    pos, _, m = inputs.clumpy_plummer(N_HEAD, seed=0)
    return pos, m


def test_headline_tree_bitexact(gpu, head):
    pos, m = head
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    gpu.gravity_tree_build(ctx, P, M, gpu.params(order=2, leaf_max=16))
    gpu.gravity_sync(ctx)
    n = len(pos)
    root = gpu.gravity_debug_export(ctx, gpu.DBG_ROOT, 1)[0]
    lo, side = oracle.root_cube(pos)
    assert root[:3].tolist() == lo.tolist() and root[3] == side
    t = oracle.Tree(pos, m, leaf_max=16, order=2)
    okeys, operm = t.order_arrays()
    assert np.array_equal(gpu.gravity_debug_export(ctx, gpu.DBG_PERM, n).astype(np.int64), operm)
    keys = gpu.gravity_debug_export(ctx, gpu.DBG_KEYS, n)
    assert np.array_equal(keys, okeys)
    topo = gpu.gravity_debug_export(ctx, gpu.DBG_TOPO, n)
    depth = gpu.gravity_debug_export(ctx, gpu.DBG_DEPTH, n)
    assert preorder_from_topo(topo, depth, keys) == preorder_from_oracle(t.nodes())
    om, oc, _ = t.moments()
    ids = oracle_node_order(topo)
    assert np.array_equal(gpu.gravity_debug_export(ctx, gpu.DBG_MASS, n)[ids], om)
    assert np.array_equal(gpu.gravity_debug_export(ctx, gpu.DBG_COM, n)[ids], oc)


def test_headline_forces_sampled(gpu, head):
    pos, m = head
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    acc = torch.empty_like(P)
    cnt = torch.empty((len(pos), 3), dtype=torch.int32, device="cuda")
    gpu.gravity_tree_build(ctx, P, M, gpu.params(order=2, leaf_max=16))
    gpu.gravity_forces(ctx, 0.5, 1e-3, acc)                 # the timed kernel
    a_timed = acc.cpu().numpy()
    gpu.gravity_forces_counted(ctx, 0.5, 1e-3, acc, cnt)
    gpu.gravity_sync(ctx)
    assert np.array_equal(acc.cpu().numpy(), a_timed)
    idx = inputs.subset(len(pos), 65536, seed=11)
    ref, absum, ocnt = oracle.Tree(pos, m, leaf_max=16, order=2).forces(0.5, 1e-3, targets=idx)
    c = cnt.cpu().numpy()[idx]
    assert np.array_equal(c[:, 0], ocnt[:, 1]) and np.array_equal(c[:, 1], ocnt[:, 2])
    assert np.array_equal(c[:, 2], ocnt[:, 0])
    check_parity(a_timed[idx], ref, absum, "fullsize/clumpy1M/theta0.5/order2/leaf16")


@pytest.fixture(scope="module")
def head_oracle(head):
    pos, m = head
    return oracle.Tree(pos, m, leaf_max=16, order=2)


@pytest.mark.parametrize("theta,accum,order,leaf", [(0.3, 0, 2, 16), (0.7, 0, 2, 16),
                                                    (0.9, 0, 2, 16), (0.5, 1, 2, 16),
                                                    (0.5, 0, 0, 16), (0.5, 0, 0, 1)])
def test_headline_theta_sweep_sampled(gpu, head, head_oracle, theta, accum, order, leaf):
    # the other opening angles of the sweep, the FP64 accumulator and the monopole trees:
    # decision counts of 16,384 seeded bodies exact, forces within the parity tolerance
    pos, m = head
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    acc = torch.empty_like(P)
    cnt = torch.empty((len(pos), 3), dtype=torch.int32, device="cuda")
    gpu.gravity_tree_build(ctx, P, M, gpu.params(order=order, leaf_max=leaf, accum=accum))
    gpu.gravity_forces(ctx, theta, 1e-3, acc)
    a_timed = acc.cpu().numpy()
    gpu.gravity_forces_counted(ctx, theta, 1e-3, acc, cnt)
    gpu.gravity_sync(ctx)
    assert np.array_equal(acc.cpu().numpy(), a_timed)
    idx = inputs.subset(len(pos), 16384, seed=int(100 * theta) + accum + 7 * leaf + order)
    tree = head_oracle if (order, leaf) == (2, 16) else oracle.Tree(pos, m, leaf_max=leaf,
                                                                    order=order)
    ref, absum, ocnt = tree.forces(theta, 1e-3, targets=idx)
    c = cnt.cpu().numpy()[idx]
    assert np.array_equal(c[:, 0], ocnt[:, 1]) and np.array_equal(c[:, 1], ocnt[:, 2])
    assert np.array_equal(c[:, 2], ocnt[:, 0])
    check_parity(a_timed[idx], ref, absum,
                 f"fullsize/clumpy1M/theta{theta}/order{order}/leaf{leaf}/accum{accum}")


def test_headline_direct_sampled(gpu, head):
    pos, m = head
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    acc = torch.empty_like(P)
    gpu.gravity_direct(ctx, P, M, 1e-3, 1.0, acc)
    gpu.gravity_sync(ctx)
    idx = inputs.subset(len(pos), 4096, seed=12)
    ref, absum = oracle.direct(pos, m, 1e-3, targets=idx)
    check_parity(acc.cpu().numpy()[idx], ref, absum, "fullsize/clumpy1M/direct", rel_tol=1e-6)


def test_ensemble_sampled_clouds(gpu):
    off, pos, _, m = inputs.ensemble(nclouds=256, seed=100)
    ctx = gpu.Context(0)
    gpu.gravity_set_clouds(ctx, off)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    acc = torch.empty_like(P)
    cnt = torch.empty((len(pos), 3), dtype=torch.int32, device="cuda")
    gpu.gravity_tree_build(ctx, P, M, gpu.params(order=2, leaf_max=16))
    gpu.gravity_forces_counted(ctx, 0.5, 1e-3, acc, cnt)
    gpu.gravity_sync(ctx)
    a, c = acc.cpu().numpy(), cnt.cpu().numpy()
    sizes = np.diff(off)
    rng = np.random.default_rng(13)
    picks = {int(np.argmin(sizes)), int(np.argmax(sizes))} | set(rng.choice(256, 4, replace=False).tolist())
    for k in sorted(picks):
        b, e = int(off[k]), int(off[k + 1])
        loc = inputs.subset(e - b, min(512, e - b), seed=14 + k)
        ref, absum, ocnt = oracle.Tree(pos[b:e], m[b:e], leaf_max=16, order=2).forces(
            0.5, 1e-3, targets=loc)
        ck = c[b:e][loc]
        assert np.array_equal(ck[:, 0], ocnt[:, 1]) and np.array_equal(ck[:, 1], ocnt[:, 2]), k
        assert np.array_equal(ck[:, 2], ocnt[:, 0]), k
        check_parity(a[b:e][loc], ref, absum, f"fullsize/ensemble/cloud{k}")


def test_rubble_pile_run(gpu):
    pos, vel, m = inputs.rubble_pile(100_000, seed=0)
    eps, dt, theta = 5e-3, 1e-3, 0.5
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    V = torch.tensor(vel, device="cuda")
    M = torch.tensor(m, device="cuda")
    A = torch.empty_like(P)
    p = gpu.params(order=2, leaf_max=16)
    gpu.gravity_tree_build(ctx, P, M, p)
    gpu.gravity_forces(ctx, theta, eps, A)
    a0 = A.cpu().numpy()
    # one step against the oracle's step from the same state
    gpu.leapfrog_step(ctx, P, V, M, A, dt, 1, theta, eps, p)
    op, ov, _ = oracle.step(pos, vel, m, a0, dt, 1, theta=theta, eps=eps, order=2, leaf_max=16)
    assert np.abs(P.cpu().numpy() - op).max() < 1e-12
    assert np.abs(V.cpu().numpy() - ov).max() < 1e-9
    # the whole run: momentum moves only by the imbalance of the FP32 / tree forces,
    # energy stays within the leapfrog's bounded oscillation plus the tree's error
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    gpu.gravity_diagnostics(ctx, torch.tensor(pos, device="cuda"), torch.tensor(vel, device="cuda"),
                            M, eps, 1.0, out)
    d0 = out.cpu().numpy().copy()
    gpu.leapfrog_step(ctx, P, V, M, A, dt, 99, theta, eps, p)
    gpu.gravity_diagnostics(ctx, P, V, M, eps, 1.0, out)
    d1 = out.cpu().numpy()
    gpu.gravity_sync(ctx)
    sa = float(np.sum(m[:, None] * np.abs(a0)))
    assert np.abs(d1[1:4] - d0[1:4]).max() <= 1e-3 * 0.1 * sa     # tree force imbalance ~1e-3
    assert abs(d1[0] - d0[0]) <= 1e-3 * abs(d0[0]), (d0[0], d1[0])


def test_gradient_workload_vjp(gpu):
    pos, _, m = inputs.uniform_sphere(65_536, seed=200)
    lam = np.random.default_rng(15).standard_normal(pos.shape)
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    gpu.gravity_tree_build(ctx, P, M, gpu.params(order=0, leaf_max=1))
    out = torch.empty_like(P)
    gpu.gravity_forces_vjp(ctx, 0.5, 1e-3, torch.tensor(lam, device="cuda"), out)
    gpu.gravity_sync(ctx)
    ref, absum = oracle.tree_vjp(oracle.Tree(pos, m, leaf_max=1), lam, 0.5, 1e-3, with_absum=True)
    err = np.linalg.norm(out.cpu().numpy() - ref, axis=1) / np.maximum(absum, 1e-300)
    assert err.max() <= 5e-6, err.max()
