"""Batched ensemble: many independent clouds in one build and one walk launch.

Every cloud must come out exactly as if it had been built alone: each is compared
with an oracle tree of that cloud only (keys, order, topology and moments
bit-exact; decision counts exact; forces within the tolerances of the single-cloud
tests)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_04197_gb300 import inputs
from util import check_parity, oracle_node_order, preorder_from_oracle, preorder_from_topo

pytestmark = pytest.mark.gpu


def _ensemble(seed=3, nclouds=21, nmax=4096):
    off, pos, vel, m = inputs.ensemble(nclouds=nclouds, seed=seed, nmin=64, nmax=nmax)
    # odd cases: a one-body cloud, a two-body cloud, a cloud of coincident bodies
    extra = [np.array([[0.3, -0.2, 0.1]]), np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]),
             np.tile([[1.0, 2.0, 3.0]], (40, 1))]
    P = [pos] + extra
    V = [vel] + [np.zeros_like(e) for e in extra]
    M = [m] + [np.full(len(e), 1.0 / len(e)) for e in extra]
    sizes = list(np.diff(off)) + [len(e) for e in extra]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return off, np.concatenate(P), np.concatenate(V), np.concatenate(M)


def _build(g, off, pos, m, **kw):
    ctx = g.Context(0)
    g.gravity_batch_tree_build(ctx, off, torch.tensor(pos, device="cuda"),
                               torch.tensor(m, device="cuda"), g.params(**kw))
    g.gravity_sync(ctx)
    return ctx


@pytest.mark.parametrize("leaf_max,order,small", [(1, 0, False), (8, 2, False), (1, 0, True)])
def test_batch_tree_per_cloud_bitexact(gpu, leaf_max, order, small):
    # small: 8 clouds of fewer than 2048 bodies in all, sorted by one block (cloud passes too)
    off, pos, _, m = _ensemble(nclouds=8, nmax=300) if small else _ensemble()
    assert (len(pos) <= 2048) == small
    K = len(off) - 1
    ctx = _build(gpu, off, pos, m, leaf_max=leaf_max, order=order)
    n = len(pos)
    roots = gpu.gravity_debug_export(ctx, gpu.DBG_ROOT, K)
    keys = gpu.gravity_debug_export(ctx, gpu.DBG_KEYS, n)
    perm = gpu.gravity_debug_export(ctx, gpu.DBG_PERM, n).astype(np.int64)
    topo = gpu.gravity_debug_export(ctx, gpu.DBG_TOPO, n)
    depth = gpu.gravity_debug_export(ctx, gpu.DBG_DEPTH, n)
    parent = gpu.gravity_debug_export(ctx, gpu.DBG_PARENT, n)
    gm = gpu.gravity_debug_export(ctx, gpu.DBG_MASS, n)
    gc = gpu.gravity_debug_export(ctx, gpu.DBG_COM, n)
    assert np.all(parent[:K] == -1)
    for k in range(K):
        b, e = int(off[k]), int(off[k + 1])
        cp, cm = pos[b:e], m[b:e]
        lo, side = oracle.root_cube(cp)
        assert roots[k][:3].tolist() == lo.tolist() and roots[k][3] == side
        okeys = oracle.morton_keys(cp, lo, side)
        operm = oracle.stable_order(okeys)
        assert np.array_equal(perm[b:e] - b, operm)
        assert np.array_equal(keys[b:e], okeys[operm])
        t = oracle.Tree(cp, cm, leaf_max=leaf_max, order=order)
        # the cloud's subtree from its root (node k), ranges made cloud-relative
        sub = np.array(topo)
        sub[:, 2:] -= b
        got = preorder_from_topo_root(sub, depth, keys[b:e], k)
        assert got == preorder_from_oracle(t.nodes()), f"cloud {k}"
        om, oc, _ = t.moments()
        ids = node_order_from_root(topo, k)
        assert np.array_equal(gm[ids], om) and np.array_equal(gc[ids], oc), f"cloud {k}"


def preorder_from_topo_root(topo, depth, sorted_keys, root):
    out, stack = [], [root]
    while stack:
        k = stack.pop()
        fc, nc, b, e = (int(v) for v in topo[k])
        d = int(depth[k])
        prefix = 0 if d == 0 else int(sorted_keys[b]) >> (3 * (21 - d))
        out.append((d, prefix, b, e, nc if fc >= 0 else 0))
        if fc >= 0:
            stack.extend(range(fc + nc - 1, fc - 1, -1))
    return out


def node_order_from_root(topo, root):
    out, stack = [], [root]
    while stack:
        k = stack.pop()
        out.append(k)
        fc, nc = int(topo[k][0]), int(topo[k][1])
        if fc >= 0:
            stack.extend(range(fc + nc - 1, fc - 1, -1))
    return np.array(out, dtype=np.int64)


@pytest.mark.parametrize("theta,leaf_max,order", [(0.5, 1, 0), (0.5, 16, 2), (0.0, 8, 0)])
def test_batch_forces_per_cloud(gpu, theta, leaf_max, order):
    off, pos, _, m = _ensemble(seed=5)
    K = len(off) - 1
    ctx = _build(gpu, off, pos, m, leaf_max=leaf_max, order=order)
    acc = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
    cnt = torch.empty((len(pos), 3), dtype=torch.int32, device="cuda")
    gpu.gravity_forces_counted(ctx, theta, 1e-3, acc, cnt)
    gpu.gravity_sync(ctx)
    a, c = acc.cpu().numpy(), cnt.cpu().numpy()
    for k in range(K):
        b, e = int(off[k]), int(off[k + 1])
        ref, absum, oc = oracle.Tree(pos[b:e], m[b:e], leaf_max=leaf_max, order=order).forces(theta, 1e-3)
        assert np.array_equal(c[b:e, 0], oc[:, 1]) and np.array_equal(c[b:e, 1], oc[:, 2])
        assert np.array_equal(c[b:e, 2], oc[:, 0])
        check_parity(a[b:e], ref, np.maximum(absum, 1e-300),
                     f"batch/theta{theta}/leaf{leaf_max}/order{order}/cloud{k}")


def test_batch_leapfrog_per_cloud(gpu):
    off, pos, vel, m = _ensemble(seed=7)
    K = len(off) - 1
    eps, dt, theta, steps = 1e-3, 1e-3, 0.5, 5
    ctx = gpu.Context(0)
    gpu.gravity_set_clouds(ctx, off)
    P = torch.tensor(pos, device="cuda")
    V = torch.tensor(vel, device="cuda")
    M = torch.tensor(m, device="cuda")
    A = torch.empty_like(P)
    p = gpu.params(order=2, leaf_max=8)
    gpu.gravity_tree_build(ctx, P, M, p)
    gpu.gravity_forces(ctx, theta, eps, A)
    a0 = A.cpu().numpy()
    gpu.leapfrog_step(ctx, P, V, M, A, dt, steps, theta, eps, p)
    gpu.gravity_sync(ctx)
    gp, gv = P.cpu().numpy(), V.cpu().numpy()
    for k in range(K):
        b, e = int(off[k]), int(off[k + 1])
        op, ov, _ = oracle.step(pos[b:e], vel[b:e], m[b:e], a0[b:e], dt, steps, theta=theta,
                                eps=eps, order=2, leaf_max=8)
        assert np.abs(gp[b:e] - op).max() < 1e-9 and np.abs(gv[b:e] - ov).max() < 1e-6, k


def test_set_clouds_validation(gpu):
    ctx = gpu.Context(0)
    for bad in ([1, 5], [0, 5, 5], [0, 4, 3]):
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_set_clouds(ctx, bad)
        assert e.value.code == gpu.GRAVITY_E_ARG
    gpu.gravity_set_clouds(ctx, [0, 5, 9])
    P = torch.zeros((8, 3), dtype=torch.float64, device="cuda")
    M = torch.ones(8, dtype=torch.float64, device="cuda")
    with pytest.raises(gpu.GravityError):                 # n must match the segmentation
        gpu.gravity_tree_build(ctx, P, M)
    gpu.gravity_set_clouds(ctx, [0, 8])                   # back to a single cloud
    gpu.gravity_tree_build(ctx, P, M)
    gpu.gravity_sync(ctx)
