"""GPU tree build (kernels 1-4 of the paper's list, Sec. 2.1) against the oracle:
keys, sort order, topology, node mass and centre of mass bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_04197_gb300 import inputs
from util import preorder_from_oracle, preorder_from_topo, oracle_node_order

pytestmark = pytest.mark.gpu


def _build(g, pos, mass, **kw):
    ctx = g.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(mass, device="cuda")
    g.gravity_tree_build(ctx, P, M, g.params(**kw))
    g.gravity_sync(ctx)
    return ctx


def _cases():
    return {
        "sphere2048": inputs.uniform_sphere(2048, seed=0),
        "sphere2085": inputs.uniform_sphere(2085, seed=1),          # ragged tail
        "clumpy100k": inputs.clumpy_plummer(100_003, seed=2, nclusters=16),
        "cube_dups": _dups(),
        "cube_dups_1tile": _dups(1500),                            # the one-block sort
        "sphere17": inputs.uniform_sphere(17, seed=4),
    }


def _dups(n=5000):
    pos, vel, m = inputs.uniform_cube(n, seed=3)
    pos[100:400] = pos[7]                                          # identical keys
    pos[1000:1003] = pos[n - 7]
    return pos, vel, m


@pytest.mark.parametrize("case", ["sphere2048", "sphere2085", "clumpy100k", "cube_dups",
                                  "cube_dups_1tile", "sphere17"])
def test_keys_and_order_bitexact(gpu, case):
    pos, _, m = _cases()[case]
    ctx = _build(gpu, pos, m)
    n = len(pos)
    root = gpu.gravity_debug_export(ctx, gpu.DBG_ROOT, 1)[0]
    lo, side = oracle.root_cube(pos)
    assert root[:3].tolist() == lo.tolist() and root[3] == side
    keys = gpu.gravity_debug_export(ctx, gpu.DBG_KEYS, n)
    perm = gpu.gravity_debug_export(ctx, gpu.DBG_PERM, n).astype(np.int64)
    okeys = oracle.morton_keys(pos, lo, side)
    operm = oracle.stable_order(okeys)
    assert np.array_equal(perm, operm)
    assert np.array_equal(keys, okeys[operm])


@pytest.mark.parametrize("case", ["sphere2085", "clumpy100k", "cube_dups", "cube_dups_1tile"])
@pytest.mark.parametrize("leaf_max", [1, 8, 16])
def test_topology_bitexact(gpu, case, leaf_max):
    pos, _, m = _cases()[case]
    ctx = _build(gpu, pos, m, leaf_max=leaf_max)
    n = len(pos)
    topo = gpu.gravity_debug_export(ctx, gpu.DBG_TOPO, n)
    depth = gpu.gravity_debug_export(ctx, gpu.DBG_DEPTH, n)
    keys = gpu.gravity_debug_export(ctx, gpu.DBG_KEYS, n)
    parent = gpu.gravity_debug_export(ctx, gpu.DBG_PARENT, n)
    t = oracle.Tree(pos, m, leaf_max=leaf_max)
    want = preorder_from_oracle(t.nodes())
    got = preorder_from_topo(topo, depth, keys)
    assert len(got) == len(want) == len(topo)
    assert got == want
    # parent pointers are consistent with the child ranges
    for k in range(len(topo)):
        fc, nc = topo[k][0], topo[k][1]
        if fc >= 0:
            assert np.all(parent[fc:fc + nc] == k)
    assert parent[0] == -1


@pytest.mark.parametrize("case", ["sphere2085", "clumpy100k", "cube_dups", "cube_dups_1tile"])
@pytest.mark.parametrize("leaf_max,order", [(1, 0), (8, 2), (16, 2)])
def test_moments_bitexact(gpu, case, leaf_max, order):
    pos, _, m = _cases()[case]
    if case == "clumpy100k":
        m = m * np.random.default_rng(4).lognormal(0, 0.5, len(m))
    ctx = _build(gpu, pos, m, leaf_max=leaf_max, order=order)
    n = len(pos)
    topo = gpu.gravity_debug_export(ctx, gpu.DBG_TOPO, n)
    gm = gpu.gravity_debug_export(ctx, gpu.DBG_MASS, n)
    gc = gpu.gravity_debug_export(ctx, gpu.DBG_COM, n)
    t = oracle.Tree(pos, m, leaf_max=leaf_max, order=order)
    om, oc, oq = t.moments()
    order_ids = oracle_node_order(topo)
    assert np.array_equal(gm[order_ids], om)
    assert np.array_equal(gc[order_ids], oc)
    if order == 2:
        # the GPU carries T = sum m y y^T up the tree (same value in exact arithmetic,
        # other roundings): compare on the node's natural scale m l^2
        gq = gpu.gravity_debug_export(ctx, gpu.DBG_QUAD, n)[order_ids]
        depth = gpu.gravity_debug_export(ctx, gpu.DBG_DEPTH, n)[order_ids]
        side = gpu.gravity_debug_export(ctx, gpu.DBG_ROOT, 1)[0][3]
        scale = (om * (side * 2.0 ** -depth.astype(np.float64)) ** 2)[:, None]
        assert np.all(np.abs(gq - oq) <= 1e-12 * scale)


def test_single_and_coincident(gpu):
    ctx = _build(gpu, np.array([[0.5, -2.0, 3.0]]), np.array([2.0]))
    topo = gpu.gravity_debug_export(ctx, gpu.DBG_TOPO, 1)
    assert topo.tolist() == [[-1, 0, 0, 1]]
    same = np.tile([[0.25, 0.5, -0.75]], (100, 1))
    ctx = _build(gpu, same, np.ones(100))
    topo = gpu.gravity_debug_export(ctx, gpu.DBG_TOPO, 100)
    depth = gpu.gravity_debug_export(ctx, gpu.DBG_DEPTH, 100)
    assert topo.tolist() == [[-1, 0, 0, 100]] and depth.tolist() == [21]
    root = gpu.gravity_debug_export(ctx, gpu.DBG_ROOT, 1)[0]
    assert root[3] == 1.0


@pytest.mark.parametrize("n", [3000, 500])             # several tiles; one block (n <= 2048)
def test_nonfinite_is_reported(gpu, n):
    pos, _, m = inputs.uniform_sphere(n, seed=5)
    for bad in (np.nan, np.inf, -np.inf):
        p = pos.copy()
        p[n // 3, 1] = bad
        ctx = gpu.Context(0)
        gpu.gravity_tree_build(ctx, torch.tensor(p, device="cuda"), torch.tensor(m, device="cuda"))
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_sync(ctx)
        assert e.value.code == gpu.GRAVITY_E_NONFINITE
        gpu.gravity_sync(ctx)                       # the latched error is cleared


def test_argument_errors(gpu):
    ctx = gpu.Context(0)
    acc = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu.GravityError) as e:
        gpu.gravity_forces(ctx, 0.5, 0.1, acc)
    assert e.value.code == gpu.GRAVITY_E_NOTREE
    P = torch.rand((10, 3), dtype=torch.float64, device="cuda")
    M = torch.ones(10, dtype=torch.float64, device="cuda")
    for kw in ({"leaf_max": 0}, {"leaf_max": 65}, {"order": 1}, {"accum": 2}):
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_tree_build(ctx, P, M, gpu.params(**kw))
        assert e.value.code == gpu.GRAVITY_E_ARG
    gpu.gravity_tree_build(ctx, P, M)
    for th, ep in ((-0.1, 0.1), (0.5, -1.0), (float("nan"), 0.1)):
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_forces(ctx, th, ep, acc)
        assert e.value.code == gpu.GRAVITY_E_ARG
    # n = 0 is a no-op
    gpu.gravity_tree_build(ctx, P[:0], M[:0])
    gpu.gravity_forces(ctx, 0.5, 0.1, acc[:0])
    gpu.gravity_sync(ctx)
