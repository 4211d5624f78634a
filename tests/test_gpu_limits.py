"""The size and shape limits of the library: the largest body count (2^24, node indices
in the walk's 25-bit fields), the largest leaf bucket (64), and depth-21 buckets of many
identical keys.  Sampled outputs against the oracle, as the full-size tests."""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_04197_gb300 import inputs
from util import check_parity

pytestmark = pytest.mark.gpu


def _sampled(g, pos, m, theta, ntarg, seed, **kw):
    ctx = g.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    A = torch.empty_like(P)
    cnt = torch.empty((len(pos), 3), dtype=torch.int32, device="cuda")
    g.gravity_tree_build(ctx, P, M, g.params(**kw))
    g.gravity_forces_counted(ctx, theta, 1e-3, A, cnt)
    g.gravity_sync(ctx)
    idx = inputs.subset(len(pos), ntarg, seed=seed)
    a, c = A.cpu().numpy()[idx], cnt.cpu().numpy()[idx]
    del P, M, A, cnt, ctx
    t = oracle.Tree(pos, m, leaf_max=kw.get("leaf_max", 1), order=kw.get("order", 0))
    ref, absum, ocnt = t.forces(theta, 1e-3, targets=idx)
    assert np.array_equal(c[:, 0], ocnt[:, 1]) and np.array_equal(c[:, 1], ocnt[:, 2])
    assert np.array_equal(c[:, 2], ocnt[:, 0])
    check_parity(a, ref, absum, f"limits/n{len(pos)}/" + "/".join(f"{k}{v}" for k, v in sorted(kw.items())))


def test_largest_body_count(gpu):
    n = 1 << 24
    pos, _, m = inputs.clumpy_plummer(n, seed=21)
    _sampled(gpu, pos, m, 0.5, 1024, seed=22, order=2, leaf_max=16)
    ctx = gpu.Context(0)
    with pytest.raises(gpu.GravityError) as e:           # one more body is refused
        gpu.gravity_tree_build(ctx, torch.zeros((n + 1, 3), dtype=torch.float64, device="cuda"),
                               torch.ones(n + 1, dtype=torch.float64, device="cuda"))
    assert e.value.code == gpu.GRAVITY_E_ARG


@pytest.mark.parametrize("leaf_max", [33, 64])
def test_largest_leaves(gpu, leaf_max):
    pos, _, m = inputs.clumpy_plummer(200_000, seed=23, nclusters=8)
    _sampled(gpu, pos, m, 0.6, 2048, seed=24, order=2, leaf_max=leaf_max)


def test_big_identical_key_buckets(gpu):
    # runs of identical positions give depth-21 buckets far larger than leaf_max
    pos, _, m = inputs.uniform_cube(60_000, seed=25)
    pos[1000:1500] = pos[3]
    pos[20000:20100] = pos[5] + 1e-12                 # same grid cell, not identical
    pos[40000:40070] = pos[7]
    _sampled(gpu, pos, m, 0.5, 2048, seed=26, order=2, leaf_max=16)
