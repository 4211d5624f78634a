"""Aggregate identification on the GPU (contact-graph components over the gravity tree)
against the oracle's depth-first search on all pairs: labels and counts bit-exact (every
edge is an FP64 pairwise test made as the oracle makes it); clouds never join across;
full size against brute-force neighbours of sampled bodies; errors from the host."""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_04197_gb300 import inputs

pytestmark = pytest.mark.gpu


def _gpu_components(g, pos, m, radius=None, dmax=0.0, ctx=None, **kw):
    ctx = ctx or g.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    g.gravity_tree_build(ctx, P, M, g.params(**kw))
    label = torch.empty(len(pos), dtype=torch.int32, device="cuda")
    counts = torch.empty(2, dtype=torch.int64, device="cuda")
    R = None if radius is None else torch.tensor(radius, device="cuda")
    g.gravity_components(ctx, label, radius=R, dmax=dmax, counts=counts)
    g.gravity_sync(ctx)
    return label.cpu().numpy(), tuple(int(x) for x in counts.cpu())


@pytest.mark.parametrize("leaf_max,order", [(1, 0), (16, 2), (64, 0)])
@pytest.mark.parametrize("dmax", [0.0, 0.004, 0.02])
def test_uniform_threshold_vs_oracle(gpu, leaf_max, order, dmax):
    pos, _, m = inputs.clumpy_plummer(20_000, seed=41, nclusters=8)
    label, counts = _gpu_components(gpu, pos, m, dmax=dmax, leaf_max=leaf_max, order=order)
    ref, rcounts = oracle.components(pos, dmax=dmax)
    assert np.array_equal(label, ref)
    assert counts == rcounts


def test_radii_vs_oracle(gpu):
    pos, _, m = inputs.rubble_pile(15_000, seed=42)
    radius = 0.6 * np.cbrt(m / m.mean()) * 0.02                 # sizes from the masses
    radius[7] = 0.0                                            # a point body
    label, counts = _gpu_components(gpu, pos, m, radius=radius, leaf_max=8)
    ref, rcounts = oracle.components(pos, radius=radius)
    assert np.array_equal(label, ref) and counts == rcounts
    assert 1 < rcounts[1] < rcounts[0]


def test_exact_boundary_and_duplicates(gpu):
    # touching at exactly dmax joins; identical positions (distance 0) join
    pos = np.array([[0, 0, 0], [0.25, 0, 0], [0.625, 0, 0], [0.625, 0, 0], [2, 2, 2], [0, 0, 1]],
                   float)
    m = np.ones(len(pos))
    for dmax in (0.25, 0.375, 0.0):
        label, counts = _gpu_components(gpu, pos, m, dmax=dmax)
        ref, rcounts = oracle.components(pos, dmax=dmax)
        assert np.array_equal(label, ref) and counts == rcounts, dmax


def test_clouds_never_join(gpu):
    # five clouds drawn around the same centre: across clouds bodies overlap in space,
    # but components are per cloud
    clouds = [inputs.uniform_sphere(n, seed=50 + k)[0] * 0.2 for k, n in
              enumerate((700, 1, 2500, 64, 1200))]
    off = np.concatenate([[0], np.cumsum([len(c) for c in clouds])])
    pos = np.concatenate(clouds)
    m = np.ones(len(pos))
    ctx = gpu.Context(0)
    gpu.gravity_set_clouds(ctx, off)
    label, counts = _gpu_components(gpu, pos, m, dmax=0.03, ctx=ctx, leaf_max=4)
    tot = [0, 0]
    for k in range(len(clouds)):
        b, e = off[k], off[k + 1]
        ref, rc = oracle.components(pos[b:e], dmax=0.03)
        assert np.array_equal(label[b:e], ref + b), k
        tot[0] += rc[0]
        tot[1] += rc[1]
    assert counts == tuple(tot)


def test_headline_aggregate_sampled(gpu):
    # 1,048,576 clumpy bodies: every sampled body's brute-force neighbours share its label,
    # the labelling is canonical, and the counts match the labels
    pos, _, m = inputs.clumpy_plummer(1_048_576, seed=0)
    dmax = 1e-3
    label, counts = _gpu_components(gpu, pos, m, dmax=dmax, leaf_max=16, order=2)
    idx = np.arange(len(pos))
    assert np.all(label <= idx) and np.array_equal(label[label], label)
    uniq, mult = np.unique(label, return_counts=True)
    assert counts == (len(uniq), int((mult > 1).sum()))
    for i in inputs.subset(len(pos), 256, seed=43):
        d = pos - pos[i]
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        nb = np.nonzero(d2 <= dmax * dmax)[0]
        assert np.all(label[nb] == label[i]), i


def test_errors(gpu):
    ctx = gpu.Context(0)
    label = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(gpu.GravityError) as e:
        gpu.gravity_components(ctx, label, dmax=0.1)            # no tree yet
    assert e.value.code == gpu.GRAVITY_E_NOTREE
    pos, _, m = inputs.uniform_sphere(4, seed=44)
    gpu.gravity_tree_build(ctx, torch.tensor(pos, device="cuda"), torch.tensor(m, device="cuda"))
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_components(ctx, label, dmax=bad)
        assert e.value.code == gpu.GRAVITY_E_ARG
    r = torch.tensor([0.1, float("nan"), 0.1, 0.1], dtype=torch.float64, device="cuda")
    gpu.gravity_components(ctx, label, radius=r)
    with pytest.raises(gpu.GravityError) as e:
        gpu.gravity_sync(ctx)                                  # the bad radius is latched
    assert e.value.code == gpu.GRAVITY_E_NONFINITE
    gpu.gravity_components(ctx, label, dmax=0.0)               # the context stays usable
    gpu.gravity_sync(ctx)
    assert label.cpu().tolist() == [0, 1, 2, 3]


def test_dt_g_closed_form(gpu):
    # Eq. (dt_g): 1 / (2 sqrt(G rho)); for asteroid material densities of 1 to 4 g/cm^3
    # (SI units) the bound is of the order of a thousand seconds, as Sec. 4.1 states
    G = 6.674e-11
    assert gpu.gravity_dt_g(G, 2000.0) == 0.5 / np.sqrt(G * 2000.0)
    assert 1.9e3 < gpu.gravity_dt_g(G, 1000.0) < 2.0e3
    assert 9.5e2 < gpu.gravity_dt_g(G, 4000.0) < 1.0e3
    assert gpu.gravity_dt_g(G, 4000.0) * 2 == pytest.approx(gpu.gravity_dt_g(G, 1000.0), rel=1e-15)
    for bad in ((0.0, 1.0), (1.0, -1.0), (float("nan"), 1.0), (1.0, float("inf"))):
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_dt_g(*bad)
        assert e.value.code == gpu.GRAVITY_E_ARG
