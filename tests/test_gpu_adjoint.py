"""Adjoint on the GPU: the frozen-tree vector-Jacobian product against the oracle's,
the checkpointed leapfrog reverse pass against the oracle's reverse pass on the same
positions, the whole adjoint against central differences of the frozen-decision map around
the GPU trajectory (theta > 0), and the gradient of the axis-ratio loss against finite
differences.

Tolerances.  The product's terms are FP32 (hi/lo or warp-relative coordinates, as the
forces), summed per body with two-sum compensation and per source by a 32-lane FP32
sum plus an FP64 atomic; each body's error is bounded by a small multiple of 2^-23
times the sum of the magnitudes of the terms it takes part in (the oracle's absum):
5e-6 of it is required for every body."""
import numpy as np
import pytest
import torch

import oracle
from util import PARITY_RECORDS
from paper_1912_04197_gb300 import inputs

pytestmark = pytest.mark.gpu

VJP_TOL = 5e-6


def _vjp_gpu(g, pos, m, lam, theta, eps, leaf_max, G=1.0, ctx=None):
    ctx = ctx or g.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    g.gravity_tree_build(ctx, P, M, g.params(leaf_max=leaf_max, order=0, G=G))
    out = torch.empty_like(P)
    g.gravity_forces_vjp(ctx, theta, eps, torch.tensor(lam, device="cuda"), out)
    g.gravity_sync(ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("kind,n,theta,eps,leaf_max,G", [
    ("sphere", 5000, 0.5, 1e-3, 1, 1.0),
    ("clumpy", 7777, 0.5, 1e-3, 16, 1.0),
    ("clumpy", 3001, 0.7, 0.0, 8, 1.3),
    ("sphere", 2049, 0.0, 1e-2, 4, 1.0),
    ("rubble", 4100, 0.3, 5e-3, 1, 0.7),
])
def test_vjp_matches_oracle(gpu, kind, n, theta, eps, leaf_max, G):
    if kind == "sphere":
        pos, _, m = inputs.uniform_sphere(n, seed=11)
    elif kind == "clumpy":
        pos, _, m = inputs.clumpy_plummer(n, seed=12, nclusters=8)
    else:
        pos, _, m = inputs.rubble_pile(n, seed=13)
    lam = np.random.default_rng(14).standard_normal(pos.shape)
    got = _vjp_gpu(gpu, pos, m, lam, theta, eps, leaf_max, G)
    ref, absum = oracle.tree_vjp(oracle.Tree(pos, m, leaf_max=leaf_max), lam, theta, eps, G,
                                 with_absum=True)
    err = np.linalg.norm(got - ref, axis=1) / np.maximum(absum, 1e-300)
    assert err.max() <= VJP_TOL, (err.max(), np.percentile(err, 99.9))
    # momentum-like invariant of the exact product: sum over bodies of the gradient is 0
    # (every term adds +w and -w); the GPU's sum vanishes to its rounding, a small
    # fraction of the total term magnitude (a dropped scatter would leave a large one)
    assert np.abs(got.sum(0)).max() <= 1e-6 * absum.sum()


def test_vjp_batched_per_cloud(gpu):
    off, pos, _, m = inputs.ensemble(nclouds=13, seed=21, nmin=40, nmax=3000)
    lam = np.random.default_rng(22).standard_normal(pos.shape)
    ctx = gpu.Context(0)
    gpu.gravity_set_clouds(ctx, off)
    got = _vjp_gpu(gpu, pos, m, lam, 0.5, 1e-3, 8, ctx=ctx)
    for k in range(len(off) - 1):
        b, e = int(off[k]), int(off[k + 1])
        ref, absum = oracle.tree_vjp(oracle.Tree(pos[b:e], m[b:e], leaf_max=8), lam[b:e], 0.5,
                                     1e-3, with_absum=True)
        err = np.linalg.norm(got[b:e] - ref, axis=1) / np.maximum(absum, 1e-300)
        assert err.max() <= VJP_TOL, (k, err.max())


def test_vjp_arguments(gpu):
    ctx = gpu.Context(0)
    P = torch.rand((100, 3), dtype=torch.float64, device="cuda")
    M = torch.full((100,), 0.01, dtype=torch.float64, device="cuda")
    L = torch.randn_like(P)
    out = torch.empty_like(P)
    with pytest.raises(gpu.GravityError) as e:
        gpu.gravity_forces_vjp(ctx, 0.5, 1e-3, L, out)
    assert e.value.code == gpu.GRAVITY_E_NOTREE
    gpu.gravity_tree_build(ctx, P, M, gpu.params(order=2))
    with pytest.raises(gpu.GravityError) as e:
        gpu.gravity_forces_vjp(ctx, 0.5, 1e-3, L, out)
    assert e.value.code == gpu.GRAVITY_E_ARG
    # one body: no terms, zero gradient
    gpu.gravity_tree_build(ctx, P[:1].contiguous(), M[:1].contiguous())
    o1 = torch.full((1, 3), 7.0, dtype=torch.float64, device="cuda")
    gpu.gravity_forces_vjp(ctx, 0.5, 1e-3, L[:1].contiguous(), o1)
    gpu.gravity_sync(ctx)
    assert torch.all(o1 == 0)


def _levels_gpu(g, pos, vel, m, dt, nsteps, theta, eps, leaf_max):
    """Positions after every step of the GPU integrator (steps taken one call at a time)."""
    ctx = g.Context(0)
    P = torch.tensor(pos, device="cuda")
    V = torch.tensor(vel, device="cuda")
    M = torch.tensor(m, device="cuda")
    A = torch.empty_like(P)
    p = g.params(leaf_max=leaf_max)
    g.gravity_tree_build(ctx, P, M, p)
    g.gravity_forces(ctx, theta, eps, A)
    levels = [P.cpu().numpy().copy()]
    for _ in range(nsteps):
        g.leapfrog_step(ctx, P, V, M, A, dt, 1, theta, eps, p)
        levels.append(P.cpu().numpy().copy())
    g.gravity_sync(ctx)
    return levels, P.cpu().numpy(), V.cpu().numpy()


@pytest.mark.parametrize("theta,leaf_max,nsteps,every", [(0.5, 1, 12, 5), (0.6, 8, 7, 7),
                                                          (0.0, 4, 4, 1)])
def test_leapfrog_adjoint_matches_oracle_reverse(gpu, theta, leaf_max, nsteps, every):
    from paper_1912_04197_gb300.adjoint import leapfrog
    pos, vel, m = inputs.rubble_pile(1500, seed=31)
    dt, eps = 1e-3, 5e-3
    levels, xN, vN = _levels_gpu(gpu, pos, vel, m, dt, nsteps, theta, eps, leaf_max)
    rng = np.random.default_rng(32)
    xbar, vbar = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)
    x0 = torch.tensor(pos, device="cuda", requires_grad=True)
    v0 = torch.tensor(vel, device="cuda", requires_grad=True)
    M = torch.tensor(m, device="cuda")
    x, v = leapfrog(x0, v0, M, dt, nsteps, theta=theta, eps=eps, leaf_max=leaf_max,
                    checkpoint_every=every)
    # the checkpointed forward is the step-by-step trajectory, bit for bit
    assert np.array_equal(x.detach().cpu().numpy(), xN)
    assert np.array_equal(v.detach().cpu().numpy(), vN)
    gx, gv = torch.autograd.grad((x, v), (x0, v0), (torch.tensor(xbar, device="cuda"),
                                                    torch.tensor(vbar, device="cuda")))
    rx, rv = oracle.leapfrog_reverse(levels, m, xbar, vbar, dt, theta=theta, eps=eps,
                                     leaf_max=leaf_max)
    gx, gv = gx.cpu().numpy(), gv.cpu().numpy()
    # without forces the reverse pass is xbar, vbar + N dt xbar; compare the part the
    # products add (the per-level errors are <= VJP_TOL of each product's magnitudes)
    fx, fv = xbar, vbar + nsteps * dt * xbar
    for got, ref, free in ((gx, rx, fx), (gv, rv, fv)):
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref - free)
        assert rel <= 2e-5, rel


def _loss_fd(g, pos, vel, m, dt, nsteps, theta, eps, leaf_max, directions, h):
    """Central differences of the axis-ratio loss of the GPU forward along directions
    (each a pair (dx, dv))."""
    from paper_1912_04197_gb300.loss import axis_ratio_loss
    ctx = g.Context(0)
    M = torch.tensor(m, device="cuda")
    p = g.params(leaf_max=leaf_max)

    def loss(x, v):
        P = torch.tensor(x, device="cuda")
        V = torch.tensor(v, device="cuda")
        A = torch.empty_like(P)
        g.gravity_tree_build(ctx, P, M, p)
        g.gravity_forces(ctx, theta, eps, A)
        g.leapfrog_step(ctx, P, V, M, A, dt, nsteps, theta, eps, p)
        return float(axis_ratio_loss(P, M))

    return np.array([(loss(pos + h * dx, vel + h * dv) - loss(pos - h * dx, vel - h * dv))
                     / (2 * h) for dx, dv in directions])


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_loss_gradient_vs_finite_differences(gpu, theta):
    """The loss is a function of the eigenvalues of S, nearly degenerate for a round cloud,
    so a central difference converges to the derivative only for steps well below the
    eigenvalue gaps (an O(h^2) error that is large at h = 1e-3 along affine directions).
    theta = 0 (the exact sum) is smooth: smooth (affine) directions at h = 1e-5 must agree
    to 1e-4 relative.  At theta = 0.5 the forward map is only piecewise smooth (opening
    decisions flip under the perturbation); the adjoint is the derivative with the
    decisions frozen, checked against differences relative to the largest derivative a
    direction of that norm can have."""
    from paper_1912_04197_gb300.adjoint import leapfrog
    from paper_1912_04197_gb300.loss import axis_ratio_loss
    pos, vel, m = inputs.rubble_pile(4096, seed=41)
    dt, eps, nsteps, leaf = 1e-3, 5e-3, 40, 1
    x0 = torch.tensor(pos, device="cuda", requires_grad=True)
    v0 = torch.tensor(vel, device="cuda", requires_grad=True)
    M = torch.tensor(m, device="cuda")
    x, _ = leapfrog(x0, v0, M, dt, nsteps, theta=theta, eps=eps, leaf_max=leaf,
                    checkpoint_every=20)
    L = axis_ratio_loss(x, M)
    gx, gv = torch.autograd.grad(L, (x0, v0))
    gx, gv = gx.cpu().numpy(), gv.cpu().numpy()
    rng = np.random.default_rng(42)
    gnorm = np.sqrt((gx * gx).sum() + (gv * gv).sum())
    if theta == 0.0:
        dirs = [(pos @ rng.standard_normal((3, 3)).T, pos @ rng.standard_normal((3, 3)).T)
                for _ in range(3)]
        fd = _loss_fd(gpu, pos, vel, m, dt, nsteps, theta, eps, leaf, dirs, h=1e-5)
        ad = np.array([(gx * dx).sum() + (gv * dv).sum() for dx, dv in dirs])
        rel = np.abs(fd - ad) / np.abs(ad)
        assert np.all(rel <= 1e-4), (rel, fd, ad)
    else:
        dirs = [(rng.standard_normal(pos.shape), rng.standard_normal(pos.shape))
                for _ in range(3)]
        dirs.append((gx / np.abs(gx).max(), gv / np.abs(gx).max()))   # along the gradient
        fd = _loss_fd(gpu, pos, vel, m, dt, nsteps, theta, eps, leaf, dirs, h=1e-4)
        ad = np.array([(gx * dx).sum() + (gv * dv).sum() for dx, dv in dirs])
        scale = np.array([gnorm * np.sqrt((dx * dx).sum() + (dv * dv).sum()) for dx, dv in dirs])
        rel = np.abs(fd - ad) / scale
        assert np.all(rel <= 1e-4), (rel, fd, ad)
        assert abs(fd[-1] - ad[-1]) <= 1e-3 * abs(ad[-1])   # along the gradient, plain relative


@pytest.mark.parametrize("theta,leaf_max", [(0.5, 1), (0.7, 8)])
def test_adjoint_matches_frozen_differences_on_gpu_trajectory(gpu, theta, leaf_max):
    # The GPU adjoint differentiates the GPU leapfrog with every step's opening decisions
    # frozen at that step's tree.  The oracle builds the same trees from the GPU levels (the
    # GPU's decisions are the FP64 ones, so they are the same decisions), and a KDK run whose
    # forces come from those frozen trees at the perturbed positions is a smooth map of
    # (x0, v0): its central differences are the derivative the adjoint must give, with no
    # decision flips in between.  The GPU products carry FP32 term rounding (<= 5e-6 of
    # each product's magnitudes), so the directional derivatives must agree to 1e-4 of
    # their own size along the gradient, and to 1e-5 of the magnitude sum along random
    # directions.
    from paper_1912_04197_gb300.adjoint import leapfrog
    pos, vel, m = inputs.rubble_pile(1500, seed=33)
    dt, eps, nsteps = 1e-3, 5e-3, 12
    levels, _, _ = _levels_gpu(gpu, pos, vel, m, dt, nsteps, theta, eps, leaf_max)
    rng = np.random.default_rng(34)
    cx, cv = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)
    x0 = torch.tensor(pos, device="cuda", requires_grad=True)
    v0 = torch.tensor(vel, device="cuda", requires_grad=True)
    M = torch.tensor(m, device="cuda")
    x, v = leapfrog(x0, v0, M, dt, nsteps, theta=theta, eps=eps, leaf_max=leaf_max,
                    checkpoint_every=5)
    gx, gv = torch.autograd.grad((x, v), (x0, v0), (torch.tensor(cx, device="cuda"),
                                                    torch.tensor(cv, device="cuda")))
    gx, gv = gx.cpu().numpy(), gv.cpu().numpy()
    trees = [oracle.Tree(xk, m, leaf_max=leaf_max) for xk in levels]

    def L(xa, va):
        xa, va = xa.copy(), va.copy()
        a = oracle.tree_forces_frozen(trees[0], xa, theta, eps)
        for k in range(nsteps):
            va = va + (0.5 * dt) * a
            xa = xa + dt * va
            a = oracle.tree_forces_frozen(trees[k + 1], xa, theta, eps)
            va = va + (0.5 * dt) * a
        return (cx * xa).sum() + (cv * va).sum()

    h = 1e-6
    dirs = [(rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)) for _ in range(3)]
    dirs.append((gx, gv))
    rels = []
    PARITY_RECORDS[f"adjoint_vs_frozen_differences_theta{theta}_leaf{leaf_max}"] = rels
    for k, (ex, ev) in enumerate(dirs):
        fd = (L(pos + h * ex, vel + h * ev) - L(pos - h * ex, vel - h * ev)) / (2 * h)
        an = (gx * ex).sum() + (gv * ev).sum()
        if k == len(dirs) - 1:
            rels.append(abs(fd - an) / abs(an))
            assert rels[-1] <= 1e-4, (rels, fd, an)
        else:
            rels.append(abs(fd - an) / (np.abs(gx * ex).sum() + np.abs(gv * ev).sum()))
            assert rels[-1] <= 1e-5, (rels, fd, an)
