"""Pins of the oracle's adjoint (vector-Jacobian product on the frozen tree, and the
reverse pass of the leapfrog) against finite differences and a symmetry of the
Jacobian that the mathematics fixes."""
import numpy as np
import pytest

import oracle
from paper_1912_04197_gb300 import inputs

pytestmark = pytest.mark.oracle


@pytest.mark.parametrize("theta,leaf_max,eps", [(0.0, 1, 1e-2), (0.5, 1, 1e-2), (0.7, 8, 0.0)])
def test_vjp_matches_frozen_finite_differences(theta, leaf_max, eps):
    pos, _, m = inputs.uniform_sphere(600, seed=1)
    m = m * np.random.default_rng(2).lognormal(0, 0.3, len(m))
    t = oracle.Tree(pos, m, leaf_max=leaf_max)
    rng = np.random.default_rng(3)
    lam = rng.standard_normal(pos.shape)
    g = oracle.tree_vjp(t, lam, theta, eps, G=1.3)
    h = 1e-6
    for _ in range(4):
        e = rng.standard_normal(pos.shape)
        fp = oracle.tree_forces_frozen(t, pos + h * e, theta, eps, G=1.3)
        fm = oracle.tree_forces_frozen(t, pos - h * e, theta, eps, G=1.3)
        fd = ((fp - fm) * lam).sum() / (2 * h)
        assert abs(fd - (g * e).sum()) <= 1e-6 * np.abs(g * e).sum(), (fd, (g * e).sum())
    # the frozen force at the tree's own positions is the ordinary tree force
    a0 = oracle.tree_forces(pos, m, theta, eps, 1.3, leaf_max=leaf_max)
    assert np.allclose(oracle.tree_forces_frozen(t, pos, theta, eps, G=1.3), a0, rtol=0,
                       atol=1e-12 * np.abs(a0).max())


def test_direct_jacobian_mass_symmetry():
    # M (d a / d x) is symmetric for the direct sum: m_i m_j J(d_ij) with J even and
    # symmetric, so u^T M J w = w^T M J u for any u, w
    pos, _, _ = inputs.uniform_sphere(300, seed=4)
    m = np.random.default_rng(5).random(300) + 0.2
    t = oracle.Tree(pos, m)
    rng = np.random.default_rng(6)
    u, w = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)
    lhs = (oracle.tree_vjp(t, m[:, None] * u, 0.0, 0.05) * w).sum()
    rhs = (oracle.tree_vjp(t, m[:, None] * w, 0.0, 0.05) * u).sum()
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + abs(rhs))


def test_leapfrog_gradient_matches_finite_differences_direct():
    # theta = 0: the dynamics is smooth (no decisions), so finite differences of the
    # whole simulation check the reverse pass
    pos, vel, m = inputs.rubble_pile(150, seed=8)
    dt, ns, eps = 2e-3, 12, 5e-2
    rng = np.random.default_rng(9)
    cx, cv = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)

    def L(x0, v0):
        a = oracle.tree_forces(x0, m, 0.0, eps)
        x, v, _ = oracle.step(x0, v0, m, a, dt, ns, theta=0.0, eps=eps)
        return (cx * x).sum() + (cv * v).sum()

    gx, gv = oracle.leapfrog_grad(pos, vel, m, cx, cv, dt, ns, theta=0.0, eps=eps)
    h = 1e-6
    for _ in range(3):
        ex, ev = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)
        fd = (L(pos + h * ex, vel + h * ev) - L(pos - h * ex, vel - h * ev)) / (2 * h)
        an = (gx * ex).sum() + (gv * ev).sum()
        assert abs(fd - an) <= 1e-6 * (np.abs(gx * ex).sum() + np.abs(gv * ev).sum()), (fd, an)


@pytest.mark.parametrize("theta,leaf_max", [(0.5, 1), (0.7, 4)])
def test_leapfrog_gradient_matches_frozen_finite_differences_tree(theta, leaf_max):
    # theta > 0: the reverse pass differentiates with every step's opening decisions frozen
    # (those of the trees of the unperturbed trajectory).  A forward run whose forces come
    # from those frozen trees (tree_forces_frozen at the perturbed positions) is a smooth
    # map, so its central differences check the whole reverse pass, decisions and all
    pos, vel, m = inputs.rubble_pile(150, seed=18)
    dt, ns, eps = 2e-3, 12, 5e-2
    rng = np.random.default_rng(19)
    cx, cv = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)
    a0 = oracle.tree_forces(pos, m, theta, eps, leaf_max=leaf_max)
    levels, x, v, a = [pos.copy()], pos.copy(), vel.copy(), a0
    for _ in range(ns):
        x, v, a = oracle.step(x, v, m, a, dt, 1, theta=theta, eps=eps, leaf_max=leaf_max)
        levels.append(x.copy())
    trees = [oracle.Tree(xk, m, leaf_max=leaf_max) for xk in levels]

    def L(x0, v0):
        # KDK leapfrog with each level's forces from that level's frozen tree
        x, v = x0.copy(), v0.copy()
        a = oracle.tree_forces_frozen(trees[0], x, theta, eps)
        for k in range(ns):
            v = v + (0.5 * dt) * a
            x = x + dt * v
            a = oracle.tree_forces_frozen(trees[k + 1], x, theta, eps)
            v = v + (0.5 * dt) * a
        return (cx * x).sum() + (cv * v).sum()

    # at zero perturbation the frozen run is the ordinary run
    assert abs(L(pos, vel) - ((cx * levels[-1]).sum() + (cv * v).sum())) <= 1e-12 * (
        np.abs(cx * levels[-1]).sum() + np.abs(cv * v).sum())
    gx, gv = oracle.leapfrog_grad(pos, vel, m, cx, cv, dt, ns, theta=theta, eps=eps,
                                  leaf_max=leaf_max)
    h = 1e-6
    for _ in range(3):
        ex, ev = rng.standard_normal(pos.shape), rng.standard_normal(pos.shape)
        fd = (L(pos + h * ex, vel + h * ev) - L(pos - h * ex, vel - h * ev)) / (2 * h)
        an = (gx * ex).sum() + (gv * ev).sum()
        assert abs(fd - an) <= 1e-6 * (np.abs(gx * ex).sum() + np.abs(gv * ev).sum()), (fd, an)


def test_vjp_absum_two_body_closed_form():
    # two bodies, d = x1 - x0: body 0 takes part in its own term (source 1, cotangent
    # u0) and as the source of body 1's term (cotangent u1), so its magnitude sum is
    # m1 |J(d) u0| + m0 |J(d) u1|, J = (I - 3 d d^T / r^2) / r^3, r^2 = |d|^2 + eps^2
    x = np.array([[0.1, -0.2, 0.3], [0.7, 0.4, -0.5]])
    m = np.array([0.3, 1.7])
    u = np.array([[1.0, -2.0, 0.5], [0.25, 0.75, -1.5]])
    eps = 0.05
    d = x[1] - x[0]
    r2 = d @ d + eps * eps
    J = (np.eye(3) - 3.0 * np.outer(d, d) / r2) / r2 ** 1.5
    g, a = oracle.tree_vjp(oracle.Tree(x, m), u, 0.0, eps, with_absum=True)
    w0, w1 = m[1] * J @ u[0], m[0] * J @ u[1]      # terms of body 0 and of body 1
    assert np.allclose(g[0], -w0 + w1, rtol=1e-14, atol=0)
    assert np.allclose(g[1], -w1 + w0, rtol=1e-14, atol=0)
    want = np.linalg.norm(w0) + np.linalg.norm(w1)
    assert np.allclose(a, [want, want], rtol=1e-14, atol=0)


def test_vjp_absum_bounds_gradient():
    # triangle inequality: |grad_j| <= absum_j for every body, with and without nodes
    pos, _, m = inputs.clumpy_plummer(800, seed=8)
    lam = np.random.default_rng(9).standard_normal(pos.shape)
    for theta, leaf in ((0.0, 1), (0.6, 4)):
        g, a = oracle.tree_vjp(oracle.Tree(pos, m, leaf_max=leaf), lam, theta, 1e-3,
                               with_absum=True)
        assert np.all(np.linalg.norm(g, axis=1) <= a * (1 + 1e-12))
