"""Pins of the axis-ratio objective: for bodies uniform in an ellipsoid with semi-axes
a >= b >= c the second-moment tensor is (M/5) diag(a^2, b^2, c^2), so the axis ratios
are b/a and c/a; the loss vanishes at the target and its gradient is that of the
closed form."""
import numpy as np
import torch

from paper_1912_04197_gb300.loss import axis_ratio_loss


def _ellipsoid(n, axes, seed=0):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    u *= rng.random((n, 1)) ** (1.0 / 3.0)
    # random rotation and offset: the loss is invariant under both
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return (u * np.asarray(axes)) @ q.T + np.array([0.3, -1.0, 2.0])


def test_axis_ratios_of_uniform_ellipsoid():
    x = torch.tensor(_ellipsoid(400_000, (1.0, 0.7, 0.4)))
    m = torch.full((len(x),), 1.0 / len(x), dtype=torch.float64)
    L = axis_ratio_loss(x, m, target=(0.7, 0.4))
    assert float(L) < 1e-5
    L2 = axis_ratio_loss(x, m, target=(0.8, 0.6))
    assert abs(float(L2) - ((0.7 - 0.8) ** 2 + (0.4 - 0.6) ** 2)) < 2e-3


def test_axis_ratio_exact_six_points_and_gradient():
    # six unit masses at +-a e1, +-b e2, +-c e3: S = 2 diag(a^2, b^2, c^2) exactly
    a, b, c = 2.0, 1.5, 0.5
    x = torch.tensor([[a, 0, 0], [-a, 0, 0], [0, b, 0], [0, -b, 0], [0, 0, c], [0, 0, -c]],
                     dtype=torch.float64, requires_grad=True)
    m = torch.ones(6, dtype=torch.float64)
    L = axis_ratio_loss(x, m)
    want = (b / a - 0.8) ** 2 + (c / a - 0.6) ** 2
    assert abs(float(L.detach()) - want) < 1e-14
    L.backward()
    # d/da of the closed form, split equally between the two bodies on the x axis
    # (each moves by +-da along e1 when a grows by da)
    dLda = 2 * (b / a - 0.8) * (-b / a ** 2) + 2 * (c / a - 0.6) * (-c / a ** 2)
    assert abs(float(x.grad[0, 0]) - dLda / 2) < 1e-12
    assert abs(float(x.grad[1, 0]) + dLda / 2) < 1e-12
    dLdb = 2 * (b / a - 0.8) / a
    assert abs(float(x.grad[2, 1]) - dLdb / 2) < 1e-12
