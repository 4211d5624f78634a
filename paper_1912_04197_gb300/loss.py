"""Aggregate-shape objective for the differentiation layer: the second-moment tensor
S = sum_i m_i (x_i - c)(x_i - c)^T about the centre of mass c, its eigenvalues
l1 >= l2 >= l3, rho_k = sqrt(l_k / l1), loss = (rho_2 - t2)^2 + (rho_3 - t3)^2 for a
target axis ratio 1 : t2 : t3.  Plain differentiable torch (any device, float64)."""
import torch


def axis_ratio_loss(x: torch.Tensor, mass: torch.Tensor, target=(0.8, 0.6)) -> torch.Tensor:
    """(rho_2 - t2)^2 + (rho_3 - t3)^2 of the mass distribution's second-moment tensor."""
    m = mass.reshape(-1, 1)
    c = (m * x).sum(0) / m.sum()
    y = x - c
    S = (m * y).T @ y
    lam = torch.linalg.eigvalsh(S)              # ascending: l3, l2, l1
    rho2 = torch.sqrt(lam[1] / lam[2])
    rho3 = torch.sqrt(lam[0] / lam[2])
    return (rho2 - target[0]) ** 2 + (rho3 - target[1]) ** 2
