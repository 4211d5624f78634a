"""Differentiation through the tree-code integrator.

`leapfrog` runs kick-drift-kick leapfrog steps (Sec. 2.3, tree rebuilt every step,
Sec. 2.1) as a torch.autograd.Function: the forward pass keeps the state (x, v) every
`checkpoint_every` steps; the backward pass walks the segments from last to first,
each one recomputing its positions from its checkpoint and applying the frozen-tree
vector-Jacobian products of the accelerations (leapfrog_adjoint in the library).
Gradients flow to the initial positions and velocities; the masses are constants.
The aggregate-shape objective used with it is loss.axis_ratio_loss."""
from __future__ import annotations

import torch

from . import gravity as _g


class _Leapfrog(torch.autograd.Function):
    @staticmethod
    def forward(fctx, x0, v0, mass, dt, nsteps, theta, eps, params, every, gctx):
        x = x0.detach().clone().contiguous()
        v = v0.detach().clone().contiguous()
        m = mass.detach().contiguous()
        acc = torch.empty_like(x)
        _g.gravity_tree_build(gctx, x, m, params)
        _g.gravity_forces(gctx, theta, eps, acc)
        ckpts = []
        s = 0
        while s < nsteps:
            k = min(every, nsteps - s)
            ckpts.append((x.clone(), v.clone(), k))
            _g.leapfrog_step(gctx, x, v, m, acc, dt, k, theta, eps, params)
            s += k
        fctx.ckpts = ckpts
        fctx.args = (m, dt, theta, eps, params, gctx)
        return x, v

    @staticmethod
    def backward(fctx, xbar, vbar):
        m, dt, theta, eps, params, gctx = fctx.args
        ckpts = fctx.ckpts
        n = m.shape[0]
        xb = (xbar if xbar is not None else torch.zeros((n, 3), dtype=torch.float64,
                                                         device=m.device)).clone().contiguous()
        vb = (vbar if vbar is not None else torch.zeros_like(xb)).clone().contiguous()
        for i in range(len(ckpts) - 1, -1, -1):
            xs, vs, k = ckpts[i]
            flags = ((_g.GRAVITY_ADJ_END if i == len(ckpts) - 1 else 0) |
                     (_g.GRAVITY_ADJ_START if i == 0 else 0))
            _g.leapfrog_adjoint(gctx, xs, vs, m, dt, k, theta, eps, params, flags, xb, vb)
        fctx.ckpts = None
        return xb, vb, None, None, None, None, None, None, None, None


def leapfrog(x0: torch.Tensor, v0: torch.Tensor, mass: torch.Tensor, dt: float, nsteps: int, *,
             theta: float = 0.5, eps: float = 1e-3, G: float = 1.0, leaf_max: int = 1,
             checkpoint_every: int = 20, ctx: _g.Context | None = None):
    """(x_N, v_N) after nsteps KDK steps from (x0, v0), differentiable in x0 and v0.
    Monopole tree forces (order 0); all tensors float64 on one CUDA device."""
    if nsteps < 1 or checkpoint_every < 1:
        raise ValueError("nsteps and checkpoint_every must be >= 1")
    gctx = ctx if ctx is not None else _g.Context(x0.device)
    params = _g.params(G=G, leaf_max=leaf_max, order=0, scheme=0)
    return _Leapfrog.apply(x0, v0, mass, float(dt), int(nsteps), float(theta), float(eps), params,
                           int(checkpoint_every), gctx)
