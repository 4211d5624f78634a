"""Seeded synthetic inputs (numpy PCG64, FP64) shaped like the paper's workloads.

This module holds none of the method's arithmetic: it only draws bodies.  Both
the CUDA path and the CPU oracle receive the arrays it returns.

The paper's own benchmark workload is bodies at rest, uniform in a cube, mutual
gravity only (Sec. 3.2); its aggregation scenarios are rubble clouds (Sec. 4).
The generators below stand in for those with the following recipes:

* ``uniform_sphere``  - radius R*U^(1/3), isotropic direction, m = M/N, v = 0.
* ``uniform_cube``    - the paper's timing workload: uniform in [-1, 1]^3, at rest.
* ``rubble_pile``     - uniform sphere R = 1, lognormal(0, 0.5) masses normalised to
  total mass 1, solid-body rotation at 0.3 of breakup about z (breakup rate
  w_b = sqrt(G M / R^3)) plus Gaussian velocity noise sigma = 0.01 w_b R.
* ``clumpy_plummer``  - k Plummer spheres of scale a, centres uniform in the unit
  sphere; radii by inverting the Plummer cumulative mass r^3/(r^2+a^2)^{3/2}
  restricted to r <= 10 a; equal masses; at rest.
* ``ensemble``        - independent clouds with N_k = floor(exp U(ln lo, ln hi)),
  uniform spheres R = 1, m = 1/N_k, spin axis uniform on the sphere, rate
  U(0, 0.3) w_b.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _directions(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    nrm = np.linalg.norm(v, axis=1, keepdims=True)
    nrm[nrm == 0] = 1.0
    return v / nrm


def uniform_sphere(n: int, seed: int = 0, radius: float = 1.0, total_mass: float = 1.0):
    """(pos[n,3], vel[n,3], mass[n]) uniform in a ball, equal masses, at rest."""
    rng = _rng(seed)
    r = radius * rng.random(n) ** (1.0 / 3.0)
    pos = _directions(rng, n) * r[:, None]
    mass = np.full(n, total_mass / max(n, 1))
    return pos, np.zeros((n, 3)), mass


def uniform_cube(n: int, seed: int = 0, half_side: float = 1.0):
    """The paper's timing workload (Sec. 3.2): uniform in a cube, at rest, m = 1/N."""
    rng = _rng(seed)
    pos = (rng.random((n, 3)) * 2.0 - 1.0) * half_side
    return pos, np.zeros((n, 3)), np.full(n, 1.0 / max(n, 1))


def rubble_pile(n: int = 100_000, seed: int = 0, G: float = 1.0):
    """Rotating rubble cloud: lognormal masses, 0.3 x breakup spin, 1 % noise."""
    rng = _rng(seed)
    R = 1.0
    r = R * rng.random(n) ** (1.0 / 3.0)
    pos = _directions(rng, n) * r[:, None]
    mass = rng.lognormal(0.0, 0.5, n)
    mass /= mass.sum()
    wb = np.sqrt(G * 1.0 / R ** 3)
    omega = np.array([0.0, 0.0, 0.3 * wb])
    vel = np.cross(np.broadcast_to(omega, pos.shape), pos)
    vel += rng.standard_normal((n, 3)) * (0.01 * wb * R)
    return pos, vel, mass


def clumpy_plummer(n: int = 1_048_576, seed: int = 0, nclusters: int = 64, a: float = 0.05,
                   rcut: float = 10.0):
    """n bodies in `nclusters` truncated Plummer spheres; equal masses, at rest."""
    rng = _rng(seed)
    per = np.full(nclusters, n // nclusters)
    per[: n - per.sum()] += 1
    rc = rng.random(nclusters) ** (1.0 / 3.0)
    centres = _directions(rng, nclusters) * rc[:, None]
    xmax = rcut ** 3 / (rcut ** 2 + 1.0) ** 1.5      # enclosed mass fraction at r = rcut*a
    out = []
    for c in range(nclusters):
        k = int(per[c])
        X = rng.random(k) * xmax
        X = np.clip(X, 1e-300, None)
        rad = a / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        out.append(centres[c] + _directions(rng, k) * rad[:, None])
    pos = np.concatenate(out, axis=0)
    return pos, np.zeros((n, 3)), np.full(n, 1.0 / n)


def ensemble(nclouds: int = 256, seed: int = 0, nmin: int = 1024, nmax: int = 65536,
             G: float = 1.0):
    """Independent spinning clouds: (offsets[nclouds+1], pos, vel, mass), concatenated."""
    rng = _rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(nmin), np.log(nmax), nclouds))).astype(np.int64)
    offsets = np.zeros(nclouds + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    P, V, M = [], [], []
    wb = np.sqrt(G * 1.0 / 1.0)
    for k in range(nclouds):
        nk = int(sizes[k])
        r = rng.random(nk) ** (1.0 / 3.0)
        pos = _directions(rng, nk) * r[:, None]
        axis = _directions(rng, 1)[0]
        w = axis * rng.uniform(0.0, 0.3) * wb
        P.append(pos)
        V.append(np.cross(np.broadcast_to(w, pos.shape), pos))
        M.append(np.full(nk, 1.0 / nk))
    return offsets, np.concatenate(P), np.concatenate(V), np.concatenate(M)


def subset(n: int, k: int, seed: int = 12345) -> np.ndarray:
    """Seeded sorted sample of k distinct caller indices out of n."""
    if k >= n:
        return np.arange(n, dtype=np.int64)
    return np.sort(_rng(seed).choice(n, size=k, replace=False)).astype(np.int64)
