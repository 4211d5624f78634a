"""Pins of the oracle's aggregate identification (Sec. 2, "Post-processing: aggregate
identification": contact-graph components by depth-first search), none of which compares
the oracle with itself: hand cases with exact boundary distances, closed forms on a
lattice, an independent graph library on random clouds, and the labelling's invariants."""
import numpy as np
import pytest

import oracle
from paper_1912_04197_gb300 import inputs


def test_chain_with_exact_boundaries():
    # distances 1 (= dmax: touching joins), 1.5, 1 and 6.5 along x
    pos = np.array([[0, 0, 0], [1, 0, 0], [2.5, 0, 0], [3.5, 0, 0], [10, 0, 0]], float)
    label, counts = oracle.components(pos, dmax=1.0)
    assert label.tolist() == [0, 0, 2, 2, 4] and counts == (3, 2)
    label, counts = oracle.components(pos, dmax=1.5)
    assert label.tolist() == [0, 0, 0, 0, 4] and counts == (2, 1)
    label, counts = oracle.components(pos, dmax=0.5)
    assert label.tolist() == [0, 1, 2, 3, 4] and counts == (5, 0)


def test_radii_touching_spheres():
    # spheres of radii 0.25 and 0.5 with centres 0.75 apart touch; 0.75 + 2^-40 apart do not
    for gap, joined in ((0.75, True), (0.75 + 2.0 ** -40, False)):
        pos = np.array([[0.0, 0.0, 0.0], [0.0, gap, 0.0]])
        label, counts = oracle.components(pos, radius=np.array([0.25, 0.5]))
        assert (label.tolist() == [0, 0]) == joined
        assert counts == ((1, 1) if joined else (2, 0))


def test_lattice_closed_form():
    h = 0.125
    k = np.arange(6) * h
    pos = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    label, counts = oracle.components(pos, dmax=h)            # nearest neighbours touch
    assert np.all(label == 0) and counts == (1, 1)
    label, counts = oracle.components(pos, dmax=h * (1 - 2.0 ** -20))
    assert np.array_equal(label, np.arange(len(pos))) and counts == (len(pos), 0)


def _canonical(n, comp):
    # smallest index of each component, from any component numbering
    first = {}
    for i in range(n):
        first.setdefault(comp[i], i)
    return np.array([first[c] for c in comp], np.int32)


@pytest.mark.parametrize("seed,use_radius", [(0, False), (1, True), (2, False)])
def test_against_scipy_connected_components(seed, use_radius):
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    sparse = pytest.importorskip("scipy.sparse")
    pos, _, _ = inputs.clumpy_plummer(3000, seed=seed, nclusters=6)
    rng = np.random.default_rng(seed)
    radius = rng.lognormal(np.log(0.004), 0.5, len(pos)) if use_radius else None
    dmax = 0.01
    d2 = ((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1)
    t = (radius[:, None] + radius[None, :]) if use_radius else dmax
    adj = sparse.csr_matrix(d2 <= t * t)
    ncomp, comp = csgraph.connected_components(adj, directed=False)
    label, counts = oracle.components(pos, radius=radius, dmax=dmax)
    assert np.array_equal(label, _canonical(len(pos), comp))
    sizes = np.bincount(comp)
    assert counts == (ncomp, int((sizes > 1).sum()))
    assert 1 < counts[1] < counts[0] < len(pos)               # a non-trivial partition


def test_label_invariants():
    pos, _, _ = inputs.uniform_sphere(2000, seed=3)
    label, counts = oracle.components(pos, dmax=0.06)
    idx = np.arange(len(pos))
    assert np.all(label <= idx)                                # the smallest index
    assert np.array_equal(label[label], label)                 # a label labels itself
    assert len(np.unique(label)) == counts[0]
    _, mult = np.unique(label, return_counts=True)
    assert int((mult > 1).sum()) == counts[1]
