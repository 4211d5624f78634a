"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a hand-derived value
(tests/golden), a closed form, a library routine, an independent construction,
or an invariant that a dropped term, wrong sign or wrong index would break.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1912_04197_gb300 import inputs
from conftest import load_golden

pytestmark = pytest.mark.oracle


# ---------------------------------------------------------------- root cube, keys, order

def test_root_cube_reading():
    pos = np.array([[0.5, -1.0, 2.0], [1.5, 3.0, 2.25], [1.0, 0.0, 2.5]])
    lo, s = oracle.root_cube(pos)
    assert lo.tolist() == [0.5, -1.0, 2.0]
    assert s == 4.0                                   # largest extent (y: -1 .. 3)
    assert oracle.root_cube(np.zeros((5, 3)))[1] == 1.0   # zero extent -> side 1
    assert oracle.root_cube(np.array([[3.0, 4.0, 5.0]]))[1] == 1.0
    bad = pos.copy()
    bad[1, 2] = np.nan
    with pytest.raises(oracle.OracleError) as e:
        oracle.root_cube(bad)
    assert e.value.code == oracle.ORC_E_NONFINITE
    bad[1, 2] = np.inf
    with pytest.raises(oracle.OracleError):
        oracle.root_cube(bad)


def test_morton_golden_unit_cube():
    rows = load_golden("morton_unit_cube.txt")
    pos = np.array([[float(v) for v in r[:3]] for r in rows])
    want = np.array([int(r[3]) for r in rows], dtype=np.uint64)
    lo, s = oracle.root_cube(pos)
    assert lo.tolist() == [0, 0, 0] and s == 1.0
    assert np.array_equal(oracle.morton_keys(pos, lo, s), want)


def _spread_bits(v):
    """Independent interleave: insert two zero bits between the bits of a 21-bit int
    using the shift-and-mask ladder (different method from the oracle's bit loop)."""
    v = np.asarray(v, dtype=np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def test_morton_vs_independent_interleave():
    pos, _, _ = inputs.clumpy_plummer(20000, seed=3, nclusters=8)
    lo, s = oracle.root_cube(pos)
    keys = oracle.morton_keys(pos, lo, s)
    scale = 2.0 ** 21 / s
    q = np.clip(np.floor((pos - lo) * scale), 0, 2 ** 21 - 1).astype(np.uint64)
    ref = (_spread_bits(q[:, 0]) << np.uint64(2)) | (_spread_bits(q[:, 1]) << np.uint64(1)) \
        | _spread_bits(q[:, 2])
    assert np.array_equal(keys, ref)
    assert keys.max() < np.uint64(1 << 63)


def test_key_order_is_octant_path_order():
    rng = np.random.default_rng(7)
    pos = rng.random((3000, 3))
    lo, s = oracle.root_cube(pos)
    keys = oracle.morton_keys(pos, lo, s)
    q = np.clip(np.floor((pos - lo) * (2.0 ** 21 / s)), 0, 2 ** 21 - 1).astype(np.int64)
    # octant path: for each level (coarse first) the digit 4*bx + 2*by + bz
    paths = [tuple(int(4 * ((qq[0] >> k) & 1) + 2 * ((qq[1] >> k) & 1) + ((qq[2] >> k) & 1))
                   for k in range(20, -1, -1)) for qq in q]
    by_path = sorted(range(len(paths)), key=lambda i: paths[i])
    assert np.array_equal(np.argsort(keys, kind="stable"), np.array(by_path))


def test_stable_order_matches_library_sort_with_ties():
    rng = np.random.default_rng(1)
    keys = rng.integers(0, 50, size=5000).astype(np.uint64)     # many duplicate keys
    perm = oracle.stable_order(keys)
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))


# ---------------------------------------------------------------- topology

def _interleave_cell(cx, cy, cz, depth):
    p = 0
    for k in range(depth):
        p |= ((cx >> k) & 1) << (3 * k + 2) | ((cy >> k) & 1) << (3 * k + 1) | ((cz >> k) & 1) << (3 * k)
    return p


def _insertion_octree(q, leaf_max):
    """Paper-style construction (Sec. 2.1): insert bodies one at a time into cells
    addressed by integer grid coordinates; a cell exceeding leaf_max bodies is
    subdivided (depth < 21).  Then chains of single-child cells are collapsed to
    their deepest member.  Returns the DFS preorder list of
    (depth, prefix, frozenset(bodies), n_child)."""
    root = {"depth": 0, "c": (0, 0, 0), "bodies": [], "kids": None}

    def octant(cell, i):
        sh = 20 - cell["depth"]
        return tuple(int((q[i, a] >> sh) & 1) for a in range(3))

    def insert(cell, i):
        while cell["kids"] is not None:
            o = octant(cell, i)
            if o not in cell["kids"]:
                cx, cy, cz = cell["c"]
                cell["kids"][o] = {"depth": cell["depth"] + 1,
                                   "c": (2 * cx + o[0], 2 * cy + o[1], 2 * cz + o[2]),
                                   "bodies": [], "kids": None}
            cell["bodies"].append(i)
            cell = cell["kids"][o]
        cell["bodies"].append(i)
        if len(cell["bodies"]) > leaf_max and cell["depth"] < 21:
            held = cell["bodies"]
            cell["bodies"], cell["kids"] = [], {}
            for j in held:
                insert(cell, j)

    for i in range(len(q)):
        insert(root, i)

    out = []

    def emit(cell):
        while cell["kids"] is not None and len(cell["kids"]) == 1:
            cell = next(iter(cell["kids"].values()))
        kids = [] if cell["kids"] is None else [cell["kids"][o] for o in sorted(cell["kids"])]
        d = cell["depth"]
        out.append((d, _interleave_cell(*cell["c"], d), frozenset(cell["bodies"]), len(kids)))
        for k in kids:
            emit(k)

    emit(root)
    return out


@pytest.mark.parametrize("n,leaf_max,seed", [(1, 1, 0), (2, 1, 0), (8, 1, 1), (60, 1, 2),
                                             (300, 1, 3), (300, 4, 4), (500, 16, 5)])
def test_topology_vs_insertion_construction(n, leaf_max, seed):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) ** 3                     # uneven density
    if n >= 60:
        pos[: n // 10] = pos[0]                       # a block of coincident bodies
    mass = np.full(n, 1.0 / n)
    t = oracle.Tree(pos, mass, leaf_max=leaf_max)
    nd = t.nodes()
    _, perm = t.order_arrays()
    got = [(int(nd["depth"][k]), int(nd["prefix"][k]),
            frozenset(perm[nd["begin"][k]:nd["end"][k]].tolist()), int(nd["n_child"][k]))
           for k in range(t.num_nodes)]
    lo, s = oracle.root_cube(pos)
    q = np.clip(np.floor((pos - lo) * (2.0 ** 21 / s)), 0, 2 ** 21 - 1).astype(np.int64)
    assert got == _insertion_octree(q, leaf_max)


def test_topology_invariants_large():
    pos, _, m = inputs.clumpy_plummer(50000, seed=1, nclusters=16)
    for leaf_max in (1, 8):
        t = oracle.Tree(pos, m, leaf_max=leaf_max)
        nd = t.nodes()
        k = t.num_nodes
        internal = nd["leaf"] == 0
        assert np.all((nd["n_child"][internal] >= 2) & (nd["n_child"][internal] <= 8))
        assert np.all(nd["n_child"][~internal] == 0)
        assert np.all(nd["depth"] <= 21)
        assert (nd["leaf"] == 1).sum() >= 50000 / leaf_max
        # children ranges partition the parent's range, in order
        kids = {}
        for c in range(1, k):
            kids.setdefault(int(nd["parent"][c]), []).append(c)
        for p, cs in kids.items():
            assert nd["begin"][cs[0]] == nd["begin"][p] and nd["end"][cs[-1]] == nd["end"][p]
            for a, b in zip(cs[:-1], cs[1:]):
                assert nd["end"][a] == nd["begin"][b]
                assert nd["depth"][b] > nd["depth"][p]


# ---------------------------------------------------------------- moments

def test_moments_closed_forms():
    rng = np.random.default_rng(5)
    pos = rng.standard_normal((4000, 3))
    mass = rng.lognormal(0, 0.5, 4000)
    for leaf_max in (1, 8):
        t = oracle.Tree(pos, mass, leaf_max=leaf_max, order=2)
        m, com, quad = t.moments()
        assert abs(m[0] - mass.sum()) <= 1e-13 * mass.sum()
        want = (mass[:, None] * pos).sum(0) / mass.sum()
        assert np.allclose(com[0], want, rtol=0, atol=1e-13)
        # every node against the definition over its own bodies
        nd = t.nodes()
        _, perm = t.order_arrays()
        for k in range(0, t.num_nodes, 37):
            idx = perm[nd["begin"][k]:nd["end"][k]]
            mk = mass[idx]
            ck = (mk[:, None] * pos[idx]).sum(0) / mk.sum()
            assert abs(m[k] - mk.sum()) <= 1e-13 * mk.sum()
            assert np.allclose(com[k], ck, rtol=0, atol=1e-12)
            y = pos[idx] - ck
            r2 = (y * y).sum(1)
            Q = np.einsum("i,ij,ik->jk", mk, 3 * y, y) - np.eye(3) * (mk * r2).sum()
            qk = quad[k]
            got = np.array([[qk[0], qk[3], qk[4]], [qk[3], qk[1], qk[5]], [qk[4], qk[5], qk[2]]])
            if len(idx) == 1:
                assert np.all(qk == 0)
            else:
                scale = (mk * r2).sum() * 3
                assert np.allclose(got, Q, rtol=0, atol=1e-11 * scale)
                assert abs(qk[0] + qk[1] + qk[2]) <= 1e-12 * scale   # traceless


def test_moments_symmetric_corners_and_two_mass_quadrupole():
    corners = np.array([[x, y, z] for x in (0.0, 1.0) for y in (0.0, 1.0) for z in (0.0, 1.0)])
    t = oracle.Tree(corners, np.full(8, 0.5))
    m, com, _ = t.moments()
    assert m[0] == 4.0 and com[0].tolist() == [0.5, 0.5, 0.5]
    # two masses m at +-a on the x axis: Q = diag(4 m a^2, -2 m a^2, -2 m a^2)
    a, mm = 0.75, 2.0
    pos = np.array([[-a, 0.0, 0.0], [a, 0.0, 0.0]])
    for leaf_max in (1, 2):
        t = oracle.Tree(pos, np.full(2, mm), leaf_max=leaf_max, order=2)
        _, com, quad = t.moments()
        assert com[0].tolist() == [0.0, 0.0, 0.0]
        assert np.allclose(quad[0], [4 * mm * a * a, -2 * mm * a * a, -2 * mm * a * a, 0, 0, 0],
                           rtol=1e-15, atol=0)


# ---------------------------------------------------------------- forces

def test_two_body_golden():
    for r in load_golden("two_body_force.txt"):
        G, eps, m1, m2, dx, dy, dz, ax, ay, az = map(float, r)
        pos = np.array([[0.0, 0.0, 0.0], [dx, dy, dz]])
        mass = np.array([m1, m2])
        acc, _ = oracle.direct(pos, mass, eps, G)
        assert np.allclose(acc[0], [ax, ay, az], rtol=1e-12, atol=1e-15)
        assert np.allclose(acc[1] * m2, -acc[0] * m1, rtol=1e-15, atol=1e-18)
        for leaf_max in (1, 2):
            at = oracle.tree_forces(pos, mass, 0.5, eps, G, leaf_max=leaf_max)
            assert np.allclose(at, acc, rtol=1e-15, atol=0)


def test_direct_newton_third_law_and_long_double():
    pos, _, _ = inputs.rubble_pile(3000, seed=2)
    mass = inputs.rubble_pile(3000, seed=2)[2]
    acc, _ = oracle.direct(pos, mass, 5e-3)
    tot = (mass[:, None] * acc).sum(0)
    assert np.linalg.norm(tot) <= 1e-12 * (mass * np.linalg.norm(acc, axis=1)).sum()
    # brute force in extended precision on a small set
    rng = np.random.default_rng(3)
    p = rng.standard_normal((48, 3))
    w = rng.random(48) + 0.5
    acc, _ = oracle.direct(p, w, 0.01, 1.7)
    P = p.astype(np.longdouble)
    W = w.astype(np.longdouble)
    d = P[None, :, :] - P[:, None, :]
    r2 = (d * d).sum(-1) + np.longdouble(0.01) ** 2
    np.fill_diagonal(r2, 1)
    f = W[None, :] / (r2 * np.sqrt(r2))
    np.fill_diagonal(f, 0)
    ref = np.longdouble(1.7) * (f[:, :, None] * d).sum(1)
    assert np.allclose(acc, ref.astype(np.float64), rtol=1e-13, atol=1e-13)


def test_direct_uniform_sphere_interior_field():
    # shell theorem: inside a uniform ball of mass M and radius R, a(r) = -G M r / R^3
    pos, _, m = inputs.uniform_sphere(20000, seed=4)
    idx = inputs.subset(20000, 400, seed=9)
    acc, _ = oracle.direct(pos, m, 1e-3, targets=idx)
    r = np.linalg.norm(pos[idx], axis=1)
    sel = (r > 0.2) & (r < 0.8)
    radial = (acc[sel] * pos[idx][sel]).sum(1) / r[sel]
    assert abs(np.median(radial / -r[sel]) - 1.0) < 0.03


def test_theta_zero_equals_direct():
    # Sec. 3.2: theta = 0 means no clustering, i.e. direct integration
    pos, _, m = inputs.clumpy_plummer(6000, seed=6, nclusters=4)
    ad, _ = oracle.direct(pos, m, 1e-3)
    for leaf_max in (1, 8):
        for order in (0, 2):
            t = oracle.Tree(pos, m, leaf_max=leaf_max, order=order)
            at, _, cnt = t.forces(0.0, 1e-3)
            assert np.all(cnt[:, 1] == 0) and np.all(cnt[:, 2] == len(pos) - 1)
            err = np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)
            assert err.max() < 1e-13


def test_large_softening_partition_of_bodies():
    # With eps much larger than the system, every term is m_k d_k / eps^3 to
    # O((size/eps)^2); sum_nodes m_N COM_N = sum_bodies m_j x_j, so the tree force
    # equals the direct force iff each body's accepted nodes and body terms cover
    # every other body exactly once.
    pos, _, _ = inputs.uniform_sphere(3000, seed=8)
    m = np.random.default_rng(8).random(3000) + 0.1
    eps = 1e4
    ad, _ = oracle.direct(pos, m, eps)
    for leaf_max, order in ((1, 0), (8, 0), (8, 2)):
        at = oracle.tree_forces(pos, m, 0.9, eps, leaf_max=leaf_max, order=order)
        assert np.abs(at - ad).max() <= 1e-7 * np.abs(ad).max()


def test_mac_equality_opens():
    pos = np.array([[0.0, 0.0, 0.0], [0.25, 0.0, 0.0], [0.125, 0.0, 1.0]])
    t = oracle.Tree(pos, np.ones(3))
    for r in load_golden("mac_equality.txt"):
        theta = float(r[0])
        _, _, cnt = t.forces(theta, 0.0, targets=[2])
        assert cnt[0].tolist() == [int(r[1]), int(r[2]), int(r[3])]


def test_far_field_error_slopes():
    # A cluster of size l at distance D seen as one node: monopole error ~ (l/D)^2
    # (the dipole vanishes about the COM), quadrupole error ~ (l/D)^3.
    rng = np.random.default_rng(11)
    base = rng.random((40, 3)) - 0.5
    w = rng.random(40) + 0.5
    D = 1.0
    ratios, e0, e2 = [], [], []
    for l in (1 / 8, 1 / 16, 1 / 32, 1 / 64):
        cl = base * l
        probe = np.array([[0.3 * D, 0.2 * D, D]])
        pos = np.vstack([cl, probe])
        mass = np.concatenate([w, [1.0]])
        exact, _ = oracle.direct(pos, mass, 0.0, targets=[40])
        errs = []
        for order in (0, 2):
            t = oracle.Tree(pos, mass, leaf_max=1, order=order)
            a, _, cnt = t.forces(0.9, 0.0, targets=[40])
            assert cnt[0, 1] == 1 and cnt[0, 2] == 0      # the cluster is one node term
            errs.append(np.linalg.norm(a[0] - exact[0]) / np.linalg.norm(exact[0]))
        ratios.append(l)
        e0.append(errs[0])
        e2.append(errs[1])
    s0 = np.polyfit(np.log(ratios), np.log(e0), 1)[0]
    s2 = np.polyfit(np.log(ratios), np.log(e2), 1)[0]
    assert 1.8 < s0 < 2.2, s0
    assert 2.8 < s2 < 3.3, s2


def test_error_monotone_in_theta():
    # Sec. 3.2 (Accuracy): the error grows monotonically with theta
    pos, _, m = inputs.uniform_cube(4000, seed=2)
    ad, _ = oracle.direct(pos, m, 1e-3)
    t = oracle.Tree(pos, m)
    meds = []
    for th in (0.1, 0.25, 0.5, 0.75):
        a, _, _ = t.forces(th, 1e-3)
        meds.append(np.median(np.linalg.norm(a - ad, axis=1) / np.linalg.norm(ad, axis=1)))
    assert all(x < y for x, y in zip(meds, meds[1:])), meds
    assert meds[-1] / meds[0] > 30


def test_edge_cases():
    a, _, _ = oracle.Tree(np.zeros((0, 3)), np.zeros(0)).forces(0.5, 0.1)
    assert a.shape == (0, 3)
    a = oracle.tree_forces(np.array([[1.0, 2.0, 3.0]]), np.ones(1), 0.5, 0.1)
    assert np.all(a == 0)
    same = np.tile([[0.3, 0.3, 0.3]], (20, 1))
    for eps in (0.0, 0.1):                         # r^2 + eps^2 = 0 contributes nothing
        t = oracle.Tree(same, np.ones(20))
        assert t.nodes()["depth"][0] == 21 and t.num_nodes == 1
        a, _, _ = t.forces(0.5, eps)
        assert np.all(a == 0)
        ad, _ = oracle.direct(same, np.ones(20), eps)
        assert np.all(ad == 0)
    with pytest.raises(oracle.OracleError):
        oracle.Tree(same, np.ones(20)).forces(-0.1, 0.1)
    with pytest.raises(oracle.OracleError):
        oracle.Tree(same, np.ones(20)).forces(0.5, -1.0)


# ---------------------------------------------------------------- integrators, invariants

def _kepler_pair(e=0.5, a=1.0, m1=1.0, m2=0.5):
    M = m1 + m2
    r_p = a * (1 - e)
    v_p = math.sqrt(M * (1 + e) / r_p)            # vis-viva at pericentre, G = 1
    pos = np.array([[-m2 / M * r_p, 0, 0], [m1 / M * r_p, 0, 0]])
    vel = np.array([[0, -m2 / M * v_p, 0], [0, m1 / M * v_p, 0]])
    return pos, vel, np.array([m1, m2])


def test_kepler_period_and_energy_leapfrog():
    # two-body conic (Sec. 3.1): period 2 pi sqrt(a^3 / (G M)), energy -G m1 m2 / (2 a)
    pos, vel, m = _kepler_pair()
    T = 2 * math.pi * math.sqrt(1.0 / 1.5)
    E_exact = -1.0 * 0.5 / 2.0
    for nper, tol_x in ((2000, 3e-3), (4000, 8e-4)):
        dt = T / nper
        acc, _ = oracle.direct(pos, m, 0.0)
        E0 = oracle.diagnostics(pos, vel, m, 0.0)[0]
        assert abs(E0 - E_exact) < 1e-14
        p, v, a = oracle.step(pos, vel, m, acc, dt, nper, use_tree=False, eps=0.0)
        assert np.abs(p - pos).max() < tol_x      # back at pericentre after one period
        E1, P1, L1 = oracle.diagnostics(p, v, m, 0.0)
        assert abs(E1 - E_exact) < 50 * (dt ** 2)
        assert np.abs(P1).max() < 1e-14
    # energy error is O(dt^2): halving dt divides it by ~4
    errs = []
    for nper in (500, 1000):
        acc, _ = oracle.direct(pos, m, 0.0)
        p, v, _ = oracle.step(pos, vel, m, acc, T / nper, nper // 4, use_tree=False, eps=0.0)
        errs.append(abs(oracle.diagnostics(p, v, m, 0.0)[0] - E_exact))
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_semi_implicit_euler_bounded_energy():
    pos, vel, m = _kepler_pair(e=0.3)
    T = 2 * math.pi * math.sqrt(1.0 / 1.5)
    acc, _ = oracle.direct(pos, m, 0.0)
    E0 = oracle.diagnostics(pos, vel, m, 0.0)[0]
    p, v, a = pos, vel, acc
    worst = 0.0
    for _ in range(10):                            # 5 periods, no secular drift
        p, v, a = oracle.step(p, v, m, a, T / 2000, 1000, scheme=1, use_tree=False, eps=0.0)
        worst = max(worst, abs(oracle.diagnostics(p, v, m, 0.0)[0] - E0))
    assert worst < 2e-2 * abs(E0)
    _, _, L = oracle.diagnostics(p, v, m, 0.0)
    assert abs(L[2] - oracle.diagnostics(pos, vel, m, 0.0)[2][2]) < 1e-12


def test_leapfrog_time_reversible():
    pos, vel, m = inputs.rubble_pile(400, seed=5)
    acc, _ = oracle.direct(pos, m, 5e-3)
    p, v, a = oracle.step(pos, vel, m, acc, 1e-3, 20, use_tree=False, eps=5e-3)
    p2, v2, _ = oracle.step(p, v, m, a, -1e-3, 20, use_tree=False, eps=5e-3)
    assert np.abs(p2 - pos).max() < 1e-12 and np.abs(v2 - vel).max() < 1e-11


def test_rubble_pile_energy_bounded_tree():
    pos, vel, m = inputs.rubble_pile(2000, seed=0)
    acc = oracle.tree_forces(pos, m, 0.5, 5e-3, order=2)
    E0, P0, L0 = oracle.diagnostics(pos, vel, m, 5e-3)
    p, v, a = pos, vel, acc
    rel = []
    for _ in range(5):
        p, v, a = oracle.step(p, v, m, a, 1e-3, 20, theta=0.5, eps=5e-3, order=2)
        rel.append(abs(oracle.diagnostics(p, v, m, 5e-3)[0] - E0) / abs(E0))
    assert max(rel) < 1e-5, rel
    _, P1, L1 = oracle.diagnostics(p, v, m, 5e-3)
    assert np.linalg.norm(L1 - L0) < 1e-4 * np.linalg.norm(L0)


def test_diagnostics_two_body_closed_form():
    pos = np.array([[0.0, 0, 0], [3.0, 4.0, 0]])
    vel = np.array([[1.0, 0, 0], [0, -2.0, 0]])
    m = np.array([2.0, 0.5])
    E, P, L = oracle.diagnostics(pos, vel, m, 0.0, G=1.0)
    assert E == pytest.approx(0.5 * 2 * 1 + 0.5 * 0.5 * 4 - 2 * 0.5 / 5, rel=1e-15)
    assert P.tolist() == [2.0, -1.0, 0.0]
    assert L.tolist() == [0.0, 0.0, 0.5 * (3.0 * -2.0)]


@pytest.mark.parametrize("scheme", [0, 1])
def test_two_time_steps_hold_gravity_between_evaluations(scheme):
    # Sec. 4.1: the stepper advances by the contact step, gravity is evaluated every k-th
    # step and held in between.  With the acceleration held at a0 for s < k steps, the
    # steppers reduce to constant-acceleration motion with closed forms:
    #   semi-implicit Euler: v_s = v0 + s dt a0, x_s = x0 + s dt v0 + dt^2 a0 s (s + 1) / 2
    #   KDK leapfrog:        v_s = v0 + s dt a0, x_s = x0 + s dt v0 + dt^2 a0 s^2 / 2
    # and at step k the acceleration is the force field at x_k (here the direct sum).
    pos, vel, m = inputs.rubble_pile(300, seed=21)
    eps, dt, k = 5e-3, 1e-3, 5
    a0, _ = oracle.direct(pos, m, eps)
    for s in range(1, k):
        p, v, a = oracle.step(pos, vel, m, a0, dt, s, scheme=scheme, use_tree=False, eps=eps,
                              grav_every=k)
        quad = s * (s + 1) / 2 if scheme == 1 else s * s / 2
        scale = np.abs(pos).max() + s * dt * np.abs(vel).max()
        assert np.abs(v - (vel + s * dt * a0)).max() <= 1e-13 * (np.abs(vel).max() + 1)
        assert np.abs(p - (pos + s * dt * vel + dt * dt * quad * a0)).max() <= 1e-14 * scale
        assert np.array_equal(a, a0)                      # held, not re-evaluated
    p, v, a = oracle.step(pos, vel, m, a0, dt, k, scheme=scheme, use_tree=False, eps=eps,
                          grav_every=k)
    assert np.array_equal(a, oracle.direct(p, m, eps)[0])   # evaluated at x_k
    # k = 1 (and 0) is the single-rate stepper; a run of 2k steps is two runs of k steps
    p1, v1, a1 = oracle.step(pos, vel, m, a0, dt, 7, scheme=scheme, use_tree=False, eps=eps)
    for ge in (0, 1):
        q = oracle.step(pos, vel, m, a0, dt, 7, scheme=scheme, use_tree=False, eps=eps,
                        grav_every=ge)
        assert all(np.array_equal(x, y) for x, y in zip(q, (p1, v1, a1)))
    r1 = oracle.step(pos, vel, m, a0, dt, 2 * k, scheme=scheme, use_tree=False, eps=eps,
                     grav_every=k)
    r2 = oracle.step(p, v, m, a, dt, k, scheme=scheme, use_tree=False, eps=eps, grav_every=k)
    assert all(np.array_equal(x, y) for x, y in zip(r1, r2))
