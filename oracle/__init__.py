"""FP64 CPU oracle for the Barnes-Hut octree gravity path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may load this package; the library under
``paper_1912_04197_gb300`` never does, and the two share no code.

The arithmetic lives in ``oracle.cpp`` (plain recursive C++, FP64, built with
``-ffp-contract=off``); this module compiles it with g++ on first use and wraps
it with ctypes.  Every function cites the passage of the paper (Ferrari,
Lavagna, Blazquez 2019, arXiv:1912.04197) that it follows in ``oracle.cpp``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_E_ARG, ORC_E_NONFINITE = 0, -1, -2


def build(force: bool = False) -> str:
    """Compile oracle.cpp into _build/liboracle.so (g++, OpenMP, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            D = ctypes.c_double
            I = ctypes.c_int
            lib.orc_root_cube.argtypes = [I64, P, P, P]
            lib.orc_root_cube.restype = I
            lib.orc_morton_keys.argtypes = [I64, P, P, D, P]
            lib.orc_morton_keys.restype = None
            lib.orc_sort.argtypes = [I64, P, P]
            lib.orc_sort.restype = None
            lib.orc_tree_build.argtypes = [I64, P, P, I, I, ctypes.POINTER(I)]
            lib.orc_tree_build.restype = P
            lib.orc_tree_free.argtypes = [P]
            lib.orc_tree_free.restype = None
            lib.orc_tree_num_nodes.argtypes = [P]
            lib.orc_tree_num_nodes.restype = I64
            lib.orc_tree_geometry.argtypes = [P, P, P]
            lib.orc_tree_geometry.restype = None
            lib.orc_tree_export_order.argtypes = [P, P, P]
            lib.orc_tree_export_order.restype = None
            lib.orc_tree_export_nodes.argtypes = [P, P, P, P, P, P, P, P]
            lib.orc_tree_export_nodes.restype = None
            lib.orc_tree_export_moments.argtypes = [P, P, P, P]
            lib.orc_tree_export_moments.restype = None
            lib.orc_tree_forces.argtypes = [P, D, D, D, I, I64, P, P, P, P]
            lib.orc_tree_forces.restype = None
            lib.orc_tree_vjp.argtypes = [P, D, D, D, I, P, P, P]
            lib.orc_tree_vjp.restype = I
            lib.orc_tree_forces_frozen.argtypes = [P, D, D, D, I, P, P]
            lib.orc_tree_forces_frozen.restype = I
            lib.orc_direct.argtypes = [I64, P, P, D, D, I64, P, P, P]
            lib.orc_direct.restype = None
            lib.orc_leapfrog.argtypes = [I64, P, P, P, P, D, I, I, I, D, D, D, I, I, I, I]
            lib.orc_leapfrog.restype = I
            lib.orc_set_threads.argtypes = [I]
            lib.orc_set_threads.restype = None
            lib.orc_diagnostics.argtypes = [I64, P, P, P, D, D, P]
            lib.orc_diagnostics.restype = None
            lib.orc_components.argtypes = [I64, P, P, D, P, P]
            lib.orc_components.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape_last=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape_last is not None and a.size and a.shape[-1] != shape_last:
        raise ValueError("expected trailing dimension %d" % shape_last)
    return a


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__({ORC_E_ARG: "invalid argument",
                          ORC_E_NONFINITE: "non-finite position"}.get(code, str(code)))
        self.code = code


def root_cube(pos):
    """Kernel 1 of the paper's list (Sec. 2.1): root cube (lo[3], side)."""
    pos = _f64(pos, 3)
    lo = np.zeros(3)
    side = np.zeros(1)
    rc = _load().orc_root_cube(len(pos), _ptr(pos), _ptr(lo), _ptr(side))
    if rc:
        raise OracleError(rc)
    return lo, float(side[0])


def morton_keys(pos, lo, side):
    """63-bit Morton keys on the 2^21 grid of the root cube (naive bit loop)."""
    pos = _f64(pos, 3)
    lo = _f64(lo)
    keys = np.zeros(len(pos), dtype=np.uint64)
    _load().orc_morton_keys(len(pos), _ptr(pos), _ptr(lo), float(side), _ptr(keys))
    return keys


def stable_order(keys):
    """Stable sort of caller indices by key ("sort bodies", Sec. 2.1)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    perm = np.zeros(len(keys), dtype=np.int64)
    _load().orc_sort(len(keys), _ptr(keys), _ptr(perm))
    return perm


class Tree:
    """Octree of kernels 1-4 of the paper's list (Sec. 2.1), FP64, DFS preorder."""

    def __init__(self, pos, mass, leaf_max: int = 1, order: int = 0):
        self.pos = _f64(pos, 3).reshape(-1, 3)
        self.mass = _f64(mass).reshape(-1)
        if len(self.mass) != len(self.pos):
            raise ValueError("pos and mass lengths differ")
        st = ctypes.c_int(0)
        lib = _load()
        self._h = lib.orc_tree_build(len(self.pos), _ptr(self.pos), _ptr(self.mass),
                                     int(leaf_max), int(order), ctypes.byref(st))
        if not self._h:
            raise OracleError(st.value)
        self.n = len(self.pos)
        self.leaf_max = leaf_max
        self.order = order

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().orc_tree_free(h)
            self._h = None

    @property
    def num_nodes(self) -> int:
        return int(_load().orc_tree_num_nodes(self._h))

    def geometry(self):
        lo = np.zeros(3)
        side = np.zeros(1)
        _load().orc_tree_geometry(self._h, _ptr(lo), _ptr(side))
        return lo, float(side[0])

    def order_arrays(self):
        keys = np.zeros(self.n, dtype=np.uint64)
        perm = np.zeros(self.n, dtype=np.int64)
        _load().orc_tree_export_order(self._h, _ptr(keys), _ptr(perm))
        return keys, perm

    def nodes(self) -> dict:
        k = self.num_nodes
        out = dict(depth=np.zeros(k, np.int32), begin=np.zeros(k, np.int64),
                   end=np.zeros(k, np.int64), n_child=np.zeros(k, np.int32),
                   parent=np.zeros(k, np.int64), prefix=np.zeros(k, np.uint64),
                   leaf=np.zeros(k, np.int32))
        _load().orc_tree_export_nodes(self._h, *(_ptr(out[f]) for f in
                                                ("depth", "begin", "end", "n_child", "parent",
                                                 "prefix", "leaf")))
        return out

    def moments(self):
        k = self.num_nodes
        m = np.zeros(k)
        com = np.zeros((k, 3))
        quad = np.zeros((k, 6))
        _load().orc_tree_export_moments(self._h, _ptr(m), _ptr(com), _ptr(quad))
        return m, com, quad

    def forces(self, theta: float, eps: float, G: float = 1.0, mac_guard: int = 1,
               targets=None):
        """Kernel 5 (Sec. 2.1): (acc[ntarg,3], absum[ntarg], counts[ntarg,3]).

        counts columns: MAC tests, node terms accepted, body-body terms."""
        if theta < 0 or eps < 0:
            raise OracleError(ORC_E_ARG)
        t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
        nt = self.n if t is None else len(t)
        acc = np.zeros((nt, 3))
        absum = np.zeros(nt)
        counts = np.zeros((nt, 3), dtype=np.int64)
        _load().orc_tree_forces(self._h, float(theta), float(eps), float(G), int(mac_guard),
                                nt, _ptr(t), _ptr(acc), _ptr(absum), _ptr(counts))
        return acc, absum, counts


def tree_vjp(tree: "Tree", lam, theta: float, eps: float, G: float = 1.0, mac_guard: int = 1,
             with_absum: bool = False):
    """(d acc / d pos)^T lam on the frozen tree (monopole), caller order (n,3).
    with_absum: also return per body the sum of |term| magnitudes it takes part in."""
    lam = _f64(lam, 3).reshape(-1, 3)
    grad = np.zeros((tree.n, 3))
    absum = np.zeros(tree.n) if with_absum else None
    rc = _load().orc_tree_vjp(tree._h, float(theta), float(eps), float(G), int(mac_guard),
                              _ptr(lam), _ptr(grad), _ptr(absum))
    if rc:
        raise OracleError(rc)
    return (grad, absum) if with_absum else grad


def tree_forces_frozen(tree: "Tree", pos_new, theta: float, eps: float, G: float = 1.0,
                       mac_guard: int = 1):
    """Accelerations at pos_new with the decisions of the tree's own positions."""
    pos_new = _f64(pos_new, 3).reshape(-1, 3)
    acc = np.zeros((tree.n, 3))
    rc = _load().orc_tree_forces_frozen(tree._h, float(theta), float(eps), float(G),
                                        int(mac_guard), _ptr(pos_new), _ptr(acc))
    if rc:
        raise OracleError(rc)
    return acc


def direct(pos, mass, eps: float, G: float = 1.0, targets=None):
    """Eq. (Newton) with softening (Eq. Force_rComp): (acc[ntarg,3], absum[ntarg])."""
    pos = _f64(pos, 3).reshape(-1, 3)
    mass = _f64(mass).reshape(-1)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = len(pos) if t is None else len(t)
    acc = np.zeros((nt, 3))
    absum = np.zeros(nt)
    _load().orc_direct(len(pos), _ptr(pos), _ptr(mass), float(eps), float(G), nt, _ptr(t),
                       _ptr(acc), _ptr(absum))
    return acc, absum


def tree_forces(pos, mass, theta, eps, G=1.0, leaf_max=1, order=0, mac_guard=1):
    """Convenience: build the tree and return accelerations of all bodies."""
    return Tree(pos, mass, leaf_max, order).forces(theta, eps, G, mac_guard)[0]


def step(pos, vel, mass, acc, dt, nsteps, *, scheme=0, use_tree=True, theta=0.5, eps=0.0,
         G=1.0, leaf_max=1, order=0, mac_guard=1, grav_every=1):
    """Symplectic stepping (Sec. 2.3): scheme 0 = KDK leapfrog, 1 = semi-implicit Euler;
    with grav_every = k > 1, gravity is evaluated only every k-th step and held in between
    (the two time steps of Sec. 4.1).

    Returns new (pos, vel, acc); inputs are not modified."""
    pos = _f64(pos, 3).reshape(-1, 3).copy()
    vel = _f64(vel, 3).reshape(-1, 3).copy()
    mass = _f64(mass).reshape(-1)
    acc = _f64(acc, 3).reshape(-1, 3).copy()
    rc = _load().orc_leapfrog(len(pos), _ptr(pos), _ptr(vel), _ptr(mass), _ptr(acc), float(dt),
                              int(nsteps), int(scheme), int(bool(use_tree)), float(theta),
                              float(eps), float(G), int(leaf_max), int(order), int(mac_guard),
                              int(grav_every))
    if rc:
        raise OracleError(rc)
    return pos, vel, acc


def set_threads(n: int = 0):
    """Host threads of the oracle's parallel loops (0 = all cores); for timing only."""
    _load().orc_set_threads(int(n))


def diagnostics(pos, vel, mass, eps, G=1.0):
    """Conserved quantities (Sec. 3.1): E, P[3], L[3]."""
    pos = _f64(pos, 3).reshape(-1, 3)
    vel = _f64(vel, 3).reshape(-1, 3)
    mass = _f64(mass).reshape(-1)
    out = np.zeros(7)
    _load().orc_diagnostics(len(pos), _ptr(pos), _ptr(vel), _ptr(mass), float(eps), float(G),
                            _ptr(out))
    return float(out[0]), out[1:4].copy(), out[4:7].copy()


def components(pos, radius=None, dmax=0.0):
    """Aggregate identification (Sec. 2): contact-graph components by depth-first search.
    Contact: |x_i - x_j| <= r_i + r_j (radius given) or <= dmax.  Returns (label, counts):
    label[i] = smallest index of i's component; counts = (components, components of > 1)."""
    pos = _f64(pos, 3).reshape(-1, 3)
    n = len(pos)
    r = None if radius is None else _f64(radius).reshape(-1)
    label = np.zeros(n, np.int32)
    counts = np.zeros(2, np.int64)
    _load().orc_components(n, _ptr(pos), _ptr(r), float(dmax), _ptr(label), _ptr(counts))
    return label, (int(counts[0]), int(counts[1]))


def leapfrog_grad(pos0, vel0, mass, xbar, vbar, dt, nsteps, *, theta=0.5, eps=1e-3, G=1.0,
                  leaf_max=1, mac_guard=1):
    """Reverse-mode gradient of KDK leapfrog (Sec. 2.3) with the tree's decisions frozen
    at every step: given the cotangents (xbar, vbar) of (x_N, v_N), return those of
    (x_0, v_0).  With h = dt/2 the step is kick(h), drift(dt), kick(h); reversing
    kick(h) adds h J(x)^T vbar to xbar, reversing drift(dt) adds dt xbar to vbar; the
    two kicks at an interior time level share one vbar, so they combine to dt."""
    mass = _f64(mass).reshape(-1)
    x = _f64(pos0, 3).reshape(-1, 3).copy()
    v = _f64(vel0, 3).reshape(-1, 3).copy()
    a = tree_forces(x, mass, theta, eps, G, leaf_max=leaf_max, mac_guard=mac_guard)
    xs = [x.copy()]
    for _ in range(nsteps):
        x, v, a = step(x, v, mass, a, dt, 1, theta=theta, eps=eps, G=G, leaf_max=leaf_max,
                       mac_guard=mac_guard)
        xs.append(x.copy())

    return leapfrog_reverse(xs, mass, xbar, vbar, dt, theta=theta, eps=eps, G=G,
                            leaf_max=leaf_max, mac_guard=mac_guard)


def leapfrog_reverse(levels, mass, xbar, vbar, dt, *, theta=0.5, eps=1e-3, G=1.0, leaf_max=1,
                     mac_guard=1):
    """The reverse pass of leapfrog_grad on given positions levels[0..N] (each (n,3)):
    xbar += h J(x_N)^T vbar; then for k = N-1 .. 0: vbar += dt xbar (drift of step k),
    xbar += c_k J(x_k)^T vbar with c_0 = h = dt/2 and c_k = dt otherwise."""
    mass = _f64(mass).reshape(-1)
    nsteps = len(levels) - 1

    def jt(xn, u):
        return tree_vjp(Tree(xn, mass, leaf_max=leaf_max), u, theta, eps, G, mac_guard)

    h = 0.5 * dt
    xb = _f64(xbar, 3).reshape(-1, 3).copy()
    vb = _f64(vbar, 3).reshape(-1, 3).copy()
    xb += h * jt(levels[nsteps], vb)
    for k in range(nsteps - 1, -1, -1):
        vb += dt * xb
        xb += (h if k == 0 else dt) * jt(levels[k], vb)
    return xb, vb
