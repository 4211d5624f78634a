"""Thin ctypes binding of libgravity (include/gravity.h): argument marshalling only.

Every function keeps the name of the C entry point it calls.  Tensors are torch
CUDA tensors (float64, contiguous); work goes to the current torch stream of the
tensors' device.  Errors raise GravityError carrying the library's code.  There
is no CPU fallback: if libgravity.so is missing this module fails to import.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

GRAVITY_OK = 0
GRAVITY_E_ARG = -1
GRAVITY_E_NONFINITE = -2
GRAVITY_E_NOMEM = -3
GRAVITY_E_CUDA = -4
GRAVITY_E_TIMEOUT = -5
GRAVITY_E_INTERNAL = -6
GRAVITY_E_NOTREE = -7
GRAVITY_ADJ_END = 1
GRAVITY_ADJ_START = 2
GRAVITY_DBGSET_STACK_CAP = 1
GRAVITY_DBGSET_SORT_STALL = 2
GRAVITY_DBGSET_MOMENTS_STALL = 3

# gravity_alloc_fn / gravity_free_fn
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t,
                            ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

DBG_ROOT, DBG_KEYS, DBG_PERM, DBG_NNODES, DBG_TOPO, DBG_DEPTH, DBG_PARENT, DBG_MASS, DBG_COM, \
    DBG_QUAD, DBG_WALKSTATS = range(11)


class GravityError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__(f"{where}: {gravity_strerror(code)} ({code})")


class gravity_params(ctypes.Structure):
    _fields_ = [("G", ctypes.c_double), ("order", ctypes.c_int32), ("leaf_max", ctypes.c_int32),
                ("accum", ctypes.c_int32), ("mac_guard", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("walk_cfg", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("grav_every", ctypes.c_int32)]


def _load() -> ctypes.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libgravity.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    PP = ctypes.POINTER(gravity_params)
    sig = {
        "gravity_params_default": (None, [PP]),
        "gravity_create": (I, [ctypes.POINTER(P), I, P]),
        "gravity_destroy": (I, [P]),
        "gravity_set_stream": (I, [P, P]),
        "gravity_set_allocator": (I, [P, ALLOC_FN, FREE_FN, P]),
        "gravity_debug_set": (I, [P, I, I64]),
        "gravity_tree_build": (I, [P, I64, P, P, PP]),
        "gravity_forces": (I, [P, D, D, P]),
        "gravity_forces_counted": (I, [P, D, D, P, P]),
        "gravity_forces_vjp": (I, [P, D, D, P, P]),
        "gravity_direct": (I, [P, I64, P, P, D, D, P]),
        "gravity_diagnostics": (I, [P, I64, P, P, P, D, D, P]),
        "gravity_components": (I, [P, P, D, P, P]),
        "gravity_dt_g": (I, [D, D, ctypes.POINTER(D)]),
        "leapfrog_step": (I, [P, I64, P, P, P, P, D, I, D, D, PP]),
        "leapfrog_adjoint": (I, [P, I64, P, P, P, D, I, D, D, PP, I, P, P]),
        "gravity_forces_host": (I, [P, I64, P, P, D, D, PP, P]),
        "gravity_forces_host_batch": (I, [P, I64, I64, P, P, D, D, PP, P]),
        "gravity_sync": (I, [P]),
        "gravity_debug_export": (I, [P, I, P, ctypes.c_size_t]),
        "gravity_strerror": (ctypes.c_char_p, [I]),
        "gravity_stats": (I, [P, ctypes.POINTER(I64)]),
        "gravity_probe_fp32": (I, [P, I64, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "gravity_direct_noalloc": (I, [I64, P, P, D, D, P, P]),
        "gravity_set_clouds": (I, [P, ctypes.c_int32, P]),
        "gravity_walk_tasks": (I, [P, ctypes.POINTER(I64)]),
        "gravity_task_bodies": (I, [P, I64, I64, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
        "gravity_forces_range": (I, [P, D, D, I64, I64, P]),
        "gravity_scatter_sorted": (I, [P, I64, I64, P, P]),
        "gravity_kick_drift": (I, [P, I64, P, P, P, D, D]),
        "gravity_kick": (I, [P, I64, P, P, D]),
        "gravity_batch_tree_build": (I, [P, ctypes.c_int32, P, P, P, PP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def gravity_strerror(code: int) -> str:
    return _lib.gravity_strerror(int(code)).decode()


def _check(rc: int, where: str):
    if rc != GRAVITY_OK:
        raise GravityError(rc, where)


def params(**kw) -> gravity_params:
    """gravity_params with the library defaults, then the given fields."""
    p = gravity_params()
    _lib.gravity_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _dev(t: torch.Tensor, name: str, shape_last=None) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in (torch.float64, torch.int32, torch.int64) or not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous float64/int32/int64")
    if shape_last is not None and t.numel() and t.shape[-1] != shape_last:
        raise ValueError(f"{name} must have trailing dimension {shape_last}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_of(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Context:
    """Owns a gravity_ctx (scratch memory, current tree) on one device."""

    def __init__(self, device=None):
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                           torch.device(device).index or 0)
        self.device = dev
        h = ctypes.c_void_p()
        _check(_lib.gravity_create(ctypes.byref(h), dev.index, _stream_of(dev)), "gravity_create")
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("context destroyed")
        _lib.gravity_set_stream(self._h, _stream_of(self.device))
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _lib.gravity_destroy(self._h)
            self._h = None
        self._alloc_keep = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gravity_set_allocator(ctx: Context, alloc=None, release=None):
    """Route the context's device memory through Python callables alloc(nbytes) -> int
    device pointer (0 on failure) and release(ptr); both None restores cudaMalloc/cudaFree.
    The context's tree and scratch are released (see gravity.h)."""
    if (alloc is None) != (release is None):
        raise ValueError("give both alloc and release, or neither")
    if alloc is None:
        fa, ff = ALLOC_FN(), FREE_FN()
    else:
        def _a(pp, nbytes, _user):
            try:
                ptr = int(alloc(int(nbytes)))
            except Exception:
                return 1
            if not ptr:
                return 1
            pp[0] = ptr
            return 0

        def _f(ptr, _user):
            release(int(ptr))
        fa, ff = ALLOC_FN(_a), FREE_FN(_f)
    h = ctx.handle
    keep_old = getattr(ctx, "_alloc_keep", None)   # old callbacks stay alive for the release
    ctx._alloc_keep = (fa, ff)
    rc = _lib.gravity_set_allocator(h, fa, ff, None)
    if rc != GRAVITY_OK and keep_old is not None:
        ctx._alloc_keep = keep_old
    _check(rc, "gravity_set_allocator")


def use_torch_allocator(ctx: Context):
    """Give the context's device memory to PyTorch's caching allocator (one pool)."""
    dev, stream = ctx.device, torch.cuda.current_stream(ctx.device)
    gravity_set_allocator(ctx, lambda nbytes: torch.cuda.caching_allocator_alloc(nbytes, dev, stream),
                          torch.cuda.caching_allocator_delete)


def gravity_debug_set(ctx: Context, what: int, value: int):
    _check(_lib.gravity_debug_set(ctx.handle, int(what), int(value)), "gravity_debug_set")


def gravity_create(device=None) -> Context:
    return Context(device)


def gravity_destroy(ctx: Context):
    ctx.close()


def gravity_tree_build(ctx: Context, pos: torch.Tensor, mass: torch.Tensor, p=None):
    n = pos.shape[0] if pos.ndim else 0
    if mass.numel() != n:
        raise ValueError("pos and mass lengths differ")
    _check(_lib.gravity_tree_build(ctx.handle, n, _dev(pos, "pos", 3), _dev(mass, "mass"),
                                   None if p is None else ctypes.byref(p)), "gravity_tree_build")


def _offsets(offsets) -> np.ndarray:
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    if off.ndim != 1 or len(off) < 2:
        raise ValueError("offsets must be a 1-D array of nclouds + 1 entries")
    return off


def gravity_set_clouds(ctx: Context, offsets):
    """Independent clouds: cloud k = bodies offsets[k]:offsets[k+1] (host array)."""
    off = _offsets(offsets)
    _check(_lib.gravity_set_clouds(ctx.handle, len(off) - 1, off.ctypes.data_as(ctypes.c_void_p)),
           "gravity_set_clouds")


def gravity_batch_tree_build(ctx: Context, offsets, pos: torch.Tensor, mass: torch.Tensor,
                             p=None):
    off = _offsets(offsets)
    if int(off[-1]) != pos.shape[0] or mass.numel() != pos.shape[0]:
        raise ValueError("offsets[-1] must equal the number of bodies")
    _check(_lib.gravity_batch_tree_build(ctx.handle, len(off) - 1,
                                         off.ctypes.data_as(ctypes.c_void_p), _dev(pos, "pos", 3),
                                         _dev(mass, "mass"), None if p is None else ctypes.byref(p)),
           "gravity_batch_tree_build")


def gravity_forces(ctx: Context, theta: float, eps: float, acc: torch.Tensor) -> torch.Tensor:
    _check(_lib.gravity_forces(ctx.handle, float(theta), float(eps), _dev(acc, "acc", 3)),
           "gravity_forces")
    return acc


def gravity_walk_tasks(ctx: Context) -> int:
    n = ctypes.c_int64()
    _check(_lib.gravity_walk_tasks(ctx.handle, ctypes.byref(n)), "gravity_walk_tasks")
    return n.value


def gravity_task_bodies(ctx: Context, first_task: int, ntasks: int) -> tuple[int, int]:
    """(first sorted body, body count) of walk tasks [first_task, first_task + ntasks)."""
    b0, nb = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.gravity_task_bodies(ctx.handle, int(first_task), int(ntasks), ctypes.byref(b0),
                                    ctypes.byref(nb)), "gravity_task_bodies")
    return b0.value, nb.value


def gravity_forces_range(ctx: Context, theta: float, eps: float, first_task: int, ntasks: int,
                         acc_sorted: torch.Tensor) -> torch.Tensor:
    _, nb = gravity_task_bodies(ctx, first_task, ntasks)
    if acc_sorted.shape[0] < nb:
        raise ValueError(f"acc_sorted needs {nb} rows")
    _check(_lib.gravity_forces_range(ctx.handle, float(theta), float(eps), int(first_task),
                                     int(ntasks), _dev(acc_sorted, "acc_sorted", 3)),
           "gravity_forces_range")
    return acc_sorted


def gravity_scatter_sorted(ctx: Context, first_body: int, src_sorted: torch.Tensor,
                           dst: torch.Tensor, nbodies: int | None = None) -> torch.Tensor:
    nb = src_sorted.shape[0] if nbodies is None else int(nbodies)
    _check(_lib.gravity_scatter_sorted(ctx.handle, int(first_body), nb,
                                       _dev(src_sorted, "src_sorted", 3), _dev(dst, "dst", 3)),
           "gravity_scatter_sorted")
    return dst


def gravity_kick_drift(ctx: Context, pos: torch.Tensor, vel: torch.Tensor, acc: torch.Tensor,
                       h_kick: float, dt: float):
    _check(_lib.gravity_kick_drift(ctx.handle, pos.shape[0], _dev(pos, "pos", 3),
                                   _dev(vel, "vel", 3), _dev(acc, "acc", 3), float(h_kick),
                                   float(dt)), "gravity_kick_drift")


def gravity_kick(ctx: Context, vel: torch.Tensor, acc: torch.Tensor, h_kick: float):
    _check(_lib.gravity_kick(ctx.handle, vel.shape[0], _dev(vel, "vel", 3), _dev(acc, "acc", 3),
                             float(h_kick)), "gravity_kick")


def gravity_forces_counted(ctx: Context, theta: float, eps: float, acc: torch.Tensor,
                           counts: torch.Tensor) -> torch.Tensor:
    _check(_lib.gravity_forces_counted(ctx.handle, float(theta), float(eps), _dev(acc, "acc", 3),
                                       _dev(counts, "counts", 3)), "gravity_forces_counted")
    return acc


def gravity_forces_vjp(ctx: Context, theta: float, eps: float, lam: torch.Tensor,
                       grad: torch.Tensor) -> torch.Tensor:
    """grad = (d acc / d pos)^T lam on the current tree's frozen decisions (order 0)."""
    _check(_lib.gravity_forces_vjp(ctx.handle, float(theta), float(eps), _dev(lam, "lambda", 3),
                                   _dev(grad, "grad", 3)), "gravity_forces_vjp")
    return grad


def gravity_direct(ctx: Context, pos, mass, eps: float, G: float, acc) -> torch.Tensor:
    _check(_lib.gravity_direct(ctx.handle, pos.shape[0], _dev(pos, "pos", 3), _dev(mass, "mass"),
                               float(eps), float(G), _dev(acc, "acc", 3)), "gravity_direct")
    return acc


def gravity_diagnostics(ctx: Context, pos, vel, mass, eps: float, G: float,
                        out: torch.Tensor) -> torch.Tensor:
    """out (device, 7 float64) = E, P xyz, L xyz."""
    _check(_lib.gravity_diagnostics(ctx.handle, pos.shape[0], _dev(pos, "pos", 3),
                                    _dev(vel, "vel", 3), _dev(mass, "mass"), float(eps), float(G),
                                    _dev(out, "out")), "gravity_diagnostics")
    return out


def gravity_components(ctx: Context, label: torch.Tensor, radius: torch.Tensor = None,
                       dmax: float = 0.0, counts: torch.Tensor = None):
    """Contact-graph components of the current tree's bodies: label (device int32, n) gets
    the smallest caller index of each body's component; counts (device int64, 2), if
    given, the number of components and of aggregates (components of > 1 body).  Contact:
    |x_i - x_j| <= radius_i + radius_j, or <= dmax without radii."""
    if counts is not None and (counts.dtype != torch.int64 or counts.numel() < 2):
        raise TypeError("counts must be an int64 tensor of 2 elements")
    if label.dtype != torch.int32:
        raise TypeError("label must be int32")
    _check(_lib.gravity_components(ctx.handle, None if radius is None else _dev(radius, "radius"),
                                   float(dmax), _dev(label, "label"),
                                   None if counts is None else _dev(counts, "counts")),
           "gravity_components")
    return label, counts


def gravity_dt_g(G: float, rho: float) -> float:
    """Largest gravity time step of Eq. (dt_g): 1 / (2 sqrt(G rho)), rho the material density."""
    out = ctypes.c_double()
    _check(_lib.gravity_dt_g(float(G), float(rho), ctypes.byref(out)), "gravity_dt_g")
    return out.value


def gravity_direct_noalloc(pos, mass, eps: float, G: float, acc) -> torch.Tensor:
    """Direct sum with no context and no allocation (n <= 65536); see gravity.h."""
    _check(_lib.gravity_direct_noalloc(pos.shape[0], _dev(pos, "pos", 3), _dev(mass, "mass"),
                                       float(eps), float(G), _dev(acc, "acc", 3),
                                       _stream_of(pos.device)), "gravity_direct_noalloc")
    return acc


def leapfrog_step(ctx: Context, pos, vel, mass, acc_cache, dt: float, nsteps: int, theta: float,
                  eps: float, p=None):
    _check(_lib.leapfrog_step(ctx.handle, pos.shape[0], _dev(pos, "pos", 3), _dev(vel, "vel", 3),
                              _dev(mass, "mass"), _dev(acc_cache, "acc_cache", 3), float(dt),
                              int(nsteps), float(theta), float(eps),
                              None if p is None else ctypes.byref(p)), "leapfrog_step")


def leapfrog_adjoint(ctx: Context, pos0, vel0, mass, dt: float, nsteps: int, theta: float,
                     eps: float, p, flags: int, xbar, vbar):
    """Reverse pass of a checkpointed leapfrog segment; xbar, vbar updated in place."""
    _check(_lib.leapfrog_adjoint(ctx.handle, pos0.shape[0], _dev(pos0, "pos0", 3),
                                 _dev(vel0, "vel0", 3), _dev(mass, "mass"), float(dt), int(nsteps),
                                 float(theta), float(eps), None if p is None else ctypes.byref(p),
                                 int(flags), _dev(xbar, "xbar", 3), _dev(vbar, "vbar", 3)),
           "leapfrog_adjoint")


def gravity_forces_host(ctx: Context, pos_host: torch.Tensor, mass_host: torch.Tensor,
                        theta: float, eps: float, p, acc_host: torch.Tensor):
    for name, t in (("pos_host", pos_host), ("mass_host", mass_host), ("acc_host", acc_host)):
        if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float64 host tensor")
    _check(_lib.gravity_forces_host(ctx.handle, pos_host.shape[0],
                                    ctypes.c_void_p(pos_host.data_ptr()),
                                    ctypes.c_void_p(mass_host.data_ptr()), float(theta),
                                    float(eps), None if p is None else ctypes.byref(p),
                                    ctypes.c_void_p(acc_host.data_ptr())), "gravity_forces_host")
    return acc_host


def gravity_forces_host_batch(ctx: Context, pos_host: list, mass_host: list, theta: float,
                              eps: float, p, acc_host: list):
    """Snapshots k = 0 .. K-1: pos_host[k] (n, 3), mass_host[k] (n,) -> acc_host[k] (n, 3),
    all contiguous float64 host tensors (pinned for overlap); the copies of a snapshot
    overlap the build and walk of its neighbours."""
    k = len(pos_host)
    if len(mass_host) != k or len(acc_host) != k:
        raise ValueError("pos_host, mass_host and acc_host need one tensor per snapshot")
    n = pos_host[0].shape[0] if k else 0
    for name, ts in (("pos_host", pos_host), ("mass_host", mass_host), ("acc_host", acc_host)):
        for t in ts:
            if t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or t.shape[0] != n:
                raise TypeError(f"{name} must hold contiguous float64 host tensors of {n} rows")
    arr = ctypes.c_void_p * max(k, 1)
    pp = arr(*[t.data_ptr() for t in pos_host])
    mp = arr(*[t.data_ptr() for t in mass_host])
    ap = arr(*[t.data_ptr() for t in acc_host])
    _check(_lib.gravity_forces_host_batch(ctx.handle, k, n, pp, mp, float(theta), float(eps),
                                          None if p is None else ctypes.byref(p), ap),
           "gravity_forces_host_batch")
    return acc_host


def gravity_stats(ctx: Context) -> int:
    """Kernels enqueued by this context so far."""
    v = ctypes.c_int64(0)
    _check(_lib.gravity_stats(ctx.handle, ctypes.byref(v)), "gravity_stats")
    return int(v.value)


def gravity_probe_fp32(ctx: Context, iters: int = 20000):
    """(ms, FLOP/s) of the FFMA-chain probe."""
    ms, fl = ctypes.c_double(0), ctypes.c_double(0)
    _check(_lib.gravity_probe_fp32(ctx.handle, int(iters), ctypes.byref(ms), ctypes.byref(fl)),
           "gravity_probe_fp32")
    return ms.value, fl.value


def gravity_sync(ctx: Context):
    _check(_lib.gravity_sync(ctx.handle), "gravity_sync")


_DBG_DTYPES = {DBG_ROOT: (np.float64, 4), DBG_KEYS: (np.uint64, 1), DBG_PERM: (np.uint32, 1),
               DBG_TOPO: (np.int32, 4), DBG_DEPTH: (np.int32, 1), DBG_PARENT: (np.int32, 1),
               DBG_MASS: (np.float64, 1), DBG_COM: (np.float64, 3), DBG_QUAD: (np.float64, 6),
               DBG_WALKSTATS: (np.uint64, 16)}


def gravity_debug_export(ctx: Context, what: int, n: int) -> np.ndarray:
    """Copy a tree array to a numpy array (n = bodies for KEYS/PERM, ignored otherwise)."""
    if what == DBG_NNODES:
        out = np.zeros(1, np.int32)
        _check(_lib.gravity_debug_export(ctx.handle, what, out.ctypes.data_as(ctypes.c_void_p), 4),
               "gravity_debug_export")
        return out
    dt, width = _DBG_DTYPES[what]
    if what == DBG_ROOT:
        count = max(1, int(n))          # n = number of clouds for the root cubes
    elif what == DBG_WALKSTATS:
        count = 1
    elif what in (DBG_KEYS, DBG_PERM):
        count = n
    else:
        count = int(gravity_debug_export(ctx, DBG_NNODES, n)[0])
    flat = what == DBG_WALKSTATS or width == 1
    out = np.zeros((count * width,) if flat else (count, width), dt)
    _check(_lib.gravity_debug_export(ctx.handle, what, out.ctypes.data_as(ctypes.c_void_p),
                                     out.nbytes), "gravity_debug_export")
    return out


# ----------------------------------------------------------------- convenience
class Gravity:
    """Octree gravity on one device: build + forces + direct + stepping."""

    def __init__(self, device=None, **param_kw):
        self.ctx = Context(device)
        self.p = params(**param_kw)

    def tree_build(self, pos, mass):
        gravity_tree_build(self.ctx, pos, mass, self.p)

    def forces(self, theta, eps, acc=None, n=None):
        if acc is None:
            acc = torch.empty((n, 3), dtype=torch.float64, device=self.ctx.device)
        return gravity_forces(self.ctx, theta, eps, acc)

    def evaluate(self, pos, mass, theta, eps, acc=None):
        self.tree_build(pos, mass)
        return self.forces(theta, eps, acc, n=pos.shape[0])

    def direct(self, pos, mass, eps, acc=None):
        if acc is None:
            acc = torch.empty_like(pos)
        return gravity_direct(self.ctx, pos, mass, eps, self.p.G, acc)

    def step(self, pos, vel, mass, acc_cache, dt, nsteps, theta, eps):
        leapfrog_step(self.ctx, pos, vel, mass, acc_cache, dt, nsteps, theta, eps, self.p)

    def sync(self):
        gravity_sync(self.ctx)
