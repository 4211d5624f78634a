"""Autotuner of the walk's launch shape (gravity_params.walk_cfg).

The walk kernel has run-time shapes (flush threshold of the term lists, resident
blocks per SM, per-SM or global task queues).  tune_walk() times gravity_forces
with each shape on the caller's tree and returns the fastest; results are cached
in a JSON file per (device, order, leaf_max, size class, clouds), so a workload
class is tuned once.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import gravity as g

N_CONFIGS = 18
CACHE = os.environ.get("GRAVITY_TUNE_CACHE",
                       os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build",
                                    "walk_tune.json"))


def _key(order, leaf_max, n, clouds, theta):
    name = torch.cuda.get_device_name()
    return f"{name}|order{order}|leaf{leaf_max}|n2^{int(round(math.log2(max(n, 1))))}" \
           f"|clouds{int(clouds > 1)}|theta{theta:g}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune_walk(ctx: g.Context, pos: torch.Tensor, mass: torch.Tensor, p, theta: float, eps: float,
              clouds: int = 1, reps: int = 3, use_cache: bool = True) -> int:
    """Best walk_cfg for this tree and workload; the tree is (re)built with p."""
    n = pos.shape[0]
    key = _key(p.order, p.leaf_max, n, clouds, theta)
    cache = _load() if use_cache else {}
    if key in cache:
        return int(cache[key]["cfg"])
    g.gravity_tree_build(ctx, pos, mass, p)
    acc = torch.empty_like(pos)
    stream = torch.cuda.current_stream()
    saved = p.walk_cfg
    times = []
    for cfg in range(N_CONFIGS):
        p.walk_cfg = cfg
        g.gravity_tree_build(ctx, pos, mass, p)           # params travel with the tree
        g.gravity_forces(ctx, theta, eps, acc)            # warm-up
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.gravity_forces(ctx, theta, eps, acc)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        times.append(best)
    g.gravity_sync(ctx)
    p.walk_cfg = saved
    cfg = min(range(N_CONFIGS), key=lambda i: times[i])
    if use_cache:
        cache = _load()
        cache[key] = {"cfg": cfg, "ms": times[cfg], "all_ms": [round(t, 4) for t in times]}
        _store(cache)
    return cfg
