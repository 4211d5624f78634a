#!/usr/bin/env python3
"""Octree body-forces/s at N = 1,048,576, theta = 0.5 on GB300, vs the direct sum.

Workload: the clumpy aggregate (64 truncated Plummer spheres of scale 0.05 with
centres uniform in the unit sphere, equal masses, at rest), eps = 1e-3, seeded
synthetic data.  One step = one full force evaluation: gravity_tree_build (root
cube, Morton keys, radix sort, octree, moments) + gravity_forces (the walk).
The reported (order, leaf_max) is the fastest that meets the <= 1e-3 median force
error against the direct sum, which is checked on every run.

Timing: W warm-up steps, then exactly K steps timed with CUDA events on the
launching stream; the L2 (129 MB) is flushed by writing a 256 MB buffer before each
timed step (outside the events).  Under torchrun each rank evaluates its own
independent cloud (weak scaling, replicas only); rank 0 prints the max over ranks.

--impl reference times the FP64 CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "octree body-forces/s at N=1M, θ=0.5 vs direct N² on GB300 at ≤1e-3 force error"
UNIT = "body-forces/s"
# Algorithmic FLOPs per unit of walk work (counted from the formulas, FMA = 2):
#   point term (node monopole or body-body): d 3, r^2 6, 1/sqrt 2, r^-3 2, m r^-3 1, accumulate 6
#   quadrupole node term: d 3, r^2 6, 1/sqrt 2, r^-3..r^-7 4, Q d 15, d.Q d 5, 5/2 dQd r^-7 2,
#                         m r^-3 + that 2, accumulate s d - Q d r^-5 12
#   opening test: d 3, D^2 5, theta^2 D^2 1, compare 1
FLOP_POINT, FLOP_QUAD, FLOP_MAC = 20, 51, 10
#   vector-Jacobian product term: d 3, r^2 6, 1/sqrt 2, r^-2 1, r^-3 1, m r^-3 1, d.u 5,
#                                 3 (d.u) r^-2 2, w = s (u - c d) 9, own sum 3, source sum 3
FLOP_VJP = 36
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--experiment", choices=["accuracy", "sweep", "vjp"], default=None,
                    help="run one of the paper's Sec. 3.2 experiments instead of the benchmark")
    ap.add_argument("--n", type=int, default=1_048_576)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--leaf-max", type=int, default=16)
    ap.add_argument("--accum", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-direct", action="store_true", help="skip the direct-sum comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="oracle targets in cpu_baseline (0 = every body: the whole evaluation)")
    ap.add_argument("--cpu-reps", type=int, default=3, help="cpu_baseline repetitions (median)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble leg")
    ap.add_argument("--no-tune", action="store_true", help="default walk shape, no autotuning")
    ap.add_argument("--ensemble-steps", type=int, default=50)
    ap.add_argument("--no-grad", action="store_true", help="skip the gradient (adjoint) leg")
    ap.add_argument("--no-pipelined", action="store_true",
                    help="skip the two-stream throughput of independent evaluations")
    ap.add_argument("--no-components", action="store_true",
                    help="skip the aggregate-identification leg")
    ap.add_argument("--sweep-sizes", default="",
                    help="--experiment sweep: comma-separated body counts (default 10 .. 1e7)")
    ap.add_argument("--sweep-thetas", default="0.1,0.25,0.5,0.75",
                    help="--experiment sweep: opening angles of the tree rows")
    ap.add_argument("--sweep-steps", type=int, default=50,
                    help="--experiment sweep: timed steps per row up to 1e6 bodies (10 above)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the theta / order / accumulator sweep (runs with the direct-sum leg)")
    ap.add_argument("--fp64-sample", type=int, default=65536,
                    help="bodies of the FP64 direct-sum reference computed by the oracle in the "
                         "cpu_baseline leg (0 = none)")
    ap.add_argument("--shard", action="store_true",
                    help="N > 1: one cloud split between the ranks (replicated build, a range "
                         "of the walk per rank, one all-gather; strong scaling) instead of one "
                         "independent cloud per rank")
    return ap.parse_args()


def workload(args):
    """The benchmark's configuration, the same for both arms (the arithmetic each arm
    computes in is reported in its own dtype / precision keys)."""
    return {"workload": f"clumpy aggregate: {args.n} bodies in 64 Plummer spheres (a=0.05, r<=10a) "
                        f"uniform in the unit sphere, equal masses, at rest",
            "n": args.n, "theta": args.theta, "eps": args.eps, "order": args.order,
            "leaf_max": args.leaf_max, "mac_guard": 1,
            "step": "tree build + walk (one full force evaluation)",
            "l2": "flushed before each timed step (256 MB write)", "seed": args.seed}


def gen(args, rank):
    from paper_1912_04197_gb300 import inputs
    return inputs.clumpy_plummer(args.n, seed=args.seed + (0 if args.shard else rank))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows
                                                         if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


# ----------------------------------------------------------------------------- CPU oracle
def max_over_ranks(x: float, world: int, device=None) -> float:
    """Largest x over all ranks: one all-reduce (the identity on a single rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n_per_rank: int, world: int, t_max_ms: float) -> float:
    """Body-forces/s of the whole job: every rank's bodies over the slowest rank's time."""
    return world * n_per_rank / (t_max_ms * 1e-3)


def oracle_eval(pos, m, args, ntarg, with_forces=False):
    """Oracle tree build (all bodies) + walk of ntarg seeded targets (every body when
    ntarg = N); returns body-forces/s of the evaluation (scaled to N targets when
    sampled), the build and walk times and, on request, the walk's (targets, acc, absum)."""
    import oracle
    from paper_1912_04197_gb300 import inputs
    idx = None if ntarg >= len(pos) else inputs.subset(len(pos), ntarg, seed=7)
    t0 = time.perf_counter()
    tree = oracle.Tree(pos, m, leaf_max=args.leaf_max, order=args.order)
    t1 = time.perf_counter()
    acc, absum, _ = tree.forces(args.theta, args.eps, targets=idx)
    t2 = time.perf_counter()
    t_build, t_walk = t1 - t0, t2 - t1
    full = t_build + t_walk * len(pos) / (len(pos) if idx is None else len(idx))
    out = (len(pos) / full, t_build, t_walk)
    return out + ((idx, acc, absum),) if with_forces else out


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def parity_figures(a_gpu, ref, absum):
    """Per-body parity of the GPU walk against the oracle's walk (the tests' rule):
    rel = |d| / max(|a|, 1e-3 rms|a|), scale = |d| / sum|t|, kappa = sum|t| / max(...)."""
    d = np.linalg.norm(a_gpu - ref, axis=1)
    r = np.linalg.norm(ref, axis=1)
    den = np.maximum(r, 1e-3 * np.sqrt(np.mean(r * r)))
    rel, scale, kappa = d / den, d / np.maximum(absum, 1e-300), absum / den
    over = rel > 1e-5
    return {"bodies": int(len(rel)), "rel_max": float(rel.max()), "rel_median": float(np.median(rel)),
            "over_1e-5": int(over.sum()), "scale_max": float(scale.max()),
            "kappa_of_over_min": float(kappa[over].min()) if over.any() else None}


def cpu_baseline_leg(pos, m, args, gpu):
    """The FP64 oracle on the host cores: (1) the whole evaluation of the benchmark's
    configuration (tree build + walk of every body), timed: the CPU baseline; its forces
    also give the GPU walk's parity figures against the oracle; (2) the oracle's FP64
    direct sum of `--fp64-sample` seeded bodies (all N sources), timed: the CPU direct-sum
    baseline, and the reference for the error of every GPU configuration sampled in
    `gpu["sampled"]` (median / 99th percentile of |a - a_FP64| / |a_FP64|)."""
    import oracle
    from paper_1912_04197_gb300 import inputs
    ntarg = args.cpu_sample if 0 < args.cpu_sample < len(pos) else len(pos)
    runs = [oracle_eval(pos, m, args, ntarg, with_forces=(k == 0))
            for k in range(max(1, args.cpu_reps))]
    idx, oacc, oabs = runs[0][3]
    val, tb, tw = sorted(r[:3] for r in runs)[len(runs) // 2]
    what = ("every body (the whole evaluation, no extrapolation)" if ntarg == len(pos)
            else f"{ntarg} seeded targets, scaled to N targets")
    cpu = {"value": val, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
           "sample": f"FP64 oracle on the same workload: tree build of all {len(pos)} bodies "
                     f"({tb:.2f} s, 1 thread) + walk of {what} ({tw:.2f} s, OpenMP); "
                     f"median of {len(runs)} runs"}
    # one core: the build is single-threaded already; a walk of a seeded sample on one thread
    oracle.set_threads(1)
    try:
        n1 = min(16384, len(pos))
        v1, tb1, tw1 = oracle_eval(pos, m, args, n1)
    finally:
        oracle.set_threads(0)
    cpu["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"tree build of all {len(pos)} bodies ({tb1:.2f} s) + walk of "
                                      f"{n1} seeded targets on one thread ({tw1:.2f} s), scaled to "
                                      f"N targets"}
    # the smaller configurations in full: direct sum and tree (build + walk of every body),
    # all cores (configs of the plain method and the rubble pile)
    from paper_1912_04197_gb300 import inputs as _inp
    small = []
    for label, (sp, _, sm), kw, eps_s in (
            ("plain method: 2048 bodies uniform in a sphere", _inp.uniform_sphere(2048, seed=0),
             dict(leaf_max=1, order=0), 1e-3),
            ("rubble pile: 100,000 bodies", _inp.rubble_pile(100_000, seed=0),
             dict(leaf_max=16, order=2), 5e-3)):
        t0 = time.perf_counter()
        oracle.direct(sp, sm, eps_s)
        t1 = time.perf_counter()
        oracle.Tree(sp, sm, **kw).forces(args.theta, eps_s)
        t2 = time.perf_counter()
        small.append({"workload": label, "n": len(sp), "direct_s": t1 - t0,
                      "direct_value": len(sp) / (t1 - t0), "tree_s": t2 - t1,
                      "tree_value": len(sp) / (t2 - t1), "unit": UNIT, "tree": kw})
    cpu["smaller_configs"] = small
    acc_gpu = gpu["acc"] if idx is None else gpu["acc"][idx]
    parity = parity_figures(acc_gpu, oacc, oabs)
    parity["against"] = "the oracle's walk of the same tree configuration (FP64)"
    accuracy = None
    if args.fp64_sample > 0:
        sidx = gpu["sample_idx"]
        t0 = time.perf_counter()
        ref, _ = oracle.direct(pos, m, args.eps, targets=sidx)
        t_dir = time.perf_counter() - t0
        rn = np.linalg.norm(ref, axis=1)
        rows = []
        for row in gpu["sampled"]:
            rel = np.linalg.norm(row.pop("acc") - ref, axis=1) / rn
            row.update({"median_vs_fp64": float(np.median(rel)),
                        "p99_vs_fp64": float(np.quantile(rel, 0.99)),
                        "meets_1e-3": bool(np.median(rel) <= 1e-3)})
            rows.append(row)
        qual = [r for r in rows if r.get("theta") == args.theta and r["meets_1e-3"]
                and r["kind"] == "tree"]
        best = min(qual, key=lambda r: r["build_ms"] + r["walk_ms"]) if qual else None
        accuracy = {"reference": f"oracle FP64 direct sum of {len(sidx)} seeded bodies (all "
                                 f"{len(pos)} sources)",
                    "rows": rows,
                    "fastest_meeting_1e-3_at_theta": None if best is None else
                    {k: best[k] for k in ("order", "leaf_max", "accum", "build_ms", "walk_ms",
                                          "median_vs_fp64")}}
        cpu["direct_sample"] = {"bodies": len(sidx), "s": t_dir, "cores": omp_threads(),
                                "value_scaled_to_N": len(pos) / (t_dir * len(pos) / len(sidx)),
                                "unit": UNIT}
    return cpu, parity, accuracy


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, as it stands, on the host cores, timed on the
    benchmark's configuration.  Each step is the whole evaluation (tree build of all
    bodies + walk of every body), so ms_per_step is measured, not extrapolated."""
    if rank != 0:
        return 0
    pos, _, m = gen(args, 0)
    for _ in range(args.warmup):
        oracle_eval(pos, m, args, args.n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_eval(pos, m, args, args.n)
    wall = time.perf_counter() - t0
    ms = 1e3 * wall / max(1, args.steps)
    value = args.n / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "precision": "FP64 throughout (the oracle)", "data": "synthetic",
            "config": workload(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
                             "sample": f"per step: FP64 tree build of all {args.n} bodies + walk "
                                       f"of every body (the whole evaluation); {args.steps} steps "
                                       f"in {wall:.1f} s"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def walk_code_hash() -> str:
    """Hash of the walk source without comments and blank space: a change of the code
    (not of its comments) makes the recorded DRAM traffic stale."""
    import re
    src = open(os.path.join(ROOT, "paper_1912_04197_gb300", "csrc", "walk.cu")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", " ", src)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def walk_traffic(order):
    """DRAM bytes per walk launch from the committed ncu summary, if the walk code has
    not changed since it was captured (else None)."""
    path = os.path.join(ROOT, "profiles", "walk_ncu_clumpy1M.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("walk_code_sha256_16") != walk_code_hash():
        return None
    key = f"dram_bytes_per_launch_order{order}"
    return float(vals[key]) if key in vals else None


def config_sweep_leg(args, g, ctx, P, M, accd, p, flush, stream, sample_idx):
    """The headline workload at other opening angles (0.3 / 0.5 / 0.7 / 0.9, with the FP32
    two-sum and the FP64 accumulator), and at theta 0.5 with the monopole (leaf 1, 16) and
    other leaf sizes: build and walk time (CUDA events, L2 flushed), FLOP rate from the
    exact decision counts, error against the GPU direct sum over every body, and the
    accelerations of the sampled bodies for the FP64 direct-sum comparison."""
    import torch
    n = P.shape[0]
    dev = P.device
    acc = torch.empty_like(P)
    cnt = torch.empty((n, 3), dtype=torch.int32, device=dev)
    sidx = None if sample_idx is None else torch.as_tensor(sample_idx, device=dev)
    rows, res = [], {}
    cfgs = [(args.order, args.leaf_max, accum, theta) for accum in (0, 1)
            for theta in (0.3, 0.5, 0.7, 0.9)]
    cfgs += [(0, 16, 0, args.theta), (0, 1, 0, args.theta), (2, 8, 0, args.theta),
             (2, 32, 0, args.theta)]
    for order, leaf, accum, theta in cfgs:
        q = g.params(order=order, leaf_max=leaf, accum=accum, walk_cfg=p.walk_cfg)
        tb = []
        for k in range(5):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.gravity_tree_build(ctx, P, M, q)
            e1.record(stream)
            e1.synchronize()
            tb.append(e0.elapsed_time(e1))
        g.gravity_forces_counted(ctx, theta, args.eps, acc, cnt)
        c = cnt.to(torch.int64).sum(0).cpu().numpy()
        f_node = FLOP_QUAD if order == 2 else FLOP_POINT
        flops = int(c[0]) * f_node + int(c[1]) * FLOP_POINT + int(c[2]) * FLOP_MAC
        ts = []
        for k in range(5):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.gravity_forces(ctx, theta, args.eps, acc)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        g.gravity_sync(ctx)
        t = float(np.median(ts))
        rel = (torch.linalg.norm(acc - accd, dim=1) / torch.linalg.norm(accd, dim=1)).cpu().numpy()
        res[(order, leaf, accum, theta)] = acc.clone()
        rows.append({"kind": "tree", "theta": theta, "order": order, "leaf_max": leaf,
                     "accum": "fp32-two-sum" if accum == 0 else "fp64",
                     "build_ms": float(np.median(tb)), "walk_ms": t,
                     "tflops": flops / (t * 1e-3) / 1e12,
                     "node_terms": int(c[0]), "body_terms": int(c[1]), "opening_tests": int(c[2]),
                     "median_error_vs_gpu_direct": float(np.median(rel)),
                     "p99_error_vs_gpu_direct": float(np.quantile(rel, 0.99)),
                     "acc": None if sidx is None else acc[sidx].cpu().numpy()})
    for r in rows:
        if r["accum"] == "fp32-two-sum" and r["order"] == args.order and r["leaf_max"] == args.leaf_max:
            a32 = res[(r["order"], r["leaf_max"], 0, r["theta"])]
            a64 = res[(r["order"], r["leaf_max"], 1, r["theta"])]
            d = (torch.linalg.norm(a32 - a64, dim=1) / torch.linalg.norm(a64, dim=1)).max()
            r["max_rel_diff_vs_fp64_accum"] = float(d)
    rows.append({"kind": "direct", "theta": None, "order": None, "leaf_max": None, "accum": None,
                 "build_ms": 0.0, "walk_ms": None,
                 "acc": None if sidx is None else accd[sidx].cpu().numpy()})
    return rows


def components_leg(args, g, ctx, P, M, p, flush, stream):
    """Aggregate identification (contact-graph components over the gravity tree) on the
    headline workload: contact = distance <= dmax; the tree of the headline is reused."""
    import torch
    n = P.shape[0]
    g.gravity_tree_build(ctx, P, M, p)
    label = torch.empty(n, dtype=torch.int32, device=P.device)
    counts = torch.empty(2, dtype=torch.int64, device=P.device)
    rows = []
    for dmax in (5e-4, 1e-3, 2e-3):
        g.gravity_components(ctx, label, dmax=dmax, counts=counts)      # warm-up
        ts = []
        for k in range(5):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.gravity_components(ctx, label, dmax=dmax, counts=counts)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        g.gravity_sync(ctx)
        c = counts.cpu().tolist()
        t = float(np.median(ts))
        rows.append({"dmax": dmax, "ms": t, "bodies_per_s": n / (t * 1e-3),
                     "components": int(c[0]), "aggregates": int(c[1])})
    return {"workload": "the headline aggregate; contact = |x_i - x_j| <= dmax; tree reused "
                        "(search + union-find + labels, 4 kernels)", "rows": rows}


def pipelined_leg(args, g, P, M, p, steps=20):
    """Throughput of independent evaluations when two contexts on two streams take turns:
    one snapshot's build and the start of its walk run while the other's walk finishes.
    The second snapshot is the workload drawn with the next seed; the two snapshots' data
    (~0.3 GB with both trees) exceed the L2."""
    import torch
    from paper_1912_04197_gb300 import inputs
    n = P.shape[0]
    pos2, _, _ = inputs.clumpy_plummer(n, seed=args.seed + 1)
    Ps = [P, torch.tensor(pos2, device=P.device)]
    As = [torch.empty_like(P), torch.empty_like(P)]
    streams = [torch.cuda.Stream(P.device), torch.cuda.Stream(P.device)]
    ctxs = []
    for k in range(2):
        with torch.cuda.stream(streams[k]):
            c = g.Context(P.device)
            ctxs.append(c)
            for _ in range(3):                               # warm-up (and task order)
                g.gravity_tree_build(c, Ps[k], M, p)
                g.gravity_forces(c, args.theta, args.eps, As[k])
    torch.cuda.synchronize(P.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(streams[0])
    streams[1].wait_event(e0)
    for k in range(steps):
        j = k % 2
        with torch.cuda.stream(streams[j]):
            g.gravity_tree_build(ctxs[j], Ps[j], M, p)
            g.gravity_forces(ctxs[j], args.theta, args.eps, As[j])
    done = torch.cuda.Event()
    done.record(streams[1])
    streams[0].wait_event(done)
    e1.record(streams[0])
    e1.synchronize()
    for c in ctxs:
        g.gravity_sync(c)
    ms = e0.elapsed_time(e1) / steps
    return {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "how": "two contexts on two streams taking turns over two independent snapshots "
                   "(each step a full build + walk); throughput, not one evaluation's latency"}


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1912_04197_gb300 import gravity as g

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    pos, _, m = gen(args, rank)
    n = len(pos)
    P = torch.tensor(pos, device=dev)
    M = torch.tensor(m, device=dev)
    acc = torch.empty_like(P)
    ctx = g.Context(dev)
    p = g.params(order=args.order, leaf_max=args.leaf_max, accum=args.accum)
    if not args.no_tune:
        from paper_1912_04197_gb300 import autotune
        p.walk_cfg = autotune.tune_walk(ctx, P, M, p, args.theta, args.eps)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream(dev)
    shard_mode = args.shard and world > 1
    if shard_mode:
        # one cloud split between the ranks: the same tree on every rank, a range of the
        # walk per rank, one all-gather of the ranges' accelerations (NCCL)
        from paper_1912_04197_gb300 import shard
        eng, comm = shard.GpuEngine(ctx, p), shard.TorchComm()

    def walk():
        if shard_mode:
            shard.sharded_forces(eng, comm, args.theta, args.eps, acc)
        else:
            g.gravity_forces(ctx, args.theta, args.eps, acc)

    def step():
        g.gravity_tree_build(ctx, P, M, p)
        walk()

    for _ in range(max(args.warmup, 3)):
        step()
    g.gravity_sync(ctx)

    # algorithmic work of one walk launch (exact per-body decision counts)
    cnt = torch.empty((n, 3), dtype=torch.int32, device=dev)
    g.gravity_tree_build(ctx, P, M, p)
    g.gravity_forces_counted(ctx, args.theta, args.eps, acc, cnt)
    g.gravity_sync(ctx)
    if shard_mode:         # this rank's range of the walk only
        first, count = shard.plan(g.gravity_walk_tasks(ctx), world)[rank]
        b0, nb = g.gravity_task_bodies(ctx, first, count)
        perm = g.gravity_debug_export(ctx, g.DBG_PERM, n).astype(np.int64)
        c = cnt.to(torch.int64)[torch.as_tensor(perm[b0:b0 + nb], device=dev)].sum(0).cpu().numpy()
    else:
        c = cnt.to(torch.int64).sum(0).cpu().numpy()
    node_terms, body_terms, tests = int(c[0]), int(c[1]), int(c[2])
    f_node = FLOP_QUAD if args.order == 2 else FLOP_POINT
    walk_flops = node_terms * f_node + body_terms * FLOP_POINT + tests * FLOP_MAC

    props = torch.cuda.get_device_properties(dev)
    gpu_id = str(getattr(props, "uuid", local_rank))
    if gpu_id and not gpu_id.startswith("GPU-") and len(gpu_id) == 36:
        gpu_id = "GPU-" + gpu_id
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches0 = g.gravity_stats(ctx)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(gpu_id)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        e0, e1, e2 = ev[k]
        e0.record(stream)
        g.gravity_tree_build(ctx, P, M, p)
        e1.record(stream)
        walk()
        e2.record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    acc_head = acc.cpu().numpy()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    g.gravity_sync(ctx)
    launches = g.gravity_stats(ctx) - launches0
    t_build = sum(e0.elapsed_time(e1) for e0, e1, _ in ev) / args.steps
    t_walk = sum(e1.elapsed_time(e2) for _, e1, e2 in ev) / args.steps
    t_step = t_build + t_walk
    t_max = max_over_ranks(t_step, world, dev)
    # sharded: one cloud of n bodies over all ranks; else one cloud per rank
    value = whole_job_value(n, 1, t_max) if shard_mode else whole_job_value(n, world, t_max)
    from paper_1912_04197_gb300 import inputs
    sample_idx = inputs.subset(n, args.fp64_sample, seed=17) if args.fp64_sample > 0 else None
    sweep_rows = []

    # error against the direct sum, and the direct-sum throughput on the same GPU
    extra = {}
    if not args.no_direct and not shard_mode:
        accd = torch.empty_like(P)
        g.gravity_direct(ctx, P, M, args.eps, 1.0, accd)       # warm-up
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        g.gravity_direct(ctx, P, M, args.eps, 1.0, accd)
        d1.record(stream)
        torch.cuda.synchronize(dev)
        t_dir = d0.elapsed_time(d1)
        step()
        g.gravity_sync(ctx)
        rel = (torch.linalg.norm(acc - accd, dim=1) / torch.linalg.norm(accd, dim=1)).cpu().numpy()
        med, p99 = float(np.median(rel)), float(np.quantile(rel, 0.99))
        extra["error_vs_direct"] = {"median": med, "p99": p99, "meets_1e-3": med <= 1e-3,
                                    "reference": "GPU direct sum (FP32 pair terms on "
                                                 "block-relative or hi/lo coordinates, within "
                                                 "1e-6 of the FP64 sum per tests)"}
        extra["direct"] = {"ms": t_dir, "value": n / (t_dir * 1e-3), "unit": UNIT,
                           "speedup_of_tree": (n / (t_step * 1e-3)) / (n / (t_dir * 1e-3)),
                           "interactions_per_s": n * (n - 1) / (t_dir * 1e-3),
                           "flops_per_s": FLOP_POINT * n * (n - 1) / (t_dir * 1e-3)}
        if not args.no_sweep:
            sweep_rows = config_sweep_leg(args, g, ctx, P, M, accd, p, flush, stream, sample_idx)

    if not args.no_components and not shard_mode:
        extra["components"] = components_leg(args, g, ctx, P, M, p, flush, stream)
    if not args.no_pipelined and not shard_mode:
        extra["pipelined"] = pipelined_leg(args, g, P, M, p)

    # rooflines: the walk is FP32-ALU bound (no dense contraction, no tensor cores)
    sm_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    peak_clock = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6
    _, probe = g.gravity_probe_fp32(ctx, 20000)
    achieved = walk_flops / (t_walk * 1e-3)
    roof = {"bound": "alu", "kernel": "k_walk", "achieved": achieved / 1e12,
            "peak": peak_clock / 1e12, "unit": "TFLOP/s", "frac": achieved / peak_clock,
            "traffic": walk_traffic(args.order),
            "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 "
                          f"x {sm_mhz:.0f} MHz (median SM clock sampled in the timed region)",
            "fp32_probe_tflops": probe / 1e12, "frac_of_probe": achieved / probe,
            "walk_ms": t_walk, "build_ms": t_build,
            "work_per_launch": {"node_terms": node_terms, "body_terms": body_terms,
                                "opening_tests": tests, "flops": walk_flops,
                                "flop_per_unit": {"node_term": f_node, "body_term": FLOP_POINT,
                                                  "opening_test": FLOP_MAC}}}

    e2e = None
    if not args.no_e2e and shard_mode:
        # host positions and masses in, build + sharded walk + all-gather, host forces out
        ph = torch.tensor(pos).pin_memory()
        mh = torch.tensor(m).pin_memory()
        ah = torch.empty((n, 3), dtype=torch.float64).pin_memory()
        ke = min(args.steps, 10)
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(ke):
            P.copy_(ph, non_blocking=True)
            M.copy_(mh, non_blocking=True)
            step()
            ah.copy_(acc, non_blocking=True)
            torch.cuda.synchronize(dev)
        te = max_over_ranks((time.perf_counter() - t0) / ke, world, dev)
        e2e = {"value": whole_job_value(n, 1, 1e3 * te), "unit": UNIT,
               "h2d_bytes_per_step": int(ph.nbytes + mh.nbytes), "d2h_bytes_per_step": int(ah.nbytes),
               "ms_per_step": 1e3 * te,
               "api": "pinned host copies + gravity_tree_build + shard.sharded_forces per rank"}
    elif not args.no_e2e:
        # K snapshots in their own pinned host buffers: every step copies its positions and
        # masses in and its accelerations out; the batch call overlaps one snapshot's copies
        # with its neighbours' build and walk
        ke = min(args.steps, 10)
        ph = [torch.tensor(pos).pin_memory() for _ in range(ke)]
        mh = [torch.tensor(m).pin_memory() for _ in range(ke)]
        ah = [torch.empty((n, 3), dtype=torch.float64).pin_memory() for _ in range(ke)]
        g.gravity_forces_host_batch(ctx, ph, mh, args.theta, args.eps, p, ah)
        t0 = time.perf_counter()
        g.gravity_forces_host_batch(ctx, ph, mh, args.theta, args.eps, p, ah)
        te = max_over_ranks((time.perf_counter() - t0) / ke, world, dev)
        # one snapshot per call (copy in, build, walk, copy out, wait): latency
        g.gravity_forces_host(ctx, ph[0], mh[0], args.theta, args.eps, p, ah[0])
        t0 = time.perf_counter()
        for k in range(ke):
            g.gravity_forces_host(ctx, ph[k], mh[k], args.theta, args.eps, p, ah[k])
        t1 = max_over_ranks((time.perf_counter() - t0) / ke, world, dev)
        e2e = {"value": whole_job_value(n, world, 1e3 * te), "unit": UNIT,
               "h2d_bytes_per_step": int(ph[0].nbytes + mh[0].nbytes),
               "d2h_bytes_per_step": int(ah[0].nbytes), "ms_per_step": 1e3 * te, "steps": ke,
               "api": "gravity_forces_host_batch (%d snapshots in pinned host buffers; each step's "
                      "copies overlap its neighbours' build and walk, and the context and its "
                      "internal twin take alternate snapshots)" % ke,
               "single_call": {"value": whole_job_value(n, world, 1e3 * t1), "ms_per_step": 1e3 * t1,
                               "api": "gravity_forces_host (copy in, build, walk, copy out, wait)"}}

    ens = None if args.no_ensemble or shard_mode else ensemble_leg(args, g, dev, rank, world)
    grad = None if args.no_grad or shard_mode else gradient_leg(args, g, dev, rank)

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        if sample_idx is not None and not sweep_rows:      # no sweep: the headline alone
            sweep_rows = [{"kind": "tree", "theta": args.theta, "order": args.order,
                           "leaf_max": args.leaf_max, "accum": "fp32-two-sum" if args.accum == 0
                           else "fp64", "build_ms": t_build, "walk_ms": t_walk,
                           "acc": acc_head[sample_idx]}]
        cpu, parity, accuracy = cpu_baseline_leg(pos, m, args, {"acc": acc_head,
                                                                "sample_idx": sample_idx,
                                                                "sampled": sweep_rows})
        extra["parity_vs_oracle"] = parity
        if accuracy is not None:
            extra["config_sweep"] = accuracy
    elif sweep_rows:
        for r in sweep_rows:
            r.pop("acc", None)
        extra["config_sweep"] = {"reference": "GPU direct sum only (no oracle leg)",
                                 "rows": sweep_rows}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max, "higher_is_better": True,
            "scaling": "strong" if shard_mode else "weak", "vs_baseline": None, "dtype": "f32",
            "dtype_note": "FP32 pair terms and opening tests on hi/lo coordinates; FP64 mass and "
                          "COM, double-float FP32 second moments, FP64 decisions in the guard "
                          "band, FP64 outputs",
            "precision": {"accum": "fp32-two-sum" if args.accum == 0 else "fp64"},
            "data": "synthetic", "config": workload(args), "phases_ms": {"build": t_build, "walk": t_walk},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps, "clocks": clk,
            "timed_wall_s": wall, "launch": {"walk_cfg": int(p.walk_cfg)}}
    if shard_mode:
        line["sharding"] = {"mode": "one cloud over all ranks: replicated build, walk task range "
                                    "per rank, one all-gather of accelerations per evaluation",
                            "ranks": world}
    if ens is not None:
        line["ensemble"] = ens
    if grad is not None:
        line["gradient"] = grad
    line.update(extra)
    print(json.dumps(line), flush=True)
    return 0


def ensemble_leg(args, g, dev, rank, world=1):
    """Batched ensemble: 256 independent spinning clouds (N_k log-uniform in
    [1024, 65536]), one build + one walk launch per step, KDK leapfrog steps
    replayed as a CUDA graph on a side stream, autotuned walk shape.  With several ranks
    the same 256 clouds are partitioned between them by cost (N_k log N_k, no exchange)
    and the whole job's rate is reported over the slowest rank."""
    import torch
    from paper_1912_04197_gb300 import autotune, inputs, shard
    off, pos, vel, m = inputs.ensemble(nclouds=256, seed=args.seed + 100)
    n_total = len(pos)
    if world > 1:
        k0, k1 = shard.partition_clouds(np.diff(off), world)[rank]
        b0, b1 = int(off[k0]), int(off[k1])
        off, pos, vel, m = off[k0:k1 + 1] - off[k0], pos[b0:b1], vel[b0:b1], m[b0:b1]
    n = len(pos)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        ctx = g.Context(dev)
        g.gravity_set_clouds(ctx, off)
        P = torch.tensor(pos, device=dev)
        V = torch.tensor(vel, device=dev)
        M = torch.tensor(m, device=dev)
        A = torch.empty_like(P)
        p = g.params(order=args.order, leaf_max=args.leaf_max)
        if not args.no_tune:
            p.walk_cfg = autotune.tune_walk(ctx, P, M, p, args.theta, args.eps, clouds=256)
        g.gravity_tree_build(ctx, P, M, p)
        g.gravity_forces(ctx, args.theta, args.eps, A)
        g.leapfrog_step(ctx, P, V, M, A, 1e-3, 3, args.theta, args.eps, p)   # warm-up + capture
        k0 = g.gravity_stats(ctx)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.leapfrog_step(ctx, P, V, M, A, 1e-3, args.ensemble_steps, args.theta, args.eps, p)
        e1.record(stream)
        e1.synchronize()
        g.gravity_sync(ctx)
        ms = e0.elapsed_time(e1)
        kernels = g.gravity_stats(ctx) - k0
    steps = args.ensemble_steps
    ms = max_over_ranks(ms, world, dev)
    return {"workload": f"256 independent clouds, {n_total} bodies (N_k log-uniform in [1024, "
                        f"65536]), uniform spheres with random spin, eps={args.eps}, "
                        f"theta={args.theta}, order {args.order}, leaf {args.leaf_max}, dt=1e-3"
                        + (f"; clouds partitioned over {world} ranks by N_k log N_k" if world > 1
                           else ""),
            "steps": steps, "ms_per_step": ms / steps, "value": n_total * steps / (ms * 1e-3),
            "unit": "body-forces/s (leapfrog steps, one force evaluation each)",
            "graph": True, "kernels_per_step": kernels / steps, "walk_cfg": int(p.walk_cfg)}


def gradient_leg(args, g, dev, rank):
    """Differentiation: N = 65536 bodies uniform in the unit sphere at rest, m = 1/N,
    eps = 1e-3, 200 KDK steps of dt = 1e-3 at theta = 0.5 (monopole, leaf 1), checkpoints
    every 20 steps; loss = axis-ratio deviation (target 1 : 0.8 : 0.6) of the final
    second-moment tensor; gradient with respect to the initial positions and velocities.
    Reports forward / backward times, the vector-Jacobian-product kernel against the FP32
    roofline, the gradient against central differences of the same GPU forward (along the
    gradient, along random directions, and on seeded single coordinates) and against the
    gradient of the exact sum (theta = 0)."""
    import torch
    from paper_1912_04197_gb300 import inputs
    from paper_1912_04197_gb300.adjoint import leapfrog
    from paper_1912_04197_gb300.loss import axis_ratio_loss
    n, nsteps, dt, eps, every = 65536, 200, 1e-3, 1e-3, 20
    theta = args.theta
    pos, vel, m = inputs.uniform_sphere(n, seed=args.seed + 200 + rank)
    stream = torch.cuda.current_stream(dev)
    ctx = g.Context(dev)
    M = torch.tensor(m, device=dev)
    p = g.params(order=0, leaf_max=1)

    def run(th):
        x0 = torch.tensor(pos, device=dev, requires_grad=True)
        v0 = torch.tensor(vel, device=dev, requires_grad=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        x, _ = leapfrog(x0, v0, M, dt, nsteps, theta=th, eps=eps, leaf_max=1,
                        checkpoint_every=every, ctx=ctx)
        L = axis_ratio_loss(x, M)
        ev[1].record(stream)
        gx, gv = torch.autograd.grad(L, (x0, v0))
        ev[2].record(stream)
        torch.cuda.synchronize(dev)
        g.gravity_sync(ctx)
        return (float(L.detach()), gx.cpu().numpy(), gv.cpu().numpy(),
                ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]))

    run(theta)                                                        # warm-up
    k0 = g.gravity_stats(ctx)
    L, gx, gv, t_fwd, t_bwd = run(theta)
    kernels = g.gravity_stats(ctx) - k0

    def loss_at(x, v, th=theta):
        P = torch.tensor(x, device=dev)
        V = torch.tensor(v, device=dev)
        A = torch.empty_like(P)
        g.gravity_tree_build(ctx, P, M, p)
        g.gravity_forces(ctx, th, eps, A)
        g.leapfrog_step(ctx, P, V, M, A, dt, nsteps, th, eps, p)
        return float(axis_ratio_loss(P, M))

    rng = np.random.default_rng(args.seed + 201)
    unit = [(f"random{k}", rng.standard_normal(pos.shape), rng.standard_normal(pos.shape))
            for k in range(4)]
    # random affine fields (x -> A x, v -> B x): smooth directions that move neighbours
    # together, so close pairs do not dominate the differences
    affine = [(f"affine{k}", pos @ rng.standard_normal((3, 3)).T, pos @ rng.standard_normal((3, 3)).T)
              for k in range(4)]

    def fd_check(th, gx_, gv_, dirs, hs, richardson=False):
        """Central differences of the loss of the same GPU forward along each direction,
        for each step h; with richardson, (4 D(h/2) - D(h)) / 3 cancels the h^2 term."""
        gn = np.sqrt((gx_ * gx_).sum() + (gv_ * gv_).sum())
        out = []
        for name, dx, dv in dirs:
            def cd(hh):
                return (loss_at(pos + hh * dx, vel + hh * dv, th) -
                        loss_at(pos - hh * dx, vel - hh * dv, th)) / (2 * hh)
            ad = float((gx_ * dx).sum() + (gv_ * dv).sum())
            cs = gn * float(np.sqrt((dx * dx).sum() + (dv * dv).sum()))
            for h in hs:
                fd = cd(h)
                if richardson:
                    fd = (4.0 * cd(0.5 * h) - fd) / 3.0
                out.append({"direction": name, "theta": th, "h": h, "richardson": richardson,
                            "fd": fd, "adjoint": ad,
                            "rel_err": abs(fd - ad) / abs(ad) if ad else None,
                            "err_over_norm_bound": abs(fd - ad) / cs})
        return out

    # The loss depends on the eigenvalues of S, which are nearly degenerate for a sphere
    # (gaps ~ N^-1/2): an affine step moves them by O(h), so central differences converge
    # to the derivative only once h is well below the gaps (O(h^2) error, seen below).
    gmax = max(np.abs(gx).max(), np.abs(gv).max())
    fd_dirs = fd_check(theta, gx, gv, [("gradient", gx / gmax, gv / gmax)], (1e-3,))
    fd_dirs += fd_check(theta, gx, gv, affine, (1e-3, 1e-4, 1e-5))
    fd_dirs += fd_check(theta, gx, gv, unit, (4e-3,), richardson=True)
    coords = rng.choice(3 * n, size=32, replace=False)
    coord_rel, h_c = [], 1e-3
    for c in coords:
        i, a = divmod(int(c), 3)
        dx = np.zeros_like(pos)
        dx[i, a] = 1.0
        fd = (loss_at(pos + h_c * dx, vel) - loss_at(pos - h_c * dx, vel)) / (2 * h_c)
        coord_rel.append(abs(fd - gx[i, a]) / (abs(gx[i, a]) + 1e-300))

    # gradient of the exact sum: the same pipeline at theta = 0 (no opening decisions,
    # so its differences carry FP32 rounding only)
    _, gx0, gv0, t_fwd0, t_bwd0 = run(0.0)
    d_exact = {"rel_l2_x": float(np.linalg.norm(gx - gx0) / np.linalg.norm(gx0)),
               "rel_l2_v": float(np.linalg.norm(gv - gv0) / np.linalg.norm(gv0)),
               "fwd_ms_theta0": t_fwd0, "bwd_ms_theta0": t_bwd0}
    fd_dirs += fd_check(0.0, gx0, gv0, affine[:2], (1e-3, 1e-4, 1e-5))
    fd_dirs += fd_check(0.0, gx0, gv0, unit[:2], (1e-3, 1e-4))

    # the vector-Jacobian-product kernel alone, on the tree of the initial positions
    P0 = torch.tensor(pos, device=dev)
    props = torch.cuda.get_device_properties(dev)
    fp32_peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * 2070e6

    def time_vjp(P_, M_, p_, th, ep):
        """Average time of one vector-Jacobian product on the tree of P_ (and its FLOP)."""
        lam_ = torch.tensor(rng.standard_normal(tuple(P_.shape)), device=dev)
        out_ = torch.empty_like(P_)
        cnt_ = torch.empty((P_.shape[0], 3), dtype=torch.int32, device=dev)
        g.gravity_tree_build(ctx, P_, M_, p_)
        g.gravity_forces_counted(ctx, th, ep, out_, cnt_)
        c_ = cnt_.to(torch.int64).sum(0).cpu().numpy()
        for _ in range(3):
            g.gravity_forces_vjp(ctx, th, ep, lam_, out_)
        reps = 20
        e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0_.record(stream)
        for _ in range(reps):
            g.gravity_forces_vjp(ctx, th, ep, lam_, out_)
        e1_.record(stream)
        torch.cuda.synchronize(dev)
        g.gravity_sync(ctx)
        ms = e0_.elapsed_time(e1_) / reps
        fl = int(c_[0] + c_[1]) * FLOP_VJP + int(c_[2]) * FLOP_MAC
        return {"ms": ms, "terms": int(c_[0] + c_[1]), "opening_tests": int(c_[2]),
                "flop_per_term": FLOP_VJP, "achieved_tflops": fl / (ms * 1e-3) / 1e12,
                "frac_of_fp32_peak_at_max_clock": fl / (ms * 1e-3) / fp32_peak,
                "includes": "VJP walk + leaf-chain finishing pass + 2 memsets"}

    vjp = time_vjp(P0, M, p, theta, eps)
    # the same kernel on the headline workload (monopole: the product covers order 0)
    hpos, _, hm = inputs.clumpy_plummer(1_048_576, seed=args.seed)
    vjp_1m = time_vjp(torch.tensor(hpos, device=dev), torch.tensor(hm, device=dev),
                      g.params(order=0, leaf_max=16), theta, 1e-3)
    vjp_1m["workload"] = "clumpy aggregate, 1,048,576 bodies, theta 0.5, monopole, leaf 16"
    return {"workload": f"N={n} uniform sphere at rest, m=1/N, eps={eps}, {nsteps} KDK steps "
                        f"dt={dt}, theta={theta} monopole, leaf 1, checkpoints every {every}; "
                        "loss (rho2-0.8)^2+(rho3-0.6)^2 of the final second-moment tensor",
            "loss": L, "forward_ms": t_fwd, "backward_ms": t_bwd,
            "backward_over_forward": t_bwd / t_fwd, "kernels": kernels,
            "vs_finite_differences": {"directions": fd_dirs,
                                      "coordinates": {"count": 32, "h": h_c,
                                                      "median_rel_err": float(np.median(coord_rel)),
                                                      "max_rel_err": float(np.max(coord_rel))}},
            "vs_exact_sum_gradient": d_exact,
            "vjp_kernel": vjp, "vjp_kernel_1M": vjp_1m}


def experiment_accuracy(args):
    """Sec. 3.2 "Accuracy": N = 1000 bodies at rest, uniform in a cube, gravity only,
    integrated through a full contraction and re-expansion; at every step the largest
    (and the median) relative position error e_i = |r_i,BH - r_i,N2| / |r_i,N2| (Eq. e_i)
    of the tree runs (theta = 0.1, 0.25, 0.5, 0.75) against the exact sum (the walk at
    theta = 0), with the paper's semi-implicit Euler.  The paper gives no softening: with
    a small one the collapse is violent (close encounters make single trajectories
    chaotic, and the largest error grows without bound); with a softening near the mean
    spacing it pulsates smoothly, as the paper describes.  e_i divides by |r_i|, so it
    depends on the origin: here a corner of the cube, as for positions drawn in [0, L]^3."""
    import torch
    from paper_1912_04197_gb300 import gravity as g, inputs
    n, dt, nsteps = 1000, 1e-3, 3600
    pos, vel, m = inputs.uniform_cube(n, seed=args.seed + 300)
    pos = pos + 1.0        # the cube [0, 2]^3: positions (and e_i) relative to a corner
    dev = torch.device("cuda", 0)
    ctx = g.Context(dev)
    M = torch.tensor(m, device=dev)
    out = {"experiment": "accuracy", "n": n, "dt": dt, "steps": nsteps, "scheme": "semi-implicit Euler",
           "workload": "1000 equal masses (1/N) uniform in the cube [0, 2]^3 at rest, G = 1",
           "every": 50, "runs": {}}

    def run(theta, eps):
        P = torch.tensor(pos, device=dev)
        V = torch.tensor(vel, device=dev)
        A = torch.empty_like(P)
        p = g.params(order=0, leaf_max=1, scheme=1)
        g.gravity_tree_build(ctx, P, M, p)
        g.gravity_forces(ctx, theta, eps, A)
        traj = [P.cpu().numpy().copy()]
        for _ in range(nsteps):
            g.leapfrog_step(ctx, P, V, M, A, dt, 1, theta, eps, p)
            traj.append(P.cpu().numpy().copy())
        g.gravity_sync(ctx)
        return np.stack(traj)

    for eps in (0.05, 0.2):
        ref = run(0.0, eps)
        rad = np.linalg.norm(ref - ref.mean(axis=1, keepdims=True), axis=2).mean(axis=1)
        res = {"mean_radius": rad[::50].tolist(), "t_min_radius": float(np.argmin(rad) * dt),
               "final_over_initial_radius": float(rad[-1] / rad[0]), "theta": {}}
        for theta in (0.1, 0.25, 0.5, 0.75):
            tr = run(theta, eps)
            e = 100.0 * np.linalg.norm(tr - ref, axis=2) / np.linalg.norm(ref, axis=2)
            emax, emed = e.max(axis=1), np.median(e, axis=1)
            res["theta"][str(theta)] = {"max_error_pct": emax[::50].tolist(),
                                        "median_error_pct": emed[::50].tolist(),
                                        "peak_max_pct": float(emax.max()),
                                        "t_peak": float(np.argmax(emax) * dt),
                                        "max_pct_at_min_radius": float(emax[np.argmin(rad)]),
                                        "peak_median_pct": float(emed.max())}
        out["runs"][f"eps={eps}"] = res
    print(json.dumps(out), flush=True)
    return 0


def experiment_sweep(args):
    """Sec. 3.2 "Computational time": time of one integration step against N (bodies at
    rest, uniform in a cube), for the tree (theta = 0.1, 0.25, 0.5, 0.75; monopole, leaf
    1 as in the paper) and the direct sum; CUDA events over steps replayed as a graph."""
    import torch
    from paper_1912_04197_gb300 import gravity as g, inputs
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    rows = []
    sizes = [10, 30, 100, 300, 1000, 3000, 10_000, 30_000, 100_000, 300_000, 1_000_000,
             3_000_000, 10_000_000]
    if args.sweep_sizes:
        sizes = [int(float(v)) for v in args.sweep_sizes.split(",")]
    thetas = [float(v) for v in args.sweep_thetas.split(",")]
    with torch.cuda.stream(stream):
        ctx = g.Context(dev)
        for n in sizes:
            pos, vel, m = inputs.uniform_cube(n, seed=args.seed + 400)
            P0 = torch.tensor(pos, device=dev)
            M = torch.tensor(m, device=dev)
            row = {"n": n}
            steps = args.sweep_steps if n <= 1_000_000 else min(args.sweep_steps, 10)
            for theta in thetas:
                P, V = P0.clone(), torch.zeros_like(P0)
                A = torch.empty_like(P)
                p = g.params(order=0, leaf_max=1)
                g.gravity_tree_build(ctx, P, M, p)
                g.gravity_forces(ctx, theta, 1e-3, A)
                g.leapfrog_step(ctx, P, V, M, A, 1e-6, 3, theta, 1e-3, p)     # capture
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.leapfrog_step(ctx, P, V, M, A, 1e-6, steps, theta, 1e-3, p)
                e1.record(stream)
                e1.synchronize()
                row[f"tree_theta{theta}_ms"] = e0.elapsed_time(e1) / steps
            if n <= 300_000:
                A = torch.empty_like(P0)
                g.gravity_direct(ctx, P0, M, 1e-3, 1.0, A)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 20 if n <= 30_000 else 3
                e0.record(stream)
                for _ in range(reps):
                    g.gravity_direct(ctx, P0, M, 1e-3, 1.0, A)
                e1.record(stream)
                e1.synchronize()
                row["direct_ms"] = e0.elapsed_time(e1) / reps
            g.gravity_sync(ctx)
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    print(json.dumps({"experiment": "sweep", "unit": "ms per step",
                      "workload": "N equal masses uniform in the cube [-1, 1]^3 at rest, eps 1e-3; "
                                  "tree step = kick-drift + build + walk with fused kick (graph "
                                  "replay); direct = one direct-sum evaluation",
                      "rows": rows}), flush=True)
    return 0


def experiment_vjp(args):
    """The vector-Jacobian product alone on the headline aggregate's tree (monopole, leaf 16):
    a few warm-up products, then --steps timed ones (CUDA events); the launch to profile."""
    import torch
    from paper_1912_04197_gb300 import gravity as g
    dev = torch.device("cuda", 0)
    pos, _, m = gen(args, 0)
    P = torch.tensor(pos, device=dev)
    M = torch.tensor(m, device=dev)
    lam = torch.tensor(np.random.default_rng(args.seed + 7).standard_normal(pos.shape), device=dev)
    out = torch.empty_like(P)
    ctx = g.Context(dev)
    g.gravity_tree_build(ctx, P, M, g.params(order=0, leaf_max=16))
    for _ in range(max(1, args.warmup)):
        g.gravity_forces_vjp(ctx, args.theta, args.eps, lam, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        g.gravity_forces_vjp(ctx, args.theta, args.eps, lam, out)
    e1.record()
    torch.cuda.synchronize(dev)
    g.gravity_sync(ctx)
    print(json.dumps({"experiment": "vjp", "n": len(pos), "theta": args.theta, "eps": args.eps,
                      "ms_per_product": e0.elapsed_time(e1) / args.steps,
                      "workload": "clumpy aggregate, monopole, leaf 16, one tree"}), flush=True)
    return 0


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.experiment == "accuracy":
        return experiment_accuracy(args)
    if args.experiment == "sweep":
        return experiment_sweep(args)
    if args.experiment == "vjp":
        return experiment_vjp(args)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
