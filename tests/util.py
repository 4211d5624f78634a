"""Helpers shared by the tests: canonical tree serialisation and error metrics."""
import numpy as np

LEVELS = 21


def preorder_from_topo(topo, depth, sorted_keys):
    """DFS preorder list of (depth, prefix, begin, end, n_child) from the GPU node
    arrays (children contiguous at topo[:,0] .. +topo[:,1], root = node 0)."""
    out = []
    stack = [0]
    while stack:
        k = stack.pop()
        fc, nc, b, e = (int(v) for v in topo[k])
        d = int(depth[k])
        prefix = 0 if d == 0 else int(sorted_keys[b]) >> (3 * (LEVELS - d))
        out.append((d, prefix, b, e, nc if fc >= 0 else 0))
        if fc >= 0:
            stack.extend(range(fc + nc - 1, fc - 1, -1))
    return out


def preorder_from_oracle(nodes):
    return [(int(nodes["depth"][k]), int(nodes["prefix"][k]), int(nodes["begin"][k]),
             int(nodes["end"][k]), int(nodes["n_child"][k])) for k in range(len(nodes["depth"]))]


def oracle_node_order(topo):
    """GPU node ids in DFS preorder (to align per-node arrays with the oracle's)."""
    order = []
    stack = [0]
    while stack:
        k = stack.pop()
        order.append(k)
        fc, nc = int(topo[k][0]), int(topo[k][1])
        if fc >= 0:
            stack.extend(range(fc + nc - 1, fc - 1, -1))
    return np.array(order, dtype=np.int64)


def force_errors(a, ref, absum):
    """Per-body errors of accelerations `a` against `ref`:
    rel   = |a - ref| / max(|ref|, 1e-3 rms|ref|)
    scale = |a - ref| / sum_k |term_k|  (the natural scale of a sum's rounding)."""
    d = np.linalg.norm(np.asarray(a) - np.asarray(ref), axis=1)
    r = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(r * r)) if len(r) else 0.0
    rel = d / np.maximum(np.maximum(r, floor), 1e-300)
    scale = d / np.maximum(absum, 1e-300)
    return rel, scale


# Parity records of this session (label -> figures); conftest writes them to the file named
# by the environment variable PARITY_LOG at the end of the session, if it is set.
PARITY_RECORDS = {}


def check_parity(a, ref, absum, label, rel_tol=1e-5, scale_tol=1e-6):
    """Per-body parity of accelerations `a` against the oracle's `ref`, for EVERY body given.

    rel   = |a - ref| / max(|ref|, 1e-3 rms|ref|)      (the stated relative bound, rel_tol)
    scale = |a - ref| / sum_k |t_k|                     (the rounding scale of a sum of terms)
    kappa = sum_k |t_k| / max(|ref|, 1e-3 rms|ref|)     (cancellation of the body's terms)

    Rule, body by body: scale <= scale_tol, and rel <= rel_tol unless kappa > rel_tol /
    scale_tol (a force cancelled that far below its terms cannot carry rel_tol with FP32
    terms, each of which rounds at a few 2^-24 of itself: there the scale bound is the
    bound).  The figures (max rel, how many bodies exceed rel_tol, their largest and
    smallest kappa, max scale) are recorded under `label` and returned."""
    a = np.asarray(a)
    ref = np.asarray(ref)
    absum = np.asarray(absum)
    rel, scale = force_errors(a, ref, absum)
    r = np.linalg.norm(ref, axis=1)
    floor = 1e-3 * np.sqrt(np.mean(r * r)) if len(r) else 0.0
    kappa = absum / np.maximum(np.maximum(r, floor), 1e-300)
    over = rel > rel_tol
    k_cut = rel_tol / scale_tol
    rec = {"bodies": int(len(rel)), "rel_tol": rel_tol, "scale_tol": scale_tol,
           "max_rel": float(rel.max()) if len(rel) else 0.0,
           "over_rel_tol": int(over.sum()),
           "kappa_of_over_min": float(kappa[over].min()) if over.any() else None,
           "kappa_of_over_max": float(kappa[over].max()) if over.any() else None,
           "max_scale": float(scale.max()) if len(scale) else 0.0,
           "median_rel": float(np.median(rel)) if len(rel) else 0.0}
    PARITY_RECORDS[label] = rec
    assert rec["max_scale"] <= scale_tol, (label, rec, int(np.argmax(scale)))
    bad = over & (kappa <= k_cut)
    assert not bad.any(), (label, rec, np.flatnonzero(bad)[:10])
    return rec
