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
