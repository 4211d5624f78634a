"""The allocation-free direct sum, gravity_direct_noalloc, called through the C ABI.

It exists for callers that cannot call cudaMalloc (an application that owns all
device memory, or a latency-critical loop that cannot take cudaMalloc's implicit
synchronisation); its staging lives in a fixed 2 MiB device array.  This file is
collected last on purpose, so a run that stops at the first failure has already
run every other test; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1912_04197_gb300 import inputs
from util import force_errors

pytestmark = pytest.mark.gpu

SCALE_TOL = 1e-6        # the direct-sum tolerance of the other GPU tests (|err| / sum |terms|)
MAX_BODIES = 65536


def _call(lib, P, M, eps, G, A):
    return lib.gravity_direct_noalloc(P.shape[0], ctypes.c_void_p(P.data_ptr()),
                                      ctypes.c_void_p(M.data_ptr()), ctypes.c_double(eps),
                                      ctypes.c_double(G), ctypes.c_void_p(A.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_direct_twice_in_a_row(gpu):
    lib = gpu._lib                                    # the C ABI itself
    ctx = gpu.Context(0)
    # a large call then a smaller one: the second must not see the first's leftovers
    for n, eps, G, seed in ((MAX_BODIES, 1e-3, 1.0, 11), (5003, 5e-3, 2.0, 12)):
        pos, _, m = inputs.uniform_sphere(n, seed=seed)
        P = torch.tensor(pos, device="cuda")
        M = torch.tensor(m, device="cuda")
        A = torch.full_like(P, float("nan"))
        assert _call(lib, P, M, eps, G, A) == gpu.GRAVITY_OK
        ref = torch.empty_like(P)
        gpu.gravity_direct(ctx, P, M, eps, G, ref)
        torch.cuda.synchronize()
        a, r = A.cpu().numpy(), ref.cpu().numpy()
        sub = inputs.subset(n, 512, seed=seed)
        _, absum = oracle.direct(pos, m, eps, G, targets=sub)
        _, scale = force_errors(a[sub], r[sub], absum)
        assert np.all(np.isfinite(a))
        assert scale.max() <= SCALE_TOL               # the two direct sums agree to rounding
        ref_o, _ = oracle.direct(pos, m, eps, G, targets=sub)
        _, scale_o = force_errors(a[sub], ref_o, absum)
        assert scale_o.max() <= SCALE_TOL             # and the allocation-free one is exact


def test_noalloc_rejects_oversize_and_bad_args(gpu):
    lib = gpu._lib
    P = torch.zeros((MAX_BODIES + 1, 3), dtype=torch.float64, device="cuda")
    M = torch.ones(MAX_BODIES + 1, dtype=torch.float64, device="cuda")
    A = torch.zeros_like(P)
    assert _call(lib, P, M, 1e-3, 1.0, A) == gpu.GRAVITY_E_ARG
    assert _call(lib, P[:10], M[:10], -1.0, 1.0, A[:10]) == gpu.GRAVITY_E_ARG
    assert _call(lib, P[:0], M[:0], 1e-3, 1.0, A[:0]) == gpu.GRAVITY_OK
    torch.cuda.synchronize()
