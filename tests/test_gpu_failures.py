"""Failure detection without a GPU fault: conditions made on the host (an allocator that
refuses, a walk stack capped below what the walk needs) must come back as error codes,
leave nothing half-made, and leave the context usable."""
import numpy as np
import pytest
import torch

from paper_1912_04197_gb300 import inputs

pytestmark = pytest.mark.gpu


class Counting:
    """Device allocator over PyTorch's caching allocator that counts live buffers and
    can refuse every allocation after the first `budget`."""

    def __init__(self, budget=None):
        self.live, self.made, self.budget = {}, 0, budget

    def alloc(self, nbytes):
        if self.budget is not None and self.made >= self.budget:
            return 0
        self.made += 1
        ptr = torch.cuda.caching_allocator_alloc(nbytes, 0, torch.cuda.current_stream(0))
        self.live[ptr] = nbytes
        return ptr

    def release(self, ptr):
        assert ptr in self.live, "freed a pointer this allocator did not make"
        del self.live[ptr]
        torch.cuda.caching_allocator_delete(ptr)


def _forces(g, ctx, pos, m, **kw):
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    A = torch.empty_like(P)
    g.gravity_tree_build(ctx, P, M, g.params(**kw))
    g.gravity_forces(ctx, 0.5, 1e-3, A)
    g.gravity_sync(ctx)
    return A.cpu().numpy()


def test_stack_cap_reports_internal_error(gpu):
    pos, _, m = inputs.clumpy_plummer(20_000, seed=3, nclusters=4)
    ctx = gpu.Context(0)
    ref = _forces(gpu, ctx, pos, m, leaf_max=8)
    gpu.gravity_debug_set(ctx, gpu.GRAVITY_DBGSET_STACK_CAP, 4)
    with pytest.raises(gpu.GravityError) as e:
        _forces(gpu, ctx, pos, m, leaf_max=8)
    assert e.value.code == gpu.GRAVITY_E_INTERNAL
    gpu.gravity_debug_set(ctx, gpu.GRAVITY_DBGSET_STACK_CAP, 0)
    assert np.array_equal(_forces(gpu, ctx, pos, m, leaf_max=8), ref)
    for bad in (-1, 1 << 20):
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_debug_set(ctx, gpu.GRAVITY_DBGSET_STACK_CAP, bad)
        assert e.value.code == gpu.GRAVITY_E_ARG


def test_caller_allocator_gives_identical_results_and_frees_everything(gpu):
    pos, vel, m = inputs.rubble_pile(30_000, seed=4)
    ref_ctx = gpu.Context(0)
    ref = _forces(gpu, ref_ctx, pos, m, order=2, leaf_max=16)
    al = Counting()
    ctx = gpu.Context(0)
    gpu.gravity_set_allocator(ctx, al.alloc, al.release)
    base = len(al.live)
    assert base > 0
    assert np.array_equal(_forces(gpu, ctx, pos, m, order=2, leaf_max=16), ref)
    # the other entry points allocate their scratch through it too
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    A = torch.empty_like(P)
    gpu.gravity_direct(ctx, P, M, 1e-3, 1.0, A)
    gpu.gravity_tree_build(ctx, P, M, gpu.params(order=0, leaf_max=8))
    gpu.gravity_forces_vjp(ctx, 0.5, 1e-3, torch.randn_like(P), A)
    out = torch.empty(7, dtype=torch.float64, device="cuda")
    gpu.gravity_diagnostics(ctx, P, torch.tensor(vel, device="cuda"), M, 1e-3, 1.0, out)
    gpu.gravity_sync(ctx)
    assert len(al.live) > base
    ctx.close()
    assert al.live == {}                       # every buffer went back to the allocator


def test_refused_allocation_is_nomem_and_context_stays_usable(gpu):
    pos, _, m = inputs.uniform_sphere(50_000, seed=5)
    ctx = gpu.Context(0)
    probe = Counting()
    gpu.gravity_set_allocator(ctx, probe.alloc, probe.release)
    base = probe.made
    al = Counting(budget=base + 5)             # the fixed buffers, then 5 tree arrays
    gpu.gravity_set_allocator(ctx, al.alloc, al.release)
    assert probe.live == {}                    # switching released the old allocator's buffers
    with pytest.raises(gpu.GravityError) as e:
        _forces(gpu, ctx, pos, m)
    assert e.value.code == gpu.GRAVITY_E_NOMEM
    assert len(al.live) == base                # the partial tree was released
    gpu.gravity_set_allocator(ctx)             # back to cudaMalloc / cudaFree
    assert al.live == {}
    ref = _forces(gpu, gpu.Context(0), pos, m)
    assert np.array_equal(_forces(gpu, ctx, pos, m), ref)


def test_allocator_refusing_the_fixed_buffers_keeps_the_previous_one(gpu):
    ctx = gpu.Context(0)
    never = Counting(budget=0)
    with pytest.raises(gpu.GravityError) as e:
        gpu.gravity_set_allocator(ctx, never.alloc, never.release)
    assert e.value.code == gpu.GRAVITY_E_NOMEM
    pos, _, m = inputs.uniform_sphere(3000, seed=6)
    assert np.isfinite(_forces(gpu, ctx, pos, m)).all()


def test_torch_pool_allocator_helper(gpu):
    # the binding's helper hands the context's memory to PyTorch's caching allocator
    pos, _, m = inputs.clumpy_plummer(40_000, seed=7, nclusters=4)
    ref = _forces(gpu, gpu.Context(0), pos, m, order=2, leaf_max=16)
    ctx = gpu.Context(0)
    before = torch.cuda.memory_allocated(0)
    gpu.use_torch_allocator(ctx)
    got = _forces(gpu, ctx, pos, m, order=2, leaf_max=16)
    held = torch.cuda.memory_allocated(0) - before
    assert np.array_equal(got, ref)
    assert held > 0                            # the tree lives in the torch pool now
    ctx.close()
    assert torch.cuda.memory_allocated(0) - before <= 0
    with pytest.raises(gpu.GravityError) as e:
        gpu.gravity_debug_set(gpu.Context(0), 99, 0)
    assert e.value.code == gpu.GRAVITY_E_ARG


def test_sort_lookback_wait_runs_out_and_context_recovers(gpu):
    # the first tile of every sort pass withholds its digit counts (a flag nothing sets),
    # so the next tile's bounded look-back wait runs out: GRAVITY_E_TIMEOUT, no fault, every
    # permutation entry still a valid index; the next build on the same context is
    # bit-identical to a fresh context's
    pos, _, m = inputs.clumpy_plummer(100_000, seed=8, nclusters=4)
    ref = _forces(gpu, gpu.Context(0), pos, m, order=2, leaf_max=16)
    ctx = gpu.Context(0)
    gpu.gravity_debug_set(ctx, gpu.GRAVITY_DBGSET_SORT_STALL, 64)
    with pytest.raises(gpu.GravityError) as e:
        _forces(gpu, ctx, pos, m, order=2, leaf_max=16)
    assert e.value.code == gpu.GRAVITY_E_TIMEOUT
    perm = gpu.gravity_debug_export(ctx, gpu.DBG_PERM, len(pos))
    assert perm.min() >= 0 and perm.max() < len(pos)
    gpu.gravity_debug_set(ctx, gpu.GRAVITY_DBGSET_SORT_STALL, 0)
    assert np.array_equal(_forces(gpu, ctx, pos, m, order=2, leaf_max=16), ref)
    for bad in (-1, (1 << 22) + 1):
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_debug_set(ctx, gpu.GRAVITY_DBGSET_SORT_STALL, bad)
        assert e.value.code == gpu.GRAVITY_E_ARG


def test_moments_level_wait_runs_out_and_context_recovers(gpu):
    # the deepest internal depth is not counted, so the next depth's bounded wait in the
    # one-launch pass over the internal nodes runs out: GRAVITY_E_TIMEOUT, no fault; the
    # next build on the same context is bit-identical to a fresh context's
    pos, _, m = inputs.clumpy_plummer(100_000, seed=9, nclusters=4)
    ref = _forces(gpu, gpu.Context(0), pos, m, order=2, leaf_max=16)
    ctx = gpu.Context(0)
    gpu.gravity_debug_set(ctx, gpu.GRAVITY_DBGSET_MOMENTS_STALL, 16)
    with pytest.raises(gpu.GravityError) as e:
        _forces(gpu, ctx, pos, m, order=2, leaf_max=16)
    assert e.value.code == gpu.GRAVITY_E_TIMEOUT
    gpu.gravity_debug_set(ctx, gpu.GRAVITY_DBGSET_MOMENTS_STALL, 0)
    assert np.array_equal(_forces(gpu, ctx, pos, m, order=2, leaf_max=16), ref)
    for bad in (-1, (1 << 18) + 1):
        with pytest.raises(gpu.GravityError) as e:
            gpu.gravity_debug_set(ctx, gpu.GRAVITY_DBGSET_MOMENTS_STALL, bad)
        assert e.value.code == gpu.GRAVITY_E_ARG
