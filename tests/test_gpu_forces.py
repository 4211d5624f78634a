"""GPU walk (kernel 5, Sec. 2.1), direct sum (Eq. Newton) and stepping (Sec. 2.3)
against the FP64 oracle on the same seeded inputs.

Tolerances (derived from the FP32 pair arithmetic), checked on every body:
  * decision counts (node terms, body terms, opening tests) per body: exact;
  * tree accelerations: |a - a_oracle| <= 1e-6 * sum_k |term_k| (FP32 terms with hi/lo
    differences carry ~2^-22 relative error each, and the two-sum accumulation adds
    ~2^-24 of the partial sums), and the relative error |a - a_oracle| /
    max(|a_oracle|, 1e-3 rms) <= 1e-5 for every body whose force is not cancelled more
    than tenfold below its terms (sum |t| / |a| <= 10); the figures (largest relative
    error, bodies above 1e-5 and their cancellation) are recorded per case;
  * direct sums: the same, with a relative bound of 1e-6 (recorded per case).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_04197_gb300 import inputs
from util import check_parity

pytestmark = pytest.mark.gpu

SCALE_TOL = 1e-6
REL_TOL = 1e-5


def _gpu_forces(g, pos, m, theta, eps, counted=False, **kw):
    ctx = g.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    g.gravity_tree_build(ctx, P, M, g.params(**kw))
    acc = torch.empty_like(P)
    if counted:
        cnt = torch.empty((len(pos), 3), dtype=torch.int32, device="cuda")
        g.gravity_forces_counted(ctx, theta, eps, acc, cnt)
        g.gravity_sync(ctx)
        return acc.cpu().numpy(), cnt.cpu().numpy()
    g.gravity_forces(ctx, theta, eps, acc)
    g.gravity_sync(ctx)
    return acc.cpu().numpy(), None


DIRECT_REL_TOL = 1e-6


def _check(a, ref, absum, label, rel_tol=REL_TOL):
    return check_parity(a, ref, absum, label, rel_tol=rel_tol, scale_tol=SCALE_TOL)


CASES = {
    "sphere2048": lambda: inputs.uniform_sphere(2048, seed=0),
    "sphere20011": lambda: inputs.uniform_sphere(20011, seed=1),
    "clumpy30000": lambda: inputs.clumpy_plummer(30_000, seed=2, nclusters=8),
    "rubble20000": lambda: inputs.rubble_pile(20_000, seed=3),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("theta", [0.0, 0.3, 0.5, 0.9])
@pytest.mark.parametrize("leaf_max,order", [(1, 0), (1, 2), (8, 0), (16, 2)])
def test_tree_forces_vs_oracle(gpu, case, theta, leaf_max, order):
    pos, _, m = CASES[case]()
    if theta == 0.0 and len(pos) > 2048 and (leaf_max, order) != (1, 0):
        pytest.skip("theta = 0 is checked on the small case for the other layouts")
    eps = 1e-3
    a, cnt = _gpu_forces(gpu, pos, m, theta, eps, counted=True, leaf_max=leaf_max, order=order)
    t = oracle.Tree(pos, m, leaf_max=leaf_max, order=order)
    ref, absum, ocnt = t.forces(theta, eps)
    assert np.array_equal(cnt[:, 0], ocnt[:, 1]), "accepted-node counts differ"
    assert np.array_equal(cnt[:, 1], ocnt[:, 2]), "body-term counts differ"
    assert np.array_equal(cnt[:, 2], ocnt[:, 0]), "opening-test counts differ"
    _check(a, ref, absum, f"tree/{case}/theta{theta}/leaf{leaf_max}/order{order}")
    # the uncounted kernel gives the same result
    a2, _ = _gpu_forces(gpu, pos, m, theta, eps, leaf_max=leaf_max, order=order)
    assert np.array_equal(a, a2)


@pytest.mark.parametrize("kind,n,eps,G", [("clumpy", 70_001, 1e-3, 1.0), ("sphere", 40_000, 0.0, 1.7)])
def test_direct_sorted_tiles_vs_oracle(gpu, kind, n, eps, G):
    # from 32768 bodies on the direct sum runs on Morton-sorted tiles (block-relative
    # coordinates for tiles away from a block, hi/lo for the others): sampled bodies
    # against the oracle's FP64 sum, a coincident pair included (eps = 0: adds nothing)
    if kind == "clumpy":
        pos, _, m = inputs.clumpy_plummer(n, seed=31, nclusters=8)
    else:
        pos, _, m = inputs.uniform_sphere(n, seed=32)
        pos[17] = pos[12345]
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    acc = torch.empty_like(P)
    gpu.gravity_direct(ctx, P, M, eps, G, acc)
    gpu.gravity_sync(ctx)
    idx = np.union1d(inputs.subset(n, 2048, seed=33), [17, 12345, 0, n - 1])
    ref, absum = oracle.direct(pos, m, eps, G, targets=idx)
    a = acc.cpu().numpy()
    assert np.all(np.isfinite(a))
    _check(a[idx], ref, absum, f"direct_sorted/{kind}{n}", rel_tol=DIRECT_REL_TOL)


@pytest.mark.parametrize("mac_guard,accum,eps", [(0, 0, 1e-3), (1, 1, 1e-3), (1, 0, 0.0)])
def test_tree_variants(gpu, mac_guard, accum, eps):
    pos, _, m = inputs.clumpy_plummer(20_000, seed=7, nclusters=4)
    a, cnt = _gpu_forces(gpu, pos, m, 0.6, eps, counted=True, mac_guard=mac_guard, accum=accum,
                         leaf_max=4)
    t = oracle.Tree(pos, m, leaf_max=4)
    ref, absum, ocnt = t.forces(0.6, eps, mac_guard=mac_guard)
    assert np.array_equal(cnt[:, 0], ocnt[:, 1]) and np.array_equal(cnt[:, 1], ocnt[:, 2])
    assert np.array_equal(cnt[:, 2], ocnt[:, 0])
    _check(a, ref, absum, f"tree/variant/guard{mac_guard}/accum{accum}/eps{eps}")


def test_theta0_equals_direct(gpu):
    pos, _, m = inputs.uniform_sphere(4099, seed=4)
    a, _ = _gpu_forces(gpu, pos, m, 0.0, 1e-3, leaf_max=8)
    ref, absum = oracle.direct(pos, m, 1e-3)
    _check(a, ref, absum, "tree/theta0_vs_direct/sphere4099")


@pytest.mark.parametrize("n,eps,G", [(2048, 1e-3, 1.0), (10_007, 5e-3, 2.5), (3, 0.0, 1.0)])
def test_direct_vs_oracle(gpu, n, eps, G):
    pos, _, m = inputs.uniform_sphere(n, seed=n)
    if n == 3:
        pos[2] = pos[1]                               # coincident pair, eps = 0: term is zero
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    acc = torch.empty_like(P)
    gpu.gravity_direct(ctx, P, M, eps, G, acc)
    gpu.gravity_sync(ctx)
    ref, absum = oracle.direct(pos, m, eps, G)
    if n == 3:
        ref[1:] = 0.0
        ref[1] = G * m[0] * (pos[0] - pos[1]) / np.linalg.norm(pos[0] - pos[1]) ** 3
        ref[2] = ref[1]
        absum = np.linalg.norm(ref, axis=1) + 1e-300
    _check(acc.cpu().numpy(), ref, absum, f"direct/sphere{n}/eps{eps}", rel_tol=DIRECT_REL_TOL)


@pytest.mark.parametrize("leaf_max,order", [(1, 0), (16, 2)])
def test_tiny_clouds_vs_oracle(gpu, leaf_max, order):
    # 1 .. 64 bodies: one-block build, tasks split eight ways, a walk of a few nodes; counts
    # exact and every body within the parity rule
    for n in (1, 2, 3, 5, 8, 17, 33, 64):
        pos, _, m = inputs.uniform_sphere(n, seed=60 + n)
        a, cnt = _gpu_forces(gpu, pos, m, 0.5, 1e-3, counted=True, leaf_max=leaf_max, order=order)
        ref, absum, ocnt = oracle.Tree(pos, m, leaf_max=leaf_max, order=order).forces(0.5, 1e-3)
        assert np.array_equal(cnt[:, 0], ocnt[:, 1]) and np.array_equal(cnt[:, 1], ocnt[:, 2]), n
        assert np.array_equal(cnt[:, 2], ocnt[:, 0]), n
        if n > 1:
            _check(a, ref, absum, f"tiny/n{n}/leaf{leaf_max}/order{order}")
        else:
            assert np.array_equal(a, np.zeros((1, 3)))


def test_two_body_closed_form(gpu):
    pos = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    m = np.array([1.0, 3.0])
    a, _ = _gpu_forces(gpu, pos, m, 0.5, 0.0)
    assert np.allclose(a[0], [0.072, 0.096, 0.0], rtol=1e-6, atol=0)
    assert np.allclose(a[1] * 3.0, -a[0], rtol=1e-6)


@pytest.mark.parametrize("scheme", [0, 1])
def test_stepping_vs_oracle(gpu, scheme):
    pos, vel, m = inputs.rubble_pile(3000, seed=6)
    eps, dt, theta, steps = 5e-3, 1e-3, 0.5, 10
    ref0 = oracle.tree_forces(pos, m, theta, eps, leaf_max=1, order=2)
    P = torch.tensor(pos, device="cuda")
    V = torch.tensor(vel, device="cuda")
    M = torch.tensor(m, device="cuda")
    A = torch.tensor(ref0, device="cuda")
    ctx = gpu.Context(0)
    p = gpu.params(order=2, scheme=scheme)
    gpu.leapfrog_step(ctx, P, V, M, A, dt, steps, theta, eps, p)
    gpu.gravity_sync(ctx)
    op, ov, oa = oracle.step(pos, vel, m, ref0, dt, steps, scheme=scheme, theta=theta, eps=eps,
                             order=2)
    dx = np.abs(P.cpu().numpy() - op).max()
    dv = np.abs(V.cpu().numpy() - ov).max()
    assert dx < 1e-9 and dv < 1e-6, (dx, dv)


def test_host_entry_point(gpu):
    pos, _, m = inputs.uniform_sphere(5000, seed=8)
    ctx = gpu.Context(0)
    ph = torch.tensor(pos).pin_memory()
    mh = torch.tensor(m).pin_memory()
    ah = torch.empty((5000, 3), dtype=torch.float64).pin_memory()
    gpu.gravity_forces_host(ctx, ph, mh, 0.5, 1e-3, gpu.params(leaf_max=8), ah)
    a, _ = _gpu_forces(gpu, pos, m, 0.5, 1e-3, leaf_max=8)
    assert np.array_equal(ah.numpy(), a)


def test_host_batch_entry_point(gpu):
    # five different snapshots through the overlapped batch call (copies on their own
    # streams, two device slots reused, two engines taking turns): each result equals the
    # one-snapshot call's bit for bit; a repeated input pointer is allowed, and so is an
    # empty batch
    n = 20_000
    snaps = [inputs.clumpy_plummer(n, seed=30 + k, nclusters=4) for k in range(4)]
    snaps.append(snaps[1])
    ph = [torch.tensor(s_[0]).pin_memory() for s_ in snaps]
    mh = [torch.tensor(s_[2]).pin_memory() for s_ in snaps]
    ah = [torch.full((n, 3), np.nan, dtype=torch.float64).pin_memory() for _ in snaps]
    p = gpu.params(order=2, leaf_max=16)
    ctx = gpu.Context(0)
    gpu.gravity_forces_host_batch(ctx, ph, mh, 0.5, 1e-3, p, ah)
    one = gpu.Context(0)
    ref = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    for k in range(len(snaps)):
        gpu.gravity_forces_host(one, ph[k], mh[k], 0.5, 1e-3, p, ref)
        assert np.array_equal(ah[k].numpy(), ref.numpy()), k
    # every other snapshot runs on the context's internal twin; the tree left in the
    # context is the last snapshot's, for an odd and an even count
    keys = lambda c: gpu.gravity_debug_export(c, gpu.DBG_KEYS, n)
    assert np.array_equal(keys(ctx), keys(one))
    ah4 = [torch.full((n, 3), np.nan, dtype=torch.float64).pin_memory() for _ in range(4)]
    gpu.gravity_forces_host_batch(ctx, ph[:4], mh[:4], 0.5, 1e-3, p, ah4)
    for k in range(4):
        assert np.array_equal(ah4[k].numpy(), ah[k].numpy()), k
    gpu.gravity_forces_host(one, ph[3], mh[3], 0.5, 1e-3, p, ref)
    assert np.array_equal(keys(ctx), keys(one))
    gpu.gravity_forces_host_batch(ctx, [], [], 0.5, 1e-3, p, [])
    with pytest.raises(gpu.GravityError) as e:
        gpu.gravity_forces_host_batch(ctx, ph[:1], mh[:1], -1.0, 1e-3, p, ah[:1])
    assert e.value.code == gpu.GRAVITY_E_ARG


@pytest.mark.parametrize("clouds", [False, True])
def test_leapfrog_graph_replay_matches_eager(gpu, clouds):
    # on a non-default stream leapfrog_step captures one step as a CUDA graph and
    # replays it; the result must equal launching every kernel (same kernels, same order)
    if clouds:
        off, pos, vel, m = inputs.ensemble(nclouds=12, seed=2, nmin=100, nmax=3000)
    else:
        off = None
        pos, vel, m = inputs.rubble_pile(20_000, seed=9)
    out = []
    for use_graph in (0, 1):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            ctx = gpu.Context(0)
            if clouds:
                gpu.gravity_set_clouds(ctx, off)
            P = torch.tensor(pos, device="cuda")
            V = torch.tensor(vel, device="cuda")
            M = torch.tensor(m, device="cuda")
            A = torch.empty_like(P)
            p = gpu.params(order=2, leaf_max=16, use_graph=use_graph)
            gpu.gravity_tree_build(ctx, P, M, p)
            gpu.gravity_forces(ctx, 0.5, 1e-3, A)
            gpu.leapfrog_step(ctx, P, V, M, A, 1e-3, 8, 0.5, 1e-3, p)
            gpu.leapfrog_step(ctx, P, V, M, A, 1e-3, 4, 0.5, 1e-3, p)   # reuses the graph
            gpu.gravity_sync(ctx)
        stream.synchronize()
        out.append((P.cpu().numpy(), V.cpu().numpy(), A.cpu().numpy()))
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)


def test_task_order_from_costs_keeps_results(gpu):
    # a full force walk takes each task queue's tasks in the order of the cycles they took
    # in the previous walk (costliest first): which warp runs a task, and when, must change
    # no result, so later walks equal the first (index-order) walk bit for bit, and so does
    # the counted walk (which keeps index order)
    pos, _, m = inputs.clumpy_plummer(200_000, seed=3, nclusters=16)
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    gpu.gravity_tree_build(ctx, P, M, gpu.params(order=2, leaf_max=16))
    first = None
    for _ in range(3):
        A = torch.full_like(P, float("nan"))
        gpu.gravity_forces(ctx, 0.5, 1e-3, A)
        gpu.gravity_sync(ctx)
        if first is None:
            first = A.cpu().numpy()
            assert np.isfinite(first).all()
        else:
            assert np.array_equal(A.cpu().numpy(), first)
    A = torch.full_like(P, float("nan"))
    C = torch.empty((len(pos), 3), dtype=torch.int32, device="cuda")
    gpu.gravity_forces_counted(ctx, 0.5, 1e-3, A, C)
    gpu.gravity_sync(ctx)
    assert np.array_equal(A.cpu().numpy(), first)


def test_leapfrog_graph_dropped_when_buffers_grow(gpu):
    # a larger tree on the same context reallocates the buffers a captured leapfrog step
    # refers to; the captured step must be dropped (and captured again), so that stepping
    # the first problem afterwards equals stepping it without the interleaved call
    pos, vel, m = inputs.rubble_pile(5_000, seed=4)
    big, _, mbig = inputs.clumpy_plummer(120_000, seed=5, nclusters=8)
    out = []
    for interleave in (False, True):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            ctx = gpu.Context(0)
            P = torch.tensor(pos, device="cuda")
            V = torch.tensor(vel, device="cuda")
            M = torch.tensor(m, device="cuda")
            A = torch.empty_like(P)
            p = gpu.params(order=2, leaf_max=16, use_graph=1)
            gpu.gravity_tree_build(ctx, P, M, p)
            gpu.gravity_forces(ctx, 0.5, 1e-3, A)
            gpu.leapfrog_step(ctx, P, V, M, A, 1e-3, 6, 0.5, 1e-3, p)    # captures a step
            if interleave:
                PB = torch.tensor(big, device="cuda")
                MB = torch.tensor(mbig, device="cuda")
                AB = torch.empty_like(PB)
                gpu.gravity_tree_build(ctx, PB, MB, p)                # buffers grow
                gpu.gravity_forces(ctx, 0.5, 1e-3, AB)
            gpu.leapfrog_step(ctx, P, V, M, A, 1e-3, 6, 0.5, 1e-3, p)
            gpu.gravity_sync(ctx)
        stream.synchronize()
        out.append((P.cpu().numpy(), V.cpu().numpy(), A.cpu().numpy()))
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("mac_guard", [1, 0])
def test_opening_band_on_a_lattice(gpu, mac_guard):
    # A 17^3 lattice on [0, 1]^3 (root side 1): depth-3 cells (side 1/8) hold 2x2x2 bodies
    # with the COM at odd multiples of 1/32, so bodies at offsets (5, 3, 3)/32 see
    # l^2 = theta^2 D^2 up to the rounding of theta^2 = 16/43 (Eq. accuracy at equality).
    # These tests land in the kernel's FP32 uncertainty band and are taken in FP64; the
    # decision counts must still equal the oracle's for every body.
    k = np.arange(17) / 16.0
    pos = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    m = np.ones(len(pos))
    theta = float(np.sqrt(16.0 / 43.0))
    ctx = gpu.Context(0)
    P = torch.tensor(pos, device="cuda")
    M = torch.tensor(m, device="cuda")
    gpu.gravity_tree_build(ctx, P, M, gpu.params(leaf_max=1, order=0, mac_guard=mac_guard))
    acc = torch.empty_like(P)
    cnt = torch.empty((len(pos), 3), dtype=torch.int32, device="cuda")
    gpu.gravity_forces_counted(ctx, theta, 1e-3, acc, cnt)
    gpu.gravity_sync(ctx)
    fp64_decisions = int(gpu.gravity_debug_export(ctx, gpu.DBG_WALKSTATS, 16)[3])
    assert fp64_decisions >= 1000, fp64_decisions
    ref, absum, ocnt = oracle.Tree(pos, m, leaf_max=1).forces(theta, 1e-3, mac_guard=mac_guard)
    c = cnt.cpu().numpy()
    assert np.array_equal(c[:, 0], ocnt[:, 1]) and np.array_equal(c[:, 1], ocnt[:, 2])
    assert np.array_equal(c[:, 2], ocnt[:, 0])
    _check(acc.cpu().numpy(), ref, absum, f"tree/lattice_band/guard{mac_guard}")


@pytest.mark.parametrize("scheme", [0, 1])
def test_two_time_steps_vs_oracle(gpu, scheme):
    # Sec. 4.1: the stepper advances by the contact step dt and gravity is evaluated every
    # grav_every-th step (Delta t_g = grav_every dt, bounded by Eq. dt_g), held in between;
    # against the oracle's run with the same schedule, and the count carries across calls
    pos, vel, m = inputs.rubble_pile(3000, seed=16)
    eps, dt, theta, k, steps = 5e-3, 1e-3, 0.5, 4, 12
    ref0 = oracle.tree_forces(pos, m, theta, eps, leaf_max=1, order=2)
    out = []
    for split in ((steps,), (5, 7)):
        ctx = gpu.Context(0)
        P = torch.tensor(pos, device="cuda")
        V = torch.tensor(vel, device="cuda")
        M = torch.tensor(m, device="cuda")
        A = torch.tensor(ref0, device="cuda")
        p = gpu.params(order=2, scheme=scheme, grav_every=k)
        for ns in split:
            gpu.leapfrog_step(ctx, P, V, M, A, dt, ns, theta, eps, p)
        gpu.gravity_sync(ctx)
        out.append((P.cpu().numpy(), V.cpu().numpy(), A.cpu().numpy()))
    for x, y in zip(*out):
        assert np.array_equal(x, y)
    op, ov, oa = oracle.step(pos, vel, m, ref0, dt, steps, scheme=scheme, theta=theta, eps=eps,
                             order=2, grav_every=k)
    P, V, A = out[0]
    assert np.abs(P - op).max() < 1e-9 and np.abs(V - ov).max() < 1e-6
    # the last step evaluated gravity: the forces at the run's own final positions
    ref, absum, _ = oracle.Tree(P, m, leaf_max=1, order=2).forces(theta, eps)
    check_parity(A, ref, absum, f"two_time_steps/scheme{scheme}")
    assert np.abs(A - oa).max() <= 1e-6 * np.abs(oa).max()
    with pytest.raises(gpu.GravityError):
        gpu.leapfrog_step(gpu.Context(0), torch.tensor(pos, device="cuda"),
                          torch.tensor(vel, device="cuda"), torch.tensor(m, device="cuda"),
                          torch.tensor(ref0, device="cuda"), dt, 1, theta, eps,
                          gpu.params(grav_every=-1))
