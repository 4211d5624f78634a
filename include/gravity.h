/*
 * gravity.h - C ABI of libgravity, a GB300 (sm_103a) Barnes-Hut octree gravity library.
 *
 * Method: Ferrari, Lavagna, Blazquez, "A parallel-GPU code for asteroid aggregation
 * problems with angular particles", MNRAS 2019 (arXiv:1912.04197), Sec. 2.1:
 * N point masses, Eq. (Newton); octree clustering with the opening test of
 * Eq. (accuracy); force rules Eqs. (Force_leaf, Force_thetaTrue) with the softened
 * distance of Eq. (Force_rComp); node moments Eq. (COMinternal); the tree is
 * rebuilt every step.  The library returns accelerations (force / body mass).
 *
 * Conventions shared by every entry point:
 *   - Array arguments are DEVICE pointers (e.g. torch.Tensor.data_ptr()) unless the
 *     name ends in _host.  They are contiguous, row-major, caller-owned, and not
 *     retained after the call returns.  pos/vel/acc are (n, 3) FP64, mass is (n) FP64.
 *   - All work is enqueued on the context's CUDA stream (the caller's stream); no
 *     call synchronises the device except gravity_sync, gravity_debug_export and
 *     the _host entry points.
 *   - Return value: GRAVITY_OK (0) or a negative GRAVITY_E_* code.  Argument and
 *     launch errors are returned immediately.  Errors found on the device (a
 *     non-finite coordinate, an exhausted walk stack, a bounded wait that ran out)
 *     are latched in the context and returned by the next gravity_sync.  After a
 *     latched error the outputs of the affected call are unspecified.
 *   - No exception crosses the ABI and nothing aborts the process.
 *   - The context owns all scratch memory (sort buffers, tree, walk records); it
 *     grows on demand and is freed by gravity_destroy.  One context must not be
 *     used from two host threads at once.
 */
#ifndef GRAVITY_H
#define GRAVITY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum gravity_status {
  GRAVITY_OK = 0,
  GRAVITY_E_ARG = -1,        /* invalid argument (n < 0, theta < 0, eps < 0, null pointer, ...) */
  GRAVITY_E_NONFINITE = -2,  /* a position coordinate is NaN or infinite, or a contact radius
                                is negative or not finite (latched) */
  GRAVITY_E_NOMEM = -3,      /* device allocation failed */
  GRAVITY_E_CUDA = -4,       /* a CUDA runtime call failed */
  GRAVITY_E_TIMEOUT = -5,    /* a bounded device-side wait ran out (latched) */
  GRAVITY_E_INTERNAL = -6,   /* walk or contact-search stack exhausted, or an inconsistent
                                tree (latched) */
  GRAVITY_E_NOTREE = -7      /* gravity_forces called before gravity_tree_build */
};

typedef struct gravity_ctx gravity_ctx;

/* Caller-supplied device allocator (see gravity_set_allocator).  alloc stores a device
 * pointer of at least `bytes` bytes (aligned to 256 bytes) in *ptr and returns 0, or
 * returns non-zero on failure; release frees a pointer alloc returned.  `user` is passed
 * through unchanged. */
typedef int (*gravity_alloc_fn)(void **ptr, size_t bytes, void *user);
typedef void (*gravity_free_fn)(void *ptr, void *user);

/* Tunables.  Fill with gravity_params_default() and change what you need. */
typedef struct gravity_params {
  double G;            /* gravitational constant of Eq. (Newton); default 1.0 */
  int32_t order;       /* 0 = monopole node terms (the paper), 2 = + traceless quadrupole */
  int32_t leaf_max;    /* bodies per leaf cell: 1 = the paper's "zero or one body"
                          (Sec. 2.1); 1..64 allowed */
  int32_t accum;       /* per-body accumulation: 0 = FP32 compensated (two-sum), 1 = FP64 */
  int32_t mac_guard;   /* 1 (default) = a cell that contains the body is always opened;
                          0 = plain opening test for every cell */
  int32_t scheme;      /* leapfrog_step only: 0 = kick-drift-kick leapfrog,
                          1 = semi-implicit (symplectic) Euler (Sec. 2.3) */
  int32_t walk_cfg;    /* -1 = default launch shape of the walk; >= 0 = index into the
                          table of walk launch shapes (autotuner use) */
  int32_t use_graph;   /* leapfrog_step with nsteps > 2 on a non-default stream: 1 (default)
                          = capture one step as a CUDA graph and replay it, 0 = launch
                          every kernel of every step.  The captured step is dropped, and
                          captured again by the next call, whenever the context frees a
                          device buffer (a larger tree, another call's scratch) */
  int32_t grav_every;  /* leapfrog_step only: evaluate gravity every grav_every-th step and hold
                          the last acceleration in between (the two time steps of Sec. 4.1:
                          a stepper at the contact step dt with gravity every Delta t_g, Eq.
                          (dt_g), i.e. grav_every = ceil(Delta t_g / dt)); 0 or 1 = every step
                          (default 1).  The context counts steps since gravity was last
                          evaluated across calls; gravity_tree_build and gravity_forces reset
                          the count (the acceleration passed in acc_cache counts as fresh). */
} gravity_params;

/* Fill *p with the defaults: G = 1, order 0, leaf_max 1, accum 0, mac_guard 1,
 * scheme 0, walk_cfg -1, use_graph 1, grav_every 1. */
void gravity_params_default(gravity_params *p);

/* Create a context on CUDA device `device` whose work goes to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the handle. */
int gravity_create(gravity_ctx **out, int device, void *cuda_stream);

/* Synchronise the context's stream and free everything it owns.  NULL is a no-op. */
int gravity_destroy(gravity_ctx *ctx);

/* Change the stream later calls are enqueued on. */
int gravity_set_stream(gravity_ctx *ctx, void *cuda_stream);

/* Route every device allocation of the context through the caller's allocator (for
 * instance an application's memory pool); alloc = release = NULL restores
 * cudaMalloc/cudaFree.  Synchronises the context's stream, then releases ALL of the
 * context's device memory (the tree, the cloud segmentation, every scratch buffer) with
 * the allocator that made it and re-creates the small fixed buffers with the new one: the
 * context is left as after gravity_create (no tree, one cloud).  An allocation the
 * allocator refuses makes the call that needed it return GRAVITY_E_NOMEM, with no buffer
 * left half-made; the context stays usable. */
int gravity_set_allocator(gravity_ctx *ctx, gravity_alloc_fn alloc, gravity_free_fn release,
                          void *user);

/* Kernels 1-4 of the paper's five-kernel list (Sec. 2.1, "CUDA implementation"):
 * bounding cube of all bodies (the root), octree construction (63-bit Morton keys,
 * stable device radix sort = "sort bodies", binary radix tree collapsed to an
 * octree), and node mass / centre of mass by Eq. (COMinternal) in FP64 (plus the
 * traceless quadrupole when p->order == 2, its second moments carried up the tree in
 * double-float FP32 arithmetic, ~47 significant bits).  The tree stays in the context until
 * the next build; pos and mass are read during this call only.
 * n = 0 is a no-op that leaves an empty tree.  p = NULL means defaults. */
int gravity_tree_build(gravity_ctx *ctx, int64_t n, const double *pos, const double *mass,
                       const gravity_params *p);

/* Kernel 5 of the list (Sec. 2.1): for every body, walk the tree from the root;
 * a node with l < theta * D (l = cell side, D = distance to the node's centre of
 * mass, Eq. (accuracy)) contributes its monopole (Eq. Force_thetaTrue) and, with
 * order 2, its quadrupole; otherwise it is opened; a single-body leaf contributes a
 * body-to-body term (Eq. Force_leaf).  Every term uses r^2 = |d|^2 + eps^2
 * (Eq. Force_rComp); a term with r^2 = 0 contributes nothing.
 * acc: (n, 3) FP64, caller order, overwritten with G-scaled accelerations.
 * theta = 0 is exact (direct summation); theta < 0 or eps < 0 -> GRAVITY_E_ARG. */
int gravity_forces(gravity_ctx *ctx, double theta, double eps, double *acc);

/* As gravity_forces, and also writes per-body decision counts (caller order,
 * int32 (n, 3): node terms accepted, body-to-body terms excluding the body
 * itself, opening tests of Eq. (accuracy) evaluated) to the device array counts.
 * Slower; meant for tests and for counting the walk's algorithmic work. */
int gravity_forces_counted(gravity_ctx *ctx, double theta, double eps, double *acc,
                           int32_t *counts);

/* ---- Sharded evaluation of one cloud (several GPUs, one context each).  Kernel 5 of the
 * paper's list (Sec. 2.1) computes every body's force from the tree independently of the
 * other bodies, so the bodies can be split between devices: every device builds the same
 * tree from the same positions (the build is deterministic), walks a contiguous range of
 * the walk's tasks, and the ranges' results are exchanged by the caller (one all-gather
 * per step; this library makes no collective call).  A task is up to 32 bodies that are
 * consecutive in the tree's (Morton) order and belong to one cloud. */

/* Number of walk tasks of the current tree.  GRAVITY_E_NOTREE before a build. */
int gravity_walk_tasks(gravity_ctx *ctx, int64_t *ntasks);

/* Bodies of tasks [first_task, first_task + ntasks): *first_body is the first sorted
 * position, *nbodies their count (the tasks' bodies are consecutive in sorted order).
 * Host arithmetic only.  GRAVITY_E_ARG for a range outside [0, gravity_walk_tasks). */
int gravity_task_bodies(gravity_ctx *ctx, int64_t first_task, int64_t ntasks,
                        int64_t *first_body, int64_t *nbodies);

/* gravity_forces restricted to tasks [first_task, first_task + ntasks): acc_sorted
 * (device, (nbodies, 3) FP64, caller-owned) receives the G-scaled accelerations of the
 * tasks' bodies in sorted order (row i = sorted body first_body + i, see
 * gravity_task_bodies).  Each row equals the one gravity_forces computes for that body,
 * bit for bit (same tasks, same launch decisions).  Asynchronous. */
int gravity_forces_range(gravity_ctx *ctx, double theta, double eps, int64_t first_task,
                         int64_t ntasks, double *acc_sorted);

/* dst[perm[first_body + i]] = src_sorted[i] for i < nbodies: rows in the tree's sorted
 * order back to the caller's order (perm = the current tree's order, gravity_tree_build).
 * Device (n,3)-row arrays, FP64; rows of dst not addressed are left unchanged. */
int gravity_scatter_sorted(gravity_ctx *ctx, int64_t first_body, int64_t nbodies,
                           const double *src_sorted, double *dst);

/* The integrator's pieces (Sec. 2.3) as separate calls, for a caller that assembles a step
 * around gravity_forces_range: kick-drift v += h_kick a; x += dt v, and the kick
 * v += h_kick a, over n bodies (device (n,3) FP64, no FMA contraction: the same roundings
 * as leapfrog_step). */
int gravity_kick_drift(gravity_ctx *ctx, int64_t n, double *pos, double *vel, const double *acc,
                       double h_kick, double dt);
int gravity_kick(gravity_ctx *ctx, int64_t n, double *vel, const double *acc, double h_kick);

/* Vector-Jacobian product of the tree accelerations with respect to the body
 * positions, the interaction decisions of the current tree held fixed (the tree
 * of the last gravity_tree_build; monopole terms of Eq. (Force_thetaTrue) and
 * Eq. (Force_leaf) with the softening of Eq. (Force_rComp)).  The paper has no
 * adjoint: this is the differentiation layer built on its force kernel.
 *   grad_pos = (d acc / d pos)^T lambda
 * For each accepted term a_i += G m_s f(s - x_i), f(d) = d / (|d|^2 + eps^2)^{3/2},
 * with w = G m_s J(d) lambda_i, J = (I - 3 d d^T / r^2) / r^3: x_i takes -w and the
 * source s takes +w; a node's COM is sum_j m_j x_j / M, so its share reaches body j
 * as (m_j / M) w.  theta, eps and the opening decisions are those of gravity_forces
 * with the same arguments.
 * lambda, grad_pos: device, (n,3) FP64 row-major, caller order; lambda is read,
 * grad_pos written (every row).  Requires order 0 (GRAVITY_E_ARG otherwise);
 * GRAVITY_E_NOTREE without a tree.  Works with several clouds as gravity_forces.
 * FP32 terms, compensated per-body sums, FP64 scatter (atomics: the last bits may
 * differ between runs).  Asynchronous on the context's stream; allocates scratch of
 * 96 bytes per body of capacity on first use (synchronises then). */
int gravity_forces_vjp(gravity_ctx *ctx, double theta, double eps, const double *lambda,
                       double *grad_pos);

/* Reverse pass (adjoint) of leapfrog_step, kick-drift-kick, over one checkpointed
 * segment of nsteps steps starting at the saved state (pos0, vel0) (device, (n,3)
 * FP64, read only).  The segment's positions x_0 .. x_nsteps are recomputed with the
 * forward kernels (identical results), then, from the last level down, each level k
 * applies xbar += c_k J(x_k)^T vbar (J = d a / d x on the tree of x_k, decisions
 * frozen: gravity_forces_vjp) followed by the reverse of the drift before it,
 * vbar += dt xbar.  c_k = dt/2 at the trajectory's two end levels, dt at interior
 * levels (two half kicks share one x_k and one vbar).  flags:
 *   GRAVITY_ADJ_END    the segment ends at the trajectory's final level: that level's
 *                      half kick is included (on entry xbar, vbar are the cotangents
 *                      of the final x, v); without it the caller already applied level
 *                      nsteps (as the first level of the following segment)
 *   GRAVITY_ADJ_START  the segment starts at the trajectory's initial level: its half
 *                      kick closes the pass and no drift follows it
 * Segments are processed from the last to the first; with both flags one call
 * reverses a whole trajectory.  xbar, vbar: device, (n,3), caller order, updated in
 * place.  With GRAVITY_ADJ_START they end as the cotangents of (pos0, vel0);
 * without it the reverse of the drift that produced pos0 is applied too, which is
 * where the preceding segment's call continues.  p: order 0 and scheme 0 only
 * (GRAVITY_E_ARG otherwise).  Allocates on first use (synchronising then)
 * (nsteps + 1) * 24 bytes per body for the positions and, when it can, about
 * (nsteps + 1) * 250 bytes per body to keep each level's tree for the reverse pass (else
 * the trees are built again); leaves the tree of the last recomputed level in the
 * context. */
enum gravity_adjoint_flags { GRAVITY_ADJ_END = 1, GRAVITY_ADJ_START = 2 };
int leapfrog_adjoint(gravity_ctx *ctx, int64_t n, const double *pos0, const double *vel0,
                     const double *mass, double dt, int nsteps, double theta, double eps,
                     const gravity_params *p, int flags, double *xbar, double *vbar);

/* Independent clouds ("batched ensemble"): many separate N-body problems handled
 * by one tree build and one walk launch.  offsets_host (host memory, nclouds + 1
 * int64) gives cloud k as bodies [offsets[k], offsets[k+1]) of the arrays passed
 * to later calls (offsets[0] = 0, strictly increasing; at most 65536 clouds).
 * Each cloud gets its own root cube and octree, exactly as if it were built alone,
 * and bodies feel only the bodies of their own cloud.  The segmentation stays in
 * effect for gravity_tree_build / gravity_forces / leapfrog_step (whose n must then
 * equal offsets[nclouds]) until changed; nclouds <= 1 returns to a single cloud.
 * Synchronises the context's stream. */
int gravity_set_clouds(gravity_ctx *ctx, int32_t nclouds, const int64_t *offsets_host);

/* gravity_set_clouds followed by gravity_tree_build of all clouds. */
int gravity_batch_tree_build(gravity_ctx *ctx, int32_t nclouds, const int64_t *offsets_host,
                             const double *pos, const double *mass, const gravity_params *p);

/* Eq. (Newton) with the softening of Eq. (Force_rComp), all N(N-1) pairs:
 * acc_i = G sum_{j != i} m_j (R_j - R_i) / (|R_j - R_i|^2 + eps^2)^{3/2}.
 * FP32 pair terms, compensated accumulation, FP64 out.  From 32768 bodies on, the
 * bodies are put in Morton order first (the context's own buffers; its tree is
 * untouched) so that each source
 * tile far from a block of targets is evaluated on FP32 coordinates relative to the
 * block, the others on hi/lo split coordinates; every term's error stays a few 2^-24 of
 * its size. */
int gravity_direct(gravity_ctx *ctx, int64_t n, const double *pos, const double *mass,
                   double eps, double G, double *acc);

/* Allocation-free direct sum (the paper has no counterpart: this is a library
 * service).  For callers that cannot call cudaMalloc - an application that owns
 * all device memory (fixed-budget pool, plugin host forbidding allocations after
 * start-up), or a latency-critical loop that cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree.  The same sum as gravity_direct (equal to
 * rounding: it keeps the caller's order and hi/lo coordinates for every pair, where
 * gravity_direct sorts the bodies first), but needs no context and allocates nothing:
 * the hi/lo staging of the
 * bodies lives in a file-scope __device__ array of 2 MiB, sized for at most
 * 65536 bodies, which every GPU that loads the library holds until the process
 * exits.
 *   n      number of bodies, 0 <= n <= 65536; larger n -> GRAVITY_E_ARG (nothing runs)
 *   pos, mass, acc  device pointers as for gravity_direct, on the CURRENT device
 *   cuda_stream     stream the two kernels are enqueued on (NULL = legacy default)
 * The first call on a device (with that device current) resolves the array's
 * device address with cudaGetSymbolAddress; make that first call before any stream
 * capture.  The address is cached for the life of the process: a process that resets
 * the device (cudaDeviceReset) must not call this entry point afterwards.  All calls on a device share the one array, which keeps the last call's
 * contents (every entry a call reads is written by that call first): calls that
 * overlap on the GPU (different streams, or different host threads) race and give
 * wrong results - serialise them. */
int gravity_direct_noalloc(int64_t n, const double *pos, const double *mass, double eps,
                           double G, double *acc, void *cuda_stream);

/* Conserved quantities of the softened N-body system (the energy and momenta that
 * Sec. 3.1 tracks), on the device:
 *   out[0] = E = sum_i m_i |v_i|^2 / 2 - G sum_{i<j} m_i m_j / sqrt(|x_j - x_i|^2 + eps^2)
 *   out[1..3] = P = sum_i m_i v_i,   out[4..6] = L = sum_i m_i x_i x v_i
 * pos, vel: device (n,3) FP64; mass: device (n) FP64; out: DEVICE, 7 doubles, written
 * asynchronously on the context's stream.  The potential is an O(n^2) sum of FP32 pair
 * terms on hi/lo coordinates (relative error ~1e-7 of |E_pot|); kinetic energy and
 * momenta are FP64 sums in a fixed order (deterministic).  A pair with r^2 = 0 adds
 * nothing.  n = 0 writes zeros. */
int gravity_diagnostics(gravity_ctx *ctx, int64_t n, const double *pos, const double *vel,
                        const double *mass, double eps, double G, double *out);

/* Aggregate identification (Sec. 2, "Post-processing: aggregate identification"): the
 * connected components of the contact graph whose vertices are the bodies of the current
 * tree.  The paper takes the edges from its collision solver's contact container; here two
 * bodies i != j of the same cloud are in contact when |x_i - x_j|^2 <= t_ij^2, in FP64 with
 * d = x_j - x_i and |d|^2 = (dx^2 + dy^2) + dz^2, each operation rounded once (every edge is
 * decided as a plain pairwise test decides it), t_ij = radius[i] + radius[j] (touching
 * bounding spheres) when radius is given, else t_ij = dmax.  The positions are those of the
 * last gravity_tree_build / gravity_batch_tree_build (the tree serves as the neighbour
 * search).
 *   radius  device, (n) doubles in caller order, each >= 0 and finite, or NULL
 *   dmax    uniform threshold (>= 0, finite), used when radius is NULL
 *   label   device, (n) int32 out, caller order: the smallest caller index of the body's
 *           component (canonical: independent of the order of the unions)
 *   counts  device, two int64 out: the number of components, and the number of
 *           aggregates (components of more than one body, the paper's count); or NULL
 * Written asynchronously on the context's stream.  Errors: GRAVITY_E_NOTREE without a
 * tree, GRAVITY_E_ARG for a bad dmax (radius NULL) or a NULL label, GRAVITY_E_NOMEM;
 * a negative or non-finite radius is latched (read by gravity_sync) and counts as 0. */
int gravity_components(gravity_ctx *ctx, const double *radius, double dmax, int32_t *label,
                       int64_t *counts);

/* Largest gravity time step of Eq. (dt_g) (Sec. 4.1): *dt_g = T_g / 2 = 1 / (2 sqrt(G rho)),
 * rho the material density of the bodies (host arithmetic, no device work).  A caller that
 * steps contacts with dt_c evaluates gravity every ceil(dt_g / dt_c) contact steps, as the
 * paper's two-time-step scheme does.  Errors: GRAVITY_E_ARG unless G > 0 and rho > 0 are
 * finite and dt_g is non-NULL. */
int gravity_dt_g(double G, double rho, double *dt_g);

/* nsteps steps of a symplectic integrator (Sec. 2.3) with the tree rebuilt every
 * step (Sec. 2.1).  p->scheme 0 (kick-drift-kick leapfrog):
 *   v += dt/2 a;  x += dt v;  a = a(x);  v += dt/2 a
 * p->scheme 1 (semi-implicit Euler):  v += dt a;  x += dt v;  a = a(x).
 * pos, vel: (n, 3) FP64, updated in place.  acc_cache: (n, 3) FP64, a(x) of the
 * incoming positions on entry (compute it once with gravity_tree_build +
 * gravity_forces) and a(x) of the outgoing positions on exit.  theta = 0 uses the
 * tree walk at theta = 0, i.e. the exact sum. */
int leapfrog_step(gravity_ctx *ctx, int64_t n, double *pos, double *vel, const double *mass,
                  double *acc_cache, double dt, int nsteps, double theta, double eps,
                  const gravity_params *p);

/* Host-buffer evaluation: copy pos_host / mass_host (ideally pinned) to the
 * device, build the tree, walk it, copy the accelerations to acc_host, and wait
 * for completion.  Returns any latched device error.  Same semantics as
 * gravity_tree_build followed by gravity_forces. */
int gravity_forces_host(gravity_ctx *ctx, int64_t n, const double *pos_host,
                        const double *mass_host, double theta, double eps,
                        const gravity_params *p, double *acc_host);

/* Host-buffer evaluation of nsnap independent snapshots of n bodies each: snapshot k
 * has positions pos_host[k] (3n doubles) and masses mass_host[k] (n doubles), and its
 * accelerations go to acc_host[k] (3n doubles); the pointers may repeat (ideally pinned
 * memory).  Each snapshot's result is the one gravity_forces_host gives.  The copies of a
 * snapshot run beside the tree build and walk of its neighbours: two device slots of
 * inputs and outputs, a host-to-device and a device-to-host copy stream of the context
 * (created on first use), ordered against the compute streams by events.  With two
 * snapshots or more (one cloud), every other snapshot is evaluated by a second context
 * that this one creates on first use, with its own tree, walk buffers and stream and the
 * same allocator: one snapshot's build runs while the other's walk finishes (the twin
 * holds as much device memory as this context; it is released by gravity_destroy and
 * gravity_set_allocator).  The tree left in the context is the last snapshot's.  Returns
 * once every copy has finished, with any latched device error of either context (on an
 * error the remaining snapshots are not evaluated).
 * GRAVITY_E_ARG for a null array or pointer, a negative count or bad theta / eps. */
int gravity_forces_host_batch(gravity_ctx *ctx, int64_t nsnap, int64_t n,
                              const double *const *pos_host, const double *const *mass_host,
                              double theta, double eps, const gravity_params *p,
                              double *const *acc_host);

/* Wait for the context's stream, then return (and clear) the first latched device
 * error, or a CUDA error, or GRAVITY_OK. */
int gravity_sync(gravity_ctx *ctx);

/* Tree introspection for tests.  Synchronises.  Copies into host memory:
 *   GRAVITY_DBG_ROOT      4 doubles per cloud: lo[3], side
 *   GRAVITY_DBG_KEYS      n uint64: Morton keys in sorted order
 *   GRAVITY_DBG_PERM      n int32: caller index of each sorted body
 *   GRAVITY_DBG_NNODES    1 int32: node count
 *   GRAVITY_DBG_TOPO      nnodes x 4 int32: first child (-1 = leaf), child count,
 *                         body begin, body end (sorted order, end exclusive); node k
 *                         (k < number of clouds) is the root of cloud k
 *   GRAVITY_DBG_DEPTH     nnodes int32
 *   GRAVITY_DBG_PARENT    nnodes int32 (-1 for the root)
 *   GRAVITY_DBG_MASS      nnodes double
 *   GRAVITY_DBG_COM       nnodes x 3 double
 *   GRAVITY_DBG_QUAD      nnodes x 6 double (xx, yy, zz, xy, xz, yz)
 *   GRAVITY_DBG_WALKSTATS 16 uint64 from the last gravity_forces_counted: batches, node items,
 *                         mixed nodes, FP64 decisions, point-list entries, quadrupole-list
 *                         entries, deepest stack, terms evaluated by active lanes, lockstep
 *                         iterations of lists split by 16 / 8 / 1 lanes, full-mask entries,
 *                         far-list entries, mixed nodes that all tested lanes decided alike,
 *                         lockstep iterations of the point list split by 1 lane, 1 reserved
 * bytes must be at least the size listed; otherwise GRAVITY_E_ARG. */
enum gravity_debug_item {
  GRAVITY_DBG_ROOT = 0,
  GRAVITY_DBG_KEYS = 1,
  GRAVITY_DBG_PERM = 2,
  GRAVITY_DBG_NNODES = 3,
  GRAVITY_DBG_TOPO = 4,
  GRAVITY_DBG_DEPTH = 5,
  GRAVITY_DBG_PARENT = 6,
  GRAVITY_DBG_MASS = 7,
  GRAVITY_DBG_COM = 8,
  GRAVITY_DBG_QUAD = 9,
  GRAVITY_DBG_WALKSTATS = 10
};
int gravity_debug_export(gravity_ctx *ctx, int what, void *host_dst, size_t bytes);

/* Settings for failure testing.  GRAVITY_DBGSET_STACK_CAP: largest number of walk stack
 * entries a warp may hold (1 .. the built-in capacity; 0 restores the full capacity); a
 * walk that needs more latches GRAVITY_E_INTERNAL (reported by gravity_sync) instead of
 * growing, as an exhausted stack does.  GRAVITY_DBGSET_SORT_STALL: value k in 1 .. 2^22
 * makes the first tile of every radix-sort pass withhold its published digit counts and
 * gives each tile's look-back wait a budget of k polls, so the next tile's wait runs out
 * and GRAVITY_E_TIMEOUT is latched (the order of that build is then wrong, every index
 * still in range, nothing faults); 0 restores normal sorting.
 * GRAVITY_DBGSET_MOMENTS_STALL: value k in 1 .. 2^18 keeps the moment pass from counting
 * the nodes of the deepest internal depth and gives each of its waits (an internal depth
 * waits for the deeper ones) a budget of k polls, so the next depth's wait runs out and
 * GRAVITY_E_TIMEOUT is latched (that build's moments may then be wrong; every index stays
 * in range, nothing faults); 0 restores the normal pass.  GRAVITY_E_ARG for an unknown
 * item or value. */
enum gravity_debug_setting {
  GRAVITY_DBGSET_STACK_CAP = 1,
  GRAVITY_DBGSET_SORT_STALL = 2,
  GRAVITY_DBGSET_MOMENTS_STALL = 3
};
int gravity_debug_set(gravity_ctx *ctx, int what, int64_t value);

/* Number of kernels this context has enqueued since it was created (host-side
 * counter, no synchronisation). */
int gravity_stats(gravity_ctx *ctx, int64_t *launches);

/* Measure the FP32 FMA throughput of the device: a grid of 8 blocks per SM runs
 * independent FFMA chains for `iters` x 16 rounds.  Synchronises.  *ms = kernel
 * time, *flops = achieved FLOP/s (2 per FMA).  Used as the measured ALU roofline. */
int gravity_probe_fp32(gravity_ctx *ctx, int64_t iters, double *ms, double *flops);

/* Static description of an error code. */
const char *gravity_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* GRAVITY_H */
