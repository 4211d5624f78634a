// C ABI of libgravity: context, scratch management, argument checks, status
// latching.  Declarations and their documentation are in include/gravity.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

struct gravity_ctx {
  grav::Ctx c;
  // gravity_forces_host_batch: a second context with its own tree and stream, created on
  // first use, that evaluates every other snapshot, so that one snapshot's build and the
  // start of its walk run while the other's walk finishes
  gravity_ctx *twin = nullptr;
  cudaStream_t twin_stream = nullptr;
};

namespace grav {

// A named range around each entry point, visible to a profiler (NVTX; no cost when none
// is attached).
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

// Largest body count: octree node indices (< 2n) must fit the walk's 25-bit fields.
constexpr int64_t kMaxBodies = (int64_t)1 << 24;

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return GRAVITY_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return GRAVITY_E_NOMEM;
  }
  return GRAVITY_E_CUDA;
}

// One step of leapfrog_step (the kernels it enqueues, in order): kick-drift, tree
// build at the new positions, walk with the closing kick fused (KDK) or plain (Euler).
int integrate_one(Ctx &c, int64_t n, double *pos, double *vel, const double *mass,
                  double *acc, double dt, double theta, double eps) {
  const bool kdk = c.params.scheme == 0;
  const double h_kick = kdk ? 0.5 * dt : dt;
  int r = launch_kick_drift(&c, n, pos, vel, acc, h_kick, dt);
  if (r) return r;
  c.n = n;
  if ((r = tree_build(&c, n, pos, mass))) return r;
  c.have_tree = true;
  return walk_forces(&c, theta, eps, acc, nullptr, kdk ? vel : nullptr, kdk ? h_kick : 0.0);
}

int ctx_malloc(Ctx *c, void **p, size_t bytes) {
  *p = nullptr;
  if (c->user_alloc) {
    if (c->user_alloc(p, bytes, c->alloc_user) != 0 || !*p) {
      *p = nullptr;
      return GRAVITY_E_NOMEM;
    }
    return GRAVITY_OK;
  }
  return cuda_status(cudaMalloc(p, bytes));
}

void ctx_free(Ctx *c, void *p) {
  if (!p) return;
  // the captured leapfrog step may hold this buffer's address: drop it, so that the next
  // step runs eagerly and captures again on the buffers then current
  if (c->graph.exec) {
    cudaGraphExecDestroy(c->graph.exec);
    c->graph = StepGraph{};
  }
  if (c->user_free) c->user_free(p, c->alloc_user);
  else cudaFree(p);
}

namespace {

void free_tree(Ctx *c) {
  Tree &t = c->t;
  ctx_release(c, t.keys); ctx_release(c, t.keys_alt); ctx_release(c, t.idx);
  ctx_release(c, t.idx_alt); ctx_release(c, t.hist);
  ctx_release(c, t.bbox_part); ctx_release(c, t.pos_s); ctx_release(c, t.mass_s);
  ctx_release(c, t.body_hi); ctx_release(c, t.body_lo); ctx_release(c, t.bchild);
  ctx_release(c, t.bparent); ctx_release(c, t.bfirst); ctx_release(c, t.blast);
  ctx_release(c, t.bplen); ctx_release(c, t.bnchild); ctx_release(c, t.bbase);
  ctx_release(c, t.topo); ctx_release(c, t.nparent); ctx_release(c, t.ndepth);
  ctx_release(c, t.nlist); ctx_release(c, t.nmass); ctx_release(c, t.ncom);
  ctx_release(c, t.nquad); ctx_release(c, t.nrec0); ctx_release(c, t.nrec1);
  ctx_release(c, t.nquadf);
}

int check_params(const gravity_params *p) {
  if (!p) return GRAVITY_OK;
  if (!std::isfinite(p->G)) return GRAVITY_E_ARG;
  if (p->order != 0 && p->order != 2) return GRAVITY_E_ARG;
  if (p->leaf_max < 1 || p->leaf_max > kMaxLeaf) return GRAVITY_E_ARG;
  if (p->accum != 0 && p->accum != 1) return GRAVITY_E_ARG;
  if (p->mac_guard != 0 && p->mac_guard != 1) return GRAVITY_E_ARG;
  if (p->scheme != 0 && p->scheme != 1) return GRAVITY_E_ARG;
  if (p->use_graph != 0 && p->use_graph != 1) return GRAVITY_E_ARG;
  if (p->grav_every < 0) return GRAVITY_E_ARG;
  return GRAVITY_OK;
}

int set_device(const Ctx &c) { return cuda_status(cudaSetDevice(c.device)); }

}  // namespace

int ensure_capacity(Ctx *c, int64_t n) {
  if (n <= c->cap) return GRAVITY_OK;
  GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
  Tree &t = c->t;
  free_tree(c);
  c->cap = 0;
  int64_t cap = n + n / 8;
  if (cap < 1024) cap = 1024;
  if (cap > kMaxBodies) cap = kMaxBodies;
  const int64_t nodes = 2 * cap;
  int rc = GRAVITY_OK;
#define GRAV_ALLOC(p, cnt) if (rc == GRAVITY_OK) rc = ctx_alloc(c, p, cnt)
  GRAV_ALLOC(t.keys, cap); GRAV_ALLOC(t.keys_alt, cap);
  GRAV_ALLOC(t.idx, cap); GRAV_ALLOC(t.idx_alt, cap);
  GRAV_ALLOC(t.hist, radix_hist_words(cap));         // radix sort: counts + tile states
  GRAV_ALLOC(t.bbox_part, 6 * (4 * (int64_t)c->num_sms + 3));
  GRAV_ALLOC(t.pos_s, 3 * cap); GRAV_ALLOC(t.mass_s, cap);
  GRAV_ALLOC(t.body_hi, cap); GRAV_ALLOC(t.body_lo, cap);
  GRAV_ALLOC(t.bchild, 2 * cap); GRAV_ALLOC(t.bparent, cap); GRAV_ALLOC(t.bfirst, cap);
  GRAV_ALLOC(t.blast, cap); GRAV_ALLOC(t.bplen, cap); GRAV_ALLOC(t.bnchild, cap);
  GRAV_ALLOC(t.bbase, cap);
  GRAV_ALLOC(t.topo, nodes); GRAV_ALLOC(t.nparent, nodes); GRAV_ALLOC(t.ndepth, nodes);
  GRAV_ALLOC(t.nlist, nodes);
  GRAV_ALLOC(t.nmass, nodes); GRAV_ALLOC(t.ncom, 3 * nodes); GRAV_ALLOC(t.nquad, 3 * nodes);
  GRAV_ALLOC(t.nrec0, nodes); GRAV_ALLOC(t.nrec1, nodes); GRAV_ALLOC(t.nquadf, 2 * nodes);
#undef GRAV_ALLOC
  if (rc != GRAVITY_OK) {
    free_tree(c);
    return rc;
  }
  c->cap = cap;
  return GRAVITY_OK;
}

namespace {
void free_segments(Ctx *c) {
  Segs &sg = c->seg;
  ctx_release(c, sg.off); ctx_release(c, sg.seg_of); ctx_release(c, sg.seg_sorted);
  ctx_release(c, sg.task_begin); ctx_release(c, sg.task_end); ctx_release(c, sg.task_seg);
  sg = Segs{};
}
}  // namespace

// Clouds given by host offsets off[0..nseg] (off[0] = 0, strictly increasing).
// nseg <= 1 returns to a single cloud.  Builds the per-body cloud ids, the walk
// task list (32 consecutive bodies of one cloud per task) and the geometry array.
int set_segments(Ctx *c, int nseg, const int64_t *off) {
  GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
  free_segments(c);
  if (nseg <= 1) return GRAVITY_OK;
  if (!off || off[0] != 0 || nseg > 65536) return GRAVITY_E_ARG;
  for (int k = 0; k < nseg; ++k)
    if (off[k + 1] <= off[k]) return GRAVITY_E_ARG;
  const int64_t n = off[nseg];
  if (n > kMaxBodies) return GRAVITY_E_ARG;
  Segs &sg = c->seg;
  sg.nseg = nseg;
  sg.cbits = 0;
  while ((1 << sg.cbits) < nseg) ++sg.cbits;
  sg.n = n;
  std::vector<int32_t> tb, te, ts;
  for (int k = 0; k < nseg; ++k)
    for (int64_t b = off[k]; b < off[k + 1]; b += 32) {
      tb.push_back((int32_t)b);
      te.push_back((int32_t)off[k + 1]);
      ts.push_back(k);
    }
  sg.ntasks = (int)tb.size();
  sg.h_task_begin = tb;
  sg.h_task_end = te;
  int rc = GRAVITY_OK;
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, sg.off, nseg + 1);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, sg.seg_of, n);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, sg.seg_sorted, n);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, sg.task_begin, sg.ntasks);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, sg.task_end, sg.ntasks);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, sg.task_seg, sg.ntasks);
  if (rc == GRAVITY_OK)
    rc = cuda_status(cudaMemcpy(sg.off, off, sizeof(int64_t) * (nseg + 1), cudaMemcpyHostToDevice));
  if (rc == GRAVITY_OK)
    rc = cuda_status(cudaMemcpy(sg.task_begin, tb.data(), sizeof(int32_t) * sg.ntasks, cudaMemcpyHostToDevice));
  if (rc == GRAVITY_OK)
    rc = cuda_status(cudaMemcpy(sg.task_end, te.data(), sizeof(int32_t) * sg.ntasks, cudaMemcpyHostToDevice));
  if (rc == GRAVITY_OK)
    rc = cuda_status(cudaMemcpy(sg.task_seg, ts.data(), sizeof(int32_t) * sg.ntasks, cudaMemcpyHostToDevice));
  if (rc == GRAVITY_OK && c->t.geom_cap < nseg) {
    double *g = nullptr;
    rc = ctx_alloc(c, g, 8 * (int64_t)nseg);
    if (rc == GRAVITY_OK) {
      ctx_release(c, c->t.geom);
      c->t.geom = g;
      c->t.geom_cap = nseg;
    }
  }
  if (rc != GRAVITY_OK) { free_segments(c); return rc; }
  return fill_segment_ids(c);
}

// A saved copy of the tree arrays the vector-Jacobian product reads (the adjoint
// keeps one per recomputed level instead of building the tree again in reverse).
struct TreeSlot {
  size_t bhi, blo, pos, mass, idx, topo, rec0, rec1, depth, parent, nmass, ncom, geom, nnodes;
  size_t bytes;
};

TreeSlot tree_slot_layout(int64_t n, int ngeom) {
  TreeSlot L{};
  size_t o = 0;
  auto take = [&](size_t b) { const size_t r = o; o += (b + 255) & ~(size_t)255; return r; };
  const size_t nodes = 2 * (size_t)n;
  L.bhi = take(sizeof(float4) * n); L.blo = take(sizeof(float4) * n);
  L.pos = take(sizeof(double) * 3 * n); L.mass = take(sizeof(double) * n);
  L.idx = take(sizeof(uint32_t) * n);
  L.topo = take(sizeof(int4) * nodes); L.rec0 = take(sizeof(float4) * nodes);
  L.rec1 = take(sizeof(float4) * nodes); L.depth = take(sizeof(int32_t) * nodes);
  L.parent = take(sizeof(int32_t) * nodes); L.nmass = take(sizeof(double) * nodes);
  L.ncom = take(sizeof(double) * 3 * nodes); L.geom = take(sizeof(double) * 8 * ngeom);
  L.nnodes = take(sizeof(int32_t));
  L.bytes = o;
  return L;
}

Tree tree_slot_view(unsigned char *b, const TreeSlot &L) {
  Tree v{};
  v.body_hi = reinterpret_cast<float4 *>(b + L.bhi);
  v.body_lo = reinterpret_cast<float4 *>(b + L.blo);
  v.pos_s = reinterpret_cast<double *>(b + L.pos);
  v.mass_s = reinterpret_cast<double *>(b + L.mass);
  v.idx = reinterpret_cast<uint32_t *>(b + L.idx);
  v.topo = reinterpret_cast<int4 *>(b + L.topo);
  v.nrec0 = reinterpret_cast<float4 *>(b + L.rec0);
  v.nrec1 = reinterpret_cast<float4 *>(b + L.rec1);
  v.ndepth = reinterpret_cast<int32_t *>(b + L.depth);
  v.nparent = reinterpret_cast<int32_t *>(b + L.parent);
  v.nmass = reinterpret_cast<double *>(b + L.nmass);
  v.ncom = reinterpret_cast<double *>(b + L.ncom);
  v.geom = reinterpret_cast<double *>(b + L.geom);
  v.nnodes = reinterpret_cast<int32_t *>(b + L.nnodes);
  return v;
}

int tree_slot_save(Ctx *c, unsigned char *b, const TreeSlot &L, int64_t n, int ngeom) {
  const Tree v = tree_slot_view(b, L);
  const Tree &t = c->t;
  const size_t nodes = 2 * (size_t)n;
  struct { void *dst; const void *src; size_t bytes; } cp[] = {
      {v.body_hi, t.body_hi, sizeof(float4) * n}, {v.body_lo, t.body_lo, sizeof(float4) * n},
      {v.pos_s, t.pos_s, sizeof(double) * 3 * n}, {v.mass_s, t.mass_s, sizeof(double) * n},
      {v.idx, t.idx, sizeof(uint32_t) * n}, {v.topo, t.topo, sizeof(int4) * nodes},
      {v.nrec0, t.nrec0, sizeof(float4) * nodes}, {v.nrec1, t.nrec1, sizeof(float4) * nodes},
      {v.ndepth, t.ndepth, sizeof(int32_t) * nodes}, {v.nparent, t.nparent, sizeof(int32_t) * nodes},
      {v.nmass, t.nmass, sizeof(double) * nodes}, {v.ncom, t.ncom, sizeof(double) * 3 * nodes},
      {v.geom, t.geom, sizeof(double) * 8 * ngeom}, {v.nnodes, t.nnodes, sizeof(int32_t)}};
  for (const auto &e : cp)
    GRAV_CUDA_TRY(cudaMemcpyAsync(e.dst, e.src, e.bytes, cudaMemcpyDeviceToDevice, c->stream));
  return GRAVITY_OK;
}

// The small fixed buffers every context holds (status word, one cloud's geometry,
// counters); and the release of everything the context owns.
int alloc_base(Ctx *c) {
  int rc = GRAVITY_OK;
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->d_status, 1);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->t.geom, 8);
  if (rc == GRAVITY_OK) c->t.geom_cap = 1;
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->t.bbox_ticket, 1);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->t.nnodes, 1);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->t.scalars, grav::kScalarWords);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->walk_stats, 16);
  if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->walk_queues, c->num_sms + 1);
  if (rc == GRAVITY_OK) rc = cuda_status(cudaMemset(c->walk_stats, 0, 16 * sizeof(unsigned long long)));
  if (rc == GRAVITY_OK) rc = cuda_status(cudaMemset(c->d_status, 0, sizeof(unsigned)));
  if (rc == GRAVITY_OK) rc = cuda_status(cudaMemset(c->t.bbox_ticket, 0, sizeof(unsigned)));
  if (rc == GRAVITY_OK) rc = cuda_status(cudaMemset(c->t.nnodes, 0, sizeof(int32_t)));
  return rc;
}

void free_all(Ctx *c) {
  free_tree(c);
  free_segments(c);
  c->cap = 0;
  c->n = 0;
  c->have_tree = false;
  ctx_release(c, c->t.geom); c->t.geom_cap = 0;
  ctx_release(c, c->t.bbox_ticket); ctx_release(c, c->t.nnodes); ctx_release(c, c->t.scalars);
  ctx_release(c, c->walk_stats); ctx_release(c, c->walk_queues);
  ctx_release(c, c->walk_gstack); c->walk_gstack_cap = 0;
  ctx_release(c, c->walk_part); c->walk_part_cap = 0;
  ctx_release(c, c->walk_cost); ctx_release(c, c->walk_order);
  c->walk_order_cap = 0; c->walk_order_n = 0; c->walk_order_nq = 0;
  ctx_release(c, c->vjp_own); ctx_release(c, c->vjp_body); ctx_release(c, c->vjp_node);
  c->vjp_cap = 0;
  ctx_release(c, c->adj_levels); ctx_release(c, c->adj_work);
  c->adj_levels_cap = c->adj_work_cap = 0;
  ctx_release(c, c->adj_bank); c->adj_bank_cap = 0;
  ctx_release(c, c->dir_hi); ctx_release(c, c->dir_lo); c->dir_cap = 0;
  ctx_release(c, c->ds_keys); ctx_release(c, c->ds_keys_alt); ctx_release(c, c->ds_idx);
  ctx_release(c, c->ds_idx_alt); ctx_release(c, c->ds_hist); ctx_release(c, c->ds_geom);
  ctx_release(c, c->ds_part); ctx_release(c, c->ds_ticket); ctx_release(c, c->ds_hi);
  ctx_release(c, c->ds_lo); ctx_release(c, c->ds_box); c->ds_cap = 0;
  ctx_release(c, c->diag_buf); c->diag_cap = 0;
  ctx_release(c, c->h2d_pos); ctx_release(c, c->h2d_mass); ctx_release(c, c->h2d_acc);
  c->h2d_cap = 0;
  for (int k = 0; k < 2; ++k) {
    ctx_release(c, c->bat_pos[k]); ctx_release(c, c->bat_mass[k]); ctx_release(c, c->bat_acc[k]);
    cudaEvent_t *ev[4] = {&c->ev_in[k], &c->ev_built[k], &c->ev_walked[k], &c->ev_out[k]};
    for (cudaEvent_t *e : ev)
      if (*e) { cudaEventDestroy(*e); *e = nullptr; }
  }
  c->bat_cap = 0;
  if (c->h2d_stream) { cudaStreamDestroy(c->h2d_stream); c->h2d_stream = nullptr; }
  if (c->d2h_stream) { cudaStreamDestroy(c->d2h_stream); c->d2h_stream = nullptr; }
  ctx_release(c, c->comp_r); ctx_release(c, c->comp_i); c->comp_cap = 0;
  if (c->graph.exec) cudaGraphExecDestroy(c->graph.exec);
  c->graph = StepGraph{};
  ctx_release(c, c->d_status);
}

}  // namespace grav

using grav::Ctx;

extern "C" {

void gravity_params_default(gravity_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->G = 1.0;
  p->order = 0;
  p->leaf_max = 1;
  p->accum = 0;
  p->mac_guard = 1;
  p->scheme = 0;
  p->walk_cfg = -1;
  p->use_graph = 1;
  p->grav_every = 1;
}

int gravity_create(gravity_ctx **out, int device, void *cuda_stream) {
  if (!out) return GRAVITY_E_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) { cudaGetLastError(); return GRAVITY_E_CUDA; }
  if (device < 0 || device >= ndev) return GRAVITY_E_ARG;
  gravity_ctx *h = new (std::nothrow) gravity_ctx();
  if (!h) return GRAVITY_E_NOMEM;
  Ctx &c = h->c;
  c.device = device;
  c.stream = static_cast<cudaStream_t>(cuda_stream);
  gravity_params_default(&c.params);
  int rc = grav::set_device(c);
  if (rc == GRAVITY_OK) rc = grav::cuda_status(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, device));
  if (rc == GRAVITY_OK) rc = grav::alloc_base(&c);
  if (rc != GRAVITY_OK) {
    gravity_destroy(h);
    return rc;
  }
  *out = h;
  return GRAVITY_OK;
}

static void drop_twin(gravity_ctx *h) {
  if (h->twin) {
    gravity_destroy(h->twin);
    h->twin = nullptr;
  }
  if (h->twin_stream) {
    cudaStreamDestroy(h->twin_stream);
    h->twin_stream = nullptr;
  }
}

int gravity_destroy(gravity_ctx *h) {
  if (!h) return GRAVITY_OK;
  Ctx &c = h->c;
  cudaSetDevice(c.device);
  drop_twin(h);
  cudaStreamSynchronize(c.stream);
  grav::free_all(&c);
  cudaGetLastError();
  delete h;
  return GRAVITY_OK;
}

int gravity_set_allocator(gravity_ctx *h, gravity_alloc_fn alloc, gravity_free_fn release,
                          void *user) {
  if (!h || (alloc == nullptr) != (release == nullptr)) return GRAVITY_E_ARG;
  Ctx &c = h->c;
  int rc = grav::set_device(c);
  if (rc) return rc;
  GRAV_CUDA_TRY(cudaStreamSynchronize(c.stream));
  drop_twin(h);                             // made again, on the new allocator, when needed
  grav::free_all(&c);                       // with the allocator that made each buffer
  const gravity_alloc_fn old_alloc = c.user_alloc;
  const gravity_free_fn old_free = c.user_free;
  void *const old_user = c.alloc_user;
  c.user_alloc = alloc;
  c.user_free = release;
  c.alloc_user = user;
  rc = grav::alloc_base(&c);
  if (rc != GRAVITY_OK) {                   // keep a usable context on the previous allocator
    grav::free_all(&c);
    c.user_alloc = old_alloc;
    c.user_free = old_free;
    c.alloc_user = old_user;
    const int rc2 = grav::alloc_base(&c);
    return rc2 != GRAVITY_OK ? rc2 : rc;
  }
  return GRAVITY_OK;
}

int gravity_debug_set(gravity_ctx *h, int what, int64_t value) {
  if (!h) return GRAVITY_E_ARG;
  switch (what) {
    case GRAVITY_DBGSET_STACK_CAP:
      if (value < 0 || value > grav::walk_stack_capacity()) return GRAVITY_E_ARG;
      h->c.stack_cap = (int)value;
      return GRAVITY_OK;
    case GRAVITY_DBGSET_SORT_STALL:
      if (value < 0 || value > (1 << 22)) return GRAVITY_E_ARG;
      h->c.sort_stall = (int)value;
      return GRAVITY_OK;
    case GRAVITY_DBGSET_MOMENTS_STALL:
      if (value < 0 || value > (1 << 18)) return GRAVITY_E_ARG;
      h->c.moments_stall = (int)value;
      return GRAVITY_OK;
    default:
      return GRAVITY_E_ARG;
  }
}

int gravity_set_stream(gravity_ctx *h, void *cuda_stream) {
  if (!h) return GRAVITY_E_ARG;
  h->c.stream = static_cast<cudaStream_t>(cuda_stream);
  return GRAVITY_OK;
}

int gravity_tree_build(gravity_ctx *h, int64_t n, const double *pos, const double *mass,
                       const gravity_params *p) {
  grav::Range range_("gravity_tree_build");
  if (!h || n < 0 || n > grav::kMaxBodies) return GRAVITY_E_ARG;
  if (n > 0 && (!pos || !mass)) return GRAVITY_E_ARG;
  int rc = grav::check_params(p);
  if (rc) return rc;
  Ctx &c = h->c;
  if (c.seg.nseg > 1 && n != c.seg.n) return GRAVITY_E_ARG;
  if (p) c.params = *p; else gravity_params_default(&c.params);
  c.have_tree = false;
  c.grav_since = 0;
  c.n = n;
  if (n == 0) { c.have_tree = true; return GRAVITY_OK; }
  if ((rc = grav::set_device(c))) return rc;
  if ((rc = grav::ensure_capacity(&c, n))) return rc;
  if ((rc = grav::tree_build(&c, n, pos, mass))) return rc;
  c.have_tree = true;
  return GRAVITY_OK;
}

static int forces_common(gravity_ctx *h, double theta, double eps, double *acc, int32_t *counts) {
  grav::Range range_("gravity_forces");
  if (!h || !(theta >= 0.0) || !(eps >= 0.0) || !std::isfinite(theta) || !std::isfinite(eps))
    return GRAVITY_E_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return GRAVITY_E_NOTREE;
  if (c.n == 0) return GRAVITY_OK;
  if (!acc) return GRAVITY_E_ARG;
  int rc = grav::set_device(c);
  if (rc) return rc;
  c.grav_since = 0;
  return grav::walk_forces(&c, theta, eps, acc, counts, nullptr, 0.0);
}

int gravity_forces(gravity_ctx *h, double theta, double eps, double *acc) {
  return forces_common(h, theta, eps, acc, nullptr);
}

int gravity_forces_counted(gravity_ctx *h, double theta, double eps, double *acc,
                           int32_t *counts) {
  if (h && h->c.n > 0 && !counts) return GRAVITY_E_ARG;
  return forces_common(h, theta, eps, acc, counts);
}

int gravity_walk_tasks(gravity_ctx *h, int64_t *ntasks) {
  if (!h || !ntasks) return GRAVITY_E_ARG;
  if (!h->c.have_tree) return GRAVITY_E_NOTREE;
  *ntasks = grav::walk_task_count(&h->c);
  return GRAVITY_OK;
}

namespace grav {
namespace {
// Sorted-order bodies [*b0, *b0 + *nb) of walk tasks [first, first + count) of the tree.
int task_bodies(const Ctx &c, int64_t first, int64_t count, int64_t *b0, int64_t *nb) {
  const int64_t total = walk_task_count(&c);
  if (first < 0 || count < 0 || first + count > total) return GRAVITY_E_ARG;
  if (count == 0) { *b0 = 0; *nb = 0; return GRAVITY_OK; }
  if (c.seg.nseg > 1) {
    const int64_t last = first + count - 1;
    const int64_t beg = c.seg.h_task_begin[(size_t)first];
    const int64_t end = std::min<int64_t>(c.seg.h_task_begin[(size_t)last] + 32,
                                          c.seg.h_task_end[(size_t)last]);
    *b0 = beg;
    *nb = end - beg;
  } else {
    *b0 = 32 * first;
    *nb = std::min<int64_t>(32 * (first + count), c.n) - 32 * first;
  }
  return GRAVITY_OK;
}
}  // namespace
}  // namespace grav

int gravity_task_bodies(gravity_ctx *h, int64_t first_task, int64_t ntasks, int64_t *first_body,
                        int64_t *nbodies) {
  if (!h || !first_body || !nbodies) return GRAVITY_E_ARG;
  if (!h->c.have_tree) return GRAVITY_E_NOTREE;
  return grav::task_bodies(h->c, first_task, ntasks, first_body, nbodies);
}

int gravity_forces_range(gravity_ctx *h, double theta, double eps, int64_t first_task,
                         int64_t ntasks, double *acc_sorted) {
  grav::Range range_("gravity_forces_range");
  if (!h || !(theta >= 0.0) || !(eps >= 0.0) || !std::isfinite(theta) || !std::isfinite(eps))
    return GRAVITY_E_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return GRAVITY_E_NOTREE;
  int64_t b0 = 0, nb = 0;
  int rc = grav::task_bodies(c, first_task, ntasks, &b0, &nb);
  if (rc) return rc;
  if (nb == 0) return GRAVITY_OK;
  if (!acc_sorted) return GRAVITY_E_ARG;
  if ((rc = grav::set_device(c))) return rc;
  return grav::walk_forces_range(&c, theta, eps, first_task, ntasks, b0, nb, acc_sorted);
}

int gravity_scatter_sorted(gravity_ctx *h, int64_t first_body, int64_t nbodies,
                           const double *src_sorted, double *dst) {
  if (!h) return GRAVITY_E_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return GRAVITY_E_NOTREE;
  if (first_body < 0 || nbodies < 0 || first_body + nbodies > c.n) return GRAVITY_E_ARG;
  if (nbodies == 0) return GRAVITY_OK;
  if (!src_sorted || !dst) return GRAVITY_E_ARG;
  int rc = grav::set_device(c);
  if (rc) return rc;
  return grav::launch_scatter_sorted(&c, first_body, nbodies, src_sorted, dst);
}

int gravity_kick_drift(gravity_ctx *h, int64_t n, double *pos, double *vel, const double *acc,
                       double h_kick, double dt) {
  if (!h || n < 0 || !std::isfinite(h_kick) || !std::isfinite(dt)) return GRAVITY_E_ARG;
  if (n == 0) return GRAVITY_OK;
  if (!pos || !vel || !acc) return GRAVITY_E_ARG;
  int rc = grav::set_device(h->c);
  if (rc) return rc;
  return grav::launch_kick_drift(&h->c, n, pos, vel, acc, h_kick, dt);
}

int gravity_kick(gravity_ctx *h, int64_t n, double *vel, const double *acc, double h_kick) {
  if (!h || n < 0 || !std::isfinite(h_kick)) return GRAVITY_E_ARG;
  if (n == 0) return GRAVITY_OK;
  if (!vel || !acc) return GRAVITY_E_ARG;
  int rc = grav::set_device(h->c);
  if (rc) return rc;
  return grav::launch_kick(&h->c, n, vel, acc, h_kick);
}

int gravity_forces_vjp(gravity_ctx *h, double theta, double eps, const double *lambda,
                       double *grad_pos) {
  grav::Range range_("gravity_forces_vjp");
  if (!h || !(theta >= 0.0) || !(eps >= 0.0) || !std::isfinite(theta) || !std::isfinite(eps))
    return GRAVITY_E_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return GRAVITY_E_NOTREE;
  if (c.params.order != 0) return GRAVITY_E_ARG;
  if (c.n == 0) return GRAVITY_OK;
  if (!lambda || !grad_pos) return GRAVITY_E_ARG;
  int rc = grav::set_device(c);
  if (rc) return rc;
  return grav::walk_vjp(&c, theta, eps, lambda, grad_pos);
}

int gravity_components(gravity_ctx *h, const double *radius, double dmax, int32_t *label,
                       int64_t *counts) {
  grav::Range range_("gravity_components");
  if (!h) return GRAVITY_E_ARG;
  if (!radius && (!(dmax >= 0.0) || !std::isfinite(dmax))) return GRAVITY_E_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return GRAVITY_E_NOTREE;
  if (c.n > 0 && !label) return GRAVITY_E_ARG;
  int rc = grav::set_device(c);
  if (rc) return rc;
  if (c.n == 0) {
    if (counts) GRAV_CUDA_TRY(cudaMemsetAsync(counts, 0, 2 * sizeof(int64_t), c.stream));
    return GRAVITY_OK;
  }
  return grav::components(&c, radius, dmax, label, counts);
}

int gravity_dt_g(double G, double rho, double *dt_g) {
  if (!dt_g || !(G > 0.0) || !(rho > 0.0) || !std::isfinite(G) || !std::isfinite(rho))
    return GRAVITY_E_ARG;
  *dt_g = 0.5 / std::sqrt(G * rho);
  return GRAVITY_OK;
}

int gravity_direct(gravity_ctx *h, int64_t n, const double *pos, const double *mass, double eps,
                   double G, double *acc) {
  grav::Range range_("gravity_direct");
  if (!h || n < 0 || !(eps >= 0.0) || !std::isfinite(eps) || !std::isfinite(G))
    return GRAVITY_E_ARG;
  if (n == 0) return GRAVITY_OK;
  if (!pos || !mass || !acc) return GRAVITY_E_ARG;
  int rc = grav::set_device(h->c);
  if (rc) return rc;
  return grav::direct_forces(&h->c, n, pos, mass, eps, G, acc);
}

int gravity_diagnostics(gravity_ctx *h, int64_t n, const double *pos, const double *vel,
                        const double *mass, double eps, double G, double *out) {
  grav::Range range_("gravity_diagnostics");
  if (!h || n < 0 || !(eps >= 0.0) || !std::isfinite(eps) || !std::isfinite(G) || !out)
    return GRAVITY_E_ARG;
  if (n > 0 && (!pos || !vel || !mass)) return GRAVITY_E_ARG;
  Ctx &c = h->c;
  int rc = grav::set_device(c);
  if (rc) return rc;
  if (n == 0) {
    GRAV_CUDA_TRY(cudaMemsetAsync(out, 0, 7 * sizeof(double), c.stream));
    return GRAVITY_OK;
  }
  return grav::diagnostics(&c, n, pos, vel, mass, eps, G, out);
}

int leapfrog_step(gravity_ctx *h, int64_t n, double *pos, double *vel, const double *mass,
                  double *acc_cache, double dt, int nsteps, double theta, double eps,
                  const gravity_params *p) {
  grav::Range range_("leapfrog_step");
  if (!h || n < 0 || n > grav::kMaxBodies || nsteps < 0 || !std::isfinite(dt)) return GRAVITY_E_ARG;
  if (!(theta >= 0.0) || !(eps >= 0.0) || !std::isfinite(theta) || !std::isfinite(eps))
    return GRAVITY_E_ARG;
  int rc = grav::check_params(p);
  if (rc) return rc;
  if (n == 0 || nsteps == 0) return GRAVITY_OK;
  if (!pos || !vel || !mass || !acc_cache) return GRAVITY_E_ARG;
  Ctx &c = h->c;
  if (c.seg.nseg > 1 && n != c.seg.n) return GRAVITY_E_ARG;
  if (p) c.params = *p; else gravity_params_default(&c.params);
  if ((rc = grav::set_device(c))) return rc;
  if ((rc = grav::ensure_capacity(&c, n))) return rc;
  auto one_step = [&]() -> int {
    return grav::integrate_one(c, n, pos, vel, mass, acc_cache, dt, theta, eps);
  };
  if (c.params.grav_every > 1) {
    // two time steps (Sec. 4.1): kick-drift every step, gravity (build + walk, with the
    // closing kick fused for KDK) every grav_every-th step, the held acceleration in between
    const bool kdk = c.params.scheme == 0;
    const double hk = kdk ? 0.5 * dt : dt;
    for (int s = 0; s < nsteps; ++s) {
      if ((rc = grav::launch_kick_drift(&c, n, pos, vel, acc_cache, hk, dt))) return rc;
      if (++c.grav_since >= c.params.grav_every) {
        c.grav_since = 0;
        c.n = n;
        if ((rc = grav::tree_build(&c, n, pos, mass))) return rc;
        c.have_tree = true;
        if ((rc = grav::walk_forces(&c, theta, eps, acc_cache, nullptr, kdk ? vel : nullptr,
                                    kdk ? hk : 0.0)))
          return rc;
      } else if (kdk && (rc = grav::launch_kick(&c, n, vel, acc_cache, hk))) {
        return rc;
      }
    }
    return GRAVITY_OK;
  }
  // The first step runs eagerly (it sizes every buffer); later steps replay a
  // CUDA graph of one step captured on the caller's stream when graphs are enabled.
  grav::StepGraph &g = c.graph;
  const bool same = g.exec && g.stream == c.stream && g.n == n && g.pos == pos && g.vel == vel &&
                    g.mass == mass && g.acc == acc_cache && g.dt == dt && g.theta == theta &&
                    g.eps == eps && g.nseg == c.seg.nseg &&
                    std::memcmp(&g.params, &c.params, sizeof(gravity_params)) == 0;
  int s0 = 0;
  if (!same) {
    if ((rc = one_step())) return rc;
    s0 = 1;
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    if (c.params.use_graph && c.stream != nullptr && nsteps > 2) {
      cudaGraph_t graph = nullptr;
      const int64_t k0 = c.launches;
      if (cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        int rs = one_step();
        cudaError_t ec = cudaStreamEndCapture(c.stream, &graph);
        if (rs == GRAVITY_OK && ec == cudaSuccess && graph &&
            cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess) {
          g.stream = c.stream; g.n = n; g.pos = pos; g.vel = vel; g.mass = mass;
          g.acc = acc_cache; g.dt = dt; g.theta = theta; g.eps = eps; g.params = c.params;
          g.nseg = c.seg.nseg; g.kernels = c.launches - k0;
        } else {
          g.exec = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
        c.launches = k0;
      }
      cudaGetLastError();
    }
  }
  for (int s = s0; s < nsteps; ++s) {
    if (g.exec) {
      GRAV_CUDA_TRY(cudaGraphLaunch(g.exec, c.stream));
      c.launches += g.kernels;
    } else if ((rc = one_step())) {
      return rc;
    }
  }
  return GRAVITY_OK;
}

int leapfrog_adjoint(gravity_ctx *h, int64_t n, const double *pos0, const double *vel0,
                     const double *mass, double dt, int nsteps, double theta, double eps,
                     const gravity_params *p, int flags, double *xbar, double *vbar) {
  grav::Range range_("leapfrog_adjoint");
  if (!h || n < 0 || n > grav::kMaxBodies || nsteps < 0 || !std::isfinite(dt)) return GRAVITY_E_ARG;
  if (!(theta >= 0.0) || !(eps >= 0.0) || !std::isfinite(theta) || !std::isfinite(eps))
    return GRAVITY_E_ARG;
  if (flags & ~(GRAVITY_ADJ_END | GRAVITY_ADJ_START)) return GRAVITY_E_ARG;
  int rc = grav::check_params(p);
  if (rc) return rc;
  gravity_params q;
  if (p) q = *p; else gravity_params_default(&q);
  if (q.order != 0 || q.scheme != 0 || q.grav_every > 1) return GRAVITY_E_ARG;
  if (n == 0) return GRAVITY_OK;
  if (!pos0 || !vel0 || !mass || !xbar || !vbar) return GRAVITY_E_ARG;
  Ctx &c = h->c;
  if (c.seg.nseg > 1 && n != c.seg.n) return GRAVITY_E_ARG;
  c.params = q;
  if ((rc = grav::set_device(c))) return rc;
  if ((rc = grav::ensure_capacity(&c, n))) return rc;
  const int64_t n3 = 3 * n;
  const int64_t lev_need = n3 * (int64_t)(nsteps + 1);
  if (c.adj_levels_cap < lev_need || c.adj_work_cap < 3 * n3) {
    GRAV_CUDA_TRY(cudaStreamSynchronize(c.stream));
    if (c.adj_levels_cap < lev_need) {
      grav::ctx_release(&c, c.adj_levels);
      c.adj_levels_cap = 0;
      if ((rc = grav::ctx_alloc(&c, c.adj_levels, lev_need))) return rc;
      c.adj_levels_cap = lev_need;
    }
    if (c.adj_work_cap < 3 * n3) {
      grav::ctx_release(&c, c.adj_work);
      c.adj_work_cap = 0;
      if ((rc = grav::ctx_alloc(&c, c.adj_work, 3 * n3))) return rc;
      c.adj_work_cap = 3 * n3;
    }
  }
  double *vel = c.adj_work, *acc = c.adj_work + n3, *g = c.adj_work + 2 * n3;
  auto level = [&](int k) { return c.adj_levels + n3 * (int64_t)k; };
  const int last = (flags & GRAVITY_ADJ_END) ? nsteps : nsteps - 1;
  // keep each recomputed level's tree (the arrays the product reads) when that fits,
  // so the reverse pass needs no second build; else build again in reverse
  const int ngeom = c.seg.nseg > 1 ? c.seg.nseg : 1;
  const grav::TreeSlot L = grav::tree_slot_layout(n, ngeom);
  const size_t bank_need = L.bytes * (size_t)(last + 1);
  bool banked = false;
  if (bank_need <= ((size_t)64 << 30)) {
    if (c.adj_bank_cap >= bank_need) {
      banked = true;
    } else {
      GRAV_CUDA_TRY(cudaStreamSynchronize(c.stream));
      grav::ctx_release(&c, c.adj_bank);
      c.adj_bank_cap = 0;
      if (grav::ctx_alloc(&c, c.adj_bank, (int64_t)bank_need) == GRAVITY_OK) {
        c.adj_bank_cap = bank_need;
        banked = true;
      } else {
        cudaGetLastError();                  // not enough memory: rebuild in reverse
      }
    }
  }
  auto slot = [&](int k) { return c.adj_bank + L.bytes * (size_t)k; };
  // recompute the segment's levels from the checkpoint with the forward kernels
  GRAV_CUDA_TRY(cudaMemcpyAsync(level(0), pos0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
  GRAV_CUDA_TRY(cudaMemcpyAsync(vel, vel0, sizeof(double) * n3, cudaMemcpyDeviceToDevice, c.stream));
  c.n = n;
  if ((rc = grav::tree_build(&c, n, level(0), mass))) return rc;
  c.have_tree = true;
  if ((rc = grav::walk_forces(&c, theta, eps, acc, nullptr, nullptr, 0.0))) return rc;
  if (banked && (rc = grav::tree_slot_save(&c, slot(0), L, n, ngeom))) return rc;
  for (int k = 0; k < last; ++k) {
    GRAV_CUDA_TRY(cudaMemcpyAsync(level(k + 1), level(k), sizeof(double) * n3,
                                  cudaMemcpyDeviceToDevice, c.stream));
    if ((rc = grav::integrate_one(c, n, level(k + 1), vel, mass, acc, dt, theta, eps))) return rc;
    if (banked && (rc = grav::tree_slot_save(&c, slot(k + 1), L, n, ngeom))) return rc;
  }
  // reverse: level k takes xbar += c_k J(x_k)^T vbar, then the drift before it
  const double hk = 0.5 * dt;
  for (int k = last; k >= 0; --k) {
    const bool top = k == nsteps;                    // only with GRAVITY_ADJ_END
    const bool first = k == 0 && (flags & GRAVITY_ADJ_START);
    if (banked) {
      rc = grav::walk_vjp_tree(&c, grav::tree_slot_view(slot(k), L), theta, eps, vbar, g);
    } else {
      if (k != last) {                               // the tree is at level `last` already
        c.n = n;
        if ((rc = grav::tree_build(&c, n, level(k), mass))) return rc;
        c.have_tree = true;
      }
      rc = grav::walk_vjp(&c, theta, eps, vbar, g);
    }
    if (rc) return rc;
    const double coef = (top || first) ? hk : dt;
    if ((rc = grav::launch_adjoint_kick_drift(&c, n, xbar, vbar, g, coef, dt, !first))) return rc;
  }
  return GRAVITY_OK;
}

int gravity_set_clouds(gravity_ctx *h, int32_t nclouds, const int64_t *offsets_host) {
  grav::Range range_("gravity_set_clouds");
  if (!h || nclouds < 0) return GRAVITY_E_ARG;
  if (nclouds > 1 && !offsets_host) return GRAVITY_E_ARG;
  if (offsets_host && nclouds >= 1) {          // off[0] = 0, strictly increasing
    if (offsets_host[0] != 0) return GRAVITY_E_ARG;
    for (int32_t k = 0; k < nclouds; ++k)
      if (offsets_host[k + 1] <= offsets_host[k]) return GRAVITY_E_ARG;
  }
  int rc = grav::set_device(h->c);
  if (rc) return rc;
  h->c.have_tree = false;
  return grav::set_segments(&h->c, nclouds, offsets_host);
}

int gravity_batch_tree_build(gravity_ctx *h, int32_t nclouds, const int64_t *offsets_host,
                             const double *pos, const double *mass, const gravity_params *p) {
  if (!h || nclouds < 1 || !offsets_host) return GRAVITY_E_ARG;
  int rc = gravity_set_clouds(h, nclouds, offsets_host);
  if (rc) return rc;
  return gravity_tree_build(h, offsets_host[nclouds], pos, mass, p);
}

int gravity_sync(gravity_ctx *h) {
  if (!h) return GRAVITY_E_ARG;
  Ctx &c = h->c;
  int rc = grav::set_device(c);
  if (rc) return rc;
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return grav::cuda_status(e);
  unsigned st = 0;
  e = cudaMemcpy(&st, c.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return grav::cuda_status(e);
  if (st) {
    e = cudaMemset(c.d_status, 0, sizeof(unsigned));
    if (e != cudaSuccess) return grav::cuda_status(e);
  }
  if (st & grav::kErrNonFinite) return GRAVITY_E_NONFINITE;
  if (st & grav::kErrTimeout) return GRAVITY_E_TIMEOUT;
  if (st & (grav::kErrStack | grav::kErrTree)) return GRAVITY_E_INTERNAL;
  return GRAVITY_OK;
}

int gravity_forces_host(gravity_ctx *h, int64_t n, const double *pos_host, const double *mass_host,
                        double theta, double eps, const gravity_params *p, double *acc_host) {
  grav::Range range_("gravity_forces_host");
  if (!h || n < 0 || n > grav::kMaxBodies) return GRAVITY_E_ARG;
  if (n > 0 && (!pos_host || !mass_host || !acc_host)) return GRAVITY_E_ARG;
  if (!(theta >= 0.0) || !(eps >= 0.0) || !std::isfinite(theta) || !std::isfinite(eps))
    return GRAVITY_E_ARG;
  int rc = grav::check_params(p);
  if (rc) return rc;
  Ctx &c = h->c;
  if ((rc = grav::set_device(c))) return rc;
  if (n > c.h2d_cap) {
    GRAV_CUDA_TRY(cudaStreamSynchronize(c.stream));
    grav::ctx_release(&c, c.h2d_pos); grav::ctx_release(&c, c.h2d_mass);
    grav::ctx_release(&c, c.h2d_acc);
    c.h2d_cap = 0;
    if ((rc = grav::ctx_alloc(&c, c.h2d_pos, 3 * n))) return rc;
    if ((rc = grav::ctx_alloc(&c, c.h2d_mass, n))) return rc;
    if ((rc = grav::ctx_alloc(&c, c.h2d_acc, 3 * n))) return rc;
    c.h2d_cap = n;
  }
  if (n > 0) {
    GRAV_CUDA_TRY(cudaMemcpyAsync(c.h2d_pos, pos_host, sizeof(double) * 3 * n,
                                  cudaMemcpyHostToDevice, c.stream));
    GRAV_CUDA_TRY(cudaMemcpyAsync(c.h2d_mass, mass_host, sizeof(double) * n,
                                  cudaMemcpyHostToDevice, c.stream));
  }
  if ((rc = gravity_tree_build(h, n, c.h2d_pos, c.h2d_mass, p))) return rc;
  if ((rc = gravity_forces(h, theta, eps, c.h2d_acc))) return rc;
  if (n > 0)
    GRAV_CUDA_TRY(cudaMemcpyAsync(acc_host, c.h2d_acc, sizeof(double) * 3 * n,
                                  cudaMemcpyDeviceToHost, c.stream));
  return gravity_sync(h);
}

int gravity_forces_host_batch(gravity_ctx *h, int64_t nsnap, int64_t n,
                              const double *const *pos_host, const double *const *mass_host,
                              double theta, double eps, const gravity_params *p,
                              double *const *acc_host) {
  grav::Range range_("gravity_forces_host_batch");
  if (!h || nsnap < 0 || n < 0 || n > grav::kMaxBodies) return GRAVITY_E_ARG;
  if (nsnap > 0 && (!pos_host || !mass_host || !acc_host)) return GRAVITY_E_ARG;
  for (int64_t k = 0; k < nsnap && n > 0; ++k)
    if (!pos_host[k] || !mass_host[k] || !acc_host[k]) return GRAVITY_E_ARG;
  if (!(theta >= 0.0) || !(eps >= 0.0) || !std::isfinite(theta) || !std::isfinite(eps))
    return GRAVITY_E_ARG;
  int rc = grav::check_params(p);
  if (rc) return rc;
  Ctx &c = h->c;
  if ((rc = grav::set_device(c))) return rc;
  if (nsnap == 0) return GRAVITY_OK;
  if (!c.h2d_stream) {
    GRAV_CUDA_TRY(cudaStreamCreateWithFlags(&c.h2d_stream, cudaStreamNonBlocking));
    GRAV_CUDA_TRY(cudaStreamCreateWithFlags(&c.d2h_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t *ev[4] = {&c.ev_in[k], &c.ev_built[k], &c.ev_walked[k], &c.ev_out[k]};
      for (cudaEvent_t *e : ev) GRAV_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
  }
  if (n > c.bat_cap) {
    GRAV_CUDA_TRY(cudaStreamSynchronize(c.stream));
    GRAV_CUDA_TRY(cudaStreamSynchronize(c.h2d_stream));
    GRAV_CUDA_TRY(cudaStreamSynchronize(c.d2h_stream));
    c.bat_cap = 0;
    for (int k = 0; k < 2; ++k) {
      grav::ctx_release(&c, c.bat_pos[k]); grav::ctx_release(&c, c.bat_mass[k]);
      grav::ctx_release(&c, c.bat_acc[k]);
    }
    for (int k = 0; k < 2; ++k) {
      if ((rc = grav::ctx_alloc(&c, c.bat_pos[k], 3 * n))) return rc;
      if ((rc = grav::ctx_alloc(&c, c.bat_mass[k], n))) return rc;
      if ((rc = grav::ctx_alloc(&c, c.bat_acc[k], 3 * n))) return rc;
    }
    c.bat_cap = n;
  }
  // two engines take turns (one cloud, two snapshots or more): this context and its twin,
  // each with its own tree, walk buffers and stream; the last snapshot goes to this context,
  // so the tree left here is the last snapshot's
  gravity_ctx *eng[2] = {h, h};
  if (nsnap >= 2 && n > 0 && c.seg.nseg <= 1) {
    if (!h->twin) {
      if (!h->twin_stream)
        GRAV_CUDA_TRY(cudaStreamCreateWithFlags(&h->twin_stream, cudaStreamNonBlocking));
      gravity_ctx *t = nullptr;
      if ((rc = gravity_create(&t, c.device, h->twin_stream))) return rc;
      if (c.user_alloc && (rc = gravity_set_allocator(t, c.user_alloc, c.user_free, c.alloc_user))) {
        gravity_destroy(t);
        return rc;
      }
      h->twin = t;
    }
    eng[(nsnap - 1) & 1] = h;                 // slot of the last snapshot
    eng[nsnap & 1] = h->twin;
  }
  // snapshot k uses slot s = k mod 2 and engine eng[s]: its inputs are copied in once the
  // build of snapshot k - 2 has read that slot, its walk writes the slot's output once the
  // copy-out of snapshot k - 2 has finished; so the copies of one snapshot run beside the
  // build and walk of its neighbours (each wait names the event's latest record, that of
  // k - 2)
  const size_t bp = sizeof(double) * 3 * (size_t)n, bm = sizeof(double) * (size_t)n;
  // (an error stops the enqueueing; the copies already in flight are waited for before
  // returning, so the caller's host buffers are no longer in use)
#define GRAV_BATCH_TRY(x) { const cudaError_t e_ = (x); if (e_ != cudaSuccess) { rc = grav::cuda_status(e_); break; } }
  for (int64_t k = 0; k < nsnap && rc == GRAVITY_OK; ++k) {
    const int s = (int)(k & 1);
    if (k >= 2) GRAV_BATCH_TRY(cudaStreamWaitEvent(c.h2d_stream, c.ev_built[s], 0));
    if (n > 0) {
      GRAV_BATCH_TRY(cudaMemcpyAsync(c.bat_pos[s], pos_host[k], bp, cudaMemcpyHostToDevice,
                                     c.h2d_stream));
      GRAV_BATCH_TRY(cudaMemcpyAsync(c.bat_mass[s], mass_host[k], bm, cudaMemcpyHostToDevice,
                                     c.h2d_stream));
    }
    gravity_ctx *e = eng[s];
    const cudaStream_t cs = e->c.stream;
    GRAV_BATCH_TRY(cudaEventRecord(c.ev_in[s], c.h2d_stream));
    GRAV_BATCH_TRY(cudaStreamWaitEvent(cs, c.ev_in[s], 0));
    if ((rc = gravity_tree_build(e, n, c.bat_pos[s], c.bat_mass[s], p))) break;
    GRAV_BATCH_TRY(cudaEventRecord(c.ev_built[s], cs));
    if (k >= 2) GRAV_BATCH_TRY(cudaStreamWaitEvent(cs, c.ev_out[s], 0));
    if ((rc = gravity_forces(e, theta, eps, c.bat_acc[s]))) break;
    GRAV_BATCH_TRY(cudaEventRecord(c.ev_walked[s], cs));
    GRAV_BATCH_TRY(cudaStreamWaitEvent(c.d2h_stream, c.ev_walked[s], 0));
    if (n > 0)
      GRAV_BATCH_TRY(cudaMemcpyAsync(acc_host[k], c.bat_acc[s], bp, cudaMemcpyDeviceToHost,
                                     c.d2h_stream));
    GRAV_BATCH_TRY(cudaEventRecord(c.ev_out[s], c.d2h_stream));
  }
#undef GRAV_BATCH_TRY
  const cudaError_t e1 = cudaStreamSynchronize(c.h2d_stream);
  const cudaError_t e2 = cudaStreamSynchronize(c.d2h_stream);
  if (rc) {
    cudaStreamSynchronize(c.stream);
    if (eng[0] != eng[1]) cudaStreamSynchronize(h->twin_stream);
    return rc;
  }
  if (e1 != cudaSuccess) return grav::cuda_status(e1);
  if (e2 != cudaSuccess) return grav::cuda_status(e2);
  if (eng[0] != eng[1] && (rc = gravity_sync(h->twin))) {
    gravity_sync(h);
    return rc;
  }
  return gravity_sync(h);
}

int gravity_debug_export(gravity_ctx *h, int what, void *dst, size_t bytes) {
  if (!h || !dst) return GRAVITY_E_ARG;
  Ctx &c = h->c;
  if (!c.have_tree) return GRAVITY_E_NOTREE;
  int rc = grav::set_device(c);
  if (rc) return rc;
  GRAV_CUDA_TRY(cudaStreamSynchronize(c.stream));
  const grav::Tree &t = c.t;
  int32_t nn = 0;
  if (c.n > 0) GRAV_CUDA_TRY(cudaMemcpy(&nn, t.nnodes, sizeof(int32_t), cudaMemcpyDeviceToHost));
  const void *src = nullptr;
  size_t need = 0;
  switch (what) {
    case GRAVITY_DBG_ROOT: {
      const int k = c.seg.nseg;
      if (bytes < 4 * sizeof(double) * k) return GRAVITY_E_ARG;
      GRAV_CUDA_TRY(cudaMemcpy2D(dst, 4 * sizeof(double), t.geom, 8 * sizeof(double),
                                 4 * sizeof(double), k, cudaMemcpyDeviceToHost));
      return GRAVITY_OK;
    }
    case GRAVITY_DBG_KEYS: src = t.keys; need = sizeof(uint64_t) * c.n; break;
    case GRAVITY_DBG_PERM: src = t.idx; need = sizeof(uint32_t) * c.n; break;
    case GRAVITY_DBG_NNODES:
      if (bytes < sizeof(int32_t)) return GRAVITY_E_ARG;
      std::memcpy(dst, &nn, sizeof(int32_t));
      return GRAVITY_OK;
    case GRAVITY_DBG_TOPO: src = t.topo; need = sizeof(int4) * nn; break;
    case GRAVITY_DBG_DEPTH: src = t.ndepth; need = sizeof(int32_t) * nn; break;
    case GRAVITY_DBG_PARENT: src = t.nparent; need = sizeof(int32_t) * nn; break;
    case GRAVITY_DBG_MASS: src = t.nmass; need = sizeof(double) * nn; break;
    case GRAVITY_DBG_COM: src = t.ncom; need = 3 * sizeof(double) * nn; break;
    case GRAVITY_DBG_QUAD: {
      // stored as T = sum m y y^T in double-float pairs; exported as Q = 3T - tr(T) I, FP64
      if (bytes < 6 * sizeof(double) * (size_t)nn) return GRAVITY_E_ARG;
      if (nn == 0) return GRAVITY_OK;
      std::vector<float> sec((size_t)12 * nn);
      GRAV_CUDA_TRY(cudaMemcpy(sec.data(), t.nquad, sizeof(float) * sec.size(),
                               cudaMemcpyDeviceToHost));
      double *q = static_cast<double *>(dst);
      for (int32_t k = 0; k < nn; ++k) {
        double T[6];
        for (int a = 0; a < 6; ++a)
          T[a] = (double)sec[12 * (size_t)k + 2 * a] + (double)sec[12 * (size_t)k + 2 * a + 1];
        const double tr = T[0] + T[1] + T[2];
        for (int a = 0; a < 3; ++a) q[6 * (size_t)k + a] = 3.0 * T[a] - tr;
        for (int a = 3; a < 6; ++a) q[6 * (size_t)k + a] = 3.0 * T[a];
      }
      return GRAVITY_OK;
    }
    case GRAVITY_DBG_WALKSTATS: src = c.walk_stats; need = 16 * sizeof(unsigned long long); break;
    default: return GRAVITY_E_ARG;
  }
  if (bytes < need) return GRAVITY_E_ARG;
  if (need == 0) return GRAVITY_OK;
  GRAV_CUDA_TRY(cudaMemcpy(dst, src, need, cudaMemcpyDeviceToHost));
  return GRAVITY_OK;
}

int gravity_stats(gravity_ctx *h, int64_t *launches) {
  if (!h || !launches) return GRAVITY_E_ARG;
  *launches = h->c.launches;
  return GRAVITY_OK;
}

int gravity_probe_fp32(gravity_ctx *h, int64_t iters, double *ms, double *flops) {
  if (!h || iters < 1 || !ms || !flops) return GRAVITY_E_ARG;
  int rc = grav::set_device(h->c);
  if (rc) return rc;
  return grav::probe_fp32(&h->c, iters, ms, flops);
}

const char *gravity_strerror(int code) {
  switch (code) {
    case GRAVITY_OK: return "ok";
    case GRAVITY_E_ARG: return "invalid argument";
    case GRAVITY_E_NONFINITE: return "non-finite position coordinate or invalid radius";
    case GRAVITY_E_NOMEM: return "device allocation failed";
    case GRAVITY_E_CUDA: return "CUDA runtime error";
    case GRAVITY_E_TIMEOUT: return "bounded device wait ran out";
    case GRAVITY_E_INTERNAL: return "walk stack exhausted or inconsistent tree";
    case GRAVITY_E_NOTREE: return "no tree built";
    default: return "unknown error";
  }
}

}  // extern "C"
