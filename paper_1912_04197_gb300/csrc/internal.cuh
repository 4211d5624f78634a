// Internal declarations of libgravity (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "gravity.h"

namespace grav {

constexpr int kLevels = 21;          // 63-bit Morton keys: 21 levels of 3 bits
constexpr int kScalarWords = 192;    // small device scalars of a tree (t.scalars)
constexpr int kMaxLeaf = 64;         // largest leaf_max accepted

// Latched device error bits (combined with atomicOr into ctx->d_status).
enum : unsigned {
  kErrNonFinite = 1u,
  kErrStack = 2u,
  kErrTree = 4u,
  kErrTimeout = 8u,
};

struct Tree {
  // geometry per cloud, 8 doubles each: lo[3], side, scale = 2^21 / side
  double *geom = nullptr;
  int geom_cap = 0;              // clouds the geometry array holds
  // keys / sort
  uint64_t *keys = nullptr, *keys_alt = nullptr;
  uint32_t *idx = nullptr, *idx_alt = nullptr;   // after the sort: idx = perm (sorted -> caller)
  uint32_t *hist = nullptr;                     // radix sort: digit counts and tile states
  double *bbox_part = nullptr;                  // [blocks][6]
  unsigned *bbox_ticket = nullptr;
  // sorted bodies
  double *pos_s = nullptr;                      // (n,3)
  double *mass_s = nullptr;                     // (n)
  float4 *body_hi = nullptr;                    // (x_hi, y_hi, z_hi, m)
  float4 *body_lo = nullptr;                    // (x_lo, y_lo, z_lo, 0)
  // binary radix tree over n-1 internal nodes; child code >= 0: internal node,
  // < 0: body ~code
  int32_t *bchild = nullptr;                    // [2*(n-1)]
  int32_t *bparent = nullptr;                   // [n-1]
  int32_t *bfirst = nullptr;                    // [n-1]
  int32_t *blast = nullptr;                     // [n-1]
  int32_t *bplen = nullptr;                     // [n-1] common prefix length (bits)
  uint32_t *bnchild = nullptr;                  // [n-1] octree children (0 if not internal)
  uint32_t *bbase = nullptr;                    // [n-1] exclusive scan of bnchild
  uint32_t *scalars = nullptr;                  // small device scalars (scan totals, buckets)
  // octree, capacity 2n nodes
  int4 *topo = nullptr;                         // first child (-1 leaf), n_child, begin, end
  int32_t *nparent = nullptr;
  int32_t *ndepth = nullptr;
  int32_t *nlist = nullptr;                     // node ids bucketed for the moment pass
  int32_t *nnodes = nullptr;                    // device scalar
  double *nmass = nullptr;                      // FP64 moments
  double *ncom = nullptr;                       // (k,3)
  float4 *nquad = nullptr;                      // (k,3) second moments T about the COM, (hi, lo) pairs
  float4 *nrec0 = nullptr;                      // (com_hi xyz, m)
  float4 *nrec1 = nullptr;                      // (com_lo xyz, l^2)
  float4 *nquadf = nullptr;                     // 2 per node, of -Q: (xx,yy,zz,xy), (xz,yz,0,0)
};

// Independent clouds (segments) handled in one build and one walk launch: bodies
// are given concatenated cloud by cloud; cloud k occupies [off[k], off[k+1]).
struct Segs {
  int nseg = 1;                  // number of clouds
  int cbits = 0;                 // bits of the cloud id in the extended key (0 for one cloud)
  int64_t *off = nullptr;        // device copy of the offsets (nseg + 1)
  int32_t *seg_of = nullptr;     // cloud id of each body, caller order (nseg > 1)
  int32_t *seg_sorted = nullptr; // cloud id of each body, sorted order (nseg > 1)
  int32_t *task_begin = nullptr; // walk tasks: first body (sorted order), cloud end, cloud id
  int32_t *task_end = nullptr;
  int32_t *task_seg = nullptr;
  int ntasks = 0;
  int64_t n = 0;                 // total bodies the segmentation describes
  int64_t body_cap = 0;
  std::vector<int32_t> h_task_begin, h_task_end;   // host copies (task ranges of a shard)
};

// Captured leapfrog step (a CUDA graph) and the arguments it was captured with.
struct StepGraph {
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  int64_t n = 0;
  const void *pos = nullptr, *vel = nullptr, *mass = nullptr, *acc = nullptr;
  double dt = 0, theta = 0, eps = 0;
  gravity_params params{};
  int nseg = 0;
  int64_t kernels = 0;         // kernels in one replay
};

struct Ctx {
  int device = 0;
  // device memory of the context: cudaMalloc/cudaFree, or the caller's allocator
  gravity_alloc_fn user_alloc = nullptr;
  gravity_free_fn user_free = nullptr;
  void *alloc_user = nullptr;
  int stack_cap = 0;           // walk stack entries allowed (0 = all); failure testing
  int sort_stall = 0;          // > 0: sort passes withhold tile 0, look-back budget (testing)
  int moments_stall = 0;       // > 0: leaves not counted, moment-pass wait budget (testing)
  int grav_since = 0;          // leapfrog_step with grav_every > 1: steps since the last force
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int64_t cap = 0;             // body capacity of the buffers
  int64_t n = 0;               // bodies in the current tree
  bool have_tree = false;
  gravity_params params{};
  unsigned *d_status = nullptr;
  Segs seg;                    // cloud segmentation (one cloud unless set)
  StepGraph graph;             // cached captured leapfrog step
  int64_t launches = 0;        // kernels enqueued by this context (introspection)
  unsigned long long *walk_stats = nullptr;   // 16 counters filled by the counted walk
  void *walk_gstack = nullptr;                // walk stack overflow, per persistent warp
  unsigned *walk_queues = nullptr;            // walk task-queue counters, one per SM
  size_t walk_gstack_cap = 0;                 // in 8-byte entries
  double *walk_part = nullptr;                // four-way split walk: partial sums
  size_t walk_part_cap = 0;                   // in doubles
  // walk task order: the SM clock cycles each task took in the last full force walk, and
  // each task queue's tasks in decreasing order of that cost for the next one
  uint32_t *walk_cost = nullptr;
  int32_t *walk_order = nullptr;
  int64_t walk_order_cap = 0;                 // tasks the two arrays hold
  int walk_order_n = 0;                       // tasks (after splitting) the order is for
  int walk_order_nq = 0;                      // and the queues it is for
  // vector-Jacobian product scratch (sorted order; nodes 2 cap)
  double *vjp_own = nullptr, *vjp_body = nullptr, *vjp_node = nullptr;
  int64_t vjp_cap = 0;
  // leapfrog adjoint: positions of the recomputed levels, velocity, acceleration
  // and product work arrays
  double *adj_levels = nullptr, *adj_work = nullptr;
  int64_t adj_levels_cap = 0, adj_work_cap = 0;   // in doubles
  unsigned char *adj_bank = nullptr;              // saved trees of the recomputed levels
  size_t adj_bank_cap = 0;                        // in bytes
  Tree t;
  // direct-sum staging (caller order hi/lo)
  float4 *dir_hi = nullptr, *dir_lo = nullptr;
  int64_t dir_cap = 0;
  // direct sum on Morton-sorted tiles: order, sorted hi/lo bodies, tile boxes
  uint64_t *ds_keys = nullptr, *ds_keys_alt = nullptr;
  uint32_t *ds_idx = nullptr, *ds_idx_alt = nullptr, *ds_hist = nullptr;
  double *ds_geom = nullptr;
  unsigned long long *ds_part = nullptr;
  unsigned *ds_ticket = nullptr;
  float4 *ds_hi = nullptr, *ds_lo = nullptr, *ds_box = nullptr;
  int64_t ds_cap = 0;
  // diagnostics: m phi per body, block partials, result (nodes of 8 doubles)
  double *diag_buf = nullptr;
  int64_t diag_cap = 0;
  // host-buffer entry point staging
  double *h2d_pos = nullptr, *h2d_mass = nullptr, *h2d_acc = nullptr;
  int64_t h2d_cap = 0;
  // batched host-buffer evaluation: two slots of device inputs and outputs, a copy stream
  // each way, and the events that order them against the context's stream
  double *bat_pos[2] = {nullptr, nullptr}, *bat_mass[2] = {nullptr, nullptr};
  double *bat_acc[2] = {nullptr, nullptr};
  int64_t bat_cap = 0;
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_built[2] = {nullptr, nullptr};
  cudaEvent_t ev_walked[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  // contact components: sorted radii + 3 words; parent, component minimum, root, size
  double *comp_r = nullptr;
  int *comp_i = nullptr;
  int64_t comp_cap = 0;
};

// ---- launchers (tree_build.cu)
int tree_build(Ctx *c, int64_t n, const double *pos, const double *mass);
struct MortonBuffers {
  uint64_t *keys, *keys_alt;
  uint32_t *idx, *idx_alt;
  uint32_t *hist;                 // radix sort counts and tile states
  double *geom;                   // 8 doubles: root cube of the bodies
  unsigned long long *part;       // bounding-box partials, 6 per block
  unsigned *ticket;               // zero before the first use; left zero
};
int morton_order(Ctx *c, int64_t n, const double *pos, const MortonBuffers &b);
int64_t radix_hist_words(int64_t n);
// ---- launchers (walk.cu)
int walk_forces(Ctx *c, double theta, double eps, double *acc, int32_t *counts,
                double *vel, double kick);
// The walk of tasks [first_task, first_task + ntasks) only, their bodies' accelerations
// written in sorted order to acc_sorted (nbodies rows, from sorted body body0).
int walk_forces_range(Ctx *c, double theta, double eps, int64_t first_task, int64_t ntasks,
                      int64_t body0, int64_t nbodies, double *acc_sorted);
// Number of walk tasks of the current tree (32 Morton-consecutive bodies of one cloud each).
int64_t walk_task_count(const Ctx *c);
int walk_vjp(Ctx *c, double theta, double eps, const double *lambda, double *grad);
// The same on a tree held elsewhere (a saved copy of the arrays the product reads).
int walk_vjp_tree(Ctx *c, const Tree &t, double theta, double eps, const double *lambda,
                  double *grad);
int walk_stack_capacity();
// ---- launchers (direct.cu)
int direct_forces(Ctx *c, int64_t n, const double *pos, const double *mass, double eps,
                  double G, double *acc);
int diagnostics(Ctx *c, int64_t n, const double *pos, const double *vel, const double *mass,
                double eps, double G, double *out_dev);
// ---- launchers (contact.cu)
int components(Ctx *c, const double *radius, double dmax, int32_t *label, int64_t *counts);
// ---- launchers (integrate.cu)
int launch_kick_drift(Ctx *c, int64_t n, double *pos, double *vel, const double *acc,
                      double h_kick, double dt);
int launch_kick(Ctx *c, int64_t n, double *vel, const double *acc, double h_kick);
int launch_scatter_sorted(Ctx *c, int64_t first_body, int64_t nbodies, const double *src,
                          double *dst);
int launch_adjoint_kick_drift(Ctx *c, int64_t n, double *xbar, double *vbar, const double *g,
                              double coef, double dt, bool drift);

// ---- probe.cu
int probe_fp32(Ctx *c, int64_t iters, double *ms, double *flops);

int ensure_capacity(Ctx *c, int64_t n);
int alloc_base(Ctx *c);
void free_all(Ctx *c);
// Context-owned device memory (through the caller's allocator when one is set).
int ctx_malloc(Ctx *c, void **p, size_t bytes);
void ctx_free(Ctx *c, void *p);
template <typename T>
int ctx_alloc(Ctx *c, T *&p, int64_t count) {
  void *q = nullptr;
  const int rc = ctx_malloc(c, &q, sizeof(T) * (size_t)(count > 0 ? count : 1));
  p = static_cast<T *>(q);
  return rc;
}
template <typename T>
void ctx_release(Ctx *c, T *&p) {
  if (p) ctx_free(c, p);
  p = nullptr;
}
int set_segments(Ctx *c, int nseg, const int64_t *off_host);
int fill_segment_ids(Ctx *c);
int cuda_status(cudaError_t e);

// ---- device helpers
__device__ __forceinline__ void latch_error(unsigned *status, unsigned bit) {
  atomicOr(status, bit);
}

// 2^-d as a double, built from its exponent bits (0 <= d <= 1022): side * pow2_neg(d)
// equals ldexp(side, -d) exactly while the product stays normal.
__device__ __forceinline__ double pow2_neg(int d) {
  return __longlong_as_double((long long)(1023 - d) << 52);
}

// hi/lo split of an FP64 value into two FP32 values with hi + lo ~ x to ~2^-48.
__device__ __forceinline__ void split_df(double x, float &hi, float &lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(__dsub_rn(x, (double)hi));
}

}  // namespace grav

#define GRAV_CUDA_TRY(expr)                         \
  do {                                              \
    cudaError_t _e = (expr);                        \
    if (_e != cudaSuccess) return grav::cuda_status(_e); \
  } while (0)
