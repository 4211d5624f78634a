// Aggregate identification (Sec. 2, "Post-processing: aggregate identification"):
// bodies are the vertices of a contact graph, aggregates its connected components
// with more than one body.  The paper fills the graph from the contact container of
// its collision solver; here contact is read as overlap of the bodies' bounding
// spheres (or a uniform distance threshold).
//
// Contact-graph components.  Bodies i != j of one cloud are joined when
//   |x_i - x_j|^2 <= t_ij^2,  t_ij = r_i + r_j (per-body radii) or a uniform dmax,
// with |d|^2 = (dx^2 + dy^2) + dz^2, d = x_j - x_i, every operation one FP64
// rounding, so each edge is decided exactly as a plain pairwise test decides it.
// The candidate pairs come from the octree already built for gravity: a node can
// hold a partner of body i only if |x_i - COM| <= (r_i + r_max) + sqrt(3) l (every
// body of a node lies in its cube of side l, and so does the COM); the test runs in
// FP32 on the hi parts of the coordinates with margins that cover their truncation
// and rounding, so it never prunes a true partner.  Each thread
// walks the tree for one body (sorted order) and joins it to every partner j > i
// with a lock-free union-find: roots only ever point to smaller indices (a root is
// hooked under the smaller of two roots by compare-and-swap; path halving keeps the
// chains short), so every loop has a bound.  A final pass labels each body with the
// smallest caller index of its component, which does not depend on the order in
// which the unions happened, and counts the components and the aggregates.
#include <climits>

#include "internal.cuh"

namespace grav {
namespace {

constexpr int kCompThreads = 128;
constexpr int kCompStack = kLevels * 8 + 8;    // DFS: at most 7 pending siblings per level
constexpr int kFindMax = 1 << 26;             // bounds of the union-find loops (never reached:
constexpr int kUniteMax = 1 << 20;            // chains strictly decrease)

__device__ __forceinline__ int ld_parent(const int *parent, int x) {
  return *(volatile const int *)(parent + x);
}

// Root of x; parent[x] <= x always holds.  Returns -1 if the bound is hit.
__device__ int find_root(int *parent, int x) {
  for (int it = 0; it < kFindMax; ++it) {
    const int p = ld_parent(parent, x);
    if (p == x) return x;
    const int gp = ld_parent(parent, p);
    if (gp != p) atomicCAS(parent + x, p, gp);   // path halving (a lost race is harmless)
    x = gp;
  }
  return -1;
}

__device__ bool unite(int *parent, int a, int b) {
  for (int it = 0; it < kUniteMax; ++it) {
    a = find_root(parent, a);
    b = find_root(parent, b);
    if (a < 0 || b < 0) return false;
    if (a == b) return true;
    if (a < b) { const int t = a; a = b; b = t; }   // hook the larger root under the smaller
    if (atomicCAS(parent + a, a, b) == a) return true;
  }
  return false;
}

// Radii in sorted order; the largest radius (non-negative doubles order like their
// bit patterns); a negative or non-finite radius latches an error and counts as 0.
__global__ void k_comp_init(const double *__restrict__ radius, const uint32_t *__restrict__ perm,
                            int64_t n, double *__restrict__ r_s, int *__restrict__ parent,
                            int *__restrict__ cmin, unsigned long long *__restrict__ rmax_bits,
                            unsigned *status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  parent[i] = (int)i;
  cmin[i] = INT_MAX;
  if (radius) {
    double r = radius[perm[i]];
    if (!(r >= 0.0) || !isfinite(r)) {
      latch_error(status, kErrNonFinite);
      r = 0.0;
    }
    r_s[i] = r;
    atomicMax(rmax_bits, (unsigned long long)__double_as_longlong(r));
  }
}

struct CompArgs {
  const int4 *topo;
  const int32_t *ndepth;
  const float4 *rec0;                // (COM hi xyz, m)
  const float4 *bhi;                 // (x hi xyz, m), sorted
  const double *geom;
  const double *pos_s;
  const double *r_s;                 // nullptr: uniform dmax
  const unsigned long long *rmax_bits;
  const int32_t *seg_sorted;         // cloud of each body (sorted), nullptr for one cloud
  const int32_t *nnodes;
  double dmax;
  int64_t n;
  int *parent;
  unsigned *status;
};

__global__ void __launch_bounds__(kCompThreads) k_comp_search(CompArgs A) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int nn = *A.nnodes;
  const int root = A.seg_sorted ? A.seg_sorted[i] : 0;
  const double *gr = A.geom + 8 * root;
  const double xi = A.pos_s[3 * i], yi = A.pos_s[3 * i + 1], zi = A.pos_s[3 * i + 2];
  const double ri = A.r_s ? A.r_s[i] : 0.0;
  const double reach = A.r_s ? __dadd_rn(ri, __longlong_as_double((long long)*A.rmax_bits)) : A.dmax;
  // FP32 pruning: hi parts differ from the FP64 values by <= 2^-24 of the largest |corner
  // coordinate| C of the root cube, FP32 differences and squares add a few 2^-24 relative;
  // the margin 2^-18 (reach + sqrt(3) l) + 2^-18 C covers both with room
  const float C = (float)fmax(fmax(fmax(fabs(gr[0]), fabs(gr[0] + gr[3])), fmax(fabs(gr[1]), fabs(gr[1] + gr[3]))),
                              fmax(fabs(gr[2]), fabs(gr[2] + gr[3])));
  const float sidef = (float)gr[3] * (1.0f + 3.814697265625e-6f);   // side, rounded up
  const float reachf = (float)reach * (1.0f + 3.814697265625e-6f) + 3.814697265625e-6f * C;
  const float4 bh = A.bhi[i];
  int stack[kCompStack];
  int sp = 0;
  stack[sp++] = root;
  while (sp > 0) {
    const int node = stack[--sp];
    if (node < 0 || node >= nn) { latch_error(A.status, kErrTree); return; }
    const int4 tp = A.topo[node];
    const float4 c = A.rec0[node];
    const float dx = c.x - bh.x, dy = c.y - bh.y, dz = c.z - bh.z;
    const float D2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float l = sidef * __int_as_float((127 - A.ndepth[node]) << 23);   // side * 2^-depth
    const float S = fmaf(1.7320509f, l, reachf) * (1.0f + 3.814697265625e-6f);
    if (D2 > S * S) continue;                   // no body of the node is in reach
    if (tp.x >= 0) {                            // internal: visit the children
      if (tp.x + tp.y > nn || sp + tp.y > kCompStack) { latch_error(A.status, kErrStack); return; }
      for (int k = 0; k < tp.y; ++k) stack[sp++] = tp.x + k;
      continue;
    }
    if (tp.z < 0 || tp.w > A.n || tp.z >= tp.w) { latch_error(A.status, kErrTree); return; }
    for (int j = max(tp.z, (int)i + 1); j < tp.w; ++j) {   // each pair once: partner j > i
      const double ex = __dsub_rn(A.pos_s[3 * j], xi), ey = __dsub_rn(A.pos_s[3 * j + 1], yi),
                   ez = __dsub_rn(A.pos_s[3 * j + 2], zi);
      const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)), __dmul_rn(ez, ez));
      const double t = A.r_s ? __dadd_rn(ri, A.r_s[j]) : A.dmax;
      if (d2 <= __dmul_rn(t, t) && !unite(A.parent, (int)i, j)) {
        latch_error(A.status, kErrTimeout);
        return;
      }
    }
  }
}

// Root of every body, the smallest caller index and the size of each component
// (kept at its root).
__global__ void k_comp_min(const uint32_t *__restrict__ perm, int64_t n, int *parent,
                           int *__restrict__ root_of, int *__restrict__ cmin,
                           int *__restrict__ csize, unsigned *status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = find_root(parent, (int)i);
  if (r < 0) { latch_error(status, kErrTimeout); root_of[i] = (int)i; return; }
  root_of[i] = r;
  atomicMin(cmin + r, (int)perm[i]);
  atomicAdd(csize + r, 1);
}

// Labels in caller order; counts[0] = components, counts[1] = components of more
// than one body (the aggregates).
__global__ void k_comp_label(const uint32_t *__restrict__ perm, int64_t n,
                             const int *__restrict__ root_of, const int *__restrict__ cmin,
                             const int *__restrict__ csize, int32_t *__restrict__ label,
                             unsigned long long *__restrict__ counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  label[perm[i]] = cmin[root_of[i]];
  if (root_of[i] == (int)i) {
    atomicAdd(counts, 1ull);
    if (csize[i] > 1) atomicAdd(counts + 1, 1ull);
  }
}

__global__ void k_comp_counts(const unsigned long long *counts, int64_t *out) {
  out[0] = (int64_t)counts[0];
  out[1] = (int64_t)counts[1];
}

}  // namespace

int components(Ctx *c, const double *radius, double dmax, int32_t *label, int64_t *counts) {
  const int64_t n = c->n;
  if (n > c->comp_cap) {
    GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
    ctx_release(c, c->comp_r);
    ctx_release(c, c->comp_i);
    c->comp_cap = 0;
    int rc = ctx_alloc(c, c->comp_r, n + 3);    // radii (sorted), largest radius, 2 counts
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->comp_i, 4 * n);   // parent, min, root, size
    if (rc) return rc;
    c->comp_cap = n;
  }
  int *parent = c->comp_i, *cmin = c->comp_i + n, *root_of = c->comp_i + 2 * n,
      *csize = c->comp_i + 3 * n;
  // three 64-bit words after the radii: the largest radius (bits), the two counts
  unsigned long long *sc = reinterpret_cast<unsigned long long *>(c->comp_r + n);
  GRAV_CUDA_TRY(cudaMemsetAsync(sc, 0, 3 * sizeof(unsigned long long), c->stream));
  GRAV_CUDA_TRY(cudaMemsetAsync(csize, 0, sizeof(int) * (size_t)n, c->stream));
  const unsigned blocks = (unsigned)((n + kCompThreads - 1) / kCompThreads);
  k_comp_init<<<blocks, kCompThreads, 0, c->stream>>>(radius, c->t.idx, n, c->comp_r, parent,
                                                      cmin, sc, c->d_status);
  CompArgs A{};
  A.topo = c->t.topo; A.ndepth = c->t.ndepth; A.rec0 = c->t.nrec0; A.bhi = c->t.body_hi;
  A.geom = c->t.geom;
  A.pos_s = c->t.pos_s; A.r_s = radius ? c->comp_r : nullptr; A.rmax_bits = sc;
  A.seg_sorted = c->seg.nseg > 1 ? c->seg.seg_sorted : nullptr;
  A.nnodes = c->t.nnodes; A.dmax = dmax; A.n = n; A.parent = parent; A.status = c->d_status;
  k_comp_search<<<blocks, kCompThreads, 0, c->stream>>>(A);
  k_comp_min<<<blocks, kCompThreads, 0, c->stream>>>(c->t.idx, n, parent, root_of, cmin, csize,
                                                     c->d_status);
  k_comp_label<<<blocks, kCompThreads, 0, c->stream>>>(c->t.idx, n, root_of, cmin, csize, label,
                                                       sc + 1);
  c->launches += 4;
  if (counts) {
    k_comp_counts<<<1, 1, 0, c->stream>>>(sc + 1, counts);
    ++c->launches;
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace grav
