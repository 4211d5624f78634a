// Octree construction on the GPU: kernels 1-4 of the paper's five-kernel list
// (Sec. 2.1, "CUDA implementation of GPU-parallel Barnes-Hut"):
//   bounding box (root cube) -> Morton keys -> stable LSD radix sort ("sort bodies")
//   -> binary radix tree over the sorted keys -> compressed octree -> node mass and
//   centre of mass, Eq. (COMinternal), bottom-up in FP64.
// The paper builds its octree by insertion with locks (Burtscher-Pingali design);
// here every step is a data-parallel pass with no lock and no spin-wait.
#include <cstdio>

#include "internal.cuh"

namespace grav {
namespace {

constexpr int kBBoxThreads = 256;
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;   // keys per radix tile
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int cap_depth(int plen) {
  int d = plen / 3;
  return d < kLevels ? d : kLevels;
}

// ------------------------------------------------------------------ a1: root cube
// Kernel 1 (Sec. 2.1): bounding box of all bodies.  Root cube: corner at the
// per-axis minimum, side = largest extent (1 if that is 0 or n <= 1).  Any
// non-finite coordinate latches kErrNonFinite.  Last-block reduction, no spin.
__global__ void __launch_bounds__(kBBoxThreads)
k_bbox(const double *__restrict__ pos, int64_t n, double *__restrict__ part,
       unsigned *__restrict__ ticket, double *__restrict__ geom, unsigned *status) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      double v = pos[3 * i + a];
      bad |= !isfinite(v);
      lo[a] = fmin(lo[a], v);
      hi[a] = fmax(hi[a], v);
    }
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  bad = __any_sync(0xffffffffu, bad);
  __shared__ double s[kBBoxThreads / 32][6];
  __shared__ int s_bad;
  __shared__ bool s_last;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    for (int a = 0; a < 3; ++a) { s[w][a] = lo[a]; s[w][3 + a] = hi[a]; }
    if (bad) s_bad = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int ww = 1; ww < kBBoxThreads / 32; ++ww)
      for (int a = 0; a < 3; ++a) {
        s[0][a] = fmin(s[0][a], s[ww][a]);
        s[0][3 + a] = fmax(s[0][3 + a], s[ww][3 + a]);
      }
    for (int a = 0; a < 6; ++a) part[6 * blockIdx.x + a] = s[0][a];
    if (s_bad) latch_error(status, kErrNonFinite);
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double glo[3] = {INFINITY, INFINITY, INFINITY}, ghi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (unsigned b = 0; b < gridDim.x; ++b)
    for (int a = 0; a < 3; ++a) {
      glo[a] = fmin(glo[a], __ldcg(&part[6 * b + a]));
      ghi[a] = fmax(ghi[a], __ldcg(&part[6 * b + 3 + a]));
    }
  double side = 0.0;
  for (int a = 0; a < 3; ++a) side = fmax(side, __dsub_rn(ghi[a], glo[a]));
  if (n <= 1 || !(side > 0.0) || !isfinite(side)) side = 1.0;
  for (int a = 0; a < 3; ++a) geom[a] = isfinite(glo[a]) ? glo[a] : 0.0;
  geom[3] = side;
  geom[4] = __ddiv_rn(2097152.0, side);   // 2^21 / side, one IEEE division
  *ticket = 0;                            // ready for the next build
}

// ------------------------------------------------------------------ a2: Morton keys
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1FFFFFu;
  x = (x | (x << 32)) & 0x1F00000000FFFFull;
  x = (x | (x << 16)) & 0x1F0000FF0000FFull;
  x = (x | (x << 8)) & 0x100F00F00F00F00Full;
  x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint32_t grid_coord(double x, double lo, double scale) {
  // q = clamp(floor((x - lo) * scale), 0, 2^21 - 1): separate IEEE sub and mul
  double f = floor(__dmul_rn(__dsub_rn(x, lo), scale));
  if (!(f >= 0.0)) f = 0.0;
  if (f > 2097151.0) f = 2097151.0;
  return (uint32_t)f;
}

__global__ void k_keys(const double *__restrict__ pos, int64_t n, const double *__restrict__ geom,
                       uint64_t *__restrict__ keys, uint32_t *__restrict__ idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double scale = geom[4];
  uint32_t qx = grid_coord(pos[3 * i + 0], geom[0], scale);
  uint32_t qy = grid_coord(pos[3 * i + 1], geom[1], scale);
  uint32_t qz = grid_coord(pos[3 * i + 2], geom[2], scale);
  keys[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
  idx[i] = (uint32_t)i;
}

// ------------------------------------------------------------------ exclusive scan (u32)
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  int l = threadIdx.x & 31;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (l >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread (blockDim = kScanThreads).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t &total) {
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  uint32_t inc = warp_incl_scan(v);
  if (l == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t x = (l < (kScanThreads >> 5)) ? s_warp[l] : 0u;
    uint32_t xi = warp_incl_scan(x);
    s_warp[l] = xi - x;
    if (l == 31) s_warp[32] = xi;
  }
  __syncthreads();
  uint32_t r = s_warp[w] + inc - v;
  total = s_warp[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(uint32_t *__restrict__ data, int64_t n, uint32_t *__restrict__ sums) {
  __shared__ uint32_t s_warp[33];
  int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
  uint32_t v[kScanItems], t = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? data[base + k] : 0u;
    t += v[k];
  }
  uint32_t total;
  uint32_t ex = block_excl_scan(t, s_warp, total);
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) data[base + k] = ex;
    ex += v[k];
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block scans all tile sums (any count, in chunks) and writes the grand total.
__global__ void __launch_bounds__(kScanThreads)
k_scan_sums(uint32_t *__restrict__ sums, int nb, uint32_t *__restrict__ total_out) {
  __shared__ uint32_t s_warp[33];
  uint32_t carry = 0;
  for (int c0 = 0; c0 < nb; c0 += kScanThreads) {
    int i = c0 + threadIdx.x;
    uint32_t v = (i < nb) ? sums[i] : 0u, tot;
    uint32_t ex = block_excl_scan(v, s_warp, tot);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_add(uint32_t *__restrict__ data, int64_t n, const uint32_t *__restrict__ sums) {
  int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanItems;
  uint32_t add = sums[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) data[base + k] += add;
}

int exclusive_scan(Ctx *c, uint32_t *data, int64_t n, uint32_t *total_out) {
  if (n <= 0) return GRAVITY_OK;
  int nb = (int)((n + kScanTile - 1) / kScanTile);
  k_scan_tiles<<<nb, kScanThreads, 0, c->stream>>>(data, n, c->t.scan_aux);
  ++c->launches;
  k_scan_sums<<<1, kScanThreads, 0, c->stream>>>(c->t.scan_aux, nb, total_out);
  ++c->launches;
  if (nb > 1) { k_scan_add<<<nb, kScanThreads, 0, c->stream>>>(data, n, c->t.scan_aux); ++c->launches; }
  return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ a3: radix sort
// Stable LSD radix sort of (key, index) pairs, 8 passes of 8-bit digits.
// Pass = per-tile digit histogram -> exclusive scan in digit-major order ->
// stable scatter (ranks from warp match + per-warp counts, in index order).
__global__ void __launch_bounds__(kRsThreads)
k_rs_hist(const uint64_t *__restrict__ keys, int64_t n, int shift, uint32_t *__restrict__ hist,
          int ntiles) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = blockIdx.x * (int64_t)kRsTile;
  for (int k = 0; k < kRsItems; ++k) {
    int64_t i = base + k * kRsThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kRsThreads)
k_rs_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
             uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
             const uint32_t *__restrict__ offs, int ntiles) {
  constexpr int W = kRsThreads / 32;
  __shared__ uint32_t s_base[256];
  __shared__ uint32_t s_w[W][256];
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const unsigned lt = (1u << l) - 1u;
  s_base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
  const int64_t base = blockIdx.x * (int64_t)kRsTile;
  for (int k = 0; k < kRsItems; ++k) {
    for (int ww = 0; ww < W; ++ww) s_w[ww][tid] = 0;
    __syncthreads();
    int64_t i = base + k * kRsThreads + tid;
    bool valid = i < n;
    uint64_t key = valid ? kin[i] : 0ull;
    uint32_t val = valid ? vin[i] : 0u;
    unsigned d = valid ? ((unsigned)(key >> shift) & 255u) : 256u;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) s_w[w][d] = __popc(peers);
    __syncthreads();
    uint32_t run = s_base[tid];
    for (int ww = 0; ww < W; ++ww) {
      uint32_t cnum = s_w[ww][tid];
      s_w[ww][tid] = run;
      run += cnum;
    }
    s_base[tid] = run;
    __syncthreads();
    if (valid) {
      uint32_t p = s_w[w][d] + rank;
      if (p < (uint64_t)n) {                 // always true for consistent histograms
        kout[p] = key;
        vout[p] = val;
      }
    }
    __syncthreads();
  }
}

int radix_sort(Ctx *c, int64_t n) {
  Tree &t = c->t;
  int ntiles = (int)((n + kRsTile - 1) / kRsTile);
  uint64_t *ka = t.keys, *kb = t.keys_alt;
  uint32_t *va = t.idx, *vb = t.idx_alt;
  for (int pass = 0; pass < 8; ++pass) {
    int shift = 8 * pass;
    k_rs_hist<<<ntiles, kRsThreads, 0, c->stream>>>(ka, n, shift, t.hist, ntiles);
    ++c->launches;
    int rc = exclusive_scan(c, t.hist, (int64_t)256 * ntiles, nullptr);
    if (rc) return rc;
    k_rs_scatter<<<ntiles, kRsThreads, 0, c->stream>>>(ka, va, kb, vb, n, shift, t.hist, ntiles);
    ++c->launches;
    uint64_t *tk = ka; ka = kb; kb = tk;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  // 8 passes: the sorted data is back in t.keys / t.idx
  return cuda_status(cudaGetLastError());
}

// ------------------------------------------------------------------ a4: gather
__global__ void k_gather(const double *__restrict__ pos, const double *__restrict__ mass,
                         const uint32_t *__restrict__ perm, int64_t n, double *__restrict__ pos_s,
                         double *__restrict__ mass_s, float4 *__restrict__ bhi,
                         float4 *__restrict__ blo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t j = perm[i];
  double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2], m = mass[j];
  pos_s[3 * i] = x; pos_s[3 * i + 1] = y; pos_s[3 * i + 2] = z;
  mass_s[i] = m;
  float xh, xl, yh, yl, zh, zl;
  split_df(x, xh, xl); split_df(y, yh, yl); split_df(z, zh, zl);
  bhi[i] = make_float4(xh, yh, zh, __double2float_rn(m));
  blo[i] = make_float4(xl, yl, zl, 0.0f);
}

// ------------------------------------------------------------------ a5: binary radix tree
// Common prefix length (bits) of the extended keys (key, sorted index) at sorted
// positions i and j; -1 outside [0, n).  Keys use 63 bits, so bit 63 is 0.
__device__ __forceinline__ int delta(const uint64_t *__restrict__ k, int n, int i, int j) {
  if (j < 0 || j >= n) return -1;
  uint64_t a = k[i], b = k[j];
  if (a != b) return __clzll((long long)(a ^ b)) - 1;
  return 63 + __clz((int)((unsigned)i ^ (unsigned)j));
}

// Karras' parallel construction: internal node i covers a key range with one end
// at i; its direction, extent and split follow from prefix-length comparisons.
__global__ void k_radix_tree(const uint64_t *__restrict__ k, int n, int32_t *__restrict__ child,
                             int32_t *__restrict__ parent, int32_t *__restrict__ first,
                             int32_t *__restrict__ last, int32_t *__restrict__ plen) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int dir = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(k, n, i, i - dir);
  int lmax = 2;
  while (delta(k, n, i, i + lmax * dir) > dmin) lmax <<= 1;
  int len = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(k, n, i, i + (len + t) * dir) > dmin) len += t;
  int j = i + len * dir;
  int dnode = delta(k, n, i, j);
  int s = 0;
  for (int div = 2;; div <<= 1) {
    int t = (len + div - 1) / div;
    if (delta(k, n, i, i + (s + t) * dir) > dnode) s += t;
    if (t <= 1) break;
  }
  int gamma = i + s * dir + (dir < 0 ? -1 : 0);
  int lo = min(i, j), hi = max(i, j);
  int left = (lo == gamma) ? ~gamma : gamma;
  int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
  child[2 * i] = left;
  child[2 * i + 1] = right;
  if (left >= 0) parent[left] = i;
  if (right >= 0) parent[right] = i;
  if (i == 0) parent[0] = -1;
  first[i] = lo;
  last[i] = hi;
  plen[i] = dnode;
}

// ------------------------------------------------------------------ a6: octree
// A binary node X is an octree cell when its capped depth floor(plen/3) exceeds
// its binary parent's (or X is the root): the cell at that depth holds exactly X's
// bodies, i.e. X is the deepest member of a chain of single-child cells.  A cell
// is internal when it holds > leaf_max bodies and is above depth 21.  Its octree
// children are the first binary descendants whose prefix reaches 3(depth+1) bits
// (or bodies), found by a DFS of at most 7 binary nodes, in key = octant order.
struct Frontier {
  int32_t item[8];
  int count;
};

__device__ __forceinline__ bool frontier(const int32_t *__restrict__ child,
                                         const int32_t *__restrict__ plen, int X, int T,
                                         Frontier &f) {
  int32_t st[16];
  int sp = 0;
  f.count = 0;
  st[sp++] = child[2 * X + 1];
  st[sp++] = child[2 * X];
  while (sp > 0) {
    int32_t c = st[--sp];
    if (c < 0 || plen[c] >= T) {
      if (f.count >= 8) return false;
      f.item[f.count++] = c;
    } else {
      if (sp + 2 > 16) return false;
      st[sp++] = child[2 * c + 1];
      st[sp++] = child[2 * c];
    }
  }
  return true;
}

__global__ void k_oct_count(int n, int leaf_max, const int32_t *__restrict__ child,
                            const int32_t *__restrict__ parent, const int32_t *__restrict__ first,
                            const int32_t *__restrict__ last, const int32_t *__restrict__ plen,
                            uint32_t *__restrict__ nchild, unsigned *status) {
  int X = blockIdx.x * blockDim.x + threadIdx.x;
  if (X >= n - 1) return;
  int d = cap_depth(plen[X]);
  bool cell = (X == 0) || cap_depth(plen[parent[X]]) < d;
  int cnt = last[X] - first[X] + 1;
  if (!(cell && cnt > leaf_max && d < kLevels)) { nchild[X] = 0; return; }
  Frontier f;
  if (!frontier(child, plen, X, 3 * (d + 1), f) || f.count < 2) {
    latch_error(status, kErrTree);
    nchild[X] = 0;
    return;
  }
  nchild[X] = (uint32_t)f.count;
}

__global__ void k_oct_write(int n, int leaf_max, const int32_t *__restrict__ child,
                            const int32_t *__restrict__ first, const int32_t *__restrict__ last,
                            const int32_t *__restrict__ plen, const uint32_t *__restrict__ nchild,
                            const uint32_t *__restrict__ base, const uint32_t *__restrict__ total,
                            int4 *__restrict__ topo, int32_t *__restrict__ depth,
                            int32_t *__restrict__ nnodes, int cap_nodes, unsigned *status) {
  int X = blockIdx.x * blockDim.x + threadIdx.x;
  if (X == 0) {
    // the root (octree node 0)
    int d0 = cap_depth(plen[0]);
    if (nchild[0] > 0) {
      topo[0] = make_int4(1 + (int)base[0], (int)nchild[0], 0, n);
      depth[0] = d0;
    } else {
      topo[0] = make_int4(-1, 0, 0, n);
      depth[0] = (n <= leaf_max) ? 0 : kLevels;
    }
    int nn = 1 + (int)*total;
    if (nn > cap_nodes) { latch_error(status, kErrTree); nn = 1; }
    *nnodes = nn;
  }
  if (X >= n - 1 || nchild[X] == 0) return;
  int d = cap_depth(plen[X]);
  Frontier f;
  frontier(child, plen, X, 3 * (d + 1), f);
  int id0 = 1 + (int)base[X];
  if (id0 + f.count > cap_nodes) { latch_error(status, kErrTree); return; }
  for (int k = 0; k < f.count; ++k) {
    int c = f.item[k], id = id0 + k;
    if (c < 0) {
      int b = ~c;
      topo[id] = make_int4(-1, 0, b, b + 1);
      depth[id] = d + 1;
    } else {
      int b = first[c], e = last[c] + 1;
      if (nchild[c] > 0) {
        topo[id] = make_int4(1 + (int)base[c], (int)nchild[c], b, e);
        depth[id] = cap_depth(plen[c]);
      } else {
        topo[id] = make_int4(-1, 0, b, e);
        depth[id] = (e - b <= leaf_max) ? d + 1 : kLevels;
      }
    }
  }
}

__global__ void k_oct_parent(int cap_nodes, const int4 *__restrict__ topo,
                             const int32_t *__restrict__ nnodes, int32_t *__restrict__ nparent,
                             unsigned *status) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  int nn = *nnodes;
  if (id >= nn || id >= cap_nodes) return;
  if (id == 0) nparent[0] = -1;
  int4 t = topo[id];
  if (t.x < 0) return;
  if (t.x <= 0 || t.x + t.y > nn) { latch_error(status, kErrTree); return; }
  for (int k = 0; k < t.y; ++k) nparent[t.x + k] = id;
}

// ------------------------------------------------------------------ a7: moments
// Eq. (COMinternal): m = sum of child masses; COM = (sum of child COM * child mass)
// / m, children in octant order; a leaf sums its bodies in sorted order.  FP64
// with explicit IEEE roundings (no contraction) so the result is reproducible.
// Quadrupole (order 2): Q = sum m (3 y y^T - |y|^2 I) about the COM, shifted to the
// parent by the parallel-axis rule; a single-body leaf has Q = 0.
// Bottom-up by arrival counters: the last child to arrive computes the parent.
struct MomArgs {
  const int4 *topo;
  const int32_t *nparent;
  const int32_t *ndepth;
  const int32_t *nnodes;
  int32_t *narrive;
  const double *pos_s;
  const double *mass_s;
  const double *geom;
  double *nmass;
  double *ncom;
  double *nquad;
  float4 *rec0;
  float4 *rec1;
  float4 *quadf;
  int order;
  int cap_nodes;
  int n;
  unsigned *status;
};

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }

// Walk records: (COM hi, m) and (COM lo, l^2).  A one-body leaf is always a
// body-to-body term, so its record holds the body position itself and l^2 = -1
// marks it as a point term.
__device__ void write_records(const MomArgs &A, int id, double m, const double *com,
                              const double *q, int single_body) {
  float h[3], lo[3];
  const double *x = single_body >= 0 ? &A.pos_s[3 * single_body] : com;
  for (int a = 0; a < 3; ++a) split_df(x[a], h[a], lo[a]);
  double l = ldexp(A.geom[3], -A.ndepth[id]);
  float l2 = single_body >= 0 ? -1.0f : __double2float_rn(dm(l, l));
  A.rec0[id] = make_float4(h[0], h[1], h[2], __double2float_rn(m));
  A.rec1[id] = make_float4(lo[0], lo[1], lo[2], l2);
  if (A.order >= 2) {
    A.quadf[2 * id] = make_float4(__double2float_rn(q[0]), __double2float_rn(q[1]),
                                  __double2float_rn(q[2]), __double2float_rn(q[3]));
    A.quadf[2 * id + 1] = make_float4(__double2float_rn(q[4]), __double2float_rn(q[5]), 0.f, 0.f);
  }
}

__global__ void k_moments(MomArgs A) {
  int id = blockIdx.x * blockDim.x + threadIdx.x;
  int nn = *A.nnodes;
  if (id >= nn || id >= A.cap_nodes) return;
  int4 t = A.topo[id];
  if (t.x >= 0) return;                       // internal nodes are done by their last child
  if (t.z < 0 || t.w > A.n || t.z >= t.w) { latch_error(A.status, kErrTree); return; }
  // leaf: bodies [t.z, t.w) in sorted order
  double msum = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
  for (int i = t.z; i < t.w; ++i) {
    double mi = A.mass_s[i];
    msum = da(msum, mi);
    sx = da(sx, dm(mi, A.pos_s[3 * i]));
    sy = da(sy, dm(mi, A.pos_s[3 * i + 1]));
    sz = da(sz, dm(mi, A.pos_s[3 * i + 2]));
  }
  double com[3] = {__ddiv_rn(sx, msum), __ddiv_rn(sy, msum), __ddiv_rn(sz, msum)};
  double q[6] = {0, 0, 0, 0, 0, 0};
  if (A.order >= 2 && t.w - t.z > 1) {
    for (int i = t.z; i < t.w; ++i) {
      double mi = A.mass_s[i];
      double y0 = ds(A.pos_s[3 * i], com[0]), y1 = ds(A.pos_s[3 * i + 1], com[1]),
             y2 = ds(A.pos_s[3 * i + 2], com[2]);
      double r2 = da(da(dm(y0, y0), dm(y1, y1)), dm(y2, y2));
      q[0] = da(q[0], dm(mi, ds(dm(dm(3.0, y0), y0), r2)));
      q[1] = da(q[1], dm(mi, ds(dm(dm(3.0, y1), y1), r2)));
      q[2] = da(q[2], dm(mi, ds(dm(dm(3.0, y2), y2), r2)));
      q[3] = da(q[3], dm(mi, dm(dm(3.0, y0), y1)));
      q[4] = da(q[4], dm(mi, dm(dm(3.0, y0), y2)));
      q[5] = da(q[5], dm(mi, dm(dm(3.0, y1), y2)));
    }
  }
  A.nmass[id] = msum;
  for (int a = 0; a < 3; ++a) A.ncom[3 * id + a] = com[a];
  if (A.order >= 2)
    for (int a = 0; a < 6; ++a) A.nquad[6 * id + a] = q[a];
  write_records(A, id, msum, com, q, t.w - t.z == 1 ? t.z : -1);

  int node = id;
  for (int guard = 0;; ++guard) {
    int p = A.nparent[node];
    if (p < 0) return;
    if (guard > 64 || p >= nn) { latch_error(A.status, kErrTree); return; }
    int4 tp = A.topo[p];
    if (tp.x <= 0 || tp.x + tp.y > nn) { latch_error(A.status, kErrTree); return; }
    __threadfence();
    int old = atomicAdd(&A.narrive[p], 1);
    if (old != tp.y - 1) return;             // not the last child
    __threadfence();
    double pm = 0.0, px = 0.0, py = 0.0, pz = 0.0;
    for (int c = tp.x; c < tp.x + tp.y; ++c) {
      double mc = __ldcg(&A.nmass[c]);
      pm = da(pm, mc);
      px = da(px, dm(__ldcg(&A.ncom[3 * c]), mc));
      py = da(py, dm(__ldcg(&A.ncom[3 * c + 1]), mc));
      pz = da(pz, dm(__ldcg(&A.ncom[3 * c + 2]), mc));
    }
    double pc[3] = {__ddiv_rn(px, pm), __ddiv_rn(py, pm), __ddiv_rn(pz, pm)};
    double pq[6] = {0, 0, 0, 0, 0, 0};
    if (A.order >= 2) {
      for (int c = tp.x; c < tp.x + tp.y; ++c) {
        double mc = __ldcg(&A.nmass[c]);
        double d0 = ds(__ldcg(&A.ncom[3 * c]), pc[0]);
        double d1 = ds(__ldcg(&A.ncom[3 * c + 1]), pc[1]);
        double d2 = ds(__ldcg(&A.ncom[3 * c + 2]), pc[2]);
        double r2 = da(da(dm(d0, d0), dm(d1, d1)), dm(d2, d2));
        const double *cq = &A.nquad[6 * c];
        pq[0] = da(pq[0], da(__ldcg(cq + 0), dm(mc, ds(dm(dm(3.0, d0), d0), r2))));
        pq[1] = da(pq[1], da(__ldcg(cq + 1), dm(mc, ds(dm(dm(3.0, d1), d1), r2))));
        pq[2] = da(pq[2], da(__ldcg(cq + 2), dm(mc, ds(dm(dm(3.0, d2), d2), r2))));
        pq[3] = da(pq[3], da(__ldcg(cq + 3), dm(mc, dm(dm(3.0, d0), d1))));
        pq[4] = da(pq[4], da(__ldcg(cq + 4), dm(mc, dm(dm(3.0, d0), d2))));
        pq[5] = da(pq[5], da(__ldcg(cq + 5), dm(mc, dm(dm(3.0, d1), d2))));
      }
    }
    A.nmass[p] = pm;
    for (int a = 0; a < 3; ++a) A.ncom[3 * p + a] = pc[a];
    if (A.order >= 2)
      for (int a = 0; a < 6; ++a) A.nquad[6 * p + a] = pq[a];
    write_records(A, p, pm, pc, pq, -1);
    node = p;
  }
}

// Root of a single body: node 0 is a leaf at depth 0.
__global__ void k_single_root(int4 *topo, int32_t *depth, int32_t *nparent, int32_t *nnodes) {
  topo[0] = make_int4(-1, 0, 0, 1);
  depth[0] = 0;
  nparent[0] = -1;
  *nnodes = 1;
}

inline unsigned blocks_for(int64_t n, int threads) {
  return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

int tree_build(Ctx *c, int64_t n, const double *pos, const double *mass) {
  Tree &t = c->t;
  cudaStream_t s = c->stream;
  const int leaf_max = c->params.leaf_max;
  // a1: root cube (also validates the coordinates)
  int64_t nb64 = (n + kBBoxThreads - 1) / kBBoxThreads;
  if (nb64 > 4 * (int64_t)c->num_sms) nb64 = 4 * (int64_t)c->num_sms;
  int nb = (int)nb64;
  if (nb < 1) nb = 1;
  k_bbox<<<nb, kBBoxThreads, 0, s>>>(pos, n, t.bbox_part, t.bbox_ticket, t.geom, c->d_status);
  ++c->launches;
  // a2: keys
  k_keys<<<blocks_for(n, 256), 256, 0, s>>>(pos, n, t.geom, t.keys, t.idx);
  ++c->launches;
  // a3: sort
  int rc = radix_sort(c, n);
  if (rc) return rc;
  // a4: gather sorted bodies
  k_gather<<<blocks_for(n, 256), 256, 0, s>>>(pos, mass, t.idx, n, t.pos_s, t.mass_s, t.body_hi,
                                               t.body_lo);
  ++c->launches;
  const int cap_nodes = (int)(2 * c->cap);
  if (n == 1) {
    k_single_root<<<1, 1, 0, s>>>(t.topo, t.ndepth, t.nparent, t.nnodes);
    ++c->launches;
  } else {
    int ni = (int)(n - 1);
    // a5: binary radix tree
    k_radix_tree<<<blocks_for(ni, 256), 256, 0, s>>>(t.keys, (int)n, t.bchild, t.bparent, t.bfirst,
                                                     t.blast, t.bplen);
    ++c->launches;
    // a6: octree
    k_oct_count<<<blocks_for(ni, 256), 256, 0, s>>>((int)n, leaf_max, t.bchild, t.bparent,
                                                    t.bfirst, t.blast, t.bplen, t.bnchild,
                                                    c->d_status);
    ++c->launches;
    uint32_t *base = t.bbase;
    GRAV_CUDA_TRY(cudaMemcpyAsync(base, t.bnchild, sizeof(uint32_t) * ni,
                                  cudaMemcpyDeviceToDevice, s));
    uint32_t *total = t.scalars;             // number of non-root octree nodes
    rc = exclusive_scan(c, base, ni, total);
    if (rc) return rc;
    k_oct_write<<<blocks_for(ni, 256), 256, 0, s>>>((int)n, leaf_max, t.bchild, t.bfirst, t.blast,
                                                    t.bplen, t.bnchild, base, total, t.topo,
                                                    t.ndepth, t.nnodes, cap_nodes, c->d_status);
    ++c->launches;
    k_oct_parent<<<blocks_for(cap_nodes, 256), 256, 0, s>>>(cap_nodes, t.topo, t.nnodes,
                                                            t.nparent, c->d_status);
    ++c->launches;
  }
  // a7: moments
  GRAV_CUDA_TRY(cudaMemsetAsync(t.narrive, 0, sizeof(int32_t) * cap_nodes, s));
  MomArgs A{t.topo, t.nparent, t.ndepth, t.nnodes, t.narrive, t.pos_s, t.mass_s, t.geom,
            t.nmass, t.ncom, t.nquad, t.nrec0, t.nrec1, t.nquadf, c->params.order, cap_nodes,
            (int)n, c->d_status};
  k_moments<<<blocks_for(cap_nodes, 256), 256, 0, s>>>(A);
  ++c->launches;
  return cuda_status(cudaGetLastError());
}

}  // namespace grav
