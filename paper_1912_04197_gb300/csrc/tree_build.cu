// Octree construction on the GPU: kernels 1-4 of the paper's five-kernel list
// (Sec. 2.1, "CUDA implementation of GPU-parallel Barnes-Hut"):
//   bounding box (root cube) -> Morton keys -> stable LSD radix sort ("sort bodies")
//   -> binary radix tree over the sorted keys -> compressed octree -> node mass and
//   centre of mass, Eq. (COMinternal), bottom-up in FP64.
// The paper builds its octree by insertion with locks (Burtscher-Pingali design);
// here every step is a data-parallel pass with no lock; the only waits (the sort's and
// the octree scan's look-backs, the moment pass's depth order) are bounded.
#include <cstdio>

#include "internal.cuh"

namespace grav {
namespace {

constexpr int kBBoxThreads = 256;
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;   // keys per radix tile
constexpr int kOctTile = 1024;                   // octree count + scan: binary nodes per tile

__device__ __forceinline__ int cap_depth(int plen) {
  int d = plen / 3;
  return d < kLevels ? d : kLevels;
}

// ------------------------------------------------------------------ a1: root cube
// Kernel 1 (Sec. 2.1): bounding box of all bodies.  Root cube: corner at the
// per-axis minimum, side = largest extent (1 if that is 0 or n <= 1).  Any
// non-finite coordinate latches kErrNonFinite.  Min/max run on order-preserving
// 64-bit integer images of the doubles (exact, and off the slow FP64 pipe); the
// last block to finish reduces the per-block partials.  No spin-wait.
__device__ __forceinline__ unsigned long long ord_of(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double of_ord(unsigned long long k) {
  unsigned long long b = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b) {
  return a < b ? a : b;
}
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// Block-wide min (lo[3]) / max (hi[3]) of ordered keys over NT threads; result valid in
// thread 0.
template <int NT = kBBoxThreads>
__device__ __forceinline__ void block_minmax(unsigned long long lo[3], unsigned long long hi[3]) {
  __shared__ unsigned long long s[NT / 32][6];
  for (int o = 16; o > 0; o >>= 1)
    for (int a = 0; a < 3; ++a) {
      lo[a] = umin64(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = umax64(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
    for (int a = 0; a < 3; ++a) { s[w][a] = lo[a]; s[w][3 + a] = hi[a]; }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int ww = 1; ww < NT / 32; ++ww)
      for (int a = 0; a < 3; ++a) {
        lo[a] = umin64(lo[a], s[ww][a]);
        hi[a] = umax64(hi[a], s[ww][3 + a]);
      }
  __syncthreads();
}

__global__ void __launch_bounds__(kBBoxThreads)
k_bbox(const double *__restrict__ pos, int64_t n, unsigned long long *__restrict__ part,
       unsigned *__restrict__ ticket, double *__restrict__ geom, unsigned *status) {
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
  unsigned long long klo = ~0ull, khi = 0ull;
  bool bad = false;
  const unsigned long long *p64 = reinterpret_cast<const unsigned long long *>(pos);
  // coalesced over the flat (n,3) array; the grid stride is a multiple of 3 (the
  // launcher makes gridDim a multiple of 3), so each thread keeps one axis
  const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = i0; i < 3 * n; i += stride) {
    unsigned long long b = p64[i];
    bad |= ((b >> 52) & 0x7FFull) == 0x7FFull;
    unsigned long long k = (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    klo = umin64(klo, k);
    khi = umax64(khi, k);
  }
  const int axis = (int)(i0 % 3);
  lo[0] = axis == 0 ? klo : lo[0]; hi[0] = axis == 0 ? khi : hi[0];
  lo[1] = axis == 1 ? klo : lo[1]; hi[1] = axis == 1 ? khi : hi[1];
  lo[2] = axis == 2 ? klo : lo[2]; hi[2] = axis == 2 ? khi : hi[2];
  bad = __syncthreads_or(bad);
  block_minmax(lo, hi);
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
    for (int a = 0; a < 3; ++a) { part[6 * blockIdx.x + a] = lo[a]; part[6 * blockIdx.x + 3 + a] = hi[a]; }
    if (bad) latch_error(status, kErrNonFinite);
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int a = 0; a < 3; ++a) { lo[a] = ~0ull; hi[a] = 0ull; }
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
    for (int a = 0; a < 3; ++a) {
      lo[a] = umin64(lo[a], __ldcg(&part[6 * b + a]));
      hi[a] = umax64(hi[a], __ldcg(&part[6 * b + 3 + a]));
    }
  block_minmax(lo, hi);
  if (threadIdx.x != 0) return;
  double glo[3], ghi[3];
  for (int a = 0; a < 3; ++a) { glo[a] = of_ord(lo[a]); ghi[a] = of_ord(hi[a]); }
  double side = 0.0;
  for (int a = 0; a < 3; ++a) side = fmax(side, __dsub_rn(ghi[a], glo[a]));
  if (n <= 1 || !(side > 0.0) || !isfinite(side)) side = 1.0;
  for (int a = 0; a < 3; ++a) geom[a] = isfinite(glo[a]) ? glo[a] : 0.0;
  geom[3] = side;
  geom[4] = __ddiv_rn(2097152.0, side);   // 2^21 / side, one IEEE division
  *ticket = 0;                            // ready for the next build
}

// Root cube of every cloud (several clouds): one block per cloud.
__global__ void __launch_bounds__(kBBoxThreads)
k_bbox_seg(const double *__restrict__ pos, const int64_t *__restrict__ off,
           double *__restrict__ geom, unsigned *status) {
  const int k = blockIdx.x;
  const int64_t b = off[k], e = off[k + 1];
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
  bool bad = false;
  const unsigned long long *p64 = reinterpret_cast<const unsigned long long *>(pos);
  for (int64_t i = 3 * b + threadIdx.x; i < 3 * e; i += blockDim.x) {
    const unsigned long long v = p64[i];
    bad |= ((v >> 52) & 0x7FFull) == 0x7FFull;
    const unsigned long long key = (v >> 63) ? ~v : (v | 0x8000000000000000ull);
    const int a = (int)((i - 3 * b) % 3);
    lo[a] = umin64(lo[a], key);
    hi[a] = umax64(hi[a], key);
  }
  bad = __syncthreads_or(bad);
  block_minmax(lo, hi);
  if (threadIdx.x != 0) return;
  if (bad) latch_error(status, kErrNonFinite);
  double glo[3], ghi[3];
  for (int a = 0; a < 3; ++a) { glo[a] = of_ord(lo[a]); ghi[a] = of_ord(hi[a]); }
  double side = 0.0;
  for (int a = 0; a < 3; ++a) side = fmax(side, __dsub_rn(ghi[a], glo[a]));
  if (e - b <= 1 || !(side > 0.0) || !isfinite(side)) side = 1.0;
  double *g = geom + 8 * k;
  for (int a = 0; a < 3; ++a) g[a] = isfinite(glo[a]) ? glo[a] : 0.0;
  g[3] = side;
  g[4] = __ddiv_rn(2097152.0, side);
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
  // q = clamp(floor((x - lo) * scale), 0, 2^21 - 1): separate IEEE sub and mul, then
  // one floor-converting conversion (saturating; NaN gives 0) and an integer clamp
  const int q = __double2int_rd(__dmul_rn(__dsub_rn(x, lo), scale));
  return (uint32_t)min(max(q, 0), 2097151);
}

__global__ void k_keys(const double *__restrict__ pos, int64_t n, const double *__restrict__ geom0,
                       const int32_t *__restrict__ seg_of, uint64_t *__restrict__ keys,
                       uint32_t *__restrict__ idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double *geom = seg_of ? geom0 + 8 * (int64_t)seg_of[i] : geom0;   // the body's cloud
  const double scale = geom[4];
  uint32_t qx = grid_coord(pos[3 * i + 0], geom[0], scale);
  uint32_t qy = grid_coord(pos[3 * i + 1], geom[1], scale);
  uint32_t qz = grid_coord(pos[3 * i + 2], geom[2], scale);
  keys[i] = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
  idx[i] = (uint32_t)i;
}

// ------------------------------------------------------------------ a3: radix sort
// Stable LSD radix sort of (key, index) pairs, 8 passes of 8-bit digits (then, with
// several clouds, passes over the cloud id), one kernel per pass ("one sweep"):
//   * one upfront kernel counts the digits of every pass (the multiset of a pass's
//     digits does not depend on the order the earlier passes leave);
//   * in a pass, each block claims the next 2048-key tile in order, ranks its keys
//     stably (warp match on the digit, per-warp running counts, items in index
//     order), publishes its per-digit counts, and finds the counts of all earlier
//     tiles by a decoupled look-back over their published values (a bounded wait on
//     tiles not yet published: those were claimed earlier by running blocks, which
//     publish before they wait themselves, so the wait always ends);
//   * destination = digit base (scan of the pass histogram) + earlier tiles' count of
//     the digit + earlier warps' count in this tile + rank within the warp.
// Digit of element i in a pass: 8 bits of the Morton key, or, for the passes that
// order clouds, 8 bits of the cloud id of the element's caller index.
// If a look-back wait runs out (kErrTimeout is latched), that tile's destinations are
// wrong and some output slots keep older contents.  Both value buffers start the sort
// holding indices below n (the identity), and every pass writes only values read from
// its input, so the permutation still holds indices below n: the kernels that index
// with it stay in bounds and the caller gets GRAVITY_E_TIMEOUT from gravity_sync.
constexpr int kRsMaxPasses = 10;                 // 8 key passes + up to 2 cloud-id passes
constexpr uint32_t kRsFlagAgg = 1u << 30, kRsFlagPre = 2u << 30, kRsValue = (1u << 30) - 1;
constexpr int kRsSpin = 1 << 22;                 // polls allowed per tile (look-back budget)
constexpr int kRsLook = 8;                       // predecessor tiles read per look-back round

__device__ __forceinline__ unsigned rs_digit(uint64_t key, uint32_t val, int shift,
                                             const int32_t *__restrict__ seg_of) {
  if (seg_of) return ((unsigned)seg_of[val] >> shift) & 255u;
  return (unsigned)(key >> shift) & 255u;
}

// Digit counts of all passes: ghist[pass][256].
__global__ void __launch_bounds__(kRsThreads)
k_rs_count(const uint64_t *__restrict__ keys, int64_t n, int key_passes, int cloud_passes,
           const int32_t *__restrict__ seg_of, uint32_t *__restrict__ ghist,
           uint32_t *__restrict__ vinit) {
  __shared__ uint32_t cnt[kRsMaxPasses][256];
  const int np = key_passes + cloud_passes;
  for (int p = 0; p < np; ++p) cnt[p][threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)kRsThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kRsThreads) {
    const uint64_t k = keys[i];
    vinit[i] = (uint32_t)i;   // the first pass's value buffer holds indices < n throughout
    for (int p = 0; p < key_passes; ++p) atomicAdd(&cnt[p][(unsigned)(k >> (8 * p)) & 255u], 1u);
    if (cloud_passes) {
      const unsigned sg = (unsigned)seg_of[i];   // caller order: same multiset of ids
      for (int p = 0; p < cloud_passes; ++p) atomicAdd(&cnt[key_passes + p][(sg >> (8 * p)) & 255u], 1u);
    }
  }
  __syncthreads();
  for (int p = 0; p < np; ++p)
    if (cnt[p][threadIdx.x]) atomicAdd(&ghist[256 * p + threadIdx.x], cnt[p][threadIdx.x]);
}

// Morton keys (as k_keys) and the digit counts of every sort pass (as k_rs_count) in one
// read of the positions: keys[i], idx[i] = i and the first pass's other value buffer
// vinit[i] = i are written, and the counts are added to ghist.
__global__ void __launch_bounds__(kRsThreads)
k_keys_count(const double *__restrict__ pos, int64_t n, const double *__restrict__ geom0,
             const int32_t *__restrict__ seg_of, uint64_t *__restrict__ keys,
             uint32_t *__restrict__ idx, uint32_t *__restrict__ vinit, int cloud_passes,
             uint32_t *__restrict__ ghist) {
  __shared__ uint32_t cnt[kRsMaxPasses][256];
  const int np = 8 + cloud_passes;
  for (int p = 0; p < np; ++p) cnt[p][threadIdx.x] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)kRsThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kRsThreads) {
    const int sg = seg_of ? seg_of[i] : 0;
    const double *geom = geom0 + 8 * (int64_t)sg;           // the body's cloud
    const double scale = geom[4];
    const uint32_t qx = grid_coord(pos[3 * i + 0], geom[0], scale);
    const uint32_t qy = grid_coord(pos[3 * i + 1], geom[1], scale);
    const uint32_t qz = grid_coord(pos[3 * i + 2], geom[2], scale);
    const uint64_t k = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    keys[i] = k;
    idx[i] = (uint32_t)i;
    vinit[i] = (uint32_t)i;
    for (int p = 0; p < 8; ++p) atomicAdd(&cnt[p][(unsigned)(k >> (8 * p)) & 255u], 1u);
    for (int p = 0; p < cloud_passes; ++p)
      atomicAdd(&cnt[8 + p][((unsigned)sg >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int p = 0; p < np; ++p)
    if (cnt[p][threadIdx.x]) atomicAdd(&ghist[256 * p + threadIdx.x], cnt[p][threadIdx.x]);
}

// Exclusive scan of one value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v, uint32_t *s_tmp) {
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (l >= o) inc += t;
  }
  if (l == 31) s_tmp[w] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t r = 0;
    for (int ww = 0; ww < kRsThreads / 32; ++ww) { const uint32_t t = s_tmp[ww]; s_tmp[ww] = r; r += t; }
  }
  __syncthreads();
  const uint32_t ex = s_tmp[w] + inc - v;
  __syncthreads();
  return ex;
}

// 4 blocks per SM (64 registers): every 2048-key tile of a 1M-key pass is resident at once
__global__ void __launch_bounds__(kRsThreads, 4)
k_rs_sweep(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
           uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int64_t n, int shift,
           const int32_t *__restrict__ seg_of, const uint32_t *__restrict__ ghist,
           uint32_t *__restrict__ status, unsigned *__restrict__ tile_counter, int ntiles,
           unsigned *err, int spin_budget) {
  constexpr int W = kRsThreads / 32;
  __shared__ uint32_t s_w[W][256];      // per-warp digit counts, then exclusive bases
  __shared__ int32_t s_off[256];        // global position of the tile's local position 0, per digit
  __shared__ uint32_t s_tloc[256];      // tile-local exclusive digit offsets
  __shared__ uint32_t s_tmp[W];
  __shared__ uint64_t s_key[kRsTile];   // the tile in local sorted order
  __shared__ uint32_t s_val[kRsTile];
  __shared__ uint8_t s_dig[kRsTile];
  __shared__ int s_tile;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const unsigned lt = (1u << l) - 1u;
  if (tid == 0) s_tile = (int)atomicAdd(tile_counter, 1u);
  for (int ww = 0; ww < W; ++ww) s_w[ww][tid] = 0;
  __syncthreads();
  const int tile = s_tile;
  if (tile >= ntiles) return;
  // ---- stable ranks within each warp (warp w holds items [w*256, w*256 + 256) of the tile)
  const int64_t base = (int64_t)tile * kRsTile + w * (32 * kRsItems);
  uint64_t key[kRsItems];
  uint32_t val[kRsItems], pos[kRsItems];
  unsigned dig[kRsItems];
#pragma unroll
  for (int k = 0; k < kRsItems; ++k) {
    const int64_t i = base + k * 32 + l;
    const bool valid = i < n;
    key[k] = valid ? kin[i] : 0ull;
    val[k] = valid ? vin[i] : 0u;
    dig[k] = valid ? rs_digit(key[k], val[k], shift, seg_of) : 256u;
  }
#pragma unroll
  for (int k = 0; k < kRsItems; ++k) {
    const unsigned d = dig[k];
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (l == leader && d < 256u) {
      before = s_w[w][d];
      s_w[w][d] = before + __popc(peers);
    }
    before = __shfl_sync(0xffffffffu, before, leader);
    pos[k] = before + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();
  // ---- per digit (thread = digit): warp bases, tile count, publish, look back
  uint32_t run = 0;
  for (int ww = 0; ww < W; ++ww) {
    const uint32_t c = s_w[ww][tid];
    s_w[ww][tid] = run;
    run += c;
  }
  const uint32_t count = run;
  volatile uint32_t *st = status + (int64_t)tile * 256 + tid;
  // (failure testing: a negative budget -k makes the first tile publish nothing, so the
  // next tile's look-back waits on a flag that is never set until its k polls run out)
  if (tile > 0 || spin_budget > 0) *st = (tile == 0 ? kRsFlagPre : kRsFlagAgg) | count;
  // look back kRsLook tiles per round (independent loads), nearest first
  uint32_t excl = 0;
  int spin = 0;                               // one bounded budget for the whole look-back
  bool found = tile == 0;
  for (int j0 = tile - 1; !found && j0 >= 0; j0 -= kRsLook) {
    uint32_t v[kRsLook];
#pragma unroll
    for (int k = 0; k < kRsLook; ++k)
      v[k] = j0 - k >= 0 ? *(const volatile uint32_t *)(status + (int64_t)(j0 - k) * 256 + tid)
                         : kRsFlagPre;
#pragma unroll
    for (int k = 0; k < kRsLook; ++k) {
      if (found) break;
      const volatile uint32_t *sj = status + (int64_t)(j0 - k) * 256 + tid;
      while ((v[k] >> 30) == 0 && ++spin < abs(spin_budget)) v[k] = *sj;
      if ((v[k] >> 30) == 0) { atomicOr(err, kErrTimeout); found = true; break; }
      excl += v[k] & kRsValue;
      found = (v[k] >> 30) == 2u;
    }
  }
  if (tile > 0) *st = kRsFlagPre | (excl + count);
  // ---- digit bases (scan of the pass histogram) and tile-local digit offsets
  const uint32_t gbase = block_excl_scan256(ghist[tid], s_tmp);
  const uint32_t tloc = block_excl_scan256(count, s_tmp);
  s_tloc[tid] = tloc;
  s_off[tid] = (int32_t)(gbase + excl) - (int32_t)tloc;
  __syncthreads();
  // ---- local sort into shared memory, then coalesced write-out of each digit's run
#pragma unroll
  for (int k = 0; k < kRsItems; ++k) {
    const unsigned d = dig[k];
    if (d < 256u) {
      const uint32_t lp = s_tloc[d] + s_w[w][d] + pos[k];
      if (lp < (uint32_t)kRsTile) {          // always true for consistent counts
        s_key[lp] = key[k];
        s_val[lp] = val[k];
        s_dig[lp] = (uint8_t)d;
      }
    }
  }
  __syncthreads();
  const int nvalid = (int)min((int64_t)kRsTile, n - (int64_t)tile * kRsTile);
  for (int lp = tid; lp < nvalid; lp += kRsThreads) {
    const int64_t p = (int64_t)s_off[s_dig[lp]] + lp;
    if (p >= 0 && p < n) {                   // always true for consistent counts
      kout[p] = s_key[lp];
      vout[p] = s_val[lp];
    }
  }
}

// The same sort for at most one tile (n <= kRsTile): one block runs every pass in shared
// memory, ranking each pass exactly as a tile of k_rs_sweep does (warp match on the digit,
// items in index order), so the result is the same stable permutation without the
// per-pass launches and look-backs.  The (key, value) pairs are in s_key / s_val on entry
// and on exit.
struct RsSmall {
  uint32_t w[kRsThreads / 32][256];     // per-warp digit counts, then exclusive bases
  uint32_t tloc[256];                   // exclusive digit offsets of the tile
  uint32_t tmp[kRsThreads / 32];
  uint64_t key[kRsTile];
  uint32_t val[kRsTile];
};
__device__ void rs_small_passes(RsSmall &S, int n, int cloud_passes,
                                const int32_t *__restrict__ seg_of) {
  constexpr int W = kRsThreads / 32;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const unsigned lt = (1u << l) - 1u;
  const int np = 8 + cloud_passes;
  for (int pass = 0; pass < np; ++pass) {
    const bool cl = pass >= 8;
    const int shift = cl ? 8 * (pass - 8) : 8 * pass;
    for (int ww = 0; ww < W; ++ww) S.w[ww][tid] = 0;
    __syncthreads();
    uint64_t key[kRsItems];
    uint32_t val[kRsItems], pos[kRsItems];
    unsigned dig[kRsItems];
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
      const int i = w * (32 * kRsItems) + k * 32 + l;
      const bool valid = i < n;
      key[k] = valid ? S.key[i] : 0ull;
      val[k] = valid ? S.val[i] : 0u;
      dig[k] = valid ? rs_digit(key[k], val[k], shift, cl ? seg_of : nullptr) : 256u;
    }
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
      const unsigned d = dig[k];
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (l == leader && d < 256u) {
        before = S.w[w][d];
        S.w[w][d] = before + __popc(peers);
      }
      before = __shfl_sync(0xffffffffu, before, leader);
      pos[k] = before + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    uint32_t run = 0;                           // thread = digit: warp bases, tile count
    for (int ww = 0; ww < W; ++ww) {
      const uint32_t c = S.w[ww][tid];
      S.w[ww][tid] = run;
      run += c;
    }
    S.tloc[tid] = block_excl_scan256(run, S.tmp);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
      const unsigned d = dig[k];
      if (d < 256u) {
        const uint32_t lp = S.tloc[d] + S.w[w][d] + pos[k];
        if (lp < (uint32_t)kRsTile) {          // always true for consistent counts
          S.key[lp] = key[k];
          S.val[lp] = val[k];
        }
      }
    }
    __syncthreads();
  }
}

// Sort of (keys, idx) in place when n <= kRsTile (several clouds: cloud_passes > 0).
__global__ void __launch_bounds__(kRsThreads)
k_rs_small(uint64_t *__restrict__ keys, uint32_t *__restrict__ idx, int n, int cloud_passes,
           const int32_t *__restrict__ seg_of) {
  __shared__ RsSmall S;
  for (int i = threadIdx.x; i < n; i += kRsThreads) {
    S.key[i] = keys[i];
    S.val[i] = idx[i];
  }
  rs_small_passes(S, n, cloud_passes, seg_of);
  for (int i = threadIdx.x; i < n; i += kRsThreads) {
    keys[i] = S.key[i];
    idx[i] = S.val[i];
  }
}

// One cloud of n <= kRsTile bodies: root cube (as k_bbox: per-axis min / max of the
// coordinates' order-preserving integer images, the side and scale by the same IEEE
// operations, non-finite coordinates latched), Morton keys (as k_keys) and the sort, in one
// block.  The sort is a bitonic network on (key, caller index): the pairs are distinct, so
// their ascending order is exactly the stable order by key.  Thread t holds positions t
// and t + 1024 in registers; a step whose partner lies in the same warp exchanges through
// shuffles, one across warps through shared memory, and the step between the two halves
// stays in the thread.
constexpr int kOrdThreads = 1024;
static_assert(2 * kOrdThreads == kRsTile, "two positions per thread cover one tile");

__device__ __forceinline__ bool pair_gt(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
  return ka > kb || (ka == kb && va > vb);
}

// One compare-exchange of the network seen from position i (pair (k, v)), whose partner
// i ^ j holds (pk, pv), in a merge of blocks of kk positions: the lower position of an
// ascending pair keeps the smaller pair, of a descending one the larger.
__device__ __forceinline__ void bitonic_keep(int i, int j, int kk, uint64_t &k, uint32_t &v,
                                             uint64_t pk, uint32_t pv) {
  const bool take_min = ((i & j) == 0) == ((i & kk) == 0);
  if (take_min == pair_gt(k, v, pk, pv)) {
    k = pk;
    v = pv;
  }
}

// Morton key of body i (as k_keys): geom = (lo xyz, side, 2^21 / side).
__device__ __forceinline__ uint64_t morton_of(const double *__restrict__ pos, int i,
                                              const double *geom) {
  const uint32_t qx = grid_coord(pos[3 * i + 0], geom[0], geom[4]);
  const uint32_t qy = grid_coord(pos[3 * i + 1], geom[1], geom[4]);
  const uint32_t qz = grid_coord(pos[3 * i + 2], geom[2], geom[4]);
  return (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
}

__global__ void __launch_bounds__(kOrdThreads)
k_order_small(const double *__restrict__ pos, int n, double *__restrict__ geom,
              uint64_t *__restrict__ keys, uint32_t *__restrict__ idx, unsigned *status) {
  __shared__ uint64_t s_key[kRsTile];
  __shared__ uint32_t s_val[kRsTile];
  __shared__ double s_geom[5];
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
  bool bad = false;
  const unsigned long long *p64 = reinterpret_cast<const unsigned long long *>(pos);
  for (int i = threadIdx.x; i < n; i += kOrdThreads) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const unsigned long long v = p64[3 * i + a];
      bad |= ((v >> 52) & 0x7FFull) == 0x7FFull;
      const unsigned long long k = (v >> 63) ? ~v : (v | 0x8000000000000000ull);
      lo[a] = umin64(lo[a], k);
      hi[a] = umax64(hi[a], k);
    }
  }
  bad = __syncthreads_or(bad);
  block_minmax<kOrdThreads>(lo, hi);
  if (threadIdx.x == 0) {
    if (bad) latch_error(status, kErrNonFinite);
    double glo[3], ghi[3];
    for (int a = 0; a < 3; ++a) { glo[a] = of_ord(lo[a]); ghi[a] = of_ord(hi[a]); }
    double side = 0.0;
    for (int a = 0; a < 3; ++a) side = fmax(side, __dsub_rn(ghi[a], glo[a]));
    if (n <= 1 || !(side > 0.0) || !isfinite(side)) side = 1.0;
    for (int a = 0; a < 3; ++a) s_geom[a] = geom[a] = isfinite(glo[a]) ? glo[a] : 0.0;
    s_geom[3] = geom[3] = side;
    s_geom[4] = geom[4] = __ddiv_rn(2097152.0, side);   // 2^21 / side, one IEEE division
  }
  __syncthreads();
  const int t = threadIdx.x, tb = t + kOrdThreads;
  uint64_t ka = ~0ull, kb = ~0ull;             // positions t and tb; pads sort last
  uint32_t va = ~0u, vb = ~0u;
  if (t < n) { ka = morton_of(pos, t, s_geom); va = (uint32_t)t; }
  if (tb < n) { kb = morton_of(pos, tb, s_geom); vb = (uint32_t)tb; }
  const bool upper = n > kOrdThreads;           // the upper half holds only pads otherwise
  int p2 = 1;
  while (p2 < n) p2 <<= 1;
  for (int kk = 2; kk <= p2; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      if (j == kOrdThreads) {                   // positions t and tb: ascending (kk = 2048)
        if (pair_gt(ka, va, kb, vb)) {
          const uint64_t tk = ka; ka = kb; kb = tk;
          const uint32_t tv = va; va = vb; vb = tv;
        }
      } else if (j >= 32) {                     // partner in another warp
        s_key[t] = ka; s_val[t] = va;
        if (upper) { s_key[tb] = kb; s_val[tb] = vb; }
        __syncthreads();
        const uint64_t pka = s_key[t ^ j];
        const uint32_t pva = s_val[t ^ j];
        uint64_t pkb = 0ull;
        uint32_t pvb = 0u;
        if (upper) { pkb = s_key[tb ^ j]; pvb = s_val[tb ^ j]; }
        __syncthreads();
        bitonic_keep(t, j, kk, ka, va, pka, pva);
        if (upper) bitonic_keep(tb, j, kk, kb, vb, pkb, pvb);
      } else {                                  // partner in this warp
        const uint64_t pka = __shfl_xor_sync(0xffffffffu, ka, j);
        const uint32_t pva = __shfl_xor_sync(0xffffffffu, va, j);
        bitonic_keep(t, j, kk, ka, va, pka, pva);
        if (upper) {
          const uint64_t pkb = __shfl_xor_sync(0xffffffffu, kb, j);
          const uint32_t pvb = __shfl_xor_sync(0xffffffffu, vb, j);
          bitonic_keep(tb, j, kk, kb, vb, pkb, pvb);
        }
      }
    }
  }
  if (t < n) { keys[t] = ka; idx[t] = va; }
  if (tb < n) { keys[tb] = kb; idx[tb] = vb; }
}

// 8 passes over the 63-bit keys, then (several clouds) stable passes over the cloud
// ids, so the order is by cloud, then key, then caller index.  Sorts (keys, idx) in
// place; keys_alt / idx_alt are the other halves of the ping-pong, hist the counts
// and tile states (257 * kRsMaxPasses + passes * tiles * 256 words).
// With counted, the caller has cleared hist (radix_sort_clear) and launched k_keys_count,
// which gives the keys, the identity value buffers and the digit counts.
int radix_sort_clear(Ctx *c, int64_t n, uint32_t *hist, int cloud_passes,
                     int64_t extra_zero_words) {
  const int ntiles = (int)((n + kRsTile - 1) / kRsTile);
  const int np = 8 + cloud_passes;
  GRAV_CUDA_TRY(cudaMemsetAsync(hist, 0,
                                sizeof(uint32_t) * ((size_t)(256 + 1) * kRsMaxPasses +
                                                    (size_t)np * ntiles * 256 +
                                                    (size_t)extra_zero_words), c->stream));
  return GRAVITY_OK;
}

int radix_sort_buffers(Ctx *c, int64_t n, uint64_t *keys, uint64_t *keys_alt, uint32_t *idx,
                       uint32_t *idx_alt, uint32_t *hist, int cloud_passes,
                       const int32_t *seg_of, int64_t extra_zero_words, bool counted = false) {
  const int ntiles = (int)((n + kRsTile - 1) / kRsTile);
  uint64_t *ka = keys, *kb = keys_alt;
  uint32_t *va = idx, *vb = idx_alt;
  const int np = 8 + cloud_passes;
  // hist: [kRsMaxPasses][256] digit counts, [kRsMaxPasses] tile counters,
  // then [kRsMaxPasses][ntiles][256] published tile counts
  uint32_t *ghist = hist, *counters = hist + 256 * kRsMaxPasses;
  uint32_t *status = counters + kRsMaxPasses;
  if (!counted) {
    const int rc = radix_sort_clear(c, n, hist, cloud_passes, extra_zero_words);
    if (rc) return rc;
  }
  if (n <= kRsTile && c->sort_stall == 0) {   // one tile: every pass in one block
    k_rs_small<<<1, kRsThreads, 0, c->stream>>>(keys, idx, (int)n, cloud_passes, seg_of);
    ++c->launches;
    return cuda_status(cudaGetLastError());
  }
  if (!counted) {
    int cb = (int)((n + kRsThreads - 1) / kRsThreads);
    if (cb > 2 * c->num_sms) cb = 2 * c->num_sms;
    k_rs_count<<<cb, kRsThreads, 0, c->stream>>>(keys, n, 8, cloud_passes, seg_of, ghist, vb);
    ++c->launches;
  }
  for (int pass = 0; pass < np; ++pass) {
    const bool cl = pass >= 8;
    const int shift = cl ? 8 * (pass - 8) : 8 * pass;
    const int32_t *so = cl ? seg_of : nullptr;
    k_rs_sweep<<<ntiles, kRsThreads, 0, c->stream>>>(ka, va, kb, vb, n, shift, so,
                                                     ghist + 256 * pass,
                                                     status + (int64_t)pass * ntiles * 256,
                                                     counters + pass, ntiles, c->d_status,
                                                     c->sort_stall > 0 ? -c->sort_stall : kRsSpin);
    ++c->launches;
    uint64_t *tk = ka; ka = kb; kb = tk;
    uint32_t *tv = va; va = vb; vb = tv;
  }
  if (np % 2) {                               // odd pass count: move the result back
    GRAV_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, c->stream));
    GRAV_CUDA_TRY(cudaMemcpyAsync(idx, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, c->stream));
  }
  return cuda_status(cudaGetLastError());
}

// The octree scan's tile counter and tile states sit in the sort's count buffer right after
// the sort's own words, so the sort's clearing memset clears them too.
int64_t oct_scan_words(int64_t n) { return (n + kOctTile - 1) / kOctTile + 1; }
uint32_t *oct_scan_state(Ctx *c, int64_t n) {
  const int np = 8 + (c->seg.nseg > 1 ? (c->seg.cbits + 7) / 8 : 0);
  const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
  return c->t.hist + (int64_t)(256 + 1) * kRsMaxPasses + (int64_t)np * ntiles * 256;
}

int radix_sort(Ctx *c, int64_t n, bool counted) {
  Tree &t = c->t;
  const int cloud_passes = c->seg.nseg > 1 ? (c->seg.cbits + 7) / 8 : 0;
  return radix_sort_buffers(c, n, t.keys, t.keys_alt, t.idx, t.idx_alt, t.hist, cloud_passes,
                            c->seg.seg_of, oct_scan_words(n), counted);
}

// Launch of k_bbox over one cloud of n bodies (grid a multiple of 3, see k_bbox).
void launch_bbox(Ctx *c, const double *pos, int64_t n, unsigned long long *part,
                 unsigned *ticket, double *geom) {
  int64_t nb64 = (3 * n + 4 * kBBoxThreads - 1) / (4 * kBBoxThreads);
  if (nb64 > 4 * (int64_t)c->num_sms) nb64 = 4 * (int64_t)c->num_sms;
  nb64 = (nb64 + 2) / 3 * 3;
  int nb = (int)nb64;
  if (nb < 1) nb = 1;
  k_bbox<<<nb, kBBoxThreads, 0, c->stream>>>(pos, n, part, ticket, geom, c->d_status);
  ++c->launches;
}

// ------------------------------------------------------------------ moment buckets
// The moment pass takes nodes bucketed so that every warp's lanes run equal loops:
// leaves by body count (1 .. 16 and more), then internal nodes by depth, deepest first.
// The octree write counts the buckets; t.scalars holds, from kSlotCnt, the bucket
// counts, fill cursors, the moment pass's done counters and its ticket (cleared by the
// gather of each build), then the bucket offsets.  Word 0 is the octree total.
constexpr int kLeafBuckets = 17;
constexpr int kBuckets = kLeafBuckets + kLevels;   // + internal depths 20 .. 0
constexpr int kSlotCnt = 1, kSlotFill = 40, kSlotDone = 80, kSlotTicket = 120, kSlotOff = 128;
static_assert(kSlotCnt + kBuckets <= kSlotFill && kSlotFill + kBuckets <= kSlotDone &&
              kSlotOff - kSlotCnt <= 256, "scalar slots");

__device__ __forceinline__ int bucket_of(int4 t, int depth) {
  const int b = t.x < 0 ? min(t.w - t.z, kLeafBuckets) - 1 : kLeafBuckets + (kLevels - 1 - depth);
  return min(max(b, 0), kBuckets - 1);
}

// ------------------------------------------------------------------ a4: gather
// (block 0 also clears the moment pass's counters, slots [kSlotCnt, kSlotOff))
__global__ void k_gather(const double *__restrict__ pos, const double *__restrict__ mass,
                         const uint32_t *__restrict__ perm, int64_t n, double *__restrict__ pos_s,
                         double *__restrict__ mass_s, float4 *__restrict__ bhi,
                         float4 *__restrict__ blo, const int32_t *__restrict__ seg_of,
                         int32_t *__restrict__ seg_sorted, uint32_t *__restrict__ slots) {
  if (blockIdx.x == 0 && threadIdx.x < kSlotOff - kSlotCnt) slots[kSlotCnt + threadIdx.x] = 0;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t j = perm[i];
  if (seg_of) seg_sorted[i] = seg_of[j];
  double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2], m = mass[j];
  pos_s[3 * i] = x; pos_s[3 * i + 1] = y; pos_s[3 * i + 2] = z;
  mass_s[i] = m;
  float xh, xl, yh, yl, zh, zl;
  split_df(x, xh, xl); split_df(y, yh, yl); split_df(z, zh, zl);
  bhi[i] = make_float4(xh, yh, zh, __double2float_rn(m));
  blo[i] = make_float4(xl, yl, zl, 0.0f);
}

// ------------------------------------------------------------------ a5: binary radix tree
// Extended key of sorted position i: (cloud id [cbits bits], 63-bit key, i).  delta
// is the common prefix length in bits of two extended keys; -1 outside [0, n).
// With one cloud cbits = 0 and the cloud part is absent.
struct KeyView {
  const uint64_t *k;
  const int32_t *seg;          // cloud of each sorted body, or nullptr (one cloud)
  int cbits;
  int n;
};

__device__ __forceinline__ int delta(const KeyView &v, int i, int j) {
  if (j < 0 || j >= v.n) return -1;
  if (v.seg) {
    const int si = v.seg[i], sj = v.seg[j];
    if (si != sj) return __clz(si ^ sj) - (32 - v.cbits);
  }
  const uint64_t a = v.k[i], b = v.k[j];
  if (a != b) return v.cbits + __clzll((long long)(a ^ b)) - 1;   // keys use 63 bits
  return v.cbits + 63 + __clz((int)((unsigned)i ^ (unsigned)j));
}

// Karras' parallel construction: internal node i covers a key range with one end
// at i; its direction, extent and split follow from prefix-length comparisons.
__global__ void k_radix_tree(KeyView v, int32_t *__restrict__ child, int32_t *__restrict__ parent,
                             int32_t *__restrict__ first, int32_t *__restrict__ last,
                             int32_t *__restrict__ plen) {
  const int n = v.n;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int dir = (delta(v, i, i + 1) - delta(v, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(v, i, i - dir);
  int lmax = 2;
  while (delta(v, i, i + lmax * dir) > dmin) lmax <<= 1;
  int len = 0;
  for (int t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(v, i, i + (len + t) * dir) > dmin) len += t;
  int j = i + len * dir;
  int dnode = delta(v, i, j);
  int s = 0;
  for (int div = 2;; div <<= 1) {
    int t = (len + div - 1) / div;
    if (delta(v, i, i + (s + t) * dir) > dnode) s += t;
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
// A binary node X is an octree cell when its capped depth floor((plen - cbits)/3)
// exceeds its binary parent's (or X is a cloud root): the cell at that depth holds
// exactly X's bodies, i.e. X is the deepest member of a chain of single-child
// cells.  A cell is internal when it holds > leaf_max bodies and is above depth 21.
// Its octree children are the first binary descendants whose prefix reaches
// cbits + 3(depth+1) bits (or bodies), found by a DFS of at most 7 binary nodes, in
// key = octant order.  With several clouds, binary nodes whose prefix is shorter
// than the cloud bits only connect clouds; their children just below are the cloud
// roots, which take octree node ids 0 .. nclouds-1.
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

__device__ __forceinline__ int cdepth(int plen, int cbits) {
  return plen < cbits ? -1 : cap_depth(plen - cbits);
}

// Children count of every binary node (0 unless it is an internal octree cell), fused with
// the exclusive scan that gives each cell the first octree id of its children: each block
// claims the next tile of kOctTile binary nodes in order (ITEMS consecutive nodes per thread:
// 4 for many tiles, 1 for a few, where the latency of each thread's chain of dependent loads
// is the kernel's time), scans it,
// publishes its total, and its first warp finds the sum of the earlier tiles by a decoupled
// look-back, 32 predecessors per round (a bounded wait on tiles not yet published: those
// were claimed earlier by running blocks, which publish before they wait themselves).  The
// last tile writes the grand total (octree nodes below the cloud roots).
constexpr uint32_t kOsAgg = 1u << 30, kOsPre = 2u << 30, kOsValue = (1u << 30) - 1;
constexpr int kOsSpin = 1 << 22;

__device__ __forceinline__ uint32_t oct_children(int X, int n, int leaf_max, int cbits,
                                                 const int32_t *__restrict__ child,
                                                 const int32_t *__restrict__ parent,
                                                 const int32_t *__restrict__ first,
                                                 const int32_t *__restrict__ last,
                                                 const int32_t *__restrict__ plen,
                                                 unsigned *status) {
  const int px = plen[X];
  const int P = parent[X];
  if (P >= n - 1) {                                     // only after a failed sort pass
    latch_error(status, kErrTree);
    return 0;
  }
  if (px < cbits) return 0;                             // connector between clouds
  const int d = cdepth(px, cbits);
  const bool cell = P < 0 || plen[P] < cbits || cdepth(plen[P], cbits) < d;
  const int count = last[X] - first[X] + 1;
  if (!(cell && count > leaf_max && d < kLevels)) return 0;
  Frontier f;
  if (!frontier(child, plen, X, cbits + 3 * (d + 1), f) || f.count < 2) {
    latch_error(status, kErrTree);
    return 0;
  }
  return (uint32_t)f.count;
}

template <int ITEMS>
__global__ void __launch_bounds__(kOctTile / ITEMS)
k_oct_count(int n, int leaf_max, int cbits, const int32_t *__restrict__ child,
            const int32_t *__restrict__ parent, const int32_t *__restrict__ first,
            const int32_t *__restrict__ last, const int32_t *__restrict__ plen,
            uint32_t *__restrict__ nchild, uint32_t *__restrict__ base, uint32_t *__restrict__ total,
            uint32_t *__restrict__ tstate, unsigned *__restrict__ tile_counter, int ntiles,
            unsigned *status) {
  __shared__ int s_tile;
  constexpr int kOctThreads = kOctTile / ITEMS;
  __shared__ uint32_t s_warp[kOctThreads / 32];
  __shared__ uint32_t s_excl;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_counter, 1u);
  __syncthreads();
  const int tile = s_tile;
  if (tile >= ntiles) return;
  const int X0 = tile * kOctTile + threadIdx.x * ITEMS;   // ITEMS consecutive nodes
  uint32_t cnt[ITEMS], sum = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int X = X0 + k;
    cnt[k] = X < n - 1 ? oct_children(X, n, leaf_max, cbits, child, parent, first, last, plen,
                                      status) : 0u;
    if (X < n - 1) nchild[X] = cnt[k];
    sum += cnt[k];
  }
  // block-wide exclusive scan of the threads' sums
  const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (l >= o) inc += t;
  }
  if (l == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t r = 0;
    if (l == 0) {
      for (int ww = 0; ww < kOctThreads / 32; ++ww) { const uint32_t t = s_warp[ww]; s_warp[ww] = r; r += t; }
      *(volatile uint32_t *)(tstate + tile) = (tile == 0 ? kOsPre : kOsAgg) | r;
    }
    r = __shfl_sync(0xffffffffu, r, 0);
    // look back 32 tiles per round: lane j reads tile j0 - j
    uint32_t excl = 0;
    int spin = 0;
    bool done = tile == 0;
    for (int j0 = tile - 1; !done; j0 -= 32) {
      const int j = j0 - l;
      uint32_t v = j >= 0 ? *(const volatile uint32_t *)(tstate + j) : kOsPre;
      // the nearest predecessor with a prefix; wait until every nearer one has published
      for (;;) {
        const unsigned pre = __ballot_sync(0xffffffffu, (v >> 30) == 2u);
        const int lim = pre ? __ffs(pre) - 1 : 31;      // lanes 0 .. lim are needed
        const bool miss = l <= lim && (v >> 30) == 0u;
        if (!__any_sync(0xffffffffu, miss)) {
          uint32_t add = l <= lim ? (v & kOsValue) : 0u;
          for (int o = 16; o > 0; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
          excl += add;
          done = pre != 0u;
          break;
        }
        if (++spin >= kOsSpin) {
          if (l == 0) latch_error(status, kErrTimeout);
          done = true;
          break;
        }
        if (miss) v = *(const volatile uint32_t *)(tstate + j);
      }
    }
    if (l == 0) {
      if (tile > 0) *(volatile uint32_t *)(tstate + tile) = kOsPre | (excl + r);
      if (tile == ntiles - 1) *total = excl + r;
      s_excl = excl;
    }
  }
  __syncthreads();
  uint32_t pre = s_excl + s_warp[w] + inc - sum;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int X = X0 + k;
    if (X < n - 1) base[X] = pre;
    pre += cnt[k];
  }
}

struct OctWriteArgs {
  int n, leaf_max, cbits, nseg, cap_nodes;
  const int32_t *child, *first, *last, *plen, *seg_sorted;
  const uint32_t *nchild, *base, *total;
  int4 *topo;
  int32_t *depth, *nnodes, *nparent;
  uint32_t *slots;             // moment bucket counts at kSlotCnt (cleared by the gather)
  unsigned *status;
};

// Parent of the octree children of binary node c (an internal octree cell written at
// octree id `id`): its children take ids nseg + base[c] .. + nchild[c] - 1.
__device__ __forceinline__ void write_parent_of_children(const OctWriteArgs &A, int c, int id) {
  const int n0 = A.nseg + (int)A.base[c], cnt = (int)A.nchild[c];
  if (n0 < A.nseg || n0 + cnt > A.cap_nodes) { latch_error(A.status, kErrTree); return; }
  for (int j = 0; j < cnt; ++j) A.nparent[n0 + j] = id;
}

// Node record (topology, depth) at octree id `id`, counted in its moment bucket (cnt: the
// block's counters in shared memory).
__device__ __forceinline__ void put_node(const OctWriteArgs &A, int id, int4 t, int depth,
                                         uint32_t *cnt) {
  A.topo[id] = t;
  A.depth[id] = depth;
  atomicAdd(&cnt[bucket_of(t, depth)], 1u);
}

// Record of a cloud root (binary internal node c, or body ~c) at octree id `id`.
__device__ __forceinline__ void write_root(const OctWriteArgs &A, int c, int id, uint32_t *cnt) {
  A.nparent[id] = -1;
  if (c < 0) {
    const int b = ~c;
    put_node(A, id, make_int4(-1, 0, b, b + 1), 0, cnt);
    return;
  }
  const int b = A.first[c], e = A.last[c] + 1;
  if (A.nchild[c] > 0) {
    put_node(A, id, make_int4(A.nseg + (int)A.base[c], (int)A.nchild[c], b, e),
             cdepth(A.plen[c], A.cbits), cnt);
    write_parent_of_children(A, c, id);
  } else {
    put_node(A, id, make_int4(-1, 0, b, e), (e - b <= A.leaf_max) ? 0 : kLevels, cnt);
  }
}

__device__ void oct_write_node(const OctWriteArgs &A, int X, uint32_t *cnt) {
  if (A.plen[X] < A.cbits) {                              // connector: place the cloud roots below
    for (int h = 0; h < 2; ++h) {
      const int c = A.child[2 * X + h];
      if (c < 0 || A.plen[c] >= A.cbits) {
        const int b = c < 0 ? ~c : A.first[c];
        write_root(A, c, A.seg_sorted[b], cnt);
      }
    }
    return;
  }
  if (A.nchild[X] == 0) return;
  const int d = cdepth(A.plen[X], A.cbits);
  Frontier f;
  frontier(A.child, A.plen, X, A.cbits + 3 * (d + 1), f);
  const int id0 = A.nseg + (int)A.base[X];
  if (id0 + f.count > A.cap_nodes) { latch_error(A.status, kErrTree); return; }
  for (int k = 0; k < f.count; ++k) {
    const int c = f.item[k], id = id0 + k;
    if (c < 0) {
      const int b = ~c;
      put_node(A, id, make_int4(-1, 0, b, b + 1), d + 1, cnt);
    } else {
      const int b = A.first[c], e = A.last[c] + 1;
      if (A.nchild[c] > 0) {
        put_node(A, id, make_int4(A.nseg + (int)A.base[c], (int)A.nchild[c], b, e),
                 cdepth(A.plen[c], A.cbits), cnt);
        write_parent_of_children(A, c, id);
      } else {
        put_node(A, id, make_int4(-1, 0, b, e), (e - b <= A.leaf_max) ? d + 1 : kLevels, cnt);
      }
    }
  }
}

// Writes the octree records: each binary node that starts an octree cell writes the
// records of that cell's children (and the parent of their children), counting every
// node in its moment bucket (per block in shared memory, then added to the global counts).
__global__ void __launch_bounds__(256) k_oct_write(OctWriteArgs A) {
  __shared__ uint32_t cnt[kBuckets];
  if (threadIdx.x < kBuckets) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int X = blockIdx.x * blockDim.x + threadIdx.x;
  if (X == 0) {
    int nn = A.nseg + (int)*A.total;
    if (nn > A.cap_nodes) { latch_error(A.status, kErrTree); nn = A.nseg; }
    *A.nnodes = nn;
    if (A.cbits == 0) write_root(A, 0, 0, cnt);           // one cloud: binary node 0 is the root
  }
  if (X < A.n - 1) oct_write_node(A, X, cnt);
  __syncthreads();
  if (threadIdx.x < kBuckets && cnt[threadIdx.x])
    atomicAdd(&A.slots[kSlotCnt + threadIdx.x], cnt[threadIdx.x]);
}

// ------------------------------------------------------------------ a7: moments
// Eq. (COMinternal): m = sum of child masses; COM = (sum of child COM * child mass)
// / m, children in octant order; a leaf of several bodies sums them in sorted
// order; a one-body leaf is the body (its mass and position).  FP64 with explicit
// IEEE roundings (no contraction) so m and COM are reproducible bit for bit.
// Quadrupole (order 2): the second moment T = sum m y y^T about the node's COM is
// carried up with the parallel-axis rule T_p = sum_c (T_c + m_c d_c d_c^T),
// d_c = COM_c - COM_p (an FP64 difference); the walk uses the traceless
// Q = 3 T - tr(T) I, identical in exact arithmetic to sum m (3 y y^T - |y|^2 I).
// The products and sums of T run in double-float arithmetic (Dbl2 below, ~47
// significant bits), not FP64: on GB300 an FP32 warp instruction issues in one cycle
// of a sub-partition and an FP64 one holds its unit ~64 cycles, so this halves the
// pass's FP64 instructions; T stays within ~1e-14 m l^2 of the FP64 value.
//
// GB300's FP64 pipe costs the same per warp instruction however many lanes are
// active, so the pass runs on full, uniform warps: nodes are counting-sorted into
// buckets (leaves by body count 1 .. 16 and more, so that the lanes of a warp loop
// equally long; then internal nodes by depth, deepest first); one launch does the
// leaves, one more every internal depth, each after the deeper ones (k_level_moments).
constexpr int kMomBlocksPerSM = 1;             // internal levels: one warp per SM sub-partition

struct MomArgs {
  const int4 *topo;
  const int32_t *ndepth;
  const int32_t *nnodes;
  const int32_t *nlist;
  const uint32_t *boff;
  const double *pos_s;
  const double *mass_s;
  const double *geom;
  const int32_t *seg_sorted;   // cloud of each sorted body, or nullptr (one cloud)
  double *nmass;
  double *ncom;
  float4 *nsec;                // second moments T, double-float (hi, lo) pairs, 3 per node:
                               // (xx, yy), (zz, xy), (xz, yz)
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

// A double-float value hi + lo (two FP32 numbers, |lo| <= ulp(hi) / 2 after every
// operation).  The operations are the classical error-free transforms (Dekker's
// product through a fused multiply-add, Knuth's two-sum) with explicit roundings, so
// no contraction can break them.
struct Dbl2 {
  float hi, lo;
};

// x as hi + lo from its FP64 bit fields, on the integer units (no FP64 instruction):
// hi = the leading 24 significant bits, lo = the next ones of the remaining 29,
// truncated to 24; |x - hi - lo| < 2^-47 |x|.  A lo below FP32's normal range is
// dropped; outside that range for hi (|x| < 2^-126 or >= 2^128), hi = x rounded to
// FP32 and lo = 0.
__device__ __forceinline__ Dbl2 dbl2_split(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)(u >> 52) & 0x7FF;
  if (e < 897 || e > 1150) return {__double2float_rn(x), 0.f};
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const float hi =
      __uint_as_float(sign | ((uint32_t)(e - 896) << 23) | ((uint32_t)(u >> 29) & 0x7FFFFFu));
  const uint32_t low = (uint32_t)u & 0x1FFFFFFFu;       // weight of bit 0: 2^(e - 1075)
  float lo = 0.f;
  if (low) {
    const int p = 31 - __clz(low);                     // leading bit of the low part
    const uint32_t mant = p >= 23 ? low >> (p - 23) : low << (23 - p);
    const int be = e - 948 + p;                        // FP32 biased exponent
    if (be > 0) lo = __uint_as_float(sign | ((uint32_t)be << 23) | (mant & 0x7FFFFFu));
  }
  return {hi, lo};
}

__device__ __forceinline__ Dbl2 dbl2_mul(Dbl2 a, Dbl2 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);                 // exact error of p
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(p, e);
  return {s, __fsub_rn(e, __fsub_rn(s, p))};
}

__device__ __forceinline__ Dbl2 dbl2_add(Dbl2 a, Dbl2 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));   // exact error of s
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

// T (6 double-float entries) to and from its 3 float4 records.
__device__ __forceinline__ void store_sec(float4 *dst, const Dbl2 *T) {
  dst[0] = make_float4(T[0].hi, T[0].lo, T[1].hi, T[1].lo);
  dst[1] = make_float4(T[2].hi, T[2].lo, T[3].hi, T[3].lo);
  dst[2] = make_float4(T[4].hi, T[4].lo, T[5].hi, T[5].lo);
}


// Scatter node ids into their buckets (order inside a bucket is irrelevant: every
// node is computed from its children only).
__global__ void k_bucket_fill(const int4 *__restrict__ topo, const int32_t *__restrict__ ndepth,
                              const int32_t *__restrict__ nnodes, int cap_nodes,
                              uint32_t *__restrict__ slots, int32_t *__restrict__ nlist) {
  __shared__ uint32_t cnt[kBuckets], base[kBuckets], off[kBuckets + 1];
  if (threadIdx.x < kBuckets) cnt[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    off[0] = 0;
    for (int b = 0; b < kBuckets; ++b) off[b + 1] = off[b] + slots[kSlotCnt + b];
    if (blockIdx.x == 0)
      for (int b = 0; b <= kBuckets; ++b) slots[kSlotOff + b] = off[b];
  }
  __syncthreads();
  const int id = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = min(*nnodes, cap_nodes);
  int b = 0;
  uint32_t local = 0;
  if (id < nn) {
    b = bucket_of(topo[id], ndepth[id]);
    local = atomicAdd(&cnt[b], 1u);
  }
  __syncthreads();
  if (threadIdx.x < kBuckets && cnt[threadIdx.x])
    base[threadIdx.x] = atomicAdd(&slots[kSlotFill + threadIdx.x], cnt[threadIdx.x]);
  __syncthreads();
  if (id < nn) nlist[off[b] + base[b] + local] = id;
}

// Quadrupole record: Q in double-float, then rounded to FP32 (the hi part of a
// normalised pair), stored negated.
__device__ void write_quad_record(const MomArgs &A, int id, const Dbl2 *T) {
  const Dbl2 tr = dbl2_add(dbl2_add(T[0], T[1]), T[2]), ntr = {-tr.hi, -tr.lo};
  const Dbl2 three = {3.f, 0.f};
  float q[6];
#pragma unroll
  for (int a = 0; a < 3; ++a) q[a] = dbl2_add(dbl2_mul(three, T[a]), ntr).hi;
#pragma unroll
  for (int a = 3; a < 6; ++a) q[a] = dbl2_mul(three, T[a]).hi;
  A.quadf[2 * id] = make_float4(-q[0], -q[1], -q[2], -q[3]);
  A.quadf[2 * id + 1] = make_float4(-q[4], -q[5], 0.f, 0.f);
}

// Walk records: (COM hi, m) and (COM lo, l^2); l^2 = -1 marks a one-body leaf
// (always a body-to-body term).  Quadrupole record: -Q = -(3T - tr(T) I) as FP32 (the
// walk's term is written with the negated tensor, which needs no negation there).
__device__ void write_records(const MomArgs &A, int id, double m, const double *com,
                              const Dbl2 *T, bool single_body) {
  float h[3], lo[3];
  for (int a = 0; a < 3; ++a) split_df(com[a], h[a], lo[a]);
  const int4 t = A.topo[id];
  const double side = A.geom[8 * (A.seg_sorted ? A.seg_sorted[t.z] : 0) + 3];
  double l = __dmul_rn(side, pow2_neg(A.ndepth[id]));
  float l2 = single_body ? -1.0f : __double2float_rn(dm(l, l));
  A.rec0[id] = make_float4(h[0], h[1], h[2], __double2float_rn(m));
  A.rec1[id] = make_float4(lo[0], lo[1], lo[2], l2);
  if (A.order >= 2) write_quad_record(A, id, T);
}

// Moments of one leaf from its bodies, in body order (mass, then m x, COM = sum / mass,
// then the second moments about the COM).
__device__ void leaf_node(const MomArgs &A, int id) {
  const int4 t = A.topo[id];
  if (t.z < 0 || t.w > A.n || t.z >= t.w) { latch_error(A.status, kErrTree); return; }
  double msum, com[3];
  Dbl2 T[6] = {};
  if (t.w - t.z == 1) {
    msum = A.mass_s[t.z];
    for (int a = 0; a < 3; ++a) com[a] = A.pos_s[3 * t.z + a];
  } else {
    double sx = 0.0, sy = 0.0, sz = 0.0;
    msum = 0.0;
    for (int i = t.z; i < t.w; ++i) {
      const double mi = A.mass_s[i];
      msum = da(msum, mi);
      sx = da(sx, dm(mi, A.pos_s[3 * i]));
      sy = da(sy, dm(mi, A.pos_s[3 * i + 1]));
      sz = da(sz, dm(mi, A.pos_s[3 * i + 2]));
    }
    com[0] = __ddiv_rn(sx, msum); com[1] = __ddiv_rn(sy, msum); com[2] = __ddiv_rn(sz, msum);
    if (A.order >= 2) {
      for (int i = t.z; i < t.w; ++i) {
        const Dbl2 mi = dbl2_split(A.mass_s[i]);
        const Dbl2 y0 = dbl2_split(ds(A.pos_s[3 * i], com[0])),
                   y1 = dbl2_split(ds(A.pos_s[3 * i + 1], com[1])),
                   y2 = dbl2_split(ds(A.pos_s[3 * i + 2], com[2]));
        const Dbl2 m0 = dbl2_mul(mi, y0), m1 = dbl2_mul(mi, y1), m2 = dbl2_mul(mi, y2);
        T[0] = dbl2_add(T[0], dbl2_mul(m0, y0)); T[1] = dbl2_add(T[1], dbl2_mul(m1, y1));
        T[2] = dbl2_add(T[2], dbl2_mul(m2, y2)); T[3] = dbl2_add(T[3], dbl2_mul(m0, y1));
        T[4] = dbl2_add(T[4], dbl2_mul(m0, y2)); T[5] = dbl2_add(T[5], dbl2_mul(m1, y2));
      }
    }
  }
  A.nmass[id] = msum;
  for (int a = 0; a < 3; ++a) A.ncom[3 * id + a] = com[a];
  if (A.order >= 2) store_sec(A.nsec + 3 * id, T);
  write_records(A, id, msum, com, T, t.w - t.z == 1);
}

// An internal node from its children, combined in octant order (tp = its topology
// record).  All children's values are loaded up front (at most 8 children: independent
// loads in flight together), through L2: they were written by other warps of the same
// launch, and an SM's L1 may hold an older copy of their cache lines.
__device__ void internal_node(const MomArgs &A, int id, int4 tp, int nn) {
  if (tp.x <= 0 || tp.y > 8 || tp.x + tp.y > nn) { latch_error(A.status, kErrTree); return; }
  double cm[8], cx[8], cy[8], cz[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const bool in = j < tp.y;
    const int c = in ? tp.x + j : tp.x;
    cm[j] = in ? __ldcg(A.nmass + c) : 0.0;
    cx[j] = __ldcg(A.ncom + 3 * c); cy[j] = __ldcg(A.ncom + 3 * c + 1);
    cz[j] = __ldcg(A.ncom + 3 * c + 2);
  }
  double pm = 0.0, px = 0.0, py = 0.0, pz = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (j < tp.y) {
      pm = da(pm, cm[j]);
      px = da(px, dm(cx[j], cm[j]));
      py = da(py, dm(cy[j], cm[j]));
      pz = da(pz, dm(cz[j], cm[j]));
    }
  }
  const double pc[3] = {__ddiv_rn(px, pm), __ddiv_rn(py, pm), __ddiv_rn(pz, pm)};
  Dbl2 T[6] = {};
  if (A.order >= 2) {
#pragma unroll
    for (int h = 0; h < 8; h += 4) {
      float4 Tc[4][3];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = (h + j < tp.y) ? tp.x + h + j : tp.x;
#pragma unroll
        for (int q = 0; q < 3; ++q) Tc[j][q] = __ldcg(A.nsec + 3 * c + q);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (h + j < tp.y) {
          const Dbl2 mc = dbl2_split(cm[h + j]);
          const Dbl2 d0 = dbl2_split(ds(cx[h + j], pc[0])), d1 = dbl2_split(ds(cy[h + j], pc[1])),
                     d2 = dbl2_split(ds(cz[h + j], pc[2]));
          const Dbl2 m0 = dbl2_mul(mc, d0), m1 = dbl2_mul(mc, d1), m2 = dbl2_mul(mc, d2);
          const Dbl2 t[6] = {dbl2_mul(m0, d0), dbl2_mul(m1, d1), dbl2_mul(m2, d2),
                             dbl2_mul(m0, d1), dbl2_mul(m0, d2), dbl2_mul(m1, d2)};
          const Dbl2 tc[6] = {{Tc[j][0].x, Tc[j][0].y}, {Tc[j][0].z, Tc[j][0].w},
                              {Tc[j][1].x, Tc[j][1].y}, {Tc[j][1].z, Tc[j][1].w},
                              {Tc[j][2].x, Tc[j][2].y}, {Tc[j][2].z, Tc[j][2].w}};
#pragma unroll
          for (int a = 0; a < 6; ++a) T[a] = dbl2_add(T[a], dbl2_add(tc[a], t[a]));
        }
      }
    }
  }
  A.nmass[id] = pm;
  for (int a = 0; a < 3; ++a) A.ncom[3 * id + a] = pc[a];
  if (A.order >= 2) store_sec(A.nsec + 3 * id, T);
  write_records(A, id, pm, pc, T, false);
}

// The same node computed by a group of 8 lanes (lane j of the group holds child j), for
// depths with few nodes.  The products m_c x_c run once per child, in parallel; every lane
// of the group then folds them in octant order with the same IEEE operations as
// internal_node, so m and COM are bitwise the same; lanes 0-2 of the group divide one COM
// component each and split it for the record; the second moments are summed over the
// group by a butterfly (another rounding order than internal_node's, the same ~1e-14 m l^2
// accuracy).  About half the FP64 instructions of a 32-node unit, for 4 nodes: the form
// pays when a depth's groups fit one warp per SM sub-partition.  Every lane of the warp
// calls this (full-warp shuffles); valid is false in lanes of a group with no node.
__device__ void internal_node_group(const MomArgs &A, int id, int4 tp, bool valid, int nn) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31, j = lane & 7, base = lane & ~7;
  if (valid && (tp.x <= 0 || tp.y > 8 || tp.x + tp.y > nn)) {
    if (j == 0) latch_error(A.status, kErrTree);
    valid = false;
  }
  const bool has = valid && j < tp.y;
  const int c = has ? tp.x + j : 0;
  double cm = 0.0, cx = 0.0, cy = 0.0, cz = 0.0;
  if (has) {
    cm = __ldcg(A.nmass + c);
    cx = __ldcg(A.ncom + 3 * c); cy = __ldcg(A.ncom + 3 * c + 1); cz = __ldcg(A.ncom + 3 * c + 2);
  }
  const double mx = dm(cx, cm), my = dm(cy, cm), mz = dm(cz, cm);
  const int nc = valid ? tp.y : 0;
  double pm = 0.0, px = 0.0, py = 0.0, pz = 0.0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double qm = __shfl_sync(kAll, cm, base + q), qx = __shfl_sync(kAll, mx, base + q);
    const double qy = __shfl_sync(kAll, my, base + q), qz = __shfl_sync(kAll, mz, base + q);
    if (q < nc) {
      pm = da(pm, qm);
      px = da(px, qx); py = da(py, qy); pz = da(pz, qz);
    }
  }
  const double num = j == 0 ? px : j == 1 ? py : pz;
  const double quo = __ddiv_rn(num, valid ? pm : 1.0);
  float h, l;
  split_df(quo, h, l);                          // lanes 0-2: one COM component each
  const double pc[3] = {__shfl_sync(kAll, quo, base), __shfl_sync(kAll, quo, base + 1),
                        __shfl_sync(kAll, quo, base + 2)};
  const float hx = __shfl_sync(kAll, h, base), hy = __shfl_sync(kAll, h, base + 1),
              hz = __shfl_sync(kAll, h, base + 2);
  const float lx = __shfl_sync(kAll, l, base), ly = __shfl_sync(kAll, l, base + 1),
              lz = __shfl_sync(kAll, l, base + 2);
  Dbl2 T[6] = {};
  if (A.order >= 2) {
    if (has) {
      const float4 t0 = __ldcg(A.nsec + 3 * c), t1 = __ldcg(A.nsec + 3 * c + 1),
                   t2 = __ldcg(A.nsec + 3 * c + 2);
      const Dbl2 mc = dbl2_split(cm);
      const Dbl2 d0 = dbl2_split(ds(cx, pc[0])), d1 = dbl2_split(ds(cy, pc[1])),
                 d2 = dbl2_split(ds(cz, pc[2]));
      const Dbl2 m0 = dbl2_mul(mc, d0), m1 = dbl2_mul(mc, d1), m2 = dbl2_mul(mc, d2);
      T[0] = dbl2_add({t0.x, t0.y}, dbl2_mul(m0, d0));
      T[1] = dbl2_add({t0.z, t0.w}, dbl2_mul(m1, d1));
      T[2] = dbl2_add({t1.x, t1.y}, dbl2_mul(m2, d2));
      T[3] = dbl2_add({t1.z, t1.w}, dbl2_mul(m0, d1));
      T[4] = dbl2_add({t2.x, t2.y}, dbl2_mul(m0, d2));
      T[5] = dbl2_add({t2.z, t2.w}, dbl2_mul(m1, d2));
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1)
#pragma unroll
      for (int a = 0; a < 6; ++a)
        T[a] = dbl2_add(T[a], {__shfl_xor_sync(kAll, T[a].hi, o), __shfl_xor_sync(kAll, T[a].lo, o)});
  }
  if (!valid || j != 0) return;
  A.nmass[id] = pm;
  for (int a = 0; a < 3; ++a) A.ncom[3 * id + a] = pc[a];
  if (A.order >= 2) store_sec(A.nsec + 3 * id, T);
  const double side = A.geom[8 * (A.seg_sorted ? A.seg_sorted[tp.z] : 0) + 3];
  const double ln = dm(side, pow2_neg(A.ndepth[id]));
  A.rec0[id] = make_float4(hx, hy, hz, __double2float_rn(pm));
  A.rec1[id] = make_float4(lx, ly, lz, __double2float_rn(dm(ln, ln)));
  if (A.order >= 2) write_quad_record(A, id, T);
}

// Leaves, one per thread (leaves of equal body counts share a warp).
__global__ void __launch_bounds__(128) k_leaf_moments(MomArgs A) {
  const uint32_t b0 = A.boff[0], b1 = A.boff[kLeafBuckets];
  for (uint32_t k = b0 + blockIdx.x * blockDim.x + threadIdx.x; k < b1;
       k += gridDim.x * blockDim.x)
    leaf_node(A, A.nlist[k]);
}

// Every internal node in one launch, after the leaves.  A work unit is up to 32 nodes of
// one depth, one per lane (full, uniform warps: the FP64 pipe's cost per instruction does
// not depend on the active lanes); a depth whose nodes fit the grid's warps 4 to a warp
// runs 4 nodes per unit instead, 8 lanes per node (internal_node_group), so its time is
// the shorter FP64 chain of that form.  Warps take units from an atomic ticket, deepest depth
// first.  A unit waits until the nearest deeper non-empty depth is complete; that depth's
// units waited likewise before they started, so every node below, and in particular every
// child, is done.  A unit waits only on units with smaller tickets, which running warps
// hold, so the waits end; each is still bounded (on running out, kErrTimeout is latched
// and the unit computed anyway, so later waits do not cascade), and polls back off
// exponentially so that the waiting warps do not crowd the counter's L2 slice.  A negative
// budget -k (failure testing) keeps the deepest depth from being counted, so the next
// depth's wait runs out after k polls.
// One node is ~290 FP64 instructions, and on GB300 an FP64 warp instruction occupies an SM
// sub-partition's FP64 unit for ~64 cycles, so a depth takes as long as the busiest
// sub-partition's units: one block of four warps per SM puts one warp on each
// sub-partition, so a depth of up to 4 x SMs units takes one unit's time (~9 us).
constexpr int kMomSpin = 1 << 18;              // polls allowed per wait (> 0.1 s)
constexpr int kMomThreads = 128;

__global__ void __launch_bounds__(kMomThreads, kMomBlocksPerSM)
k_level_moments(MomArgs A, uint32_t *__restrict__ ticket, uint32_t *__restrict__ done,
                int spin_budget) {
  __shared__ uint32_t s_uoff[kLevels + 1];     // first unit of each depth bucket; total units
  __shared__ int s_widx[kLevels];              // depth bucket a bucket's units wait on (-1: none)
  __shared__ uint32_t s_wneed[kLevels];        // and its node count
  __shared__ uint32_t s_per[kLevels];          // nodes per unit: 32, or 4 (8 lanes per node)
  if (threadIdx.x == 0) {
    uint32_t u = 0;
    int prev = -1;                             // latest non-empty depth bucket
    const uint32_t warps = gridDim.x * (kMomThreads / 32);
    for (int i = 0; i < kLevels; ++i) {
      const int b = kLeafBuckets + i;
      const uint32_t sz = A.boff[b + 1] - A.boff[b];
      s_uoff[i] = u;
      s_per[i] = (sz + 3u) / 4u <= warps ? 4u : 32u;
      u += (sz + s_per[i] - 1u) / s_per[i];
      s_widx[i] = prev;
      s_wneed[i] = prev < 0 ? 0u : A.boff[kLeafBuckets + prev + 1] - A.boff[kLeafBuckets + prev];
      if (sz) prev = i;
    }
    s_uoff[kLevels] = u;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t nunits = s_uoff[kLevels];
  const int nn = min(*A.nnodes, A.cap_nodes);
  const int budget = abs(spin_budget);
  for (;;) {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(ticket, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= nunits) break;
    // depth bucket of unit u = the number of bucket starts 1 .. kLevels-1 at or before it
    const int i = __popc(__ballot_sync(0xffffffffu, 1 + lane < kLevels && s_uoff[1 + lane] <= u));
    const int b = kLeafBuckets + i;
    const uint32_t per = s_per[i];
    const uint32_t k0 = A.boff[b] + (u - s_uoff[i]) * per;
    const uint32_t k1 = min(k0 + per, A.boff[b + 1]);
    const uint32_t k = k0 + (uint32_t)(per == 4u ? lane >> 3 : lane);
    // the unit's node ids and topology come from earlier launches: load them before the
    // wait, so that only the children's moments are loaded after it
    int id = 0;
    int4 tp = make_int4(0, 0, 0, 0);
    if (k < k1) {
      id = __ldg(A.nlist + k);
      tp = __ldg(A.topo + id);
    }
    if (s_widx[i] >= 0) {
      // every lane polls (one coalesced load): a wait taken by lane 0 alone left the
      // warp running as two halves afterwards, doubling the FP64 time of the unit
      const volatile uint32_t *w = done + s_widx[i];
      const uint32_t need = s_wneed[i];
      unsigned ns = 32;
      for (int spin = 0; __any_sync(0xffffffffu, *w < need); ++spin) {
        if (spin >= budget) {
          if (lane == 0) latch_error(A.status, kErrTimeout);
          break;
        }
        __nanosleep(ns);
        ns = min(2u * ns, 1024u);
      }
      __threadfence();
    }
    if (per == 4u)
      internal_node_group(A, id, tp, k < k1, nn);
    else if (k < k1)
      internal_node(A, id, tp, nn);
    __threadfence();                            // this unit's moments before its count
    __syncwarp();
    if (lane == 0 && !(spin_budget < 0 && s_widx[i] < 0)) atomicAdd(done + i, k1 - k0);
  }
}

// Cloud id of every body (caller order), one block per cloud.
__global__ void k_fill_seg(const int64_t *__restrict__ off, int32_t *__restrict__ seg_of) {
  const int k = blockIdx.x;
  for (int64_t i = off[k] + threadIdx.x; i < off[k + 1]; i += blockDim.x) seg_of[i] = k;
}

// Root of a single body: node 0 is a leaf at depth 0 (moment bucket 0: one body).
__global__ void k_single_root(int4 *topo, int32_t *depth, int32_t *nparent, int32_t *nnodes,
                              uint32_t *slots) {
  topo[0] = make_int4(-1, 0, 0, 1);
  depth[0] = 0;
  nparent[0] = -1;
  *nnodes = 1;
  slots[kSlotCnt + bucket_of(topo[0], 0)] = 1;
}

inline unsigned blocks_for(int64_t n, int threads) {
  return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

int fill_segment_ids(Ctx *c) {
  k_fill_seg<<<c->seg.nseg, 256, 0, c->stream>>>(c->seg.off, c->seg.seg_of);
  ++c->launches;
  return cuda_status(cudaGetLastError());
}

int tree_build(Ctx *c, int64_t n, const double *pos, const double *mass) {
  Tree &t = c->t;
  Segs &sg = c->seg;
  cudaStream_t s = c->stream;
  const int leaf_max = c->params.leaf_max;
  const bool multi = sg.nseg > 1;
  int rc = GRAVITY_OK;
  if (!multi && n <= kRsTile && c->sort_stall == 0) {
    // a1-a3 for one cloud that fits one sort tile: root cube, keys and sort in one block
    // (the octree scan's tile states, kept after the sort's words, are cleared here)
    GRAV_CUDA_TRY(cudaMemsetAsync(oct_scan_state(c, n), 0, sizeof(uint32_t) * oct_scan_words(n), s));
    k_order_small<<<1, kOrdThreads, 0, s>>>(pos, (int)n, t.geom, t.keys, t.idx, c->d_status);
    ++c->launches;
  } else {
    // a1: root cube of each cloud (also validates the coordinates)
    if (!multi) {
      launch_bbox(c, pos, n, reinterpret_cast<unsigned long long *>(t.bbox_part), t.bbox_ticket,
                  t.geom);
    } else {
      k_bbox_seg<<<sg.nseg, kBBoxThreads, 0, s>>>(pos, sg.off, t.geom, c->d_status);
      ++c->launches;
    }
    // a2: keys, with the digit counts of every sort pass (one read of the positions)
    const int cloud_passes = multi ? (sg.cbits + 7) / 8 : 0;
    if ((rc = radix_sort_clear(c, n, t.hist, cloud_passes, oct_scan_words(n)))) return rc;
    int cb = (int)((n + kRsThreads - 1) / kRsThreads);
    if (cb > 2 * c->num_sms) cb = 2 * c->num_sms;
    k_keys_count<<<cb, kRsThreads, 0, s>>>(pos, n, t.geom, multi ? sg.seg_of : nullptr, t.keys,
                                           t.idx, t.idx_alt, cloud_passes, t.hist);
    ++c->launches;
    // a3: sort (by cloud, then key, then caller index)
    rc = radix_sort(c, n, true);
    if (rc) return rc;
  }
  // a4: gather sorted bodies
  k_gather<<<blocks_for(n, 256), 256, 0, s>>>(pos, mass, t.idx, n, t.pos_s, t.mass_s, t.body_hi,
                                               t.body_lo, multi ? sg.seg_of : nullptr,
                                               sg.seg_sorted, t.scalars);
  ++c->launches;
  const int cap_nodes = (int)(2 * c->cap);
  if (n == 1) {
    k_single_root<<<1, 1, 0, s>>>(t.topo, t.ndepth, t.nparent, t.nnodes, t.scalars);
    ++c->launches;
  } else {
    const int ni = (int)(n - 1);
    const KeyView kv{t.keys, multi ? sg.seg_sorted : nullptr, multi ? sg.cbits : 0, (int)n};
    // a5: binary radix tree
    k_radix_tree<<<blocks_for(ni, 256), 256, 0, s>>>(kv, t.bchild, t.bparent, t.bfirst, t.blast,
                                                     t.bplen);
    ++c->launches;
    // a6: octree
    // a6: octree children counts and their exclusive scan (one launch; tile states zeroed
    // with the sort's counters)
    uint32_t *base = t.bbase;
    uint32_t *total = t.scalars;             // number of octree nodes below the cloud roots
    uint32_t *oct_state = oct_scan_state(c, n);
    const int otiles = (int)((ni + kOctTile - 1) / kOctTile);
    const bool few = otiles <= 32;
    auto oct_count = few ? k_oct_count<1> : k_oct_count<4>;
    oct_count<<<otiles, few ? kOctTile : kOctTile / 4, 0, s>>>(
        (int)n, leaf_max, kv.cbits, t.bchild, t.bparent, t.bfirst, t.blast, t.bplen, t.bnchild,
        base, total, oct_state + 1, oct_state, otiles, c->d_status);
    ++c->launches;
    // (with the parent of every node: a cell writes its children's records and the parent
    // of their children)
    OctWriteArgs W{(int)n, leaf_max, kv.cbits, sg.nseg, cap_nodes, t.bchild, t.bfirst, t.blast,
                   t.bplen, kv.seg, t.bnchild, base, total, t.topo, t.ndepth, t.nnodes,
                   t.nparent, t.scalars, c->d_status};
    k_oct_write<<<blocks_for(ni, 256), 256, 0, s>>>(W);
    ++c->launches;
  }
  // a7: moments (nodes bucketed by the octree write's counts; full warps)
  static_assert(kSlotDone + kLevels <= kSlotTicket && kSlotOff + kBuckets + 1 <= kScalarWords,
                "scalar slots overlap");
  const unsigned nb_nodes = blocks_for(cap_nodes, 256);
  k_bucket_fill<<<nb_nodes, 256, 0, s>>>(t.topo, t.ndepth, t.nnodes, cap_nodes, t.scalars,
                                         t.nlist);
  ++c->launches;
  MomArgs A{t.topo, t.ndepth, t.nnodes, t.nlist, t.scalars + kSlotOff, t.pos_s, t.mass_s,
            t.geom, multi ? sg.seg_sorted : nullptr, t.nmass, t.ncom, t.nquad, t.nrec0, t.nrec1,
            t.nquadf, c->params.order, cap_nodes, (int)n, c->d_status};
  k_leaf_moments<<<(unsigned)(8 * c->num_sms), 128, 0, s>>>(A);
  ++c->launches;
  k_level_moments<<<(unsigned)(kMomBlocksPerSM * c->num_sms), kMomThreads, 0, s>>>(
      A, t.scalars + kSlotTicket, t.scalars + kSlotDone,
      c->moments_stall > 0 ? -c->moments_stall : kMomSpin);
  ++c->launches;
  return cuda_status(cudaGetLastError());
}

// Morton order of n bodies of one cloud (for the direct sum's tiling): root cube,
// keys and the radix sort into caller-provided buffers; idx ends as the permutation
// (sorted position -> caller index).
int64_t radix_hist_words(int64_t n) {
  const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
  return (int64_t)257 * kRsMaxPasses + (int64_t)kRsMaxPasses * 256 * ntiles +
         (n + kOctTile - 1) / kOctTile + 2;    // + the octree scan's tile counter and states
}

int morton_order(Ctx *c, int64_t n, const double *pos, const MortonBuffers &b) {
  launch_bbox(c, pos, n, b.part, b.ticket, b.geom);
  k_keys<<<blocks_for(n, 256), 256, 0, c->stream>>>(pos, n, b.geom, nullptr, b.keys, b.idx);
  ++c->launches;
  return radix_sort_buffers(c, n, b.keys, b.keys_alt, b.idx, b.idx_alt, b.hist, 0, nullptr, 0);
}

}  // namespace grav
