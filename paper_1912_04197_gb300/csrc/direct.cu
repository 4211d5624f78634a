// Direct N^2 gravity, Eq. (Newton) (Sec. 2.1), with the softened distance of
// Eq. (Force_rComp): a_i = G sum_{j != i} m_j d_ij / (|d_ij|^2 + eps^2)^{3/2}.
// FP32 pair terms, source tiles staged in shared memory, each tile's partial sum added
// to a (hi, lo) two-sum accumulator.  The self term has d = 0 and adds zero.
// From 32768 bodies on, gravity_direct first puts the bodies in Morton order, so that a
// block's 512 bodies and a 256-body source tile are each compact: a tile away from the
// block (gap between their boxes at least half the block's diagonal w) is evaluated on
// FP32 coordinates relative to the block's first body, d = s_rel - x_rel, whose error is
// then below 2^-24 (2 |d| + 2 w) <= 6 * 2^-24 |d|; nearer tiles use hi/lo split
// coordinates, d = (x_j,hi - x_i,hi) + (x_j,lo - x_i,lo).  Smaller sums, and the
// allocation-free entry point, keep the caller's order and the hi/lo form throughout.
#include "internal.cuh"

namespace grav {
namespace {

constexpr int kDirThreads = 256;
constexpr int kDirPerThread = 2;     // bodies per thread (register blocking)

__global__ void k_split(const double *__restrict__ pos, const double *__restrict__ mass, int64_t n,
                        float4 *__restrict__ hi, float4 *__restrict__ lo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float xh, xl, yh, yl, zh, zl;
  split_df(pos[3 * i], xh, xl);
  split_df(pos[3 * i + 1], yh, yl);
  split_df(pos[3 * i + 2], zh, zl);
  hi[i] = make_float4(xh, yh, zh, __double2float_rn(mass[i]));
  lo[i] = make_float4(xl, yl, zl, 0.f);
}

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float p) {
  float s = hi + p;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (p - bp);
  hi = s;
  lo += err;
}

template <bool EPS0>
__global__ void __launch_bounds__(kDirThreads)
k_direct(const float4 *__restrict__ hi, const float4 *__restrict__ lo, int64_t n, float eps2,
         double G, double *__restrict__ acc);

// Sorted hi/lo bodies (Morton order) and the box of each 256-body tile (hi parts).
__global__ void k_split_sorted(const double *__restrict__ pos, const double *__restrict__ mass,
                               const uint32_t *__restrict__ perm, int64_t n,
                               float4 *__restrict__ hi, float4 *__restrict__ lo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j = perm[i];
  float xh, xl, yh, yl, zh, zl;
  split_df(pos[3 * j], xh, xl);
  split_df(pos[3 * j + 1], yh, yl);
  split_df(pos[3 * j + 2], zh, zl);
  hi[i] = make_float4(xh, yh, zh, __double2float_rn(mass[j]));
  lo[i] = make_float4(xl, yl, zl, 0.f);
}

__global__ void __launch_bounds__(kDirThreads)
k_tile_box(const float4 *__restrict__ hi, int64_t n, float4 *__restrict__ box) {
  const int64_t i = blockIdx.x * (int64_t)kDirThreads + threadIdx.x;
  const bool v = i < n;
  const float4 h = v ? hi[i] : make_float4(0, 0, 0, 0);
  float lx = v ? h.x : INFINITY, ly = v ? h.y : INFINITY, lz = v ? h.z : INFINITY;
  float ux = v ? h.x : -INFINITY, uy = v ? h.y : -INFINITY, uz = v ? h.z : -INFINITY;
  for (int o = 16; o > 0; o >>= 1) {
    lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
    ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
    lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
    ux = fmaxf(ux, __shfl_xor_sync(0xffffffffu, ux, o));
    uy = fmaxf(uy, __shfl_xor_sync(0xffffffffu, uy, o));
    uz = fmaxf(uz, __shfl_xor_sync(0xffffffffu, uz, o));
  }
  __shared__ float s[kDirThreads / 32][6];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { s[w][0] = lx; s[w][1] = ly; s[w][2] = lz; s[w][3] = ux; s[w][4] = uy; s[w][5] = uz; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kDirThreads / 32; ++k) {
      lx = fminf(lx, s[k][0]); ly = fminf(ly, s[k][1]); lz = fminf(lz, s[k][2]);
      ux = fmaxf(ux, s[k][3]); uy = fmaxf(uy, s[k][4]); uz = fmaxf(uz, s[k][5]);
    }
    box[2 * blockIdx.x] = make_float4(lx, ly, lz, 0.f);
    box[2 * blockIdx.x + 1] = make_float4(ux, uy, uz, 0.f);
  }
}

// Packed two-wide FP32 arithmetic (sm_100+): one issue slot for the same operation on the
// two bodies a thread holds; each half is the scalar IEEE operation, so the result equals
// the one-body-at-a-time arithmetic bit for bit.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 xy2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 zw2(float4 v) { return make_float2(v.z, v.w); }

// Caller order, hi/lo coordinates for every pair: each thread's two bodies (i0 and
// i0 + 256) evaluated as one packed pair against every 256-body tile, sources staged
// duplicated as in k_direct_sorted.
template <bool EPS0>
__global__ void __launch_bounds__(kDirThreads)
k_direct(const float4 *__restrict__ hi, const float4 *__restrict__ lo, int64_t n, float eps2,
         double G, double *__restrict__ acc) {
  __shared__ float4 sA[kDirThreads], sB[kDirThreads], sC[kDirThreads], sD[kDirThreads];
  static_assert(kDirPerThread == 2, "the two bodies of a thread form one packed pair");
  const int64_t i0 = (blockIdx.x * (int64_t)kDirThreads) * 2 + threadIdx.x;
  float nh[2][3], nl[2][3];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int64_t i = i0 + p * kDirThreads;
    const float4 h = i < n ? hi[i] : make_float4(0, 0, 0, 0);
    const float4 l = i < n ? lo[i] : make_float4(0, 0, 0, 0);
    nh[p][0] = -h.x; nh[p][1] = -h.y; nh[p][2] = -h.z;
    nl[p][0] = -l.x; nl[p][1] = -l.y; nl[p][2] = -l.z;
  }
  const float2 nhx = make_float2(nh[0][0], nh[1][0]), nhy = make_float2(nh[0][1], nh[1][1]),
               nhz = make_float2(nh[0][2], nh[1][2]);
  const float2 nlx = make_float2(nl[0][0], nl[1][0]), nly = make_float2(nl[0][1], nl[1][1]),
               nlz = make_float2(nl[0][2], nl[1][2]);
  const float2 e2 = make_float2(eps2, eps2);
  float ahx[2] = {0.f, 0.f}, ahy[2] = {0.f, 0.f}, ahz[2] = {0.f, 0.f};
  float alx[2] = {0.f, 0.f}, aly[2] = {0.f, 0.f}, alz[2] = {0.f, 0.f};
  for (int64_t t0 = 0; t0 < n; t0 += kDirThreads) {
    const int64_t j = t0 + threadIdx.x;
    const float4 h = j < n ? hi[j] : make_float4(0, 0, 0, 0);
    const float4 l = j < n ? lo[j] : make_float4(0, 0, 0, 0);
    sA[threadIdx.x] = make_float4(h.x, h.x, h.y, h.y);
    sB[threadIdx.x] = make_float4(h.z, h.z, h.w, h.w);
    sC[threadIdx.x] = make_float4(l.x, l.x, l.y, l.y);
    sD[threadIdx.x] = make_float4(l.z, l.z, 0.f, 0.f);
    __syncthreads();
    float2 px = make_float2(0.f, 0.f), py = px, pz = px;
#pragma unroll 4
    for (int k = 0; k < kDirThreads; ++k) {
      const float4 A = sA[k], B = sB[k], Cc = sC[k], D = sD[k];
      const float2 dx = add2(add2(xy2(A), nhx), add2(xy2(Cc), nlx));
      const float2 dy = add2(add2(zw2(A), nhy), add2(zw2(Cc), nly));
      const float2 dz = add2(add2(xy2(B), nhz), add2(xy2(D), nlz));
      const float2 r2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, e2)));
      float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
      // with eps > 0, r^2 >= eps^2 > 0 and the self pair (d = 0) adds m * 0;
      // with eps = 0 a pair at r^2 = 0 must add nothing
      if (EPS0) {
        inv.x = r2.x > 0.f ? inv.x : 0.f;
        inv.y = r2.y > 0.f ? inv.y : 0.f;
      }
      const float2 sc = mul2(zw2(B), mul2(mul2(inv, inv), inv));
      px = fma2(sc, dx, px);
      py = fma2(sc, dy, py);
      pz = fma2(sc, dz, pz);
    }
    two_sum_add(ahx[0], alx[0], px.x); two_sum_add(ahx[1], alx[1], px.y);
    two_sum_add(ahy[0], aly[0], py.x); two_sum_add(ahy[1], aly[1], py.y);
    two_sum_add(ahz[0], alz[0], pz.x); two_sum_add(ahz[1], alz[1], pz.y);
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int64_t i = i0 + p * kDirThreads;
    if (i < n) {
      acc[3 * i] = G * ((double)ahx[p] + (double)alx[p]);
      acc[3 * i + 1] = G * ((double)ahy[p] + (double)aly[p]);
      acc[3 * i + 2] = G * ((double)ahz[p] + (double)alz[p]);
    }
  }
}

// One block: 512 Morton-consecutive bodies (2 per thread, evaluated as one packed pair)
// against every 256-body tile; the tile's sources are staged duplicated, (x, x, y, y) and
// (z, z, m, m), so that each shared-memory load gives a packed operand.
template <bool EPS0>
__global__ void __launch_bounds__(kDirThreads)
k_direct_sorted(const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                const float4 *__restrict__ box, const uint32_t *__restrict__ perm, int64_t n,
                float eps2, double G, double *__restrict__ acc) {
  __shared__ float4 sA[kDirThreads], sB[kDirThreads], sC[kDirThreads], sD[kDirThreads];
  static_assert(kDirPerThread == 2, "the two bodies of a thread form one packed pair");
  const int64_t b0 = blockIdx.x * (int64_t)kDirThreads * 2;
  const int64_t ntiles = (n + kDirThreads - 1) / kDirThreads;
  // origin (the block's first body) and the block's box from its tiles' boxes
  const float4 oh = hi[b0], ol = lo[b0];
  float bl[3] = {INFINITY, INFINITY, INFINITY}, bu[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int64_t t = b0 / kDirThreads + p;
    if (t < ntiles) {
      const float4 a = box[2 * t], c = box[2 * t + 1];
      bl[0] = fminf(bl[0], a.x); bl[1] = fminf(bl[1], a.y); bl[2] = fminf(bl[2], a.z);
      bu[0] = fmaxf(bu[0], c.x); bu[1] = fmaxf(bu[1], c.y); bu[2] = fmaxf(bu[2], c.z);
    }
  }
  const float ex = bu[0] - bl[0], ey = bu[1] - bl[1], ez = bu[2] - bl[2];
  const float C = fmaxf(fmaxf(fabsf(bl[0]), fabsf(bu[0])),
                        fmaxf(fmaxf(fabsf(bl[1]), fabsf(bu[1])), fmaxf(fabsf(bl[2]), fabsf(bu[2]))));
  // far: gap >= diag / 2 (the hi parts' rounding is taken off the gap below)
  const float far2 = 0.25f * fmaf(ex, ex, fmaf(ey, ey, ez * ez)) * 1.01f + 1e-30f;
  const float slack = C * 2.4e-7f;            // 2^-22 |x|: hi parts are within 2^-24 |x|
  // the thread's two bodies, negated (d = source - body is source + (-body))
  float nh[2][3], nl[2][3], nr[2][3];
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int64_t i = b0 + threadIdx.x + p * kDirThreads;
    const float4 h = i < n ? hi[i] : oh;
    const float4 l = i < n ? lo[i] : ol;
    nh[p][0] = -h.x; nh[p][1] = -h.y; nh[p][2] = -h.z;
    nl[p][0] = -l.x; nl[p][1] = -l.y; nl[p][2] = -l.z;
    nr[p][0] = -((h.x - oh.x) + (l.x - ol.x));
    nr[p][1] = -((h.y - oh.y) + (l.y - ol.y));
    nr[p][2] = -((h.z - oh.z) + (l.z - ol.z));
  }
  const float2 nhx = make_float2(nh[0][0], nh[1][0]), nhy = make_float2(nh[0][1], nh[1][1]),
               nhz = make_float2(nh[0][2], nh[1][2]);
  const float2 nlx = make_float2(nl[0][0], nl[1][0]), nly = make_float2(nl[0][1], nl[1][1]),
               nlz = make_float2(nl[0][2], nl[1][2]);
  const float2 nrx = make_float2(nr[0][0], nr[1][0]), nry = make_float2(nr[0][1], nr[1][1]),
               nrz = make_float2(nr[0][2], nr[1][2]);
  const float2 e2 = make_float2(eps2, eps2);
  float ahx[2] = {0.f, 0.f}, ahy[2] = {0.f, 0.f}, ahz[2] = {0.f, 0.f};
  float alx[2] = {0.f, 0.f}, aly[2] = {0.f, 0.f}, alz[2] = {0.f, 0.f};
  for (int64_t t = 0; t < ntiles; ++t) {
    const float4 a0 = box[2 * t], a1 = box[2 * t + 1];
    float gx = fmaxf(fmaxf(a0.x - bu[0], bl[0] - a1.x) - slack, 0.f);
    float gy = fmaxf(fmaxf(a0.y - bu[1], bl[1] - a1.y) - slack, 0.f);
    float gz = fmaxf(fmaxf(a0.z - bu[2], bl[2] - a1.z) - slack, 0.f);
    const bool far = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) >= far2;     // block-uniform
    const int64_t j = t * kDirThreads + threadIdx.x;
    const float4 h = j < n ? hi[j] : make_float4(0, 0, 0, 0);
    const float4 l = j < n ? lo[j] : make_float4(0, 0, 0, 0);
    if (far) {   // sources relative to the origin; past the end: massless and very far
      const float4 r = j < n ? make_float4((h.x - oh.x) + (l.x - ol.x), (h.y - oh.y) + (l.y - ol.y),
                                           (h.z - oh.z) + (l.z - ol.z), h.w)
                             : make_float4(1e30f, 1e30f, 1e30f, 0.f);
      sA[threadIdx.x] = make_float4(r.x, r.x, r.y, r.y);
      sB[threadIdx.x] = make_float4(r.z, r.z, r.w, r.w);
    } else {
      sA[threadIdx.x] = make_float4(h.x, h.x, h.y, h.y);
      sB[threadIdx.x] = make_float4(h.z, h.z, h.w, h.w);
      sC[threadIdx.x] = make_float4(l.x, l.x, l.y, l.y);
      sD[threadIdx.x] = make_float4(l.z, l.z, 0.f, 0.f);
    }
    __syncthreads();
    float2 px = make_float2(0.f, 0.f), py = px, pz = px;
    if (far) {
#pragma unroll 4
      for (int k = 0; k < kDirThreads; ++k) {
        const float4 A = sA[k], B = sB[k];
        const float2 dx = add2(xy2(A), nrx), dy = add2(zw2(A), nry), dz = add2(xy2(B), nrz);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, e2)));
        // r2 > 0: the tile is away from the block
        const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 sc = mul2(zw2(B), mul2(mul2(inv, inv), inv));
        px = fma2(sc, dx, px);
        py = fma2(sc, dy, py);
        pz = fma2(sc, dz, pz);
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < kDirThreads; ++k) {
        const float4 A = sA[k], B = sB[k], Cc = sC[k], D = sD[k];
        const float2 dx = add2(add2(xy2(A), nhx), add2(xy2(Cc), nlx));
        const float2 dy = add2(add2(zw2(A), nhy), add2(zw2(Cc), nly));
        const float2 dz = add2(add2(xy2(B), nhz), add2(xy2(D), nlz));
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, e2)));
        float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        // with eps > 0, r^2 >= eps^2 > 0 and the self pair (d = 0) adds m * 0;
        // with eps = 0 a pair at r^2 = 0 must add nothing
        if (EPS0) {
          inv.x = r2.x > 0.f ? inv.x : 0.f;
          inv.y = r2.y > 0.f ? inv.y : 0.f;
        }
        const float2 sc = mul2(zw2(B), mul2(mul2(inv, inv), inv));
        px = fma2(sc, dx, px);
        py = fma2(sc, dy, py);
        pz = fma2(sc, dz, pz);
      }
    }
    two_sum_add(ahx[0], alx[0], px.x); two_sum_add(ahx[1], alx[1], px.y);
    two_sum_add(ahy[0], aly[0], py.x); two_sum_add(ahy[1], aly[1], py.y);
    two_sum_add(ahz[0], alz[0], pz.x); two_sum_add(ahz[1], alz[1], pz.y);
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const int64_t i = b0 + threadIdx.x + p * kDirThreads;
    if (i < n) {
      const int64_t ci = perm[i];
      acc[3 * ci] = G * ((double)ahx[p] + (double)alx[p]);
      acc[3 * ci + 1] = G * ((double)ahy[p] + (double)aly[p]);
      acc[3 * ci + 2] = G * ((double)ahz[p] + (double)alz[p]);
    }
  }
}

// Softened potential of every body, phi_i = sum_{j != i} m_j / sqrt(|d_ij|^2 + eps^2)
// (the Plummer potential consistent with the softened force; Sec. 3.1's energy),
// same tiling and arithmetic as k_direct; the self pair is excluded by index and a
// pair with r^2 = 0 adds nothing.  Writes m_i phi_i (FP64).
__global__ void __launch_bounds__(kDirThreads)
k_potential(const float4 *__restrict__ hi, const float4 *__restrict__ lo, const double *mass,
            int64_t n, float eps2, double *__restrict__ mphi) {
  __shared__ float4 sh[kDirThreads], sl[kDirThreads];
  const int64_t i = blockIdx.x * (int64_t)kDirThreads + threadIdx.x;
  const float4 h = i < n ? hi[i] : make_float4(0, 0, 0, 0);
  const float4 l = i < n ? lo[i] : make_float4(0, 0, 0, 0);
  float sh_hi = 0.f, sh_lo = 0.f;
  for (int64_t t0 = 0; t0 < n; t0 += kDirThreads) {
    const int64_t j = t0 + threadIdx.x;
    sh[threadIdx.x] = j < n ? hi[j] : make_float4(0, 0, 0, 0);
    sl[threadIdx.x] = j < n ? lo[j] : make_float4(0, 0, 0, 0);
    __syncthreads();
    float ps = 0.f;
    const int64_t self = i - t0;
#pragma unroll 8
    for (int k = 0; k < kDirThreads; ++k) {
      const float4 a = sh[k], b = sl[k];
      const float dx = (a.x - h.x) + (b.x - l.x);
      const float dy = (a.y - h.y) + (b.y - l.y);
      const float dz = (a.z - h.z) + (b.z - l.z);
      const float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
      const float inv = (r2 > 0.f && k != self) ? rsqrtf(r2) : 0.f;
      ps = fmaf(a.w, inv, ps);
    }
    two_sum_add(sh_hi, sh_lo, ps);
    __syncthreads();
  }
  if (i < n) mphi[i] = mass[i] * ((double)sh_hi + (double)sh_lo);
}

// Per-block FP64 partial sums of kinetic energy, m phi, momentum and angular
// momentum (8 values per block, fixed grid and order: deterministic).
constexpr int kDiagThreads = 256;
constexpr int kDiagBlocks = 256;

__global__ void __launch_bounds__(kDiagThreads)
k_diag_partial(const double *__restrict__ pos, const double *__restrict__ vel,
               const double *__restrict__ mass, const double *__restrict__ mphi, int64_t n,
               double *__restrict__ part) {
  double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)kDiagThreads + threadIdx.x; i < n;
       i += (int64_t)kDiagBlocks * kDiagThreads) {
    const double m = mass[i];
    const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
    const double vx = vel[3 * i], vy = vel[3 * i + 1], vz = vel[3 * i + 2];
    q[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
    q[1] += mphi[i];
    q[2] += m * vx; q[3] += m * vy; q[4] += m * vz;
    q[5] += m * (y * vz - z * vy);
    q[6] += m * (z * vx - x * vz);
    q[7] += m * (x * vy - y * vx);
  }
  __shared__ double red[8][kDiagThreads];
#pragma unroll
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = q[k];
  __syncthreads();
  for (int s = kDiagThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
#pragma unroll
      for (int k = 0; k < 8; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 8) part[8 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// Sums the block partials in block order: out = E, P xyz, L xyz.
__global__ void k_diag_final(const double *__restrict__ part, double G, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < kDiagBlocks; ++b)
    for (int k = 0; k < 8; ++k) q[k] += part[8 * b + k];
  out[0] = q[0] - 0.5 * G * q[1];     // every pair appears twice in sum_i m_i phi_i
  for (int k = 0; k < 6; ++k) out[1 + k] = q[2 + k];
}

}  // namespace

// Below this many bodies the Morton order costs more than the far tiles save.
constexpr int64_t kDirSortMin = 32768;

int direct_forces(Ctx *c, int64_t n, const double *pos, const double *mass, double eps, double G,
                  double *acc) {
  if (n < kDirSortMin) {                       // caller order, hi/lo for every pair
    if (n > c->dir_cap) {
      GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
      ctx_release(c, c->dir_hi);
      ctx_release(c, c->dir_lo);
      c->dir_cap = 0;
      int rc = ctx_alloc(c, c->dir_hi, n);
      if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->dir_lo, n);
      if (rc) return rc;
      c->dir_cap = n;
    }
    k_split<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(pos, mass, n, c->dir_hi, c->dir_lo);
    const int64_t per_block = (int64_t)kDirThreads * kDirPerThread;
    const unsigned blocks = (unsigned)((n + per_block - 1) / per_block);
    const float eps2 = (float)(eps * eps);
    if (eps2 > 0.f)
      k_direct<false><<<blocks, kDirThreads, 0, c->stream>>>(c->dir_hi, c->dir_lo, n, eps2, G, acc);
    else
      k_direct<true><<<blocks, kDirThreads, 0, c->stream>>>(c->dir_hi, c->dir_lo, n, eps2, G, acc);
    c->launches += 2;
    return cuda_status(cudaGetLastError());
  }
  if (n > c->ds_cap) {
    GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
    ctx_release(c, c->ds_keys); ctx_release(c, c->ds_keys_alt); ctx_release(c, c->ds_idx);
    ctx_release(c, c->ds_idx_alt); ctx_release(c, c->ds_hist); ctx_release(c, c->ds_geom);
    ctx_release(c, c->ds_part); ctx_release(c, c->ds_ticket); ctx_release(c, c->ds_hi);
    ctx_release(c, c->ds_lo); ctx_release(c, c->ds_box);
    c->ds_cap = 0;
    const int64_t ntiles = (n + kDirThreads - 1) / kDirThreads;
    int rc = ctx_alloc(c, c->ds_keys, n);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_keys_alt, n);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_idx, n);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_idx_alt, n);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_hist, radix_hist_words(n));
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_geom, 8);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_part, 6 * (4 * (int64_t)c->num_sms + 3));
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_ticket, 1);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_hi, n);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_lo, n);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->ds_box, 2 * ntiles);
    if (rc == GRAVITY_OK) rc = cuda_status(cudaMemset(c->ds_ticket, 0, sizeof(unsigned)));
    if (rc) return rc;
    c->ds_cap = n;
  }
  const MortonBuffers b{c->ds_keys, c->ds_keys_alt, c->ds_idx, c->ds_idx_alt, c->ds_hist,
                        c->ds_geom, c->ds_part, c->ds_ticket};
  int rc = morton_order(c, n, pos, b);
  if (rc) return rc;
  k_split_sorted<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(pos, mass, c->ds_idx, n,
                                                                    c->ds_hi, c->ds_lo);
  const int64_t ntiles = (n + kDirThreads - 1) / kDirThreads;
  k_tile_box<<<(unsigned)ntiles, kDirThreads, 0, c->stream>>>(c->ds_hi, n, c->ds_box);
  const int64_t per_block = (int64_t)kDirThreads * kDirPerThread;
  const unsigned blocks = (unsigned)((n + per_block - 1) / per_block);
  const float eps2 = (float)(eps * eps);
  if (eps2 > 0.f)
    k_direct_sorted<false><<<blocks, kDirThreads, 0, c->stream>>>(c->ds_hi, c->ds_lo, c->ds_box,
                                                                 c->ds_idx, n, eps2, G, acc);
  else
    k_direct_sorted<true><<<blocks, kDirThreads, 0, c->stream>>>(c->ds_hi, c->ds_lo, c->ds_box,
                                                                c->ds_idx, n, eps2, G, acc);
  c->launches += 3;
  return cuda_status(cudaGetLastError());
}

int diagnostics(Ctx *c, int64_t n, const double *pos, const double *vel, const double *mass,
                double eps, double G, double *out_dev) {
  if (n > c->dir_cap) {
    GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
    ctx_release(c, c->dir_hi);
    ctx_release(c, c->dir_lo);
    c->dir_cap = 0;
    int rc = ctx_alloc(c, c->dir_hi, n);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->dir_lo, n);
    if (rc) return rc;
    c->dir_cap = n;
  }
  if (n > c->diag_cap) {
    GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
    ctx_release(c, c->diag_buf);
    c->diag_cap = 0;
    const int rc = ctx_alloc(c, c->diag_buf, n + 8 * kDiagBlocks + 8);
    if (rc) return rc;
    c->diag_cap = n;
  }
  double *mphi = c->diag_buf, *part = c->diag_buf + n;
  k_split<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(pos, mass, n, c->dir_hi, c->dir_lo);
  k_potential<<<(unsigned)((n + kDirThreads - 1) / kDirThreads), kDirThreads, 0, c->stream>>>(
      c->dir_hi, c->dir_lo, mass, n, (float)(eps * eps), mphi);
  k_diag_partial<<<kDiagBlocks, kDiagThreads, 0, c->stream>>>(pos, vel, mass, mphi, n, part);
  k_diag_final<<<1, 32, 0, c->stream>>>(part, G, out_dev);
  c->launches += 4;
  return cuda_status(cudaGetLastError());
}

}  // namespace grav

// ---------------------------------------------------------------------------
// Allocation-free direct sum.
//
// Some callers cannot call cudaMalloc: code embedded in a host application that
// owns every byte of device memory (a fixed-budget pool, or a plugin host that
// forbids allocations once it has started), and latency-critical loops where the
// implicit device-wide synchronisation of cudaMalloc/cudaFree is not acceptable.
// gravity_direct_noalloc serves them: it runs the same two kernels as
// gravity_direct, but its hi/lo staging lives in the file-scope array below
// instead of context-owned scratch, and it needs no context at all.
#include <mutex>

#include <nvtx3/nvToolsExt.h>

namespace grav {
namespace {

constexpr int64_t kNoAllocMaxBodies = 65536;     // 2 x 65536 x 16 B = 2 MiB per device
constexpr int kNoAllocMaxDevices = 64;

// hi/lo staging of gravity_direct_noalloc: [0, max) = (x_hi, y_hi, z_hi, m),
// [max, 2 max) = (x_lo, y_lo, z_lo, 0).  Every GPU that loads this library holds it
// until the process exits.  Host code must not pass this name to a kernel: on the
// host it is only a stand-in for the symbol; the device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) float4 g_direct_scratch[2 * kNoAllocMaxBodies];

// The device address of the array, resolved once per device.  It belongs to the device's
// primary context: after a cudaDeviceReset the cached value is stale (the array's module
// is loaded again in the new context), so this entry point is not for processes that
// reset a device while using it.
std::mutex g_noalloc_mu;
float4 *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// A named range for a profiler's timeline, as around the context entry points.
struct NoAllocRange {
  NoAllocRange() { nvtxRangePushA("gravity_direct_noalloc"); }
  ~NoAllocRange() { nvtxRangePop(); }
};

}  // namespace
}  // namespace grav

extern "C" int gravity_direct_noalloc(int64_t n, const double *pos, const double *mass,
                                      double eps, double G, double *acc, void *cuda_stream) {
  using namespace grav;
  NoAllocRange range_;
  if (n < 0 || n > kNoAllocMaxBodies || !(eps >= 0.0) || !isfinite(eps) || !isfinite(G))
    return GRAVITY_E_ARG;
  if (n == 0) return GRAVITY_OK;
  if (!pos || !mass || !acc) return GRAVITY_E_ARG;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= kNoAllocMaxDevices) return GRAVITY_E_ARG;
  float4 *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {               // first call on this device: resolve the address
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_direct_scratch);
      if (e != cudaSuccess) return cuda_status(e);
      g_noalloc_ptr[dev] = static_cast<float4 *>(p);
    }
    base = g_noalloc_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  float4 *hi = base, *lo = base + kNoAllocMaxBodies;
  // every staging entry the sum reads (j < n) is written first by k_split in this call
  k_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(pos, mass, n, hi, lo);
  const int64_t per_block = (int64_t)kDirThreads * kDirPerThread;
  const unsigned blocks = (unsigned)((n + per_block - 1) / per_block);
  const float eps2 = (float)(eps * eps);
  if (eps2 > 0.f) k_direct<false><<<blocks, kDirThreads, 0, s>>>(hi, lo, n, eps2, G, acc);
  else k_direct<true><<<blocks, kDirThreads, 0, s>>>(hi, lo, n, eps2, G, acc);
  return cuda_status(cudaGetLastError());
}
