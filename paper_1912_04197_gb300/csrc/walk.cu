// Kernel 5 of the paper's list (Sec. 2.1, "compute forces"): the tree walk.
//
// The paper assigns one thread per body and relies on body sorting so that
// neighbouring threads traverse similar sub-trees.  Here a warp owns 32 bodies
// that are consecutive in Morton order and walks ONE shared stack for all of them,
// while every decision stays per body:
//   * stack entries are ranges of sibling nodes (children are contiguous), each with
//     the 32-bit mask of lanes that still need them; the bodies of an opened leaf go
//     straight to the body-term list instead;
//   * up to 32 stacked items are taken at once, one per lane, and classified
//     against the bounding box of the warp's bodies: "accepted by every lane",
//     "opened by every lane" or "mixed";
//   * a mixed node is tested by each lane with the exact opening test of
//     Eq. (accuracy): l^2 < theta^2 D^2 in FP32 on hi/lo coordinates; a result
//     within a relative 2^-16 of the boundary is recomputed in FP64 exactly as
//     the oracle does, so every decision equals the FP64 one;
//   * accepted terms go to shared-memory lists that all lanes evaluate with the
//     softened r of Eq. (Force_rComp); inactive lanes add zero.  Three lists:
//       point  - body-to-body terms (Eq. Force_leaf), and with monopoles only the
//                node terms not in the far list, d = (c_hi - x_hi) + (c_lo - x_lo);
//       far    - node terms (Eq. Force_thetaTrue; + quadrupole) of cells at least
//                theta R_w / 2 wide (R_w = extent of the warp's bodies), on FP32
//                coordinates relative to the warp's first body: every accepting
//                body is then more than R_w / 2 away, which bounds the error of
//                d = c_rel - x_rel by 5.5 * 2^-23 |d| (2^-23 (1.5 |d| + 2 R_w));
//       near   - (quadrupole) the other node terms, on hi/lo coordinates;
//   * the lists are stored pair-interleaved in shared memory, so that each lane
//     evaluates two entries at once with packed two-wide FP32 instructions (f32x2 FMA,
//     add and multiply of sm_100 and later: one issue slot for two operations);
//   * each flushed list's partial sum enters a (hi, lo) two-sum accumulator (or an
//     FP64 one).
// The kernel is persistent: each warp takes 32-body tasks from per-SM task queues (atomic
// counters; the queues of a full force walk hold their tasks costliest first, by the cycles
// each took in the previous one), and owns an overflow area in global memory for the deep
// part of its stack.  When
// there are too few tasks to fill the GPU (small N), each task is split in two, four or
// eight: warps walk the same 32 bodies, each from its share of the root's children (the root
// contains every body, so the guard opens it for all of them); two partial sums are added
// to the zeroed output with FP64 atomics (two addends: the result does not depend on their
// order), more are written to scratch and added in a fixed order by a closing pass.  Very
// small trees split in 64: eight parts per root child decide it alike, and each walks an
// eighth of its children; only the first takes the child's own term or its bodies.
// A second mode computes the vector-Jacobian product of the accelerations on the
// same decisions (see flush_vjp and k_vjp_finish); a third counts decisions and
// collects walk statistics.
#include <type_traits>

#include "internal.cuh"

namespace grav {
namespace {

constexpr int kWalkWarps = 4;
constexpr int kSmemStack = 128;                // stack entries in shared memory
constexpr int kGlobStack = 1152;               // further entries in global memory, per warp
constexpr int kStackCap = kSmemStack + kGlobStack;
constexpr int kFlushMax = 16;                  // lists are evaluated once they hold flush_at
constexpr int kListCap = kFlushMax + 32;       // (<= kFlushMax) terms; a batch appends <= 32

// Walk launch shapes selectable at run time (gravity_params.walk_cfg, autotuned):
// cfg = fi + 3 bi + 9 qi with flush_at = {16, 12, 8}[fi], resident blocks per SM =
// occupancy maximum - bi, and task queues per SM (qi = 0) or one global queue (qi = 1).
constexpr int kWalkConfigs = 18;
struct WalkShape { int flush_at, blocks_less, one_queue; };
inline WalkShape walk_shape(int cfg) {
  if (cfg < 0 || cfg >= kWalkConfigs) cfg = 0;
  const int fl[3] = {16, 12, 8};
  return WalkShape{fl[cfg % 3], (cfg / 3) % 3, cfg / 9};
}
constexpr int kSplitWarpsPerSM = 28;           // resident warps per SM of the monopole walk
constexpr uint32_t kFirstMask = 0x01FFFFFFu;   // 25-bit first index
constexpr int kCntShift = 25;                  // 6-bit (count - 1)

enum { kModeForce = 0, kModeCount = 1, kModeVjp = 2 };

// Walk statistics accumulated by the counted variant (introspection, not used on
// the timed path): batches, items, mixed nodes, FP64 decisions, point-list entries,
// node-term entries, deepest stack, lane-terms evaluated by active lanes, lockstep
// iterations of lists split by 16 / 8 / 1 lanes, full-mask entries, far entries,
// mixed nodes every tested lane decided alike, per-lane lockstep iterations of the
// point list.
enum { kStatBatches, kStatItems, kStatMixed, kStatFp64, kStatMono, kStatQuad, kStatMaxSp,
       kStatLaneTerms, kStatSplit2, kStatSplit4, kStatSplit32, kStatFull, kStatFar,
       kStatMixedUnanimous, kStatPointLane, kStatCount = 16 };

// The interaction lists are stored pair-interleaved: pair j holds entries 2j (a) and
// 2j + 1 (b), each float4 two fields of both, (f_a, f_b, g_a, g_b), so that one
// shared-memory load yields the operands of the packed instructions for both entries.
constexpr int kPairCap = kListCap / 2;
struct WarpSmem {
  uint2 st[kSmemStack];           // (first | (count-1) << 25, lane mask)
  float4 pA[kPairCap];            // point list: (x_hi, y_hi) of a pair of entries
  float4 pB[kPairCap];            //             (z_hi, m)
  float4 pC[kPairCap];            //             (x_lo, y_lo)
  float4 pD[kPairCap];            //             (z_lo, lane mask bits)
  float4 fA[kPairCap];            // far list:   (c_rel x, c_rel y)
  float4 fB[kPairCap];            //             (c_rel z, m)
  uint2 fM[kPairCap];             //             lane masks of entries a, b
  int32_t ltag[kListCap];         // counting / VJP: -(node+1) node term, else sorted body index
  float4 org_h, org_l;            // the warp origin (lane 0's body), hi and lo parts
  int32_t part;                   // split task: which share of the root's children
  float band_k, band_c;           // mixed-node test: FP64 band = 2^-16 l^2 + k D^2 + c
  int32_t bitem[32];              // node id of each lane's item (mixed nodes' FP64 decisions)
  float4 bcr[32];                 // a lane's mixed node: COM relative to the origin, l^2
  int4 lfx[32];                   // opened leaves of a batch: first body, bodies, lane mask
};

// Vector-Jacobian product (order 0): far-list sources and the lane-to-source
// transposition buffer (chunks of kVjpChunk entries; rows of 36 floats, so that a row
// starts on 16 bytes and the eight rows one quarter-warp reads as float4 fall in distinct
// banks).
constexpr int kVjpChunk = 8;
constexpr int kVjpRow = 36;
struct WarpSmemV {
  WarpSmem base;
  int32_t ftag[kListCap];         // node of each far entry
  __align__(16) float vt[3][kVjpChunk][kVjpRow];   // per component, entry and lane: gradient
};

// Quadrupole lists hold -Q (see the moments pass): (xx, yy), (zz, xy), (xz, yz).
struct WarpSmemQ {
  WarpSmem base;
  float4 fC[kPairCap], fD[kPairCap], fE[kPairCap];                  // far list -Q
  float4 nA[kPairCap], nB[kPairCap], nC[kPairCap], nD[kPairCap];    // near list, as point
  float4 nE[kPairCap], nF[kPairCap], nG[kPairCap];                  // near list -Q
};

// Field k (0: the x/y slots, 1: the z/w slots) of entry p of a pair-interleaved array.
__device__ __forceinline__ void put(float4 *a, int p, int k, float v) {
  reinterpret_cast<float *>(a + (p >> 1))[2 * k + (p & 1)] = v;
}
__device__ __forceinline__ float getf(const float4 *a, int p, int k) {
  return reinterpret_cast<const float *>(a + (p >> 1))[2 * k + (p & 1)];
}
// Zero the b half of pair j (an odd list's pad entry: mask 0, finite fields, adds 0).
__device__ __forceinline__ void zero_b(float4 &v) { v.y = 0.f; v.w = 0.f; }

// Packed two-wide FP32 arithmetic (IEEE round to nearest per element).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 xy2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 zw2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

struct WalkArgs {
  const float4 *bhi, *blo;
  const double *pos_s;
  const float4 *rec0, *rec1, *quadf;
  const int4 *topo;
  const int32_t *ndepth;
  const double *ncom;
  const double *geom;
  const uint32_t *perm;
  const int32_t *nnodes;
  int n;
  int ntasks;                     // tasks after splitting (base tasks x split)
  int split;                      // 1, 2, 4, 8 or 64 warps per base task (see above)
  double *part;                   // split >= 4: partial sums [split][rows][3] (rows = n or nrange)
  int rows;
  float theta2f;
  double theta2d;
  float eps2;
  double G;
  int mac_guard;
  int acc64;
  double *acc;
  int32_t *counts;
  double *vel;
  double kick;
  unsigned *status;
  int max_iter;
  unsigned *task_counter;         // [nqueues] per-queue counters, zeroed before the launch
  const int32_t *order;           // full force walk: the task of each queue slot (else null)
  uint32_t *cost;                 // full force walk: SM clock cycles each task took (else null)
  int nqueues;
  int flush_at;
  int stack_cap;                  // stack entries allowed (<= kStackCap)
  uint2 *gstack;                  // [persistent warps][kGlobStack] (first|cnt, mask)
  const int32_t *task_begin;      // several clouds: per task first body, cloud end, cloud id
  const int32_t *task_end;
  const int32_t *task_seg;
  unsigned long long *stats;      // counted variant only
  int task0;                      // first task of the walked range (0: all tasks)
  int split_basis;                // task count the split decision is taken on (the whole tree's)
  double *acc_sorted;             // range walk: rows in sorted order from body body0 (else null)
  int body0;
  int nrange;                     // bodies of the range (rows of acc_sorted)
  const double *lambda;           // VJP: cotangent of the accelerations, caller order (n,3)
  double *g_own;                  // VJP: gradient of each body from its own terms, sorted order
  double *g_body;                 // VJP: gradient scattered to body sources, sorted order
  double *g_node;                 // VJP: gradient scattered to node COMs
};

__device__ __forceinline__ int warp_incl_scan_i(int v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float p) {
  float s = hi + p;
  float bp = s - hi;
  float err = (hi - (s - bp)) + (p - bp);
  hi = s;
  lo += err;
}

// Per-body accumulator: a (hi, lo) two-sum pair per component, or (accum = 1) an FP64
// sum whose bits live in the same two 32-bit registers (hi word, lo word).
__device__ __forceinline__ void add64(float &h, float &l, float p) {
  const double d = __hiloint2double(__float_as_int(h), __float_as_int(l)) + (double)p;
  h = __int_as_float(__double2hiint(d));
  l = __int_as_float(__double2loint(d));
}
__device__ __forceinline__ double get64(float h, float l) {
  return __hiloint2double(__float_as_int(h), __float_as_int(l));
}

struct Accum {
  float hx = 0, hy = 0, hz = 0, lx = 0, ly = 0, lz = 0;   // all-zero bits = 0.0 as FP64 too
  __device__ __forceinline__ void add(bool acc64, float px, float py, float pz) {
    if (acc64) { add64(hx, lx, px); add64(hy, ly, py); add64(hz, lz, pz); }
    else { two_sum_add(hx, lx, px); two_sum_add(hy, ly, py); two_sum_add(hz, lz, pz); }
  }
  __device__ __forceinline__ void get(bool acc64, double &x, double &y, double &z) const {
    if (acc64) { x = get64(hx, lx); y = get64(hy, ly); z = get64(hz, lz); }
    else { x = (double)hx + (double)lx; y = (double)hy + (double)ly; z = (double)hz + (double)lz; }
  }
};

// 1/sqrt(r2) for an active lane, 0 otherwise.  With eps > 0, r2 >= eps^2 > 0;
// with eps = 0 a term with r2 = 0 (coincident bodies) contributes nothing.
template <bool EPS0>
__device__ __forceinline__ float inv_r(float r2, bool act) {
  const float inv = rsqrtf(r2);
  if (EPS0) return (act && r2 > 0.f) ? inv : 0.f;
  return act ? inv : 0.f;
}

template <bool EPS0>
__device__ __forceinline__ float2 inv_r2(float2 r2, unsigned ma, unsigned mb, unsigned lbit) {
  return make_float2(inv_r<EPS0>(r2.x, (ma & lbit) != 0u), inv_r<EPS0>(r2.y, (mb & lbit) != 0u));
}

// Counting variant only: decision counts of the entries of pair j.
template <bool POINT>
__device__ __forceinline__ void count_pair(const WarpSmem &S, int j, int cnt, unsigned ma,
                                           unsigned mb, unsigned lbit, int gi, int &c_m2p,
                                           int &c_p2p) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int k = 2 * j + h;
    if (k < cnt && ((h ? mb : ma) & lbit)) {
      if (!POINT) ++c_m2p;
      else if (S.ltag[k] < 0) ++c_m2p;
      else if (S.ltag[k] != gi) ++c_p2p;
    }
  }
}

// Point terms: a += m d / (|d|^2 + eps^2)^{3/2}, d = source - body (hi/lo), two
// entries per step.
template <bool EPS0, bool COUNT>
__device__ __forceinline__ void flush_point(WarpSmem &S, int cnt, int lane, float xh, float yh,
                                            float zh, float xl, float yl, float zl, float eps2,
                                            float &px, float &py, float &pz, int gi, int &c_m2p,
                                            int &c_p2p) {
  if (cnt & 1) {
    if (lane == 0) {
      const int j = cnt >> 1;
      zero_b(S.pA[j]); zero_b(S.pB[j]); zero_b(S.pC[j]); zero_b(S.pD[j]);
    }
    __syncwarp();
  }
  const unsigned lbit = 1u << lane;
  const float2 nxh = dup2(-xh), nyh = dup2(-yh), nzh = dup2(-zh);
  const float2 nxl = dup2(-xl), nyl = dup2(-yl), nzl = dup2(-zl), e2 = dup2(eps2);
  float2 ax = dup2(0.f), ay = dup2(0.f), az = dup2(0.f);
  const int np = (cnt + 1) >> 1;
#pragma unroll (EPS0 ? 1 : 2)
  for (int j = 0; j < np; ++j) {
    const float4 A = S.pA[j], B = S.pB[j], C = S.pC[j], D = S.pD[j];
    const float2 dx = add2(add2(xy2(A), nxh), add2(xy2(C), nxl));
    const float2 dy = add2(add2(zw2(A), nyh), add2(zw2(C), nyl));
    const float2 dz = add2(add2(xy2(B), nzh), add2(xy2(D), nzl));
    const float2 r2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, e2)));
    const unsigned ma = __float_as_uint(D.z), mb = __float_as_uint(D.w);
    const float2 inv = inv_r2<EPS0>(r2, ma, mb, lbit);
    const float2 sc = mul2(zw2(B), mul2(mul2(inv, inv), inv));
    ax = fma2(sc, dx, ax);
    ay = fma2(sc, dy, ay);
    az = fma2(sc, dz, az);
    if (COUNT) count_pair<true>(S, j, cnt, ma, mb, lbit, gi, c_m2p, c_p2p);
  }
  px = ax.x + ax.y;
  py = ay.x + ay.y;
  pz = az.x + az.y;
}

// Quadrupole node terms of two entries, with d = source - body and qn = -Q:
//   a += m d r^-3 - Q d r^-5 + (5/2) (d.Q d) d r^-7,  r^2 = |d|^2 + eps^2
// (the negative gradient of -m/r - y.Q y/(2 r^5), y = -d); with qn = -Q the signs are
// folded into the constant -5/2.
__device__ __forceinline__ void quad_term2(float2 dx, float2 dy, float2 dz, float2 m, float2 qxx,
                                           float2 qyy, float2 qzz, float2 qxy, float2 qxz,
                                           float2 qyz, float2 inv, float2 &ax, float2 &ay,
                                           float2 &az) {
  const float2 inv2 = mul2(inv, inv);
  const float2 inv3 = mul2(inv2, inv);
  const float2 inv5 = mul2(inv3, inv2);
  const float2 inv7 = mul2(inv5, inv2);
  const float2 qx = fma2(qxx, dx, fma2(qxy, dy, mul2(qxz, dz)));
  const float2 qy = fma2(qxy, dx, fma2(qyy, dy, mul2(qyz, dz)));
  const float2 qz = fma2(qxz, dx, fma2(qyz, dy, mul2(qzz, dz)));
  const float2 dqd = fma2(dx, qx, fma2(dy, qy, mul2(dz, qz)));
  const float2 sc = fma2(m, inv3, mul2(dup2(-2.5f), mul2(dqd, inv7)));
  ax = fma2(sc, dx, fma2(qx, inv5, ax));
  ay = fma2(sc, dy, fma2(qy, inv5, ay));
  az = fma2(sc, dz, fma2(qz, inv5, az));
}

// Far node terms on warp-relative coordinates (monopole, or + quadrupole), two entries
// per step.
template <int ORDER, bool EPS0, bool COUNT>
__device__ __forceinline__ void flush_far(void *Sv, int cnt, int lane, float xr, float yr,
                                          float zr, float eps2, float &px, float &py, float &pz,
                                          int &c_m2p) {
  WarpSmem &S = *reinterpret_cast<WarpSmem *>(Sv);
  if (cnt & 1) {
    if (lane == 0) {
      const int j = cnt >> 1;
      zero_b(S.fA[j]); zero_b(S.fB[j]); S.fM[j].y = 0u;
      if constexpr (ORDER == 2) {
        WarpSmemQ &Q = *reinterpret_cast<WarpSmemQ *>(Sv);
        zero_b(Q.fC[j]); zero_b(Q.fD[j]); zero_b(Q.fE[j]);
      }
    }
    __syncwarp();
  }
  const unsigned lbit = 1u << lane;
  const float2 nx = dup2(-xr), ny = dup2(-yr), nz = dup2(-zr), e2 = dup2(eps2);
  float2 ax = dup2(0.f), ay = dup2(0.f), az = dup2(0.f);
  const int np = (cnt + 1) >> 1;
#pragma unroll (ORDER == 2 ? 1 : 2)
  for (int j = 0; j < np; ++j) {
    const float4 A = S.fA[j], B = S.fB[j];
    const uint2 mk = S.fM[j];
    const float2 dx = add2(xy2(A), nx), dy = add2(zw2(A), ny), dz = add2(xy2(B), nz);
    const float2 r2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, e2)));
    const float2 inv = inv_r2<EPS0>(r2, mk.x, mk.y, lbit);
    if constexpr (ORDER == 2) {
      const WarpSmemQ &Q = *reinterpret_cast<const WarpSmemQ *>(Sv);
      const float4 C = Q.fC[j], D = Q.fD[j], E = Q.fE[j];
      quad_term2(dx, dy, dz, zw2(B), xy2(C), zw2(C), xy2(D), zw2(D), xy2(E), zw2(E), inv, ax, ay,
                 az);
    } else {
      const float2 sc = mul2(zw2(B), mul2(mul2(inv, inv), inv));
      ax = fma2(sc, dx, ax);
      ay = fma2(sc, dy, ay);
      az = fma2(sc, dz, az);
    }
    if (COUNT) {
      int unused = 0;
      count_pair<false>(S, j, cnt, mk.x, mk.y, lbit, 0, c_m2p, unused);
    }
  }
  px = ax.x + ax.y;
  py = ay.x + ay.y;
  pz = az.x + az.y;
}

// Near quadrupole node terms on hi/lo coordinates, two entries per step.
template <bool EPS0, bool COUNT>
__device__ __forceinline__ void flush_near(WarpSmemQ &Q, int cnt, int lane, float xh, float yh,
                                           float zh, float xl, float yl, float zl, float eps2,
                                           float &px, float &py, float &pz, int &c_m2p) {
  if (cnt & 1) {
    if (lane == 0) {
      const int j = cnt >> 1;
      zero_b(Q.nA[j]); zero_b(Q.nB[j]); zero_b(Q.nC[j]); zero_b(Q.nD[j]);
      zero_b(Q.nE[j]); zero_b(Q.nF[j]); zero_b(Q.nG[j]);
    }
    __syncwarp();
  }
  const unsigned lbit = 1u << lane;
  const float2 nxh = dup2(-xh), nyh = dup2(-yh), nzh = dup2(-zh);
  const float2 nxl = dup2(-xl), nyl = dup2(-yl), nzl = dup2(-zl), e2 = dup2(eps2);
  float2 ax = dup2(0.f), ay = dup2(0.f), az = dup2(0.f);
  const int np = (cnt + 1) >> 1;
#pragma unroll 1
  for (int j = 0; j < np; ++j) {
    const float4 A = Q.nA[j], B = Q.nB[j], C = Q.nC[j], D = Q.nD[j];
    const float2 dx = add2(add2(xy2(A), nxh), add2(xy2(C), nxl));
    const float2 dy = add2(add2(zw2(A), nyh), add2(zw2(C), nyl));
    const float2 dz = add2(add2(xy2(B), nzh), add2(xy2(D), nzl));
    const float2 r2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, e2)));
    const unsigned ma = __float_as_uint(D.z), mb = __float_as_uint(D.w);
    const float2 inv = inv_r2<EPS0>(r2, ma, mb, lbit);
    const float4 E = Q.nE[j], F = Q.nF[j], G = Q.nG[j];
    quad_term2(dx, dy, dz, zw2(B), xy2(E), zw2(E), xy2(F), zw2(F), xy2(G), zw2(G), inv, ax, ay, az);
    if (COUNT) {
      int unused = 0;
      count_pair<false>(Q.base, j, cnt, ma, mb, lbit, 0, c_m2p, unused);
    }
  }
  px = ax.x + ax.y;
  py = ay.x + ay.y;
  pz = az.x + az.y;
}

// Vector-Jacobian product of the monopole terms of a point (FAR = false) or far
// list.  A term a_i += m f(d), f(d) = d (|d|^2 + eps^2)^{-3/2}, d = s - x_i, with
// cotangent u_i gives w = m J(d) u_i, J = (I - 3 d d^T / r^2) / r^3 (symmetric):
// the body's own gradient takes -w (the sum over the list is returned in p*), the
// source s (a body, or a node whose COM moves with its bodies) takes +w.  The +w of
// the 32 lanes are summed per entry through shared memory (one lane per entry and
// component) and added with one FP64 atomic per entry and component.  The point
// list's own-body entry is skipped: its term does not depend on x_i.
template <bool FAR, bool EPS0>
__device__ __forceinline__ void flush_vjp(WarpSmemV &V, int cnt, int lane, float xh, float yh,
                                          float zh, float xl, float yl, float zl, float xr,
                                          float yr, float zr, float eps2, float ux, float uy,
                                          float uz, int gi, float &px, float &py, float &pz,
                                          double *g_body, double *g_node) {
  WarpSmem &S = V.base;
  if (cnt & 1) {                                  // pad entry: mask 0, finite fields
    if (lane == 0) {
      const int j = cnt >> 1;
      if (FAR) { zero_b(S.fA[j]); zero_b(S.fB[j]); S.fM[j].y = 0u; }
      else { zero_b(S.pA[j]); zero_b(S.pB[j]); zero_b(S.pC[j]); zero_b(S.pD[j]); }
    }
    __syncwarp();
  }
  const unsigned lbit = 1u << lane;
  const float2 e2 = dup2(eps2), u_x = dup2(ux), u_y = dup2(uy), u_z = dup2(uz), m3 = dup2(-3.f);
  const float2 nxh = dup2(FAR ? -xr : -xh), nyh = dup2(FAR ? -yr : -yh), nzh = dup2(FAR ? -zr : -zh);
  const float2 nxl = dup2(-xl), nyl = dup2(-yl), nzl = dup2(-zl);
  float2 ox = dup2(0.f), oy = dup2(0.f), oz = dup2(0.f);
  for (int c0 = 0; c0 < cnt; c0 += kVjpChunk) {
    const int ce = min(kVjpChunk, cnt - c0);
#pragma unroll
    for (int q = 0; q < kVjpChunk / 2; ++q) {
      if (2 * q < ce) {
        const int j = (c0 >> 1) + q;
        float2 dx, dy, dz, m;
        unsigned ma, mb;
        if (FAR) {
          const float4 A = S.fA[j], B = S.fB[j];
          const uint2 mk = S.fM[j];
          dx = add2(xy2(A), nxh); dy = add2(zw2(A), nyh); dz = add2(xy2(B), nzh);
          m = zw2(B);
          ma = mk.x; mb = mk.y;
        } else {
          const float4 A = S.pA[j], B = S.pB[j], C = S.pC[j], D = S.pD[j];
          dx = add2(add2(xy2(A), nxh), add2(xy2(C), nxl));
          dy = add2(add2(zw2(A), nyh), add2(zw2(C), nyl));
          dz = add2(add2(xy2(B), nzh), add2(xy2(D), nzl));
          m = zw2(B);
          ma = __float_as_uint(D.z); mb = __float_as_uint(D.w);
          if (S.ltag[2 * j] == gi) ma = 0u;       // the body's own entry: no dependence
          if (2 * j + 1 < cnt && S.ltag[2 * j + 1] == gi) mb = 0u;
        }
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, e2)));
        const float2 inv = inv_r2<EPS0>(r2, ma, mb, lbit);
        const float2 inv2 = mul2(inv, inv);
        const float2 sc = mul2(m, mul2(inv2, inv));
        const float2 c3n = mul2(mul2(m3, fma2(dx, u_x, fma2(dy, u_y, mul2(dz, u_z)))), inv2);
        const float2 wx = mul2(sc, fma2(c3n, dx, u_x));
        const float2 wy = mul2(sc, fma2(c3n, dy, u_y));
        const float2 wz = mul2(sc, fma2(c3n, dz, u_z));
        ox = add2(ox, wx); oy = add2(oy, wy); oz = add2(oz, wz);
        V.vt[0][2 * q][lane] = wx.x; V.vt[0][2 * q + 1][lane] = wx.y;
        V.vt[1][2 * q][lane] = wy.x; V.vt[1][2 * q + 1][lane] = wy.y;
        V.vt[2][2 * q][lane] = wz.x; V.vt[2][2 * q + 1][lane] = wz.y;
      }
    }
    __syncwarp();
    const int e = lane & (kVjpChunk - 1), comp = lane / kVjpChunk;
    if (comp < 3 && e < ce) {
      // the 32 lanes' terms of this entry and component, read as eight float4 and summed
      // as two packed pairs
      const float4 *row = reinterpret_cast<const float4 *>(V.vt[comp][e]);
      float2 sa = dup2(0.f), sb = dup2(0.f);
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const float4 v = row[jj];
        sa = add2(sa, xy2(v));
        sb = add2(sb, zw2(v));
      }
      const float sum = (sa.x + sa.y) + (sb.x + sb.y);
      if (sum != 0.f) {
        const int tag = FAR ? V.ftag[c0 + e] : S.ltag[c0 + e];
        double *dst = (!FAR && tag >= 0) ? g_body + 3 * (int64_t)tag
                                         : g_node + 3 * (int64_t)(FAR ? tag : -tag - 1);
        atomicAdd(dst + comp, (double)sum);
      }
    }
    __syncwarp();
  }
  px = ox.x + ox.y;
  py = oy.x + oy.y;
  pz = oz.x + oz.y;
}

// Counted variant only: lockstep iteration counts of lane-group-split lists (masks in
// the z/w slots of a pair-interleaved array, or, with m4 = nullptr, in a mask array).
__device__ __forceinline__ void split_costs(const float4 *m4, const uint2 *mu, int cnt, int lane,
                                            unsigned long long *st) {
  int c2 = 0, c4 = 0, c32 = 0, full = 0;
  const unsigned h = 0xFFFFu << (16 * (lane >> 4)), q = 0xFFu << (8 * (lane >> 3));
  for (int k = 0; k < cnt; ++k) {
    const unsigned m = m4 ? __float_as_uint(getf(m4, k, 1))
                          : reinterpret_cast<const unsigned *>(mu)[k];
    c2 += (m & h) != 0;
    c4 += (m & q) != 0;
    c32 += (m >> lane) & 1u;
    full += m == 0xFFFFFFFFu;
  }
  c2 = __reduce_max_sync(0xffffffffu, c2);
  c4 = __reduce_max_sync(0xffffffffu, c4);
  c32 = __reduce_max_sync(0xffffffffu, c32);
  if (lane == 0) {
    st[0] += c2; st[1] += c4; st[2] += c32; st[3] += full;
  }
}

// Stack slot access: [0, kSmemStack) in shared memory, the rest in the warp's
// global overflow area.
struct Stack {
  uint2 *s, *g;
  __device__ __forceinline__ void get(int i, uint32_t &a, uint32_t &m) const {
    uint2 v;
    if (i < kSmemStack) v = s[i];
    else v = g[i - kSmemStack];
    a = v.x; m = v.y;
  }
  __device__ __forceinline__ void set(int i, uint32_t a, uint32_t m) const {
    if (i < kSmemStack) s[i] = make_uint2(a, m);
    else g[i - kSmemStack] = make_uint2(a, m);
  }
  __device__ __forceinline__ void set_a(int i, uint32_t a) const {
    if (i < kSmemStack) s[i].x = a;
    else g[i - kSmemStack].x = a;
  }
};

// The force mode is held to 6 (quadrupole: 80 registers; the shared memory of its lists
// allows no more) or 7 (monopole: 72 registers) resident blocks of 4 warps per SM, the VJP
// mode to 6 (80 registers); the counted mode is not held to any.
// 64-way split: the start of part `sub` of a task (see the kernel).  The root child c
// (first_entry) is decided per lane by the FP64 test the walk's exact decisions equal (a
// body inside c opens it under the guard).  Share 0 keeps c for the accepting lanes (the walk
// takes their term, and counts their test, when it pops c) and counts the opening lanes'
// test; every share walks its eighth of c's children for the opening lanes.  A leaf c is
// walked whole by share 0.  Returns the number of stack entries set.  Not inlined: its FP64
// registers stay out of the walk's register budget.
template <bool COUNT>
__device__ __noinline__ int split64_start(const WalkArgs &A, const Stack &st, uint32_t first_entry,
                                          int sub, int gi, bool valid, unsigned vm, int root,
                                          int &c_tests) {
  const int lane = threadIdx.x & 31;
  const int cnode = (int)(first_entry & kFirstMask);
  const int4 ct = A.topo[cnode];
  if (ct.x < 0) {
    if (sub != 0) return 0;
    if (lane == 0) st.set(0, first_entry, vm);
    return 1;
  }
  bool op = false;
  if (valid) {
    op = A.mac_guard && ct.z <= gi && gi < ct.w;
    if (!op) {
      const double X = A.ncom[3 * cnode], Y = A.ncom[3 * cnode + 1], Z = A.ncom[3 * cnode + 2];
      const double x = A.pos_s[3 * gi], y = A.pos_s[3 * gi + 1], z = A.pos_s[3 * gi + 2];
      const double ddx = __dsub_rn(X, x), ddy = __dsub_rn(Y, y), ddz = __dsub_rn(Z, z);
      const double D2d = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)),
                                   __dmul_rn(ddz, ddz));
      const double l = __dmul_rn(A.geom[8 * root + 3], pow2_neg(A.ndepth[cnode]));
      op = !(__dmul_rn(l, l) < __dmul_rn(A.theta2d, D2d));
      if (COUNT && op && sub == 0) ++c_tests;
    }
  }
  const unsigned openv = __ballot_sync(0xffffffffu, valid && op);
  const unsigned accv = vm & ~openv;
  const int h2 = (ct.y + 7) >> 3, f2 = sub * h2, c2 = min(h2, ct.y - f2);
  int sp = 0;
  if (sub == 0 && accv) {
    if (lane == 0) st.set(sp, first_entry, accv);
    ++sp;
  }
  if (openv && c2 > 0) {
    if (lane == 0) st.set(sp, (uint32_t)(ct.x + f2) | ((uint32_t)(c2 - 1) << kCntShift), openv);
    ++sp;
  }
  return sp;
}

template <int ORDER, bool EPS0, int MODE, bool S64>
__global__ void __launch_bounds__(32 * kWalkWarps, MODE == kModeCount ? 1 : (ORDER == 2 || MODE == kModeVjp ? 6 : 7))
k_walk(WalkArgs A) {
  constexpr bool COUNT = MODE == kModeCount;
  constexpr bool VJP = MODE == kModeVjp;
  static_assert(!VJP || ORDER == 0, "the vector-Jacobian product covers monopole terms");
  using Smem = typename std::conditional<
      ORDER == 2, WarpSmemQ, typename std::conditional<VJP, WarpSmemV, WarpSmem>::type>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  Smem &S = reinterpret_cast<Smem *>(smem_raw)[wib];
  WarpSmem &M = *reinterpret_cast<WarpSmem *>(&S);
  const Stack st{M.st, A.gstack + (size_t)(blockIdx.x * kWalkWarps + wib) * kGlobStack};

  const int n = A.n;
  const int nn = *A.nnodes;
  const float theta2f = A.theta2f;
  const float eps2 = A.eps2;
  const bool acc64 = A.acc64 != 0;

  // Tasks (32 consecutive bodies) are split into one contiguous queue per SM, so
  // that the warps resident on an SM walk neighbouring bodies and share node
  // records in L1; a warp whose queue is empty takes tasks from the next queues.
  unsigned smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  const int nq = A.nqueues;
  int q = (int)(smid % (unsigned)nq);
  int visited = 0;                            // queues moved past (each found exhausted)
  for (;;) {
    int task = -1;
    while (visited < nq) {
      if (lane == 0) {
        const int qbeg = (int)(((long long)A.ntasks * q) / nq);
        const int qend = (int)(((long long)A.ntasks * (q + 1)) / nq);
        if (qbeg < qend) {
          const int t = qbeg + (int)atomicAdd(&A.task_counter[q], 1u);
          if (t < qend) task = t;
        }
      }
      task = __shfl_sync(0xffffffffu, task, 0);
      if (task >= 0) break;
      // queue q is exhausted (counters only grow): read the counters of the queues after it
      // 32 at a time from L2, without atomics, and go on to the first that still has tasks
      int adv = 0;
      for (int base = 1; base < nq - visited && adv == 0; base += 32) {
        bool live = false;
        if (base + lane < nq - visited) {
          int qq = q + base + lane;
          if (qq >= nq) qq -= nq;
          const int qb = (int)(((long long)A.ntasks * qq) / nq);
          const int qe = (int)(((long long)A.ntasks * (qq + 1)) / nq);
          live = qb + (int)__ldcg(&A.task_counter[qq]) < qe;
        }
        const unsigned lv = __ballot_sync(0xffffffffu, live);
        if (lv) adv = base + __ffs(lv) - 1;
      }
      if (adv == 0) { visited = nq; break; }
      visited += adv;
      q += adv;
      if (q >= nq) q -= nq;
    }
    if (task < 0) break;
    if (A.order) task = A.order[task];          // the queue's tasks, costliest first
    const int slot_task = task;
    const long long t_task = A.cost ? clock64() : 0;

    // task: up to 32 consecutive bodies of one cloud; the walk starts at the cloud root
    const int part = A.split > 1 ? task % A.split : 0;
    task = (A.split > 1 ? task / A.split : task) + A.task0;
    const int wbeg = A.task_begin ? A.task_begin[task] : task * 32;
    const int wend = min(A.task_begin ? A.task_end[task] : n, wbeg + 32);
    const int root = A.task_seg ? A.task_seg[task] : 0;
    // first stack entry: the root, or (split) this part's share of the root's children;
    // 64 parts (S64): root child part / 8, of whose children the part walks share part % 8
    uint32_t first_entry = (uint32_t)root;
    if (A.split > 1) {
      const int4 rt = A.topo[root];
      if (rt.x < 0) {                           // a one-leaf tree: part 0 takes it whole
        if (part != 0) continue;
      } else {
        const int p1 = S64 ? part >> 3 : part;
        const int h = (rt.y + (S64 ? 8 : A.split) - 1) / (S64 ? 8 : A.split);
        const int cnt = min(h, rt.y - p1 * h);
        if (cnt <= 0) continue;
        first_entry = (uint32_t)(rt.x + p1 * h) | ((uint32_t)(cnt - 1) << kCntShift);
      }
    }
    const int gi = wbeg + lane;
    const bool valid = gi < wend;

    float xh = 0, yh = 0, zh = 0, xl = 0, yl = 0, zl = 0;
    if (valid) {
      const float4 h = A.bhi[gi], l = A.blo[gi];
      xh = h.x; yh = h.y; zh = h.z; xl = l.x; yl = l.y; zl = l.z;
    }
    float ux = 0.f, uy = 0.f, uz = 0.f;       // VJP: cotangent of this body's acceleration, x G
    if (VJP && valid) {
      const int64_t ci = A.perm[gi];
      ux = (float)(A.G * A.lambda[3 * ci]);
      uy = (float)(A.G * A.lambda[3 * ci + 1]);
      uz = (float)(A.G * A.lambda[3 * ci + 2]);
    }
    // warp origin = lane 0's body (always valid); warp-relative FP32 coordinates
    const float ohx = __shfl_sync(0xffffffffu, xh, 0), ohy = __shfl_sync(0xffffffffu, yh, 0),
                ohz = __shfl_sync(0xffffffffu, zh, 0), olx = __shfl_sync(0xffffffffu, xl, 0),
                oly = __shfl_sync(0xffffffffu, yl, 0), olz = __shfl_sync(0xffffffffu, zl, 0);
    if (lane == 0) {                            // kept in shared memory for the far appends
      M.org_h = make_float4(ohx, ohy, ohz, 0.f);
      M.org_l = make_float4(olx, oly, olz, 0.f);
      M.part = part;                            // (read back when the sums are written)
    }
    const float xr = valid ? (xh - ohx) + (xl - olx) : 0.f;
    const float yr = valid ? (yh - ohy) + (yl - oly) : 0.f;
    const float zr = valid ? (zh - ohz) + (zl - olz) : 0.f;
    // bounding box of the bodies (hi parts) and extent around the origin
    float bminx = valid ? xh : INFINITY, bminy = valid ? yh : INFINITY, bminz = valid ? zh : INFINITY;
    float bmaxx = valid ? xh : -INFINITY, bmaxy = valid ? yh : -INFINITY, bmaxz = valid ? zh : -INFINITY;
    float rw2 = fmaf(xr, xr, fmaf(yr, yr, zr * zr));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      bminx = fminf(bminx, __shfl_xor_sync(0xffffffffu, bminx, o));
      bminy = fminf(bminy, __shfl_xor_sync(0xffffffffu, bminy, o));
      bminz = fminf(bminz, __shfl_xor_sync(0xffffffffu, bminz, o));
      bmaxx = fmaxf(bmaxx, __shfl_xor_sync(0xffffffffu, bmaxx, o));
      bmaxy = fmaxf(bmaxy, __shfl_xor_sync(0xffffffffu, bmaxy, o));
      bmaxz = fmaxf(bmaxz, __shfl_xor_sync(0xffffffffu, bmaxz, o));
      rw2 = fmaxf(rw2, __shfl_xor_sync(0xffffffffu, rw2, o));
    }
    {
      // widen the box by del = 2^-19 (R + C), R = the bodies' largest |coordinate| and C a
      // bound of every node COM's (the root cube's largest |corner coordinate|): a bound on
      // the hi/lo truncation and rounding of the box distances below
      const double *gr = A.geom + 8 * root;
      const float C = (float)fmax(fmax(fmax(fabs(gr[0]), fabs(gr[0] + gr[3])),
                                       fmax(fabs(gr[1]), fabs(gr[1] + gr[3]))),
                                  fmax(fabs(gr[2]), fabs(gr[2] + gr[3])));
      const float bR = fmaxf(fmaxf(fmaxf(fabsf(bminx), fabsf(bmaxx)), fmaxf(fabsf(bminy), fabsf(bmaxy))),
                             fmaxf(fabsf(bminz), fabsf(bmaxz)));
      const float del = (bR + C) * 1.9073486e-6f;
      bminx -= del; bminy -= del; bminz -= del;
      bmaxx += del; bmaxy += del; bmaxz += del;
    }
    // a node with l^2 >= farl2 is at least R_w / 2 from every body that accepts it
    // (D > l / theta), which bounds the far-path error of d by 5.5 * 2^-23 |d|
    const float farl2 = 0.25f * theta2f * rw2 * 1.01f;
    if (lane == 0) {
      // the per-lane test of a mixed node runs on warp-relative coordinates: with R_w^2 =
      // rw2, the error of d = c_rel - x_rel is below 2^-23 (1.5 D + 2 R_w) (the origin
      // offset being exact to 2^-24 of each coordinate), that of the FP32 D^2 below
      // 2^-22 (3.25 D^2 + R_w^2); a result within 2^-16 l^2 + theta^2 2^-20 (D^2 + R_w^2) of
      // the boundary (four times that bound) is taken in FP64, so the decision is exact
      M.band_k = theta2f * 9.5367431640625e-7f;
      M.band_c = theta2f * 9.5367431640625e-7f * rw2;
    }

    Accum acc;
    int c_m2p = 0, c_p2p = 0, c_tests = 0;
    unsigned long long w_batches = 0, w_items = 0, w_mixed = 0, w_mono = 0, w_quad = 0, w_far = 0;
    unsigned long long w_split[4] = {0, 0, 0, 0};
    unsigned long long w_psplit[4] = {0, 0, 0, 0};   // the point list alone
    int w_maxsp = 0;
    int npt = 0, nfar = 0, nnear = 0;
    int sp = 1;
    bool abort = false;
    {
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      if constexpr (S64) {
        sp = split64_start<COUNT>(A, st, first_entry, part & 7, gi, valid, vm, root, c_tests);
      } else {
        if (lane == 0) st.set(0, first_entry, vm);    // root (or a share of its children)
      }
    }
    __syncwarp();

    // evaluates the point list into the accumulator and empties it
    auto flush_pt = [&]() {
      if (COUNT) {
        w_mono += npt;
        split_costs(M.pD, nullptr, npt, lane, w_split);
        split_costs(M.pD, nullptr, npt, lane, w_psplit);
      }
      float px, py, pz;
      if constexpr (VJP)
        flush_vjp<false, EPS0>(S, npt, lane, xh, yh, zh, xl, yl, zl, xr, yr, zr, eps2, ux, uy, uz,
                               gi, px, py, pz, A.g_body, A.g_node);
      else
        flush_point<EPS0, COUNT>(M, npt, lane, xh, yh, zh, xl, yl, zl, eps2, px, py, pz, gi,
                                 c_m2p, c_p2p);
      acc.add(acc64, px, py, pz);
      npt = 0;
      __syncwarp();
    };
    for (int iter = 0; sp > 0; ++iter) {
      if (iter > A.max_iter) {                  // cannot happen on a well-formed tree
        if (lane == 0) latch_error(A.status, kErrTree);
        abort = true;
        break;
      }
      // ---- pop up to 32 items from the top entries (lane 0 = top of stack)
      const int ke = sp - 1 - lane;
      uint32_t ea = 0, em = 0;
      int ecnt = 0;
      if (ke >= 0) {
        st.get(ke, ea, em);
        ecnt = (int)((ea >> kCntShift) & 63u) + 1;
      }
      const int incl = warp_incl_scan_i(ecnt, lane);
      const int excl = incl - ecnt;
      const int take = max(0, min(ecnt, 32 - excl));
      const unsigned fullm = __ballot_sync(0xffffffffu, ecnt > 0 && take == ecnt);
      const int nfull = __popc(fullm);
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      const int nitems = min(total, 32);
      __syncwarp();
      if (take > 0 && take < ecnt) {           // the one partially consumed entry stays
        st.set_a(ke, (((ea & kFirstMask) + take) & kFirstMask) |
                         ((uint32_t)(ecnt - take - 1) << kCntShift));
      }
      sp -= nfull;
      const unsigned starts = __reduce_or_sync(0xffffffffu, take > 0 ? (1u << excl) : 0u);
      const unsigned starts_le = starts & (0xffffffffu >> (31 - lane));
      const int stpos = 31 - __clz(starts_le);
      const int owner = __popc(starts_le) - 1;
      const uint32_t oa = __shfl_sync(0xffffffffu, ea, owner);
      const uint32_t omask = __shfl_sync(0xffffffffu, em, owner);
      const bool have = lane < nitems;
      if (COUNT) { ++w_batches; w_items += nitems; }
      const int item = (int)(oa & kFirstMask) + (lane - stpos);

      // ---- load and classify (lane = item)
      float4 r0 = make_float4(0, 0, 0, 0), r1 = make_float4(0, 0, 0, 0);
      float4 q0 = make_float4(0, 0, 0, 0), q1 = make_float4(0, 0, 0, 0);
      int4 tp = make_int4(-1, 0, 0, 0);
      bool single = false;                     // a one-body leaf: a point term
      bool bad = false;
      if (have) {
        bad = item >= nn;
        if (!bad) {
          tp = A.topo[item];
          r0 = A.rec0[item];
          r1 = A.rec1[item];
          if constexpr (ORDER == 2) {          // in flight during classification
            q0 = A.quadf[2 * item];
            q1 = A.quadf[2 * item + 1];
          }
          single = r1.w < 0.f;                 // the record holds the body itself
          bad = (tp.x >= 0 && (tp.x <= 0 || tp.x + tp.y > nn)) || tp.z < 0 || tp.w > n ||
                tp.z >= tp.w;
        }
      }
      if (__any_sync(0xffffffffu, bad)) {
        if (lane == 0) latch_error(A.status, kErrTree);
        abort = true;
        break;
      }
      unsigned accm = 0, openm = 0;
      unsigned tmask = 0;                      // mixed node: the lanes that test it themselves
      bool mixed = false;
      if (have) {
        if (single) {
          accm = omask;
        } else {
          const float cx = r0.x, cy = r0.y, cz = r0.z, l2 = r1.w;
          const float gx = fmaxf(fmaxf(bminx - cx, cx - bmaxx), 0.f);    // widened box
          const float gy = fmaxf(fmaxf(bminy - cy, cy - bmaxy), 0.f);
          const float gz = fmaxf(fmaxf(bminz - cz, cz - bmaxz), 0.f);
          const float fx = fmaxf(fabsf(cx - bminx), fabsf(cx - bmaxx));
          const float fy = fmaxf(fabsf(cy - bminy), fabsf(cy - bmaxy));
          const float fz = fmaxf(fabsf(cz - bminz), fabsf(cz - bmaxz));
          const float dmin2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
          const float dmax2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
          const bool guard_any = A.mac_guard && tp.z < wend && tp.w > wbeg;
          if (!guard_any && l2 < theta2f * dmin2 * 0.999f) {
            accm = omask;
          } else if (l2 > theta2f * dmax2 * 1.001f) {
            openm = omask;
          } else {
            mixed = true;
            unsigned gm = 0;                   // lanes whose body is in the node: opened
            if (A.mac_guard) {
              const int lo = min(max(tp.z - wbeg, 0), 32), hi = min(max(tp.w - wbeg, 0), 32);
              gm = (unsigned)(((1ull << hi) - 1ull) & ~((1ull << lo) - 1ull));
            }
            tmask = omask & ~gm;
          }
        }
      }
      if (COUNT) {                             // MAC tests per body (introspection only)
        for (int j = 0; j < nitems; ++j) {
          const bool sj = __shfl_sync(0xffffffffu, single, j);
          const unsigned mj = __shfl_sync(0xffffffffu, omask, j);
          const int bj = __shfl_sync(0xffffffffu, tp.z, j), ej = __shfl_sync(0xffffffffu, tp.w, j);
          if (!sj && ((mj >> lane) & 1u) && !(A.mac_guard && bj <= gi && gi < ej)) ++c_tests;
        }
      }
      // ---- exact per-lane test for mixed nodes: the owner lane broadcasts the node's
      // record and the mask of lanes that test it; every other lane of the node's mask
      // has its body inside the node and opens it
      unsigned mixed_bits = __ballot_sync(0xffffffffu, mixed);
      if (COUNT) w_mixed += __popc(mixed_bits);
      if (mixed_bits) {
        if (mixed) {                           // the node's COM relative to the warp origin
          M.bitem[lane] = item;
          const float4 oh = M.org_h, ol = M.org_l;
          M.bcr[lane] = make_float4((r0.x - oh.x) + (r1.x - ol.x), (r0.y - oh.y) + (r1.y - ol.y),
                                    (r0.z - oh.z) + (r1.z - ol.z), r1.w);
        }
        __syncwarp();
      }
      while (mixed_bits) {
        const int j = __ffs(mixed_bits) - 1;
        mixed_bits &= mixed_bits - 1;
        const unsigned tk = __shfl_sync(0xffffffffu, tmask, j);
        bool a_i = false;
        if (tk & (1u << lane)) {
          const float4 c = M.bcr[j];
          const float dx = c.x - xr, dy = c.y - yr, dz = c.z - zr;
          const float D2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          const float diff = c.w - theta2f * D2;
          if (fabsf(diff) <= fmaf(M.band_k, D2, fmaf(1.52587890625e-5f, c.w, M.band_c))) {
            // within the band of the FP32 test's error: decide in FP64
            const int node = M.bitem[j];
            const double X = A.ncom[3 * node], Y = A.ncom[3 * node + 1], Z = A.ncom[3 * node + 2];
            const double x = A.pos_s[3 * gi], y = A.pos_s[3 * gi + 1], z = A.pos_s[3 * gi + 2];
            const double ddx = __dsub_rn(X, x), ddy = __dsub_rn(Y, y), ddz = __dsub_rn(Z, z);
            const double D2d = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)),
                                         __dmul_rn(ddz, ddz));
            const double l = __dmul_rn(A.geom[8 * root + 3], pow2_neg(A.ndepth[node]));
            a_i = __dmul_rn(l, l) < __dmul_rn(A.theta2d, D2d);
            if (COUNT) atomicAdd(&A.stats[kStatFp64], 1ull);
          } else {
            a_i = diff < 0.f;
          }
        }
        const unsigned am = __ballot_sync(0xffffffffu, a_i);
        if (lane == j) { accm = am; openm = omask & ~am; }   // tested lanes accept or open
        if (COUNT) {
          const unsigned mk = __shfl_sync(0xffffffffu, omask, j);
          if (lane == 0 && (am == mk || am == 0u)) atomicAdd(&A.stats[kStatMixedUnanimous], 1ull);
        }
      }

      // ---- append accepted terms: point / far / near
      const bool node_term = accm != 0 && !single;
      const bool to_far = node_term && r1.w >= farl2;
      const bool to_near = (ORDER == 2) && node_term && !to_far;
      const bool to_pt = accm != 0 && !to_far && !to_near;
      {
        const unsigned bm = __ballot_sync(0xffffffffu, to_pt);
        if (to_pt) {
          const int p = npt + __popc(bm & ((1u << lane) - 1u));
          put(M.pA, p, 0, r0.x); put(M.pA, p, 1, r0.y); put(M.pB, p, 0, r0.z); put(M.pB, p, 1, r0.w);
          put(M.pC, p, 0, r1.x); put(M.pC, p, 1, r1.y); put(M.pD, p, 0, r1.z);
          put(M.pD, p, 1, __uint_as_float(accm));
          if (COUNT || VJP) M.ltag[p] = single ? tp.z : -(item + 1);
        }
        npt += __popc(bm);
      }
      {
        const unsigned bf = __ballot_sync(0xffffffffu, to_far);
        if (to_far) {
          const int p = nfar + __popc(bf & ((1u << lane) - 1u));
          const float4 oh = M.org_h, ol = M.org_l;
          const float cx = (r0.x - oh.x) + (r1.x - ol.x);
          const float cy = (r0.y - oh.y) + (r1.y - ol.y);
          const float cz = (r0.z - oh.z) + (r1.z - ol.z);
          put(M.fA, p, 0, cx); put(M.fA, p, 1, cy); put(M.fB, p, 0, cz); put(M.fB, p, 1, r0.w);
          reinterpret_cast<unsigned *>(M.fM)[p] = accm;
          if constexpr (VJP) S.ftag[p] = item;
          if constexpr (ORDER == 2) {
            put(S.fC, p, 0, q0.x); put(S.fC, p, 1, q0.y); put(S.fD, p, 0, q0.z);
            put(S.fD, p, 1, q0.w); put(S.fE, p, 0, q1.x); put(S.fE, p, 1, q1.y);
          }
        }
        nfar += __popc(bf);
        if (COUNT) w_far += __popc(bf);
      }
      if constexpr (ORDER == 2) {
        const unsigned bq = __ballot_sync(0xffffffffu, to_near);
        if (to_near) {
          const int p = nnear + __popc(bq & ((1u << lane) - 1u));
          put(S.nA, p, 0, r0.x); put(S.nA, p, 1, r0.y); put(S.nB, p, 0, r0.z); put(S.nB, p, 1, r0.w);
          put(S.nC, p, 0, r1.x); put(S.nC, p, 1, r1.y); put(S.nD, p, 0, r1.z);
          put(S.nD, p, 1, __uint_as_float(accm));
          put(S.nE, p, 0, q0.x); put(S.nE, p, 1, q0.y); put(S.nF, p, 0, q0.z);
          put(S.nF, p, 1, q0.w); put(S.nG, p, 0, q1.x); put(S.nG, p, 1, q1.y);
        }
        nnear += __popc(bq);
      }

      // ---- push opened internal nodes (their children range)
      const bool push = openm != 0 && tp.x >= 0;
      const unsigned pb = __ballot_sync(0xffffffffu, push);
      const int ptotal = __popc(pb);
      if (sp + ptotal > A.stack_cap) {
        if (lane == 0) latch_error(A.status, kErrStack);
        abort = true;
        break;
      }
      if (push)
        st.set(sp + __popc(pb & ((1u << lane) - 1u)),
               (uint32_t)tp.x | ((uint32_t)(tp.y - 1) << kCntShift), openm);
      sp += ptotal;
      if (COUNT) w_maxsp = max(w_maxsp, sp);

      // ---- opened leaves: their bodies go straight to the point list as body terms of
      // the opening lanes, packed 32 to a round (leaves compacted in shared memory first);
      // the point list is evaluated when a round might not fit, and when full at the end
      const bool open_leaf = openm != 0 && tp.x < 0;
      const unsigned lm = __ballot_sync(0xffffffffu, open_leaf);
      int4 lf = make_int4(0, 0, 0, 0);
      int lincl = 0, ltot = 0;
      if (lm) {
        if (open_leaf) M.lfx[__popc(lm & ((1u << lane) - 1u))] = make_int4(tp.z, tp.w - tp.z, (int)openm, 0);
        __syncwarp();
        if (lane < __popc(lm)) lf = M.lfx[lane];
        lincl = warp_incl_scan_i(lf.y, lane);
        ltot = __shfl_sync(0xffffffffu, lincl, 31);
      }
      __syncwarp();
      for (int base = 0;; base += 32) {
        const bool more = base < ltot;
        if (more ? npt > kListCap - 32 : npt >= A.flush_at) flush_pt();
        if (!more) break;
        // round [base, base + 32): the leaves overlapping it are consecutive, from the
        // first one not ended before it; slot base + lane belongs to the last of them
        // starting at or before the slot
        const int lexcl = lincl - lf.y;
        const bool in_round = lf.y > 0 && lexcl < base + 32 && lincl > base;
        const unsigned starts = __reduce_or_sync(0xffffffffu, in_round ? 1u << max(lexcl - base, 0) : 0u);
        const int first = __popc(__ballot_sync(0xffffffffu, lf.y > 0 && lincl <= base));
        const int li = first + __popc(starts & (0xffffffffu >> (31 - lane))) - 1;
        const int b0 = __shfl_sync(0xffffffffu, lf.x, li);
        const int bx = __shfl_sync(0xffffffffu, lexcl, li);
        const unsigned bm = (unsigned)__shfl_sync(0xffffffffu, lf.z, li);
        const int take = min(32, ltot - base);
        if (lane < take) {
          const int body = b0 + (base + lane - bx);
          const float4 h = A.bhi[body], l = A.blo[body];
          const int p = npt + lane;
          put(M.pA, p, 0, h.x); put(M.pA, p, 1, h.y); put(M.pB, p, 0, h.z); put(M.pB, p, 1, h.w);
          put(M.pC, p, 0, l.x); put(M.pC, p, 1, l.y); put(M.pD, p, 0, l.z);
          put(M.pD, p, 1, __uint_as_float(bm));
          if (COUNT || VJP) M.ltag[npt + lane] = body;
        }
        npt += take;
        __syncwarp();
      }

      // ---- evaluate the other full lists
      if (nfar >= A.flush_at) {
        if (COUNT) { w_quad += nfar; split_costs(nullptr, M.fM, nfar, lane, w_split); }
        float px, py, pz;
        if constexpr (VJP)
          flush_vjp<true, EPS0>(S, nfar, lane, xh, yh, zh, xl, yl, zl, xr, yr, zr, eps2, ux, uy, uz,
                                gi, px, py, pz, A.g_body, A.g_node);
        else
          flush_far<ORDER, EPS0, COUNT>(&S, nfar, lane, xr, yr, zr, eps2, px, py, pz, c_m2p);
        acc.add(acc64, px, py, pz);
        nfar = 0;
        __syncwarp();
      }
      if constexpr (ORDER == 2) {
        if (nnear >= A.flush_at) {
          if (COUNT) { w_quad += nnear; split_costs(S.nD, nullptr, nnear, lane, w_split); }
          float px, py, pz;
          flush_near<EPS0, COUNT>(S, nnear, lane, xh, yh, zh, xl, yl, zl, eps2, px, py, pz,
                                  c_m2p);
          acc.add(acc64, px, py, pz);
          nnear = 0;
          __syncwarp();
        }
      }
    }
    if (!abort) {
      if (COUNT) {
        w_mono += npt; w_quad += nfar + nnear;
        if (npt > 0) {
          split_costs(M.pD, nullptr, npt, lane, w_split);
          split_costs(M.pD, nullptr, npt, lane, w_psplit);
        }
        if (nfar > 0) split_costs(nullptr, M.fM, nfar, lane, w_split);
        if constexpr (ORDER == 2) { if (nnear > 0) split_costs(S.nD, nullptr, nnear, lane, w_split); }
      }
      float px, py, pz;
      if (npt > 0) {
        if constexpr (VJP)
          flush_vjp<false, EPS0>(S, npt, lane, xh, yh, zh, xl, yl, zl, xr, yr, zr, eps2, ux, uy, uz,
                                 gi, px, py, pz, A.g_body, A.g_node);
        else
          flush_point<EPS0, COUNT>(M, npt, lane, xh, yh, zh, xl, yl, zl, eps2, px, py, pz, gi,
                                   c_m2p, c_p2p);
        acc.add(acc64, px, py, pz);
      }
      if (nfar > 0) {
        if constexpr (VJP)
          flush_vjp<true, EPS0>(S, nfar, lane, xh, yh, zh, xl, yl, zl, xr, yr, zr, eps2, ux, uy, uz,
                                gi, px, py, pz, A.g_body, A.g_node);
        else
          flush_far<ORDER, EPS0, COUNT>(&S, nfar, lane, xr, yr, zr, eps2, px, py, pz, c_m2p);
        acc.add(acc64, px, py, pz);
      }
      if constexpr (ORDER == 2) {
        if (nnear > 0) {
          flush_near<EPS0, COUNT>(S, nnear, lane, xh, yh, zh, xl, yl, zl, eps2, px, py, pz, c_m2p);
          acc.add(acc64, px, py, pz);
        }
      }
    }
    __syncwarp();
    if (COUNT) {
      const unsigned long long lt =
          __reduce_add_sync(0xffffffffu, (unsigned)(valid ? c_m2p + c_p2p : 0));
      if (lane == 0) {
        atomicAdd(&A.stats[kStatBatches], w_batches);
        atomicAdd(&A.stats[kStatItems], w_items);
        atomicAdd(&A.stats[kStatMixed], w_mixed);
        atomicAdd(&A.stats[kStatMono], w_mono);
        atomicAdd(&A.stats[kStatQuad], w_quad);
        atomicMax(&A.stats[kStatMaxSp], (unsigned long long)w_maxsp);
        atomicAdd(&A.stats[kStatLaneTerms], lt);
        atomicAdd(&A.stats[kStatSplit2], w_split[0]);
        atomicAdd(&A.stats[kStatSplit4], w_split[1]);
        atomicAdd(&A.stats[kStatSplit32], w_split[2]);
        atomicAdd(&A.stats[kStatFull], w_split[3]);
        atomicAdd(&A.stats[kStatFar], w_far);
        atomicAdd(&A.stats[kStatPointLane], w_psplit[2]);
      }
    }
    if (VJP && valid) {                         // own-term gradient, sorted order
      double gx, gy, gz;
      acc.get(acc64, gx, gy, gz);
      if (A.split > 1) {
        atomicAdd(&A.g_own[3 * gi], -gx);
        atomicAdd(&A.g_own[3 * gi + 1], -gy);
        atomicAdd(&A.g_own[3 * gi + 2], -gz);
      } else {
        A.g_own[3 * gi] = -gx;
        A.g_own[3 * gi + 1] = -gy;
        A.g_own[3 * gi + 2] = -gz;
      }
    }
    if (!VJP && valid && A.split > 1) {         // partial sums of a split task
      double ax, ay, az;
      acc.get(acc64, ax, ay, az);
      double *dst;
      if (A.part) {                             // four or more parts: added in a fixed order later
        dst = A.part + 3 * ((int64_t)M.part * A.rows + (gi - A.body0));
      } else {                                  // two parts: two addends, order-free
        dst = A.acc_sorted ? A.acc_sorted + 3 * (int64_t)(gi - A.body0)
                           : A.acc + 3 * (int64_t)A.perm[gi];
      }
      if (A.part) {
        dst[0] = ax * A.G;
        dst[1] = ay * A.G;
        dst[2] = az * A.G;
      } else {
        atomicAdd(dst, ax * A.G);
        atomicAdd(dst + 1, ay * A.G);
        atomicAdd(dst + 2, az * A.G);
      }
      if (COUNT) {
        const int64_t ci = A.perm[gi];
        atomicAdd(&A.counts[3 * ci], c_m2p);
        atomicAdd(&A.counts[3 * ci + 1], c_p2p);
        atomicAdd(&A.counts[3 * ci + 2], c_tests);
      }
    }
    if (!VJP && valid && A.split == 1 && A.acc_sorted) {   // range walk: sorted rows
      double ax, ay, az;
      acc.get(acc64, ax, ay, az);
      double *dst = A.acc_sorted + 3 * (int64_t)(gi - A.body0);
      dst[0] = ax * A.G;
      dst[1] = ay * A.G;
      dst[2] = az * A.G;
    }
    if (!VJP && valid && A.split == 1 && !A.acc_sorted) {
      double ax, ay, az;
      acc.get(acc64, ax, ay, az);
      ax *= A.G; ay *= A.G; az *= A.G;
      const int64_t ci = A.perm[gi];
      A.acc[3 * ci] = ax;
      A.acc[3 * ci + 1] = ay;
      A.acc[3 * ci + 2] = az;
      if (A.vel) {                              // fused closing kick of the leapfrog
        A.vel[3 * ci] = __dadd_rn(A.vel[3 * ci], __dmul_rn(A.kick, ax));
        A.vel[3 * ci + 1] = __dadd_rn(A.vel[3 * ci + 1], __dmul_rn(A.kick, ay));
        A.vel[3 * ci + 2] = __dadd_rn(A.vel[3 * ci + 2], __dmul_rn(A.kick, az));
      }
      if (COUNT) {
        A.counts[3 * ci] = c_m2p;
        A.counts[3 * ci + 1] = c_p2p;
        A.counts[3 * ci + 2] = c_tests;
      }
    }
    if (A.cost && lane == 0)
      A.cost[slot_task] = (uint32_t)min(clock64() - t_task, (long long)0xFFFFFFFFu);
  }
}

// Split in four or more: the parts' partial sums added in a fixed order (so results do not
// depend on which warp finished first), written in caller order (or as range rows), with
// the leapfrog's closing kick when asked for.
__device__ __forceinline__ void finish_row(int i, const double *a, const uint32_t *__restrict__ perm,
                                           double *__restrict__ acc, double *__restrict__ acc_sorted,
                                           double *__restrict__ vel, double kick) {
  if (acc_sorted) {
    acc_sorted[3 * (int64_t)i] = a[0];
    acc_sorted[3 * (int64_t)i + 1] = a[1];
    acc_sorted[3 * (int64_t)i + 2] = a[2];
    return;
  }
  const int64_t ci = perm[i];
  acc[3 * ci] = a[0];
  acc[3 * ci + 1] = a[1];
  acc[3 * ci + 2] = a[2];
  if (vel) {
    vel[3 * ci] = __dadd_rn(vel[3 * ci], __dmul_rn(kick, a[0]));
    vel[3 * ci + 1] = __dadd_rn(vel[3 * ci + 1], __dmul_rn(kick, a[1]));
    vel[3 * ci + 2] = __dadd_rn(vel[3 * ci + 2], __dmul_rn(kick, a[2]));
  }
}

// Up to 8 parts: one thread per row, every part loaded before the sums (part by part).
__global__ void k_walk_finish(const double *__restrict__ part, int rows, int nparts,
                              const uint32_t *__restrict__ perm, double *__restrict__ acc,
                              double *__restrict__ acc_sorted, double *__restrict__ vel,
                              double kick) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  double v[8][3];
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int k = 0; k < 3; ++k) v[q][k] = q < nparts ? part[3 * ((int64_t)q * rows + i) + k] : 0.0;
  double a[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double sum = v[0][k];
#pragma unroll
    for (int q = 1; q < 8; ++q)
      if (q < nparts) sum = __dadd_rn(sum, v[q][k]);
    a[k] = sum;
  }
  finish_row(i, a, perm, acc, acc_sorted, vel, kick);
}

// 64 parts: 8 lanes per row, lane g summing parts 8g .. 8g+7 in order, then a butterfly
// over the row's lanes (every lane ends with the same sum, a + b and b + a being equal).
__global__ void __launch_bounds__(256) k_walk_finish64(const double *__restrict__ part, int rows,
                                                       const uint32_t *__restrict__ perm,
                                                       double *__restrict__ acc,
                                                       double *__restrict__ acc_sorted,
                                                       double *__restrict__ vel, double kick) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = t >> 3, g = t & 7;
  const bool in = i < rows;                    // alike in the 8 lanes of a row
  double a[3] = {0.0, 0.0, 0.0};
  if (in) {
    double v[8][3];
#pragma unroll
    for (int q = 0; q < 8; ++q)
#pragma unroll
      for (int k = 0; k < 3; ++k) v[q][k] = part[3 * ((int64_t)(8 * g + q) * rows + i) + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double sum = v[0][k];
#pragma unroll
      for (int q = 1; q < 8; ++q) sum = __dadd_rn(sum, v[q][k]);
      a[k] = sum;
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < 3; ++k) a[k] = __dadd_rn(a[k], __shfl_xor_sync(0xffffffffu, a[k], o));
  if (in && g == 0) finish_row(i, a, perm, acc, acc_sorted, vel, kick);
}

// Task order of the next full force walk: the tasks of each queue (the queues' contiguous
// ranges of the task list) sorted by the cycles they took in the last one, costliest first
// (ties by task index), so that the long tasks start early and the queue ends with short
// ones.  The order decides only which warp takes a task when: every task computes the same
// result wherever it runs.  A queue of more than kOrderMax tasks keeps its order.
constexpr int kOrderMax = 4096;
__global__ void __launch_bounds__(512) k_order_tasks(const uint32_t *__restrict__ cost,
                                                     int32_t *__restrict__ order, int ntasks,
                                                     int nq) {
  __shared__ unsigned long long key[kOrderMax];
  const int q = blockIdx.x;
  const int qbeg = (int)(((long long)ntasks * q) / nq);
  const int qend = (int)(((long long)ntasks * (q + 1)) / nq);
  const int m = qend - qbeg;
  if (m <= 1 || m > kOrderMax) return;
  int p2 = 1;
  while (p2 < m) p2 <<= 1;
  // key: cost in the high word, the complement of the task index in the low word (so that
  // a descending sort puts equal costs in ascending index order); pads are 0 and sort last
  for (int i = threadIdx.x; i < p2; i += blockDim.x)
    key[i] = i < m ? ((unsigned long long)cost[qbeg + i] << 32) | (0xFFFFFFFFu - (unsigned)(qbeg + i))
                   : 0ull;
  __syncthreads();
  for (int k = 2; k <= p2; k <<= 1) {              // bitonic sort, descending
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < p2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long a = key[i], b = key[l];
          const bool desc = (i & k) == 0;
          if (desc ? a < b : a > b) { key[i] = b; key[l] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    order[qbeg + i] = (int32_t)(0xFFFFFFFFu - (unsigned)(key[i] & 0xFFFFFFFFull));
}

// Identity task order and zero costs (a new task count or queue count).
__global__ void k_order_reset(int32_t *__restrict__ order, uint32_t *__restrict__ cost, int ntasks) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ntasks; i += gridDim.x * blockDim.x) {
    order[i] = i;
    cost[i] = 0u;
  }
}

// Warps per base task: split tasks when the tree has no more of them than a full GPU of
// warps, in four when it has no more than half as many, in eight when no more than a
// quarter, in 64 when no more than a 32nd (force and counted walks; each root child's
// children shared by eight parts).  The decision depends only on the whole tree's task count
// and the SM count (not on the kernel variant, the launch shape or a range), so every
// variant and a range walk compute what the full walk does; the VJP adds its parts' own-term
// gradients with FP64 atomics (its source scatter is order-dependent in the last bits anyway).
int walk_split(const Ctx *c, const WalkArgs &A, bool allow64) {
  const int basis = A.split_basis > 0 ? A.split_basis : A.ntasks;
  const int slots = kSplitWarpsPerSM * c->num_sms;
  if (!A.mac_guard) return 1;
  if (allow64 && 32 * basis <= slots) return 64;
  return 4 * basis <= slots ? 8 : 2 * basis <= slots ? 4 : basis <= slots ? 2 : 1;
}

template <int ORDER, bool EPS0, int MODE, bool S64>
int launch_walk_s(Ctx *c, WalkArgs A) {
  using Smem = typename std::conditional<
      ORDER == 2, WarpSmemQ,
      typename std::conditional<MODE == kModeVjp, WarpSmemV, WarpSmem>::type>::type;
  const size_t smem = sizeof(Smem) * kWalkWarps;
  auto kern = k_walk<ORDER, EPS0, MODE, S64>;
  static int blocks_per_sm[64] = {0};
  const int dev = c->device < 64 ? c->device : 63;
  if (blocks_per_sm[dev] == 0) {
    GRAV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaFuncAttributes fa{};
    GRAV_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    int regs_blocks = 65536 / (fa.numRegs * 32 * kWalkWarps);
    if (regs_blocks < 1) regs_blocks = 1;
    int smem_sm = 0;
    GRAV_CUDA_TRY(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device));
    const double need = (double)regs_blocks * (smem + 1024);
    int pct = (int)(100.0 * need / smem_sm) + 1;
    if (pct > 100) pct = 100;
    GRAV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    int b = 0;
    GRAV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 32 * kWalkWarps, smem));
    blocks_per_sm[dev] = b > 0 ? b : 1;
  }
  const WalkShape shape = walk_shape(c->params.walk_cfg);
  A.flush_at = shape.flush_at;
  A.stack_cap = (c->stack_cap > 0 && c->stack_cap < kStackCap) ? c->stack_cap : kStackCap;
  int bps = blocks_per_sm[dev] - shape.blocks_less;
  if (bps < 1) bps = 1;
  int blocks = bps * c->num_sms;
  const int base_tasks = A.ntasks;
  A.split = walk_split(c, A, MODE != kModeVjp);  // 64 exactly when S64 (launch_walk)
  A.ntasks = base_tasks * A.split;
  const int rows = A.acc_sorted ? A.nrange : A.n;
  A.rows = rows;
  A.part = nullptr;
  if (A.split >= 4 && MODE != kModeVjp) {
    const size_t need_part = (size_t)3 * A.split * rows;
    if (need_part > c->walk_part_cap) {
      GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
      ctx_release(c, c->walk_part);
      c->walk_part_cap = 0;
      const int rc = ctx_alloc(c, c->walk_part, (int64_t)need_part);
      if (rc) return rc;
      c->walk_part_cap = need_part;
    }
    A.part = c->walk_part;
    GRAV_CUDA_TRY(cudaMemsetAsync(A.part, 0, sizeof(double) * need_part, c->stream));
    if (MODE == kModeCount)
      GRAV_CUDA_TRY(cudaMemsetAsync(A.counts, 0, sizeof(int32_t) * 3 * (size_t)A.n, c->stream));
  } else if (A.split > 1) {
    const size_t n3 = 3 * (size_t)A.n;
    if (MODE == kModeVjp) {
      GRAV_CUDA_TRY(cudaMemsetAsync(A.g_own, 0, sizeof(double) * n3, c->stream));
    } else if (A.acc_sorted) {
      GRAV_CUDA_TRY(cudaMemsetAsync(A.acc_sorted, 0, sizeof(double) * 3 * (size_t)A.nrange,
                                    c->stream));
    } else {
      GRAV_CUDA_TRY(cudaMemsetAsync(A.acc, 0, sizeof(double) * n3, c->stream));
      if (MODE == kModeCount)
        GRAV_CUDA_TRY(cudaMemsetAsync(A.counts, 0, sizeof(int32_t) * n3, c->stream));
    }
  }
  double *kick_vel = A.vel;                 // the fused kick needs the whole sum
  if (A.split > 1) A.vel = nullptr;
  const int need = (A.ntasks + kWalkWarps - 1) / kWalkWarps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  const size_t gneed = (size_t)blocks * kWalkWarps * kGlobStack;
  if (gneed > c->walk_gstack_cap) {
    GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
    ctx_release(c, c->walk_gstack);
    c->walk_gstack_cap = 0;
    void *gs = nullptr;
    const int rc = ctx_malloc(c, &gs, gneed * sizeof(uint2));
    if (rc) return rc;
    c->walk_gstack = gs;
    c->walk_gstack_cap = gneed;
  }
  A.gstack = reinterpret_cast<uint2 *>(c->walk_gstack);
  A.nqueues = shape.one_queue ? 1 : c->num_sms;
  GRAV_CUDA_TRY(cudaMemsetAsync(A.task_counter, 0, sizeof(unsigned) * A.nqueues, c->stream));
  // a full force walk takes its tasks in the order the last one's costs give and records
  // its own; the range, counted and VJP walks take them in index order, and so does a walk
  // with no more tasks than resident warps (all of them start at once: no order to keep)
  A.order = nullptr;
  A.cost = nullptr;
  const bool ordered = MODE == kModeForce && A.task0 == 0 && !A.acc_sorted &&
                       A.ntasks > bps * c->num_sms * kWalkWarps;
  if (ordered) {
    if (A.ntasks > c->walk_order_cap) {
      GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
      ctx_release(c, c->walk_cost);
      ctx_release(c, c->walk_order);
      c->walk_order_cap = 0;
      c->walk_order_n = 0;
      int rc = ctx_alloc(c, c->walk_cost, (int64_t)A.ntasks);
      if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->walk_order, (int64_t)A.ntasks);
      if (rc) return rc;
      c->walk_order_cap = A.ntasks;
    }
    if (c->walk_order_n != A.ntasks || c->walk_order_nq != A.nqueues) {
      const int tb = 256;
      const int gb = (int)std::min<int64_t>((A.ntasks + tb - 1) / tb, 4 * (int64_t)c->num_sms);
      k_order_reset<<<gb > 0 ? gb : 1, tb, 0, c->stream>>>(c->walk_order, c->walk_cost, A.ntasks);
      ++c->launches;
      GRAV_CUDA_TRY(cudaGetLastError());
      c->walk_order_n = A.ntasks;
      c->walk_order_nq = A.nqueues;
    }
    A.order = c->walk_order;
    A.cost = c->walk_cost;
  }
  kern<<<blocks, 32 * kWalkWarps, smem, c->stream>>>(A);
  ++c->launches;
  GRAV_CUDA_TRY(cudaGetLastError());
  if (ordered) {
    k_order_tasks<<<A.nqueues, 512, 0, c->stream>>>(c->walk_cost, c->walk_order, A.ntasks,
                                                    A.nqueues);
    ++c->launches;
    GRAV_CUDA_TRY(cudaGetLastError());
  }
  if (A.split >= 4 && MODE != kModeVjp) {
    if (A.split == 64)
      k_walk_finish64<<<(unsigned)((8 * (int64_t)rows + 255) / 256), 256, 0, c->stream>>>(
          A.part, rows, A.perm, A.acc_sorted ? nullptr : A.acc, A.acc_sorted, kick_vel, A.kick);
    else
      k_walk_finish<<<(unsigned)((rows + 255) / 256), 256, 0, c->stream>>>(
          A.part, rows, A.split, A.perm, A.acc_sorted ? nullptr : A.acc, A.acc_sorted, kick_vel,
          A.kick);
    ++c->launches;
    return cuda_status(cudaGetLastError());
  }
  if (A.split > 1 && kick_vel) return launch_kick(c, A.n, kick_vel, A.acc, A.kick);
  return GRAVITY_OK;
}

template <int ORDER, bool EPS0, int MODE>
int launch_walk(Ctx *c, WalkArgs A) {
  if constexpr (MODE != kModeVjp) {
    if (walk_split(c, A, true) == 64) return launch_walk_s<ORDER, EPS0, MODE, true>(c, A);
  }
  return launch_walk_s<ORDER, EPS0, MODE, false>(c, A);
}

}  // namespace

int walk_stack_capacity() { return kStackCap; }

int64_t walk_task_count(const Ctx *c) {
  return c->seg.nseg > 1 ? (int64_t)c->seg.ntasks : (c->n + 31) / 32;
}

int walk_forces_range(Ctx *c, double theta, double eps, int64_t first_task, int64_t ntasks,
                      int64_t body0, int64_t nbodies, double *acc_sorted) {
  Tree &t = c->t;
  WalkArgs A{};
  A.bhi = t.body_hi; A.blo = t.body_lo; A.pos_s = t.pos_s;
  A.rec0 = t.nrec0; A.rec1 = t.nrec1; A.quadf = t.nquadf;
  A.topo = t.topo; A.ndepth = t.ndepth; A.ncom = t.ncom; A.geom = t.geom;
  A.perm = t.idx; A.nnodes = t.nnodes;
  A.n = (int)c->n;
  if (c->seg.nseg > 1) {
    A.task_begin = c->seg.task_begin;
    A.task_end = c->seg.task_end;
    A.task_seg = c->seg.task_seg;
  }
  A.ntasks = (int)ntasks;
  A.task0 = (int)first_task;
  A.split_basis = (int)walk_task_count(c);
  A.acc_sorted = acc_sorted;
  A.body0 = (int)body0;
  A.nrange = (int)nbodies;
  A.theta2d = theta * theta;
  A.theta2f = (float)(theta * theta);
  A.eps2 = (float)(eps * eps);
  A.G = c->params.G;
  A.mac_guard = c->params.mac_guard;
  A.acc64 = c->params.accum == 1;
  A.status = c->d_status;
  A.max_iter = (int)(8 * c->n + 64);
  A.task_counter = c->walk_queues;
  A.stats = c->walk_stats;
  const bool q = c->params.order == 2;
  const bool e0 = !(A.eps2 > 0.f);
  if (q) return e0 ? launch_walk<2, true, kModeForce>(c, A) : launch_walk<2, false, kModeForce>(c, A);
  return e0 ? launch_walk<0, true, kModeForce>(c, A) : launch_walk<0, false, kModeForce>(c, A);
}

int walk_forces(Ctx *c, double theta, double eps, double *acc, int32_t *counts, double *vel,
                double kick) {
  Tree &t = c->t;
  WalkArgs A{};
  A.bhi = t.body_hi; A.blo = t.body_lo; A.pos_s = t.pos_s;
  A.rec0 = t.nrec0; A.rec1 = t.nrec1; A.quadf = t.nquadf;
  A.topo = t.topo; A.ndepth = t.ndepth; A.ncom = t.ncom; A.geom = t.geom;
  A.perm = t.idx; A.nnodes = t.nnodes;
  A.n = (int)c->n;
  if (c->seg.nseg > 1) {
    A.ntasks = c->seg.ntasks;
    A.task_begin = c->seg.task_begin;
    A.task_end = c->seg.task_end;
    A.task_seg = c->seg.task_seg;
  } else {
    A.ntasks = (int)((c->n + 31) / 32);
  }
  A.theta2d = theta * theta;
  A.theta2f = (float)(theta * theta);
  A.eps2 = (float)(eps * eps);
  A.G = c->params.G;
  A.mac_guard = c->params.mac_guard;
  A.acc64 = c->params.accum == 1;
  A.acc = acc; A.counts = counts; A.vel = vel; A.kick = kick;
  A.status = c->d_status;
  A.max_iter = (int)(8 * c->n + 64);
  A.task_counter = c->walk_queues;
  A.stats = c->walk_stats;
  if (counts) {
    GRAV_CUDA_TRY(cudaMemsetAsync(c->walk_stats, 0, sizeof(unsigned long long) * 16, c->stream));
  }
  const bool q = c->params.order == 2;
  const bool e0 = !(A.eps2 > 0.f);
  if (counts) {
    if (q) return e0 ? launch_walk<2, true, kModeCount>(c, A) : launch_walk<2, false, kModeCount>(c, A);
    return e0 ? launch_walk<0, true, kModeCount>(c, A) : launch_walk<0, false, kModeCount>(c, A);
  }
  if (q) return e0 ? launch_walk<2, true, kModeForce>(c, A) : launch_walk<2, false, kModeForce>(c, A);
  return e0 ? launch_walk<0, true, kModeForce>(c, A) : launch_walk<0, false, kModeForce>(c, A);
}

namespace {

// Closing pass of the vector-Jacobian product: a node COM is sum_j m_j x_j / M over
// its bodies, so the gradient scattered to a node reaches each of its bodies j as
// (m_j / M) g_node.  One thread per leaf sums g_node / M along the leaf's ancestor
// chain and writes, for each of its bodies, own + body-source + m_j * that sum in
// caller order.
__global__ void k_vjp_finish(const int4 *__restrict__ topo, const int32_t *__restrict__ nparent,
                             const double *__restrict__ nmass, const int32_t *__restrict__ nnodes,
                             const double *__restrict__ mass_s, const uint32_t *__restrict__ perm,
                             const double *__restrict__ g_own, const double *__restrict__ g_body,
                             const double *__restrict__ g_node, double *__restrict__ grad,
                             int64_t node_cap, unsigned *status) {
  const int64_t nn = *nnodes;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nn && k < node_cap;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int4 tp = topo[k];
    if (tp.x >= 0) continue;                  // leaves only
    double sx = 0.0, sy = 0.0, sz = 0.0;
    int a = (int)k, guard = 0;
    for (; a >= 0 && guard < 4 * kLevels + 8; a = nparent[a], ++guard) {
      const double M = nmass[a];
      if (M > 0.0) {
        sx = __dadd_rn(sx, __ddiv_rn(g_node[3 * (int64_t)a], M));
        sy = __dadd_rn(sy, __ddiv_rn(g_node[3 * (int64_t)a + 1], M));
        sz = __dadd_rn(sz, __ddiv_rn(g_node[3 * (int64_t)a + 2], M));
      }
    }
    if (a >= 0) { latch_error(status, kErrTree); continue; }
    for (int j = tp.z; j < tp.w; ++j) {
      const double m = mass_s[j];
      const int64_t ci = perm[j];
      grad[3 * ci] = g_own[3 * (int64_t)j] + g_body[3 * (int64_t)j] + m * sx;
      grad[3 * ci + 1] = g_own[3 * (int64_t)j + 1] + g_body[3 * (int64_t)j + 1] + m * sy;
      grad[3 * ci + 2] = g_own[3 * (int64_t)j + 2] + g_body[3 * (int64_t)j + 2] + m * sz;
    }
  }
}

}  // namespace

int walk_vjp(Ctx *c, double theta, double eps, const double *lambda, double *grad) {
  return walk_vjp_tree(c, c->t, theta, eps, lambda, grad);
}

int walk_vjp_tree(Ctx *c, const Tree &t, double theta, double eps, const double *lambda,
                  double *grad) {
  const int64_t n = c->n;
  const int64_t node_cap = 2 * c->cap;
  if (c->vjp_cap < c->cap) {
    GRAV_CUDA_TRY(cudaStreamSynchronize(c->stream));
    ctx_release(c, c->vjp_own);
    ctx_release(c, c->vjp_body);
    ctx_release(c, c->vjp_node);
    c->vjp_cap = 0;
    int rc = ctx_alloc(c, c->vjp_own, 3 * c->cap);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->vjp_body, 3 * c->cap);
    if (rc == GRAVITY_OK) rc = ctx_alloc(c, c->vjp_node, 3 * node_cap);
    if (rc) return rc;
    c->vjp_cap = c->cap;
  }
  GRAV_CUDA_TRY(cudaMemsetAsync(c->vjp_body, 0, sizeof(double) * 3 * n, c->stream));
  GRAV_CUDA_TRY(cudaMemsetAsync(c->vjp_node, 0, sizeof(double) * 3 * 2 * n, c->stream));
  WalkArgs A{};
  A.bhi = t.body_hi; A.blo = t.body_lo; A.pos_s = t.pos_s;
  A.rec0 = t.nrec0; A.rec1 = t.nrec1; A.quadf = t.nquadf;
  A.topo = t.topo; A.ndepth = t.ndepth; A.ncom = t.ncom; A.geom = t.geom;
  A.perm = t.idx; A.nnodes = t.nnodes;
  A.n = (int)n;
  if (c->seg.nseg > 1) {
    A.ntasks = c->seg.ntasks;
    A.task_begin = c->seg.task_begin;
    A.task_end = c->seg.task_end;
    A.task_seg = c->seg.task_seg;
  } else {
    A.ntasks = (int)((n + 31) / 32);
  }
  A.theta2d = theta * theta;
  A.theta2f = (float)(theta * theta);
  A.eps2 = (float)(eps * eps);
  A.G = c->params.G;
  A.mac_guard = c->params.mac_guard;
  A.acc64 = c->params.accum == 1;
  A.status = c->d_status;
  A.max_iter = (int)(8 * n + 64);
  A.task_counter = c->walk_queues;
  A.lambda = lambda;
  A.g_own = c->vjp_own; A.g_body = c->vjp_body; A.g_node = c->vjp_node;
  const bool e0 = !(A.eps2 > 0.f);
  int rc = e0 ? launch_walk<0, true, kModeVjp>(c, A) : launch_walk<0, false, kModeVjp>(c, A);
  if (rc) return rc;
  const int threads = 256;
  int64_t blocks = (2 * n + threads - 1) / threads;
  if (blocks > 8 * (int64_t)c->num_sms) blocks = 8 * (int64_t)c->num_sms;
  if (blocks < 1) blocks = 1;
  k_vjp_finish<<<(int)blocks, threads, 0, c->stream>>>(t.topo, t.nparent, t.nmass, t.nnodes,
                                                       t.mass_s, t.idx, c->vjp_own, c->vjp_body,
                                                       c->vjp_node, grad, node_cap, c->d_status);
  ++c->launches;
  return cuda_status(cudaGetLastError());
}

}  // namespace grav
