// Kernel 5 of the paper's list (Sec. 2.1, "compute forces"): the tree walk.
//
// The paper assigns one thread per body and relies on body sorting so that
// neighbouring threads traverse similar sub-trees.  Here a warp owns 32 bodies
// that are consecutive in Morton order and walks ONE shared stack for all of them,
// while every decision stays per body:
//   * stack entries are ranges of sibling nodes (children are contiguous) or of
//     bucket bodies, each with the 32-bit mask of lanes that still need them;
//   * up to 32 stacked items are taken at once, one per lane, and classified
//     against the bounding box of the warp's bodies: "accepted by every lane",
//     "opened by every lane" or "mixed";
//   * a mixed node is tested by each lane with the exact opening test of
//     Eq. (accuracy): l^2 < theta^2 D^2 in FP32 on hi/lo coordinates; a result
//     within a relative 2^-16 of the boundary is recomputed in FP64 exactly as
//     the oracle does, so every decision equals the FP64 one;
//   * accepted nodes (Eq. Force_thetaTrue; + quadrupole) and body-to-body terms
//     (Eq. Force_leaf) go to a shared-memory list that all lanes evaluate with
//     the softened r of Eq. (Force_rComp); inactive lanes add zero.
// Pair terms are FP32 with d = (c_hi - x_hi) + (c_lo - x_lo); each flushed list's
// partial sum enters a (hi, lo) two-sum accumulator (or an FP64 one).
#include <type_traits>

#include "internal.cuh"

namespace grav {
namespace {

constexpr int kWalkWarps = 4;
constexpr int kStackCap = 512;
constexpr int kListCap = 64;
constexpr int kFlushAt = 32;
constexpr uint32_t kKindBody = 0x80000000u;
constexpr uint32_t kFirstMask = 0x01FFFFFFu;   // 25-bit first index
constexpr int kCntShift = 25;                  // 6-bit (count - 1)

// Walk statistics accumulated by the counted variant (introspection, not used on the
// timed path): batches, items, mixed nodes, FP64 decisions, point-list entries,
// quadrupole-list entries, deepest stack, lane-terms evaluated by active lanes.
enum { kStatBatches, kStatItems, kStatMixed, kStatFp64, kStatMono, kStatQuad, kStatMaxSp,
       kStatLaneTerms, kStatCount };

struct WarpSmemMono {
  uint32_t st_a[kStackCap];       // first | (count-1) << 25 | kind
  uint32_t st_m[kStackCap];       // lane mask
  float4 la[kListCap];            // (x_hi, y_hi, z_hi, m)
  float4 lb[kListCap];            // (x_lo, y_lo, z_lo, lane mask bits)
  int32_t ltag[kListCap];         // counting: -1 node term, else sorted body index
};

struct WarpSmemQuad {
  WarpSmemMono mono;
  float4 qa[kListCap], qb[kListCap], qc[kListCap], qd[kListCap];
};

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
  float theta2f;
  double theta2d;
  float eps2;
  double G;
  int mac_guard;
  double *acc;
  int32_t *counts;
  double *vel;
  double kick;
  unsigned *status;
  int max_iter;
  unsigned long long *stats;     // counted variant only: walk statistics (see kStat*)
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

template <bool ACC64>
struct Accum {
  float hx = 0, hy = 0, hz = 0, lx = 0, ly = 0, lz = 0;
  double dx = 0, dy = 0, dz = 0;
  __device__ __forceinline__ void add(float px, float py, float pz) {
    if (ACC64) { dx += (double)px; dy += (double)py; dz += (double)pz; }
    else { two_sum_add(hx, lx, px); two_sum_add(hy, ly, py); two_sum_add(hz, lz, pz); }
  }
  __device__ __forceinline__ void get(double &x, double &y, double &z) const {
    if (ACC64) { x = dx; y = dy; z = dz; }
    else { x = (double)hx + (double)lx; y = (double)hy + (double)ly; z = (double)hz + (double)lz; }
  }
};

// Monopole / body terms: a += m d / (|d|^2 + eps^2)^{3/2}, d = source - body.
template <bool COUNT>
__device__ __forceinline__ void flush_mono(const WarpSmemMono &S, int cnt, int lane, float xh,
                                           float yh, float zh, float xl, float yl, float zl,
                                           float eps2, float &px, float &py, float &pz,
                                           int gi, int &c_m2p, int &c_p2p) {
  px = py = pz = 0.f;
#pragma unroll 4
  for (int k = 0; k < cnt; ++k) {
    float4 a = S.la[k];
    float4 b = S.lb[k];
    bool act = (__float_as_uint(b.w) >> lane) & 1u;
    float dx = (a.x - xh) + (b.x - xl);
    float dy = (a.y - yh) + (b.y - yl);
    float dz = (a.z - zh) + (b.z - zl);
    float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
    float inv = rsqrtf(r2);
    inv = (act && r2 > 0.f) ? inv : 0.f;
    float s = a.w * (inv * inv * inv);
    px = fmaf(s, dx, px);
    py = fmaf(s, dy, py);
    pz = fmaf(s, dz, pz);
    if (COUNT && act) {
      int tag = S.ltag[k];
      if (tag < 0) ++c_m2p;
      else if (tag != gi) ++c_p2p;
    }
  }
}

// Quadrupole node terms: a += m d r^-3 - Q d r^-5 + (5/2) (d.Q d) d r^-7 with
// r^2 = |d|^2 + eps^2 (the negative gradient of -m/r - y.Q y/(2 r^5), y = -d).
template <bool COUNT>
__device__ __forceinline__ void flush_quad(const WarpSmemQuad &S, int cnt, int lane, float xh,
                                           float yh, float zh, float xl, float yl, float zl,
                                           float eps2, float &px, float &py, float &pz,
                                           int &c_m2p) {
  px = py = pz = 0.f;
#pragma unroll 2
  for (int k = 0; k < cnt; ++k) {
    float4 a = S.qa[k], b = S.qb[k], q0 = S.qc[k], q1 = S.qd[k];
    bool act = (__float_as_uint(b.w) >> lane) & 1u;
    float dx = (a.x - xh) + (b.x - xl);
    float dy = (a.y - yh) + (b.y - yl);
    float dz = (a.z - zh) + (b.z - zl);
    float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
    float inv = rsqrtf(r2);
    inv = (act && r2 > 0.f) ? inv : 0.f;
    float inv2 = inv * inv;
    float inv3 = inv2 * inv;
    float inv5 = inv3 * inv2;
    float inv7 = inv5 * inv2;
    float qx = fmaf(q0.x, dx, fmaf(q0.w, dy, q1.x * dz));
    float qy = fmaf(q0.w, dx, fmaf(q0.y, dy, q1.y * dz));
    float qz = fmaf(q1.x, dx, fmaf(q1.y, dy, q0.z * dz));
    float dqd = fmaf(dx, qx, fmaf(dy, qy, dz * qz));
    float s = fmaf(a.w, inv3, 2.5f * dqd * inv7);
    px = fmaf(s, dx, fmaf(-qx, inv5, px));
    py = fmaf(s, dy, fmaf(-qy, inv5, py));
    pz = fmaf(s, dz, fmaf(-qz, inv5, pz));
    if (COUNT && act) ++c_m2p;
  }
}

template <int ORDER, bool ACC64, bool COUNT>
__global__ void __launch_bounds__(32 * kWalkWarps)
k_walk(WalkArgs A) {
  using Smem = typename std::conditional<ORDER == 2, WarpSmemQuad, WarpSmemMono>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  Smem &S = reinterpret_cast<Smem *>(smem_raw)[wib];
  WarpSmemMono &M = *reinterpret_cast<WarpSmemMono *>(&S);

  const int n = A.n;
  const int wbeg = (blockIdx.x * kWalkWarps + wib) * 32;
  if (wbeg >= n) return;                       // warp-uniform
  const int wend = min(n, wbeg + 32);
  const int gi = wbeg + lane;
  const bool valid = gi < n;
  const int nn = *A.nnodes;

  float xh = 0, yh = 0, zh = 0, xl = 0, yl = 0, zl = 0;
  if (valid) {
    float4 h = A.bhi[gi], l = A.blo[gi];
    xh = h.x; yh = h.y; zh = h.z; xl = l.x; yl = l.y; zl = l.z;
  }
  // warp bounding box of the bodies (hi parts), and its magnitude
  float bminx = valid ? xh : INFINITY, bminy = valid ? yh : INFINITY, bminz = valid ? zh : INFINITY;
  float bmaxx = valid ? xh : -INFINITY, bmaxy = valid ? yh : -INFINITY, bmaxz = valid ? zh : -INFINITY;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bminx = fminf(bminx, __shfl_xor_sync(0xffffffffu, bminx, o));
    bminy = fminf(bminy, __shfl_xor_sync(0xffffffffu, bminy, o));
    bminz = fminf(bminz, __shfl_xor_sync(0xffffffffu, bminz, o));
    bmaxx = fmaxf(bmaxx, __shfl_xor_sync(0xffffffffu, bmaxx, o));
    bmaxy = fmaxf(bmaxy, __shfl_xor_sync(0xffffffffu, bmaxy, o));
    bmaxz = fmaxf(bmaxz, __shfl_xor_sync(0xffffffffu, bmaxz, o));
  }
  const float bR = fmaxf(fmaxf(fmaxf(fabsf(bminx), fabsf(bmaxx)), fmaxf(fabsf(bminy), fabsf(bmaxy))),
                         fmaxf(fabsf(bminz), fabsf(bmaxz)));
  const double side = A.geom[3];
  const float theta2f = A.theta2f;
  const float eps2 = A.eps2;

  Accum<ACC64> acc;
  int c_m2p = 0, c_p2p = 0, c_tests = 0;
  unsigned long long w_batches = 0, w_items = 0, w_mixed = 0, w_fp64 = 0, w_mono = 0, w_quad = 0;
  int w_maxsp = 0;
  int nmono = 0, nquad = 0;
  int sp = 0;
  bool abort = false;
  if (lane == 0) {
    M.st_a[0] = 0u;                            // root node, count 1, kind node
    M.st_m[0] = __ballot_sync(0xffffffffu, valid);
  } else {
    __ballot_sync(0xffffffffu, valid);
  }
  sp = 1;
  __syncwarp();

  for (int iter = 0; sp > 0; ++iter) {
    if (iter > A.max_iter) {                    // cannot happen on a well-formed tree
      if (lane == 0) latch_error(A.status, kErrTree);
      abort = true;
      break;
    }
    // ---- pop up to 32 items from the top entries (lane 0 = top of stack)
    const int ke = sp - 1 - lane;
    uint32_t ea = 0, em = 0;
    int ecnt = 0;
    if (ke >= 0) {
      ea = M.st_a[ke];
      em = M.st_m[ke];
      ecnt = (int)((ea >> kCntShift) & 63u) + 1;
    }
    const int incl = warp_incl_scan_i(ecnt, lane);
    const int excl = incl - ecnt;
    const int take = max(0, min(ecnt, 32 - excl));
    const unsigned full = __ballot_sync(0xffffffffu, ecnt > 0 && take == ecnt);
    const int nfull = __popc(full);
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int nitems = min(total, 32);
    __syncwarp();
    if (take > 0 && take < ecnt) {             // the one partially consumed entry stays
      M.st_a[ke] = (((ea & kFirstMask) + take) & kFirstMask) |
                   ((uint32_t)(ecnt - take - 1) << kCntShift) | (ea & kKindBody);
    }
    sp -= nfull;
    const unsigned starts = __reduce_or_sync(0xffffffffu, take > 0 ? (1u << excl) : 0u);
    const int stpos = 31 - __clz(starts & (0xffffffffu >> (31 - lane)));
    const int owner = __popc(starts & ((1u << stpos) - 1u));
    const uint32_t oa = __shfl_sync(0xffffffffu, ea, owner);
    const uint32_t omask = __shfl_sync(0xffffffffu, em, owner);
    const bool have = lane < nitems;
    if (COUNT) { ++w_batches; w_items += nitems; }
    const bool kbody = (oa & kKindBody) != 0;
    const int item = (int)(oa & kFirstMask) + (lane - stpos);

    // ---- load and classify (lane = item)
    float4 r0 = make_float4(0, 0, 0, 0), r1 = make_float4(0, 0, 0, 0);
    int4 tp = make_int4(-1, 0, 0, 0);
    bool single = false;                       // a point term (body or one-body leaf)
    bool bad = false;
    if (have) {
      if (kbody) {
        bad = item >= n;
        if (!bad) { r0 = A.bhi[item]; r1 = A.blo[item]; }
        tp = make_int4(-1, 0, item, item + 1);
        single = true;
      } else {
        bad = item >= nn;
        if (!bad) {
          tp = A.topo[item];
          r0 = A.rec0[item];
          r1 = A.rec1[item];
          single = r1.w < 0.f;                 // one-body leaf: record holds the body itself
          bad = (tp.x >= 0 && (tp.x <= 0 || tp.x + tp.y > nn)) || tp.z < 0 || tp.w > n ||
                tp.z >= tp.w;
        }
      }
    }
    if (__any_sync(0xffffffffu, bad)) {
      if (lane == 0) latch_error(A.status, kErrTree);
      abort = true;
      break;
    }
    unsigned accm = 0, openm = 0;
    bool mixed = false;
    if (have) {
      if (single) {
        accm = omask;
      } else {
        const float cx = r0.x, cy = r0.y, cz = r0.z, l2 = r1.w;
        const float C = fmaxf(fabsf(cx), fmaxf(fabsf(cy), fabsf(cz)));
        const float del = (bR + C) * 1.9073486e-6f;      // 2^-19 (R + C): bound on hi/lo + rounding
        float gx = fmaxf(fmaxf(bminx - cx, cx - bmaxx), 0.f);
        float gy = fmaxf(fmaxf(bminy - cy, cy - bmaxy), 0.f);
        float gz = fmaxf(fmaxf(bminz - cz, cz - bmaxz), 0.f);
        gx = fmaxf(gx - del, 0.f); gy = fmaxf(gy - del, 0.f); gz = fmaxf(gz - del, 0.f);
        float fx = fmaxf(fabsf(cx - bminx), fabsf(cx - bmaxx)) + del;
        float fy = fmaxf(fabsf(cy - bminy), fabsf(cy - bmaxy)) + del;
        float fz = fmaxf(fabsf(cz - bminz), fabsf(cz - bmaxz)) + del;
        float dmin2 = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
        float dmax2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
        bool guard_any = A.mac_guard && tp.z < wend && tp.w > wbeg;
        if (!guard_any && l2 < theta2f * dmin2 * 0.999f) accm = omask;
        else if (l2 > theta2f * dmax2 * 1.001f) openm = omask;
        else mixed = true;
      }
    }
    if (COUNT) {                               // MAC tests per body (introspection only)
      for (int j = 0; j < nitems; ++j) {
        const bool sj = __shfl_sync(0xffffffffu, single, j);
        const unsigned mj = __shfl_sync(0xffffffffu, omask, j);
        const int bj = __shfl_sync(0xffffffffu, tp.z, j), ej = __shfl_sync(0xffffffffu, tp.w, j);
        if (!sj && ((mj >> lane) & 1u) && !(A.mac_guard && bj <= gi && gi < ej)) ++c_tests;
      }
    }
    // ---- exact per-lane test for mixed nodes
    unsigned mixed_bits = __ballot_sync(0xffffffffu, mixed);
    if (COUNT) w_mixed += __popc(mixed_bits);
    while (mixed_bits) {
      const int j = __ffs(mixed_bits) - 1;
      mixed_bits &= mixed_bits - 1;
      const float cx = __shfl_sync(0xffffffffu, r0.x, j);
      const float cy = __shfl_sync(0xffffffffu, r0.y, j);
      const float cz = __shfl_sync(0xffffffffu, r0.z, j);
      const float clx = __shfl_sync(0xffffffffu, r1.x, j);
      const float cly = __shfl_sync(0xffffffffu, r1.y, j);
      const float clz = __shfl_sync(0xffffffffu, r1.z, j);
      const float l2 = __shfl_sync(0xffffffffu, r1.w, j);
      const unsigned mk = __shfl_sync(0xffffffffu, omask, j);
      const int nb = __shfl_sync(0xffffffffu, tp.z, j);
      const int ne = __shfl_sync(0xffffffffu, tp.w, j);
      const int node = __shfl_sync(0xffffffffu, item, j);
      bool a_i = false, o_i = false;
      if ((mk >> lane) & 1u) {
        if (A.mac_guard && nb <= gi && gi < ne) {
          o_i = true;
        } else {
          float dx = (cx - xh) + (clx - xl);
          float dy = (cy - yh) + (cly - yl);
          float dz = (cz - zh) + (clz - zl);
          float D2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          float diff = l2 - theta2f * D2;
          if (fabsf(diff) <= 1.52587890625e-5f * l2) {     // 2^-16 band: decide in FP64
            const double X = A.ncom[3 * node], Y = A.ncom[3 * node + 1], Z = A.ncom[3 * node + 2];
            const double x = A.pos_s[3 * gi], y = A.pos_s[3 * gi + 1], z = A.pos_s[3 * gi + 2];
            const double ddx = __dsub_rn(X, x), ddy = __dsub_rn(Y, y), ddz = __dsub_rn(Z, z);
            const double D2d = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)),
                                         __dmul_rn(ddz, ddz));
            const double l = ldexp(side, -A.ndepth[node]);
            a_i = __dmul_rn(l, l) < __dmul_rn(A.theta2d, D2d);
            if (COUNT) atomicAdd(&A.stats[kStatFp64], 1ull);
          } else {
            a_i = diff < 0.f;
          }
          o_i = !a_i;
        }
      }
      const unsigned am = __ballot_sync(0xffffffffu, a_i);
      const unsigned om = __ballot_sync(0xffffffffu, o_i);
      if (lane == j) { accm = am; openm = om; }
    }

    // ---- append accepted terms to the lists
    const bool to_quad = (ORDER == 2) && accm != 0 && !single;
    const bool to_mono = accm != 0 && !to_quad;
    {
      const unsigned bm = __ballot_sync(0xffffffffu, to_mono);
      if (to_mono) {
        int p = nmono + __popc(bm & ((1u << lane) - 1u));
        M.la[p] = r0;
        M.lb[p] = make_float4(r1.x, r1.y, r1.z, __uint_as_float(accm));
        if (COUNT) M.ltag[p] = single ? tp.z : -1;
      }
      nmono += __popc(bm);
    }
    if constexpr (ORDER == 2) {
      const unsigned bq = __ballot_sync(0xffffffffu, to_quad);
      if (to_quad) {
        int p = nquad + __popc(bq & ((1u << lane) - 1u));
        WarpSmemQuad &QS = S;
        QS.qa[p] = r0;
        QS.qb[p] = make_float4(r1.x, r1.y, r1.z, __uint_as_float(accm));
        QS.qc[p] = A.quadf[2 * item];
        QS.qd[p] = A.quadf[2 * item + 1];
      }
      nquad += __popc(bq);
    }

    // ---- push opened nodes (children range) or bucket bodies (chunks of <= 32)
    int npush = 0;
    if (openm != 0) npush = (tp.x >= 0) ? 1 : (tp.w - tp.z + 31) / 32;
    const int pincl = warp_incl_scan_i(npush, lane);
    const int ptotal = __shfl_sync(0xffffffffu, pincl, 31);
    if (sp + ptotal > kStackCap) {
      if (lane == 0) latch_error(A.status, kErrStack);
      abort = true;
      break;
    }
    if (npush > 0) {
      int p = sp + pincl - npush;
      if (tp.x >= 0) {
        M.st_a[p] = (uint32_t)tp.x | ((uint32_t)(tp.y - 1) << kCntShift);
        M.st_m[p] = openm;
      } else {
        for (int b = tp.z; b < tp.w; b += 32, ++p) {
          int c = min(32, tp.w - b);
          M.st_a[p] = (uint32_t)b | ((uint32_t)(c - 1) << kCntShift) | kKindBody;
          M.st_m[p] = openm;
        }
      }
    }
    sp += ptotal;
    if (COUNT) w_maxsp = max(w_maxsp, sp);
    __syncwarp();

    // ---- evaluate full lists
    if (nmono >= kFlushAt) {
      if (COUNT) w_mono += nmono;
      float px, py, pz;
      flush_mono<COUNT>(M, nmono, lane, xh, yh, zh, xl, yl, zl, eps2, px, py, pz, gi, c_m2p, c_p2p);
      acc.add(px, py, pz);
      nmono = 0;
      __syncwarp();
    }
    if constexpr (ORDER == 2) {
      if (nquad >= kFlushAt) {
        if (COUNT) w_quad += nquad;
        float px, py, pz;
        flush_quad<COUNT>(S, nquad, lane, xh, yh, zh, xl, yl, zl,
                          eps2, px, py, pz, c_m2p);
        acc.add(px, py, pz);
        nquad = 0;
        __syncwarp();
      }
    }
  }
  if (COUNT) { w_mono += nmono; w_quad += nquad; }
  if (!abort) {
    if (nmono > 0) {
      float px, py, pz;
      flush_mono<COUNT>(M, nmono, lane, xh, yh, zh, xl, yl, zl, eps2, px, py, pz, gi, c_m2p, c_p2p);
      acc.add(px, py, pz);
    }
    if constexpr (ORDER == 2) {
      if (nquad > 0) {
        float px, py, pz;
        flush_quad<COUNT>(S, nquad, lane, xh, yh, zh, xl, yl, zl, eps2, px, py, pz, c_m2p);
        acc.add(px, py, pz);
      }
    }
  }
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
    }
  }
  if (!valid) return;
  double ax, ay, az;
  acc.get(ax, ay, az);
  ax *= A.G; ay *= A.G; az *= A.G;
  const int64_t ci = A.perm[gi];
  A.acc[3 * ci] = ax;
  A.acc[3 * ci + 1] = ay;
  A.acc[3 * ci + 2] = az;
  if (A.vel) {                                // fused closing kick of the leapfrog
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

template <int ORDER, bool ACC64, bool COUNT>
int launch_walk(Ctx *c, const WalkArgs &A) {
  using Smem = typename std::conditional<ORDER == 2, WarpSmemQuad, WarpSmemMono>::type;
  const size_t smem = sizeof(Smem) * kWalkWarps;
  auto kern = k_walk<ORDER, ACC64, COUNT>;
  static bool configured[64] = {false};
  int dev = c->device < 64 ? c->device : 63;
  if (!configured[dev]) {
    GRAV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured[dev] = true;
  }
  const int warps = (A.n + 31) / 32;
  const int blocks = (warps + kWalkWarps - 1) / kWalkWarps;
  kern<<<blocks, 32 * kWalkWarps, smem, c->stream>>>(A);
  ++c->launches;
  return cuda_status(cudaGetLastError());
}

}  // namespace

int walk_forces(Ctx *c, double theta, double eps, double *acc, int32_t *counts, double *vel,
                double kick) {
  Tree &t = c->t;
  WalkArgs A;
  A.bhi = t.body_hi; A.blo = t.body_lo; A.pos_s = t.pos_s;
  A.rec0 = t.nrec0; A.rec1 = t.nrec1; A.quadf = t.nquadf;
  A.topo = t.topo; A.ndepth = t.ndepth; A.ncom = t.ncom; A.geom = t.geom;
  A.perm = t.idx; A.nnodes = t.nnodes;
  A.n = (int)c->n;
  A.theta2d = theta * theta;
  A.theta2f = (float)(theta * theta);
  A.eps2 = (float)(eps * eps);
  A.G = c->params.G;
  A.mac_guard = c->params.mac_guard;
  A.acc = acc; A.counts = counts; A.vel = vel; A.kick = kick;
  A.status = c->d_status;
  A.max_iter = (int)(8 * c->n + 64);
  A.stats = c->walk_stats;
  if (counts) {
    GRAV_CUDA_TRY(cudaMemsetAsync(c->walk_stats, 0, sizeof(unsigned long long) * 8, c->stream));
  }
  const bool q = c->params.order == 2;
  const bool d64 = c->params.accum == 1;
  if (counts) {
    if (q) return d64 ? launch_walk<2, true, true>(c, A) : launch_walk<2, false, true>(c, A);
    return d64 ? launch_walk<0, true, true>(c, A) : launch_walk<0, false, true>(c, A);
  }
  if (q) return d64 ? launch_walk<2, true, false>(c, A) : launch_walk<2, false, false>(c, A);
  return d64 ? launch_walk<0, true, false>(c, A) : launch_walk<0, false, false>(c, A);
}

}  // namespace grav
