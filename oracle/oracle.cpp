// Oracle for the Barnes-Hut octree gravity path.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 CPU statement of
// what the GPU path computes.  It shares no code, header, table or helper with
// the CUDA library; only tests, the smoke check and the benchmark's CPU-baseline
// leg may load it.  Build flags: -O2 -ffp-contract=off (no fused multiply-add,
// so every product and sum is one IEEE-754 rounding, in the order written here).
//
// Paper: Ferrari, Lavagna, Blazquez, "A parallel-GPU code for asteroid
// aggregation problems with angular particles" (MNRAS 2019, arXiv:1912.04197).
//   Eq. (Newton)         - direct N^2 gravity                      (Sec. 2.1)
//   Hierarchical treecode - octree split until 0 or 1 body/cell    (Sec. 2.1)
//   Eq. (COMinternal)    - node mass and centre of mass            (Sec. 2.1, Clustering)
//   Eq. (accuracy)       - opening test theta_BN vs theta          (Sec. 2.1, Force computation)
//   Eqs. (Force_leaf, Force_thetaTrue, Force_rComp) - force rules  (Sec. 2.1)
//   Five-kernel list     - bbox, build, mass, sort, forces         (Sec. 2.1, CUDA implementation)
//   Sec. 2.3             - symplectic integrators (semi-implicit Euler, leapfrog)
//   Sec. 3.1             - conservation of energy and momenta
//
// Readings where the paper is silent (each is restated at its function):
//   * root cell = cube of side s = max per-axis extent, cornered at the per-axis
//     minimum; s := 1 when the extent is 0 or n <= 1;
//   * cells are addressed by 63-bit Morton keys (21 levels); a cell that holds
//     more than leaf_max bodies and has depth < 21 is split into its non-empty
//     octants; a chain of cells with a single non-empty child is replaced by its
//     deepest member; a leaf keeps its natural depth (parent depth + 1);
//   * "Radius of N" in Eq. (accuracy) is the cell side l = s * 2^-depth and the
//     distance is from the body to the node centre of mass; equality opens;
//   * every term (leaf, node) uses the softened r of Eq. (Force_rComp);
//   * a node whose cell contains the body is always opened (mac_guard = 1);
//   * a leaf holding a single body is always a body-to-body term (Eq. Force_leaf);
//     a leaf holding several bodies is tested like an internal node.

#include <omp.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <utility>
#include <vector>

namespace {

constexpr int kLevels = 21;                       // 3 * 21 = 63 key bits
constexpr uint32_t kGridMax = (1u << kLevels) - 1;

struct Node {
  int depth = 0;
  int64_t begin = 0, end = 0;                     // body range in sorted order
  int64_t parent = -1;
  bool leaf = false;
  std::vector<int64_t> children;                  // preorder indices, octant order
  double m = 0.0;
  double com[3] = {0.0, 0.0, 0.0};
  double q[6] = {0, 0, 0, 0, 0, 0};               // xx, yy, zz, xy, xz, yz (traceless)
};

struct Tree {
  int64_t n = 0;
  int leaf_max = 1;
  int order = 0;
  double lo[3] = {0, 0, 0};
  double side = 1.0;
  std::vector<uint64_t> keys;                     // sorted keys
  std::vector<int64_t> perm;                      // sorted index -> caller index
  std::vector<double> x;                          // sorted positions (n,3)
  std::vector<double> m;                          // sorted masses
  std::vector<Node> nodes;                        // DFS preorder, root = 0
};

// Octant digit of a key for the split of a cell at `depth` (children at depth+1).
inline unsigned digit_at(uint64_t key, int depth) {
  return (unsigned)((key >> (3 * (kLevels - 1 - depth))) & 7u);
}

// Top-down recursive construction (Sec. 2.1, "Hierarchical treecode algorithm"):
// a cell is split into its octants until it holds at most leaf_max bodies
// (paper: 0 or 1); depth is capped at 21 where identical keys form one bucket.
// A chain of cells with one non-empty octant is replaced by its deepest member.
int64_t build_rec(Tree &t, int depth, int64_t b, int64_t e, int64_t parent) {
  for (;;) {
    if (e - b <= t.leaf_max || depth == kLevels) {
      Node nd;
      nd.depth = depth; nd.begin = b; nd.end = e; nd.parent = parent; nd.leaf = true;
      t.nodes.push_back(nd);
      return (int64_t)t.nodes.size() - 1;
    }
    int nonempty = 0;
    unsigned first = digit_at(t.keys[b], depth), last = digit_at(t.keys[e - 1], depth);
    nonempty = (first == last) ? 1 : 2;
    if (nonempty == 1) { depth += 1; continue; }  // collapse the chain
    break;
  }
  Node nd;
  nd.depth = depth; nd.begin = b; nd.end = e; nd.parent = parent; nd.leaf = false;
  t.nodes.push_back(nd);
  int64_t me = (int64_t)t.nodes.size() - 1;
  // children: maximal runs of equal octant digit, in digit order 0..7
  int64_t s = b;
  while (s < e) {
    unsigned d = digit_at(t.keys[s], depth);
    int64_t r = s;
    while (r < e && digit_at(t.keys[r], depth) == d) ++r;
    int64_t c = build_rec(t, depth + 1, s, r, me);
    t.nodes[me].children.push_back(c);
    s = r;
  }
  return me;
}

// Eq. (COMinternal): node mass = sum of child masses, node centre of mass =
// (sum of child COM * child mass) / node mass, children in octant order.
// A leaf of several bodies sums them in sorted order; a one-body leaf is the body.
// The traceless quadrupole (not in the paper) is Q = sum m (3 y y^T - |y|^2 I)
// about the COM, shifted to the parent with the parallel-axis rule; a one-body
// leaf has Q = 0.
void moments_rec(Tree &t, int64_t k) {
  Node &nd = t.nodes[k];
  if (nd.leaf && nd.end - nd.begin == 1) {
    // a one-body leaf is the body itself (leaves are bodies, Sec. 2.1): its mass
    // and position, no sum and no division
    nd.m = t.m[nd.begin];
    for (int a = 0; a < 3; ++a) nd.com[a] = t.x[3 * nd.begin + a];
    for (double &v : nd.q) v = 0.0;
    return;
  }
  if (nd.leaf) {
    double msum = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t i = nd.begin; i < nd.end; ++i) {
      double mi = t.m[i];
      msum = msum + mi;
      sx = sx + mi * t.x[3 * i + 0];
      sy = sy + mi * t.x[3 * i + 1];
      sz = sz + mi * t.x[3 * i + 2];
    }
    nd.m = msum;
    nd.com[0] = sx / msum; nd.com[1] = sy / msum; nd.com[2] = sz / msum;
    for (double &v : nd.q) v = 0.0;
    if (t.order >= 2 && nd.end - nd.begin > 1) {
      for (int64_t i = nd.begin; i < nd.end; ++i) {
        double mi = t.m[i];
        double y0 = t.x[3 * i + 0] - nd.com[0];
        double y1 = t.x[3 * i + 1] - nd.com[1];
        double y2 = t.x[3 * i + 2] - nd.com[2];
        double r2 = (y0 * y0 + y1 * y1) + y2 * y2;
        nd.q[0] = nd.q[0] + mi * (3.0 * y0 * y0 - r2);
        nd.q[1] = nd.q[1] + mi * (3.0 * y1 * y1 - r2);
        nd.q[2] = nd.q[2] + mi * (3.0 * y2 * y2 - r2);
        nd.q[3] = nd.q[3] + mi * (3.0 * y0 * y1);
        nd.q[4] = nd.q[4] + mi * (3.0 * y0 * y2);
        nd.q[5] = nd.q[5] + mi * (3.0 * y1 * y2);
      }
    }
    return;
  }
  for (int64_t c : nd.children) moments_rec(t, c);
  double msum = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
  for (int64_t c : nd.children) {
    const Node &ch = t.nodes[c];
    msum = msum + ch.m;
    sx = sx + ch.com[0] * ch.m;
    sy = sy + ch.com[1] * ch.m;
    sz = sz + ch.com[2] * ch.m;
  }
  nd.m = msum;
  nd.com[0] = sx / msum; nd.com[1] = sy / msum; nd.com[2] = sz / msum;
  for (double &v : nd.q) v = 0.0;
  if (t.order >= 2) {
    for (int64_t c : nd.children) {
      const Node &ch = t.nodes[c];
      double d0 = ch.com[0] - nd.com[0];
      double d1 = ch.com[1] - nd.com[1];
      double d2 = ch.com[2] - nd.com[2];
      double r2 = (d0 * d0 + d1 * d1) + d2 * d2;
      nd.q[0] = nd.q[0] + (ch.q[0] + ch.m * (3.0 * d0 * d0 - r2));
      nd.q[1] = nd.q[1] + (ch.q[1] + ch.m * (3.0 * d1 * d1 - r2));
      nd.q[2] = nd.q[2] + (ch.q[2] + ch.m * (3.0 * d2 * d2 - r2));
      nd.q[3] = nd.q[3] + (ch.q[3] + ch.m * (3.0 * d0 * d1));
      nd.q[4] = nd.q[4] + (ch.q[4] + ch.m * (3.0 * d0 * d2));
      nd.q[5] = nd.q[5] + (ch.q[5] + ch.m * (3.0 * d1 * d2));
    }
  }
}

struct WalkOut {
  double a[3] = {0, 0, 0};
  double absum = 0.0;            // sum of |term| (the natural scale of the sum's rounding)
  int64_t tests = 0, m2p = 0, p2p = 0;
};

// Softened point-mass term (Eqs. Force_leaf, Force_thetaTrue, Force_rComp),
// per unit mass of the body: m d / r^3 with r^2 = |d|^2 + eps^2, d = source - body.
// A term with r^2 = 0 contributes nothing.
inline void point_term(WalkOut &o, double mj, const double *src, const double *xb, double eps2) {
  double d0 = src[0] - xb[0], d1 = src[1] - xb[1], d2 = src[2] - xb[2];
  double r2 = ((d0 * d0 + d1 * d1) + d2 * d2) + eps2;
  if (r2 == 0.0) return;
  double r = std::sqrt(r2);
  double inv3 = 1.0 / (r2 * r);
  double s = mj * inv3;
  o.a[0] = o.a[0] + s * d0;
  o.a[1] = o.a[1] + s * d1;
  o.a[2] = o.a[2] + s * d2;
  o.absum = o.absum + s * std::sqrt((d0 * d0 + d1 * d1) + d2 * d2);
}

// Softened quadrupole term (not in the paper): the negative gradient of
//   phi = -m / r_e - (y^T Q y) / (2 r_e^5),  y = body - COM,  r_e^2 = |y|^2 + eps^2,
// i.e. a = -m y / r_e^3 + Q y / r_e^5 - (5/2) (y^T Q y) y / r_e^7.
inline void quad_term(WalkOut &o, const Node &nd, const double *xb, double eps2) {
  double y0 = xb[0] - nd.com[0], y1 = xb[1] - nd.com[1], y2 = xb[2] - nd.com[2];
  double r2 = ((y0 * y0 + y1 * y1) + y2 * y2) + eps2;
  if (r2 == 0.0) return;
  double r = std::sqrt(r2);
  double inv = 1.0 / r;
  double inv2 = inv * inv;
  double inv3 = inv2 * inv;
  double inv5 = inv3 * inv2;
  double inv7 = inv5 * inv2;
  const double *q = nd.q;
  double qy0 = (q[0] * y0 + q[3] * y1) + q[4] * y2;
  double qy1 = (q[3] * y0 + q[1] * y1) + q[5] * y2;
  double qy2 = (q[4] * y0 + q[5] * y1) + q[2] * y2;
  double yqy = (y0 * qy0 + y1 * qy1) + y2 * qy2;
  double c = 2.5 * yqy * inv7;
  double t0 = (-nd.m * inv3 * y0 + qy0 * inv5) - c * y0;
  double t1 = (-nd.m * inv3 * y1 + qy1 * inv5) - c * y1;
  double t2 = (-nd.m * inv3 * y2 + qy2 * inv5) - c * y2;
  o.a[0] = o.a[0] + t0;
  o.a[1] = o.a[1] + t1;
  o.a[2] = o.a[2] + t2;
  o.absum = o.absum + std::sqrt((t0 * t0 + t1 * t1) + t2 * t2);
}

struct WalkCtx {
  const Tree *t;
  double theta2, eps2;
  int mac_guard;
  int64_t ib;                    // sorted index of the body
  const double *xb;
};

// Force computation (Sec. 2.1): traverse from the root; a single-body leaf is a
// body-to-body term; otherwise test l < theta * D (l = cell side, D = distance
// to the node COM); accept -> node term and stop; open -> all children (or, for a
// bucket leaf, its bodies).  The decisions are made here once; the visitor
// receives the accepted node terms (node(k)), body-to-body terms (body(j), j != B)
// and opening tests (test()).
template <class V>
void decide_rec(const WalkCtx &w, int64_t k, V &v) {
  const Tree &t = *w.t;
  const Node &nd = t.nodes[k];
  int64_t cnt = nd.end - nd.begin;
  if (nd.leaf && cnt == 1) {
    if (nd.begin != w.ib) v.body(nd.begin);
    return;
  }
  bool contains = (nd.begin <= w.ib && w.ib < nd.end);
  bool open = true;
  if (!(w.mac_guard && contains)) {
    double d0 = nd.com[0] - w.xb[0], d1 = nd.com[1] - w.xb[1], d2 = nd.com[2] - w.xb[2];
    double D2 = (d0 * d0 + d1 * d1) + d2 * d2;
    double l = std::ldexp(t.side, -nd.depth);
    v.test();
    if (l * l < w.theta2 * D2) open = false;
  }
  if (!open) {
    v.node(k);
    return;
  }
  if (nd.leaf) {
    for (int64_t j = nd.begin; j < nd.end; ++j)
      if (j != w.ib) v.body(j);
    return;
  }
  for (int64_t c : nd.children) decide_rec(w, c, v);
}

// Visitor: accelerations (Eqs. Force_leaf, Force_thetaTrue, Force_rComp).
struct ForceVisitor {
  const WalkCtx &w;
  WalkOut &o;
  void test() { o.tests++; }
  void node(int64_t k) {
    const Tree &t = *w.t;
    const Node &nd = t.nodes[k];
    o.m2p++;
    if (t.order >= 2) quad_term(o, nd, w.xb, w.eps2);
    else point_term(o, nd.m, nd.com, w.xb, w.eps2);
  }
  void body(int64_t j) {
    const Tree &t = *w.t;
    point_term(o, t.m[j], &t.x[3 * j], w.xb, w.eps2);
    o.p2p++;
  }
};

void walk_rec(const WalkCtx &w, int64_t k, WalkOut &o) {
  ForceVisitor v{w, o};
  decide_rec(w, k, v);
}

// Jacobian of the softened point term f(d) = d / (|d|^2 + eps^2)^{3/2} with respect
// to d: J = (I - 3 d d^T / r^2) / r^3, r^2 = |d|^2 + eps^2 (symmetric).  Returns
// J u for a vector u; zero when r^2 = 0.
inline void jac_times(const double *d, double eps2, const double *u, double *out) {
  double r2 = ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]) + eps2;
  if (r2 == 0.0) { out[0] = out[1] = out[2] = 0.0; return; }
  double r = std::sqrt(r2);
  double inv3 = 1.0 / (r2 * r);
  double du = (d[0] * u[0] + d[1] * u[1]) + d[2] * u[2];
  double c = 3.0 * du / r2;
  for (int a = 0; a < 3; ++a) out[a] = inv3 * (u[a] - c * d[a]);
}

// Visitor: vector-Jacobian product of the accelerations on the frozen tree
// (monopole terms).  For a term a_B += m_s f(s - x_B) with cotangent u = lambda_B:
// grad x_B -= m_s J u, and grad s += m_s J u, where s is a body or a node COM.
struct VjpVisitor {
  const WalkCtx &w;
  const double *lam;            // cotangent of body B's acceleration (times G)
  double *gb;                   // gradient of x_B
  double *ab;                   // sum of |m J u| over B's terms
  std::vector<double> &gnode;   // gradient of node COMs (this target's share)
  std::vector<double> &anode;   // sum of |m J u| per node
  std::vector<std::pair<int64_t, std::array<double, 4>>> &gbody;
  void test() {}
  double term(const double *src, double m, double *gs) {
    double d[3] = {src[0] - w.xb[0], src[1] - w.xb[1], src[2] - w.xb[2]};
    double ju[3];
    jac_times(d, w.eps2, lam, ju);
    for (int a = 0; a < 3; ++a) { gb[a] -= m * ju[a]; gs[a] += m * ju[a]; }
    double mag = m * std::sqrt((ju[0] * ju[0] + ju[1] * ju[1]) + ju[2] * ju[2]);
    *ab += mag;
    return mag;
  }
  void node(int64_t k) {
    const Node &nd = w.t->nodes[k];
    anode[k] += term(nd.com, nd.m, &gnode[3 * k]);
  }
  void body(int64_t j) {
    std::array<double, 4> gs{0, 0, 0, 0};
    gs[3] = term(&w.t->x[3 * j], w.t->m[j], gs.data());
    gbody.push_back({j, gs});
  }
};

// Visitor: accelerations with the decisions already taken but every source at new
// positions (node COMs recomputed from the new body positions): the force of the
// frozen tree, for finite-difference checks of the product above.
struct FrozenVisitor {
  const WalkCtx &w;
  const double *xnew;           // sorted new positions
  const std::vector<double> &cnew;   // new node COMs
  const double *xb_new;
  WalkOut &o;
  void test() {}
  void node(int64_t k) { point_term(o, w.t->nodes[k].m, &cnew[3 * k], xb_new, w.eps2); }
  void body(int64_t j) { point_term(o, w.t->m[j], &xnew[3 * j], xb_new, w.eps2); }
};

}  // namespace

extern "C" {

enum { ORC_OK = 0, ORC_E_ARG = -1, ORC_E_NONFINITE = -2 };

// Kernel 1 of the five-kernel list (Sec. 2.1): bounding box of all bodies = root.
// Reading: a cube of side s = max_a (max_a - min_a) at the per-axis minimum;
// s = 1 when that extent is 0 or n <= 1.  Any non-finite coordinate is an error.
int orc_root_cube(int64_t n, const double *pos, double *lo, double *side) {
  lo[0] = lo[1] = lo[2] = 0.0;
  *side = 1.0;
  if (n <= 0) return ORC_OK;
  double hi[3];
  for (int a = 0; a < 3; ++a) { lo[a] = pos[a]; hi[a] = pos[a]; }
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      double v = pos[3 * i + a];
      if (!std::isfinite(v)) return ORC_E_NONFINITE;
      if (v < lo[a]) lo[a] = v;
      if (v > hi[a]) hi[a] = v;
    }
  double s = 0.0;
  for (int a = 0; a < 3; ++a) {
    double e = hi[a] - lo[a];
    if (e > s) s = e;
  }
  if (n <= 1 || s == 0.0) s = 1.0;
  *side = s;
  return ORC_OK;
}

// Morton key of each body (our reading of the octree addressing; the paper
// inserts bodies with floating-point cell tests).  Grid coordinate per axis:
// q = clamp(floor((x - lo) * (2^21 / s)), 0, 2^21 - 1), one IEEE subtraction and
// one IEEE multiplication, the scale being one IEEE division.  Key bit 3k+2 is
// bit k of q_x, bit 3k+1 of q_y, bit 3k of q_z (naive bit loop).
void orc_morton_keys(int64_t n, const double *pos, const double *lo, double side,
                     uint64_t *keys) {
  const double scale = 2097152.0 / side;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
      double u = pos[3 * i + a] - lo[a];
      double v = u * scale;
      double f = std::floor(v);
      if (!(f >= 0.0)) f = 0.0;
      if (f > (double)kGridMax) f = (double)kGridMax;
      q[a] = (uint32_t)f;
    }
    uint64_t key = 0;
    for (int k = 0; k < kLevels; ++k) {
      key |= (uint64_t)((q[0] >> k) & 1u) << (3 * k + 2);
      key |= (uint64_t)((q[1] >> k) & 1u) << (3 * k + 1);
      key |= (uint64_t)((q[2] >> k) & 1u) << (3 * k);
    }
    keys[i] = key;
  }
}

// Kernel 4 of the list (Sec. 2.1) "sort bodies by distance": read as spatial
// (Morton) order, stable, so equal keys keep ascending caller index.
void orc_sort(int64_t n, const uint64_t *keys, int64_t *perm) {
  std::vector<int64_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(),
                   [keys](int64_t a, int64_t b) { return keys[a] < keys[b]; });
  std::memcpy(perm, idx.data(), sizeof(int64_t) * n);
}

// Kernels 1-4 of the list: root cube, keys, sort, octree and moments.
// Returns nullptr (and *status < 0) on invalid input.
void *orc_tree_build(int64_t n, const double *pos, const double *mass, int leaf_max,
                     int order, int *status) {
  *status = ORC_OK;
  if (n < 0 || leaf_max < 1 || (order != 0 && order != 2)) { *status = ORC_E_ARG; return nullptr; }
  Tree *t = new Tree();
  t->n = n; t->leaf_max = leaf_max; t->order = order;
  int rc = orc_root_cube(n, pos, t->lo, &t->side);
  if (rc != ORC_OK) { delete t; *status = rc; return nullptr; }
  if (n == 0) return t;
  std::vector<uint64_t> keys(n);
  orc_morton_keys(n, pos, t->lo, t->side, keys.data());
  t->perm.resize(n);
  orc_sort(n, keys.data(), t->perm.data());
  t->keys.resize(n); t->x.resize(3 * n); t->m.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t j = t->perm[i];
    t->keys[i] = keys[j];
    for (int a = 0; a < 3; ++a) t->x[3 * i + a] = pos[3 * j + a];
    t->m[i] = mass[j];
  }
  build_rec(*t, 0, 0, n, -1);
  moments_rec(*t, 0);
  return t;
}

void orc_tree_free(void *h) { delete (Tree *)h; }

int64_t orc_tree_num_nodes(const void *h) { return (int64_t)((const Tree *)h)->nodes.size(); }

void orc_tree_geometry(const void *h, double *lo, double *side) {
  const Tree *t = (const Tree *)h;
  for (int a = 0; a < 3; ++a) lo[a] = t->lo[a];
  *side = t->side;
}

void orc_tree_export_order(const void *h, uint64_t *sorted_keys, int64_t *perm) {
  const Tree *t = (const Tree *)h;
  for (int64_t i = 0; i < t->n; ++i) { sorted_keys[i] = t->keys[i]; perm[i] = t->perm[i]; }
}

// Canonical serialisation, DFS preorder: depth, body range, child count, parent,
// key prefix (the first 3*depth key bits), leaf flag.
void orc_tree_export_nodes(const void *h, int32_t *depth, int64_t *begin, int64_t *end,
                           int32_t *n_child, int64_t *parent, uint64_t *prefix,
                           int32_t *leaf) {
  const Tree *t = (const Tree *)h;
  for (size_t k = 0; k < t->nodes.size(); ++k) {
    const Node &nd = t->nodes[k];
    depth[k] = nd.depth; begin[k] = nd.begin; end[k] = nd.end;
    n_child[k] = (int32_t)nd.children.size();
    parent[k] = nd.parent;
    prefix[k] = nd.depth == 0 ? 0 : (t->keys[nd.begin] >> (3 * (kLevels - nd.depth)));
    leaf[k] = nd.leaf ? 1 : 0;
  }
}

void orc_tree_export_moments(const void *h, double *mass, double *com, double *quad) {
  const Tree *t = (const Tree *)h;
  for (size_t k = 0; k < t->nodes.size(); ++k) {
    const Node &nd = t->nodes[k];
    mass[k] = nd.m;
    for (int a = 0; a < 3; ++a) com[3 * k + a] = nd.com[a];
    for (int a = 0; a < 6; ++a) quad[6 * k + a] = nd.q[a];
  }
}

// Kernel 5 of the list (Sec. 2.1): accelerations (force / body mass) of the
// target bodies (caller indices; all bodies if targets == nullptr), G applied
// once to each sum.  counts[3*i] = MAC tests, [3*i+1] = node terms accepted,
// [3*i+2] = body-body terms; absum[i] = sum over terms of |term| (times G).
void orc_tree_forces(const void *h, double theta, double eps, double G, int mac_guard,
                     int64_t ntarg, const int64_t *targets, double *acc, double *absum,
                     int64_t *counts) {
  const Tree *t = (const Tree *)h;
  std::vector<int64_t> inv(t->n);
  for (int64_t i = 0; i < t->n; ++i) inv[t->perm[i]] = i;
  const double theta2 = theta * theta, eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < ntarg; ++k) {
    int64_t ci = targets ? targets[k] : k;
    WalkCtx w{t, theta2, eps2, mac_guard, inv[ci], &t->x[3 * inv[ci]]};
    WalkOut o;
    if (t->n > 0) walk_rec(w, 0, o);
    for (int a = 0; a < 3; ++a) acc[3 * k + a] = G * o.a[a];
    if (absum) absum[k] = G * o.absum;
    if (counts) { counts[3 * k] = o.tests; counts[3 * k + 1] = o.m2p; counts[3 * k + 2] = o.p2p; }
  }
}

// Vector-Jacobian product of the tree accelerations (monopole, order 0) with the
// interaction decisions frozen: grad = (d acc / d pos)^T lambda, both (n,3) in caller
// order, G applied.  A node COM is sum m_j x_j / M over its bodies, so its gradient
// reaches each member j as (m_j / M) times the node's share.  absum (optional, n)
// receives for each body the sum of |m J u| over the terms it takes part in (as target,
// as source body, and its m_j / M share of each node's), the scale of the rounding.
int orc_tree_vjp(const void *h, double theta, double eps, double G, int mac_guard,
                 const double *lambda, double *grad, double *absum) {
  const Tree *t = (const Tree *)h;
  if (t->order != 0) return ORC_E_ARG;
  const int64_t n = t->n;
  const double theta2 = theta * theta, eps2 = eps * eps;
  std::vector<double> gs(3 * n, 0.0), as(n, 0.0);      // sorted order
  std::vector<double> gnode(3 * t->nodes.size(), 0.0), anode(t->nodes.size(), 0.0);
  for (int64_t ib = 0; ib < n; ++ib) {
    int64_t ci = t->perm[ib];
    double lam[3] = {G * lambda[3 * ci], G * lambda[3 * ci + 1], G * lambda[3 * ci + 2]};
    WalkCtx w{t, theta2, eps2, mac_guard, ib, &t->x[3 * ib]};
    std::vector<std::pair<int64_t, std::array<double, 4>>> gbody;
    VjpVisitor v{w, lam, &gs[3 * ib], &as[ib], gnode, anode, gbody};
    decide_rec(w, 0, v);
    for (auto &p : gbody) {
      for (int a = 0; a < 3; ++a) gs[3 * p.first + a] += p.second[a];
      as[p.first] += p.second[3];
    }
  }
  for (size_t k = 0; k < t->nodes.size(); ++k) {
    const Node &nd = t->nodes[k];
    for (int64_t j = nd.begin; j < nd.end; ++j) {
      for (int a = 0; a < 3; ++a) gs[3 * j + a] += (t->m[j] / nd.m) * gnode[3 * k + a];
      as[j] += (t->m[j] / nd.m) * anode[k];
    }
  }
  for (int64_t ib = 0; ib < n; ++ib) {
    for (int a = 0; a < 3; ++a) grad[3 * t->perm[ib] + a] = gs[3 * ib + a];
    if (absum) absum[t->perm[ib]] = as[ib];
  }
  return ORC_OK;
}

// Accelerations of the frozen tree at new positions pos_new (caller order), the
// decisions being those taken at the tree's own positions (monopole terms).
int orc_tree_forces_frozen(const void *h, double theta, double eps, double G, int mac_guard,
                           const double *pos_new, double *acc) {
  const Tree *t = (const Tree *)h;
  if (t->order != 0) return ORC_E_ARG;
  const int64_t n = t->n;
  std::vector<double> xs(3 * n);
  for (int64_t i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) xs[3 * i + a] = pos_new[3 * t->perm[i] + a];
  std::vector<double> cnew(3 * t->nodes.size());
  for (size_t k = 0; k < t->nodes.size(); ++k) {
    const Node &nd = t->nodes[k];
    double s[3] = {0, 0, 0};
    for (int64_t j = nd.begin; j < nd.end; ++j)
      for (int a = 0; a < 3; ++a) s[a] = s[a] + t->m[j] * xs[3 * j + a];
    for (int a = 0; a < 3; ++a) cnew[3 * k + a] = s[a] / nd.m;
  }
  const double theta2 = theta * theta, eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t ib = 0; ib < n; ++ib) {
    WalkCtx w{t, theta2, eps2, mac_guard, ib, &t->x[3 * ib]};
    WalkOut o;
    FrozenVisitor v{w, xs.data(), cnew, &xs[3 * ib], o};
    decide_rec(w, 0, v);
    for (int a = 0; a < 3; ++a) acc[3 * t->perm[ib] + a] = G * o.a[a];
  }
  return ORC_OK;
}

// Eq. (Newton), per unit mass of body i, with the softened r of Eq. (Force_rComp):
// a_i = G sum_{j != i} m_j (R_j - R_i) / (|R_j - R_i|^2 + eps^2)^{3/2}, in index order.
void orc_direct(int64_t n, const double *pos, const double *mass, double eps, double G,
                int64_t ntarg, const int64_t *targets, double *acc, double *absum) {
  const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < ntarg; ++k) {
    int64_t i = targets ? targets[k] : k;
    WalkOut o;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      point_term(o, mass[j], &pos[3 * j], &pos[3 * i], eps2);
    }
    for (int a = 0; a < 3; ++a) acc[3 * k + a] = G * o.a[a];
    if (absum) absum[k] = G * o.absum;
  }
}

// Accelerations of all bodies with the tree (use_tree = 1) or the direct sum.
static int forces_all(int64_t n, const double *pos, const double *mass, int use_tree,
                      double theta, double eps, double G, int leaf_max, int order,
                      int mac_guard, double *acc) {
  if (!use_tree) { orc_direct(n, pos, mass, eps, G, n, nullptr, acc, nullptr); return ORC_OK; }
  int st = 0;
  void *h = orc_tree_build(n, pos, mass, leaf_max, order, &st);
  if (!h) return st;
  orc_tree_forces(h, theta, eps, G, mac_guard, n, nullptr, acc, nullptr, nullptr);
  orc_tree_free(h);
  return ORC_OK;
}

// Symplectic steppers (Sec. 2.3).  scheme 0 = kick-drift-kick leapfrog:
//   v += dt/2 a(x); x += dt v; a = a(x) (tree rebuilt every step); v += dt/2 a.
// scheme 1 = semi-implicit Euler: v += dt a(x); x += dt v; a = a(x).
// acc holds a(x) on entry and on exit.
// Two time steps (Sec. 4.1): the stepper advances by the contact step dt, gravity is
// evaluated only every grav_every-th step (about Delta t_g / Delta t_c, Eq. dt_g bounds
// Delta t_g) and the last evaluated acceleration is used in between; grav_every <= 1
// evaluates it every step.  The count starts at the call.
int orc_leapfrog(int64_t n, double *pos, double *vel, const double *mass, double *acc,
                 double dt, int nsteps, int scheme, int use_tree, double theta, double eps,
                 double G, int leaf_max, int order, int mac_guard, int grav_every) {
  const int every = grav_every > 1 ? grav_every : 1;
  int since = 0;                        // steps since gravity was last evaluated
  for (int s = 0; s < nsteps; ++s) {
    const double h = scheme == 0 ? 0.5 * dt : dt;
    for (int64_t i = 0; i < 3 * n; ++i) vel[i] = vel[i] + h * acc[i];
    for (int64_t i = 0; i < 3 * n; ++i) pos[i] = pos[i] + dt * vel[i];
    since = since + 1;
    if (since == every) {
      int rc = forces_all(n, pos, mass, use_tree, theta, eps, G, leaf_max, order, mac_guard, acc);
      if (rc != ORC_OK) return rc;
      since = 0;
    }
    if (scheme == 0)
      for (int64_t i = 0; i < 3 * n; ++i) vel[i] = vel[i] + h * acc[i];
  }
  return ORC_OK;
}

// Conserved quantities (Sec. 3.1): out = {E, Px, Py, Pz, Lx, Ly, Lz} with
// E = sum m v^2 / 2 - sum_{i<j} G m_i m_j / sqrt(r_ij^2 + eps^2) (the Plummer
// potential whose gradient is the softened force), P = sum m v, L = sum m x cross v.
void orc_diagnostics(int64_t n, const double *pos, const double *vel, const double *mass,
                     double eps, double G, double *out) {
  const double eps2 = eps * eps;
  std::vector<double> pot(n, 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = i + 1; j < n; ++j) {
      double d0 = pos[3 * j] - pos[3 * i], d1 = pos[3 * j + 1] - pos[3 * i + 1],
             d2 = pos[3 * j + 2] - pos[3 * i + 2];
      double r2 = ((d0 * d0 + d1 * d1) + d2 * d2) + eps2;
      if (r2 > 0.0) s = s + mass[j] / std::sqrt(r2);
    }
    pot[i] = mass[i] * s;
  }
  double ekin = 0.0, epot = 0.0, P[3] = {0, 0, 0}, L[3] = {0, 0, 0};
  for (int64_t i = 0; i < n; ++i) {
    const double *x = &pos[3 * i], *v = &vel[3 * i];
    double mi = mass[i];
    ekin = ekin + 0.5 * mi * ((v[0] * v[0] + v[1] * v[1]) + v[2] * v[2]);
    epot = epot + pot[i];
    for (int a = 0; a < 3; ++a) P[a] = P[a] + mi * v[a];
    L[0] = L[0] + mi * (x[1] * v[2] - x[2] * v[1]);
    L[1] = L[1] + mi * (x[2] * v[0] - x[0] * v[2]);
    L[2] = L[2] + mi * (x[0] * v[1] - x[1] * v[0]);
  }
  out[0] = ekin - G * epot;
  for (int a = 0; a < 3; ++a) { out[1 + a] = P[a]; out[4 + a] = L[a]; }
}

// Aggregate identification (Sec. 2, "Post-processing: aggregate identification"):
// bodies are the vertices of a graph, contacts its edges, aggregates its connected
// components of more than one body, found by depth-first search.  Our reading of
// "contact" (the paper takes it from its collision solver): bodies i != j touch when
// |x_i - x_j|^2 <= t_ij^2 with t_ij = r_i + r_j (radii given) or t_ij = dmax, and
// |d|^2 = (d0*d0 + d1*d1) + d2*d2, d = x_j - x_i.  The edges are every such pair
// (brute force); the search starts from each unvisited body in index order, so a
// component's first body is its smallest index, which is the label.
// counts[0] = components, counts[1] = components of more than one body.
void orc_components(int64_t n, const double *pos, const double *radius, double dmax,
                    int32_t *label, int64_t *counts) {
  std::vector<std::vector<int64_t>> adj(n);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = i + 1; j < n; ++j) {
      double d0 = pos[3 * j] - pos[3 * i], d1 = pos[3 * j + 1] - pos[3 * i + 1],
             d2 = pos[3 * j + 2] - pos[3 * i + 2];
      double r2 = (d0 * d0 + d1 * d1) + d2 * d2;
      double t = radius ? radius[i] + radius[j] : dmax;
      if (r2 <= t * t) {
        adj[i].push_back(j);
        adj[j].push_back(i);
      }
    }
  }
  std::vector<char> seen(n, 0);
  std::vector<int64_t> stack;
  counts[0] = counts[1] = 0;
  for (int64_t s = 0; s < n; ++s) {
    if (seen[s]) continue;
    int64_t size = 0;
    seen[s] = 1;
    stack.push_back(s);
    while (!stack.empty()) {
      int64_t v = stack.back();
      stack.pop_back();
      label[v] = (int32_t)s;
      ++size;
      for (int64_t w : adj[v])
        if (!seen[w]) { seen[w] = 1; stack.push_back(w); }
    }
    ++counts[0];
    if (size > 1) ++counts[1];
  }
}

// Number of host threads the OpenMP loops use (timing at one core and at all cores);
// n <= 0 restores the default.  No arithmetic depends on it.
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }

}  // extern "C"
