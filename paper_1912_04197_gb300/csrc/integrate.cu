// Symplectic steppers (Sec. 2.3: semi-implicit Euler and leapfrog) in FP64.
// Kick-drift: v += h a; x += dt v (one fused pass); the closing kick of the
// leapfrog is fused into the walk's output (see walk.cu).
#include "internal.cuh"

namespace grav {
namespace {

__global__ void k_kick_drift(int64_t n3, double *__restrict__ pos, double *__restrict__ vel,
                             const double *__restrict__ acc, double h, double dt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double v = __dadd_rn(vel[i], __dmul_rn(h, acc[i]));   // same roundings as written, no FMA
  vel[i] = v;
  pos[i] = __dadd_rn(pos[i], __dmul_rn(dt, v));
}

__global__ void k_kick(int64_t n3, double *__restrict__ vel, const double *__restrict__ acc,
                       double h) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n3) return;
  vel[i] = __dadd_rn(vel[i], __dmul_rn(h, acc[i]));
}

// Reverse of one time level of the leapfrog: xbar += c g (g = J(x)^T vbar from the
// vector-Jacobian product), then, unless this is the trajectory's first level, the
// reverse of the drift before it: vbar += dt xbar.
__global__ void k_adjoint_kick_drift(int64_t n3, double *__restrict__ xbar,
                                     double *__restrict__ vbar, const double *__restrict__ g,
                                     double c, double dt, int drift) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const double xb = __dadd_rn(xbar[i], __dmul_rn(c, g[i]));
  xbar[i] = xb;
  if (drift) vbar[i] = __dadd_rn(vbar[i], __dmul_rn(dt, xb));
}

}  // namespace

int launch_adjoint_kick_drift(Ctx *c, int64_t n, double *xbar, double *vbar, const double *g,
                              double coef, double dt, bool drift) {
  int64_t n3 = 3 * n;
  k_adjoint_kick_drift<<<(unsigned)((n3 + 255) / 256), 256, 0, c->stream>>>(n3, xbar, vbar, g,
                                                                           coef, dt, drift ? 1 : 0);
  ++c->launches;
  return cuda_status(cudaGetLastError());
}

// dst rows perm[first + i] = src rows i (sorted order back to the caller's order).
__global__ void k_scatter_sorted(int64_t first, int64_t nb, int64_t n,
                                 const uint32_t *__restrict__ perm, const double *__restrict__ src,
                                 double *__restrict__ dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nb) return;
  const int64_t j = perm[first + i];
  if (j >= n) return;                         // only after a failed sort (status latched)
  dst[3 * j] = src[3 * i];
  dst[3 * j + 1] = src[3 * i + 1];
  dst[3 * j + 2] = src[3 * i + 2];
}

int launch_kick_drift(Ctx *c, int64_t n, double *pos, double *vel, const double *acc,
                      double h_kick, double dt) {
  int64_t n3 = 3 * n;
  k_kick_drift<<<(unsigned)((n3 + 255) / 256), 256, 0, c->stream>>>(n3, pos, vel, acc, h_kick, dt);
  ++c->launches;
  return cuda_status(cudaGetLastError());
}

int launch_kick(Ctx *c, int64_t n, double *vel, const double *acc, double h_kick) {
  int64_t n3 = 3 * n;
  k_kick<<<(unsigned)((n3 + 255) / 256), 256, 0, c->stream>>>(n3, vel, acc, h_kick);
  ++c->launches;
  return cuda_status(cudaGetLastError());
}

int launch_scatter_sorted(Ctx *c, int64_t first_body, int64_t nbodies, const double *src,
                          double *dst) {
  if (nbodies <= 0) return GRAVITY_OK;
  k_scatter_sorted<<<(unsigned)((nbodies + 255) / 256), 256, 0, c->stream>>>(
      first_body, nbodies, c->n, c->t.idx, src, dst);
  ++c->launches;
  return cuda_status(cudaGetLastError());
}

}  // namespace grav
