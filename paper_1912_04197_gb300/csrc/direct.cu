// Direct N^2 gravity, Eq. (Newton) (Sec. 2.1), with the softened distance of
// Eq. (Force_rComp): a_i = G sum_{j != i} m_j d_ij / (|d_ij|^2 + eps^2)^{3/2}.
// FP32 pair terms on hi/lo split coordinates (d = (x_j,hi - x_i,hi) + (x_j,lo - x_i,lo)),
// source tiles staged in shared memory, each tile's partial sum added to a
// (hi, lo) two-sum accumulator.  The self term has d = 0 and adds zero.
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

__global__ void __launch_bounds__(kDirThreads)
k_direct(const float4 *__restrict__ hi, const float4 *__restrict__ lo, int64_t n, float eps2,
         double G, double *__restrict__ acc) {
  __shared__ float4 sh[kDirThreads], sl[kDirThreads];
  constexpr int P = kDirPerThread;
  float xh[P], yh[P], zh[P], xl[P], yl[P], zl[P];
  float ahx[P], ahy[P], ahz[P], alx[P], aly[P], alz[P];
  int64_t i0 = (blockIdx.x * (int64_t)kDirThreads) * P + threadIdx.x;
#pragma unroll
  for (int p = 0; p < P; ++p) {
    int64_t i = i0 + p * kDirThreads;
    float4 h = i < n ? hi[i] : make_float4(0, 0, 0, 0);
    float4 l = i < n ? lo[i] : make_float4(0, 0, 0, 0);
    xh[p] = h.x; yh[p] = h.y; zh[p] = h.z; xl[p] = l.x; yl[p] = l.y; zl[p] = l.z;
    ahx[p] = ahy[p] = ahz[p] = alx[p] = aly[p] = alz[p] = 0.f;
  }
  for (int64_t t0 = 0; t0 < n; t0 += kDirThreads) {
    int64_t j = t0 + threadIdx.x;
    sh[threadIdx.x] = j < n ? hi[j] : make_float4(0, 0, 0, 0);
    sl[threadIdx.x] = j < n ? lo[j] : make_float4(0, 0, 0, 0);
    __syncthreads();
    float px[P], py[P], pz[P];
#pragma unroll
    for (int p = 0; p < P; ++p) px[p] = py[p] = pz[p] = 0.f;
#pragma unroll 8
    for (int k = 0; k < kDirThreads; ++k) {
      const float4 a = sh[k], b = sl[k];
#pragma unroll
      for (int p = 0; p < P; ++p) {
        float dx = (a.x - xh[p]) + (b.x - xl[p]);
        float dy = (a.y - yh[p]) + (b.y - yl[p]);
        float dz = (a.z - zh[p]) + (b.z - zl[p]);
        float r2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, eps2)));
        float inv = rsqrtf(r2);
        inv = r2 > 0.f ? inv : 0.f;
        float s = a.w * (inv * inv * inv);
        px[p] = fmaf(s, dx, px[p]);
        py[p] = fmaf(s, dy, py[p]);
        pz[p] = fmaf(s, dz, pz[p]);
      }
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
      two_sum_add(ahx[p], alx[p], px[p]);
      two_sum_add(ahy[p], aly[p], py[p]);
      two_sum_add(ahz[p], alz[p], pz[p]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < P; ++p) {
    int64_t i = i0 + p * kDirThreads;
    if (i < n) {
      acc[3 * i] = G * ((double)ahx[p] + (double)alx[p]);
      acc[3 * i + 1] = G * ((double)ahy[p] + (double)aly[p]);
      acc[3 * i + 2] = G * ((double)ahz[p] + (double)alz[p]);
    }
  }
}

}  // namespace

int direct_forces(Ctx *c, int64_t n, const double *pos, const double *mass, double eps, double G,
                  double *acc) {
  if (n > c->dir_cap) {
    if (c->dir_hi) cudaFree(c->dir_hi);
    if (c->dir_lo) cudaFree(c->dir_lo);
    c->dir_hi = c->dir_lo = nullptr;
    c->dir_cap = 0;
    GRAV_CUDA_TRY(cudaMalloc(&c->dir_hi, sizeof(float4) * n));
    GRAV_CUDA_TRY(cudaMalloc(&c->dir_lo, sizeof(float4) * n));
    c->dir_cap = n;
  }
  k_split<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(pos, mass, n, c->dir_hi, c->dir_lo);
  ++c->launches;
  const int64_t per_block = (int64_t)kDirThreads * kDirPerThread;
  k_direct<<<(unsigned)((n + per_block - 1) / per_block), kDirThreads, 0, c->stream>>>(
      c->dir_hi, c->dir_lo, n, (float)(eps * eps), G, acc);
  ++c->launches;
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

std::mutex g_noalloc_mu;
float4 *g_noalloc_ptr[kNoAllocMaxDevices] = {};

}  // namespace
}  // namespace grav

extern "C" int gravity_direct_noalloc(int64_t n, const double *pos, const double *mass,
                                      double eps, double G, double *acc, void *cuda_stream) {
  using namespace grav;
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
  k_direct<<<(unsigned)((n + per_block - 1) / per_block), kDirThreads, 0, s>>>(
      hi, lo, n, (float)(eps * eps), G, acc);
  return cuda_status(cudaGetLastError());
}
