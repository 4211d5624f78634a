// FP32 FMA-pipe probe: measures the achievable FP32 FLOP/s of this GPU with
// independent FFMA chains (8 per thread, no memory traffic), for the roofline
// of the ALU-bound kernels (walk and direct sum).
#include "internal.cuh"

namespace grav {
namespace {

__global__ void __launch_bounds__(256) k_ffma(int64_t iters, float seed, float *sink) {
  float a0 = seed + threadIdx.x, a1 = a0 + 1.f, a2 = a0 + 2.f, a3 = a0 + 3.f;
  float a4 = a0 + 4.f, a5 = a0 + 5.f, a6 = a0 + 6.f, a7 = a0 + 7.f;
  const float m = 0.999999f, c = 1e-7f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fmaf(a0, m, c); a1 = fmaf(a1, m, c); a2 = fmaf(a2, m, c); a3 = fmaf(a3, m, c);
      a4 = fmaf(a4, m, c); a5 = fmaf(a5, m, c); a6 = fmaf(a6, m, c); a7 = fmaf(a7, m, c);
    }
  }
  float r = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (r == 12345.678f) sink[threadIdx.x] = r;   // keeps the chains alive
}

}  // namespace

int probe_fp32(Ctx *c, int64_t iters, double *ms, double *flops) {
  float *sink = nullptr;
  const int rc = ctx_alloc(c, sink, 256);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = c->num_sms * 8;
  k_ffma<<<blocks, 256, 0, c->stream>>>(iters / 4 + 1, 1.0f, sink);   // warm-up
  ++c->launches;
  cudaEventRecord(e0, c->stream);
  k_ffma<<<blocks, 256, 0, c->stream>>>(iters, 1.0f, sink);
  ++c->launches;
  cudaEventRecord(e1, c->stream);
  cudaError_t err = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx_release(c, sink);
  if (err != cudaSuccess) return cuda_status(err);
  *ms = t;
  *flops = 2.0 * 8 * 16 * (double)iters * blocks * 256 / (t * 1e-3);
  return cuda_status(cudaGetLastError());
}

}  // namespace grav
