// Throughput probes of the FP64 units, timed by the caller: the measured
// denominators of the roofline fractions the benchmark reports for the FP64-bound
// kernels (the reaction Newton, the rates, the smoother). Not part of the method.
//
//  kind 0: FP64 FMA (DFMA). Every thread runs 8 independent FMA chains, so the
//          pipe sees 8 independent instructions per warp between dependences.
//  kind 1: FP64 tensor-core MMA (mma.sync m8n8k4 f64, 512 flops each). Every warp
//          runs 4 independent accumulator chains.
//  kind 2: FP32 FMA, 8 chains per thread (the FP32 roof of the mixed kernels).
// The result of every chain is summed into out[thread] so nothing is eliminated.
#include "misdc_internal.cuh"

namespace misdc {
namespace {

__global__ void __launch_bounds__(256) k_probe_dfma(int iters, double seed, double *out) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + 0.001 * (threadIdx.x + k);
  const double m = 0.999999999, c = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_probe_ffma(int iters, double seed, double *out) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = (float)seed + 0.001f * (threadIdx.x + k);
  const float m = 0.9999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_probe_dmma(int iters, double seed, double *out) {
  const int lane = threadIdx.x & 31;
  double d[4][2];
#pragma unroll
  for (int k = 0; k < 4; ++k) { d[k][0] = 0.0; d[k][1] = 0.0; }
  const double a = seed * 1e-3 * (lane + 1), b = 1e-3 * (32 - lane);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(d[k][0]), "+d"(d[k][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += d[k][0] + d[k][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace misdc

using namespace misdc;

extern "C" misdc_status misdc_probe_flops(int kind, int blocks, int iters, double *out, double *flops,
                                          void *stream) {
  if (kind < 0 || kind > 2 || blocks < 1 || iters < 1 || !out || !flops) return MISDC_E_INVALID;
  const int threads = 256;
  cudaStream_t s = (cudaStream_t)stream;
  if (kind == 0) {
    k_probe_dfma<<<blocks, threads, 0, s>>>(iters, 1.0, out);
    *flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  } else if (kind == 1) {
    k_probe_dmma<<<blocks, threads, 0, s>>>(iters, 1.0, out);
    *flops = 512.0 * 4.0 * iters * (double)blocks * (threads / 32);
  } else {
    k_probe_ffma<<<blocks, threads, 0, s>>>(iters, 1.0, out);
    *flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  }
  return cudaGetLastError() == cudaSuccess ? MISDC_OK : MISDC_E_CUDA;
}
