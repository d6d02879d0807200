// Compute-throughput microbenchmarks for the roofline denominators of the SIMT
// kernels: FP32 fused multiply-add (scalar and packed two-lane), the MUFU tanh
// approximation, the CUDA library's accurate tanhf (the FP32 kernels form tanh from
// ex2 and rcp instead, two MUFU operations), and FP64 FMA; plus the
// SM clock seen while they run.  Each kernel runs many independent chains per
// thread on a grid of 4 CTAs of 256 threads per SM, so that issue, not latency,
// limits it.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "lrnr_internal.cuh"

namespace lrnr {
namespace {

constexpr int PK_CHAINS = 8;
constexpr int PK_THREADS = 256;

enum PeakOp { OP_FFMA = 0, OP_FFMA2 = 1, OP_TANH_APPROX = 2, OP_TANHF = 3, OP_DFMA = 4 };

template <int OP>
__global__ void __launch_bounds__(PK_THREADS) k_peak(int iters, float seed, float *sink,
                                                     long long *cycles) {
  const long long c0 = clock64();
  float acc = 0.0f;
  if constexpr (OP == OP_FFMA) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = seed + c + threadIdx.x * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) x[c] = fmaf(x[c], 0.999f, 1e-3f);
    }
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) acc += x[c];
  } else if constexpr (OP == OP_FFMA2) {
    float2 x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = make_float2(seed + c, seed - c + threadIdx.x * 1e-3f);
    const float2 a = make_float2(0.999f, 0.998f), b = make_float2(1e-3f, 2e-3f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) x[c] = __ffma2_rn(x[c], a, b);
    }
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) acc += x[c].x + x[c].y;
  } else if constexpr (OP == OP_TANH_APPROX || OP == OP_TANHF) {
    float x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = 0.1f * (seed + c) + threadIdx.x * 1e-4f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < PK_CHAINS; ++c) {
        if constexpr (OP == OP_TANH_APPROX) {
          float y;
          asm volatile("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x[c]));
          x[c] = y;
        } else {
          x[c] = tanhf(x[c]);
        }
      }
    }
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) acc += x[c];
  } else {
    double x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = (double)seed + c + threadIdx.x * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) x[c] = fma(x[c], 0.999, 1e-3);
    }
    double d = 0.0;
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) d += x[c];
    acc = (float)d;
  }
  const long long c1 = clock64();
  if (acc == 12345.678f) sink[blockIdx.x] = acc;   // keeps the chains alive
  if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

template <int OP>
cudaError_t run_peak(int blocks, int iters, float *sink, long long *cycles, cudaStream_t st,
                     float *ms) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) { cudaEventDestroy(a); return e; }
  k_peak<OP><<<blocks, PK_THREADS, 0, st>>>(std::max(1, iters / 8), 1.0f, sink, cycles);   // warm-up
  cudaEventRecord(a, st);
  k_peak<OP><<<blocks, PK_THREADS, 0, st>>>(iters, 1.0f, sink, cycles);
  cudaEventRecord(b, st);
  e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

}  // namespace
}  // namespace lrnr

using namespace lrnr;

extern "C" lrnr_status lrnr_measure_peaks(lrnr_peaks *out, void *stream) {
  if (!out) return LRNR_EINVAL;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return LRNR_ECUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int blocks = 4 * sms;
  float *sink = nullptr;
  long long *cycles = nullptr;
  if (cudaMalloc(&sink, sizeof(float) * blocks) != cudaSuccess) return LRNR_ENOMEM;
  if (cudaMalloc(&cycles, sizeof(long long) * blocks) != cudaSuccess) {
    cudaFree(sink);
    return LRNR_ENOMEM;
  }
  const double threads = (double)blocks * PK_THREADS;
  float ms[5] = {0, 0, 0, 0, 0};
  const int it_fma = 1 << 14, it_tanh = 1 << 12, it_dfma = 1 << 8;
  cudaError_t e = run_peak<OP_FFMA>(blocks, it_fma, sink, cycles, st, &ms[0]);
  // SM clock: the longest block of the FP32 FMA run (it spans the kernel) in cycles,
  // over that kernel's CUDA-event time
  std::vector<long long> cyc(blocks, 0);
  if (e == cudaSuccess)
    e = cudaMemcpy(cyc.data(), cycles, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
  const long long cmax = *std::max_element(cyc.begin(), cyc.end());
  if (e == cudaSuccess) e = run_peak<OP_FFMA2>(blocks, it_fma, sink, cycles, st, &ms[1]);
  if (e == cudaSuccess) e = run_peak<OP_TANH_APPROX>(blocks, it_tanh, sink, cycles, st, &ms[2]);
  if (e == cudaSuccess) e = run_peak<OP_TANHF>(blocks, it_tanh, sink, cycles, st, &ms[3]);
  if (e == cudaSuccess) e = run_peak<OP_DFMA>(blocks, it_dfma, sink, cycles, st, &ms[4]);
  cudaFree(sink);
  cudaFree(cycles);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LRNR_ENOMEM : LRNR_ECUDA;
  // flops: threads x iterations x 4 unrolled x chains x (2 per FMA, x 2 lanes packed)
  out->fp32_fma_tflops = threads * it_fma * 4 * PK_CHAINS * 2 / (ms[0] * 1e-3) / 1e12;
  out->fp32_fma2_tflops = threads * it_fma * 4 * PK_CHAINS * 4 / (ms[1] * 1e-3) / 1e12;
  out->tanh_approx_gops = threads * it_tanh * PK_CHAINS / (ms[2] * 1e-3) / 1e9;
  out->tanhf_gops = threads * it_tanh * PK_CHAINS / (ms[3] * 1e-3) / 1e9;
  out->fp64_fma_tflops = threads * it_dfma * 4 * PK_CHAINS * 2 / (ms[4] * 1e-3) / 1e12;
  out->sm_mhz = (double)cmax / (ms[0] * 1e-3) / 1e6;
  out->sms = sms;
  return LRNR_OK;
}
