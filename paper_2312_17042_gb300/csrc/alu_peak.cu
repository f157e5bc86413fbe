// alu_peak.cu -- FMA throughput of the current GPU in FP64 and FP32, the denominator of the
// ALU roofline of the FP64 path. Independent FMA chains per thread, a fixed trip count and a
// grid of blocks_per_SM x SMs; timed with CUDA events after a warm-up launch.
#include <cuda_runtime.h>

#include "cteno.h"

namespace {

template <typename T>
__global__ void fma_chains(T *sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  if (s == (T)-1) sink[blockIdx.x] = s;  // never true; keeps the chains alive
}

template <typename T>
int measure(double *tflops) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CTENO_ERR_CUDA;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nsm * 8, threads = 256, iters = 1000;
  T *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * blocks) != cudaSuccess) return CTENO_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_chains<T><<<blocks, threads>>>(sink, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e0);
  const int reps = 3;
  for (int r = 0; r < reps; ++r) fma_chains<T><<<blocks, threads>>>(sink, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess || ms <= 0.f) return CTENO_ERR_CUDA;
  const double flops = 2.0 * 64.0 * iters * (double)blocks * threads * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return CTENO_OK;
}

}  // namespace

extern "C" int cteno_measure_alu_peak(double *fp64_tflops, double *fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return CTENO_ERR_ARG;
  int rc = measure<double>(fp64_tflops);
  if (rc) return rc;
  return measure<float>(fp32_tflops);
}
