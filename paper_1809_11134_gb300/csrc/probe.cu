// probe.cu -- qe_measure_alu_peaks: FMA throughput of this GPU in binary32 and
// binary64, the denominators of the arithmetic rooflines of the circuit and
// rescoring kernels.  Not part of the method: a measurement utility.
//
// Every thread runs kChains independent FMA chains for kIters iterations (no
// memory traffic but one store per thread, so the result is not optimised
// away); the grid fills every SM with 8 blocks of 256 threads.  Rate =
// 2 flops x FMAs / time of the second of two launches (CUDA events).
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/qe.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T *out, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t time_fma(uint32_t blocks, double *tflops) {
  T *out = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * 256 * sizeof(T));
  if (e != cudaSuccess) return e;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float ms = 0.f;
  if (e == cudaSuccess) {
    k_fma_chain<T><<<blocks, 256>>>(out, (T)0.999, (T)0.001);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a);
  if (e == cudaSuccess) {
    k_fma_chain<T><<<blocks, 256>>>(out, (T)0.999, (T)0.001);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess) {
    const double flops = 2.0 * (double)blocks * 256.0 * kIters * kChains;
    *tflops = flops / (ms * 1e-3) / 1e12;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  return e;
}

}  // namespace

extern "C" qe_status qe_measure_alu_peaks(double *fp32_tflops, double *fp64_tflops) {
  if (!fp32_tflops || !fp64_tflops) return QE_EINVAL;
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return QE_ECUDA;
  const uint32_t blocks = (uint32_t)prop.multiProcessorCount * 8;
  if (time_fma<float>(blocks, fp32_tflops) != cudaSuccess) return QE_ECUDA;
  if (time_fma<double>(blocks, fp64_tflops) != cudaSuccess) return QE_ECUDA;
  return QE_OK;
}
