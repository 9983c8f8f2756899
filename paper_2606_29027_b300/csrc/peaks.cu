// Measured ALU peaks for the roofline of the entry evaluator: a kernel of independent FMA
// chains (8 per thread, fully unrolled), enough CTAs for every SM, timed with CUDA events
// on the caller's stream.  Flops = 2 per FMA.
#include <cuda_runtime.h>

#include "common.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == (T)-1.2345) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <typename T>
cudaError_t run(int iters, double* tflops, cudaStream_t s) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blocks = nsm * 8;
  T* out = nullptr;
  if ((e = cudaMalloc(&out, sizeof(T) * blocks * 256)) != cudaSuccess) return e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  slar::count_launch(), k_fma<T><<<blocks, 256, 0, s>>>(out, 16, (T)0.999, (T)1e-3);   // warm-up
  cudaEventRecord(a, s);
  slar::count_launch(), k_fma<T><<<blocks, 256, 0, s>>>(out, iters, (T)0.999, (T)1e-3);
  cudaEventRecord(b, s);
  e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * 8 * 16 * (double)iters * blocks * 256;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return cudaSuccess;
}

}  // namespace

extern "C" slar_status slar_fma_peak(int fp64, int iters, double* tflops, void* stream) {
  if (!tflops || iters < 1 || iters > (1 << 24)) return SLAR_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = fp64 ? run<double>(iters, tflops, s) : run<float>(iters, tflops, s);
  return e == cudaSuccess ? SLAR_OK : SLAR_ECUDA;
}
