// Arithmetic-pipe throughput probes used to derive the roofline peaks: independent FMA chains
// per thread (8 per thread, no memory traffic), a grid of 8 blocks of 256 threads per SM.
#include <cuda_runtime.h>

#include "mgx.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = x[i] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(int device, int iters, double* tflops) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MGX_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  T* d = nullptr;
  if (cudaMalloc(&d, sizeof(T) * blocks * threads) != cudaSuccess) return MGX_ERR_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int w = 0; w < 3; ++w) fma_chains<T><<<blocks, threads>>>(d, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e0);
  fma_chains<T><<<blocks, threads>>>(d, iters, (T)0.999, (T)0.001);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  const bool ok = cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  if (!ok || ms <= 0.0f) return MGX_ERR_CUDA;
  *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
  return MGX_OK;
}

}  // namespace

extern "C" int mgx_measure_fma_tflops(int device, int precision, double* tflops) {
  if (!tflops) return MGX_ERR_INVALID_ARGUMENT;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cudaSetDevice(device) != cudaSuccess) return MGX_ERR_INVALID_ARGUMENT;
  const int rc = precision == 64 ? run<double>(device, 4096, tflops)
                 : precision == 32 ? run<float>(device, 16384, tflops) : MGX_ERR_INVALID_ARGUMENT;
  cudaSetDevice(cur);
  return rc;
}
