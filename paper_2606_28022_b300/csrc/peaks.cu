// fmo_fma_peak: measured FP32 / FP64 FMA throughput of the device (the
// denominators of the SCC kernel's roofline; the paper has no counterpart).
//
// Every thread runs kChains independent FMA chains for `iters` steps; the
// grid is 8 blocks of 256 threads per SM, so every SM sub-partition has
// enough independent FMAs in flight to keep its FMA pipe busy.  Timed with
// CUDA events on a private stream, best of five launches.
#include <cuda_runtime.h>

#include "../../include/fmo_xtb.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_loop_kernel(int iters, T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;   // contracted to one FMA
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == T(12345.678)) out[0] = s;   // keeps the chains live; never taken for these inputs
}

template <typename T>
cudaError_t measure(int device, double* tflops) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return e;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = 8 * sms, threads = 256;
  const int iters = sizeof(T) == 8 ? 1 << 12 : 1 << 16;
  T* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaMalloc(&out, sizeof(T))) != cudaSuccess) return e;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0.0;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(e0, st);
    fma_loop_kernel<T><<<blocks, threads, 0, st>>>(iters, T(0.999999), T(1e-7), out);
    cudaEventRecord(e1, st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * kChains * double(iters) * blocks * threads;
    if (rep > 0 && ms > 0.f) best = flops / (ms * 1e-3) / 1e12 > best ? flops / (ms * 1e-3) / 1e12 : best;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  cudaFree(out);
  *tflops = best;
  return e;
}

}  // namespace

extern "C" fmo_status fmo_fma_peak(int32_t precision, int32_t device, double* tflops) {
  if (!tflops || (precision != FMO_PREC_FP64 && precision != FMO_PREC_MIXED)) return FMO_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FMO_ERR_CUDA;
  const cudaError_t e = precision == FMO_PREC_FP64 ? measure<double>(device, tflops) : measure<float>(device, tflops);
  return e == cudaSuccess ? FMO_OK : FMO_ERR_CUDA;
}
