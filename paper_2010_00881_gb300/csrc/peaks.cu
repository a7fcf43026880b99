// Measured arithmetic peaks of the GPU the library runs on (benchmark hook).
//
// The FP64 path of the solver (plain FP64 shared-matrix products) and the
// compensated df32 products of the mixed path are bound by FMA issue, not by
// memory, so their rooflines need the FMA throughput of this GPU.  Each
// thread runs kChains independent FMA chains (enough to cover the pipeline
// latency) for `iters` steps; the grid fills every SM several times over.
// Timed with CUDA events on a private stream, after one warm-up launch.
#include <cuda_runtime.h>

#include "fcm_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_kernel(T* out, int iters, T a, T b) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  // a store the compiler cannot drop, practically never taken
  if (s == (T)-1.2345e-30) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
cudaError_t measure(double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = sms * 8;
  const int iters = sizeof(T) == 8 ? 1 << 14 : 1 << 16;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  T* out = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(T));
  if (e == cudaSuccess) {
    // a close to 1 keeps the chains finite over the whole run
    fma_kernel<T><<<blocks, kThreads, 0, s>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e0, s);
    fma_kernel<T><<<blocks, kThreads, 0, s>>>(out, iters, (T)0.999999, (T)1e-7);
    cudaEventRecord(e1, s);
    e = cudaStreamSynchronize(s);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess)
    *tflops = 2.0 * kChains * (double)iters * blocks * kThreads / (ms * 1e-3) / 1e12;
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  return e;
}

}  // namespace

extern "C" fcm_status fcm_measure_fma_peak(int prec, double* tflops) {
  if (!tflops || (prec != FCM_FP64 && prec != FCM_MIXED)) {
    fcm::set_last_error("fcm_measure_fma_peak: invalid argument");
    return FCM_E_INVALID;
  }
  cudaError_t e = prec == FCM_FP64 ? measure<double>(tflops) : measure<float>(tflops);
  if (e != cudaSuccess) {
    fcm::set_last_error(cudaGetErrorString(e));
    return FCM_E_CUDA;
  }
  return FCM_OK;
}
