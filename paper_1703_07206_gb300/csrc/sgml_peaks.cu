// sgml_peaks.cu -- measured arithmetic throughput of the current GPU, the denominator of the FP64
// form's roofline.  The FP64 form of the cycle runs every stencil sum, Jacobi update and residual in
// FP64 (Sec. 2's pseudo-time iteration without a precision split); on a GPU whose FP64 pipe is narrow
// that pipe, not HBM, bounds it, so the benchmark needs its measured rate.  The paper has no
// counterpart: this is a measurement aid.
//
// Kernel: every thread runs kChains independent FMA chains (a = a * b + c) for `iters` iterations,
// enough independent work per warp to keep the pipe busy whatever its latency; the grid fills every
// SM several times over.  Rate = FMA instructions (thread level) / elapsed time (CUDA events on the
// caller's stream, after a warm-up launch).
#include <cuda_runtime.h>

#include "sgml.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_chains_kernel(T* out, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = (T)0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  // never true for the arguments used (|a| stays below 2): keeps the chains alive without a store
  if (s == (T)-12345.0) out[blockIdx.x] = s;
}

template <typename T>
int measure(cudaStream_t st, T* buf, int sms, double* rate) {
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  const T b = (T)0.999, c = (T)1e-3;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SGML_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SGML_ERR_CUDA;
  }
  fma_chains_kernel<T><<<blocks, threads, 0, st>>>(buf, iters, b, c);  // warm-up
  cudaEventRecord(e0, st);
  const int reps = 3;
  for (int r = 0; r < reps; ++r) fma_chains_kernel<T><<<blocks, threads, 0, st>>>(buf, iters, b, c);
  cudaEventRecord(e1, st);
  float ms = 0.0f;
  int status = SGML_OK;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f)
    status = SGML_ERR_CUDA;
  else
    *rate = (double)reps * blocks * threads * (double)iters * kChains / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}

}  // namespace

extern "C" int sgml_measure_fma_rates(void* cuda_stream, double* fp64_fma_per_s, double* fp32_fma_per_s) {
  if (!fp64_fma_per_s || !fp32_fma_per_s) return SGML_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SGML_ERR_CUDA;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * sms * 8) != cudaSuccess) return SGML_ERR_CUDA;
  int s = measure<double>(st, buf, sms, fp64_fma_per_s);
  if (s == SGML_OK) s = measure<float>(st, (float*)buf, sms, fp32_fma_per_s);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  return s;
}
