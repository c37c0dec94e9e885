// Arithmetic issue-rate measurement behind the "alu" rooflines of bench.py: the FP64 collision
// kernels are bound by the FP64 pipe (about two lanes per clock per SM on this part), the FP32 forms
// by FP32 issue, so their peaks are derived from unit counts and clocks; this measures the rates
// those counts predict.  Each thread runs eight independent dependency chains of one operation
// (fma, add or mul) for a fixed number of iterations; a launch of 8 blocks of 256 threads per SM is
// timed with CUDA events after one warm-up launch.
#include <cuda_runtime.h>

#include "../../include/qbe.h"

namespace {

constexpr int kChains = 8;
constexpr int kRateThreads = 256;

template <class T, int OP>
__global__ void __launch_bounds__(kRateThreads) k_issue_rate(T* sink, int iters, T a, T b) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
#pragma unroll 1
  for (int i = 0; i < iters; i += 8) {   // iters a multiple of 8: 64 operations per loop trip
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if (OP == 0) x[c] = fma(x[c], a, b);
        else if (OP == 1) x[c] = x[c] + b;
        else x[c] = x[c] * a;
      }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  sink[blockIdx.x * kRateThreads + threadIdx.x] = s;   // keeps the chains live
}

template <class T, int OP>
cudaError_t time_rate(T* sink, int blocks, int iters, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* rate) {
  const T a = (T)0.9999999, b = (T)1e-7;
  k_issue_rate<T, OP><<<blocks, kRateThreads, 0, s>>>(sink, iters, a, b);   // warm-up
  cudaError_t e = cudaEventRecord(e0, s);
  if (e != cudaSuccess) return e;
  k_issue_rate<T, OP><<<blocks, kRateThreads, 0, s>>>(sink, iters, a, b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaEventRecord(e1, s)) != cudaSuccess) return e;
  if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return e;
  float ms = 0.f;
  if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) return e;
  *rate = (double)blocks * kRateThreads * (double)iters * kChains / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace

int qbe_arith_issue_rates(int device, void* stream, double* rates) {
  if (!rates || device < 0) return QBE_ERR_ARG;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return QBE_ERR_CUDA;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  const int blocks = 8 * (nsm > 0 ? nsm : 1);
  cudaStream_t s = (cudaStream_t)stream;
  void* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, (size_t)blocks * kRateThreads * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // FP64 at about 2 lanes per clock per SM runs 4096 iterations in some 20 ms; FP32 needs 32x more
  if (e == cudaSuccess) e = time_rate<double, 0>((double*)sink, blocks, 4096, s, e0, e1, &rates[0]);
  if (e == cudaSuccess) e = time_rate<double, 1>((double*)sink, blocks, 4096, s, e0, e1, &rates[1]);
  if (e == cudaSuccess) e = time_rate<double, 2>((double*)sink, blocks, 4096, s, e0, e1, &rates[2]);
  if (e == cudaSuccess) e = time_rate<float, 0>((float*)sink, blocks, 131072, s, e0, e1, &rates[3]);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  cudaSetDevice(prev);
  return e == cudaSuccess ? QBE_OK : QBE_ERR_CUDA;
}
