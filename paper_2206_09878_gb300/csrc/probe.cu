// Issue-rate probe of the arithmetic pipes the kernels of this library are bound by (no paper counterpart:
// it supplies the denominators of the roofline fractions the benchmark reports).
//
// Every thread runs 8 independent chains of one operation (no chain waits on another, so the pipe, not the
// latency, sets the rate) over `iters` iterations; 8 CTAs of 256 threads per SM. The result is operations
// per second: one FMA, add or multiply per chain per iteration. The chains' final values are stored so that
// nothing is optimised away.
#include <cuda_runtime.h>

#include "lmvd_internal.h"

namespace lmvd {

template <class T, int OP>
__global__ void __launch_bounds__(256) k_rate(T* out, int iters, T b, T c) {
  T a[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) a[q] = (T)(threadIdx.x + q) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (OP == 0) a[q] = fma(a[q], b, c);
      else if (OP == 1) a[q] = a[q] + b;
      else a[q] = a[q] * b;
    }
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += a[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T, int OP>
static int rate(int sms, int iters, cudaStream_t st, double* ops) {
  const int blocks = 8 * sms, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return LMVD_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // b close to 1 and c small keep the chains finite and normal over any number of iterations
  const T b = OP == 1 ? (T)1e-7 : (T)0.9999999, c = (T)1e-7;
  k_rate<T, OP><<<blocks, threads, 0, st>>>(out, iters / 8 + 1, b, c);  // warm-up
  cudaEventRecord(e0, st);
  k_rate<T, OP><<<blocks, threads, 0, st>>>(out, iters, b, c);
  cudaEventRecord(e1, st);
  int err = LMVD_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
    err = LMVD_ERR_CUDA;
  else
    *ops = (double)blocks * threads * 8.0 * iters / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return err;
}

}  // namespace lmvd

extern "C" int lmvd_rate_probe(int op, int iters, double* ops_per_second, void* cuda_stream) {
  using namespace lmvd;
  if (!ops_per_second || iters < 1 || op < 0 || op > 3) return LMVD_ERR_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LMVD_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  switch (op) {
    case 0: return rate<double, 0>(sms, iters, st, ops_per_second);
    case 1: return rate<double, 1>(sms, iters, st, ops_per_second);
    case 2: return rate<double, 2>(sms, iters, st, ops_per_second);
    default: return rate<float, 0>(sms, iters, st, ops_per_second);
  }
}
