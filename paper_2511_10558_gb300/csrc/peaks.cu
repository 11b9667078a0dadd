// FMA-throughput probe: the measured FP64 and FP32 peaks that the ALU
// rooflines of the solver divide by. Each thread runs kChains independent
// dependent-FMA chains a_k <- a_k * b + c for `iters` iterations (2 flops per
// FMA), so with enough resident warps the FMA pipe, not latency, bounds the
// kernel. The result is kept live by a store that never happens for the
// chosen constants (the chains converge to c / (1 - b) = 0.1 per chain).
#include <cuda_runtime.h>

#include "carbox_peaks.h"

namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void fma_chains(T* sink, int iters, T b, T c) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x & 7) * T(0.01) + T(k) * T(0.001);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == T(-1)) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int cbx_peak_fma(int fp64, int grid, int block, int iters, void* stream, void* sink) {
  if (grid < 1 || block < 32 || block > 1024 || block % 32 || iters < 1 || !sink) return -1;
  cudaStream_t st = (cudaStream_t)stream;
  if (fp64)
    fma_chains<double><<<grid, block, 0, st>>>((double*)sink, iters, 1.0 - 1e-6, 1e-7);
  else
    fma_chains<float><<<grid, block, 0, st>>>((float*)sink, iters, 1.0f - 1e-4f, 1e-5f);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" double cbx_peak_fma_flops(int grid, int block, int iters) {
  return 2.0 * kChains * (double)grid * block * iters;
}
