// Arithmetic-peak probe: the measured FP64 FMA, FP32 FMA and 32 × 32 → 64-bit
// integer multiply-add (mad.wide.s32) rates of the GPU, the denominators of
// the ALU-bound rooflines of the library's kernels (the FP64 patch mat-vecs and
// stage operator, the fixed-point patch mat-vecs).  Each thread runs eight
// independent chains of `iters` multiply-adds on values that stay bounded; one
// launch of 152 × 8 CTAs of 256 threads, timed with CUDA events on the given
// stream.  Not part of the solver.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/irkmg_probe.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T a, T b, int64_t iters, T* out) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);  // a = -1: x alternates, stays bounded
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == (T)12345.678) out[0] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(256) k_madwide_chain(int32_t a, int64_t iters, int64_t* out) {
  int64_t x[8];
  int32_t v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    x[k] = threadIdx.x + k;
    v[k] = (int32_t)(threadIdx.x * 7 + k);
  }
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      int64_t d;
      asm volatile("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(v[k]), "r"(a), "l"(x[k]));
      x[k] = d;
    }
  }
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= x[k];
  if (s == 0x123456789abcll) out[0] = s;
}

}  // namespace

extern "C" int irkmg_probe_peak(int kind, int64_t iters, void* cuda_stream, double* ops_per_s) {
  if (!ops_per_s || iters <= 0 || kind < 0 || kind > 2) return 1;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 3;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 3;
  void* out = nullptr;
  if (cudaMalloc(&out, 64) != cudaSuccess) return 2;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const unsigned grid = (unsigned)nsm * 8, block = 256;
  auto launch = [&](int64_t it) {
    if (kind == 0)
      k_fma_chain<double><<<grid, block, 0, st>>>(-1.0, 0.5, it, (double*)out);
    else if (kind == 1)
      k_fma_chain<float><<<grid, block, 0, st>>>(-1.0f, 0.5f, it, (float*)out);
    else
      k_madwide_chain<<<grid, block, 0, st>>>(3, it, (int64_t*)out);
  };
  launch(iters / 16 + 1);  // warm-up
  cudaEventRecord(e0, st);
  launch(iters);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) return 3;
  // FMA kinds: 2 flop per multiply-add; mad.wide: 1 operation per multiply-add
  const double ops = (double)grid * block * 8.0 * (double)iters * (kind < 2 ? 2.0 : 1.0);
  *ops_per_s = ops / (ms * 1e-3);
  return 0;
}
