// Throughput probes that give the rooflines of the hot path their measured
// denominators on the GPU at hand: FP32 and FP64 fused multiply-add issue,
// shared-memory atomic adds (the ray-shooting histogram) and 16-byte
// gathers from a window resident in L1 or in L2 (the map lookups).
#include <cuda_runtime.h>
#include <stdint.h>

#include "morse_internal.cuh"

namespace morse {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;  // independent dependency chains per thread

// kChains chains of n dependent FMAs per thread; the result is stored only
// under a condition the host never meets, so nothing is optimised away.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads)
    k_fma(int n, T b, T c, T *sink, int flag) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + i);
  for (int k = 0; k < n; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = a[i] * b + c;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (flag == 12345) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// n shared-memory atomic adds per thread to pseudo-random bins of a
// 128 x 128 window (the ray-shooting window size).
__global__ void __launch_bounds__(kProbeThreads)
    k_smem_atomic(int n, unsigned *sink, int flag) {
  extern __shared__ unsigned bins[];  // kRayWin * kRayWin
  for (int i = threadIdx.x; i < kRayWin * kRayWin; i += blockDim.x)
    bins[i] = 0;
  __syncthreads();
  unsigned x = 2654435761u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
  for (int k = 0; k < n; ++k) {
    x = x * 1664525u + 1013904223u;
    atomicAdd(&bins[x >> 18], 1u);  // 14 bits: 16384 bins
  }
  __syncthreads();
  if (flag == 12345 && threadIdx.x == 0) sink[blockIdx.x] = bins[0];
}

// n 16-byte loads per thread at pseudo-random cells of a window of
// `mask + 1` float4 (a power of two), summed.
__global__ void __launch_bounds__(kProbeThreads)
    k_gather(const float4 *__restrict__ win, unsigned mask, int n,
             float *sink, int flag) {
  unsigned x = 2654435761u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
  float s = 0.f;
  for (int k = 0; k < n; k += 4) {
    float4 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x = x * 1664525u + 1013904223u;
      v[j] = __ldg(&win[(x >> 8) & mask]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) s += v[j].x + v[j].y + v[j].z + v[j].w;
  }
  if (flag == 12345) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t probe_fma32(int blocks, int n, float *sink, cudaStream_t st) {
  k_fma<float><<<blocks, kProbeThreads, 0, st>>>(n, 0.999f, 1e-3f, sink, 0);
  return cudaGetLastError();
}

cudaError_t probe_fma64(int blocks, int n, double *sink, cudaStream_t st) {
  k_fma<double><<<blocks, kProbeThreads, 0, st>>>(n, 0.999, 1e-3, sink, 0);
  return cudaGetLastError();
}

cudaError_t probe_smem_atomic(int blocks, int n, unsigned *sink,
                              cudaStream_t st) {
  const int smem = (int)sizeof(unsigned) * kRayWin * kRayWin;
  cudaError_t e = cudaFuncSetAttribute(
      k_smem_atomic, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_smem_atomic<<<blocks, kProbeThreads, smem, st>>>(n, sink, 0);
  return cudaGetLastError();
}

cudaError_t probe_gather(const float4 *win, unsigned mask, int blocks, int n,
                         float *sink, cudaStream_t st) {
  k_gather<<<blocks, kProbeThreads, 0, st>>>(win, mask, n, sink, 0);
  return cudaGetLastError();
}

int probe_threads() { return kProbeThreads; }
int probe_chains() { return kChains; }

}  // namespace morse
