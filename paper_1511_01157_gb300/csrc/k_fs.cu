// Finite-source maps (§4.1: each point-source map convolved with radially
// symmetric, limb-darkened source profiles of fixed radii).
//
// out(i, j) = sum_{dx, dy} W(dx, dy) A(i + dx, j + dy), W the source
// profile integrated over the texels within R of the centre (normalised),
// a texel outside the map taking the Paczynski magnification of its centre
// (the lookup's outside rule).
//
// GB300 design: a block computes a 64 x 16 tile of outputs, four per
// thread, the threads of a warp on consecutive columns.  For each kernel
// row dy it stages the 16 input rows the tile needs, 64 + 2R texels wide,
// and that row's weights in shared memory, then every thread sums
// w * A along the row in FP32 (at most 2R + 1 terms) and adds the row sum
// to an FP64 accumulator, so the rounding does not grow with the source
// area.  Rows of zero weight beyond the disc are skipped by their
// half-width.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"

namespace morse {

namespace {

constexpr int kFsTX = 64, kFsTY = 16, kFsOut = 4;  // outputs per thread
constexpr int kFsThreads = (kFsTX / kFsOut) * kFsTY;

// Paczynski A of the centre of texel (x, y) outside the map, in FP32
// (relative error a few 1e-7; halo texels of a large source are many)
__device__ __forceinline__ float pspl_at(int x, int y, float L, float dlt) {
  const float y1 = __fmaf_rn((float)x + 0.5f, dlt, -L);
  const float y2 = __fmaf_rn((float)y + 0.5f, dlt, -L);
  const float u2 = __fmaf_rn(y1, y1, y2 * y2);
  return (u2 + 2.0f) * rsqrtf(u2 * (u2 + 4.0f));
}

__global__ void __launch_bounds__(kFsThreads)
    k_fs_conv(const float *__restrict__ A, int npix, double L, int R,
              const float *__restrict__ W, const int *__restrict__ rowhw,
              float *__restrict__ out) {
  extern __shared__ float fs_smem[];
  const int width = kFsTX + 2 * R;
  float *s_in = fs_smem;                 // [kFsTY][width]
  float *s_w = s_in + kFsTY * width;     // [2R + 1]
  const int tx = threadIdx.x % (kFsTX / kFsOut);
  const int ty = threadIdx.x / (kFsTX / kFsOut);
  const int x0 = blockIdx.x * kFsTX, y0 = blockIdx.y * kFsTY;
  const float Lf = (float)L, dltf = (float)((2.0 * L) / (double)npix);
  double acc[kFsOut];
#pragma unroll
  for (int k = 0; k < kFsOut; ++k) acc[k] = 0.0;
  for (int dy = -R; dy <= R; ++dy) {
    const int hw = rowhw[dy + R];  // weights nonzero for |dx| <= hw
    if (hw < 0) continue;          // block-uniform
    for (int t = threadIdx.x; t < kFsTY * width; t += blockDim.x) {
      const int r = t / width, c = t - r * width;
      const int x = x0 - R + c, y = y0 + dy + r;
      s_in[t] = (x >= 0 && x < npix && y >= 0 && y < npix)
                    ? A[(size_t)y * npix + x]
                    : pspl_at(x, y, Lf, dltf);
    }
    for (int t = threadIdx.x; t <= 2 * R; t += blockDim.x)
      s_w[t] = W[(size_t)(dy + R) * (2 * R + 1) + t];
    __syncthreads();
    float row[kFsOut];
#pragma unroll
    for (int k = 0; k < kFsOut; ++k) row[k] = 0.f;
    const float *base = s_in + ty * width + R + tx;
    for (int dx = -hw; dx <= hw; ++dx) {
      const float w = s_w[dx + R];
#pragma unroll
      for (int k = 0; k < kFsOut; ++k)
        row[k] = __fmaf_rn(w, base[dx + k * (kFsTX / kFsOut)], row[k]);
    }
#pragma unroll
    for (int k = 0; k < kFsOut; ++k) acc[k] += (double)row[k];
    __syncthreads();
  }
  const int y = y0 + ty;
#pragma unroll
  for (int k = 0; k < kFsOut; ++k) {
    const int x = x0 + tx + k * (kFsTX / kFsOut);
    if (x < npix && y < npix) out[(size_t)y * npix + x] = (float)acc[k];
  }
}

}  // namespace

size_t fs_smem_bytes(int R) {
  return sizeof(float) * ((size_t)kFsTY * (kFsTX + 2 * R) + 2 * R + 1);
}

cudaError_t launch_fs_conv(const float *A, int npix, double L, int R,
                           const float *W, const int *rowhw, float *out,
                           cudaStream_t st) {
  const size_t smem = fs_smem_bytes(R);
  cudaError_t e = cudaFuncSetAttribute(
      k_fs_conv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((npix + kFsTX - 1) / kFsTX, (npix + kFsTY - 1) / kFsTY);
  k_fs_conv<<<grid, kFsThreads, smem, st>>>(A, npix, L, R, W, rowhw, out);
  return cudaGetLastError();
}

}  // namespace morse
