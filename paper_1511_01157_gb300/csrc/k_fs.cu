// Finite-source maps (§4.1: each point-source map convolved with radially
// symmetric, limb-darkened source profiles of fixed radii).
//
// out(i, j) = sum_{dx, dy} W(dx, dy) A(i + dx, j + dy), W the source
// profile integrated over the texels within R of the centre (normalised),
// a texel outside the map taking the Paczynski magnification of its centre
// (the lookup's outside rule).
//
// GB300 design: a block computes a 64 x 16 tile of outputs, four adjacent
// ones per thread.  The 16 input rows the tile needs at kernel row dy, 64 +
// 2R texels wide, sit in a circular buffer in shared memory that takes one
// new row per dy, next to that row's weights;
// a thread then walks the row in aligned 16-byte chunks, so one chunk of
// texels and one of weights feed 16 FMAs (4 taps x 4 outputs).  Each row's
// sum is FP32 (at most 2R + 4 terms) and is added to an FP64 accumulator,
// so the rounding does not grow with the source area.  Rows of zero weight
// beyond the disc are skipped by their half-width.
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

// Staged row layout: column c holds x = x0 - Ra + c, Ra = R rounded up to a
// multiple of 4, so that the four outputs of a thread (x0 + 4 tx + k) and
// the taps of any dx fall in 16-byte chunks; Wd = row width in floats.
__host__ __device__ __forceinline__ int fs_ra(int R) { return (R + 3) & ~3; }
__host__ __device__ __forceinline__ int fs_width(int R) {
  return kFsTX + 2 * fs_ra(R) + 4;
}

__global__ void __launch_bounds__(kFsThreads)
    k_fs_conv(const float *__restrict__ A, int npix, double L, int R,
              const float *__restrict__ W, const int *__restrict__ rowhw,
              float *__restrict__ out) {
  extern __shared__ __align__(16) float fs_smem[];
  const int Ra = fs_ra(R), width = fs_width(R);
  float *s_in = fs_smem;                 // [kFsTY][width]
  float *s_w = s_in + kFsTY * width;     // [2 Ra + 4], zero outside the row
  const int tx = threadIdx.x % (kFsTX / kFsOut);
  const int ty = threadIdx.x / (kFsTX / kFsOut);
  const int x0 = blockIdx.x * kFsTX, y0 = blockIdx.y * kFsTY;
  const float Lf = (float)L, dltf = (float)((2.0 * L) / (double)npix);
  double acc[kFsOut];
#pragma unroll
  for (int k = 0; k < kFsOut; ++k) acc[k] = 0.0;
  // Circular buffer of kFsTY staged input rows: at kernel row dy the tile
  // needs rows y0 + dy + r, r < kFsTY, and input row y lives in slot
  // (y - y0 + R) mod kFsTY, so each step stages one new row.
  auto stage = [&](int y, int slot) {
    float *dst = s_in + slot * width;
    for (int c = threadIdx.x; c < width; c += blockDim.x) {
      const int x = x0 - Ra + c;
      dst[c] = (x >= 0 && x < npix && y >= 0 && y < npix)
                   ? A[(size_t)y * npix + x]
                   : pspl_at(x, y, Lf, dltf);
    }
  };
  for (int r = 0; r < kFsTY - 1; ++r) stage(y0 - R + r, r);
  for (int dy = -R; dy <= R; ++dy) {
    stage(y0 + dy + kFsTY - 1, (dy + R + kFsTY - 1) % kFsTY);
    const int hw = rowhw[dy + R];  // weights nonzero for |dx| <= hw
    if (hw < 0) {                  // block-uniform: nothing to add
      __syncthreads();
      continue;
    }
    // weights of this row at dx + Ra, zero beyond the disc
    for (int t = threadIdx.x; t < 2 * Ra + 4; t += blockDim.x) {
      const int dx = t - Ra;
      s_w[t] = (dx >= -hw && dx <= hw)
                   ? W[(size_t)(dy + R) * (2 * R + 1) + (dx + R)]
                   : 0.f;
    }
    __syncthreads();
    // taps dx = dxa - Ra for dxa in [Ra - hw, Ra + hw], in aligned groups
    // of four: output k needs s_in[4 tx + dxa + k]
    const int a0 = (Ra - hw) & ~3, a1 = Ra + hw;
    const float4 *row4 = reinterpret_cast<const float4 *>(
                             s_in + ((ty + dy + R) % kFsTY) * width) +
                         tx;
    const float4 *w4 = reinterpret_cast<const float4 *>(s_w);
    float rs[kFsOut] = {0.f, 0.f, 0.f, 0.f};
    float4 cur = row4[a0 >> 2];
    for (int dxa = a0; dxa <= a1; dxa += 4) {
      const float4 nxt = row4[(dxa >> 2) + 1];
      const float4 w = w4[dxa >> 2];
      const float v[8] = {cur.x, cur.y, cur.z, cur.w,
                          nxt.x, nxt.y, nxt.z, nxt.w};
      const float ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int o = 0; o < 4; ++o)
#pragma unroll
        for (int k = 0; k < kFsOut; ++k)
          rs[k] = __fmaf_rn(ww[o], v[o + k], rs[k]);
      cur = nxt;
    }
#pragma unroll
    for (int k = 0; k < kFsOut; ++k) acc[k] += (double)rs[k];
    __syncthreads();
  }
  const int y = y0 + ty;
#pragma unroll
  for (int k = 0; k < kFsOut; ++k) {
    const int x = x0 + kFsOut * tx + k;
    if (x < npix && y < npix) out[(size_t)y * npix + x] = (float)acc[k];
  }
}

// Source profile integrated over texel (dx, dy), |dx|, |dy| <= R, on
// kSub x kSub midpoint points (unnormalised), one thread per texel.
constexpr int kFsSub = 8;
__global__ void k_fs_weights(double rho, double gamma, int R,
                             double *__restrict__ w) {
  const int side = 2 * R + 1;
  const int n = side * side;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += gridDim.x * blockDim.x) {
    const int dy = k / side - R, dx = k % side - R;
    double acc = 0.0;
    for (int b = 0; b < kFsSub; ++b) {
      const double y = dy - 0.5 + (b + 0.5) / kFsSub;
      for (int a = 0; a < kFsSub; ++a) {
        const double x = dx - 0.5 + (a + 0.5) / kFsSub;
        const double u2 = (x * x + y * y) / (rho * rho);
        if (u2 < 1.0) acc += 1.0 - gamma * (1.0 - 1.5 * sqrt(1.0 - u2));
      }
    }
    w[k] = acc;
  }
}

}  // namespace

cudaError_t launch_fs_weights(double rho_px, double gamma, int R, double *w,
                              cudaStream_t st) {
  const int n = (2 * R + 1) * (2 * R + 1);
  int blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_fs_weights<<<blocks, 256, 0, st>>>(rho_px, gamma, R, w);
  return cudaGetLastError();
}

size_t fs_smem_bytes(int R) {
  return sizeof(float) *
         ((size_t)kFsTY * fs_width(R) + 2 * (size_t)fs_ra(R) + 4);
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
