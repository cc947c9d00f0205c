// Largest magnification along every (u0, alpha) line of a grid, for the
// minimum-magnification cut of §4.3 (i): a trajectory whose line never
// reaches the magnification the light curve requires cannot fit it, and
// the search skips every (t0, tE) of that line.
//
// Per line (one warp): inside the map the bilinear interpolant along the
// line is a quadratic in tau between consecutive crossings of texel-centre
// lines, so its maximum is at a crossing, an end of the inside interval or
// the vertex of a piece; outside the map the Paczynski A(|y|),
// |y|^2 = tau^2 + u0^2, is largest at the outside tau nearest 0.  The
// inside interval is cut into 32 equal parts, one per lane; a lane steps
// through its part's crossings in order (the next x- and y-crossings from
// integer indices, so that it always advances) and evaluates the pieces in
// FP64 from the FP32 texels.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"
#include "search_common.cuh"

namespace morse {

namespace {

using namespace dev;

// Bilinear interpolant at pixel coordinates (px, py), clamped to the
// outermost texel centres.
__device__ __forceinline__ double bil_px(const float *__restrict__ A,
                                         int npix, double px, double py) {
  const double hi = (double)(npix - 1);
  px = fmin(fmax(px, 0.0), hi);
  py = fmin(fmax(py, 0.0), hi);
  int i0 = (int)floor(px), j0 = (int)floor(py);
  i0 = min(max(i0, 0), max(npix - 2, 0));
  j0 = min(max(j0, 0), max(npix - 2, 0));
  const int i1 = min(i0 + 1, npix - 1), j1 = min(j0 + 1, npix - 1);
  const double fx = px - (double)i0, fy = py - (double)j0;
  const double a00 = __ldg(&A[(size_t)j0 * npix + i0]);
  const double a10 = __ldg(&A[(size_t)j0 * npix + i1]);
  const double a01 = __ldg(&A[(size_t)j1 * npix + i0]);
  const double a11 = __ldg(&A[(size_t)j1 * npix + i1]);
  return (1.0 - fy) * ((1.0 - fx) * a00 + fx * a10) +
         fy * ((1.0 - fx) * a01 + fx * a11);
}

__device__ __forceinline__ double pspl64(double u) {
  return (u * u + 2.0) / (u * sqrt(u * u + 4.0));
}

__global__ void k_line_max(const float *__restrict__ A, int npix, double L,
                           const double *__restrict__ u0v,
                           const double *__restrict__ ca,
                           const double *__restrict__ sa, int n_u0,
                           int n_alpha, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int line = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (line >= n_u0 * n_alpha) return;  // warp-uniform
  const int iu = line / n_alpha, ia = line - iu * n_alpha;
  const double u = u0v[iu], c = ca[ia], s = sa[ia];
  double lo, hi;
  slab_tau(L, u, c, s, lo, hi);
  double best;
  if (!(lo < hi)) {
    if (lane == 0) out[line] = pspl64(fabs(u));
    return;
  }
  {
    const double tn = (lo > 0.0 || hi < 0.0) ? 0.0 : (-lo < hi ? lo : hi);
    best = pspl64(sqrt(tn * tn + u * u));
  }
  const double dlt = (2.0 * L) / (double)npix;
  const double ax = c / dlt, bx = (-u * s + L) / dlt - 0.5;
  const double ay = s / dlt, by = (u * c + L) / dlt - 0.5;
  auto f = [&](double t) { return bil_px(A, npix, ax * t + bx, ay * t + by); };
  const double w = (hi - lo) / 32.0;
  const double ta = lo + lane * w;
  const double tb = lane == 31 ? hi : lo + (lane + 1) * w;
  // next crossing index along each axis, stepping in the direction of
  // increasing tau
  const double pxa = ax * ta + bx, pya = ay * ta + by;
  double kx = ax > 0.0 ? floor(pxa) + 1.0 : ceil(pxa) - 1.0;
  double ky = ay > 0.0 ? floor(pya) + 1.0 : ceil(pya) - 1.0;
  const double sx = ax > 0.0 ? 1.0 : -1.0, sy = ay > 0.0 ? 1.0 : -1.0;
  const double iax = ax != 0.0 ? 1.0 / ax : 0.0;
  const double iay = ay != 0.0 ? 1.0 / ay : 0.0;
  double prev = ta, fprev = f(ta);
  best = fmax(best, fprev);
  const int cap = 2 * npix + 8;  // crossings in a lane's part, at most
  for (int it = 0; it < cap; ++it) {
    const double tx = ax != 0.0 ? (kx - bx) * iax : CUDART_INF;
    const double ty = ay != 0.0 ? (ky - by) * iay : CUDART_INF;
    double cur = fmin(fmin(tx, ty), tb);
    if (!(cur > prev)) cur = prev;  // a crossing at prev: advance the index
    if (cur > prev) {
      const double fc = f(cur);
      const double tm = 0.5 * (prev + cur), h = 0.5 * (cur - prev);
      const double fm = f(tm);
      best = fmax(best, fmax(fc, fm));
      const double g2 = (fprev + fc - 2.0 * fm) / (2.0 * h * h);
      if (g2 < 0.0) {
        const double g1 = (fc - fprev) / (2.0 * h);
        const double tv = tm - g1 / (2.0 * g2);
        if (tv > prev && tv < cur) best = fmax(best, f(tv));
      }
      prev = cur;
      fprev = fc;
    }
    if (prev >= tb) break;
    if (tx <= ty) kx += sx;
    else ky += sy;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) best = fmax(best, __shfl_xor_sync(kFull, best, o));
  if (lane == 0) out[line] = best;
}

}  // namespace

cudaError_t launch_line_max(const float *A, int npix, double L,
                            const double *u0v, const double *ca,
                            const double *sa, int n_u0, int n_alpha,
                            double *out, cudaStream_t st) {
  const long long warps = (long long)n_u0 * n_alpha;
  const int threads = 128;
  const long long blocks = (warps * 32 + threads - 1) / threads;
  k_line_max<<<(unsigned)blocks, threads, 0, st>>>(A, npix, L, u0v, ca, sa,
                                                   n_u0, n_alpha, out);
  return cudaGetLastError();
}

}  // namespace morse
