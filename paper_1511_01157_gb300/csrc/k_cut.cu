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
// integer indices, so that it always advances) and evaluates each piece in
// FP64 from its cell's four FP32 texels, loaded once.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"
#include "search_common.cuh"

namespace morse {

namespace {

using namespace dev;

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
  const double pmax = (double)(npix - 1);
  // One piece [t0, t1] lies in one cell (i0, j0) with the clamping state
  // fixed, so the lookup is a0 + d1 fx + d2 fy + d3 fx fy with fx, fy
  // linear in tau: its four texels are loaded once and the ends and the
  // vertex evaluated from them.
  auto piece = [&](double t0, double t1) {
    const double tm = 0.5 * (t0 + t1);
    const double pxm = ax * tm + bx, pym = ay * tm + by;
    const bool cx = pxm < 0.0 || pxm > pmax, cy = pym < 0.0 || pym > pmax;
    const double qx = fmin(fmax(pxm, 0.0), pmax), qy = fmin(fmax(pym, 0.0), pmax);
    int i0 = (int)floor(qx), j0 = (int)floor(qy);
    i0 = min(max(i0, 0), max(npix - 2, 0));
    j0 = min(max(j0, 0), max(npix - 2, 0));
    const int i1 = min(i0 + 1, npix - 1), j1 = min(j0 + 1, npix - 1);
    const double a00 = __ldg(&A[(size_t)j0 * npix + i0]);
    const double a10 = __ldg(&A[(size_t)j0 * npix + i1]);
    const double a01 = __ldg(&A[(size_t)j1 * npix + i0]);
    const double a11 = __ldg(&A[(size_t)j1 * npix + i1]);
    const double d1 = a10 - a00, d2 = a01 - a00, d3 = a00 - a10 - a01 + a11;
    // fx = ux + vx t, fy = uy + vy t (constant when clamped)
    const double vx = cx ? 0.0 : ax, ux = cx ? qx - i0 : bx - i0;
    const double vy = cy ? 0.0 : ay, uy = cy ? qy - j0 : by - j0;
    auto val = [&](double t) {
      const double fx = ux + vx * t, fy = uy + vy * t;
      return a00 + d1 * fx + d2 * fy + d3 * fx * fy;
    };
    double m = fmax(val(t0), val(t1));
    const double c2 = d3 * vx * vy;
    if (c2 < 0.0) {
      const double c1 = d1 * vx + d2 * vy + d3 * (ux * vy + uy * vx);
      const double tv = -c1 / (2.0 * c2);
      if (tv > t0 && tv < t1) m = fmax(m, val(tv));
    }
    return m;
  };
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
  double prev = ta;
  const int cap = 2 * npix + 8;  // crossings in a lane's part, at most
  for (int it = 0; it < cap; ++it) {
    const double tx = ax != 0.0 ? (kx - bx) * iax : CUDART_INF;
    const double ty = ay != 0.0 ? (ky - by) * iay : CUDART_INF;
    const double cur = fmin(fmin(tx, ty), tb);
    if (cur > prev) {
      best = fmax(best, piece(prev, cur));
      prev = cur;
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
