// Critical curves and caustics of the binary lens, for trajectory grids
// about the caustic centres (§4.2: a search over fixed distances r from the
// central regions of caustics, scaled by their sizes, and angles phi).
//
// On a critical curve det J = 0 (Eq. 4), i.e. D = sum_k eps_k /
// (conj(z) - x_k)^2 has modulus one: D = exp(-i psi).  For each psi that is
// the quartic in w = conj(z)
//     eps1 (w - x2)^2 + eps2 (w - x1)^2 - exp(-i psi) (w - x1)^2 (w - x2)^2,
// whose four roots one thread finds together by the Aberth-Ehrlich
// iteration in FP64; their images by Eq. 2 are the caustic points.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"

namespace morse {

namespace {

struct c2 {
  double re, im;
};
__device__ __forceinline__ c2 cadd(c2 a, c2 b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ c2 csub(c2 a, c2 b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ c2 cmul(c2 a, c2 b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ c2 cdiv(c2 a, c2 b) {
  const double d = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}

__global__ void k_critical(double s, double q, int n_psi, double2 *z_out,
                           double2 *zeta_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_psi) return;
  const double e1 = 1.0 / (1.0 + q), e2 = q / (1.0 + q);
  const double x1 = -s * e2, x2 = s * e1;
  double sn, cs;
  sincospi(2.0 * (double)k / (double)n_psi, &sn, &cs);
  const c2 ph = {cs, -sn};  // exp(-i psi)
  // (w - x1)^2 = w^2 + p1 w + p0 and (w - x2)^2 = w^2 + r1 w + r0
  const double p1 = -2.0 * x1, p0 = x1 * x1, r1 = -2.0 * x2, r0 = x2 * x2;
  // their product, real coefficients by power
  const double m[5] = {p0 * r0, p0 * r1 + p1 * r0, p0 + p1 * r1 + r0,
                       p1 + r1, 1.0};
  c2 c[5];
  for (int t = 0; t < 5; ++t) c[t] = cmul({-m[t], 0.0}, ph);
  c[0].re += e1 * r0 + e2 * p0;
  c[1].re += e1 * r1 + e2 * p1;
  c[2].re += e1 + e2;
  // monic: b_t = c_t / c_4
  c2 b[4];
  for (int t = 0; t < 4; ++t) b[t] = cdiv(c[t], c[4]);
  double R = 0.0;
  for (int t = 0; t < 4; ++t) R = fmax(R, hypot(b[t].re, b[t].im));
  R = 0.5 * (1.0 + R);
  c2 w[4];
  for (int t = 0; t < 4; ++t) {
    double a, bb;
    sincos(0.3 + 0.5 * CUDART_PI * t, &a, &bb);
    w[t] = {R * bb, R * a};
  }
  const c2 one = {1.0, 0.0};
  for (int it = 0; it < 200; ++it) {
    double moved = 0.0;
    for (int t = 0; t < 4; ++t) {
      c2 p = one, dp = {0.0, 0.0};
      for (int u = 3; u >= 0; --u) {
        dp = cadd(cmul(dp, w[t]), p);
        p = cadd(cmul(p, w[t]), b[u]);
      }
      if (p.re == 0.0 && p.im == 0.0) continue;
      const c2 nw = cdiv(p, dp);
      c2 sum = {0.0, 0.0};
      for (int u = 0; u < 4; ++u)
        if (u != t) sum = cadd(sum, cdiv(one, csub(w[t], w[u])));
      const c2 step = cdiv(nw, csub(one, cmul(nw, sum)));
      if (isfinite(step.re) && isfinite(step.im)) {
        w[t] = csub(w[t], step);
        moved = fmax(moved, hypot(step.re, step.im) /
                                (1.0 + hypot(w[t].re, w[t].im)));
      }
    }
    if (moved < 1e-15) break;
  }
  for (int t = 0; t < 4; ++t) {
    const c2 z = {w[t].re, -w[t].im};  // z = conj(w)
    // zeta = z - e1/(conj(z) - x1) - e2/(conj(z) - x2), conj(z) = w
    const c2 za = cdiv(one, csub(w[t], {x1, 0.0}));
    const c2 zb = cdiv(one, csub(w[t], {x2, 0.0}));
    const c2 zeta = csub(csub(z, {e1 * za.re, e1 * za.im}),
                         {e2 * zb.re, e2 * zb.im});
    z_out[4 * k + t] = make_double2(z.re, z.im);
    zeta_out[4 * k + t] = make_double2(zeta.re, zeta.im);
  }
}

}  // namespace

cudaError_t launch_critical(double s, double q, int n_psi, double2 *z,
                            double2 *zeta, cudaStream_t st) {
  const int threads = 128;
  k_critical<<<(n_psi + threads - 1) / threads, threads, 0, st>>>(s, q, n_psi,
                                                                  z, zeta);
  return cudaGetLastError();
}

}  // namespace morse
