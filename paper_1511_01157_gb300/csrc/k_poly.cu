// Point-source magnification map by the lens polynomial (§4.1: the fifth-
// order polynomial inversion of Eq. 2 solved for a uniform grid of source
// positions, one GPU thread per map pixel), the paper's own map generator.
//
// Per texel centre zeta (FP64 throughout):
//  * The quintic is written in the frame centred on the midpoint of the two
//    masses, w = z - m, lenses at w = -a (primary, eps1) and w = +a
//    (secondary, eps2), a = s/2, omega = zeta - m.  Conjugating Eq. 2 gives
//    conj(w) = N / Dn with Dn = w^2 - a^2 and N = conj(omega) Dn + w + a d,
//    d = eps2 - eps1; substituting back and clearing the denominators
//    (N + a Dn)(N - a Dn) gives
//        (omega - w)(N^2 - a^2 Dn^2) + Dn N + a d Dn^2 = 0,
//    a quintic in w whose roots contain the images.
//  * Its five roots are found together by the Aberth-Ehrlich iteration
//    (each root moves by the Newton step corrected for the other roots),
//    from starting points on a circle enclosing them: in FP32 to a relative
//    move of 1e-5 (FP64 is 1/70 of the FP32 rate on this GPU), then in FP64
//    to 1e-12.
//  * Each root is polished by Newton's method on Eq. 2 itself (the step dw
//    solves f + dw + D conj(dw) = 0, D = d zeta / d conj(z)), which
//    sharpens images next to a low-mass lens where the polynomial's
//    coefficients lose digits.
//  * A root is an image when its Eq. 2 residual, relative to the size of
//    the terms Eq. 2 sums, is below 1e-4 before the polish and below 1e-9
//    after it, and it is not a repeat of an earlier root;
//    A = sum over images of 1/|det J| with det J = 1 - |D|^2 (Eq. 3-4).
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"

namespace morse {

namespace {

template <typename T>
struct cx {
  T re, im;
};
using cd = cx<double>;
template <typename T>
__device__ __forceinline__ cx<T> mk(T r, T i) { return {r, i}; }
template <typename T>
__device__ __forceinline__ cx<T> add(cx<T> a, cx<T> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename T>
__device__ __forceinline__ cx<T> sub(cx<T> a, cx<T> b) {
  return {a.re - b.re, a.im - b.im};
}
template <typename T>
__device__ __forceinline__ cx<T> mul(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cx<T> scl(T s, cx<T> a) {
  return {s * a.re, s * a.im};
}
template <typename T>
__device__ __forceinline__ cx<T> cnj(cx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ T ab2(cx<T> a) {
  return a.re * a.re + a.im * a.im;
}
__device__ __forceinline__ double ab(cd a) { return hypot(a.re, a.im); }
__device__ __forceinline__ float ab(cx<float> a) { return hypotf(a.re, a.im); }
template <typename T>
__device__ __forceinline__ cx<T> dvd(cx<T> a, cx<T> b) {
  // a / b by scaling with the larger component of b (two divisions)
  if (fabs(b.re) >= fabs(b.im)) {
    const T r = b.im / b.re, id = T(1) / (b.re + b.im * r);
    return {(a.re + a.im * r) * id, (a.im - a.re * r) * id};
  }
  const T r = b.re / b.im, id = T(1) / (b.re * r + b.im);
  return {(a.re * r + a.im) * id, (a.im * r - a.re) * id};
}

// Aberth-Ehrlich iterations on the monic quintic with coefficients b
// (z^5 + b4 z^4 + ... + b0) in precision T until the largest relative move
// is below tol or `iters` sweeps are done.
template <typename T>
__device__ __forceinline__ void aberth(const cx<T> (&b)[5], cx<T> (&z)[5],
                                       int iters, T tol) {
  const cx<T> one = mk<T>(1, 0);
  for (int it = 0; it < iters; ++it) {
    T moved = 0;
    for (int t = 0; t < 5; ++t) {
      cx<T> p = one, dp = mk<T>(0, 0);  // p and p' by Horner
      for (int u = 4; u >= 0; --u) {
        dp = add(mul(dp, z[t]), p);
        p = add(mul(p, z[t]), b[u]);
      }
      if (ab2(p) == T(0)) continue;
      const cx<T> nw = dvd(p, dp);  // Newton step p/p'
      cx<T> sum = mk<T>(0, 0);
      for (int u = 0; u < 5; ++u)
        if (u != t) sum = add(sum, dvd(one, sub(z[t], z[u])));
      // Aberth step: nw / (1 - nw * sum)
      const cx<T> step = dvd(nw, sub(one, mul(nw, sum)));
      if (isfinite(step.re) && isfinite(step.im)) {
        z[t] = sub(z[t], step);
        moved = fmax(moved, ab(step) / (T(1) + ab(z[t])));
      }
    }
    if (moved < tol) break;
  }
}

// The roots need only be good starting points for the polish on Eq. 2,
// which takes each image to full precision: FP32 sweeps stop at a relative
// move of 1e-5, FP64 sweeps at 1e-12 (a tighter test would sit at the
// rounding floor of ill-conditioned roots and use up the sweeps).
constexpr int kPolyIters = 30;    // FP64 sweeps at most
constexpr int kPolyItersF = 60;   // FP32 sweeps at most
constexpr int kPolishIters = 8;

// Lens equation in the midpoint frame: omega(w) and D = d omega/d conj(w).
__device__ __forceinline__ void lens(cd w, double a, double e1, double e2,
                                     cd *om, cd *D) {
  const cd wa = mk(w.re + a, -w.im);  // conj(w) + a
  const cd wb = mk(w.re - a, -w.im);  // conj(w) - a
  const cd ia = dvd(mk(1.0, 0.0), wa), ib = dvd(mk(1.0, 0.0), wb);
  *om = sub(sub(w, scl(e1, ia)), scl(e2, ib));
  *D = add(scl(e1, mul(ia, ia)), scl(e2, mul(ib, ib)));
}

__global__ void k_poly_map(double s, double q, double L, int npix,
                           float *__restrict__ A) {
  const size_t n = (size_t)npix * npix;
  const double e1 = 1.0 / (1.0 + q), e2 = q / (1.0 + q);
  const double a = 0.5 * s, dl = e2 - e1;
  // midpoint of the masses: the primary sits at -s e2, the secondary at
  // +s e1 (origin at the centre of mass)
  const double m = 0.5 * s * (e1 - e2);
  const double dlt = (2.0 * L) / (double)npix;
  const double a2 = a * a;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(k % npix), j = (int)(k / npix);
    const cd om = mk(-L + ((double)i + 0.5) * dlt - m,
                     -L + ((double)j + 0.5) * dlt);
    const cd omc = cnj(om);
    // Dn = w^2 - a^2; N = conj(omega) Dn + w + a d (coefficients by power)
    const cd N0 = mk(-a2 * omc.re + a * dl, -a2 * omc.im);
    const cd N1 = mk(1.0, 0.0);
    const cd N2 = omc;
    // Q = N^2 - a^2 Dn^2, Dn^2 = w^4 - 2 a^2 w^2 + a^4
    cd Q[5];
    Q[0] = sub(mul(N0, N0), mk(a2 * a2 * a2, 0.0));
    Q[1] = scl(2.0, mul(N0, N1));
    Q[2] = add(add(scl(2.0, mul(N0, N2)), mul(N1, N1)),
               mk(2.0 * a2 * a2, 0.0));
    Q[3] = scl(2.0, mul(N1, N2));
    Q[4] = sub(mul(N2, N2), mk(a2, 0.0));
    // p = (omega - w) Q + Dn N + a d Dn^2
    cd c[6];
    for (int t = 0; t < 6; ++t) c[t] = mk(0.0, 0.0);
    for (int t = 0; t < 5; ++t) {
      c[t] = add(c[t], mul(om, Q[t]));
      c[t + 1] = sub(c[t + 1], Q[t]);
    }
    // Dn N = (w^2 - a^2)(N0 + N1 w + N2 w^2)
    c[0] = sub(c[0], scl(a2, N0));
    c[1] = sub(c[1], scl(a2, N1));
    c[2] = add(c[2], sub(N0, scl(a2, N2)));
    c[3] = add(c[3], N1);
    c[4] = add(c[4], N2);
    // a d Dn^2
    const double ad = a * dl;
    c[0] = add(c[0], mk(ad * a2 * a2, 0.0));
    c[2] = add(c[2], mk(-2.0 * ad * a2, 0.0));
    c[4] = add(c[4], mk(ad, 0.0));
    double A_sum = 0.0;
    if (ab2(c[5]) > 0.0) {
      // monic form
      cd b[5];
      for (int t = 0; t < 5; ++t) b[t] = dvd(c[t], c[5]);
      // roots lie within 1 + max |b_t| (Cauchy's bound); start on a circle
      // of half that radius, rotated off the axes
      double R = 0.0;
      for (int t = 0; t < 5; ++t) R = fmax(R, ab(b[t]));
      R = 0.5 * (1.0 + R);
      // roots to single precision in FP32 from a circle of starting
      // points, then to double precision in FP64 (a few cubically
      // converging sweeps)
      cx<float> bf[5], zf[5];
      for (int t = 0; t < 5; ++t) {
        bf[t] = mk((float)b[t].re, (float)b[t].im);
        float sn, cs;
        sincosf(0.4f + 2.0f * (float)CUDART_PI * t / 5.0f, &sn, &cs);
        zf[t] = mk((float)R * cs, (float)R * sn);
      }
      aberth(bf, zf, kPolyItersF, 1e-5f);
      cd z[5];
      bool ok = true;
      for (int t = 0; t < 5; ++t) {
        z[t] = mk((double)zf[t].re, (double)zf[t].im);
        ok = ok && isfinite(z[t].re) && isfinite(z[t].im);
      }
      if (!ok)  // FP32 out of range: start the FP64 sweeps from the circle
        for (int t = 0; t < 5; ++t) {
          double sn, cs;
          sincos(0.4 + 2.0 * CUDART_PI * t / 5.0, &sn, &cs);
          z[t] = mk(R * cs, R * sn);
        }
      aberth(b, z, kPolyIters, 1e-12);
      // polish on Eq. 2 and keep the images
      cd img[5];
      int ni = 0;
      for (int t = 0; t < 5; ++t) {
        cd w = z[t], best = w;
        // the quintic has roots that are not images (3-image sources): they
        // leave Eq. 2 with an O(1) relative residual and are not polished,
        // lest Newton carry them onto an image found already
        {
          cd o, D;
          lens(w, a, e1, e2, &o, &D);
          const double sc0 = ab(w) + ab(om) + e1 / ab(mk(w.re + a, w.im)) +
                             e2 / ab(mk(w.re - a, w.im));
          if (!(ab(sub(o, om)) < 1e-4 * sc0)) continue;
        }
        double best_r = CUDART_INF;
        for (int it = 0; it <= kPolishIters; ++it) {
          cd o, D;
          lens(w, a, e1, e2, &o, &D);
          const cd f = sub(o, om);
          const double r = ab(f);
          if (!(r < best_r)) break;  // no longer improving: at the floor
          best_r = r;
          best = w;
          if (r == 0.0 || it == kPolishIters) break;
          const double det = 1.0 - ab2(D);
          if (det == 0.0) break;
          const cd dw = scl(1.0 / det, sub(mul(D, cnj(f)), f));
          w = add(w, dw);
          if (ab2(dw) <= 1e-32 * (1.0 + ab2(w))) {  // converged: one check
            lens(w, a, e1, e2, &o, &D);
            const double r2 = ab(sub(o, om));
            if (r2 < best_r) {
              best_r = r2;
              best = w;
            }
            break;
          }
        }
        // residual relative to the size of the terms of Eq. 2
        const double sc = ab(best) + ab(om) +
                          e1 / ab(mk(best.re + a, best.im)) +
                          e2 / ab(mk(best.re - a, best.im));
        if (!(best_r < 1e-9 * sc)) continue;
        bool dup = false;
        for (int u = 0; u < ni; ++u)
          if (ab(sub(best, img[u])) <= 1e-9 * (1.0 + ab(img[u]))) dup = true;
        if (dup) continue;
        img[ni++] = best;
        cd o, D;
        lens(best, a, e1, e2, &o, &D);
        A_sum += 1.0 / fabs(1.0 - ab2(D));
      }
    }
    A[k] = __double2float_rn(A_sum);
  }
}

}  // namespace

cudaError_t launch_poly_map(double s, double q, double L, int npix, float *A,
                            int sm_count, cudaStream_t st) {
  const size_t n = (size_t)npix * npix;
  size_t blocks = (n + 127) / 128;
  const size_t cap = (size_t)sm_count * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_poly_map<<<(unsigned)blocks, 128, 0, st>>>(s, q, L, npix, A);
  return cudaGetLastError();
}

}  // namespace morse
