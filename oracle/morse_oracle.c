/*
 * Plain, slow, FP64 CPU oracle for the MORSE hot path (McDougall & Albrow,
 * "MORSE code for GPUs", MNRAS 2015).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library; the two are independent
 * statements of the same mathematics.
 *
 * Every function follows the plain definition of what it computes, one ray /
 * one epoch / one trajectory at a time, with no blocking, fusion or
 * reordering:
 *
 *   lens geometry ........ §4.1 (origin at the centre of mass, masses on the
 *                          first axis) and §3 Eq. 2 (mass fractions eps_k)
 *   inverse ray shooting .. §3 (ray-shooting magnification maps) and §5
 *                          (inverse ray shooting); binned on the uniform
 *                          source grid of §4.1
 *   quintic + roots ....... §3 (inversion of Eq. 2 gives a fifth-order
 *                          polynomial with 3 or 5 image solutions); roots by
 *                          Laguerre's iteration (derived from the root sums
 *                          of p'/p and its derivative), damped and
 *                          restarted, with deflation and re-convergence on
 *                          the full polynomial
 *   magnification ......... §3 Eq. 3-4 (A_j = 1/det J, J = d zeta / d z,
 *                          total = sum over images; absolute value taken)
 *   Paczynski curve ....... §4.3 (ii) single-lens light curve
 *   map lookup ............ §4.2 (bilinear interpolation of the map at the
 *                          source position of each data point)
 *   flux model + fit ...... §4.1 Eq. 5-6 (F = Fs A + Fb, linear in A), chi^2
 *                          as the sum of per-data-point contributions (§4.2)
 *   seeds (top-K) ......... §4.4 (best local minima of the coarse search)
 *   peak library .......... §4.3 (iii) (peaks along a line: the
 *                          magnification turning from rising to falling)
 *   FP16 log10 map ........ storage form of the map values: log10 A rounded
 *                          to IEEE binary16 (round to nearest, ties to
 *                          even), decoded as 10^x
 *
 * Readings where the paper is silent (all mirrored by the CUDA path and
 * listed in the design notes): cell-centred image rays; half-open source
 * bins [-L, L); q = m2/m1 with the primary at -s q/(1+q); outside the map
 * the magnification is the Paczynski A(|y|) about the centre of mass; the
 * degenerate-fit rule; top-K order by (chi^2, index).
 *
 * Parity pins: every function here is pinned by a CPU test against closed
 * forms, invariants or brute force (Witt-Mao sum, q->0 Paczynski limit,
 * equal-mass on-axis closed form, ray conservation and mirror symmetry,
 * least-squares by QR, argmin by exhaustive search).
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * FMA contraction must stay off: the ray-shooting counts are compared
 * bit-for-bit with the GPU's FP64 path.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* Lens geometry (§4.1, §3 Eq. 2)                                       */
/* ------------------------------------------------------------------ */

/* q = m2/m1; eps1 = 1/(1+q), eps2 = q/(1+q); the origin is the centre of
 * mass, so the primary sits at -s*eps2 and the secondary at +s*eps1. */
void orc_lens(double s, double q, double *eps1, double *eps2, double *xa,
              double *xb) {
  double e1 = 1.0 / (1.0 + q);
  double e2 = q / (1.0 + q);
  *eps1 = e1;
  *eps2 = e2;
  *xa = -(s * e2);
  *xb = s * e1;
}

/* ------------------------------------------------------------------ */
/* Inverse ray shooting (§3, §5)                                        */
/* ------------------------------------------------------------------ */

/* Shoot nray x nray image-plane rays on the cell-centred grid over
 * [-X, X]^2 through Eq. 2 (real form) and histogram them on the npix x npix
 * source grid over [-L, L)^2.  counts is row-major, second source
 * coordinate major: counts[iy*npix + ix].  Rays landing outside the map are
 * counted in off_map; rays exactly on a lens are counted in lost.
 * nthreads > 1 splits image rows over OpenMP threads with private
 * histograms (integer sums: identical result for any thread count). */
int orc_rayshoot(double s, double q, double L, int npix, long long nray,
                 double X, uint32_t *counts, uint64_t *off_map, uint64_t *lost,
                 int nthreads) {
  if (npix <= 0 || nray <= 0 || !(L > 0.0) || !(X > 0.0)) return -1;
  double e1, e2, xa, xb;
  orc_lens(s, q, &e1, &e2, &xa, &xb);
  double h = (2.0 * X) / (double)nray;
  double dlt = (2.0 * L) / (double)npix;
  size_t nbin = (size_t)npix * (size_t)npix;
  memset(counts, 0, nbin * sizeof(uint32_t));
  uint64_t off_total = 0, lost_total = 0;
  if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads) reduction(+ : off_total, lost_total)
#endif
  {
    uint32_t *mine = counts;
    int tid = 0, nth = 1;
#ifdef _OPENMP
    tid = omp_get_thread_num();
    nth = omp_get_num_threads();
#endif
    if (nth > 1) mine = (uint32_t *)calloc(nbin, sizeof(uint32_t));
    for (long long j = tid; j < nray; j += nth) {
      double x2 = -X + ((double)j + 0.5) * h;
      for (long long i = 0; i < nray; ++i) {
        double x1 = -X + ((double)i + 0.5) * h;
        double d1x = x1 - xa;
        double r1 = d1x * d1x + x2 * x2;
        double d2x = x1 - xb;
        double r2 = d2x * d2x + x2 * x2;
        if (r1 == 0.0 || r2 == 0.0) {
          lost_total += 1;
          continue;
        }
        double y1 = x1 - e1 * d1x / r1 - e2 * d2x / r2;
        double y2 = x2 - e1 * x2 / r1 - e2 * x2 / r2;
        double v1 = (y1 + L) / dlt;
        double v2 = (y2 + L) / dlt;
        if (!(v1 >= 0.0 && v1 < (double)npix && v2 >= 0.0 &&
              v2 < (double)npix)) {
          off_total += 1;
          continue;
        }
        long ix = (long)floor(v1);
        long iy = (long)floor(v2);
        mine[(size_t)iy * (size_t)npix + (size_t)ix] += 1u;
      }
    }
    if (nth > 1) {
#ifdef _OPENMP
#pragma omp critical
#endif
      {
        for (size_t k = 0; k < nbin; ++k) counts[k] += mine[k];
      }
      free(mine);
    }
  }
  *off_map = off_total;
  *lost = lost_total;
  return 0;
}

/* Map value = area-averaged magnification of the pixel: ray count times the
 * image-plane area of a ray over the source-plane area of a pixel,
 * A = n h^2 / Delta^2, evaluated in FP64 and rounded to FP32. */
void orc_counts_to_mag(const uint32_t *counts, int npix, double L,
                       long long nray, double X, float *A) {
  double h = (2.0 * X) / (double)nray;
  double dlt = (2.0 * L) / (double)npix;
  double f = (h * h) / (dlt * dlt);
  size_t nbin = (size_t)npix * (size_t)npix;
  for (size_t k = 0; k < nbin; ++k) A[k] = (float)((double)counts[k] * f);
}

/* ------------------------------------------------------------------ */
/* Fifth-order lens polynomial (§3)                                     */
/* ------------------------------------------------------------------ */

/* polynomials as coefficient arrays, c[k] multiplies z^k */
static void pmul(const cplx *a, int na, const cplx *b, int nb, cplx *out) {
  for (int k = 0; k <= na + nb; ++k) out[k] = 0.0;
  for (int i = 0; i <= na; ++i)
    for (int j = 0; j <= nb; ++j) out[i + j] += a[i] * b[j];
}

/* Build the quintic whose roots contain the images of source zeta.
 * Conjugating Eq. 2 gives conj(z) = conj(zeta) + e1/(z-z1) + e2/(z-z2)
 * = N(z)/D(z) with D = (z-z1)(z-z2), N = conj(zeta) D + e1 (z-z2) +
 * e2 (z-z1).  Substituting back into Eq. 2, with conj(z) - z_k = P_k/D and
 * P_k = N - z_k D, and clearing denominators:
 *     (zeta - z) P1 P2 + e1 D P2 + e2 D P1 = 0.
 * c[0..5] receive the coefficients.  Returns -1 if the leading coefficient
 * vanishes (source exactly on a lens). */
int orc_quintic(double s, double q, double y1, double y2, double *cre,
                double *cim) {
  double e1, e2, xa, xb;
  orc_lens(s, q, &e1, &e2, &xa, &xb);
  cplx zeta = y1 + I * y2;
  cplx zc = conj(zeta);
  cplx D[3], Nn[3], P1[3], P2[3], lin[2], a[6], b[6], c6[6];
  /* D = z^2 - (z1+z2) z + z1 z2 */
  D[0] = xa * xb;
  D[1] = -(xa + xb);
  D[2] = 1.0;
  for (int k = 0; k < 3; ++k) Nn[k] = zc * D[k];
  /* + e1 (z - z2) + e2 (z - z1) */
  Nn[0] += -e1 * xb - e2 * xa;
  Nn[1] += e1 + e2;
  for (int k = 0; k < 3; ++k) {
    P1[k] = Nn[k] - xa * D[k];
    P2[k] = Nn[k] - xb * D[k];
  }
  /* (zeta - z) P1 P2 */
  {
    cplx p12[5];
    pmul(P1, 2, P2, 2, p12);
    lin[0] = zeta;
    lin[1] = -1.0;
    pmul(lin, 1, p12, 4, a); /* degree 5 */
  }
  /* e1 D P2 + e2 D P1 */
  {
    cplx dp2[5], dp1[5];
    pmul(D, 2, P2, 2, dp2);
    pmul(D, 2, P1, 2, dp1);
    for (int k = 0; k < 6; ++k) b[k] = 0.0;
    for (int k = 0; k < 5; ++k) b[k] = e1 * dp2[k] + e2 * dp1[k];
  }
  for (int k = 0; k < 6; ++k) c6[k] = a[k] + b[k];
  for (int k = 0; k < 6; ++k) {
    cre[k] = creal(c6[k]);
    cim[k] = cimag(c6[k]);
  }
  return (cabs(c6[5]) == 0.0) ? -1 : 0;
}

/* Value, first and second derivative of p(z) = sum_k a[k] z^k (degree m)
 * at x by Horner's scheme, and the scale b = sum_k |a[k]| |x|^k of the
 * terms: the rounding error of the computed p(x) is at most about
 * 2 m 2^-53 b, so |p(x)| below that is indistinguishable from zero. */
static cplx poly_eval(const cplx *a, int m, cplx x, cplx *d1, cplx *d2,
                      double *scale) {
  cplx p = a[m], q = 0.0, r = 0.0;
  double b = cabs(a[m]), ax = cabs(x);
  for (int j = m - 1; j >= 0; --j) {
    r = r * x + q;  /* p''/2 */
    q = q * x + p;  /* p'    */
    p = p * x + a[j];
    b = b * ax + cabs(a[j]);
  }
  *d1 = q;
  *d2 = 2.0 * r;
  *scale = b;
  return p;
}

/* One root of p (degree m >= 1) by Laguerre's iteration from *x.
 *
 * Derivation: with roots r_i, G = p'/p = sum 1/(x - r_i) and H = G^2 -
 * p''/p = sum 1/(x - r_i)^2.  Supposing the nearest root at distance d and
 * the other m - 1 all at one distance e, G = 1/d + (m-1)/e and H = 1/d^2 +
 * (m-1)/e^2; eliminating e gives d = m / (G +- sqrt((m-1)(m H - G^2))),
 * the sign that makes the denominator larger in modulus (the nearer root).
 *
 * Safeguards of this implementation:
 *  - damping: the step is taken only if it lowers |p|; otherwise it is
 *    halved, up to six times, and the trial with the smallest |p| is kept;
 *  - restart: after three steps in a row that could not lower |p|, or a
 *    vanishing denominator, the iterate moves to a point of the circle of
 *    radius |x| + R/4 (R = 1 + max_k |a_k / a_m|, a bound on every root's
 *    modulus) at the angle j * 2.39996 rad (the golden angle: restarts
 *    never repeat a direction);
 *  - stop: |p(x)| at the rounding floor 2 m 2^-53 sum |a_k| |x|^k, or a
 *    step below 2^-52 |x|, or 200 iterations (returns -1 then; the caller
 *    keeps the last iterate, which the Eq. 2 residual test then judges).
 * Returns the iterations used. */
static int laguerre_root(const cplx *a, int m, cplx *x) {
  const double u = 1.1102230246251565e-16; /* 2^-53 */
  double R = 0.0;
  for (int k = 0; k < m; ++k) {
    double t = cabs(a[k]) / cabs(a[m]);
    if (t > R) R = t;
  }
  R += 1.0;
  int stalls = 0, restarts = 0;
  for (int it = 1; it <= 200; ++it) {
    cplx d1, d2;
    double b;
    cplx p = poly_eval(a, m, *x, &d1, &d2, &b);
    double ap = cabs(p);
    if (ap <= 2.0 * m * u * b) return it;
    cplx G = d1 / p;
    cplx H = G * G - d2 / p;
    cplx root = csqrt((double)(m - 1) * ((double)m * H - G * G));
    cplx den = cabs(G + root) >= cabs(G - root) ? G + root : G - root;
    if (cabs(den) == 0.0 || !isfinite(creal(den)) ||
        !isfinite(cimag(den)) || stalls >= 3) {
      ++restarts;
      double ang = 2.39996322972865332 * (double)restarts;
      *x = (cabs(*x) + 0.25 * R) * (cos(ang) + I * sin(ang));
      stalls = 0;
      continue;
    }
    cplx dx = (double)m / den;
    if (cabs(dx) <= 2.0 * u * cabs(*x)) return it;
    cplx best = *x - dx;
    double best_ap = cabs(poly_eval(a, m, best, &d1, &d2, &b));
    for (int h = 0; h < 6 && !(best_ap < ap); ++h) {
      dx = 0.5 * dx;
      cplx trial = *x - dx;
      double t = cabs(poly_eval(a, m, trial, &d1, &d2, &b));
      if (t < best_ap) {
        best = trial;
        best_ap = t;
      }
    }
    stalls = (best_ap < ap) ? 0 : stalls + 1;
    *x = best;
  }
  return -1;
}

/* All 5 roots of the quintic: each by laguerre_root on the polynomial
 * deflated by the roots found so far (starting from z = 0, so the smaller
 * roots come off first and the deflation stays well conditioned), the
 * deflation being synthetic division by (z - root); then every root is
 * re-converged on the undeflated polynomial, which removes the error the
 * deflated coefficients carried. */
int orc_roots5(const double *cre, const double *cim, double *rre,
               double *rim) {
  cplx a[6], d[6], r[5];
  for (int k = 0; k < 6; ++k) a[k] = d[k] = cre[k] + I * cim[k];
  for (int m = 5; m >= 1; --m) {
    cplx x = 0.0;
    laguerre_root(d, m, &x);
    r[m - 1] = x;
    cplx carry = d[m]; /* d(z) = (z - x) d'(z) + remainder */
    for (int j = m - 1; j >= 0; --j) {
      cplx t = d[j];
      d[j] = carry;
      carry = t + x * carry;
    }
  }
  for (int k = 0; k < 5; ++k) laguerre_root(a, 5, &r[k]);
  for (int k = 0; k < 5; ++k) {
    rre[k] = creal(r[k]);
    rim[k] = cimag(r[k]);
  }
  return 0;
}

/* zeta(z) from Eq. 2 with real lens positions */
static cplx lens_map(cplx z, double e1, double e2, double xa, double xb) {
  cplx zc = conj(z);
  return z - e1 / (zc - xa) - e2 / (zc - xb);
}

/* det J = 1 - |d zeta / d conj(z)|^2 with d zeta/d conj(z) =
 * sum_k eps_k / (conj(z) - z_k)^2  (Eq. 4) */
static double detj(cplx z, double e1, double e2, double xa, double xb) {
  cplx zc = conj(z);
  cplx dz = e1 / ((zc - xa) * (zc - xa)) + e2 / ((zc - xb) * (zc - xb));
  double m = cabs(dz);
  return 1.0 - m * m;
}

/* Newton's method on Eq. 2 itself, from a root of the quintic.  With
 * f = zeta(z) - zeta and d = d zeta / d conj(z), a step dz solves
 * f + dz + d conj(dz) = 0, i.e. dz = (d conj(f) - f) / (1 - |d|^2).
 * Keeps the iterate of smallest residual.  This sharpens images next to a
 * low-mass lens, where the quintic's coefficients lose digits. */
static cplx newton_polish(cplx z, cplx zeta, double e1, double e2, double xa,
                          double xb, double *res_out) {
  cplx best = z;
  double best_res = cabs(lens_map(z, e1, e2, xa, xb) - zeta);
  for (int it = 0; it < 30 && best_res > 0.0; ++it) {
    cplx zc = conj(z);
    cplx f = lens_map(z, e1, e2, xa, xb) - zeta;
    cplx d = e1 / ((zc - xa) * (zc - xa)) + e2 / ((zc - xb) * (zc - xb));
    double den = 1.0 - creal(d * conj(d));
    if (den == 0.0 || !isfinite(den)) break;
    cplx dz = (d * conj(f) - f) / den;
    z = z + dz;
    double r = cabs(lens_map(z, e1, e2, xa, xb) - zeta);
    if (!(r < best_res)) {
      if (!(r <= 2.0 * best_res)) break; /* diverging: keep the best */
    } else {
      best = z;
      best_res = r;
    }
  }
  *res_out = best_res;
  return best;
}

/* Images of a point source at (y1, y2): the quintic's roots, each polished
 * by Newton on Eq. 2, ranked by their relative Eq. 2 residual
 * (a root that lands on an image already taken counts as spurious).  The
 * images are the roots that satisfy Eq. 2 to tol: 3 or 5 of them (§3).
 * For q below ~1e-7 the faint image next to the secondary sits closer to
 * it than FP64 resolves and only 2 are returned; its magnification is of
 * order q^2 and is dropped.  Outputs are ordered by residual.  Returns the
 * image count, or -1 on failure. */
int orc_images(double s, double q, double y1, double y2, double tol,
               double *zre, double *zim, double *dj, double *resid) {
  double cre[6], cim[6], rre[5], rim[5];
  double e1, e2, xa, xb;
  if (orc_quintic(s, q, y1, y2, cre, cim) != 0) return -1;
  orc_roots5(cre, cim, rre, rim);
  orc_lens(s, q, &e1, &e2, &xa, &xb);
  cplx zeta = y1 + I * y2;
  int order[5] = {0, 1, 2, 3, 4};
  double res[5];
  for (int k = 0; k < 5; ++k) {
    cplx z = newton_polish(rre[k] + I * rim[k], zeta, e1, e2, xa, xb, &res[k]);
    rre[k] = creal(z);
    rim[k] = cimag(z);
  }
  for (int k = 0; k < 5; ++k) /* duplicates: keep the first, drop the rest */
    for (int j = 0; j < k; ++j)
      if (cabs((rre[k] + I * rim[k]) - (rre[j] + I * rim[j])) <=
          1e-9 * (1.0 + cabs(rre[j] + I * rim[j])))
        res[k] = INFINITY;
  /* a residual is judged against the size of the terms that Eq. 2 sums,
   * |z| + |zeta| + sum_k eps_k/|z - z_k|, so that an image next to a lens
   * (large, cancelling terms) is held to the same relative precision */
  double scale[5];
  for (int k = 0; k < 5; ++k) {
    cplx z = rre[k] + I * rim[k];
    scale[k] = cabs(z) + cabs(zeta) + e1 / cabs(z - xa) + e2 / cabs(z - xb);
    if (isfinite(res[k])) res[k] = res[k] / scale[k];
  }
  for (int i = 1; i < 5; ++i) /* insertion sort by residual */
    for (int j = i; j > 0 && res[order[j]] < res[order[j - 1]]; --j) {
      int t = order[j];
      order[j] = order[j - 1];
      order[j - 1] = t;
    }
  int n = 0;
  while (n < 5 && res[order[n]] < tol) ++n;
  for (int k = 0; k < 5; ++k) {
    int o = order[k];
    zre[k] = rre[o];
    zim[k] = rim[o];
    resid[k] = res[o];
    dj[k] = detj(rre[o] + I * rim[o], e1, e2, xa, xb);
  }
  return n;
}

/* Point-source magnification, sum over images of 1/|det J| (Eq. 3). */
double orc_mag_point(double s, double q, double y1, double y2, int *nimg) {
  double zre[5], zim[5], dj[5], res[5];
  int n = orc_images(s, q, y1, y2, 1e-9, zre, zim, dj, res);
  if (nimg) *nimg = n;
  if (n < 0) return NAN;
  double A = 0.0;
  for (int k = 0; k < n; ++k) A += 1.0 / fabs(dj[k]);
  return A;
}

/* Gradient of the point-source magnification with respect to the source
 * position, by implicit differentiation of Eq. 2 at each image.  With
 * D = sum_k eps_k/(conj z - z_k)^2 and E = sum_k eps_k/(conj z - z_k)^3,
 * Eq. 2 gives d zeta = dz + D d conj(z), so
 *   dz = (d zeta - D conj(d zeta)) / (1 - |D|^2),
 * and det J = 1 - |D|^2 (Eq. 4) moves by d det J = 4 Re(D conj(E) dz).
 * A_j = 1/|det J_j| then changes by -sign(det J_j) d det J_j / det J_j^2.
 * d zeta = 1 for y1 and i for y2.  Returns A; g[0] = dA/dy1, g[1] = dA/dy2. */
double orc_mag_point_grad(double s, double q, double y1, double y2,
                          double *g) {
  double zre[5], zim[5], dj[5], res[5];
  double e1, e2, xa, xb;
  int n = orc_images(s, q, y1, y2, 1e-9, zre, zim, dj, res);
  g[0] = g[1] = 0.0;
  if (n < 0) return NAN;
  orc_lens(s, q, &e1, &e2, &xa, &xb);
  double A = 0.0;
  for (int k = 0; k < n; ++k) {
    cplx zc = zre[k] - I * zim[k];
    cplx ua = zc - xa, ub = zc - xb;
    cplx D = e1 / (ua * ua) + e2 / (ub * ub);
    cplx E = e1 / (ua * ua * ua) + e2 / (ub * ub * ub);
    double det = 1.0 - creal(D * conj(D));
    double sg = det > 0.0 ? 1.0 : -1.0;
    A += 1.0 / fabs(det);
    for (int c = 0; c < 2; ++c) {
      cplx dzeta = (c == 0) ? 1.0 : I;
      cplx dz = (dzeta - D * conj(dzeta)) / det;
      double ddet = 4.0 * creal(D * conj(E) * dz);
      g[c] += -sg * ddet / (det * det);
    }
  }
  return A;
}

/* Point-source map by the polynomial (§4.1: "solving the fifth-order
 * polynomial ... for a uniform grid of source positions"): texel (i, j)
 * holds the magnification at its centre (-L + (i+1/2) Delta, ...), rounded
 * to FP32.  Rows are independent (OpenMP). */
void orc_poly_map(double s, double q, double L, int npix, float *A,
                  int nthreads) {
  double dlt = (2.0 * L) / (double)npix;
  if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
  for (int j = 0; j < npix; ++j)
    for (int i = 0; i < npix; ++i)
      A[(size_t)j * npix + i] = (float)orc_mag_point(
          s, q, -L + ((double)i + 0.5) * dlt, -L + ((double)j + 0.5) * dlt,
          NULL);
}

/* IEEE 754 binary16 encoding of a finite double, round to nearest with
 * ties to even, from the format's definition: 1 sign bit, 5 exponent bits
 * (bias 15), 10 fraction bits; normal values (1 + f/1024) 2^(E-15) for
 * E = 1..30, subnormal values f 2^-24.  Magnitudes from 65520 up round to
 * infinity.  frexp/ldexp scale exactly and rint rounds to nearest even in
 * the default rounding mode, so the result is the correctly rounded one. */
uint16_t orc_half_bits(double x) {
  uint16_t sign = (signbit(x) ? 0x8000u : 0u);
  double a = fabs(x);
  if (a == 0.0) return sign;
  if (a >= 65520.0) return sign | 0x7C00u;
  int e;
  frexp(a, &e); /* a = m 2^e, m in [0.5, 1): binade 2^(e-1) */
  if (e - 1 >= -14) {
    double sig = rint(ldexp(a, 11 - e)); /* in [1024, 2048] */
    if (sig == 2048.0) {
      sig = 1024.0;
      e += 1;
    }
    int E = e - 1 + 15;
    if (E >= 31) return sign | 0x7C00u;
    return sign | (uint16_t)(E << 10) | (uint16_t)(sig - 1024.0);
  }
  /* subnormal (a rounded count of 2^-24 reaching 1024 is the smallest
   * normal, whose bit pattern is that count) */
  return sign | (uint16_t)rint(ldexp(a, 24));
}

/* binary16 bits -> double (exact). */
double orc_half_value(uint16_t h) {
  int E = (h >> 10) & 31, f = h & 1023;
  double v;
  if (E == 0)
    v = ldexp((double)f, -24);
  else if (E == 31)
    v = f ? NAN : INFINITY;
  else
    v = ldexp((double)(1024 + f), E - 25);
  return (h & 0x8000u) ? -v : v;
}

/* FP16 storage form of a map: code = half(log10(max(A, A_floor))) per
 * texel, with A the FP32 map value. */
void orc_log10_half(const float *A, long long n, double a_floor,
                    uint16_t *codes) {
  for (long long k = 0; k < n; ++k) {
    double a = (double)A[k];
    codes[k] = orc_half_bits(log10(a > a_floor ? a : a_floor));
  }
}

/* Decoded FP16 map: A = 10^x of each code, rounded to FP32. */
void orc_half_decode(const uint16_t *codes, long long n, float *A) {
  for (long long k = 0; k < n; ++k)
    A[k] = (float)pow(10.0, orc_half_value(codes[k]));
}

/* Finite-source kernel (§4.1: maps convolved with radially symmetric,
 * limb-darkened source profiles).  Surface brightness of a source of
 * radius rho (in texels) with linear limb darkening in the Gamma form,
 *     I(r) = 1 - Gamma (1 - 3/2 sqrt(1 - r^2/rho^2)),  r < rho,
 * integrated over each texel (dx, dy), |dx|, |dy| <= R, by the midpoint
 * rule on sub x sub points, then normalised to sum 1.  W is
 * (2R+1)^2, row-major in dy.  A source smaller than a texel falls on the
 * centre texel alone. */
void orc_fs_weights(double rho, double gamma, int R, int sub, double *W) {
  int side = 2 * R + 1;
  double tot = 0.0;
  for (int dy = -R; dy <= R; ++dy)
    for (int dx = -R; dx <= R; ++dx) {
      double acc = 0.0;
      for (int b = 0; b < sub; ++b)
        for (int a = 0; a < sub; ++a) {
          double x = dx - 0.5 + (a + 0.5) / sub;
          double y = dy - 0.5 + (b + 0.5) / sub;
          double r2 = (x * x + y * y) / (rho * rho);
          if (r2 < 1.0) acc += 1.0 - gamma * (1.0 - 1.5 * sqrt(1.0 - r2));
        }
      W[(dy + R) * side + (dx + R)] = acc;
      tot += acc;
    }
  if (tot <= 0.0) { /* sub-texel source */
    for (int k = 0; k < side * side; ++k) W[k] = 0.0;
    W[R * side + R] = 1.0;
    return;
  }
  for (int k = 0; k < side * side; ++k) W[k] /= tot;
}

double orc_pspl(double u);

/* Convolution of a map with weights W (2R+1)^2: out[j][i] =
 * sum W[dy][dx] A(i+dx, j+dy), where a texel outside the map takes the
 * Paczynski A of its centre's distance from the origin (the outside rule
 * of the lookup). */
void orc_fs_convolve(const float *A, int npix, double L, const double *W,
                     int R, double *out, int nthreads) {
  double dlt = 2.0 * L / npix;
  int side = 2 * R + 1;
  if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1)
#endif
  for (int j = 0; j < npix; ++j)
    for (int i = 0; i < npix; ++i) {
      double acc = 0.0;
      for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
          double w = W[(dy + R) * side + (dx + R)];
          if (w == 0.0) continue;
          int x = i + dx, y = j + dy;
          double a;
          if (x >= 0 && x < npix && y >= 0 && y < npix) {
            a = (double)A[(size_t)y * npix + x];
          } else {
            double y1 = -L + (x + 0.5) * dlt, y2 = -L + (y + 0.5) * dlt;
            a = orc_pspl(sqrt(y1 * y1 + y2 * y2));
          }
          acc += w * a;
        }
      out[(size_t)j * npix + i] = acc;
    }
}

/* Single-lens (Paczynski) magnification A(u) = (u^2+2)/(u sqrt(u^2+4)). */
double orc_pspl(double u) {
  return (u * u + 2.0) / (u * sqrt(u * u + 4.0));
}

/* ------------------------------------------------------------------ */
/* Map lookup along a straight trajectory (§4.2)                        */
/* ------------------------------------------------------------------ */

/* Source position at time t: tau = (t - t0)/tE, moving along angle alpha
 * from the lens axis with closest approach u0 to the centre of mass. */
void orc_traj_point(double t, double t0, double tE, double u0, double alpha,
                    double *y1, double *y2) {
  double tau = (t - t0) / tE;
  double ca = cos(alpha), sa = sin(alpha);
  *y1 = tau * ca - u0 * sa;
  *y2 = tau * sa + u0 * ca;
}

/* Bilinear interpolation between texel centres (texel (i,j) centred at
 * -L + (i+1/2) Delta).  Coordinates are clamped to the outermost texel
 * centres.  Outside the map (|y1| >= L or |y2| >= L) the Paczynski
 * magnification at |y| about the centre of mass is used. */
double orc_map_A(const float *A, int npix, double L, double y1, double y2) {
  if (fabs(y1) >= L || fabs(y2) >= L) return orc_pspl(sqrt(y1 * y1 + y2 * y2));
  double dlt = (2.0 * L) / (double)npix;
  double px = (y1 + L) / dlt - 0.5;
  double py = (y2 + L) / dlt - 0.5;
  double hi = (double)(npix - 1);
  if (px < 0.0) px = 0.0;
  if (px > hi) px = hi;
  if (py < 0.0) py = 0.0;
  if (py > hi) py = hi;
  long i0 = (long)floor(px), j0 = (long)floor(py);
  if (i0 > npix - 2) i0 = npix - 2;
  if (j0 > npix - 2) j0 = npix - 2;
  if (i0 < 0) i0 = 0; /* npix == 1 */
  if (j0 < 0) j0 = 0;
  double fx = px - (double)i0, fy = py - (double)j0;
  long i1 = (i0 + 1 < npix) ? i0 + 1 : i0, j1 = (j0 + 1 < npix) ? j0 + 1 : j0;
  double a00 = A[j0 * npix + i0], a10 = A[j0 * npix + i1];
  double a01 = A[j1 * npix + i0], a11 = A[j1 * npix + i1];
  return (1.0 - fy) * ((1.0 - fx) * a00 + fx * a10) +
         fy * ((1.0 - fx) * a01 + fx * a11);
}

/* ------------------------------------------------------------------ */
/* Linear flux fit and chi^2 (§4.1 Eq. 5-6, §4.2)                       */
/* ------------------------------------------------------------------ */

/* Bilinear interpolant of the map at (y1, y2) with the coordinates clamped
 * to the outermost texel centres (the lookup inside the map, continued to
 * the edge). */
static double bil_clamped(const float *A, int npix, double L, double y1,
                          double y2) {
  double dlt = (2.0 * L) / (double)npix;
  double px = (y1 + L) / dlt - 0.5, py = (y2 + L) / dlt - 0.5;
  double hi = (double)(npix - 1);
  px = px < 0.0 ? 0.0 : (px > hi ? hi : px);
  py = py < 0.0 ? 0.0 : (py > hi ? hi : py);
  long i0 = (long)floor(px), j0 = (long)floor(py);
  if (i0 > npix - 2) i0 = npix - 2;
  if (j0 > npix - 2) j0 = npix - 2;
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  long i1 = (i0 + 1 < npix) ? i0 + 1 : i0, j1 = (j0 + 1 < npix) ? j0 + 1 : j0;
  double fx = px - (double)i0, fy = py - (double)j0;
  return (1.0 - fy) * ((1.0 - fx) * A[j0 * npix + i0] + fx * A[j0 * npix + i1]) +
         fy * ((1.0 - fx) * A[j1 * npix + i0] + fx * A[j1 * npix + i1]);
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Largest magnification a source meets anywhere on the straight line
 * (u0, alpha) (§4.3 (i): the magnification along a trajectory read from
 * the point-source map).  Inside the map the bilinear interpolant along
 * the line is a quadratic in tau between consecutive crossings of texel-
 * centre lines, so its maximum is at a crossing, at an end of the inside
 * interval, or at the vertex of a piece; outside the map (tau <= tau_lo or
 * tau >= tau_hi, or everywhere when the line misses the map) the Paczynski
 * A(|y|), |y|^2 = tau^2 + u0^2, is largest at the outside tau nearest 0. */
double orc_line_max(const float *A, int npix, double L, double u,
                    double alpha) {
  double c = cos(alpha), s = sin(alpha);
  /* tau interval inside |y1| < L, |y2| < L */
  double lo = -INFINITY, hi = INFINITY;
  if (c != 0.0) {
    double a0 = (-L + u * s) / c, a1 = (L + u * s) / c;
    lo = fmax(lo, fmin(a0, a1));
    hi = fmin(hi, fmax(a0, a1));
  } else if (!(fabs(u * s) < L)) {
    hi = lo;
  }
  if (s != 0.0) {
    double b0 = (-L - u * c) / s, b1 = (L - u * c) / s;
    lo = fmax(lo, fmin(b0, b1));
    hi = fmin(hi, fmax(b0, b1));
  } else if (!(fabs(u * c) < L)) {
    hi = lo;
  }
  double best;
  /* outside part */
  if (!(lo < hi)) {
    best = orc_pspl(fabs(u));
    return best;
  }
  {
    double tn = (lo > 0.0 || hi < 0.0) ? 0.0 : (-lo < hi ? lo : hi);
    best = orc_pspl(sqrt(tn * tn + u * u));
  }
  /* inside: breakpoints where a texel-centre coordinate is an integer */
  double dlt = (2.0 * L) / (double)npix;
  double ax = c / dlt, bx = (-u * s + L) / dlt - 0.5;
  double ay = s / dlt, by = (u * c + L) / dlt - 0.5;
  size_t cap = 2 * (size_t)npix + 4, nb = 0;
  double *tb = (double *)malloc(cap * sizeof(double));
  tb[nb++] = lo;
  tb[nb++] = hi;
  for (int k = 0; k < npix; ++k) {
    if (ax != 0.0) {
      double t = ((double)k - bx) / ax;
      if (t > lo && t < hi) tb[nb++] = t;
    }
    if (ay != 0.0) {
      double t = ((double)k - by) / ay;
      if (t > lo && t < hi) tb[nb++] = t;
    }
  }
  qsort(tb, nb, sizeof(double), cmp_double);
  for (size_t k = 0; k + 1 < nb; ++k) {
    double ta = tb[k], tc = tb[k + 1];
    double fa = bil_clamped(A, npix, L, ta * c - u * s, ta * s + u * c);
    if (fa > best) best = fa;
    if (!(tc > ta)) continue;
    double tm = 0.5 * (ta + tc), h = 0.5 * (tc - ta);
    double fc = bil_clamped(A, npix, L, tc * c - u * s, tc * s + u * c);
    double fm = bil_clamped(A, npix, L, tm * c - u * s, tm * s + u * c);
    if (fc > best) best = fc;
    if (fm > best) best = fm;
    double g2 = (fa + fc - 2.0 * fm) / (2.0 * h * h); /* curvature / 2 */
    if (g2 < 0.0) {
      double g1 = (fc - fa) / (2.0 * h);
      double tv = tm - g1 / (2.0 * g2);
      if (tv > ta && tv < tc) {
        double fv = bil_clamped(A, npix, L, tv * c - u * s, tv * s + u * c);
        if (fv > best) best = fv;
      }
    }
  }
  free(tb);
  return best;
}

/* ------------------------------------------------------------------ */
/* Peak library along a line (§4.3 (iii)-(v))                           */
/* ------------------------------------------------------------------ */

/* Peaks of the map along the line of impact u and direction (c, s) =
 * (cos alpha, sin alpha) about the origin, positions measured from the
 * line's reference point, which lies tau = shift past the closest approach
 * to the origin.
 *
 * Definition (§4.3 (iii)): a peak is where the magnification along the
 * line turns from rising to falling.  The profile (the paper does not say
 * how a line is sampled): samples at tau_k = k h, h = Delta / sub, for
 * |k| <= sub npix, kept where the point y = tau_k (c, s) + u (-s, c) is
 * inside the map (|y1| < L and |y2| < L); the value is the map's bilinear
 * lookup between texel centres, coordinates clamped to the outermost
 * centres, everything in FP64.  A rise is confirmed once a value exceeds
 * r = 1 + delta times the lowest value since the last peak; the highest
 * value after it is a peak once a later value lies below it by the factor
 * r (delta = 0: every turn; a plateau counts once, at its first sample).
 * The profile must rise before its first peak, so the first sample is
 * never one.
 *
 * Error bounds for a comparison with an FP32 evaluation of the same
 * profile.  An FP32 evaluation places the sample at texel coordinates off
 * by at most dp = 2 2^-24 (4 |a tau| + |b| + |p| + 1) per axis (p = a tau +
 * b with a, b and h rounded to FP32, tau = k h, a tau and the sum rounded:
 * five roundings, doubled as a margin), which moves the value by at most
 * G dp per axis, G the largest texel difference along that axis over the
 * cells within dp, and the FP32 bilinear itself adds at most 16 2^-24 max
 * A of those cells.  err_k is that sum.  A decision
 * of the detector whose two sides are closer than the sum of their bounds
 * (including the inside-the-map test and the max_peaks-th versus the next
 * highest peak) could go either way in FP32; such a line is flagged
 * *uncertain.  Every decision of an unflagged line is the same in any
 * evaluation within the bounds, so its count and peak positions are
 * exactly determined and its heights are within herr.
 *
 * Returns the number of peaks.  pos / height / herr receive the max_peaks
 * highest (ties: the earlier one), in increasing tau, as (k h - shift,
 * value, err); unused slots are NaN. */
static double texel_at(const float *A, int npix, long i, long j) {
  if (i < 0) i = 0;
  if (j < 0) j = 0;
  if (i > npix - 1) i = npix - 1;
  if (j > npix - 1) j = npix - 1;
  return (double)A[(size_t)j * (size_t)npix + (size_t)i];
}

/* Bounds of |d v / d px| and |d v / d py| of the clamped bilinear lookup
 * over the texel coordinates within (dpx, dpy) of (qx, qy): the largest
 * texel difference along each axis over the cells those positions touch
 * (the lookup is linear along each axis within a cell), and max A of those
 * cells. */
static void cell_slopes(const float *A, int npix, double qx, double qy,
                        double dpx, double dpy, double *gx, double *gy,
                        double *amax) {
  long ia = (long)floor(qx - dpx), ib = (long)floor(qx + dpx);
  long ja = (long)floor(qy - dpy), jb = (long)floor(qy + dpy);
  double sx = 0.0, sy = 0.0, am = 0.0;
  for (long j = ja; j <= jb; ++j)
    for (long i = ia; i <= ib; ++i)
      for (long b = 0; b <= 1; ++b)
        for (long a = 0; a <= 1; ++a) {
          double t = texel_at(A, npix, i + a, j + b);
          if (t > am) am = t;
          if (a == 0) {
            double d = fabs(texel_at(A, npix, i + 1, j + b) - t);
            if (d > sx) sx = d;
          }
          if (b == 0) {
            double d = fabs(texel_at(A, npix, i + a, j + 1) - t);
            if (d > sy) sy = d;
          }
        }
  *gx = sx;
  *gy = sy;
  *amax = am;
}

/* The detector of orc_line_peaks over samples (v[i], e[i]), i < n, in
 * order, skipping those with skip[i] set.  Writes every peak's height,
 * bound and sample index and returns the count.
 *
 * Near-ties: a decision whose two sides lie within their bounds (which
 * sample tops a peak, whether a value confirms a fall, whether it confirms
 * a rise) is recorded in ties[] as 4 i + type (type 0 top, 1 fall, 2 rise)
 * when ties is not NULL (at most max_ties; *n_ties counts them all).  The
 * decisions whose codes are listed in flips[0 .. n_flips) are taken the
 * other way, so that a caller can see whether they matter. */
static int is_flipped(const int *flips, int n_flips, int code) {
  for (int i = 0; i < n_flips; ++i)
    if (flips[i] == code) return 1;
  return 0;
}

static int detect_peaks(const double *v, const double *e, const int *kk,
                        const char *skip, int n, double r, double *ph,
                        double *pe, int *pk, const int *flips, int n_flips,
                        int *ties, int max_ties, int *n_ties) {
  int count = 0, rising_seen = 0, have = 0, kmx = 0;
  double mn = 0.0, emn = 0.0, mx = 0.0, emx = 0.0;
  if (n_ties) *n_ties = 0;
#define NEAR_TIE(type, cond)                                   \
  do {                                                         \
    if (cond) {                                                \
      if (ties && n_ties) {                                    \
        if (*n_ties < max_ties) ties[*n_ties] = 4 * i + (type); \
        ++*n_ties;                                             \
      }                                                        \
    }                                                          \
  } while (0)
  for (int i = 0; i < n; ++i) {
    if (skip && skip[i]) continue;
    double x = v[i], ex = e[i];
    if (!have) { /* first sample: the running minimum starts here */
      have = 1;
      mn = x;
      emn = ex;
      continue;
    }
    if (rising_seen) { /* looking for the top of a rise */
      int up = x > mx, fall = mx > r * x;
      NEAR_TIE(0, fabs(x - mx) <= ex + emx);
      NEAR_TIE(1, fabs(mx - r * x) <= emx + r * ex);
      if (is_flipped(flips, n_flips, 4 * i + 0)) up = !up;
      if (is_flipped(flips, n_flips, 4 * i + 1)) fall = !fall;
      if (up) {
        mx = x;
        emx = ex;
        kmx = kk[i];
      } else if (fall) { /* the fall confirms the peak at kmx */
        ph[count] = mx;
        pe[count] = emx;
        pk[count] = kmx;
        ++count;
        rising_seen = 0;
        mn = x;
        emn = ex;
      }
    } else { /* looking for a rise */
      int rise = x > r * mn;
      NEAR_TIE(2, fabs(x - r * mn) <= ex + r * emn);
      if (is_flipped(flips, n_flips, 4 * i + 2)) rise = !rise;
      if (x < mn && !rise) {
        /* a near-tie with the old minimum widens the new one's bound by
         * their difference (an FP32 evaluation may keep either) */
        double d = mn - x, eo = emn;
        mn = x;
        emn = (d <= ex + eo) ? fmax(ex, eo) + d : ex;
      } else if (rise) {
        rising_seen = 1;
        mx = x;
        emx = ex;
        kmx = kk[i];
      } else if (x - mn <= ex + emn) {
        emn = fmax(ex, emn) + (x - mn);
      }
    }
  }
#undef NEAR_TIE
  return count;
}

/* the max_peaks highest of n peaks (ties: the earlier), then in increasing
 * tau: indices into the peak arrays in sel[0 .. return value) */
static int keep_highest(const double *ph, const double *pe, const int *pk,
                        int n, int P, int *sel, int *unsure) {
  for (int i = 0; i < n; ++i) sel[i] = i;
  for (int i = 1; i < n; ++i) /* stable insertion sort, highest first */
    for (int j = i; j > 0 && ph[sel[j]] > ph[sel[j - 1]]; --j) {
      int t = sel[j];
      sel[j] = sel[j - 1];
      sel[j - 1] = t;
    }
  int nkept = n < P ? n : P;
  if (n > P && unsure) {
    int a = sel[P - 1], b = sel[P];
    if (fabs(ph[a] - ph[b]) <= pe[a] + pe[b]) *unsure = 1;
  }
  for (int i = 1; i < nkept; ++i)
    for (int j = i; j > 0 && pk[sel[j]] < pk[sel[j - 1]]; --j) {
      int t = sel[j];
      sel[j] = sel[j - 1];
      sel[j - 1] = t;
    }
  return nkept;
}

/* Whether every evaluation within the bounds gives the library (count,
 * kept positions pos[0 .. nkept)): the detector is run with the decisions
 * flips[0 .. n_flips) inverted, and recursively with each later near-tie
 * of that run inverted as well, to a depth of 3 inverted decisions (a
 * plateau of up to four samples that FP32 rounding makes wiggle).  More
 * than *budget runs in all counts as undetermined. */
#define PEAK_FLIP_DEPTH 3
static int same_library(const double *v, const double *e, const int *kk,
                        const char *skip, int n, double r, int P, double h,
                        double shift, int *flips, int n_flips, int count,
                        int nkept, const double *pos, int *budget) {
  if (--*budget < 0) return 0;
  int cap = n + 2;
  double *ph = (double *)malloc((size_t)cap * sizeof(double));
  double *pe = (double *)malloc((size_t)cap * sizeof(double));
  int *pk = (int *)malloc((size_t)cap * sizeof(int));
  int *ksel = (int *)malloc((size_t)cap * sizeof(int));
  int max_ties = 4 * n + 4, n_ties = 0;
  int *ties = (int *)malloc((size_t)max_ties * sizeof(int));
  int c2 = detect_peaks(v, e, kk, skip, n, r, ph, pe, pk, flips, n_flips,
                        ties, max_ties, &n_ties);
  int n2 = keep_highest(ph, pe, pk, c2, P, ksel, NULL);
  int same = (c2 == count && n2 == nkept);
  for (int m = 0; same && m < n2; ++m)
    if ((double)pk[ksel[m]] * h - shift != pos[m]) same = 0;
  if (same && n_flips < PEAK_FLIP_DEPTH) {
    int last = n_flips > 0 ? flips[n_flips - 1] : -1;
    for (int t = 0; t < n_ties && t < max_ties && same; ++t) {
      if (ties[t] <= last) continue; /* earlier ones: other branches */
      flips[n_flips] = ties[t];
      same = same_library(v, e, kk, skip, n, r, P, h, shift, flips,
                          n_flips + 1, count, nkept, pos, budget);
    }
    if (n_ties > max_ties) same = 0;
  }
  free(ph);
  free(pe);
  free(pk);
  free(ksel);
  free(ties);
  return same;
}

int orc_line_peaks(const float *A, int npix, double L, double u, double c,
                   double s, double shift, int sub, double delta,
                   int max_peaks, double *pos, double *height, double *herr,
                   int *uncertain) {
  const double f32 = 5.9604644775390625e-8; /* 2^-24 */
  double dlt = (2.0 * L) / (double)npix;
  double h = dlt / (double)sub;
  double r = 1.0 + delta;
  int K = sub * npix;
  int P = max_peaks > 0 ? max_peaks : 1;
  int cap = 2 * K + 1;
  /* the profile: every sample inside the map, plus those whose inside test
   * an FP32 evaluation could decide either way (amb = 1; then v, e are
   * those of the clamped lookup, which is what such a sample reads) */
  double *v = (double *)malloc((size_t)cap * sizeof(double));
  double *e = (double *)malloc((size_t)cap * sizeof(double));
  int *kk = (int *)malloc((size_t)cap * sizeof(int));
  char *amb = (char *)malloc((size_t)cap);
  char *inc = (char *)malloc((size_t)cap);
  int n = 0;
  for (int k = -K; k <= K; ++k) {
    double tau = (double)k * h;
    double y1 = tau * c - u * s, y2 = tau * s + u * c;
    /* texel coordinates and the FP32 placement bound */
    double px = (y1 + L) / dlt - 0.5, py = (y2 + L) / dlt - 0.5;
    double atx = fabs(c / dlt * tau), aty = fabs(s / dlt * tau);
    double dpx = 2.0 * f32 * (4.0 * atx + fabs(px - c / dlt * tau) +
                              fabs(px) + 1.0);
    double dpy = 2.0 * f32 * (4.0 * aty + fabs(py - s / dlt * tau) +
                              fabs(py) + 1.0);
    double lo = -0.5, hi = (double)npix - 0.5;
    int inside = fabs(y1) < L && fabs(y2) < L;
    int nearx = fabs(px - lo) <= dpx || fabs(px - hi) <= dpx;
    int neary = fabs(py - lo) <= dpy || fabs(py - hi) <= dpy;
    int outx = px < lo - dpx || px > hi + dpx;
    int outy = py < lo - dpy || py > hi + dpy;
    int ambiguous = (nearx && !outy) || (neary && !outx);
    if (!inside && !ambiguous) continue;
    double qx = px < 0.0 ? 0.0 : (px > npix - 1.0 ? npix - 1.0 : px);
    double qy = py < 0.0 ? 0.0 : (py > npix - 1.0 ? npix - 1.0 : py);
    double gx, gy, amax;
    cell_slopes(A, npix, qx, qy, dpx, dpy, &gx, &gy, &amax);
    v[n] = bil_clamped(A, npix, L, y1, y2);
    e[n] = gx * dpx + gy * dpy + 16.0 * f32 * amax;
    kk[n] = k;
    amb[n] = (char)ambiguous;
    inc[n] = (char)!inside; /* skip mask of the definition's profile */
    ++n;
  }
  double *ph = (double *)malloc((size_t)(cap + 1) * sizeof(double));
  double *pe = (double *)malloc((size_t)(cap + 1) * sizeof(double));
  int *pk = (int *)malloc((size_t)(cap + 1) * sizeof(int));
  int *sel = (int *)malloc((size_t)(cap + 1) * sizeof(int));
  int unsure = 0;
  int count = detect_peaks(v, e, kk, inc, n, r, ph, pe, pk, NULL, 0, NULL,
                           0, NULL);
  int nkept = keep_highest(ph, pe, pk, count, P, sel, &unsure);
  for (int m = 0; m < max_peaks; ++m) {
    if (m < nkept) {
      pos[m] = (double)pk[sel[m]] * h - shift;
      height[m] = ph[sel[m]];
      if (herr) herr[m] = pe[sel[m]];
    } else {
      pos[m] = NAN;
      height[m] = NAN;
      if (herr) herr[m] = NAN;
    }
  }
  /* The library is determined when no combination of up to
   * PEAK_FLIP_DEPTH near-tie decisions taken the other way changes the
   * count or the kept positions, for every way an FP32 evaluation could
   * classify the samples at the ends of the run whose inside test is
   * within its bounds (variants: the ambiguous samples of each end in or
   * out). */
  int flips[PEAK_FLIP_DEPTH + 1];
  int budget = 4096;
  int any_amb = 0;
  for (int i = 0; i < n; ++i) any_amb |= amb[i];
  for (int var = 0; var < (any_amb ? 4 : 1) && !unsure; ++var) {
    if (var > 0)
      for (int i = 0; i < n; ++i)
        inc[i] = amb[i] ? (char)!((i < n / 2) ? (var & 1)
                                               : ((var >> 1) & 1))
                        : 0;
    if (!same_library(v, e, kk, inc, n, r, P, h, shift, flips, 0, count,
                      nkept, pos, &budget))
      unsure = 1;
  }
  if (uncertain) *uncertain = unsure;
  free(v);
  free(e);
  free(kk);
  free(amb);
  free(inc);
  free(ph);
  free(pe);
  free(pk);
  free(sel);
  return count;
}

/* Given magnifications A[i] at the epochs, the weighted least-squares
 * (Fs, Fb) of F = Fs A + Fb (normal equations, closed form) and the chi^2
 * as the sum of per-point contributions w (F - Fs A - Fb)^2.
 * Degenerate rule: if det <= 1e-12 S_AA S_1 (A constant along the track)
 * then Fs = 0, Fb = S_F / S_1 and flag = 1. */
double orc_fit_A(const double *A, const double *F, const double *w, long n,
                 double *Fs, double *Fb, int *flag) {
  double S1 = 0, SA = 0, SAA = 0, SF = 0, SAF = 0;
  for (long i = 0; i < n; ++i) {
    S1 += w[i];
    SA += w[i] * A[i];
    SAA += w[i] * A[i] * A[i];
    SF += w[i] * F[i];
    SAF += w[i] * A[i] * F[i];
  }
  double det = SAA * S1 - SA * SA;
  double fs, fb;
  int fl = 0;
  if (!(det > 1e-12 * SAA * S1)) {
    fs = 0.0;
    fb = SF / S1;
    fl = 1;
  } else {
    fs = (S1 * SAF - SA * SF) / det;
    fb = (SAA * SF - SA * SAF) / det;
  }
  double chi2 = 0.0;
  for (long i = 0; i < n; ++i) {
    double r = F[i] - fs * A[i] - fb;
    chi2 += w[i] * r * r;
  }
  if (Fs) *Fs = fs;
  if (Fb) *Fb = fb;
  if (flag) *flag = fl;
  return chi2;
}

/* chi^2 (and the fitted Fs, Fb) of one trajectory at arbitrary
 * (t0, tE, u0, alpha): magnifications from the map (mode 0) or from the
 * point-source polynomial (mode 1), then the linear fit of Eq. 6. */
double orc_chi2_theta(const float *Amap, int npix, double L, double s,
                      double q, int mode, const double *t, const double *F,
                      const double *w, long n, double t0, double tE, double u0,
                      double alpha, double *Fs, double *Fb) {
  double *A = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  for (long i = 0; i < n; ++i) {
    double y1, y2;
    orc_traj_point(t[i], t0, tE, u0, alpha, &y1, &y2);
    A[i] = (mode == 0) ? orc_map_A(Amap, npix, L, y1, y2)
                       : orc_mag_point(s, q, y1, y2, NULL);
  }
  int fl;
  double c = orc_fit_A(A, F, w, n, Fs, Fb, &fl);
  free(A);
  return c;
}

/* chi^2 of the polynomial point-source light curve of one trajectory and
 * its gradient in theta = (t0, tE, u0, alpha).  Fs and Fb are the least-
 * squares solution (Eq. 5-6), so the partial derivatives of chi^2 in them
 * vanish there and, with r_i = F_i - Fs A_i - Fb,
 *   d chi^2 / d theta = sum_i -2 w_i r_i Fs (dA/dy1 dy1/dtheta
 *                                            + dA/dy2 dy2/dtheta),
 * where tau = (t - t0)/tE, y1 = tau cos(alpha) - u0 sin(alpha),
 * y2 = tau sin(alpha) + u0 cos(alpha) (§4.2). */
double orc_chi2_grad_poly(double s, double q, const double *t,
                          const double *F, const double *w, long n,
                          double t0, double tE, double u0, double alpha,
                          double *grad, double *Fs, double *Fb) {
  size_t m = (size_t)(n > 0 ? n : 1);
  double *A = (double *)malloc(m * sizeof(double));
  double *g1 = (double *)malloc(m * sizeof(double));
  double *g2 = (double *)malloc(m * sizeof(double));
  double ca = cos(alpha), sa = sin(alpha);
  for (long i = 0; i < n; ++i) {
    double y1, y2, g[2];
    orc_traj_point(t[i], t0, tE, u0, alpha, &y1, &y2);
    A[i] = orc_mag_point_grad(s, q, y1, y2, g);
    g1[i] = g[0];
    g2[i] = g[1];
  }
  int fl;
  double c = orc_fit_A(A, F, w, n, Fs, Fb, &fl);
  for (int k = 0; k < 4; ++k) grad[k] = 0.0;
  for (long i = 0; i < n; ++i) {
    double tau = (t[i] - t0) / tE;
    double y1 = tau * ca - u0 * sa, y2 = tau * sa + u0 * ca;
    double r = F[i] - *Fs * A[i] - *Fb;
    double f = -2.0 * w[i] * r * *Fs;
    /* d tau/d t0 = -1/tE, d tau/d tE = -tau/tE */
    double dtau = g1[i] * ca + g2[i] * sa; /* dA/dtau */
    grad[0] += f * dtau * (-1.0 / tE);
    grad[1] += f * dtau * (-tau / tE);
    grad[2] += f * (g1[i] * (-sa) + g2[i] * ca);
    grad[3] += f * (g1[i] * (-y2) + g2[i] * y1);
  }
  free(A);
  free(g1);
  free(g2);
  return c;
}

/* Grid axis values: linear lo + (hi-lo) i/(n-1), or logarithmic
 * lo (hi/lo)^(i/(n-1)); n == 1 gives lo. */
void orc_axis(double lo, double hi, int n, int logsp, double *out) {
  for (int i = 0; i < n; ++i) {
    double f = (n > 1) ? (double)i / (double)(n - 1) : 0.0;
    out[i] = logsp ? exp(log(lo) + (log(hi) - log(lo)) * f) : lo + (hi - lo) * f;
  }
}

/* Trajectory index = ((i_u0 * n_alpha + i_alpha) * n_t0 + i_t0) * n_tE +
 * i_tE; alpha_k = 2 pi k / n_alpha. */
void orc_traj_params(const double *u0v, int nu, int na, const double *t0v,
                     int nt0, const double *tEv, int ntE, long long idx,
                     double *t0, double *tE, double *u0, double *alpha) {
  long long itE = idx % ntE;
  long long r = idx / ntE;
  long long it0 = r % nt0;
  r /= nt0;
  long long ia = r % na;
  long long iu = r / na;
  (void)nu;
  *t0 = t0v[it0];
  *tE = tEv[itE];
  *u0 = u0v[iu];
  *alpha = 2.0 * M_PI * (double)ia / (double)na;
}

/* Dense chi^2 over the whole (u0, alpha, t0, tE) grid on a map (mode 0) or
 * on the point-source polynomial magnification (mode 1, s and q used).
 * chi2/Fs/Fb/flag receive one entry per trajectory index. */
int orc_grid_chi2(const float *Amap, int npix, double L, double s, double q,
                  int mode, const double *t, const double *F, const double *w,
                  long n, const double *u0v, int nu, int na, const double *t0v,
                  int nt0, const double *tEv, int ntE, long long first,
                  long long count, double *chi2, double *Fs, double *Fb,
                  int *flag, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  long long total = (long long)nu * na * nt0 * ntE;
  if (first < 0 || first + count > total) return -1;
  int bad = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads) reduction(| : bad)
#endif
  {
    double *A = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
    for (long long k = 0; k < count; ++k) {
      double t0, tE, u0, al;
      orc_traj_params(u0v, nu, na, t0v, nt0, tEv, ntE, first + k, &t0, &tE,
                      &u0, &al);
      for (long i = 0; i < n; ++i) {
        double y1, y2;
        orc_traj_point(t[i], t0, tE, u0, al, &y1, &y2);
        if (mode == 0)
          A[i] = orc_map_A(Amap, npix, L, y1, y2);
        else
          A[i] = orc_mag_point(s, q, y1, y2, NULL);
      }
      double fs, fb;
      int fl;
      chi2[k] = orc_fit_A(A, F, w, n, &fs, &fb, &fl);
      if (Fs) Fs[k] = fs;
      if (Fb) Fb[k] = fb;
      if (flag) flag[k] = fl;
      if (!isfinite(chi2[k])) bad = 1;
    }
    free(A);
  }
  return bad ? 1 : 0;
}

/* ------------------------------------------------------------------ */
/* Seeds: the K best trajectories (§4.4) by a full sort on (chi^2, idx)  */
/* ------------------------------------------------------------------ */

typedef struct {
  double c;
  long long i;
} orc_key;

static int cmp_key(const void *a, const void *b) {
  const orc_key *x = (const orc_key *)a, *y = (const orc_key *)b;
  if (x->c < y->c) return -1;
  if (x->c > y->c) return 1;
  return (x->i < y->i) ? -1 : (x->i > y->i);
}

/* idx_out receives the k smallest (chi2[j], first + j) in ascending order. */
int orc_topk(const double *chi2, long long count, long long first, int k,
             long long *idx_out, double *chi2_out) {
  orc_key *keys = (orc_key *)malloc((size_t)count * sizeof(orc_key));
  if (!keys) return -1;
  for (long long j = 0; j < count; ++j) {
    keys[j].c = chi2[j];
    keys[j].i = first + j;
  }
  qsort(keys, (size_t)count, sizeof(orc_key), cmp_key);
  int m = (k < count) ? k : (int)count;
  for (int j = 0; j < m; ++j) {
    idx_out[j] = keys[j].i;
    chi2_out[j] = keys[j].c;
  }
  free(keys);
  return m;
}
