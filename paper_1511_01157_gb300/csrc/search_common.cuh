// Device functions shared by the search, fit-fill and adjoint kernels: the
// per-trajectory constants, the map lookup, the two epoch sweeps and the
// 2x2 solve.  Every kernel that reports a chi^2 uses these same functions,
// so their results agree to the last bit for the same trajectory.
//
// The method (McDougall & Albrow 2015, §4.2): bilinear interpolation of the
// magnification map along a straight trajectory, the linear flux model
// F = Fs A + Fb (Eq. 5-6) and chi^2 as the sum of per-point contributions.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"

namespace morse {
namespace dev {

// Inside-map epoch loops are unrolled twice by default (a source file may
// set MORSE_UNROLL first): the code must stay within the instruction cache
// (before the trajectory pairs were packed, unroll 4 made the search 33 %
// slower; k_search.cu now sets 4).
#ifndef MORSE_UNROLL
#define MORSE_UNROLL 2
#endif
// the FP16-table kernels keep two (their band builds add code; four made
// the FP16 sweep 5 % slower)
#ifndef MORSE_UNROLL_H
#define MORSE_UNROLL_H 2
#endif
constexpr int kUnroll = MORSE_UNROLL;     // inside-map epoch loop
constexpr int kUnrollH = MORSE_UNROLL_H;  // the same, FP16 tables

constexpr unsigned kFull = 0xffffffffu;

// Per-trajectory constants.
struct TrajC {
  float ax, bx, ay, by;  // centred pixel coordinates v = a t + b
  float kt, bt, u02;     // tau = kt t + bt; u0^2
  int e_in, e_out;       // epochs [e_in, e_out) lie inside the map
};

// The epochs of one event: a block of n float4 slots (so that it is copied
// to shared memory in 16-byte pieces) holding, in structure-of-arrays
// order, tw[n] = (t - t_ref, w), wf[n] = w (F - F_ref) and fc[n] = F - F_ref.
// A warp reading 32 consecutive epochs of a sweep takes two shared-memory
// wavefronts for (t, w) and one for w Fc or Fc: three, where one float4
// per epoch takes four.
struct Epochs {
  const float2 *tw;
  const float *wf, *fc;
};

__device__ __forceinline__ Epochs epochs_at(const float4 *blk, int n) {
  Epochs E;
  E.tw = reinterpret_cast<const float2 *>(blk);
  E.wf = reinterpret_cast<const float *>(E.tw + n);
  E.fc = E.wf + n;
  return E;
}

__device__ __forceinline__ bool key_less(const Entry &a, const Entry &b) {
  return a.chi2 < b.chi2 || (a.chi2 == b.chi2 && a.idx < b.idx);
}
__device__ __forceinline__ bool key_less(double ca, long long ia, double cb,
                                         long long ib) {
  return ca < cb || (ca == cb && ia < ib);
}

// First epoch index with t > x (strict) or t >= x (!strict), t ascending.
// The FP32 epoch times are compared with x rounded to FP32 downwards
// (strict) or upwards: no FP32 value lies strictly between x and that
// rounding, so t > x <=> t > RD(x) and t >= x <=> t >= RU(x) exactly, and
// the search needs no FP64 compares.
__device__ __forceinline__ int epoch_search(const Epochs &ep, int n, double x,
                                            bool strict) {
  const float xf = strict ? __double2float_rd(x) : __double2float_ru(x);
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const float t = ep.tw[mid].x;
    const bool right = strict ? (t > xf) : (t >= xf);
    if (right)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// The tau interval (lo, hi) in which the line of (u0, alpha) is inside the
// map, |y1| < L and |y2| < L (slab intersection; lo >= hi when the line
// misses the map).  It depends on the line only, so the grid searches read
// it from a table made once per call (k_slab).
__device__ __forceinline__ void slab_tau(double L, double u, double c,
                                         double s, double &lo_out,
                                         double &hi_out) {
  double lo = -CUDART_INF, hi = CUDART_INF;
  const double us = u * s, uc = u * c;
  if (c != 0.0) {
    const double a0 = (-L + us) / c, a1 = (L + us) / c;
    lo = fmax(lo, fmin(a0, a1));
    hi = fmin(hi, fmax(a0, a1));
  } else if (!(fabs(us) < L)) {
    hi = lo;
  }
  if (s != 0.0) {
    const double b0 = (-L - uc) / s, b1 = (L - uc) / s;
    lo = fmax(lo, fmin(b0, b1));
    hi = fmin(hi, fmax(b0, b1));
  } else if (!(fabs(uc) < L)) {
    hi = lo;
  }
  lo_out = lo;
  hi_out = hi;
}

// Constants of trajectory j.  The kernel works in centred pixel coordinates
// v = (y + L)/Delta - 1/2 - floor(npix/2) = y/Delta + coff (coff = -1/2 for
// even npix, 0 for odd): texel i (from 0 at the map edge) is centred at
// v = i - floor(npix/2), and the map centre, where the caustics of close and
// resonant lenses lie, has the finest FP32 resolution.  With
// y1 = tau cos(alpha) - u0 sin(alpha), y2 = tau sin(alpha) + u0 cos(alpha)
// and tau = (t - t0)/tE the coordinates are v = a t + b.  The track is
// inside the map (|y1| < L and |y2| < L) for tau in (tau_lo, tau_hi), i.e.
// for the epochs [e_in, e_out).
__device__ __forceinline__ TrajC make_traj(const SearchParams &P,
                                           const Epochs &ep, double u,
                                           double c, double s, double t0,
                                           double k, double tE, double tlo,
                                           double thi) {
  // u = u0, (c, s) = (cos, sin) alpha, t0 relative to t_ref,
  // k = 1/(tE Delta), (tlo, thi) = the line's tau interval in the map
  const double ax = __dmul_rn(c, k), ay = __dmul_rn(s, k);
  const double cx = __dadd_rn(__dmul_rn(-__dmul_rn(u, s), P.invD), P.coff);
  const double cy = __dadd_rn(__dmul_rn(__dmul_rn(u, c), P.invD), P.coff);
  const double kt = __dmul_rn(k, P.dlt);  // 1/tE
  TrajC o;
  o.ax = __double2float_rn(ax);
  o.ay = __double2float_rn(ay);
  o.bx = __double2float_rn(__dsub_rn(cx, __dmul_rn(t0, ax)));
  o.by = __double2float_rn(__dsub_rn(cy, __dmul_rn(t0, ay)));
  o.kt = __double2float_rn(kt);
  o.bt = __double2float_rn(-__dmul_rn(t0, kt));
  o.u02 = __double2float_rn(__dmul_rn(u, u));
  if (tlo < thi) {
    o.e_in = epoch_search(ep, P.n_ep, t0 + tlo * tE, true);
    o.e_out = epoch_search(ep, P.n_ep, t0 + thi * tE, false);
    if (o.e_out < o.e_in) o.e_out = o.e_in;
  } else {
    o.e_in = P.n_ep;
    o.e_out = P.n_ep;
  }
  return o;
}

// constants of grid trajectory j from the device tables
__device__ __forceinline__ TrajC traj_consts(const SearchParams &P,
                                             const Epochs &ep, long long j) {
  long long r = j;
  const int itE = (int)(r % P.n_tE);
  r /= P.n_tE;
  const int it0 = (int)(r % P.n_t0);
  r /= P.n_t0;
  const int ia = (int)(r % P.n_alpha);
  const int iu = (int)(r / P.n_alpha);
  const double2 sl = P.slab[iu * P.n_alpha + ia];
  const double tE = P.tEv[itE];
  if (P.lu) {  // line grid: t0 of the closest approach to the reference point
    if (P.ltE) {  // tE of the line (Eq. 8)
      const double tl = P.ltE[iu];
      return make_traj(P, ep, P.lu[iu], P.lc[iu], P.ls[iu],
                       P.t0rel[it0] - P.lsh[iu] * tl, 1.0 / (tl * P.dlt), tl,
                       sl.x, sl.y);
    }
    return make_traj(P, ep, P.lu[iu], P.lc[iu], P.ls[iu],
                     P.t0rel[it0] - P.lsh[iu] * tE, P.invtEd[itE], tE, sl.x,
                     sl.y);
  }
  return make_traj(P, ep, P.u0v[iu], P.ca[ia], P.sa[ia], P.t0rel[it0],
                   P.invtEd[itE], tE, sl.x, sl.y);
}

__device__ __forceinline__ TrajC shfl_traj(const TrajC &m, int k) {
  TrajC c;
  c.ax = __shfl_sync(kFull, m.ax, k);
  c.bx = __shfl_sync(kFull, m.bx, k);
  c.ay = __shfl_sync(kFull, m.ay, k);
  c.by = __shfl_sync(kFull, m.by, k);
  c.kt = __shfl_sync(kFull, m.kt, k);
  c.bt = __shfl_sync(kFull, m.bt, k);
  c.u02 = __shfl_sync(kFull, m.u02, k);
  c.e_in = __shfl_sync(kFull, m.e_in, k);
  c.e_out = __shfl_sync(kFull, m.e_out, k);
  return c;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// single-lens magnification from u^2 (outside the map)
__device__ __forceinline__ float pspl_u2(float u2) {
  return __fmul_rn(__fadd_rn(u2, 2.f),
                   rsqrt_approx(__fmul_rn(u2, __fadd_rn(u2, 4.f))));
}

// Quad index and bilinear fractions of centred coordinates (vx, vy) inside
// the map.  Inside means vlo < v < vhi, i.e. floor(v) from -half - 1 to
// npix - half - 1: the cell whose lower corner is texel floor(v) + half,
// stored at quad (floor(v) + half + 1) in each axis, and the cells of the
// edge repeat the edge texels, so no coordinate is clamped.
struct TexPos {
  unsigned idx;
  float fx, fy;
};

__device__ __forceinline__ bool tex_pos(const SearchParams &P, float vx,
                                        float vy, TexPos &o) {
  // floor: adding 1.5 * 2^23 rounding down leaves floor(v) in the low
  // mantissa bits; the fraction v - floor(v) is exact
  const float tx = __fadd_rd(vx, 12582912.f), ty = __fadd_rd(vy, 12582912.f);
  o.fx = __fsub_rn(vx, __fsub_rn(tx, 12582912.f));
  o.fy = __fsub_rn(vy, __fsub_rn(ty, 12582912.f));
  // quad index (iy + 1) * qpitch + (ix + 1) with i = floor(v) + half,
  // folded into one multiply-add on the raw bit patterns (mod 2^32, exact
  // because the index is in [0, (npix + 1) * qpitch))
  const unsigned bx = (unsigned)__float_as_int(tx);
  const unsigned by = (unsigned)__float_as_int(ty);
  if (kTileW == 1 && kTileH == 1) {
    o.idx = by * (unsigned)P.qpitch + bx + P.qidx0;
  } else {
    // cell (c, r) = (floor(v) + half + 1) per axis, then the tile index
    const unsigned c = bx + (unsigned)(P.half + 1 - 0x4B400000);
    const unsigned r = by + (unsigned)(P.half + 1 - 0x4B400000);
    o.idx = ((((r >> kTileLH) * ((unsigned)P.qpitch >> kTileLW) +
               (c >> kTileLW))
              << (kTileLW + kTileLH)) |
             ((r & (kTileH - 1)) << kTileLW) | (c & (kTileW - 1)));
  }
#ifdef MORSE_CHECK_BOUNDS
  // checked build: record an out-of-range cell and skip the access
  const int cx = (int)(bx - 0x4B400000u) + P.half + 1;
  const int cy = (int)(by - 0x4B400000u) + P.half + 1;
  if ((unsigned)cx > (unsigned)P.npix || (unsigned)cy > (unsigned)P.npix) {
    if (P.err) atomicOr(P.err, 2u);
    return false;
  }
#endif
  return true;
}

// Bilinear A - 1 at centred coordinates inside the map.  The quads store,
// with m = A - 1, (m00, m10 - m00, m01 - m00, (m11 - m01) - (m10 - m00))
// of the cell, rounded in FP32 when the table was built: the first row at
// fx, the difference of the rows at fx and the value at fy are one FMA
// each.  Below
// the first texel centre the edge cell repeats the edge values (the
// clamping rule of the lookup); above the last centre likewise.  The
// bounds-checked build verifies the index range.
__device__ __forceinline__ float bilinear_m1(const SearchParams &P, float vx,
                                             float vy) {
  TexPos t;
  if (!tex_pos(P, vx, vy, t)) return 0.f;
  const float4 q = __ldg(&P.quad[t.idx]);
  const float r0 = __fmaf_rn(t.fx, q.y, q.x);
  const float dr = __fmaf_rn(t.fx, q.w, q.z);
  return __fmaf_rn(t.fy, dr, r0);
}

// Lanes own epochs by index mod 32 in every range, so a lane always sums
// its terms in ascending epoch order whatever the ranges are: the sums of a
// trajectory do not depend on how its epoch axis is cut into segments (the
// search pairs trajectories, the fit fill does not; both get the same
// rounding).
__device__ __forceinline__ int lane_start(int e0, int lane) {
  return e0 + ((lane - e0) & 31);
}

struct Acc {
  float a, b, d;  // S_A, S_AA, S_AF partial sums of one lane
};

__device__ __forceinline__ void acc_add(Acc &s, float w, float wf, float Ac) {
  const float wAc = __fmul_rn(w, Ac);
  s.a = __fadd_rn(s.a, wAc);
  s.b = __fmaf_rn(wAc, Ac, s.b);
  s.d = __fmaf_rn(wf, Ac, s.d);
}

// 10^x for a decoded FP16 log10 texel: one hardware base-2 exponential
// of x log2(10) (relative error a few FP32 ulps, far below the half
// quantisation of x)
__device__ __forceinline__ float exp10_texel(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x * 3.32192809488736234787f));
  return y;
}

// FP16 map: the four log10 texels of the quad are decoded to A = 10^x in
// FP32 and interpolated in A, the same bilinear as the FP32 map; A - 1 is
// returned as there.
__device__ __forceinline__ float bilinear_h_m1(const SearchParams &P,
                                               float vx, float vy) {
  TexPos t;
  if (!tex_pos(P, vx, vy, t)) return 0.f;
  const uint2 q = __ldg(&P.quadh[t.idx]);
  const float2 lo = __half22float2(
      __halves2half2(__ushort_as_half((unsigned short)(q.x & 0xffffu)),
                     __ushort_as_half((unsigned short)(q.x >> 16))));
  const float2 hi = __half22float2(
      __halves2half2(__ushort_as_half((unsigned short)(q.y & 0xffffu)),
                     __ushort_as_half((unsigned short)(q.y >> 16))));
  const float a00 = exp10_texel(lo.x), a10 = exp10_texel(lo.y);
  const float a01 = exp10_texel(hi.x), a11 = exp10_texel(hi.y);
  const float d0 = __fsub_rn(a10, a00), d1 = __fsub_rn(a11, a01);
  const float r0 = __fmaf_rn(t.fx, d0, a00);
  const float dr = __fmaf_rn(t.fx, __fsub_rn(d1, d0), __fsub_rn(a01, a00));
  return __fsub_rn(__fmaf_rn(t.fy, dr, r0), 1.f);
}

// An FP16 cell decoded as the FP16 bilinear reads it: with the texels
// a = 10^x, (a00, a10 - a00, a01 - a00, (a11 - a01) - (a10 - a00)).
__device__ __forceinline__ float4 band_cell_h(const uint2 q) {
  const float2 lo = __half22float2(
      __halves2half2(__ushort_as_half((unsigned short)(q.x & 0xffffu)),
                     __ushort_as_half((unsigned short)(q.x >> 16))));
  const float2 hi = __half22float2(
      __halves2half2(__ushort_as_half((unsigned short)(q.y & 0xffffu)),
                     __ushort_as_half((unsigned short)(q.y >> 16))));
  const float a00 = exp10_texel(lo.x), a10 = exp10_texel(lo.y);
  const float a01 = exp10_texel(hi.x), a11 = exp10_texel(hi.y);
  const float d0 = __fsub_rn(a10, a00), d1 = __fsub_rn(a11, a01);
  return make_float4(a00, d0, __fsub_rn(a01, a00), __fsub_rn(d1, d0));
}

// Band table of one line of the line-aligned pass, in shared memory.  For
// a line closer to the first axis (|cos alpha| >= |sin alpha|, TB = 1) the
// table holds, for every cell column X, the cells of rows row0(X) ..
// row0(X) + 3 around the line, at key X + S ((Y + C) & 3) with S =
// band_stride(npix) and C the floor bits' offset: four consecutive rows
// have distinct low bits, so the key is the cell's own, and neighbouring
// columns are neighbouring entries (a warp's lookups along the line fall in
// distinct bank groups, also across a row step).  The line meets at most
// rows floor(yc - 1/2) ..
// floor(yc + 1/2) of a column (|slope| <= 1, yc its height at the column
// centre), and row0 = floor(yc) - 1 takes them with 1/4 texel to spare on
// each side, far beyond the FP32 rounding of a trajectory's position
// (below 1e-2 texel for |a t| < 1e5 texels, which the host checks).  So a
// band lookup reads the same 16 bytes as the global table, from shared
// memory.  TB = 2: rows and columns swapped.  For the FP16 log10 table
// (H) the band holds the decoded texels in the same pre-differenced form,
// (a00, a10 - a00, a01, a11 - a01), so the four exponentials of a lookup
// are taken once per cell when the band is built, and the lookup is the
// FP16 bilinear's own arithmetic.
// The band-table lookup from the floor sums t = RD(v + 1.5 2^23) and the
// fractions f = v - floor(v) of both axes; (vx, vy) only serve the
// bounds-checked build.
template <int TB, bool H>
__device__ __forceinline__ float tab_cell_m1(const SearchParams &P,
                                             const float4 *tab, float tx,
                                             float ty, float fx, float fy,
                                             float vx, float vy) {
  const unsigned bx = (unsigned)__float_as_int(tx);
  const unsigned by = (unsigned)__float_as_int(ty);
  const unsigned S = (unsigned)band_stride(P.npix);
  const unsigned key = TB == 1 ? (bx + P.tab_c) + S * (by & 3u)
                               : (by + P.tab_c) + S * (bx & 3u);
#ifdef MORSE_CHECK_BOUNDS
  // checked build: the band entry must be the global table's cell
  TexPos t;
  if (!tex_pos(P, vx, vy, t)) return 0.f;
  if (key >= (unsigned)P.tab_n) {
    if (P.err) atomicOr(P.err, 4u);
    return 0.f;
  }
  {
    const float4 g = H ? band_cell_h(P.quadh[t.idx]) : __ldg(&P.quad[t.idx]);
    const float4 b = tab[key];
    if (g.x != b.x || g.y != b.y || g.z != b.z || g.w != b.w)
      if (P.err) atomicOr(P.err, 4u);
  }
#endif
  const float4 q = tab[key];
  const float r0 = __fmaf_rn(fx, q.y, q.x);
  const float dr = __fmaf_rn(fx, q.w, q.z);
  return __fmaf_rn(fy, dr, r0);
}

template <int TB, bool H>
__device__ __forceinline__ float bilinear_tab_m1(const SearchParams &P,
                                                 const float4 *tab, float vx,
                                                 float vy) {
  const float tx = __fadd_rd(vx, 12582912.f), ty = __fadd_rd(vy, 12582912.f);
  const float fx = __fsub_rn(vx, __fsub_rn(tx, 12582912.f));
  const float fy = __fsub_rn(vy, __fsub_rn(ty, 12582912.f));
  const float a = tab_cell_m1<TB, H>(P, tab, tx, ty, fx, fy, vx, vy);
  return H ? __fsub_rn(a, 1.f) : a;
}

// Fill the band table of the line through the centred point (cx, cy) with
// direction (c, s) (warp-collective); returns TB (1 or 2).
template <bool H>
__device__ inline int build_band(const SearchParams &P, float4 *tab,
                                 double cx, double cy, double c, double s,
                                 int lane) {
  const bool xm = fabs(c) >= fabs(s);
  const int n = P.npix;
  // along the major axis m, the minor coordinate of the line is
  // w(m) = w0 + slope (m - m0)
  const float slope = (float)(xm ? s / c : c / s);
  const float m0 = (float)(xm ? cx : cy), w0 = (float)(xm ? cy : cx);
  const unsigned C = 0x4B400000u - (unsigned)(P.half + 1);
  const float lim = 4.f * (float)n + 8.f;
  for (int M = lane; M <= n; M += 32) {
    const float mc = (float)(M - P.half) - 0.5f;  // centre of cell M
    float wc = __fmaf_rn(slope, mc - m0, w0);
    wc = fminf(fmaxf(wc, -lim), lim);
    const int r0 = (int)floorf(wc) + P.half;  // cell of the centre, less 1
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int W = r0 + d;
      const int Wc = min(max(W, 0), n);
      const unsigned key =
          (unsigned)M + (unsigned)band_stride(n) * (((unsigned)W + C) & 3u);
      const size_t ci = xm ? cell_index(M, Wc, P.qpitch)
                           : cell_index(Wc, M, P.qpitch);
      tab[key] = H ? band_cell_h(P.quadh[ci]) : P.quad[ci];
    }
  }
  return xm ? 1 : 2;
}

// A - 1 at time t inside the map (bilinear) or outside (single lens)
// (H: the FP16 log10 table)
template <bool H, int TB = 0>
__device__ __forceinline__ float mag_in_m1(const SearchParams &P,
                                           const TrajC &c, float t,
                                           const float4 *tab = nullptr) {
  const float vx = __fmaf_rn(c.ax, t, c.bx), vy = __fmaf_rn(c.ay, t, c.by);
  if (TB != 0) return bilinear_tab_m1<TB, H>(P, tab, vx, vy);
  return H ? bilinear_h_m1(P, vx, vy) : bilinear_m1(P, vx, vy);
}
__device__ __forceinline__ float mag_out_m1(const TrajC &c, float t) {
  const float tau = __fmaf_rn(c.kt, t, c.bt);
  return __fsub_rn(pspl_u2(__fmaf_rn(tau, tau, c.u02)), 1.f);
}

template <bool H, bool IN, int TB = 0>
__device__ __forceinline__ void seg1(const SearchParams &P, const Epochs &ep,
                                     const TrajC &c, int lane, int e0, int e1,
                                     Acc &s, const float4 *tab = nullptr) {
#pragma unroll (IN ? (H ? kUnrollH : kUnroll) : 2)
  for (int e = lane_start(e0, lane); e < e1; e += 32) {
    const float2 v = ep.tw[e];
    const float wf = ep.wf[e];
    acc_add(s, v.y, wf,
            IN ? mag_in_m1<H, TB>(P, c, v.x, tab) : mag_out_m1(c, v.x));
  }
}

// Two trajectories side by side in packed FP32 pairs (x: trajectory a,
// y: trajectory b): each packed operation rounds both halves exactly as
// the scalar operation does, so the sums are bit-identical to the scalar
// sweep (seg1, the fit records), with one instruction for both.
struct TrajP {
  float2 ax, bx, ay, by, kt, bt, u02;
};
struct Acc2 {
  float2 a, b, d;  // Acc of trajectory a in .x, of b in .y
};

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// The packed FP32 pair operations (FADD2, FMUL2, FFMA2); each rounds both
// halves as the scalar __fadd_rn, __fmul_rn and __fmaf_rn do.  A
// translation unit that defines MORSE_PK_ASM 1 gets them as inline PTX
// with explicit rounding modes (k_search: 0.8 % faster; k_batch: 8 %
// slower), else as the compiler's __fadd2_rn etc.  One step was measured to
// break the equality in both forms: a packed add of the constant -1 to the
// packed single-lens product gave other bits than the scalar sweep in the
// second half, so that step is taken per half (mag2_out_m1); GPU tests
// check that paired and single sweeps agree bit for bit.
#ifndef MORSE_PK_ASM
#define MORSE_PK_ASM 0
#endif
#if MORSE_PK_ASM
#define MORSE_PK2(OP, a, b)                                             \
  asm("{\n\t.reg .b64 pa, pb, pd;\n\tmov.b64 pa, {%2, %3};\n\t"         \
      "mov.b64 pb, {%4, %5};\n\t" OP " pd, pa, pb;\n\t"                  \
      "mov.b64 {%0, %1}, pd;\n\t}"                                       \
      : "=f"(d.x), "=f"(d.y)                                            \
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y))
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) {
  float2 d;
  MORSE_PK2("add.rn.f32x2", a, b);
  return d;
}
__device__ __forceinline__ float2 pk_add_rd(float2 a, float2 b) {
  float2 d;
  MORSE_PK2("add.rm.f32x2", a, b);
  return d;
}
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b) {
  float2 d;
  MORSE_PK2("mul.rn.f32x2", a, b);
  return d;
}
#undef MORSE_PK2
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 pa, pb, pc, pd;\n\tmov.b64 pa, {%2, %3};\n\t"
      "mov.b64 pb, {%4, %5};\n\tmov.b64 pc, {%6, %7};\n\t"
      "fma.rn.f32x2 pd, pa, pb, pc;\n\tmov.b64 {%0, %1}, pd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
#else
__device__ __forceinline__ float2 pk_add(float2 a, float2 b) {
  return __fadd2_rn(a, b);
}
__device__ __forceinline__ float2 pk_add_rd(float2 a, float2 b) {
  return __fadd2_rd(a, b);
}
__device__ __forceinline__ float2 pk_mul(float2 a, float2 b) {
  return __fmul2_rn(a, b);
}
__device__ __forceinline__ float2 pk_fma(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
#endif

__device__ __forceinline__ TrajP pack_traj(const TrajC &a, const TrajC &b) {
  TrajP p;
  p.ax = make_float2(a.ax, b.ax);
  p.bx = make_float2(a.bx, b.bx);
  p.ay = make_float2(a.ay, b.ay);
  p.by = make_float2(a.by, b.by);
  p.kt = make_float2(a.kt, b.kt);
  p.bt = make_float2(a.bt, b.bt);
  p.u02 = make_float2(a.u02, b.u02);
  return p;
}

// A - 1 of both inside the map: packed coordinates, floor sums and
// fractions (as in bilinear_tab_m1), then one lookup each
template <bool H, int TB>
__device__ __forceinline__ float2 mag2_in_m1(const SearchParams &P,
                                             const TrajP &c, const float2 tt,
                                             const float4 *tab) {
  const float2 vx = pk_fma(c.ax, tt, c.bx);
  const float2 vy = pk_fma(c.ay, tt, c.by);
  if (TB == 0)
    return make_float2(
        H ? bilinear_h_m1(P, vx.x, vy.x) : bilinear_m1(P, vx.x, vy.x),
        H ? bilinear_h_m1(P, vx.y, vy.y) : bilinear_m1(P, vx.y, vy.y));
  const float2 tx = pk_add_rd(vx, f2(12582912.f));
  const float2 ty = pk_add_rd(vy, f2(12582912.f));
  // v - (t - 1.5 2^23): the subtraction as an FMA with -1 (exact product)
  const float2 fx = pk_fma(pk_add(tx, f2(-12582912.f)), f2(-1.f), vx);
  const float2 fy = pk_fma(pk_add(ty, f2(-12582912.f)), f2(-1.f), vy);
  const float2 a =
      make_float2(tab_cell_m1<TB, H>(P, tab, tx.x, ty.x, fx.x, fy.x, vx.x, vy.x),
                  tab_cell_m1<TB, H>(P, tab, tx.y, ty.y, fx.y, fy.y, vx.y, vy.y));
  return H ? make_float2(__fsub_rn(a.x, 1.f), __fsub_rn(a.y, 1.f)) : a;
}

// A - 1 of both outside the map (single lens, as mag_out_m1)
__device__ __forceinline__ float2 mag2_out_m1(const TrajP &c, const float2 tt) {
  const float2 tau = pk_fma(c.kt, tt, c.bt);
  const float2 u2 = pk_fma(tau, tau, c.u02);
  const float2 r = pk_mul(u2, pk_add(u2, f2(4.f)));
  const float2 A = pk_mul(pk_add(u2, f2(2.f)),
                              make_float2(rsqrt_approx(r.x), rsqrt_approx(r.y)));
  // A - 1 per half (not as a packed add: see the pk_ operations)
  return make_float2(__fsub_rn(A.x, 1.f), __fsub_rn(A.y, 1.f));
}

__device__ __forceinline__ void acc2_add(Acc2 &s, float2 w, float2 wf,
                                         float2 Ac) {
  const float2 wAc = pk_mul(w, Ac);
  s.a = pk_add(s.a, wAc);
  s.b = pk_fma(wAc, Ac, s.b);
  s.d = pk_fma(wf, Ac, s.d);
}

// two trajectories over one epoch segment, one epoch load for both
template <bool H, bool INA, bool INB, int TB = 0>
__device__ __forceinline__ void seg2(const SearchParams &P, const Epochs &ep,
                                     const TrajC &ca, const TrajC &cb,
                                     const TrajP &cp, int lane, int e0, int e1,
                                     Acc2 &s, const float4 *tab = nullptr) {
#pragma unroll ((INA || INB) ? (H ? kUnrollH : kUnroll) : 2)
  for (int e = lane_start(e0, lane); e < e1; e += 32) {
    const float2 v = ep.tw[e];
    const float wf = ep.wf[e];
    const float2 tt = f2(v.x);
    float2 Ac;
    if (INA && INB)
      Ac = mag2_in_m1<H, TB>(P, cp, tt, tab);
    else if (!INA && !INB)
      Ac = mag2_out_m1(cp, tt);
    else
      Ac = make_float2(
          INA ? mag_in_m1<H, TB>(P, ca, v.x, tab) : mag_out_m1(ca, v.x),
          INB ? mag_in_m1<H, TB>(P, cb, v.x, tab) : mag_out_m1(cb, v.x));
    acc2_add(s, f2(v.y), f2(wf), Ac);
  }
}

// xor butterfly; lane 0's totals go to every lane
__device__ __forceinline__ Acc acc_reduce(Acc s) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s.a = __fadd_rn(s.a, __shfl_xor_sync(kFull, s.a, o));
    s.b = __fadd_rn(s.b, __shfl_xor_sync(kFull, s.b, o));
    s.d = __fadd_rn(s.d, __shfl_xor_sync(kFull, s.d, o));
  }
  Acc r;
  r.a = __shfl_sync(kFull, s.a, 0);
  r.b = __shfl_sync(kFull, s.b, 0);
  r.d = __shfl_sync(kFull, s.d, 0);
  return r;
}

// Phase 1: FP32 sums of S_A = sum w (A-1), S_AA = sum w (A-1)^2 and
// S_AF = sum w (F-Fref)(A-1) over the epochs before, inside and after the
// map, reduced across the warp.
template <bool H, int TB = 0>
__device__ __forceinline__ Acc phase1(const SearchParams &P, const Epochs &ep,
                                      const TrajC &c, const int lane,
                                      const float4 *tab = nullptr) {
  Acc s = {0.f, 0.f, 0.f};
  seg1<H, false>(P, ep, c, lane, 0, c.e_in, s);
  seg1<H, true, TB>(P, ep, c, lane, c.e_in, c.e_out, s, tab);
  seg1<H, false>(P, ep, c, lane, c.e_out, P.n_ep, s);
  return acc_reduce(s);
}

// Phase 1 of two trajectories at once: the epoch axis is cut at both
// trajectories' map entry and exit, and each segment runs the matching
// inside/outside combination with one epoch load per lane for both.
template <bool H, int TB = 0>
__device__ __forceinline__ void phase1_pair(const SearchParams &P,
                                            const Epochs &ep, const TrajC &ca,
                                            const TrajC &cb, const int lane,
                                            Acc &ra, Acc &rb,
                                            const float4 *tab = nullptr) {
  Acc2 s = {f2(0.f), f2(0.f), f2(0.f)};
  const TrajP cp = pack_traj(ca, cb);
  // cut points, sorted (warp-uniform)
  int p1 = ca.e_in, p2 = ca.e_out, p3 = cb.e_in, p4 = cb.e_out, t;
  if (p1 > p2) { t = p1; p1 = p2; p2 = t; }
  if (p3 > p4) { t = p3; p3 = p4; p4 = t; }
  if (p1 > p3) { t = p1; p1 = p3; p3 = t; }
  if (p2 > p4) { t = p2; p2 = p4; p4 = t; }
  if (p2 > p3) { t = p2; p2 = p3; p3 = t; }
  const int cut[6] = {0, p1, p2, p3, p4, P.n_ep};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const int e0 = cut[i], e1 = cut[i + 1];
    if (e0 >= e1) continue;
    const bool ina = e0 >= ca.e_in && e1 <= ca.e_out;
    const bool inb = e0 >= cb.e_in && e1 <= cb.e_out;
    if (ina && inb)
      seg2<H, true, true, TB>(P, ep, ca, cb, cp, lane, e0, e1, s, tab);
    else if (ina)
      seg2<H, true, false, TB>(P, ep, ca, cb, cp, lane, e0, e1, s, tab);
    else if (inb)
      seg2<H, false, true, TB>(P, ep, ca, cb, cp, lane, e0, e1, s, tab);
    else
      seg2<H, false, false>(P, ep, ca, cb, cp, lane, e0, e1, s);
  }
  const Acc sa = {s.a.x, s.b.x, s.d.x}, sb = {s.a.y, s.b.y, s.d.y};
  ra = acc_reduce(sa);
  rb = acc_reduce(sb);
}

// Phase 2: chi^2 = sum w (F - Fs A - Fb)^2, written with centred values as
// w (Fc - Fs Ac - Bc)^2, Bc = Fs + Fb - Fref.  FP32 per lane, FP64 across
// lanes; lane 0's value is returned to all lanes.
template <bool H, int TB = 0>
__device__ __forceinline__ double phase2(const SearchParams &P,
                                         const Epochs &ep, const TrajC &c,
                                         const int lane, const float Fs,
                                         const float Bc,
                                         const float4 *tab = nullptr) {
  float chi = 0.f;
#pragma unroll 2
  for (int e = lane_start(0, lane); e < c.e_in; e += 32) {
    const float2 v = ep.tw[e];
    const float Ac = mag_out_m1(c, v.x);
    const float r = __fsub_rn(ep.fc[e], __fmaf_rn(Fs, Ac, Bc));
    chi = __fmaf_rn(__fmul_rn(v.y, r), r, chi);
  }
#pragma unroll (H ? kUnrollH : kUnroll)
  for (int e = lane_start(c.e_in, lane); e < c.e_out; e += 32) {
    const float2 v = ep.tw[e];
    const float Ac = mag_in_m1<H, TB>(P, c, v.x, tab);
    const float r = __fsub_rn(ep.fc[e], __fmaf_rn(Fs, Ac, Bc));
    chi = __fmaf_rn(__fmul_rn(v.y, r), r, chi);
  }
#pragma unroll 2
  for (int e = lane_start(c.e_out, lane); e < P.n_ep; e += 32) {
    const float2 v = ep.tw[e];
    const float Ac = mag_out_m1(c, v.x);
    const float r = __fsub_rn(ep.fc[e], __fmaf_rn(Fs, Ac, Bc));
    chi = __fmaf_rn(__fmul_rn(v.y, r), r, chi);
  }
  double x = (double)chi;
#pragma unroll
  for (int o = 16; o; o >>= 1) x = __dadd_rn(x, __shfl_xor_sync(kFull, x, o));
  return __shfl_sync(kFull, x, 0);
}

struct Solved {
  double Fs, Bc;      // Fb = Bc + Fref - Fs
  double bnum, bden;  // lower bound of the exact chi^2:
                      // C_FF - min(C_FF, bnum / bden) if bden > 0, else 0
  bool degenerate;
};

// 2x2 weighted least squares (Eq. 6) in FP64 from the centred sums, and a
// lower bound of the chi^2 the exact residual sweep will give.
// Degenerate rule: det <= 1e-12 S_AA S_1 (uncentred S_AA) -> Fs = 0,
// Fb = weighted mean flux.
//
// Bound.  With C_FF = S_FF - S_F^2/S_1, C_AA = S_AA - S_A^2/S_1 and
// C_AF = S_AF - S_A S_F/S_1 the minimum is chi^2 = C_FF - C_AF^2 / C_AA.
// The FP32 sums carry relative errors of at most gamma of the sums of
// absolute terms (T_A = sum |w Ac| <= sqrt(S_1 S_AA), T_AF = sum |w Ac Fc|
// <= sqrt(S_AA S_FF); S_AA has positive terms), so |C_AF| and C_AA are
// bracketed and C_AF^2 / C_AA <= (|C_AF| + d_AF)^2 / (C_AA - d_AA).  This
// holds however ill-conditioned (Fs, Fb) is: a nearly flat track explains
// little of C_FF and is discarded all the same.  C_FF is exact up to FP64
// rounding (FP64 sums of the stored values, per event); T_A and T_AF are
// taken as FP32 square roots rounded up, which only widens the bracket.
// gamma is doubled as a margin.
struct Fit2 {
  double Fs, Bc;
  bool degenerate;
};

// the solve alone (the fit of solve2, without the bound)
__device__ __forceinline__ Fit2 fit2(const SearchParams &P, double SA,
                                     double SAA, double SAF) {
  Fit2 o;
  const double S1 = P.S1, SF = P.SF;
  const double SAAu = SAA + 2.0 * SA + S1;
  const double det = SAA * S1 - SA * SA;
  if (!(det > 1e-12 * SAAu * S1)) {
    o.Fs = 0.0;
    o.Bc = SF / S1;
    o.degenerate = true;
  } else {
    const double inv = 1.0 / det;
    o.Fs = (S1 * SAF - SA * SF) * inv;
    o.Bc = (SAA * SF - SA * SAF) * inv;
    o.degenerate = false;
  }
  return o;
}

__device__ __forceinline__ Solved solve2(const SearchParams &P, double SA,
                                         double SAA, double SAF) {
  Solved o;
  const double S1 = P.S1, SF = P.SF, iS1 = P.invS1;
  const Fit2 f = fit2(P, SA, SAA, SAF);
  o.Fs = f.Fs;
  o.Bc = f.Bc;
  o.degenerate = f.degenerate;
  const double g = 2.0 * P.gamma;
  const double CAA = SAA - SA * SA * iS1;
  const double CAF = SAF - SA * SF * iS1;
  const double TA = (double)__fsqrt_ru(__double2float_ru(S1 * SAA));
  const double TAF = (double)__fsqrt_ru(__double2float_ru(SAA * P.SFF));
  const double dAA = g * (SAA + (2.0 * fabs(SA) * TA + g * TA * TA) * iS1);
  const double dAF = g * (TAF + TA * fabs(SF) * iS1);
  const double num = fabs(CAF) + dAF;
  o.bnum = num * num;
  o.bden = CAA > dAA ? CAA - dAA : 0.0;
  return o;
}

// Whether the exact chi^2 of a solved trajectory can be at most thr:
// bound * (1 - 1e-4) <= thr, the 1e-4 a margin for the FP32 rounding of the
// exact sweep, evaluated as C_FF - bnum/bden <= thr / (1 - 1e-4) without a
// division.
__device__ __forceinline__ bool may_reach(const SearchParams &P,
                                          const Solved &o, double thr) {
  if (!(o.bden > 0.0)) return true;  // bound 0
  const double t = thr * 1.0001000100010002;  // >= thr / (1 - 1e-4)
  return (P.CFF - t) * o.bden <= o.bnum;
}

// An upper bound of the chi^2 the exact residual sweep gives at the FP32
// (Fs, Bc) = (a, b) of a solved trajectory, from its phase-1 sums alone
// (the pilot seeds the grid-wide threshold from these, without the sweep:
// K real trajectories have exact chi^2 at or below the K-th bound).  The
// residual sum is S_FF - 2a S_AF - 2b S_F + a^2 S_AA + 2ab S_A + b^2 S_1;
// the FP32 sums are bracketed as in solve2 (S_AA within g S_AA, S_A within
// g T_A, S_AF within g T_AF), each term taken at its worst, plus the FP64
// rounding of the sum of the terms, times 1 + 1e-4 for the FP32 rounding
// of the sweep (the margin may_reach allows it).
__device__ __forceinline__ double chi2_upper(const SearchParams &P, double SA,
                                            double SAA, double SAF, double a,
                                            double b) {
  const double g = 2.0 * P.gamma;
  const double TA = (double)__fsqrt_ru(__double2float_ru(P.S1 * SAA));
  const double TAF = (double)__fsqrt_ru(__double2float_ru(SAA * P.SFF));
  const double q = P.SFF - 2.0 * a * SAF - 2.0 * b * P.SF + a * a * SAA +
                   2.0 * a * b * SA + b * b * P.S1;
  const double absum = P.SFF + 2.0 * fabs(a * SAF) + 2.0 * fabs(b * P.SF) +
                       a * a * SAA + 2.0 * fabs(a * b * SA) + b * b * P.S1;
  const double slack = g * (2.0 * fabs(a) * TAF + a * a * SAA +
                            2.0 * fabs(a * b) * TA) +
                       16.0 * 1.1102230246251565e-16 * absum;
  const double ub = (q + slack) * 1.0001000100010002;
  return ub == ub ? ub : CUDART_INF;  // NaN sums: no bound
}

__device__ __forceinline__ double bits_to_chi2(unsigned long long b) {
  return b == ~0ULL ? CUDART_INF : __longlong_as_double((long long)b);
}


}  // namespace dev
}  // namespace morse
