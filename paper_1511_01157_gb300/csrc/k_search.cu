// Trajectory chi^2 grid search (K2), top-K merge (K2b), fit fill (K2c) and
// the single-trajectory light curve.
//
// The method (McDougall & Albrow 2015, §4.2): a trajectory is a straight
// source track through the (s, q) magnification map; each data point's
// magnification A(t_i) is read from the map by bilinear interpolation, the
// flux model F = Fs A + Fb (Eq. 5-6) is linear in A, and chi^2 is the sum
// of the per-point contributions.  §4.4 keeps the best trajectories as
// seeds.  Here (Fs, Fb) are profiled out by the closed-form weighted
// least-squares solve, and the grid covers (u0, alpha, t0, tE).
//
// GB300 design.
//  * One 32-warp block per SM.  The light curve (t, w, wF, F per epoch,
//    time-sorted) is staged once per block in shared memory.
//  * Warps take groups of 32 trajectories.  For each, the lanes walk
//    consecutive epochs, so the 32 bilinear gathers of a warp fall within a
//    few texels (one 16-byte float4 load fetches a texel's 2x2
//    neighbourhood) and the L2-resident map is served mostly from L1.
//  * A straight track crosses the square map in one interval of time, and
//    the epochs are sorted, so each trajectory's epochs split into three
//    contiguous ranges found by binary search: before the map and after it
//    (single-lens magnification from tau^2 + u0^2, no memory), and inside
//    (bilinear lookup with no per-epoch edge test, coordinates clamped so
//    that every gather stays inside the map).
//  * Phase 1 accumulates the normal-equation sums in FP32 per lane (the
//    magnification centred on 1, the flux on its weighted mean), reduces
//    them across the warp, and solves the 2x2 system in FP64 with one
//    trajectory per lane (32 solves per warp instruction).
//  * The closed-form chi^2 from those sums, C_FF - C_AF^2 / C_AA, loses
//    digits to cancellation, so it is used only as a rigorous lower bound
//    (error-bracketed sums) to discard trajectories that cannot enter the
//    top-K.  Every reported chi^2 comes from phase 2: a second sweep that
//    sums the per-point residuals w (F - Fs A - Fb)^2 (FP32 per lane, FP64
//    across lanes).
//  * Each block keeps a sorted top-K in shared memory.  A warp merges its
//    own candidates under a shared-memory lock (bounded spin), so warps
//    never wait at a block barrier; the block's K-th chi^2 and a grid-wide
//    minimum of K-th values (atomicMin on the bit pattern) are the pruning
//    threshold.  The grid-wide value is seeded by a pilot search over a
//    strided subset of about sqrt(K N) trajectories, so that it is tight
//    from the start.  A tree of pairwise merges gives the global
//    top-K and k_fill recomputes the winners' records with the same device
//    functions.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"

namespace morse {

namespace {

#ifndef MORSE_UNROLL
#define MORSE_UNROLL 4
#endif
constexpr int kUnroll = MORSE_UNROLL;  // inside-map epoch loop

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kLockSpinLimit = 1u << 20;

// Per-trajectory constants.
struct TrajC {
  float ax, bx, ay, by;  // centred pixel coordinates v = a t + b
  float kt, bt, u02;     // tau = kt t + bt; u0^2
  int e_in, e_out;       // epochs [e_in, e_out) lie inside the map
};

__device__ __forceinline__ bool key_less(const Entry &a, const Entry &b) {
  return a.chi2 < b.chi2 || (a.chi2 == b.chi2 && a.idx < b.idx);
}
__device__ __forceinline__ bool key_less(double ca, long long ia, double cb,
                                         long long ib) {
  return ca < cb || (ca == cb && ia < ib);
}

// first epoch index with t > x (strict) or t >= x (!strict), t ascending
__device__ __forceinline__ int epoch_search(const float4 *ep, int n, double x,
                                            bool strict) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const double t = (double)ep[mid].x;
    const bool right = strict ? (t > x) : (t >= x);
    if (right)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
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
__device__ __forceinline__ TrajC traj_consts(const SearchParams &P,
                                             const float4 *ep, long long j) {
  long long r = j;
  const int itE = (int)(r % P.n_tE);
  r /= P.n_tE;
  const int it0 = (int)(r % P.n_t0);
  r /= P.n_t0;
  const int ia = (int)(r % P.n_alpha);
  const int iu = (int)(r / P.n_alpha);
  const double k = P.invtEd[itE];  // 1/(tE Delta)
  const double c = P.ca[ia], s = P.sa[ia];
  const double u = P.u0v[iu], t0 = P.t0rel[it0];
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
  // slab intersection of the line with |y1| < L, |y2| < L
  double lo = -CUDART_INF, hi = CUDART_INF;
  const double us = u * s, uc = u * c;
  if (c != 0.0) {
    const double a0 = (-P.L + us) / c, a1 = (P.L + us) / c;
    lo = fmax(lo, fmin(a0, a1));
    hi = fmin(hi, fmax(a0, a1));
  } else if (!(fabs(us) < P.L)) {
    hi = lo;
  }
  if (s != 0.0) {
    const double b0 = (-P.L - uc) / s, b1 = (P.L - uc) / s;
    lo = fmax(lo, fmin(b0, b1));
    hi = fmin(hi, fmax(b0, b1));
  } else if (!(fabs(uc) < P.L)) {
    hi = lo;
  }
  if (lo < hi) {
    const double tE = 1.0 / kt;
    o.e_in = epoch_search(ep, P.n_ep, t0 + lo * tE, true);
    o.e_out = epoch_search(ep, P.n_ep, t0 + hi * tE, false);
    if (o.e_out < o.e_in) o.e_out = o.e_in;
  } else {
    o.e_in = P.n_ep;
    o.e_out = P.n_ep;
  }
  return o;
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

// Bilinear A - 1 at centred coordinates inside the map (the quads store
// A - 1).  Coordinates below the first texel centre are clamped to it (the
// lookup rule).  Above the last centre no clamp is needed: the caller only
// passes epochs strictly inside the map, so floor(v) <= npix - half - 1, and
// the last texel's quad repeats its edge values.  The bounds-checked build
// verifies the index range.
__device__ __forceinline__ float bilinear_m1(const SearchParams &P, float vx,
                                             float vy) {
  const float cx = fmaxf(vx, P.vmin);
  const float cy = fmaxf(vy, P.vmin);
  // floor: adding 1.5 * 2^23 rounding down leaves floor(c) in the low
  // mantissa bits; the fraction c - floor(c) is exact
  const float tx = __fadd_rd(cx, 12582912.f), ty = __fadd_rd(cy, 12582912.f);
  const float fx = __fsub_rn(cx, __fsub_rn(tx, 12582912.f));
  const float fy = __fsub_rn(cy, __fsub_rn(ty, 12582912.f));
  // texel (ix, iy) = floor(c) + half; quad index iy * qpitch + ix, folded
  // into one multiply-add on the raw bit patterns (mod 2^32, exact because
  // the index is in [0, npix * qpitch))
  const unsigned bx = (unsigned)__float_as_int(tx);
  const unsigned by = (unsigned)__float_as_int(ty);
  const unsigned idx = by * (unsigned)P.qpitch + bx + P.qidx0;
#ifdef MORSE_CHECK_BOUNDS
  // checked build: record an out-of-range texel and skip the access
  const int ix = (int)(bx - 0x4B400000u) + P.half;
  const int iy = (int)(by - 0x4B400000u) + P.half;
  if ((unsigned)ix >= (unsigned)P.npix || (unsigned)iy >= (unsigned)P.npix) {
    if (P.err) atomicOr(P.err, 2u);
    return 0.f;
  }
#endif
  const float4 q = __ldg(&P.quad[idx]);
  const float r0 = __fmaf_rn(fx, __fsub_rn(q.y, q.x), q.x);
  const float r1 = __fmaf_rn(fx, __fsub_rn(q.w, q.z), q.z);
  return __fmaf_rn(fy, __fsub_rn(r1, r0), r0);
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

__device__ __forceinline__ void acc_add(Acc &s, const float4 &v, float Ac) {
  const float wAc = __fmul_rn(v.y, Ac);
  s.a = __fadd_rn(s.a, wAc);
  s.b = __fmaf_rn(wAc, Ac, s.b);
  s.d = __fmaf_rn(v.z, Ac, s.d);
}

// A - 1 at time t inside the map (bilinear) or outside (single lens)
__device__ __forceinline__ float mag_in_m1(const SearchParams &P,
                                           const TrajC &c, float t) {
  return bilinear_m1(P, __fmaf_rn(c.ax, t, c.bx), __fmaf_rn(c.ay, t, c.by));
}
__device__ __forceinline__ float mag_out_m1(const TrajC &c, float t) {
  const float tau = __fmaf_rn(c.kt, t, c.bt);
  return __fsub_rn(pspl_u2(__fmaf_rn(tau, tau, c.u02)), 1.f);
}

template <bool IN>
__device__ __forceinline__ void seg1(const SearchParams &P, const float4 *ep,
                                     const TrajC &c, int lane, int e0, int e1,
                                     Acc &s) {
#pragma unroll (IN ? kUnroll : 2)
  for (int e = lane_start(e0, lane); e < e1; e += 32) {
    const float4 v = ep[e];
    acc_add(s, v, IN ? mag_in_m1(P, c, v.x) : mag_out_m1(c, v.x));
  }
}

// two trajectories over one epoch segment, one epoch load for both
template <bool INA, bool INB>
__device__ __forceinline__ void seg2(const SearchParams &P, const float4 *ep,
                                     const TrajC &ca, const TrajC &cb,
                                     int lane, int e0, int e1, Acc &sa,
                                     Acc &sb) {
#pragma unroll ((INA || INB) ? kUnroll : 2)
  for (int e = lane_start(e0, lane); e < e1; e += 32) {
    const float4 v = ep[e];
    acc_add(sa, v, INA ? mag_in_m1(P, ca, v.x) : mag_out_m1(ca, v.x));
    acc_add(sb, v, INB ? mag_in_m1(P, cb, v.x) : mag_out_m1(cb, v.x));
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
__device__ __forceinline__ Acc phase1(const SearchParams &P, const float4 *ep,
                                      const TrajC &c, const int lane) {
  Acc s = {0.f, 0.f, 0.f};
  seg1<false>(P, ep, c, lane, 0, c.e_in, s);
  seg1<true>(P, ep, c, lane, c.e_in, c.e_out, s);
  seg1<false>(P, ep, c, lane, c.e_out, P.n_ep, s);
  return acc_reduce(s);
}

// Phase 1 of two trajectories at once: the epoch axis is cut at both
// trajectories' map entry and exit, and each segment runs the matching
// inside/outside combination with one epoch load per lane for both.
__device__ __forceinline__ void phase1_pair(const SearchParams &P,
                                            const float4 *ep, const TrajC &ca,
                                            const TrajC &cb, const int lane,
                                            Acc &ra, Acc &rb) {
  Acc sa = {0.f, 0.f, 0.f}, sb = {0.f, 0.f, 0.f};
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
      seg2<true, true>(P, ep, ca, cb, lane, e0, e1, sa, sb);
    else if (ina)
      seg2<true, false>(P, ep, ca, cb, lane, e0, e1, sa, sb);
    else if (inb)
      seg2<false, true>(P, ep, ca, cb, lane, e0, e1, sa, sb);
    else
      seg2<false, false>(P, ep, ca, cb, lane, e0, e1, sa, sb);
  }
  ra = acc_reduce(sa);
  rb = acc_reduce(sb);
}

// Phase 2: chi^2 = sum w (F - Fs A - Fb)^2, written with centred values as
// w (Fc - Fs Ac - Bc)^2, Bc = Fs + Fb - Fref.  FP32 per lane, FP64 across
// lanes; lane 0's value is returned to all lanes.
__device__ __forceinline__ double phase2(const SearchParams &P,
                                         const float4 *ep, const TrajC &c,
                                         const int lane, const float Fs,
                                         const float Bc) {
  float chi = 0.f;
#pragma unroll 2
  for (int e = lane_start(0, lane); e < c.e_in; e += 32) {
    const float4 v = ep[e];
    const float Ac = mag_out_m1(c, v.x);
    const float r = __fsub_rn(v.w, __fmaf_rn(Fs, Ac, Bc));
    chi = __fmaf_rn(__fmul_rn(v.y, r), r, chi);
  }
#pragma unroll (kUnroll)
  for (int e = lane_start(c.e_in, lane); e < c.e_out; e += 32) {
    const float4 v = ep[e];
    const float Ac = mag_in_m1(P, c, v.x);
    const float r = __fsub_rn(v.w, __fmaf_rn(Fs, Ac, Bc));
    chi = __fmaf_rn(__fmul_rn(v.y, r), r, chi);
  }
#pragma unroll 2
  for (int e = lane_start(c.e_out, lane); e < P.n_ep; e += 32) {
    const float4 v = ep[e];
    const float Ac = mag_out_m1(c, v.x);
    const float r = __fsub_rn(v.w, __fmaf_rn(Fs, Ac, Bc));
    chi = __fmaf_rn(__fmul_rn(v.y, r), r, chi);
  }
  double x = (double)chi;
#pragma unroll
  for (int o = 16; o; o >>= 1) x = __dadd_rn(x, __shfl_xor_sync(kFull, x, o));
  return __shfl_sync(kFull, x, 0);
}

struct Solved {
  double Fs, Bc;      // Fb = Bc + Fref - Fs
  double lb;          // rigorous lower bound of the exact chi^2
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
// little of C_FF and is discarded all the same.  C_FF is exact (FP64 sums
// of the stored values).  gamma is doubled as a margin.
__device__ __forceinline__ Solved solve2(const SearchParams &P, double SA,
                                         double SAA, double SAF) {
  Solved o;
  const double S1 = P.S1, SF = P.SF, SFF = P.SFF;
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
  const double g = 2.0 * P.gamma;
  const double CFF = SFF - SF * SF / S1;
  const double CAA = SAA - SA * SA / S1;
  const double CAF = SAF - SA * SF / S1;
  const double TA = sqrt(S1 * SAA), TAF = sqrt(SAA * SFF);
  const double dAA = g * (SAA + (2.0 * fabs(SA) * TA + g * TA * TA) / S1);
  const double dAF = g * (TAF + TA * fabs(SF) / S1);
  double X = CFF;  // upper bound of the part of C_FF the fit explains
  if (CAA > dAA) {
    const double num = fabs(CAF) + dAF;
    X = fmin(CFF, num * num / (CAA - dAA));
  }
  o.lb = CFF - X;
  return o;
}

__device__ __forceinline__ double bits_to_chi2(unsigned long long b) {
  return b == ~0ULL ? CUDART_INF : __longlong_as_double((long long)b);
}

// Block-wide top-K state in shared memory.
struct BlockTopK {
  Entry *buf0, *buf1; // the sorted list and its merge target, alternating
  Entry *wbuf;        // per-warp staging of sorted candidates (32 each)
  int *cur, *nk, *lock;
  volatile double *thr;
};

// Warp-collective: merge this lane's candidate (if any) into the block's
// sorted top-K under the block lock.  Candidates are first sorted across
// the warp (bitonic); each existing entry and each candidate then moves to
// its rank in the union, and the first K are kept.
__device__ void warp_merge(const SearchParams &P, BlockTopK &T, const int K,
                           const int warp, const int lane, bool has,
                           double chi2, long long idx) {
  const unsigned m = __ballot_sync(kFull, has);
  if (!m) return;
  const int nc = __popc(m);
  double key = has ? chi2 : CUDART_INF;
  long long id = has ? idx : 0x7fffffffffffffffLL;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const double ok = __shfl_xor_sync(kFull, key, j);
      const long long oi = __shfl_xor_sync(kFull, id, j);
      const bool keep_min = (((lane & k) == 0) == ((lane & j) == 0));
      const bool other_less = key_less(ok, oi, key, id);
      if (keep_min == other_less) {
        key = ok;
        id = oi;
      }
    }
  }
  Entry *wb = T.wbuf + warp * 32;
  if (lane < nc) {
    wb[lane].chi2 = key;
    wb[lane].idx = id;
  }
  // acquire the block lock (bounded spin)
  int ok = 1;
  if (lane == 0) {
    unsigned it = 0;
    while (atomicCAS(T.lock, 0, 1) != 0) {
      if (++it > kLockSpinLimit) {
        ok = 0;
        if (P.err) atomicOr(P.err, 1u);
        break;
      }
      __nanosleep(64);
    }
    __threadfence_block();
  }
  ok = __shfl_sync(kFull, ok, 0);
  __syncwarp();
  if (!ok) return;
  const int c0 = *T.cur;
  const int nk = *T.nk;
  const Entry *cur = c0 ? T.buf1 : T.buf0;
  Entry *nxt = c0 ? T.buf0 : T.buf1;
  for (int i = lane; i < nk; i += 32) {
    const Entry e = cur[i];
    int lo = 0, hi = nc;  // candidates below e
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (key_less(wb[mid], e))
        lo = mid + 1;
      else
        hi = mid;
    }
    const int r = i + lo;
    if (r < K) nxt[r] = e;
  }
  if (lane < nc) {
    const Entry e = wb[lane];
    int lo = 0, hi = nk;  // kept entries below e
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (key_less(cur[mid], e))
        lo = mid + 1;
      else
        hi = mid;
    }
    const int r = lane + lo;
    if (r < K) nxt[r] = e;
  }
  __syncwarp();
  if (lane == 0) {
    const int nn = min(K, nk + nc);
    *T.nk = nn;
    *T.cur = c0 ^ 1;
    const double th = (nn == K) ? nxt[K - 1].chi2 : CUDART_INF;
    *T.thr = th;
    if (P.gthr && nn == K)
      atomicMin(P.gthr, (unsigned long long)__double_as_longlong(th));
    __threadfence_block();
    atomicExch(T.lock, 0);
  }
  __syncwarp();
}

template <bool DENSE, bool EP_SMEM>
__global__ void __launch_bounds__(kSearchWarps * 32, 1)
    k_search(const SearchParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int K = P.top_k;

  const float4 *ep = P.ep;
  BlockTopK T;
  __shared__ int s_cur, s_nk, s_lock;
  __shared__ double s_thr;
  {
    unsigned char *p = smem;
    if (EP_SMEM) {
      float4 *s = reinterpret_cast<float4 *>(p);
      for (int e = threadIdx.x; e < P.n_ep; e += blockDim.x) s[e] = P.ep[e];
      ep = s;
      p += sizeof(float4) * (size_t)P.n_ep;
    }
    if (!DENSE) {
      T.buf0 = reinterpret_cast<Entry *>(p);
      T.buf1 = T.buf0 + K;
      T.wbuf = T.buf1 + K;
    }
    T.cur = &s_cur;
    T.nk = &s_nk;
    T.lock = &s_lock;
    T.thr = &s_thr;
  }
  if (threadIdx.x == 0) {
    s_cur = 0;
    s_nk = 0;
    s_lock = 0;
    s_thr = CUDART_INF;
  }
  __syncthreads();

  // Warp groups.  A strided sample (pilot, stride > 1) is cut into runs of
  // tpg sample indices.  Otherwise groups are aligned to (u0, alpha) lines
  // (P.line consecutive trajectories share the track's line), ng_line
  // groups per line, so that the warps of a block, which take consecutive
  // groups, walk the same line of the map and share its texels in L1.
  const int tpg = P.tpg;  // trajectories per warp group (1..32)
  const bool lined = P.stride == 1 && P.line > 0;
  long long n_groups, line0 = 0;
  if (lined) {
    line0 = P.first / P.line;
    const long long line1 = (P.first + P.count - 1) / P.line;
    n_groups = (line1 - line0 + 1) * P.ng_line;
  } else {
    n_groups = (P.count + tpg - 1) / tpg;
  }
  const long long gstride = (long long)gridDim.x * kSearchWarps;
  unsigned long long n_exact = 0;

  for (long long g = (long long)blockIdx.x * kSearchWarps + warp;
       g < n_groups; g += gstride) {
    long long lo, hi;  // absolute indices (lined) or sample indices
    if (lined) {
      const long long L = line0 + g / P.ng_line;
      const long long gi = g % P.ng_line;
      lo = max(P.first, L * P.line + gi * tpg);
      hi = min(P.first + P.count, L * P.line + min((gi + 1) * tpg, P.line));
    } else {
      lo = g * tpg;
      hi = min(lo + tpg, P.count);
    }
    const int nvalid = (int)max(0LL, hi - lo);
    if (nvalid == 0) continue;  // warp-uniform
    const int ml = lane < nvalid ? lane : 0;
    const long long my = lined ? lo + ml : P.first + (lo + ml) * P.stride;
    const long long out_off = lined ? lo - P.first : lo;  // dense output
    const TrajC mine = traj_consts(P, ep, my);
    Acc mine_s = {0.f, 0.f, 0.f};
    for (int k = 0; k < nvalid; k += 2) {
      const TrajC ca = shfl_traj(mine, k);
      if (k + 1 < nvalid) {
        const TrajC cb = shfl_traj(mine, k + 1);
        Acc ra, rb;
        phase1_pair(P, ep, ca, cb, lane, ra, rb);
        if (lane == k) mine_s = ra;
        if (lane == k + 1) mine_s = rb;
      } else {
        const Acc ra = phase1(P, ep, ca, lane);
        if (lane == k) mine_s = ra;
      }
    }
    const Solved sol =
        solve2(P, (double)mine_s.a, (double)mine_s.b, (double)mine_s.d);
    double thr = CUDART_INF;
    if (!DENSE) {
      thr = *T.thr;
      if (P.gthr) thr = fmin(thr, bits_to_chi2(__ldcg(P.gthr)));
    }
    bool cand_me = lane < nvalid;
    // 1e-4: margin for the FP32 rounding of the exact sweep itself
    if (!DENSE && cand_me && thr < CUDART_INF)
      cand_me = sol.lb * (1.0 - 1e-4) <= thr;
    unsigned todo = __ballot_sync(kFull, cand_me);
    n_exact += __popc(todo);
    const float myFs = __double2float_rn(sol.Fs);
    const float myBc = __double2float_rn(sol.Bc);
    double my_chi2 = CUDART_INF;
    while (todo) {
      const int k = __ffs(todo) - 1;
      todo &= todo - 1;
      const TrajC c = shfl_traj(mine, k);
      const float Fs = __shfl_sync(kFull, myFs, k);
      const float Bc = __shfl_sync(kFull, myBc, k);
      const double chi2 = phase2(P, ep, c, lane, Fs, Bc);
      if (lane == k) my_chi2 = isnan(chi2) ? CUDART_INF : chi2;
    }
    if (DENSE) {
      if (lane < nvalid) {
        const long long o = out_off + lane;
        P.dchi2[o] = my_chi2;
        if (P.dFs) P.dFs[o] = sol.Fs;
        if (P.dFb) P.dFb[o] = sol.Bc + P.Fref - sol.Fs;
      }
    } else {
      const bool keep = lane < nvalid && my_chi2 <= thr && my_chi2 < CUDART_INF;
      warp_merge(P, T, K, warp, lane, keep, my_chi2, my);
    }
  }
  if (P.stat_exact && lane == 0 && n_exact)
    atomicAdd(P.stat_exact, n_exact);
  if (!DENSE) {
    __syncthreads();
    const int nk = s_nk;
    const Entry *cur = s_cur ? T.buf1 : T.buf0;
    Entry *out = P.partial + (size_t)blockIdx.x * K;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      Entry e;
      if (i < nk) {
        e = cur[i];
      } else {
        e.chi2 = CUDART_INF;  // unique sentinel keys sort after real ones
        e.idx = 0x7fffffffffffffffLL - ((long long)blockIdx.x * K + i);
      }
      out[i] = e;
    }
  }
}

// One level of the merge tree: list pairs (2p, 2p+1) -> list p, keeping the
// first k of each merged pair.  An odd last list is copied.
__global__ void k_merge_level(const Entry *__restrict__ in,
                              Entry *__restrict__ out, int lists, int k) {
  const int pairs = (lists + 1) / 2;
  const long long total = (long long)pairs * 2 * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       t < total; t += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(t / (2 * k));
    const int side = (int)((t / k) & 1);
    const int i = (int)(t % k);
    const int la = 2 * p, lb = 2 * p + 1;
    if (lb >= lists) {  // odd list out: copy
      if (side == 0) out[(size_t)p * k + i] = in[(size_t)la * k + i];
      continue;
    }
    const Entry *A = in + (size_t)(side ? lb : la) * k;
    const Entry *B = in + (size_t)(side ? la : lb) * k;
    const Entry e = A[i];
    int lo = 0, hi = k;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (key_less(B[mid], e))
        lo = mid + 1;
      else
        hi = mid;
    }
    const int r = i + lo;
    if (r < k) out[(size_t)p * k + r] = e;
  }
}

// Fit fill: one warp per selected trajectory recomputes the phase-1 sums,
// the solve and the phase-2 chi^2 with the same device functions as the
// search, and writes the public morse_fit record.
__global__ void k_fill(const FillParams F) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= F.k) return;
  const SearchParams &P = F.S;
  const Entry e = F.sel[w];
  morse_fit r;
  const long long total = (long long)P.n_u0 * P.n_alpha * P.n_t0 * P.n_tE;
  if (e.idx < 0 || e.idx >= total) {
    if (lane == 0) {
      r.chi2 = CUDART_INF;
      r.t0 = r.tE = r.u0 = r.alpha = r.Fs = r.Fb = 0.0;
      r.idx = -1;
      r.flags = 0;
      r.reserved = 0;
      F.out[w] = r;
    }
    return;
  }
  const TrajC c = traj_consts(P, P.ep, e.idx);
  const Acc s = phase1(P, P.ep, c, lane);
  const Solved sol = solve2(P, (double)s.a, (double)s.b, (double)s.d);
  const double chi2 = phase2(P, P.ep, c, lane, __double2float_rn(sol.Fs),
                             __double2float_rn(sol.Bc));
  if (lane == 0) {
    long long q = e.idx;
    const int itE = (int)(q % P.n_tE);
    q /= P.n_tE;
    const int it0 = (int)(q % P.n_t0);
    q /= P.n_t0;
    const int ia = (int)(q % P.n_alpha);
    const int iu = (int)(q / P.n_alpha);
    r.chi2 = isnan(chi2) ? CUDART_INF : chi2;
    r.t0 = F.t0abs[it0];
    r.tE = F.tEv[itE];
    r.u0 = P.u0v[iu];
    r.alpha = 2.0 * CUDART_PI * (double)ia / (double)P.n_alpha;
    r.Fs = sol.Fs;
    r.Fb = sol.Bc + P.Fref - sol.Fs;
    r.idx = e.idx;
    r.flags = sol.degenerate ? MORSE_FIT_DEGENERATE : 0;
    r.reserved = 0;
    F.out[w] = r;
  }
}

// Seed the grid-wide threshold with the K-th chi^2 of a pilot search over
// a subset of the grid: K trajectories at or below it exist, so anything
// above it cannot enter the global top-K.
__global__ void k_seed_threshold(const Entry *sel, int k,
                                 unsigned long long *gthr) {
  const Entry e = sel[k - 1];
  if (e.chi2 < CUDART_INF && e.idx >= 0 && e.idx < 0x7fff000000000000LL)
    atomicMin(gthr, (unsigned long long)__double_as_longlong(e.chi2));
}

// A(t) along one trajectory given by (ax, bx, ay, by) with v = a t + b, and
// tau = kt t + bt, u0^2 for the single-lens part outside the map.
__global__ void k_lightcurve(const SearchParams P, float ax, float bx,
                             float ay, float by, float kt, float bt, float u02,
                             const float *__restrict__ t, int n,
                             float *__restrict__ A) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += gridDim.x * blockDim.x) {
    const float vx = __fmaf_rn(ax, t[i], bx);
    const float vy = __fmaf_rn(ay, t[i], by);
    const bool inside =
        (vx > P.vlo) & (vx < P.vhi) & (vy > P.vlo) & (vy < P.vhi);
    if (inside) {
      A[i] = __fadd_rn(bilinear_m1(P, vx, vy), 1.f);
    } else {
      const float tau = __fmaf_rn(kt, t[i], bt);
      A[i] = pspl_u2(__fmaf_rn(tau, tau, u02));
    }
  }
}

}  // namespace

size_t search_smem_bytes(int n_ep_smem, int top_k) {
  return sizeof(float4) * (size_t)n_ep_smem +
         sizeof(Entry) * ((size_t)2 * top_k + kSearchWarps * 32);
}

#ifndef MORSE_SMEM_CARVEOUT
#define MORSE_SMEM_CARVEOUT 1
#endif

template <bool D, bool E>
static int occupancy(size_t smem) {
  cudaFuncSetAttribute(k_search<D, E>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
#if MORSE_SMEM_CARVEOUT
  // ask for the smallest shared-memory carveout that holds the block, so
  // the rest of the SM's 256 KB serves as L1 for the map gathers
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                         dev);
  if (optin > 0) {
    int pct = (int)((100.0 * (double)(smem + 2048)) / (double)optin) + 1;
    if (pct > 100) pct = 100;
    cudaFuncSetAttribute(k_search<D, E>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  }
#endif
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &b, k_search<D, E>, kSearchWarps * 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b;
}

int search_blocks_per_sm(bool dense, bool ep_smem, size_t smem) {
  if (dense && ep_smem) return occupancy<true, true>(smem);
  if (dense) return occupancy<true, false>(smem);
  if (ep_smem) return occupancy<false, true>(smem);
  return occupancy<false, false>(smem);
}

cudaError_t launch_search(const SearchParams &P, bool dense, bool ep_smem,
                          int grid, size_t smem, cudaStream_t st) {
  const int threads = kSearchWarps * 32;
  if (dense && ep_smem)
    k_search<true, true><<<grid, threads, smem, st>>>(P);
  else if (dense)
    k_search<true, false><<<grid, threads, smem, st>>>(P);
  else if (ep_smem)
    k_search<false, true><<<grid, threads, smem, st>>>(P);
  else
    k_search<false, false><<<grid, threads, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_topk_merge(Entry *a, Entry *b, int lists, int k,
                              Entry **result, int *levels, cudaStream_t st) {
  Entry *in = a, *out = b;
  *levels = 0;
  while (lists > 1) {
    const int pairs = (lists + 1) / 2;
    const long long total = (long long)pairs * 2 * k;
    long long g = (total + 255) / 256;
    if (g > 65535) g = 65535;
    k_merge_level<<<(int)g, 256, 0, st>>>(in, out, lists, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++*levels;
    lists = pairs;
    Entry *t = in;
    in = out;
    out = t;
  }
  *result = in;
  return cudaSuccess;
}

cudaError_t launch_fill(const FillParams &F, cudaStream_t st) {
  const int threads = 256;
  const int blocks = (F.k * 32 + threads - 1) / threads;
  k_fill<<<blocks, threads, 0, st>>>(F);
  return cudaGetLastError();
}

cudaError_t launch_seed_threshold(const Entry *sel, int k,
                                  unsigned long long *gthr, cudaStream_t st) {
  k_seed_threshold<<<1, 1, 0, st>>>(sel, k, gthr);
  return cudaGetLastError();
}

cudaError_t launch_lightcurve(const SearchParams &P, float ax, float bx,
                              float ay, float by, float kt, float bt,
                              float u02, const float *t, int n, float *A,
                              cudaStream_t st) {
  int blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_lightcurve<<<blocks, 256, 0, st>>>(P, ax, bx, ay, by, kt, bt, u02, t, n,
                                       A);
  return cudaGetLastError();
}

}  // namespace morse
