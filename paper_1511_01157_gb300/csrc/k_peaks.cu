// Peak library and peak-aligned trajectories (§4.3 (iii)-(v)).
//
// (iii) A peak of a trajectory is where the magnification along it turns
// from rising to falling; the library holds, for every line of the grid,
// the number of peaks of the map along it and their positions M_p (Einstein
// radii from the line's reference point).  Trajectories whose line has
// fewer peaks than the light curve needs are not searched.
// (iv) One peak time t_p ties t0 to tE: t0 = t_p - M_p tE (Eq. 7).
// (v) Two peak times fix both: tE = (t_p2 - t_p1) / (M_p2 - M_p1) (Eq. 8),
// then Eq. 7.
//
// The profile a line's peaks are read from (the paper leaves the sampling
// open): samples every h = Delta / sub along the part of the line inside
// the map, the bilinear lookup between texel centres in FP32, and a rise
// or fall confirmed when it exceeds the factor r = 1 + delta.  FP32 decides
// the count, with every operation rounded explicitly (no contraction), so
// the result is the same bit for bit wherever it is computed.
//
// GB300 design: one warp per line.  The line's FP64 set-up (its texel
// coordinates and sample run) is spread over lanes, the FP64 pipe being
// narrow on this part.
// The lanes evaluate 32 consecutive samples at once (the line's texels
// stream through L1/L2, the map having just been built); the sequential
// peak detector then steps through them with every lane holding the same
// state: a chunk whose extremes show that it cannot change the state
// (most chunks: a line has a few peaks) only moves the running extreme;
// otherwise a warp scan of the running maximum (or minimum) finds the
// first sample of the 32 that changes the state, everything before it
// moves only the running extreme, and the scan resumes after it -- no
// shared memory, no divergence.  The highest peaks are kept one per lane,
// the list shifted by a warp shuffle on the rare insertion.  The expansion
// into trajectory entries is one thread per (line, slot).
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"

namespace morse {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPkWarps = 4;

// The sequential peak detector on one line of one map, with the line's
// set-up (FP32 line p = a tau + b, the sample run [k0, k1]) done by the
// caller; writes count[out], pos and height[out * max_peaks + q].
__device__ __forceinline__ void detect_line(
    const float *__restrict__ A, int npix, int lane, int K, int k0, int k1,
    float axf, float ayf, float bxf, float byf, float hf, double h,
    double sh, float r, int max_peaks, long long out, int *__restrict__ count,
    double *__restrict__ pos, double *__restrict__ height,
    unsigned *__restrict__ err) {
  const float lo = -0.5f, hi = (float)npix - 0.5f, pmax = (float)(npix - 1);
  // The detector's state is the same in every lane (each step reads one
  // broadcast sample), so its branches are warp-uniform.  Kept peak q
  // (highest first) lives in lane q.
  int cnt = 0, nkept = 0, kmx = 0;
  bool look_max = false;
  float mn = CUDART_INF_F, mx = -CUDART_INF_F;
  float kh = -CUDART_INF_F;
  int kk = 0;
  // The superset must start and end outside the map (unless it reaches
  // the ends of the sampled range): otherwise samples were missed.  The
  // first sample and the last are tested once, as the chunk loop below
  // decides inside.
  if (k0 <= k1) {
    const int ke = lane == 0 ? k0 : k1;
    const float te = __fmul_rn((float)ke, hf);
    const float ex = __fadd_rn(__fmul_rn(axf, te), bxf);
    const float ey = __fadd_rn(__fmul_rn(ayf, te), byf);
    const bool ein = ex > lo && ex < hi && ey > lo && ey < hi;
    if ((lane == 0 && ein && k0 > -K) || (lane == 1 && ein && k1 < K))
      atomicOr(err, 1u);
  }
  for (int kb = k0; kb <= k1; kb += 32) {
    // Every lane evaluates its sample, branch-free: the clamps keep the
    // texel reads inside the map, and only the samples of the run inside
    // the map (in) count.
    const int k = kb + lane;
    const float tk = __fmul_rn((float)k, hf);
    const float px = __fadd_rn(__fmul_rn(axf, tk), bxf);
    const float py = __fadd_rn(__fmul_rn(ayf, tk), byf);
    const bool in = k <= k1 && px > lo && px < hi && py > lo && py < hi;
    float qx = px < 0.f ? 0.f : px, qy = py < 0.f ? 0.f : py;
    if (qx > pmax) qx = pmax;
    if (qy > pmax) qy = pmax;
    int i0 = (int)floorf(qx), j0 = (int)floorf(qy);
    if (i0 > npix - 2) i0 = npix - 2;
    if (j0 > npix - 2) j0 = npix - 2;
    const float fx = __fsub_rn(qx, (float)i0);
    const float fy = __fsub_rn(qy, (float)j0);
    const float *row = A + (size_t)j0 * npix + i0;
    const float a00 = __ldg(row), a10 = __ldg(row + 1);
    const float a01 = __ldg(row + npix), a11 = __ldg(row + npix + 1);
    const float gx = __fsub_rn(1.f, fx), gy = __fsub_rn(1.f, fy);
    const float r0 = __fadd_rn(__fmul_rn(gx, a00), __fmul_rn(fx, a10));
    const float r1 = __fadd_rn(__fmul_rn(gx, a01), __fmul_rn(fx, a11));
    const float v = __fadd_rn(__fmul_rn(gy, r0), __fmul_rn(fy, r1));
    const unsigned m = __ballot_sync(kFull, in);
    if (m == 0u) continue;
    // Most chunks cannot change the detector's state, which the chunk's
    // extremes show (one integer reduction each: the samples are
    // non-negative, so their bit patterns order as the values): looking
    // for a maximum, no sample ends a peak if max(mx, chunk max) <=
    // r x (chunk min), since every running maximum is at most the former
    // and every r x_i at least the latter (rounding is monotone); looking
    // for a rise, none starts one if chunk max <= r x min(mn, chunk min).
    // Such a chunk only moves the running extreme, exactly as the scan
    // below would.
    {
      const unsigned vb = __float_as_uint(v);
      const float cmax =
          __uint_as_float(__reduce_max_sync(kFull, in ? vb : 0u));
      const float cmin =
          __uint_as_float(__reduce_min_sync(kFull, in ? vb : 0x7f800000u));
      if (look_max) {
        if (fmaxf(mx, cmax) <= __fmul_rn(r, cmin)) {
          if (cmax > mx) {
            kmx = kb + __ffs(__ballot_sync(kFull, in && v == cmax)) - 1;
            mx = cmax;
          }
          continue;
        }
      } else {
        const float low = fminf(mn, cmin);
        if (cmax <= __fmul_rn(r, low)) {
          mn = low;
          continue;
        }
      }
    }
    // The chunk's samples in order, a run at a time.  With the inclusive
    // running maximum pm_i (of mx and the run's samples up to i), sample i
    // ends a peak exactly when pm_i > r x_i (a sample above the running
    // maximum has pm_i = x_i <= r x_i); with the running minimum pn_i, a
    // rise starts exactly when x_i > r pn_i.  Up to the first such sample
    // j only the running extreme (and its position) moves; j changes the
    // state, and the next run starts after it.
    unsigned act = m;  // inside lanes not yet stepped through
    for (int guard = 0; act != 0u && guard < 33; ++guard) {
      const bool a = (act >> lane) & 1u;
      if (look_max) {
        float pm = a ? v : -CUDART_INF_F;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float y = __shfl_up_sync(kFull, pm, o);
          pm = fmaxf(pm, y);  // lanes below o get their own value
        }
        pm = fmaxf(pm, mx);
        const unsigned f = __ballot_sync(kFull, a && pm > __fmul_rn(r, v));
        const int j = f ? __ffs(f) - 1 : 32;
        const unsigned before = act & (j < 32 ? (1u << j) - 1u : kFull);
        if (before) {
          const float cm = __shfl_sync(kFull, pm, 31 - __clz(before));
          if (cm > mx) {
            kmx = kb + __ffs(__ballot_sync(
                           kFull, ((before >> lane) & 1u) && v == cm)) - 1;
            mx = cm;
          }
        }
        if (j == 32) break;
        // a peak (mx at kmx) ends at sample j; kept if among the max_peaks
        // highest (ties: the earlier)
        ++cnt;
        const int at = __popc(__ballot_sync(kFull, lane < nkept && kh >= mx));
        if (at < max_peaks) {
          const float kh_up = __shfl_up_sync(kFull, kh, 1);
          const int kk_up = __shfl_up_sync(kFull, kk, 1);
          if (lane == at) {
            kh = mx;
            kk = kmx;
          } else if (lane > at && lane < max_peaks) {
            kh = kh_up;
            kk = kk_up;
          }
          if (nkept < max_peaks) ++nkept;
        }
        look_max = false;
        mn = __shfl_sync(kFull, v, j);
        act &= j < 31 ? ~((2u << j) - 1u) : 0u;
      } else {
        float pn = a ? v : CUDART_INF_F;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const float y = __shfl_up_sync(kFull, pn, o);
          pn = fminf(pn, y);
        }
        pn = fminf(pn, mn);
        const unsigned f = __ballot_sync(kFull, a && v > __fmul_rn(r, pn));
        const int j = f ? __ffs(f) - 1 : 32;
        const unsigned before = act & (j < 32 ? (1u << j) - 1u : kFull);
        if (before) mn = __shfl_sync(kFull, pn, 31 - __clz(before));
        if (j == 32) break;
        // a rise confirmed at sample j: the peak search starts there
        look_max = true;
        mx = __shfl_sync(kFull, v, j);
        kmx = kb + j;
        act &= j < 31 ? ~((2u << j) - 1u) : 0u;
      }
    }
  }
  // kept peaks in increasing tau: lane q's rank among the kept k
  int rank = 0;
  for (int p = 0; p < nkept; ++p) {
    const int kp = __shfl_sync(kFull, kk, p);
    rank += (kp < kk) ? 1 : 0;
  }
  if (lane == 0) count[out] = cnt;
  if (lane < max_peaks) {
    if (lane < nkept) {
      const size_t o = (size_t)out * max_peaks + rank;
      pos[o] = __dsub_rn(__dmul_rn((double)kk, h), sh);
      height[o] = (double)kh;
    } else {
      const size_t o = (size_t)out * max_peaks + lane;
      pos[o] = CUDART_NAN;
      height[o] = CUDART_NAN;
    }
  }
}

// Warp w takes line w % n_lines of map w / n_lines: the map A0, or As[m]
// of a batch of maps of one geometry (more warps per SM than one map's
// lines give).  Outputs of map m, line j at index m n_lines + j.  Slower
// on 64 maps, and not kept: a warp running one line on several maps (its
// set-up shared; fewer warps), reading a chunk's texels while the chunk
// before it is scanned, and steps of 2 or 4 chunks under one test.
__global__ void __launch_bounds__(kPkWarps * 32)
    k_line_peaks(const float *__restrict__ A0,
                 const float *const *__restrict__ As, int n_maps, int npix,
                 double L, double dlt, double h,
                 const double *__restrict__ lu,
                 const double *__restrict__ lc,
                 const double *__restrict__ ls, const double *__restrict__ lsh,
                 int n_lines, int sub, float r, int max_peaks,
                 int *__restrict__ count, double *__restrict__ pos,
                 double *__restrict__ height, unsigned *__restrict__ err) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= (long long)n_lines * n_maps) return;  // warp-uniform, no barrier
  const int mi = (int)(w / n_lines);
  const int line = (int)(w - (long long)mi * n_lines);
  const double u = lu[line], c = lc[line], s = ls[line], sh = lsh[line];
  // The line in texel coordinates, p = a tau + b, in FP64 then FP32, with
  // the texel size dlt = 2 L / npix and the step h = dlt / sub (both
  // rounded once, by the caller).  The set-up's divisions are spread over
  // lanes 0-3, one quotient each (the FP64 pipe is narrow): ax, ay, bx, by.
  const int l4 = lane & 3;
  const double num = l4 == 0   ? c
                     : l4 == 1 ? s
                     : l4 == 2 ? __dsub_rn(L, __dmul_rn(u, s))
                               : __dadd_rn(L, __dmul_rn(u, c));
  double q = __ddiv_rn(num, dlt);
  if (l4 >= 2) q = __dsub_rn(q, 0.5);
  const float qf = __double2float_rn(q);
  const double ax = __shfl_sync(kFull, q, 0), ay = __shfl_sync(kFull, q, 1);
  const double bx = __shfl_sync(kFull, q, 2), by = __shfl_sync(kFull, q, 3);
  const float axf = __shfl_sync(kFull, qf, 0), ayf = __shfl_sync(kFull, qf, 1);
  const float bxf = __shfl_sync(kFull, qf, 2), byf = __shfl_sync(kFull, qf, 3);
  const float hf = __double2float_rn(h);
  const float lo = -0.5f, hi = (float)npix - 0.5f;
  const int K = sub * npix;
  // Samples inside the map form one run of k (p is monotone in k); a
  // superset of it from the FP64 line, two samples wider on each side:
  // per axis the k where p crosses -0.5 and npix - 0.5 (lanes 0-3 again:
  // x low, x high, y low, y high), then lanes 0 (x) and 1 (y) round and
  // clamp their axis's interval, [-K, -K - 1] (empty) for an axis along
  // which the line is constant outside the map.
  const double ahx = ax * h, ahy = ay * h;
  const double bb = l4 < 2 ? bx : by;
  const double kq =
      ((l4 & 1) ? ((double)npix - 0.5 - bb) : (-0.5 - bb)) /
      (l4 < 2 ? ahx : ahy);  // unused where the divisor is 0
  int c0 = -K, c1 = K;
  {
    const int ax_i = lane & 1;
    const double ka = __shfl_sync(kFull, kq, 2 * ax_i);
    const double kb = __shfl_sync(kFull, kq, 2 * ax_i + 1);
    const double ah = ax_i ? ahy : ahx;
    const float bf = ax_i ? byf : bxf;
    if (ah != 0.0) {
      double f0 = floor(fmin(ka, kb)) - 2.0, f1 = ceil(fmax(ka, kb)) + 2.0;
      f0 = fmin(fmax(f0, (double)-K), (double)K + 1.0);
      f1 = fmin(fmax(f1, (double)-K - 1.0), (double)K);
      c0 = (int)f0;
      c1 = (int)f1;
    } else if (!(bf > lo && bf < hi)) {  // a = 0: p = b for every sample
      c1 = -K - 1;
    }
  }
  const int k0 = max(__shfl_sync(kFull, c0, 0), __shfl_sync(kFull, c0, 1));
  const int k1 = min(__shfl_sync(kFull, c1, 0), __shfl_sync(kFull, c1, 1));
  detect_line(As ? As[mi] : A0, npix, lane, K, k0, k1, axf, ayf, bxf, byf, hf,
              h, sh, r, max_peaks, w, count, pos, height, err);
}

// Entry (line j, slot) of the peak-aligned line grid, one thread each.
// mode 0: one slot, the line itself; mode 1 (one peak time): slot m = the
// line's m-th kept peak, whose time along the trajectory is the grid t0
// (shift = its tau from the origin's closest approach); mode 2 (two peak
// times): slot = the pair (a, b), a < b, of kept peaks, tE by Eq. 8 and the
// grid t0 at peak a.  keep = 1 for a slot in use, else 0.
__global__ void k_peak_entries(int n_lines, const double *__restrict__ lu,
                               const double *__restrict__ lc,
                               const double *__restrict__ ls,
                               const double *__restrict__ lsh,
                               const double *__restrict__ la,
                               const int *__restrict__ count,
                               const double *__restrict__ pos, int P,
                               int mode, int need, double tp0, double tp1,
                               PeakEntries E) {
  const int S = mode == 0 ? 1 : mode == 1 ? P : P * (P - 1) / 2;
  const long long n = (long long)n_lines * S;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / S), slot = (int)(e - (long long)j * S);
    const int cnt = count[j];
    const int kept = cnt < P ? cnt : P;
    const bool ok = cnt >= need;
    E.u[e] = lu[j];
    E.c[e] = lc[j];
    E.s[e] = ls[j];
    E.alpha[e] = la[j];
    double shift = 0.0, tE = 1.0;
    bool used;
    if (mode == 0) {
      used = ok;
      shift = lsh[j];
    } else if (mode == 1) {
      used = ok && slot < kept;
      if (used) shift = __dadd_rn(pos[(size_t)j * P + slot], lsh[j]);
    } else {
      int a = 0, t = slot;
      while (t >= P - 1 - a) {  // row a holds the pairs (a, a+1 .. P-1)
        t -= P - 1 - a;
        ++a;
      }
      const int b = a + 1 + t;
      used = ok && b < kept;
      if (used) {
        const double pa = pos[(size_t)j * P + a], pb = pos[(size_t)j * P + b];
        shift = __dadd_rn(pa, lsh[j]);
        tE = __ddiv_rn(__dsub_rn(tp1, tp0), __dsub_rn(pb, pa));
      }
    }
    E.shift[e] = shift;
    if (E.tE) E.tE[e] = tE;
    E.keep[e] = used ? 1.0 : 0.0;
  }
}

}  // namespace

cudaError_t launch_line_peaks(const float *A, const float *const *As,
                              int n_maps, int npix, double L,
                              const double *lu, const double *lc,
                              const double *ls, const double *lsh,
                              int n_lines, int sub, float r, int max_peaks,
                              int *count, double *pos, double *height,
                              unsigned *err, cudaStream_t st) {
  const long long warps = (long long)n_lines * n_maps;
  if (warps <= 0) return cudaSuccess;
  const long long blocks = (warps + kPkWarps - 1) / kPkWarps;
  // texel size and step, each one correctly rounded FP64 operation
  const double dlt = (2.0 * L) / (double)npix;
  const double h = dlt / (double)sub;
  k_line_peaks<<<(unsigned)blocks, kPkWarps * 32, 0, st>>>(
      A, As, n_maps, npix, L, dlt, h, lu, lc, ls, lsh, n_lines, sub, r,
      max_peaks, count, pos, height, err);
  return cudaGetLastError();
}

cudaError_t launch_peak_entries(int n_lines, const double *lu,
                                const double *lc, const double *ls,
                                const double *lsh, const double *la,
                                const int *count, const double *pos, int P,
                                int mode, int need, double tp0, double tp1,
                                const PeakEntries &E, cudaStream_t st) {
  const int S = mode == 0 ? 1 : mode == 1 ? P : P * (P - 1) / 2;
  const long long n = (long long)n_lines * S;
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_peak_entries<<<(unsigned)blocks, 256, 0, st>>>(n_lines, lu, lc, ls, lsh,
                                                    la, count, pos, P, mode,
                                                    need, tp0, tp1, E);
  return cudaGetLastError();
}

}  // namespace morse
