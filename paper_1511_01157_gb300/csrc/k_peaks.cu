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
// GB300 design: one warp per line.  The lanes evaluate 32 consecutive
// samples at once (the line's texels stream through L1/L2, the map having
// just been built), then lane 0 runs the sequential peak detector over
// them from shared memory and keeps the highest peaks in a short sorted
// list there.  A line has at most 2 sub npix sqrt(2) samples inside the
// map, so a line costs a few tens of microseconds and every line of a grid
// runs at once.  The expansion into trajectory entries is one thread per
// (line, slot).
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"

namespace morse {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kPkWarps = 4;

__global__ void __launch_bounds__(kPkWarps * 32)
    k_line_peaks(const float *__restrict__ A, int npix, double L,
                 const double *__restrict__ lu, const double *__restrict__ lc,
                 const double *__restrict__ ls, const double *__restrict__ lsh,
                 int n_lines, int sub, float r, int max_peaks,
                 int *__restrict__ count, double *__restrict__ pos,
                 double *__restrict__ height, unsigned *__restrict__ err) {
  __shared__ float s_v[kPkWarps][32];
  __shared__ float s_kh[kPkWarps][kPeakMax];
  __shared__ int s_kk[kPkWarps][kPeakMax];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int line = blockIdx.x * kPkWarps + w;
  if (line >= n_lines) return;  // warp-uniform; the kernel has no barrier
  const double u = lu[line], c = lc[line], s = ls[line], sh = lsh[line];
  // the line in texel coordinates, p = a tau + b, in FP64 then FP32
  const double dlt = __ddiv_rn(__dmul_rn(2.0, L), (double)npix);
  const double h = __ddiv_rn(dlt, (double)sub);
  const double ax = __ddiv_rn(c, dlt), ay = __ddiv_rn(s, dlt);
  const double bx =
      __dsub_rn(__ddiv_rn(__dsub_rn(L, __dmul_rn(u, s)), dlt), 0.5);
  const double by =
      __dsub_rn(__ddiv_rn(__dadd_rn(L, __dmul_rn(u, c)), dlt), 0.5);
  const float axf = __double2float_rn(ax), ayf = __double2float_rn(ay);
  const float bxf = __double2float_rn(bx), byf = __double2float_rn(by);
  const float hf = __double2float_rn(h);
  const float lo = -0.5f, hi = (float)npix - 0.5f, pmax = (float)(npix - 1);
  const int K = sub * npix;
  // Samples inside the map form one run of k (p is monotone in k); a
  // superset of it from the FP64 line, two samples wider on each side.
  int k0 = -K, k1 = K;
  auto clip = [&](double a, double b, float bf) {
    const double ah = a * h;
    if (ah != 0.0) {
      const double ka = (-0.5 - b) / ah, kb = ((double)npix - 0.5 - b) / ah;
      double f0 = floor(fmin(ka, kb)) - 2.0, f1 = ceil(fmax(ka, kb)) + 2.0;
      f0 = fmin(fmax(f0, (double)-K), (double)K + 1.0);
      f1 = fmin(fmax(f1, (double)-K - 1.0), (double)K);
      k0 = max(k0, (int)f0);
      k1 = min(k1, (int)f1);
    } else if (!(bf > lo && bf < hi)) {  // a = 0: p = b for every sample
      k1 = k0 - 1;
    }
  };
  clip(ax, bx, bxf);
  clip(ay, by, byf);
  int cnt = 0, nkept = 0, kmx = 0;
  bool look_max = false;
  float mn = CUDART_INF_F, mx = -CUDART_INF_F;
  for (int kb = k0; kb <= k1; kb += 32) {
    const int k = kb + lane;
    float v = 0.f;
    bool in = false;
    if (k <= k1) {
      const float tk = __fmul_rn((float)k, hf);
      const float px = __fadd_rn(__fmul_rn(axf, tk), bxf);
      const float py = __fadd_rn(__fmul_rn(ayf, tk), byf);
      in = px > lo && px < hi && py > lo && py < hi;
      if (in) {
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
        v = __fadd_rn(__fmul_rn(gy, r0), __fmul_rn(fy, r1));
      }
    }
    const unsigned m = __ballot_sync(kFull, in);
    // the superset must start and end outside the map (unless it reaches
    // the ends of the sampled range): otherwise samples were missed
    if (lane == 0) {
      if (kb == k0 && (m & 1u) && k0 > -K) atomicOr(err, 1u);
      if (k1 - kb < 32 && ((m >> (k1 - kb)) & 1u) && k1 < K)
        atomicOr(err, 1u);
    }
    s_v[w][lane] = v;
    __syncwarp();
    if (lane == 0) {
      for (unsigned mm = m; mm; mm &= mm - 1) {
        const int i = __ffs(mm) - 1;
        const float x = s_v[w][i];
        if (look_max) {
          if (x > mx) {
            mx = x;
            kmx = kb + i;
          } else if (mx > __fmul_rn(r, x)) {
            // a peak; kept if among the max_peaks highest (ties: earlier)
            ++cnt;
            int at = nkept;
            while (at > 0 && mx > s_kh[w][at - 1]) --at;
            if (at < max_peaks) {
              const int last = nkept < max_peaks ? nkept : max_peaks - 1;
              for (int q = last; q > at; --q) {
                s_kh[w][q] = s_kh[w][q - 1];
                s_kk[w][q] = s_kk[w][q - 1];
              }
              s_kh[w][at] = mx;
              s_kk[w][at] = kmx;
              if (nkept < max_peaks) ++nkept;
            }
            look_max = false;
            mn = x;
          }
        } else {
          if (x < mn) {
            mn = x;
          } else if (x > __fmul_rn(r, mn)) {
            look_max = true;
            mx = x;
            kmx = kb + i;
          }
        }
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    // kept peaks in increasing tau
    for (int a = 1; a < nkept; ++a)
      for (int b = a; b > 0 && s_kk[w][b] < s_kk[w][b - 1]; --b) {
        const int ti = s_kk[w][b];
        s_kk[w][b] = s_kk[w][b - 1];
        s_kk[w][b - 1] = ti;
        const float tf = s_kh[w][b];
        s_kh[w][b] = s_kh[w][b - 1];
        s_kh[w][b - 1] = tf;
      }
    count[line] = cnt;
    for (int q = 0; q < max_peaks; ++q) {
      const size_t o = (size_t)line * max_peaks + q;
      if (q < nkept) {
        pos[o] = __dsub_rn(__dmul_rn((double)s_kk[w][q], h), sh);
        height[o] = (double)s_kh[w][q];
      } else {
        pos[o] = CUDART_NAN;
        height[o] = CUDART_NAN;
      }
    }
  }
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

cudaError_t launch_line_peaks(const float *A, int npix, double L,
                              const double *lu, const double *lc,
                              const double *ls, const double *lsh,
                              int n_lines, int sub, float r, int max_peaks,
                              int *count, double *pos, double *height,
                              unsigned *err, cudaStream_t st) {
  if (n_lines <= 0) return cudaSuccess;
  const int blocks = (n_lines + kPkWarps - 1) / kPkWarps;
  k_line_peaks<<<blocks, kPkWarps * 32, 0, st>>>(A, npix, L, lu, lc, ls, lsh,
                                                 n_lines, sub, r, max_peaks,
                                                 count, pos, height, err);
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
