// Adjoint gradient of the profiled chi^2 and the batched Levenberg-Marquardt
// refinement of grid minima.
//
// The paper refines its coarse-grid seeds (§4.4) by MCMC with finite-source
// magnifications (§5).  This library refines them on the same point-source
// map instead: chi^2(theta), theta = (t0, tE, u0, alpha), with (Fs, Fb)
// profiled out by the 2x2 solve of Eq. 6.  Because (Fs, Fb) minimise chi^2
// for every theta, the envelope theorem gives
//     d chi^2 / d theta_k = sum_i -2 w_i r_i Fs dA_i/dtheta_k,
// r_i = F_i - Fs A_i - Fb, and the Gauss-Newton matrix
//     H_kl = sum_i w_i Fs^2 (dA_i/dtheta_k)(dA_i/dtheta_l).
// dA/dtheta follows the lookup: inside the map the bilinear gradient in
// pixel units times dy/dtheta / Delta; outside, the single-lens dA/du times
// du/dtheta.  With tau = (t - t0)/tE, y = tau (c, s) + u0 (-s, c),
// (c, s) = (cos alpha, sin alpha), G = grad_y A, Gp = G.(c, s) and
// Gn = G.(-s, c):
//     dA/dt0 = -Gp / tE,   dA/dtE = -tau Gp / tE,
//     dA/du0 = Gn,         dA/dalpha = tau Gn - u0 Gp.
// One warp per trajectory; FP32 per lane, FP64 across lanes.
// Inside-map epoch loops unrolled four times: the sweeps wait on texel
// gathers from L2, and four independent gathers per warp are in flight.
#ifndef MORSE_UNROLL
#define MORSE_UNROLL 4
#endif
#include <cuda_runtime.h>
#include <math_constants.h>

#include "morse_internal.cuh"
#include "search_common.cuh"

namespace morse {

namespace {

using namespace dev;

// GB300 design.  A block of kAdjWarps warps takes kAdjWarps trajectories,
// one warp each for the two epoch sweeps (lanes over epochs, as the search).
// The per-trajectory FP64 work -- sin/cos of alpha, the track constants and
// epoch ranges, the 2x2 solve, and the final assembly of the gradient and
// the Gauss-Newton matrix -- is done by warp 0 with one lane per
// trajectory: GB300's FP64 rate is 1/73 of its FP32 rate, and a warp-wide
// FP64 instruction costs the same whether one lane or 32 need it.  The
// light curve is staged in shared memory when it fits.
//
// Sweep 1 is the search's phase 1 (same device function, same sums), so
// Fs, Fb and chi^2 at a grid point equal the search's to the last bit.
// Sweep 2 takes the residuals r = F - Fs A - Fb (chi^2 summed as the
// search's phase 2 sums it) and accumulates the gradient in the map's
// pixel axes: with g = (gx, gy) = Delta grad_y A (the bilinear cell's
// slopes inside the map, Delta D y with D = (dA/du)/u outside),
// X1 = sum w r gx, Y1 = sum w r gy, X2 = sum w r tau gx, Y2 = sum w r tau gy.
// Rotated once per trajectory into the track's axes, Gp = g.(c, s)/Delta
// and Gn = g.(-s, c)/Delta, they give every component of
//     d chi^2/d theta = -2 Fs sum w r dA/dtheta,
//     dA/dt0 = -Gp/tE, dA/dtE = -tau Gp/tE, dA/du0 = Gn,
//     dA/dalpha = tau Gn - u0 Gp,
// with 7 FP32 instructions per epoch beyond the residual.  The Gauss-Newton
// matrix likewise from the nine sums w tau^m g_a g_b (m = 0, 1, 2).
constexpr int kAdjWarps = 16;          // warps (trajectories) per block
constexpr int kAdjEpSmemMax = 6144;    // epochs staged in shared memory

struct AdjTraj {
  TrajC c;
  float cs, sn, u0, dD;  // direction, u0, Delta (FP32)
  double kt, u0d, csd, snd;
  const float4 *quad;    // the trajectory's map (cell table)
};

struct AdjSums {
  float x1, y1, x2, y2;  // sum w r g, sum w r tau g (pixel axes)
  float h[9];            // sum w tau^m g_a g_b: m-major, (xx, xy, yy)
};

template <bool WITH_H>
__device__ __forceinline__ void adj_add(AdjSums &a, float &chi, float w,
                                        float fc, float Ac, float tau,
                                        float gx, float gy, float Fs,
                                        float Bc) {
  const float r = __fsub_rn(fc, __fmaf_rn(Fs, Ac, Bc));
  const float wr = __fmul_rn(w, r);
  chi = __fmaf_rn(wr, r, chi);
  const float wrt = __fmul_rn(wr, tau);
  a.x1 = __fmaf_rn(wr, gx, a.x1);
  a.y1 = __fmaf_rn(wr, gy, a.y1);
  a.x2 = __fmaf_rn(wrt, gx, a.x2);
  a.y2 = __fmaf_rn(wrt, gy, a.y2);
  if (WITH_H) {
    const float wgx = __fmul_rn(w, gx), wgy = __fmul_rn(w, gy);
    const float pxx = __fmul_rn(wgx, gx), pxy = __fmul_rn(wgx, gy);
    const float pyy = __fmul_rn(wgy, gy);
    const float t2 = __fmul_rn(tau, tau);
    a.h[0] = __fadd_rn(a.h[0], pxx);
    a.h[1] = __fadd_rn(a.h[1], pxy);
    a.h[2] = __fadd_rn(a.h[2], pyy);
    a.h[3] = __fmaf_rn(tau, pxx, a.h[3]);
    a.h[4] = __fmaf_rn(tau, pxy, a.h[4]);
    a.h[5] = __fmaf_rn(tau, pyy, a.h[5]);
    a.h[6] = __fmaf_rn(t2, pxx, a.h[6]);
    a.h[7] = __fmaf_rn(t2, pxy, a.h[7]);
    a.h[8] = __fmaf_rn(t2, pyy, a.h[8]);
  }
}

// A - 1, tau and the pixel-axis gradient of an epoch outside the map
// (single lens in u^2 = tau^2 + u0^2, the search's arithmetic for A)
__device__ __forceinline__ float out_point(const AdjTraj &T, float t,
                                           float &tau, float &gx, float &gy) {
  tau = __fmaf_rn(T.c.kt, t, T.c.bt);
  const float u2 = __fmaf_rn(tau, tau, T.c.u02);
  const float rr = rsqrt_approx(__fmul_rn(u2, __fadd_rn(u2, 4.f)));
  const float am1 = __fsub_rn(__fmul_rn(__fadd_rn(u2, 2.f), rr), 1.f);
  // Delta D, D = (dA/du)/u = -8 (u^2 (u^2 + 4))^(-3/2)
  const float dD = __fmul_rn(__fmul_rn(-8.f, T.dD),
                             __fmul_rn(rr, __fmul_rn(rr, rr)));
  const float y1 = __fmaf_rn(tau, T.cs, -__fmul_rn(T.u0, T.sn));
  const float y2 = __fmaf_rn(tau, T.sn, __fmul_rn(T.u0, T.cs));
  gx = __fmul_rn(dD, y1);
  gy = __fmul_rn(dD, y2);
  return am1;
}

// A - 1, tau and the pixel-axis gradient inside the map (the search's
// bilinear lookup; the cell's slopes at (fx, fy))
__device__ __forceinline__ float in_point(const SearchParams &P,
                                          const AdjTraj &T, float t,
                                          float &tau, float &gx, float &gy) {
  const float vx = __fmaf_rn(T.c.ax, t, T.c.bx);
  const float vy = __fmaf_rn(T.c.ay, t, T.c.by);
  tau = __fmaf_rn(T.c.kt, t, T.c.bt);
  TexPos p;
  if (!tex_pos(P, vx, vy, p)) {
    gx = gy = 0.f;
    return 0.f;
  }
  const float4 q = __ldg(&P.quad[p.idx]);
  const float r0 = __fmaf_rn(p.fx, q.y, q.x);
  const float dr = __fmaf_rn(p.fx, q.w, q.z);
  gx = __fmaf_rn(p.fy, q.w, q.y);
  gy = dr;
  return __fmaf_rn(p.fy, dr, r0);
}

__device__ __forceinline__ float warp_sum_f32(float x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x = __fadd_rn(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

// theta_i = (t0, tE, u0, alpha) with absolute t0, on the map P.quad or,
// when tq is set, on the map tq[i] (maps of one geometry).  Outputs (any
// may be null): chi2[i], grad[4 i + k], H[10 i + m] (upper triangle,
// row-major), Fs[i], Fb[i], flags[i].
template <bool WITH_H, bool EP_SMEM>
__global__ void __launch_bounds__(kAdjWarps * 32, 2)
    k_theta(const SearchParams P, const double *__restrict__ theta,
            const float4 *const *__restrict__ tq, int n, double t_ref,
            double *chi2, double *grad, double *H, double *Fs, double *Fb,
            int *flags) {
  extern __shared__ __align__(16) float4 s_ep[];
  __shared__ AdjTraj s_tr[kAdjWarps];
  __shared__ Acc s_acc[kAdjWarps];
  __shared__ double s_Fs[kAdjWarps], s_Bc[kAdjWarps];
  __shared__ int s_deg[kAdjWarps];
  __shared__ AdjSums s_sum[kAdjWarps];
  __shared__ double s_chi[kAdjWarps];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int i0 = blockIdx.x * kAdjWarps;
  const int i = i0 + warp;
  if (EP_SMEM)
    for (int e = threadIdx.x; e < P.n_ep; e += blockDim.x) s_ep[e] = P.ep[e];
  // set-up, one lane per trajectory (the epoch ranges from the global copy:
  // the shared one is still being written)
  if (warp == 0 && lane < kAdjWarps && i0 + lane < n) {
    const int j = i0 + lane;
    const double t0 = theta[4 * j + 0], tE = theta[4 * j + 1];
    const double u0 = theta[4 * j + 2], al = theta[4 * j + 3];
    double sn, cs;
    sincos(al, &sn, &cs);
    const double tEc = (tE > 1e-6) ? tE : 1e-6;  // the host rejects tE <= 0
    double tlo, thi;
    slab_tau(P.L, u0, cs, sn, tlo, thi);
    AdjTraj T;
    T.c = make_traj(P, epochs_at(P.ep, P.n_ep), u0, cs, sn, t0 - t_ref,
                    1.0 / (tEc * P.dlt), tEc, tlo, thi);
    T.cs = (float)cs;
    T.sn = (float)sn;
    T.u0 = (float)u0;
    T.dD = P.dltf;
    T.kt = 1.0 / tEc;
    T.u0d = u0;
    T.csd = cs;
    T.snd = sn;
    T.quad = tq ? tq[j] : P.quad;
    s_tr[lane] = T;
  }
  __syncthreads();
  const Epochs ep = epochs_at(EP_SMEM ? s_ep : P.ep, P.n_ep);
  const bool live = i < n;
  AdjTraj T;
  if (live) T = s_tr[warp];
  SearchParams Q = P;  // this warp's map
  Q.quad = live ? T.quad : P.quad;
  // sweep 1: the normal-equation sums (the search's phase 1)
  if (live) {
    const Acc a = phase1<false>(Q, ep, T.c, lane);
    if (lane == 0) s_acc[warp] = a;
  }
  __syncthreads();
  if (warp == 0 && lane < kAdjWarps && i0 + lane < n) {
    const Acc a = s_acc[lane];
    const Fit2 f = fit2(P, (double)a.a, (double)a.b, (double)a.d);
    s_Fs[lane] = f.Fs;
    s_Bc[lane] = f.Bc;
    s_deg[lane] = f.degenerate ? 1 : 0;
  }
  __syncthreads();
  // sweep 2: residuals, chi^2 and the gradient (and Gauss-Newton) sums
  if (live) {
    const float fFs = __double2float_rn(s_Fs[warp]);
    const float fBc = __double2float_rn(s_Bc[warp]);
    AdjSums a;
    a.x1 = a.y1 = a.x2 = a.y2 = 0.f;
#pragma unroll
    for (int k = 0; k < 9; ++k) a.h[k] = 0.f;
    float chi = 0.f;
#pragma unroll 2
    for (int e = lane_start(0, lane); e < T.c.e_in; e += 32) {
      const float2 v = ep.tw[e];
      float tau, gx, gy;
      const float Ac = out_point(T, v.x, tau, gx, gy);
      adj_add<WITH_H>(a, chi, v.y, ep.fc[e], Ac, tau, gx, gy, fFs, fBc);
    }
#pragma unroll kUnroll
    for (int e = lane_start(T.c.e_in, lane); e < T.c.e_out; e += 32) {
      const float2 v = ep.tw[e];
      float tau, gx, gy;
      const float Ac = in_point(Q, T, v.x, tau, gx, gy);
      adj_add<WITH_H>(a, chi, v.y, ep.fc[e], Ac, tau, gx, gy, fFs, fBc);
    }
#pragma unroll 2
    for (int e = lane_start(T.c.e_out, lane); e < P.n_ep; e += 32) {
      const float2 v = ep.tw[e];
      float tau, gx, gy;
      const float Ac = out_point(T, v.x, tau, gx, gy);
      adj_add<WITH_H>(a, chi, v.y, ep.fc[e], Ac, tau, gx, gy, fFs, fBc);
    }
    // chi^2 across lanes in FP64 (as the search's phase 2), the rest FP32
    double x = (double)chi;
#pragma unroll
    for (int o = 16; o; o >>= 1) x = __dadd_rn(x, __shfl_xor_sync(kFull, x, o));
    a.x1 = warp_sum_f32(a.x1);
    a.y1 = warp_sum_f32(a.y1);
    a.x2 = warp_sum_f32(a.x2);
    a.y2 = warp_sum_f32(a.y2);
    if (WITH_H) {
#pragma unroll
      for (int k = 0; k < 9; ++k) a.h[k] = warp_sum_f32(a.h[k]);
    }
    if (lane == 0) {
      s_chi[warp] = x;
      s_sum[warp] = a;
    }
  }
  __syncthreads();
  // assembly of the outputs, one lane per trajectory
  if (warp == 0 && lane < kAdjWarps && i0 + lane < n) {
    const int j = i0 + lane;
    const AdjTraj &Tj = s_tr[lane];
    const AdjSums &a = s_sum[lane];
    const double c = Tj.csd, s = Tj.snd, u0 = Tj.u0d, kt = Tj.kt;
    const double iD = P.invD, fs = s_Fs[lane];
    const double P1 = (c * a.x1 + s * a.y1) * iD;
    const double N1 = (c * a.y1 - s * a.x1) * iD;
    const double P2 = (c * a.x2 + s * a.y2) * iD;
    const double N2 = (c * a.y2 - s * a.x2) * iD;
    const double x2 = s_chi[lane];
    if (chi2) chi2[j] = isnan(x2) ? CUDART_INF : x2;
    if (grad) {
      const double m2 = -2.0 * fs;
      grad[4 * j + 0] = m2 * (-kt * P1);
      grad[4 * j + 1] = m2 * (-kt * P2);
      grad[4 * j + 2] = m2 * N1;
      grad[4 * j + 3] = m2 * (N2 - u0 * P1);
    }
    if (WITH_H && H) {
      const double d2 = iD * iD, f2 = fs * fs;
      double spp[3], spn[3], snn[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const double xx = a.h[3 * m], xy = a.h[3 * m + 1], yy = a.h[3 * m + 2];
        spp[m] = (c * c * xx + 2.0 * c * s * xy + s * s * yy) * d2;
        snn[m] = (s * s * xx - 2.0 * c * s * xy + c * c * yy) * d2;
        spn[m] = (c * s * (yy - xx) + (c * c - s * s) * xy) * d2;
      }
      double *h = H + 10 * (size_t)j;
      h[0] = f2 * kt * kt * spp[0];
      h[1] = f2 * kt * kt * spp[1];
      h[2] = f2 * -kt * spn[0];
      h[3] = f2 * -kt * (spn[1] - u0 * spp[0]);
      h[4] = f2 * kt * kt * spp[2];
      h[5] = f2 * -kt * spn[1];
      h[6] = f2 * -kt * (spn[2] - u0 * spp[1]);
      h[7] = f2 * snn[0];
      h[8] = f2 * (snn[1] - u0 * spn[0]);
      h[9] = f2 * (snn[2] - 2.0 * u0 * spn[1] + u0 * u0 * spp[0]);
    }
    if (Fs) Fs[j] = fs;
    if (Fb) Fb[j] = s_Bc[lane] + P.Fref - fs;
    if (flags) flags[j] = s_deg[lane] ? MORSE_FIT_DEGENERATE : 0;
  }
}

// Solve (H + lam diag(H) + eps I) x = b for a 4x4 symmetric H given as its
// upper triangle; Cholesky in FP64.  Returns false if not positive definite.
__device__ bool lm_solve(const double *h, double lam, const double *b,
                         double *x) {
  double M[4][4];
  int m = 0;
  for (int k = 0; k < 4; ++k)
    for (int l = k; l < 4; ++l) {
      M[k][l] = M[l][k] = h[m];
      ++m;
    }
  for (int k = 0; k < 4; ++k) M[k][k] = M[k][k] * (1.0 + lam) + 1e-300;
  double L[4][4] = {{0}};
  for (int j = 0; j < 4; ++j) {
    double sum = M[j][j];
    for (int k = 0; k < j; ++k) sum -= L[j][k] * L[j][k];
    if (!(sum > 0.0)) return false;
    L[j][j] = sqrt(sum);
    for (int i2 = j + 1; i2 < 4; ++i2) {
      double t = M[i2][j];
      for (int k = 0; k < j; ++k) t -= L[i2][k] * L[j][k];
      L[i2][j] = t / L[j][j];
    }
  }
  double y[4];
  for (int i2 = 0; i2 < 4; ++i2) {
    double t = b[i2];
    for (int k = 0; k < i2; ++k) t -= L[i2][k] * y[k];
    y[i2] = t / L[i2][i2];
  }
  for (int i2 = 3; i2 >= 0; --i2) {
    double t = y[i2];
    for (int k = i2 + 1; k < 4; ++k) t -= L[k][i2] * x[k];
    x[i2] = t / L[i2][i2];
  }
  return true;
}

// One Levenberg-Marquardt step per trajectory (one thread each).  The
// evaluation at theta_cur is accepted if it lowered chi^2 (damping / 3) or
// rejected (damping x 4, back to theta_best); then the next point is
// theta_best - (H + lam diag H)^-1 g at the best point.
__global__ void k_lm_step(RefineState S, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double lam = S.lam[i];
  const double c = S.chi2_cur[i];
  if (c < S.chi2_best[i]) {
    S.chi2_best[i] = c;
    for (int k = 0; k < 4; ++k) {
      S.th_best[4 * i + k] = S.th_cur[4 * i + k];
      S.g_best[4 * i + k] = S.g_cur[4 * i + k];
    }
    for (int k = 0; k < 10; ++k) S.H_best[10 * i + k] = S.H_cur[10 * i + k];
    lam = fmax(lam / 3.0, 1e-12);
  } else {
    lam = fmin(lam * 4.0, 1e12);
  }
  double neg_g[4], dx[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4; ++k) neg_g[k] = -S.g_best[4 * i + k];
  bool ok = false;
  for (int tries = 0; tries < 8 && !ok; ++tries) {
    ok = lm_solve(S.H_best + 10 * i, lam, neg_g, dx);
    if (!ok) lam = fmin(lam * 10.0, 1e12);
  }
  if (!ok)
    for (int k = 0; k < 4; ++k) dx[k] = 0.0;
  S.lam[i] = lam;
  for (int k = 0; k < 4; ++k)
    S.th_cur[4 * i + k] = S.th_best[4 * i + k] + dx[k];
  // keep tE positive
  const double tE = S.th_cur[4 * i + 1];
  const double tEb = S.th_best[4 * i + 1];
  if (!(tE > 0.05 * tEb)) S.th_cur[4 * i + 1] = 0.5 * tEb;
}

__global__ void k_lm_init(RefineState S, const morse_fit *starts, int n,
                          double lam0) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const morse_fit f = starts[i];
  S.th_cur[4 * i + 0] = f.t0;
  S.th_cur[4 * i + 1] = f.tE;
  S.th_cur[4 * i + 2] = f.u0;
  S.th_cur[4 * i + 3] = f.alpha;
  for (int k = 0; k < 4; ++k) S.th_best[4 * i + k] = S.th_cur[4 * i + k];
  S.chi2_best[i] = CUDART_INF;
  S.lam[i] = lam0;
}

// records of the refined trajectories: theta_best, its chi^2 and fluxes
__global__ void k_lm_finish(RefineState S, const morse_fit *starts, int n,
                            morse_fit *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  morse_fit f;
  f.t0 = S.th_best[4 * i + 0];
  f.tE = S.th_best[4 * i + 1];
  f.u0 = S.th_best[4 * i + 2];
  f.alpha = S.th_best[4 * i + 3];
  f.chi2 = S.chi2_cur[i];
  f.Fs = S.Fs[i];
  f.Fb = S.Fb[i];
  f.idx = starts[i].idx;
  f.flags = S.flags[i] | MORSE_FIT_REFINED;
  f.reserved = 0;
  out[i] = f;
}

}  // namespace

template <bool WITH_H>
static cudaError_t launch_theta_h(const SearchParams &P, const double *theta,
                                  const float4 *const *tq, int n,
                                  double t_ref, double *chi2, double *grad,
                                  double *H, double *Fs, double *Fb,
                                  int *flags, cudaStream_t st) {
  const int threads = kAdjWarps * 32;
  const int blocks = (n + kAdjWarps - 1) / kAdjWarps;
  if (P.n_ep <= kAdjEpSmemMax)
    k_theta<WITH_H, true><<<blocks, threads, sizeof(float4) * P.n_ep, st>>>(
        P, theta, tq, n, t_ref, chi2, grad, H, Fs, Fb, flags);
  else
    k_theta<WITH_H, false><<<blocks, threads, 0, st>>>(
        P, theta, tq, n, t_ref, chi2, grad, H, Fs, Fb, flags);
  return cudaGetLastError();
}

cudaError_t adjoint_setup() {
  const int bytes = (int)(sizeof(float4) * kAdjEpSmemMax);
  cudaError_t e = cudaFuncSetAttribute(
      k_theta<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_theta<false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  return e;
}

cudaError_t launch_theta(const SearchParams &P, const double *theta, int n,
                         double t_ref, double *chi2, double *grad, double *H,
                         double *Fs, double *Fb, int *flags, cudaStream_t st,
                         const float4 *const *tq) {
  if (n <= 0) return cudaSuccess;
  if (H)
    return launch_theta_h<true>(P, theta, tq, n, t_ref, chi2, grad, H, Fs,
                                Fb, flags, st);
  return launch_theta_h<false>(P, theta, tq, n, t_ref, chi2, grad, nullptr,
                               Fs, Fb, flags, st);
}

cudaError_t launch_lm_init(const RefineState &S, const morse_fit *starts,
                           int n, double lam0, cudaStream_t st) {
  k_lm_init<<<(n + 127) / 128, 128, 0, st>>>(S, starts, n, lam0);
  return cudaGetLastError();
}

cudaError_t launch_lm_step(const RefineState &S, int n, cudaStream_t st) {
  k_lm_step<<<(n + 127) / 128, 128, 0, st>>>(S, n);
  return cudaGetLastError();
}

cudaError_t launch_lm_finish(const RefineState &S, const morse_fit *starts,
                             int n, morse_fit *out, cudaStream_t st) {
  k_lm_finish<<<(n + 127) / 128, 128, 0, st>>>(S, starts, n, out);
  return cudaGetLastError();
}

}  // namespace morse
