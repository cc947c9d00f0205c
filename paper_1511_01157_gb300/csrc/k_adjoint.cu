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
#include <cuda_runtime.h>
#include <math_constants.h>

#include "morse_internal.cuh"
#include "search_common.cuh"

namespace morse {

namespace {

using namespace dev;

constexpr int kAdjWarps = 8;  // warps (trajectories) per block

struct Deriv {
  float d[4];
};

// A - 1 and dA/dtheta at time t inside the map
__device__ __forceinline__ float in_grad(const SearchParams &P, const TrajC &c,
                                         float cs, float sn, float u0,
                                         float t, Deriv &g) {
  const float vx = __fmaf_rn(c.ax, t, c.bx), vy = __fmaf_rn(c.ay, t, c.by);
  TexPos p;
  if (!tex_pos(P, vx, vy, p)) {
    g.d[0] = g.d[1] = g.d[2] = g.d[3] = 0.f;
    return 0.f;
  }
  const float4 q = __ldg(&P.quad[p.idx]);
  // q = (m00, m10 - m00, m01 - m00, second difference)
  const float r0 = __fmaf_rn(p.fx, q.y, q.x);
  const float dr = __fmaf_rn(p.fx, q.w, q.z);  // row difference at fx
  const float am1 = __fmaf_rn(p.fy, dr, r0);
  // gradient in pixel units; the edge cells below and above the map have
  // zero differences across the edge, so the gradient there is zero along
  // that axis (the lookup is constant)
  const float gx = __fmaf_rn(p.fy, q.w, q.y);
  const float gy = dr;
  // per unit of y: divide by Delta
  const float Gx = __fmul_rn(gx, P.invDf), Gy = __fmul_rn(gy, P.invDf);
  const float Gp = __fmaf_rn(Gx, cs, __fmul_rn(Gy, sn));
  const float Gn = __fmaf_rn(Gy, cs, -__fmul_rn(Gx, sn));
  const float tau = __fmaf_rn(c.kt, t, c.bt);
  g.d[0] = -__fmul_rn(Gp, c.kt);
  g.d[1] = __fmul_rn(tau, g.d[0]);
  g.d[2] = Gn;
  g.d[3] = __fmaf_rn(tau, Gn, -__fmul_rn(u0, Gp));
  return am1;
}

// A - 1 and dA/dtheta at time t outside the map (single lens in
// u^2 = tau^2 + u0^2): dA/du / u = -8 (u^2 (u^2 + 4))^(-3/2)
__device__ __forceinline__ float out_grad(const TrajC &c, float u0, float t,
                                          Deriv &g) {
  const float tau = __fmaf_rn(c.kt, t, c.bt);
  const float u2 = __fmaf_rn(tau, tau, c.u02);
  const float rr = rsqrt_approx(__fmul_rn(u2, __fadd_rn(u2, 4.f)));
  const float am1 = __fsub_rn(__fmul_rn(__fadd_rn(u2, 2.f), rr), 1.f);
  const float D = __fmul_rn(-8.f, __fmul_rn(rr, __fmul_rn(rr, rr)));
  g.d[0] = __fmul_rn(D, -__fmul_rn(tau, c.kt));
  g.d[1] = __fmul_rn(g.d[0], tau);
  g.d[2] = __fmul_rn(D, u0);
  g.d[3] = 0.f;
  return am1;
}

struct GradAcc {
  float chi, g[4], h[10];
};

template <bool WITH_H>
__device__ __forceinline__ void grad_add(GradAcc &a, float w, float fc,
                                         float Ac, const Deriv &d, float Fs,
                                         float Bc) {
  const float r = __fsub_rn(fc, __fmaf_rn(Fs, Ac, Bc));
  const float wr = __fmul_rn(w, r);
  a.chi = __fmaf_rn(wr, r, a.chi);
  const float s = __fmul_rn(-2.f, __fmul_rn(wr, Fs));
#pragma unroll
  for (int k = 0; k < 4; ++k) a.g[k] = __fmaf_rn(s, d.d[k], a.g[k]);
  if (WITH_H) {
    const float wf2 = __fmul_rn(w, __fmul_rn(Fs, Fs));
    int m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float t = __fmul_rn(wf2, d.d[k]);
#pragma unroll
      for (int l = k; l < 4; ++l) {
        a.h[m] = __fmaf_rn(t, d.d[l], a.h[m]);
        ++m;
      }
    }
  }
}

__device__ __forceinline__ double warp_sum_f64(float x) {
  double y = (double)x;
#pragma unroll
  for (int o = 16; o; o >>= 1) y = __dadd_rn(y, __shfl_xor_sync(kFull, y, o));
  return __shfl_sync(kFull, y, 0);
}

// theta_i = (t0, tE, u0, alpha) with absolute t0.  Outputs (any may be
// null): chi2[i], grad[4 i + k], H[10 i + m] (upper triangle, row-major),
// Fs[i], Fb[i], flags[i].
template <bool WITH_H>
__global__ void __launch_bounds__(kAdjWarps * 32)
    k_theta(const SearchParams P, const double *__restrict__ theta, int n,
            double t_ref, double *chi2, double *grad, double *H, double *Fs,
            double *Fb, int *flags) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  const double t0 = theta[4 * i + 0], tE = theta[4 * i + 1];
  const double u0 = theta[4 * i + 2], al = theta[4 * i + 3];
  double sn, cs;
  sincos(al, &sn, &cs);
  const double tEc = (tE > 1e-6) ? tE : 1e-6;  // the host rejects tE <= 0
  double tlo, thi;
  slab_tau(P.L, u0, cs, sn, tlo, thi);
  const Epochs ep = epochs_at(P.ep, P.n_ep);
  const TrajC c =
      make_traj(P, ep, u0, cs, sn, t0 - t_ref, 1.0 / (tEc * P.dlt), tEc,
                tlo, thi);
  const Acc s1 = phase1<false>(P, ep, c, lane);
  const Solved sol = solve2(P, (double)s1.a, (double)s1.b, (double)s1.d);
  const float fFs = __double2float_rn(sol.Fs);
  const float fBc = __double2float_rn(sol.Bc);
  const float fcs = (float)cs, fsn = (float)sn, fu0 = (float)u0;
  GradAcc a;
  a.chi = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) a.g[k] = 0.f;
#pragma unroll
  for (int k = 0; k < 10; ++k) a.h[k] = 0.f;
  Deriv d;
  for (int e = lane_start(0, lane); e < c.e_in; e += 32) {
    const float2 v = ep.tw[e];
    const float Ac = out_grad(c, fu0, v.x, d);
    grad_add<WITH_H>(a, v.y, ep.fc[e], Ac, d, fFs, fBc);
  }
#pragma unroll 2
  for (int e = lane_start(c.e_in, lane); e < c.e_out; e += 32) {
    const float2 v = ep.tw[e];
    const float Ac = in_grad(P, c, fcs, fsn, fu0, v.x, d);
    grad_add<WITH_H>(a, v.y, ep.fc[e], Ac, d, fFs, fBc);
  }
  for (int e = lane_start(c.e_out, lane); e < P.n_ep; e += 32) {
    const float2 v = ep.tw[e];
    const float Ac = out_grad(c, fu0, v.x, d);
    grad_add<WITH_H>(a, v.y, ep.fc[e], Ac, d, fFs, fBc);
  }
  const double x2 = warp_sum_f64(a.chi);
  double gg[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) gg[k] = warp_sum_f64(a.g[k]);
  double hh[10];
  if (WITH_H) {
#pragma unroll
    for (int k = 0; k < 10; ++k) hh[k] = warp_sum_f64(a.h[k]);
  }
  if (lane == 0) {
    if (chi2) chi2[i] = isnan(x2) ? CUDART_INF : x2;
    if (grad)
      for (int k = 0; k < 4; ++k) grad[4 * i + k] = gg[k];
    if (WITH_H && H)
      for (int k = 0; k < 10; ++k) H[10 * i + k] = hh[k];
    if (Fs) Fs[i] = sol.Fs;
    if (Fb) Fb[i] = sol.Bc + P.Fref - sol.Fs;
    if (flags) flags[i] = sol.degenerate ? MORSE_FIT_DEGENERATE : 0;
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

cudaError_t launch_theta(const SearchParams &P, const double *theta, int n,
                         double t_ref, double *chi2, double *grad, double *H,
                         double *Fs, double *Fb, int *flags,
                         cudaStream_t st) {
  const int threads = kAdjWarps * 32;
  const int blocks = (n + kAdjWarps - 1) / kAdjWarps;
  if (H)
    k_theta<true><<<blocks, threads, 0, st>>>(P, theta, n, t_ref, chi2, grad,
                                              H, Fs, Fb, flags);
  else
    k_theta<false><<<blocks, threads, 0, st>>>(P, theta, n, t_ref, chi2, grad,
                                               nullptr, Fs, Fb, flags);
  return cudaGetLastError();
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
