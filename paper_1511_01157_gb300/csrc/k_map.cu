// Magnification-map kernels: inverse ray shooting into a shared-memory
// histogram (K1) and ray counts -> magnification texels (K1b).
//
// The method (McDougall & Albrow 2015, §3 ray-shooting maps, §4.1 uniform
// source grid, §5 inverse ray shooting): image-plane rays on a uniform grid
// are deflected by the binary lens (Eq. 2) and counted in source-plane
// pixels; a pixel's magnification is its ray count times the image area of
// one ray over the source area of one pixel.
//
// GB300 design.  A persistent grid of 512-thread blocks walks 256x256-ray
// image tiles.  A tile's rays land in a compact source window (the lens map
// is smooth away from the lenses), so each block bins into a 128x128-bin
// shared-memory window placed on the deflected tile, using shared-memory
// atomics; rays that fall outside the window go straight to the global map
// with red.global.add, and the window is flushed with one global add per
// non-empty bin (four bins per 16-byte read).  Threads own 8x16-ray
// sub-blocks so that the 32 lanes of a warp sit 8 rays (~1.2 pixels) apart
// and rarely hit the same bin.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "morse_internal.cuh"

namespace morse {

namespace {

constexpr int kSubX = 8;    // rays per thread sub-block along x (the
                            // rows along y, RayParams::sub_rows, are chosen
                            // per launch)
static_assert(kRayThreads == (kRayTileX / kSubX) * kRayWarps,
              "one sub-block per thread");
static_assert(kSubX == 8 && kRayTileX / kSubX == 32,
              "a warp is one row of sub-blocks across the tile");

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// FP64 deflection with the operation order of the plain definition:
//   d1x = x1 - xa; r1 = d1x d1x + x2 x2; d2x = x1 - xb; r2 = d2x d2x + x2 x2
//   y1 = x1 - (e1 d1x)/r1 - (e2 d2x)/r2;  y2 = x2 - (e1 x2)/r1 - (e2 x2)/r2
//   v = (y + L)/Delta, bin = floor(v), on the map iff 0 <= v < npix.
// Every operation is an explicitly rounded IEEE op (no FMA contraction) so
// the counts equal those of the FP64 definition evaluated on a CPU.
// Returns 0 on map (bin in *ix, *iy), 1 off map, 2 lost (ray on a lens).
__device__ __forceinline__ int deflect64(const RayParams &P, long long i,
                                         double x2, double x2sq, int *ix,
                                         int *iy) {
  double x1 = __dadd_rn(-P.X, __dmul_rn(__dadd_rn((double)i, 0.5), P.h));
  double d1x = __dsub_rn(x1, P.xa);
  double r1 = __dadd_rn(__dmul_rn(d1x, d1x), x2sq);
  double d2x = __dsub_rn(x1, P.xb);
  double r2 = __dadd_rn(__dmul_rn(d2x, d2x), x2sq);
  if (r1 == 0.0 || r2 == 0.0) return 2;
  double y1 = __dsub_rn(__dsub_rn(x1, __ddiv_rn(__dmul_rn(P.e1, d1x), r1)),
                        __ddiv_rn(__dmul_rn(P.e2, d2x), r2));
  double y2 = __dsub_rn(__dsub_rn(x2, __ddiv_rn(__dmul_rn(P.e1, x2), r1)),
                        __ddiv_rn(__dmul_rn(P.e2, x2), r2));
  double v1 = __ddiv_rn(__dadd_rn(y1, P.L), P.dlt);
  double v2 = __ddiv_rn(__dadd_rn(y2, P.L), P.dlt);
  double np = (double)P.npix;
  if (!(v1 >= 0.0 && v1 < np && v2 >= 0.0 && v2 < np)) return 1;
  *ix = (int)v1;  // truncation == floor for v >= 0
  *iy = (int)v2;
  return 0;
}

// FP32 deflection: one approximate reciprocal of r1 r2 serves both lenses.
// The bin of v by one add rounded down: adding 1.5 * 2^23 leaves floor(v)
// in the low mantissa bits for |v| < 2^22; any other v (far off the map,
// infinite, NaN) gives a value that the unsigned range test rejects.
__device__ __forceinline__ unsigned bin_of(float v) {
  return (unsigned)__float_as_int(__fadd_rd(v, 12582912.f)) - 0x4B400000u;
}

__device__ __forceinline__ int deflect32(const RayParams &P, float x1,
                                         float x2, float x2sq, int *ix,
                                         int *iy) {
  float d1 = x1 - P.xaf;
  float d2 = x1 - P.xbf;
  float r1 = fmaf(d1, d1, x2sq);
  float r2 = fmaf(d2, d2, x2sq);
  float rr = r1 * r2;
  if (rr == 0.0f) return 2;
  float inv = rcp_approx(rr);
  float a1 = P.e1f * (r2 * inv);
  float a2 = P.e2f * (r1 * inv);
  float y1 = fmaf(-a2, d2, fmaf(-a1, d1, x1));
  float y2 = fmaf(-(a1 + a2), x2, x2);
  const unsigned a = bin_of(fmaf(y1, P.invdf, P.offf));
  const unsigned b = bin_of(fmaf(y2, P.invdf, P.offf));
  if (a >= (unsigned)P.npix || b >= (unsigned)P.npix) return 1;
  *ix = (int)a;
  *iy = (int)b;
  return 0;
}

// Bin of a sample ray (FP64), clamped into the map; used only to place the
// shared-memory window, never to count.
// Bin of ray (i, j) for placing a tile's window (a cache: where a ray is
// binned does not change the counts), in FP32 for both paths.
__device__ bool sample_bin(const RayParams &P, long long i, long long j,
                           int *bx, int *by) {
  const float x2 = fmaf((float)j, P.hf, P.x0f);
  const float x1 = fmaf((float)i, P.hf, P.x0f);
  int ix = 0, iy = 0;
  const int st = deflect32(P, x1, x2, x2 * x2, &ix, &iy);
  if (st != 0) return false;
  *bx = ix;
  *by = iy;
  return true;
}

__device__ __forceinline__ float2 f2r(float v) { return make_float2(v, v); }

// Bin one FP32 ray from its floor sums tx, ty = RD(v + 1.5 2^23) (the bin
// of v in the low mantissa bits, as bin_of).  cx, cy: the window's corner
// plus the bit offset 0x4B400000, so one unsigned compare per axis tests
// "on the map and in the window" (the window lies inside the map; W is its
// side, the map's side when the map is smaller).
__device__ __forceinline__ void bin_ray(const RayParams &P, uint32_t *win,
                                        unsigned cx, unsigned cy, unsigned W,
                                        float tx, float ty, bool lost,
                                        unsigned &n_off, unsigned &n_lost) {
  const unsigned ux = (unsigned)__float_as_int(tx);
  const unsigned uy = (unsigned)__float_as_int(ty);
  const unsigned lx = ux - cx, ly = uy - cy;
  if (lost) {
    ++n_lost;
  } else if (lx < W && ly < W) {
    atomicAdd(&win[ly * kRayWin + lx], 1u);
  } else {
    const unsigned a = ux - 0x4B400000u, b = uy - 0x4B400000u;
    if (a >= (unsigned)P.npix || b >= (unsigned)P.npix)
      ++n_off;
    else
      atomicAdd(&P.counts[(size_t)b * P.npix + a], 1u);
  }
}

// The FP32 rays of one thread's sub-block: columns ib .. ib + na - 1
// (FULL: na = kSubX), rows jb .. jb + P.sub_rows - 1, two columns per packed
// FP32 instruction.  The deflection works in bin units: with x' = x/Delta +
// L/Delta and e' = e/Delta (taken once per sub-block and per row), the
// bin coordinates are
//     v1 = x1' - e1' d1 r2/(r1 r2) - e2' d2 r1/(r1 r2),
//     v2 = x2' - (e1' r2 + e2' r1)/(r1 r2) x2,
// d_k = x1 - x_k, r_k = d_k^2 + x2^2, one approximate reciprocal of r1 r2
// for both lenses.  The lens terms are those of deflect32 (the window's
// sample rays); the ray coordinates start from the sub-block, so a ray's
// bin may differ from deflect32's by the last rounding.
template <bool FULL>
__device__ __forceinline__ void shoot_f32(const RayParams &P, uint32_t *win,
                                          int wx0, int wy0, long long jb,
                                          int na, float x1b, unsigned &n_off,
                                          unsigned &n_lost) {
  constexpr int NP = kSubX / 2;
  float2 x1s[NP], d1[NP], d2[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float2 x1 = make_float2(fmaf((float)(2 * p), P.hf, x1b),
                                  fmaf((float)(2 * p + 1), P.hf, x1b));
    d1[p] = __fadd2_rn(x1, f2r(-P.xaf));
    d2[p] = __fadd2_rn(x1, f2r(-P.xbf));
    x1s[p] = __ffma2_rn(x1, f2r(P.invdf), f2r(P.offf));
  }
  const float2 ne1 = f2r(-P.e1f * P.invdf), ne2 = f2r(-P.e2f * P.invdf);
  const float2 M = f2r(12582912.f);
  const unsigned W = (unsigned)min(kRayWin, P.npix);
  const unsigned cx = 0x4B400000u + (unsigned)wx0;
  const unsigned cy = 0x4B400000u + (unsigned)wy0;
#pragma unroll 1
  for (int b = 0; b < P.sub_rows; ++b) {
    const long long j = jb + b;
    if (j >= P.nray) break;
    const float x2 = fmaf((float)j, P.hf, P.x0f);
    const float2 x2p = f2r(x2), x2sq = f2r(x2 * x2);
    const float2 x2s = f2r(fmaf(x2, P.invdf, P.offf));
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      if (!FULL && 2 * p >= na) break;
      const float2 r1 = __ffma2_rn(d1[p], d1[p], x2sq);
      const float2 r2 = __ffma2_rn(d2[p], d2[p], x2sq);
      const float2 rr = __fmul2_rn(r1, r2);
      const float2 inv = make_float2(rcp_approx(rr.x), rcp_approx(rr.y));
      const float2 a1 = __fmul2_rn(ne1, __fmul2_rn(r2, inv));  // -e1' / r1
      const float2 a2 = __fmul2_rn(ne2, __fmul2_rn(r1, inv));  // -e2' / r2
      const float2 v1 = __ffma2_rn(a2, d2[p], __ffma2_rn(a1, d1[p], x1s[p]));
      const float2 v2 = __ffma2_rn(__fadd2_rn(a1, a2), x2p, x2s);
      const float2 tx = __fadd2_rd(v1, M);
      const float2 ty = __fadd2_rd(v2, M);
      if (FULL || 2 * p + 1 < na) {
        // both rays in the window (the common case): one test for the
        // pair; a lost ray (rr = 0) has an infinite or NaN bin sum and
        // fails it
        const unsigned lx0 = (unsigned)__float_as_int(tx.x) - cx;
        const unsigned ly0 = (unsigned)__float_as_int(ty.x) - cy;
        const unsigned lx1 = (unsigned)__float_as_int(tx.y) - cx;
        const unsigned ly1 = (unsigned)__float_as_int(ty.y) - cy;
        if (max(max(lx0, ly0), max(lx1, ly1)) < W) {
          atomicAdd(&win[ly0 * kRayWin + lx0], 1u);
          atomicAdd(&win[ly1 * kRayWin + lx1], 1u);
          continue;
        }
        // both rays off the map (the next most common case: 38 % of the
        // rays of [-3, 3]^2 miss the [-2, 2]^2 map): one test for the pair
        // on the map-relative floor bits, unless a ray is lost
        const unsigned ax0 = (unsigned)__float_as_int(tx.x) - 0x4B400000u;
        const unsigned ay0 = (unsigned)__float_as_int(ty.x) - 0x4B400000u;
        const unsigned ax1 = (unsigned)__float_as_int(tx.y) - 0x4B400000u;
        const unsigned ay1 = (unsigned)__float_as_int(ty.y) - 0x4B400000u;
        if (min(max(ax0, ay0), max(ax1, ay1)) >= (unsigned)P.npix &&
            rr.x != 0.0f && rr.y != 0.0f) {
          n_off += 2;
          continue;
        }
        bin_ray(P, win, cx, cy, W, tx.x, ty.x, rr.x == 0.0f, n_off, n_lost);
        bin_ray(P, win, cx, cy, W, tx.y, ty.y, rr.y == 0.0f, n_off, n_lost);
      } else {
        bin_ray(P, win, cx, cy, W, tx.x, ty.x, rr.x == 0.0f, n_off, n_lost);
      }
    }
  }
}

// FP32: two blocks per SM (at most 64 registers: the packed sub-block loop
// keeps its twelve column pairs in registers).
template <bool FP64>
__global__ void __launch_bounds__(kRayThreads, FP64 ? 1 : 2)
    k_rayshoot(const RayParams P) {
  extern __shared__ __align__(16) uint32_t win[];  // kRayWin^2 bins
  __shared__ int s_wx, s_wy, s_tile;
  const int tid = threadIdx.x;
  uint4 *win4 = reinterpret_cast<uint4 *>(win);
  for (int k = tid; k < kRayWin * kRayWin / 4; k += kRayThreads)
    win4[k] = make_uint4(0u, 0u, 0u, 0u);
  unsigned int n_off = 0, n_lost = 0;
  const int ntiles = P.tiles_x * P.tiles_y;
  const int sx = tid & 31;   // sub-block column (lane)
  const int sy = tid >> 5;   // sub-block row (warp)

  const long long tile_h = (long long)kRayWarps * P.sub_rows;
  for (;;) {
    // tiles from a counter: blocks whose tiles were cheap take more
    if (tid == 0) s_tile = (int)atomicAdd(&P.tot[2], 1ULL);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ntiles) break;  // block-uniform
    const long long i0 = (long long)(tile % P.tiles_x) * kRayTileX;
    const long long j0 = (long long)(tile / P.tiles_x) * tile_h;
    if (tid < 32) {
      // place the window on the bounding box of 9 deflected sample rays
      int bx = 0, by = 0;
      bool ok = false;
      if (tid < 9) {
        long long ii = i0 + (tid % 3) * (long long)(kRayTileX - 1) / 2;
        long long jj = j0 + (tid / 3) * (tile_h - 1) / 2;
        if (ii >= P.nray) ii = P.nray - 1;
        if (jj >= P.nray) jj = P.nray - 1;
        ok = sample_bin(P, ii, jj, &bx, &by);
      }
      int lo_x = ok ? bx : 0x7fffffff, hi_x = ok ? bx : -1;
      int lo_y = ok ? by : 0x7fffffff, hi_y = ok ? by : -1;
      for (int o = 16; o; o >>= 1) {
        lo_x = min(lo_x, __shfl_xor_sync(0xffffffffu, lo_x, o));
        hi_x = max(hi_x, __shfl_xor_sync(0xffffffffu, hi_x, o));
        lo_y = min(lo_y, __shfl_xor_sync(0xffffffffu, lo_y, o));
        hi_y = max(hi_y, __shfl_xor_sync(0xffffffffu, hi_y, o));
      }
      if (tid == 0) {
        int cx = (hi_x >= 0) ? (lo_x + hi_x) / 2 : P.npix / 2;
        int cy = (hi_y >= 0) ? (lo_y + hi_y) / 2 : P.npix / 2;
        int wx = cx - kRayWin / 2, wy = cy - kRayWin / 2;
        int wmax = P.npix - kRayWin;
        if (wmax < 0) wmax = 0;
        s_wx = min(max(wx, 0), wmax);
        s_wy = min(max(wy, 0), wmax);
      }
    }
    __syncthreads();
    const int wx0 = s_wx, wy0 = s_wy;
    const long long ib = i0 + sx * kSubX;
    const long long jb = j0 + sy * P.sub_rows;
    // rays of the sub-block row inside the grid, and the first one's x1
    const int na = (int)max(0LL, min((long long)kSubX, P.nray - ib));
    const float x1b = fmaf((float)ib, P.hf, P.x0f);
    if (!FP64) {
      if (na == kSubX)
        shoot_f32<true>(P, win, wx0, wy0, jb, na, x1b, n_off, n_lost);
      else if (na > 0)
        shoot_f32<false>(P, win, wx0, wy0, jb, na, x1b, n_off, n_lost);
    } else {
#pragma unroll 1
      for (int b = 0; b < P.sub_rows; ++b) {
        const long long j = jb + b;
        if (j >= P.nray) break;
        const double x2d = __dadd_rn(-P.X, __dmul_rn(__dadd_rn((double)j, 0.5), P.h));
        const double x2sqd = __dmul_rn(x2d, x2d);
#pragma unroll
        for (int a = 0; a < kSubX; ++a) {
          if (a < na) {
            int ix = 0, iy = 0;
            const int st = deflect64(P, ib + a, x2d, x2sqd, &ix, &iy);
            if (st == 0) {
              unsigned lx = (unsigned)(ix - wx0), ly = (unsigned)(iy - wy0);
              if (lx < (unsigned)kRayWin && ly < (unsigned)kRayWin)
                atomicAdd(&win[ly * kRayWin + lx], 1u);
              else
                atomicAdd(&P.counts[(size_t)iy * P.npix + ix], 1u);
            } else if (st == 1) {
              ++n_off;
            } else {
              ++n_lost;
            }
          }
        }
      }
    }
    __syncthreads();
    // flush the window: four bins per read, one global add per non-empty
    // bin, then clear (a bin beyond a map narrower than the window is
    // never counted, so it is zero and skipped)
    for (int k4 = tid; k4 < kRayWin * kRayWin / 4; k4 += kRayThreads) {
      const uint4 v = win4[k4];
      if ((v.x | v.y | v.z | v.w) == 0u) continue;
      win4[k4] = make_uint4(0u, 0u, 0u, 0u);
      const int k = 4 * k4;
      const int gx = wx0 + (k % kRayWin), gy = wy0 + (k / kRayWin);
      uint32_t *dst = &P.counts[(size_t)gy * P.npix + gx];
      if (v.x) atomicAdd(dst, v.x);
      if (v.y) atomicAdd(dst + 1, v.y);
      if (v.z) atomicAdd(dst + 2, v.z);
      if (v.w) atomicAdd(dst + 3, v.w);
    }
    __syncthreads();
  }
  // off-map and lost totals
  unsigned long long o = n_off, l = n_lost;
  for (int s = 16; s; s >>= 1) {
    o += __shfl_xor_sync(0xffffffffu, o, s);
    l += __shfl_xor_sync(0xffffffffu, l, s);
  }
  if ((tid & 31) == 0) {
    if (o) atomicAdd(&P.tot[0], o);
    if (l) atomicAdd(&P.tot[1], l);
  }
}

// Texel tables.  Quad (c, r), c, r in [0, npix], describes the bilinear
// cell whose lower corner is texel (c - 1, r - 1): the column and row below
// the map repeat its edge (so that a lookup below the first texel centre
// reads the edge value, the clamping rule, without a clamp), and so do the
// column and row at npix - 1.  With m = A - 1 the FP32 quad holds
//   (m00, m10 - m00, m01 - m00, (m11 - m01) - (m10 - m00)),
// rounded in FP32, so that a lookup is three FMAs: the first row at fx,
// the row difference at fx, and the value at fy.
__device__ __forceinline__ int clampi(int v, int n) {
  return v < 0 ? 0 : (v >= n ? n - 1 : v);
}


__device__ __forceinline__ float4 quad_of(float a00, float a10, float a01,
                                          float a11) {
  // A - 1: FP32 of the FP32 value, exact for A <= 2
  const float m00 = a00 - 1.0f, m10 = a10 - 1.0f;
  const float m01 = a01 - 1.0f, m11 = a11 - 1.0f;
  const float d0 = __fsub_rn(m10, m00), d1 = __fsub_rn(m11, m01);
  return make_float4(m00, d0, __fsub_rn(m01, m00), __fsub_rn(d1, d0));
}

// counts -> A, one FP64 product per texel (the cells are then built from A
// by k_quads_from_A: one product per texel instead of four per cell, the
// FP64 pipe being the limiter of a fused form)
__global__ void k_counts_to_A(const uint32_t *__restrict__ counts, int npix,
                              double f, float *__restrict__ A) {
  const size_t n = (size_t)npix * npix;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    A[k] = __double2float_rn(__dmul_rn((double)counts[k], f));
}

__global__ void k_quads_from_A(const float *__restrict__ A, int npix,
                               float4 *__restrict__ quad, int qpitch) {
  const int side = npix + 1;
  const size_t n = (size_t)side * side;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(k % side), r = (int)(k / side);
    const int x0 = clampi(c - 1, npix), x1 = clampi(c, npix);
    const int y0 = clampi(r - 1, npix), y1 = clampi(r, npix);
    quad[cell_index(c, r, qpitch)] = quad_of(
        A[(size_t)y0 * npix + x0], A[(size_t)y0 * npix + x1],
        A[(size_t)y1 * npix + x0], A[(size_t)y1 * npix + x1]);
  }
}

// FP16 storage code of one FP32 value: log10 in FP64, rounded once to
// binary16 (round to nearest even)
__device__ __forceinline__ uint16_t half_code(float a, double a_floor) {
  const double v = (double)a;
  return __half_as_ushort(__double2half(log10(v > a_floor ? v : a_floor)));
}

__global__ void k_half_codes(const float *__restrict__ A, size_t n,
                             double a_floor, uint16_t *__restrict__ codes) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    codes[k] = half_code(A[k], a_floor);
}

// (x00, x10) in .x and (x01, x11) in .y, low half first; same cells and
// edge repetition as the FP32 quads, codes undifferenced
__global__ void k_half_quads(const uint16_t *__restrict__ codes, int npix,
                             uint2 *__restrict__ quadh, int qpitch) {
  const int side = npix + 1;
  const size_t n = (size_t)side * side;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(k % side), r = (int)(k / side);
    const int x0 = clampi(c - 1, npix), x1 = clampi(c, npix);
    const int y0 = clampi(r - 1, npix), y1 = clampi(r, npix);
    const unsigned c00 = codes[(size_t)y0 * npix + x0];
    const unsigned c10 = codes[(size_t)y0 * npix + x1];
    const unsigned c01 = codes[(size_t)y1 * npix + x0];
    const unsigned c11 = codes[(size_t)y1 * npix + x1];
    quadh[cell_index(c, r, qpitch)] = make_uint2(c00 | (c10 << 16),
                                               c01 | (c11 << 16));
  }
}

}  // namespace

static size_t ray_smem() { return sizeof(uint32_t) * kRayWin * kRayWin; }

int rayshoot_blocks_per_sm() {
  static int cached = -1;
  if (cached > 0) return cached;
  cudaFuncSetAttribute(k_rayshoot<true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ray_smem());
  cudaFuncSetAttribute(k_rayshoot<false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)ray_smem());
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &b, k_rayshoot<false>, kRayThreads, ray_smem()) != cudaSuccess ||
      b < 1)
    b = 1;
  cached = b;
  return b;
}

cudaError_t launch_rayshoot(const RayParams &P, bool fp64, int grid,
                            cudaStream_t st) {
  rayshoot_blocks_per_sm();  // sets the shared-memory attribute once
  if (fp64)
    k_rayshoot<true><<<grid, kRayThreads, ray_smem(), st>>>(P);
  else
    k_rayshoot<false><<<grid, kRayThreads, ray_smem(), st>>>(P);
  return cudaGetLastError();
}

static size_t quad_cells(int npix) {
  return (size_t)(npix + 1) * (size_t)(npix + 1);
}

static int elementwise_grid(size_t n) {
  size_t g = (n + 255) / 256;
  if (g > 8192) g = 8192;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_counts_to_map(const uint32_t *counts, int npix, double f,
                                 float *A, float4 *quad, int qpitch,
                                 cudaStream_t st) {
  k_counts_to_A<<<elementwise_grid((size_t)npix * npix), 256, 0, st>>>(
      counts, npix, f, A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_quads_from_A<<<elementwise_grid(quad_cells(npix)), 256, 0, st>>>(
      A, npix, quad, qpitch);
  return cudaGetLastError();
}

cudaError_t launch_quads_from_A(const float *A, int npix, float4 *quad,
                                int qpitch, cudaStream_t st) {
  k_quads_from_A<<<elementwise_grid(quad_cells(npix)), 256, 0, st>>>(
      A, npix, quad, qpitch);
  return cudaGetLastError();
}

cudaError_t launch_half_from_A(const float *A, int npix, double a_floor,
                               uint16_t *codes, uint2 *quadh, int qpitch,
                               cudaStream_t st) {
  size_t n = (size_t)npix * npix;
  k_half_codes<<<elementwise_grid(n), 256, 0, st>>>(A, n, a_floor, codes);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_half_quads<<<elementwise_grid(quad_cells(npix)), 256, 0, st>>>(
      codes, npix, quadh, qpitch);
  return cudaGetLastError();
}

}  // namespace morse
