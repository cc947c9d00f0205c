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
//  * One 16-warp block per SM.  The light curve (t, w, wF, F per epoch,
//    time-sorted) is staged once per block in shared memory.
//  * Warps take groups of up to 32 trajectories from a block counter.  For each, the lanes walk
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
//    from the start.  A tree of 4-way merges gives the global
//    top-K and k_fill recomputes the winners' records with the same device
//    functions.
// The search kernels unroll their inside-map epoch loops four times: with
// a trajectory pair in packed FP32 the loop body is small enough for the
// instruction cache, and more independent shared loads are in flight
// (unroll 2: 1 % slower on the config-1 sweep, 1: 10 %, 3: 0.5 %).  The
// other kernels keep the default of search_common.cuh.
#ifndef MORSE_UNROLL
#define MORSE_UNROLL 4
#endif
#ifndef MORSE_PK_ASM
#define MORSE_PK_ASM 1  // packed pair operations as inline PTX (faster here)
#endif
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <algorithm>

#include "morse_internal.cuh"
#include "search_common.cuh"
#include "search_group.cuh"

namespace morse {

namespace {

using namespace dev;

template <bool DENSE, bool EP_SMEM, bool H>
__global__ void __launch_bounds__(kSearchWarps * 32, 1)
    k_search(const SearchParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int K = P.top_k;

  const float4 *blk = P.ep;
  BlockTopK T;
  float4 *tabs = nullptr;  // two band tables (P.tab_n entries each)
  __shared__ int s_cur, s_nk, s_lock, s_next;
  __shared__ double s_thr;
  // band table words: ((round + 1) << 7) | (ready << 6) | users; 0 = empty
  __shared__ unsigned s_tw[2];
  __shared__ int s_tb[2];  // orientation (1: x-major, 2: y-major)
  {
    unsigned char *p = smem;
    if (EP_SMEM) {
      float4 *s = reinterpret_cast<float4 *>(p);
      for (int e = threadIdx.x; e < P.n_ep; e += blockDim.x) s[e] = P.ep[e];
      blk = s;
      p += sizeof(float4) * (size_t)P.n_ep;
    }
    if (!DENSE) {
      T.buf0 = reinterpret_cast<Entry *>(p);
      T.buf1 = T.buf0 + K;
      T.wbuf = T.buf1 + K;
      p += sizeof(Entry) * ((size_t)2 * K + kSearchWarps * 32);
    }
    if (P.tab_n > 0) tabs = reinterpret_cast<float4 *>(p);
    T.cur = &s_cur;
    T.nk = &s_nk;
    T.lock = &s_lock;
    T.thr = &s_thr;
  }
  if (threadIdx.x == 0) {
    s_cur = 0;
    s_nk = 0;
    s_lock = P.lock0;
    s_next = 0;
    s_thr = CUDART_INF;
    s_tw[0] = 0u;
    s_tw[1] = 0u;
  }
  __syncthreads();
  const Epochs ep = epochs_at(blk, P.n_ep);

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

  // Band tables.  With kSearchWarps groups per line (the host enables the
  // tables only then) the block's round r is one line; its table lives in
  // buffer r & 1 (search_group.cuh: band_try_build, band_try_acquire).
  const bool use_tab = tabs != nullptr && lined &&
                       P.ng_line == (long long)kSearchWarps;
  BandTabs B;
  B.tabs = tabs;
  B.tw = s_tw;
  B.tb = s_tb;
  // the line of block round r, or -1 past the block's last group
  auto round_line = [&](long long r) -> long long {
    const long long g0 = (long long)blockIdx.x * kSearchWarps + r * gstride;
    if (g0 >= n_groups) return -1;
    return line0 + g0 / P.ng_line;
  };
  if (use_tab) {  // the first two rounds' tables before any group starts
    if (warp < 2) {
      const long long L = round_line(warp);
      if (L >= 0) band_try_build<H>(P, B, warp, L, lane);
    }
    __syncthreads();
  }

  // The block's groups come in rounds of kSearchWarps consecutive groups,
  // round r starting at blockIdx.x kSearchWarps + r gstride.  Its warps
  // take them one at a time, in order, from a shared counter: a warp whose
  // groups were cheap takes more, so the warps finish together, and the
  // warps of a block still walk neighbouring groups.
  for (;;) {
    int k = 0;
    if (lane == 0) k = atomicAdd(&s_next, 1);
    k = __shfl_sync(kFull, k, 0);
    const long long g = (long long)blockIdx.x * kSearchWarps +
                        (long long)(k / kSearchWarps) * gstride +
                        k % kSearchWarps;
    if (g >= n_groups) break;  // g grows with k: every later k is out too
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
    int tb = 0;
    const long long r = k / kSearchWarps;
    if (use_tab) {
      band_try_build<H>(P, B, r, round_line(r), lane);
      const long long L1 = round_line(r + 1);
      if (L1 >= 0) band_try_build<H>(P, B, r + 1, L1, lane);
      tb = band_try_acquire(B, r, lane);
    }
    const float4 *tab = tabs + (size_t)(r & 1) * (use_tab ? P.tab_n : 0);
    if (tb == 1)
      search_group<DENSE, H, 1>(P, ep, T, K, warp, lane, lo, hi, lined,
                                n_exact, tab);
    else if (tb == 2)
      search_group<DENSE, H, 2>(P, ep, T, K, warp, lane, lo, hi, lined,
                                n_exact, tab);
    else
      search_group<DENSE, H>(P, ep, T, K, warp, lane, lo, hi, lined,
                             n_exact);
    if (tb != 0) band_release(B, r, lane);
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
        e.chi2 = CUDART_INF;  // unique sentinel keys, ascending
        e.idx = 0x7fff000000000000LL + ((long long)blockIdx.x * K + i);
      }
      out[i] = e;
    }
  }
}

// One level of the merge tree: lists 4p .. 4p + 3 -> list p, keeping the
// first k of their union (a short last group merges what it has).
constexpr int kMergeWays = 4;  // lists merged into one per level

__global__ void k_merge_level(const Entry *__restrict__ in,
                              Entry *__restrict__ out, int lists, int k) {
  // one thread per input entry: its rank in its group of kMergeWays lists
  // is its index plus the entries of the group's other lists below it
  // (keys are unique across lists), and the first k ranks are kept
  const long long total = (long long)lists * k;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       t < total; t += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(t / k), i = (int)(t % k);
    const int grp = l / kMergeWays, l0 = grp * kMergeWays;
    const int l1 = min(l0 + kMergeWays, lists);
    const Entry e = in[(size_t)l * k + i];
    int r = i;
    for (int m = l0; m < l1; ++m) {
      if (m == l) continue;
      const Entry *B = in + (size_t)m * k;
      int lo = 0, hi = k;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_less(B[mid], e))
          lo = mid + 1;
        else
          hi = mid;
      }
      r += lo;
    }
    if (r < k) out[(size_t)grp * k + r] = e;
  }
}

// The same merge, W = 4 or 16 lists at a time, with one block per input
// list: the block stages its group's lists in shared memory (so the binary
// searches of the ranks cost shared-memory latency, not L2 latency), ranks
// its own list's entries against the others and writes those of rank < k
// to the group's output list.  With `seed` on the last level, the entry of
// final rank k - 1 lowers *seed to its chi^2 (as k_seed_threshold).
// Rank of key (kb, id) in a sorted list of k keys: the entries of smaller
// chi^2 (bit patterns of non-negative doubles order as integers), plus
// those of equal chi^2 and smaller index.
__device__ __forceinline__ int lower_rank(const unsigned long long *K,
                                          const long long *I, int k,
                                          unsigned long long kb,
                                          long long id) {
  int lo = 0, hi = k;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (K[mid] < kb)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo < k && K[lo] == kb) {  // a tie in chi^2 (rare but for sentinels)
    int e = lo + 1, top = k;
    while (e < top) {  // end of the tie run
      const int mid = (e + top) >> 1;
      if (K[mid] == kb)
        e = mid + 1;
      else
        top = mid;
    }
    hi = e;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (I[mid] < id)
        lo = mid + 1;
      else
        hi = mid;
    }
  }
  return lo;
}

// S = ways / 4 consecutive threads rank one entry, each against a quarter
// of the group's other lists; their counts are summed by shuffles.  The
// lists are staged as separate key and index arrays, so a step of the
// binary search reads 8 bytes.
__global__ void __launch_bounds__(1024)
    k_merge_rank(const Entry *__restrict__ in, Entry *__restrict__ out,
                 int lists, int k, int ways, unsigned long long *seed) {
  extern __shared__ __align__(16) unsigned char msm[];
  const int l = blockIdx.x;
  const int g = l / ways, l0 = g * ways;
  const int n = min(ways, lists - l0);
  unsigned long long *ky = reinterpret_cast<unsigned long long *>(msm);
  long long *id = reinterpret_cast<long long *>(ky + (size_t)n * k);
  {
    // the group's lists, four independent 16-byte loads per thread in
    // flight (the copy is bound by L2 latency otherwise)
    const float4 *src = reinterpret_cast<const float4 *>(in + (size_t)l0 * k);
    const int nv = n * k;
    const int st = blockDim.x;
    for (int i0 = threadIdx.x; i0 < nv; i0 += 4 * st) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u * st < nv) v[u] = __ldcg(src + i0 + u * st);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u * st < nv) {
          const double2 d = *reinterpret_cast<const double2 *>(&v[u]);
          ky[i0 + u * st] = (unsigned long long)__double_as_longlong(d.x);
          id[i0 + u * st] = __double_as_longlong(d.y);
        }
    }
  }
  __syncthreads();
  const int me = l - l0;
  const int S = ways >= 16 ? 4 : 1;  // threads per entry (a power of 2)
  const int part = threadIdx.x & (S - 1);
  const int per = blockDim.x / S;
  for (int i0 = 0; i0 < k; i0 += per) {  // block-uniform trip count
    const int i = i0 + (int)threadIdx.x / S;
    const bool has = i < k;
    unsigned long long kb = 0;
    long long ie = 0;
    int r = 0;
    if (has) {
      kb = ky[(size_t)me * k + i];
      ie = id[(size_t)me * k + i];
      for (int m = part; m < n; m += S)
        if (m != me)
          r += lower_rank(ky + (size_t)m * k, id + (size_t)m * k, k, kb, ie);
    }
    for (int o = 1; o < S; o <<= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    r += i;
    if (has && part == 0 && r < k) {
      Entry e;
      e.chi2 = __longlong_as_double((long long)kb);
      e.idx = ie;
      out[(size_t)g * k + r] = e;
      if (seed && r == k - 1 && e.chi2 < CUDART_INF && e.idx >= 0 &&
          e.idx < 0x7fff000000000000LL)
        atomicMin(seed, kb);
    }
  }
}

// Fit fill: one warp per selected trajectory recomputes the phase-1 sums
// and the solve with the same device functions as the search, and writes
// the public morse_fit record with the search's chi^2.
// With EPS the block first stages the light curve in shared memory, so a
// warp's walk over the epochs waits only on the cell gathers.
template <bool H, bool EPS>
__global__ void k_fill(const FillParams F) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const float4 *blk = nullptr;
  if (EPS) {
    float4 *s = reinterpret_cast<float4 *>(fsm);
    for (int e = threadIdx.x; e < F.S.n_ep; e += blockDim.x) s[e] = F.S.ep[e];
    __syncthreads();
    blk = s;
  }
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= F.k) return;  // after the block's only barrier
  fill_one<H>(F.S, F.sel[w], F.t0abs, F.tEv, lane, &F.out[w], blk);
}

// The tau interval of every (u0, alpha) line inside the map.
__global__ void k_slab(const double *__restrict__ u0v,
                       const double *__restrict__ ca,
                       const double *__restrict__ sa, int n_u0, int n_alpha,
                       double L, double2 *__restrict__ slab) {
  const int n = n_u0 * n_alpha;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += gridDim.x * blockDim.x) {
    const int iu = i / n_alpha, ia = i - iu * n_alpha;
    double lo, hi;
    slab_tau(L, u0v[iu], ca[ia], sa[ia], lo, hi);
    slab[i] = make_double2(lo, hi);
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
template <bool H>
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
      A[i] = __fadd_rn(H ? bilinear_h_m1(P, vx, vy) : bilinear_m1(P, vx, vy),
                       1.f);
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

template <bool D, bool E, bool H>
static int occupancy(size_t smem) {
  cudaFuncSetAttribute(k_search<D, E, H>,
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
    cudaFuncSetAttribute(k_search<D, E, H>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  }
#endif
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &b, k_search<D, E, H>, kSearchWarps * 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b;
}

template <bool H>
static int occupancy_h(bool dense, bool ep_smem, size_t smem) {
  if (dense && ep_smem) return occupancy<true, true, H>(smem);
  if (dense) return occupancy<true, false, H>(smem);
  if (ep_smem) return occupancy<false, true, H>(smem);
  return occupancy<false, false, H>(smem);
}

int search_blocks_per_sm(bool dense, bool ep_smem, bool h16, size_t smem) {
  return h16 ? occupancy_h<true>(dense, ep_smem, smem)
             : occupancy_h<false>(dense, ep_smem, smem);
}

template <bool H>
static void launch_search_h(const SearchParams &P, bool dense, bool ep_smem,
                            int grid, size_t smem, cudaStream_t st) {
  const int threads = kSearchWarps * 32;
  if (dense && ep_smem)
    k_search<true, true, H><<<grid, threads, smem, st>>>(P);
  else if (dense)
    k_search<true, false, H><<<grid, threads, smem, st>>>(P);
  else if (ep_smem)
    k_search<false, true, H><<<grid, threads, smem, st>>>(P);
  else
    k_search<false, false, H><<<grid, threads, smem, st>>>(P);
}

cudaError_t launch_search(const SearchParams &P, bool dense, bool ep_smem,
                          int grid, size_t smem, cudaStream_t st) {
  if (P.quadh)
    launch_search_h<true>(P, dense, ep_smem, grid, smem, st);
  else
    launch_search_h<false>(P, dense, ep_smem, grid, smem, st);
  return cudaGetLastError();
}

cudaError_t launch_topk_merge(Entry *a, Entry *b, int lists, int k,
                              Entry **result, int *levels, cudaStream_t st,
                              unsigned long long *seed) {
  Entry *in = a, *out = b;
  *levels = 0;
  // the device's shared-memory limit, and the rank kernel's limit raised
  // to it, once per device
  static int optin_of[64];
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = dev < 64 ? optin_of[dev] : 0;
  if (optin == 0) {
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                           dev);
    cudaFuncSetAttribute(k_merge_rank,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (dev < 64) optin_of[dev] = optin;
  }
  bool seeded = false;
  while (lists > 1) {
    // 16 lists per group when they fit in shared memory (k <= 908 at
    // 227 KB), else 4 (k <= 3632), else the global-memory 4-way levels
    const size_t per = sizeof(Entry) * (size_t)k;
    const int ways = lists > kMergeWays && 16 * per <= (size_t)optin ? 16
                     : kMergeWays * per <= (size_t)optin ? kMergeWays : 0;
    const int next = (lists + (ways ? ways : kMergeWays) - 1) /
                     (ways ? ways : kMergeWays);
    if (ways > 0) {
      const size_t sm = (size_t)min(ways, lists) * per;
      unsigned long long *sd = next == 1 ? seed : nullptr;
      // threads: S per entry for up to all k entries at once, whole warps
      const int S = ways >= 16 ? 4 : 1;
      const int threads = std::min(1024, ((k * S + 31) / 32) * 32);
      k_merge_rank<<<lists, threads, sm, st>>>(in, out, lists, k, ways, sd);
      seeded = sd != nullptr;
    } else {
      const long long total = (long long)lists * k;
      long long g = (total + 255) / 256;
      if (g > 65535) g = 65535;
      k_merge_level<<<(int)g, 256, 0, st>>>(in, out, lists, k);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++*levels;
    lists = next;
    Entry *t = in;
    in = out;
    out = t;
  }
  *result = in;
  if (seed && !seeded) {
    cudaError_t e = launch_seed_threshold(in, k, seed, st);
    if (e != cudaSuccess) return e;
    ++*levels;
  }
  return cudaSuccess;
}

cudaError_t launch_fill(const FillParams &F, cudaStream_t st) {
  // Each record's warp walks the epochs once (latency-bound).  Light curves
  // that fit are staged in shared memory by blocks of eight warps; others
  // are read from global memory by blocks of two warps, spread over the SMs.
  static int optin_of[64];
  int dev = 0;
  cudaGetDevice(&dev);
  int optin = dev < 64 ? optin_of[dev] : 0;
  if (optin == 0) {
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                           dev);
    cudaFuncSetAttribute(k_fill<true, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    cudaFuncSetAttribute(k_fill<false, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (dev < 64) optin_of[dev] = optin;
  }
  const size_t sm = sizeof(float4) * (size_t)F.S.n_ep;
  if (sm <= (size_t)optin) {
    const int threads = 256;
    const int blocks = (F.k * 32 + threads - 1) / threads;
    if (F.S.quadh)
      k_fill<true, true><<<blocks, threads, sm, st>>>(F);
    else
      k_fill<false, true><<<blocks, threads, sm, st>>>(F);
  } else {
    const int threads = 64;
    const int blocks = (F.k * 32 + threads - 1) / threads;
    if (F.S.quadh)
      k_fill<true, false><<<blocks, threads, 0, st>>>(F);
    else
      k_fill<false, false><<<blocks, threads, 0, st>>>(F);
  }
  return cudaGetLastError();
}

__global__ void k_slab_lines(const double *__restrict__ u,
                             const double *__restrict__ c,
                             const double *__restrict__ s, int n, double L,
                             double2 *__restrict__ slab) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += gridDim.x * blockDim.x) {
    double lo, hi;
    slab_tau(L, u[i], c[i], s[i], lo, hi);
    slab[i] = make_double2(lo, hi);
  }
}

cudaError_t launch_slab_lines(const double *u, const double *c,
                              const double *s, int n, double L, double2 *slab,
                              cudaStream_t st) {
  int blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  k_slab_lines<<<blocks, 256, 0, st>>>(u, c, s, n, L, slab);
  return cudaGetLastError();
}

cudaError_t launch_slab(const double *u0v, const double *ca, const double *sa,
                        int n_u0, int n_alpha, double L, double2 *slab,
                        cudaStream_t st) {
  const int n = n_u0 * n_alpha;
  int blocks = (n + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  if (blocks < 1) blocks = 1;
  k_slab<<<blocks, 256, 0, st>>>(u0v, ca, sa, n_u0, n_alpha, L, slab);
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
  if (P.quadh)
    k_lightcurve<true><<<blocks, 256, 0, st>>>(P, ax, bx, ay, by, kt, bt, u02,
                                               t, n, A);
  else
    k_lightcurve<false><<<blocks, 256, 0, st>>>(P, ax, bx, ay, by, kt, bt,
                                                u02, t, n, A);
  return cudaGetLastError();
}

}  // namespace morse
