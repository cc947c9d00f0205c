// Batched trajectory search: many light curves of uneven length against a
// bank of maps in one persistent launch (the §4.2 grid search of every
// (event, map) pair, with the §4.4 top-K seeds of each pair).
//
// GB300 design.
//  * One 16-warp block per SM loops over work units taken from a global
//    counter.  A unit is a run of warp groups of one (event, map) pair; the
//    host lists the units map by map (one map at a time is read from HBM
//    into L2) and within a map longest event first, so the long light
//    curves start early and the short ones fill the tail.
//  * Within a unit the warps take groups from a shared-memory counter, so a
//    warp that drew cheap trajectories (mostly outside the map) takes more.
//  * The event's epochs are staged in shared memory when the unit's shape
//    says so (copied once per block while consecutive units share the
//    event); long light curves are read from global memory through L1.
//  * Each pair has its own pruning threshold (seeded by a strided pilot
//    pass of the same kernel), and each unit its own block top-K, flushed
//    to a partial list at the end of the unit.  Per pair, one block merges
//    the pair's lists; a warp per kept trajectory writes its record.
//  * Every trajectory's chi^2 is computed by the same device functions as
//    the single-pair search (k_search), so the results of a batch are those
//    of one morse_grid_chi2 call per pair, bit for bit.
// Inside-map epoch loops unrolled four times for the FP32 table (as
// k_search; FP16-table variants: twice).  The map cells come from the
// global table through L1: light curves of more than 4096 epochs, which
// carry about 80 % of a batch's evaluations, cannot be staged in shared
// memory and stream their epochs through L1 too, and the 131 KB of
// k_search's band tables would take that L1 away (tried: 9.75e11 ->
// 9.2e11 evaluations/s, L1 hit rate 90 % -> 41 %).
#ifndef MORSE_UNROLL
#define MORSE_UNROLL 4
#endif
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"
#include "search_common.cuh"
#include "search_group.cuh"

namespace morse {

namespace {

using namespace dev;

// Search parameters of one pair: the shared ones with the event's and the
// map's fields filled in.
template <bool H>
__device__ __forceinline__ SearchParams pair_params(const BatchParams &B,
                                                    const BatchEvent &E,
                                                    int mi) {
  SearchParams Q = B.S;
  if (H)
    Q.quadh = static_cast<const uint2 *>(B.tab[mi]);
  else
    Q.quad = static_cast<const float4 *>(B.tab[mi]);
  Q.ep = E.ep;
  Q.n_ep = E.n_ep;
  Q.S1 = E.S1;
  Q.SF = E.SF;
  Q.SFF = E.SFF;
  Q.Fref = E.Fref;
  Q.invS1 = E.invS1;
  Q.CFF = E.CFF;
  Q.gamma = E.gamma;
  Q.t0rel = E.t0rel;
  return Q;
}

// The warps of the block run the unit's groups, taking them from *s_next.
template <bool H, bool STAGE>
__device__ __forceinline__ void run_unit(const BatchParams &B,
                                         const BatchUnit &U,
                                         const BatchEvent &E, int mi,
                                         const float4 *sep, BlockTopK &T,
                                         int *s_next, int warp, int lane,
                                         unsigned long long &n_exact) {
  SearchParams Q = pair_params<H>(B, E, mi);
  Q.tpg = U.tpg;
  Q.ng_line = (Q.line + U.tpg - 1) / U.tpg;
  Q.gthr = B.gthr + U.pair;
  if (Q.pub) {  // the pair's lists' published quantiles
    const int l0 = B.list0[U.pair];
    Q.pub += l0;
    Q.pub_nb = B.list0[U.pair + 1] - l0;
    Q.pub_me = U.list - l0;
  }
  const Epochs ep = epochs_at(STAGE ? sep : E.ep, E.n_ep);
  const bool lined = Q.stride == 1 && Q.line > 0;
  for (;;) {
    int gi = 0;
    if (lane == 0) gi = atomicAdd(s_next, 1);
    gi = __shfl_sync(kFull, gi, 0);
    if (gi >= U.ng) break;
    const long long g = (long long)U.g0 + gi;
    long long lo, hi;
    if (lined) {
      const long long L = g / Q.ng_line;
      const long long j = g % Q.ng_line;
      lo = L * Q.line + j * U.tpg;
      hi = min(Q.count, L * Q.line + min((j + 1) * U.tpg, Q.line));
    } else {
      lo = g * U.tpg;
      hi = min(lo + U.tpg, Q.count);
    }
    search_group<false, H>(Q, ep, T, Q.top_k, warp, lane, lo, hi, lined,
                           n_exact);
  }
}

// V only names a second copy of the kernel (V = 1: the launch of unstaged
// light curves), so that each launch has its own shared-memory carveout.
template <bool H, int V>
__global__ void __launch_bounds__(kSearchWarps * 32, 1)
    k_batch(const BatchParams B) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int K = B.S.top_k;
  float4 *sep = reinterpret_cast<float4 *>(smem);
  BlockTopK T;
  T.buf0 = reinterpret_cast<Entry *>(smem + sizeof(float4) * (size_t)B.ep_cap);
  T.buf1 = T.buf0 + K;
  T.wbuf = T.buf1 + K;
  __shared__ int s_unit, s_ev, s_next, s_cur, s_nk, s_lock;
  __shared__ double s_thr;
  T.cur = &s_cur;
  T.nk = &s_nk;
  T.lock = &s_lock;
  T.thr = &s_thr;
  if (threadIdx.x == 0) s_ev = -1;
  unsigned long long n_exact = 0;
  for (;;) {
    if (threadIdx.x == 0) s_unit = (int)atomicAdd(B.counter, 1u);
    __syncthreads();
    const int u = s_unit;
    if (u >= B.n_units) break;  // block-uniform
    const BatchUnit U = B.units[u];
    const int e = U.pair / B.n_maps;
    const int mi = U.pair - e * B.n_maps;
    const BatchEvent E = B.ev[e];
    const bool stage = U.stage && E.n_ep <= B.ep_cap;
    if (stage && s_ev != e)
      for (int i = threadIdx.x; i < E.n_ep; i += blockDim.x) sep[i] = E.ep[i];
    __syncthreads();  // copy done, s_ev read by every thread
    if (threadIdx.x == 0) {
      if (stage) s_ev = e;
      s_cur = 0;
      s_nk = 0;
      s_lock = B.S.lock0;
      s_thr = CUDART_INF;
      s_next = 0;
    }
    __syncthreads();
    if (stage)
      run_unit<H, true>(B, U, E, mi, sep, T, &s_next, warp, lane, n_exact);
    else
      run_unit<H, false>(B, U, E, mi, sep, T, &s_next, warp, lane, n_exact);
    __syncthreads();
    const int nk = s_nk;
    const Entry *cur = s_cur ? T.buf1 : T.buf0;
    Entry *out = B.partial + (size_t)U.list * K;
    for (int i = threadIdx.x; i < K; i += blockDim.x) {
      Entry en;
      if (i < nk) {
        en = cur[i];
      } else {  // unique sentinel keys after the real ones, ascending
        en.chi2 = CUDART_INF;
        en.idx = 0x7fff000000000000LL + ((long long)U.list * K + i);
      }
      out[i] = en;
    }
  }
  if (B.S.stat_exact && lane == 0 && n_exact)
    atomicAdd(B.S.stat_exact, n_exact);
}

// One block per pair: tree of pairwise merges over the pair's lists,
// ping-ponging between a and b within the pair's range.
__global__ void k_batch_merge(Entry *a, Entry *b, const int *__restrict__ list0,
                              int k, Entry *__restrict__ result,
                              unsigned long long *gthr) {
  const int p = blockIdx.x;
  int n = list0[p + 1] - list0[p];
  Entry *in = a + (size_t)list0[p] * k;
  Entry *out = b + (size_t)list0[p] * k;
  while (n > 1) {
    const int pairs = (n + 1) / 2;
    const long long total = (long long)pairs * 2 * k;
    for (long long t = threadIdx.x; t < total; t += blockDim.x) {
      const int q = (int)(t / (2 * k));
      const int side = (int)((t / k) & 1);
      const int i = (int)(t % k);
      const int la = 2 * q, lb = 2 * q + 1;
      if (lb >= n) {  // odd list out: copy
        if (side == 0) out[(size_t)q * k + i] = in[(size_t)la * k + i];
        continue;
      }
      const Entry *A = in + (size_t)(side ? lb : la) * k;
      const Entry *Bl = in + (size_t)(side ? la : lb) * k;
      const Entry e = A[i];
      int lo = 0, hi = k;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (key_less(Bl[mid], e))
          lo = mid + 1;
        else
          hi = mid;
      }
      const int r = i + lo;
      if (r < k) out[(size_t)q * k + r] = e;
    }
    __syncthreads();
    Entry *t = in;
    in = out;
    out = t;
    n = pairs;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    result[(size_t)p * k + i] = in[i];
  if (gthr && threadIdx.x == 0) {
    const Entry e = in[k - 1];
    if (e.chi2 < CUDART_INF && e.idx >= 0 && e.idx < 0x7fff000000000000LL)
      atomicMin(&gthr[p], (unsigned long long)__double_as_longlong(e.chi2));
  }
}

// One warp per kept trajectory of every pair.
template <bool H>
__global__ void k_batch_fill(const BatchParams B, const Entry *result,
                             int pairs, const double *t0abs, const double *tEv,
                             morse_fit *out) {
  const int lane = threadIdx.x & 31;
  const long long w =
      ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int K = B.S.top_k;
  if (w >= (long long)pairs * K) return;
  const int p = (int)(w / K);
  const int e = p / B.n_maps;
  const int mi = p - e * B.n_maps;
  const BatchEvent E = B.ev[e];
  const SearchParams Q = pair_params<H>(B, E, mi);
  fill_one<H>(Q, result[w], t0abs, tEv, lane, &out[w]);
}

}  // namespace

size_t batch_smem_bytes(int ep_cap, int top_k) {
  return sizeof(float4) * (size_t)ep_cap +
         sizeof(Entry) * ((size_t)2 * top_k + kSearchWarps * 32);
}

template <bool H, int V>
static int batch_occupancy(size_t smem) {
  cudaFuncSetAttribute(k_batch<H, V>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // smallest shared-memory carveout that holds the block: the rest of the
  // SM's 256 KB serves as L1 for the map gathers
  int dev = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                         dev);
  if (per_sm > 0) {
    int pct = (int)((100.0 * (double)(smem + 2048)) / (double)per_sm) + 1;
    if (pct > 100) pct = 100;
    cudaFuncSetAttribute(k_batch<H, V>,
                         cudaFuncAttributePreferredSharedMemoryCarveout, pct);
  }
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &b, k_batch<H, V>, kSearchWarps * 32, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return b;
}

int batch_blocks_per_sm(bool h16, size_t smem, int variant) {
  if (variant)
    return h16 ? batch_occupancy<true, 1>(smem)
               : batch_occupancy<false, 1>(smem);
  return h16 ? batch_occupancy<true, 0>(smem) : batch_occupancy<false, 0>(smem);
}

cudaError_t launch_batch(const BatchParams &B, bool h16, int grid,
                         size_t smem, cudaStream_t st, int variant) {
  const int threads = kSearchWarps * 32;
  if (variant) {
    if (h16)
      k_batch<true, 1><<<grid, threads, smem, st>>>(B);
    else
      k_batch<false, 1><<<grid, threads, smem, st>>>(B);
  } else if (h16) {
    k_batch<true, 0><<<grid, threads, smem, st>>>(B);
  } else {
    k_batch<false, 0><<<grid, threads, smem, st>>>(B);
  }
  return cudaGetLastError();
}

cudaError_t launch_batch_merge(Entry *a, Entry *b, const int *list0,
                               int pairs, int k, Entry *result,
                               unsigned long long *gthr, cudaStream_t st) {
  k_batch_merge<<<pairs, 256, 0, st>>>(a, b, list0, k, result, gthr);
  return cudaGetLastError();
}

cudaError_t launch_batch_fill(const BatchParams &B, bool h16,
                              const Entry *result, int pairs,
                              const double *t0abs, const double *tEv,
                              morse_fit *out, cudaStream_t st) {
  const long long warps = (long long)pairs * B.S.top_k;
  const long long blocks = (warps * 32 + 255) / 256;
  if (h16)
    k_batch_fill<true><<<(unsigned)blocks, 256, 0, st>>>(B, result, pairs,
                                                         t0abs, tEv, out);
  else
    k_batch_fill<false><<<(unsigned)blocks, 256, 0, st>>>(B, result, pairs,
                                                          t0abs, tEv, out);
  return cudaGetLastError();
}

}  // namespace morse
