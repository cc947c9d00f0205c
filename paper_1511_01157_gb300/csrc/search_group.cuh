// Shared-memory top-K of a search block and the per-warp-group body of the
// trajectory search, used by the single-pair search (k_search) and the
// batched persistent search (k_batch).
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "morse_internal.cuh"
#include "search_common.cuh"

namespace morse {
namespace dev {

// Block-wide top-K state in shared memory.
struct BlockTopK {
  Entry *buf0, *buf1; // the sorted list and its merge target, alternating
  Entry *wbuf;        // per-warp staging of sorted candidates (32 each)
  int *cur, *nk, *lock;
  volatile double *thr;
};

// Published block quantiles: the grid-wide threshold's second source.  A
// block whose list holds j entries at or below v, with c - 1 other lists
// whose published j-th values are at most v, makes c j distinct
// trajectories (lists hold disjoint sets) of chi^2 at most v; when
// c j >= K, v bounds the K-th best and may lower the threshold.  Level q
// (1..kPubLevels) publishes the ceil(K / 4^q)-th best and needs c >= 4^q;
// the block's K-th (c = 1) lowers the threshold directly.  Early in a pass
// each block has seen a small share of the grid, so its K-th is far above
// the global K-th while its first few entries are not.
__device__ __forceinline__ int pub_groups(int q) { return 1 << (2 * q); }

// Warp-collective, outside the block lock: publish this block's level
// values (lane q holds level q's, +inf if the list is shorter) and lower
// the grid-wide threshold where enough blocks agree.
static __device__ __noinline__ void pub_update(const SearchParams &P, double pv,
                                        const int lane) {
  const int nb = P.pub_nb;
  const int me = P.pub_me >= 0 ? P.pub_me : (int)blockIdx.x;
  const size_t row = (size_t)P.pub_stride;
  unsigned fb[kPubLevels];
#pragma unroll
  for (int q = 1; q <= kPubLevels; ++q) {
    const double v = __shfl_sync(kFull, pv, q);
    const float f = __double2float_ru(v);
    fb[q - 1] = (pub_groups(q) <= nb && f < CUDART_INF_F)
                    ? __float_as_uint(f) : 0xFFFFFFFFu;
    if (lane == 0 && fb[q - 1] != 0xFFFFFFFFu)
      __stcg(&P.pub[(size_t)(q - 1) * row + me],
             ((unsigned long long)P.pub_tag << 32) | fb[q - 1]);
  }
  int c[kPubLevels] = {};
  for (int b = lane; b < nb; b += 32) {
    if (b == me) continue;  // counted below
#pragma unroll
    for (int q = 0; q < kPubLevels; ++q) {
      const unsigned long long w = __ldcg(&P.pub[(size_t)q * row + b]);
      c[q] += ((unsigned)(w >> 32) == P.pub_tag) && ((unsigned)w <= fb[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < kPubLevels; ++q) {
    const int n = __reduce_add_sync(kFull, (unsigned)c[q]) + 1;
    if (lane == 0 && fb[q] != 0xFFFFFFFFu && n >= pub_groups(q + 1))
      atomicMin(P.gthr, (unsigned long long)__double_as_longlong(
                            (double)__uint_as_float(fb[q])));
  }
}

// Warp-collective: merge this lane's candidate (if any) into the block's
// sorted top-K under the block lock.  Candidates are first sorted across
// the warp (bitonic); each existing entry and each candidate then moves to
// its rank in the union, and the first K are kept.
__device__ inline void warp_merge(const SearchParams &P, BlockTopK &T, const int K,
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
  // acquire the block lock (bounded spin: P.spin_limit waits of ~64 ns)
  int ok = 1;
  if (lane == 0) {
    const unsigned lim = P.spin_limit ? P.spin_limit : (1u << 20);
    unsigned it = 0;
    while (atomicCAS(T.lock, 0, 1) != 0) {
      if (++it > lim) {
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
  // the published levels' values, read while the lock is held
  double pv = CUDART_INF;
  if (P.pub && lane >= 1 && lane <= kPubLevels) {
    const int j = (K + pub_groups(lane) - 1) / pub_groups(lane);
    if (min(K, nk + nc) >= j) pv = nxt[j - 1].chi2;
  }
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
  if (P.pub && P.gthr) pub_update(P, pv, lane);
}

// One warp group: trajectories [lo, hi) of the line-aligned pass (lined),
// or sample positions [lo, hi) of a strided pass, each lane owning one.
// Phase 1 in pairs of trajectories, the FP64 solve, the pruning test
// against min(block K-th, grid-wide threshold), phase 2 for the survivors,
// then the dense store or the merge into the block's top-K.
template <bool DENSE, bool H, int TB = 0>
__device__ __forceinline__ void search_group(const SearchParams &P,
                                             const Epochs &ep, BlockTopK &T,
                                             const int K, const int warp,
                                             const int lane, long long lo,
                                             long long hi, const bool lined,
                                             unsigned long long &n_exact,
                                             const float4 *tab = nullptr) {
  const int nvalid = (int)max(0LL, hi - lo);
  if (nvalid == 0) return;  // warp-uniform
  if (P.linemax && lined &&
      __ldg(&P.linemax[lo / P.line]) < P.a_min) {
    // minimum-magnification cut: the whole group's line is too faint
    if (DENSE && lane < nvalid) {
      const long long o = lo - P.first + lane;
      P.dchi2[o] = CUDART_INF;
      if (P.dFs) P.dFs[o] = 0.0;
      if (P.dFb) P.dFb[o] = 0.0;
    }
    return;
  }
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
      phase1_pair<H, TB>(P, ep, ca, cb, lane, ra, rb, tab);
      if (lane == k) mine_s = ra;
      if (lane == k + 1) mine_s = rb;
    } else {
      const Acc ra = phase1<H, TB>(P, ep, ca, lane, tab);
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
    cand_me = may_reach(P, sol, thr);
  const float myFs = __double2float_rn(sol.Fs);
  const float myBc = __double2float_rn(sol.Bc);
  double my_chi2 = CUDART_INF;
  if (!DENSE && P.pilot_ub) {
    // pilot: the bound from the sums, no sweep
    if (cand_me)
      my_chi2 = chi2_upper(P, (double)mine_s.a, (double)mine_s.b,
                           (double)mine_s.d, (double)myFs, (double)myBc);
    cand_me = false;
  }
  unsigned todo = __ballot_sync(kFull, cand_me);
  n_exact += __popc(todo);
  while (todo) {
    const int k = __ffs(todo) - 1;
    todo &= todo - 1;
    const TrajC c = shfl_traj(mine, k);
    const float Fs = __shfl_sync(kFull, myFs, k);
    const float Bc = __shfl_sync(kFull, myBc, k);
    const double chi2 = phase2<H, TB>(P, ep, c, lane, Fs, Bc, tab);
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
    bool keep = lane < nvalid && my_chi2 <= thr && my_chi2 < CUDART_INF;
    // a strided (pilot) sample mixes lines: drop the cut ones here
    if (keep && P.linemax && !lined)
      keep = __ldg(&P.linemax[my / P.line]) >= P.a_min;
    warp_merge(P, T, K, warp, lane, keep, my_chi2, my);
  }
}

// Shared-memory band tables of the line-aligned pass (build_band), two of
// them, alternating by block round (round r in buffer r & 1, one line per
// round).  A warp that claims a group of round r builds the tables of
// rounds r and r + 1 when their buffers are free (no user left of the
// round two back) and nobody has; it reads round r's table only after
// taking a user count on a ready word, and otherwise uses the global table
// (same bits).  Nothing ever waits.  Words: ((round + 1) << 7) | (ready <<
// 6) | users; 0 = empty.
struct BandTabs {
  float4 *tabs;  // 2 tables of P.tab_n entries
  unsigned *tw;  // [2] words
  int *tb;       // [2] orientations (1: x-major, 2: y-major)
};

// Centred coordinates of the point of line L nearest the origin, and its
// direction (the line's row of the grid tables, or of a line grid).
__device__ __forceinline__ void band_line(const SearchParams &P, long long L,
                                          double &cx, double &cy, double &c,
                                          double &s) {
  const long long iu = L / P.n_alpha;
  const int ia = (int)(L - iu * P.n_alpha);
  double u;
  if (P.lu) {
    u = P.lu[iu];
    c = P.lc[iu];
    s = P.ls[iu];
  } else {
    u = P.u0v[iu];
    c = P.ca[ia];
    s = P.sa[ia];
  }
  cx = -u * s * P.invD + P.coff;
  cy = u * c * P.invD + P.coff;
}

// warp-collective: build the table of round r (line L) if its buffer is
// free and nobody has
template <bool H>
__device__ __forceinline__ void band_try_build(const SearchParams &P,
                                               BandTabs &B, long long r,
                                               long long L, int lane) {
  const int b = (int)(r & 1);
  const unsigned want = (unsigned)(r + 1) << 7;
  int got = 0;
  if (lane == 0) {
    const unsigned w = *(volatile unsigned *)&B.tw[b];
    const bool idle = w == 0u || (w & 0x40u);  // empty or ready
    if (idle && (w & 0x3Fu) == 0u && (w >> 7) < (unsigned)(r + 1))
      got = atomicCAS(&B.tw[b], w, want) == w;
  }
  got = __shfl_sync(kFull, got, 0);
  if (!got) return;
  double cx, cy, c, s;
  band_line(P, L, cx, cy, c, s);
  const int tb = build_band<H>(P, B.tabs + (size_t)b * P.tab_n, cx, cy, c, s,
                               lane);
  __threadfence_block();
  __syncwarp();
  if (lane == 0) {
    B.tb[b] = tb;
    __threadfence_block();
    atomicExch(&B.tw[b], want | 0x40u);
  }
  __syncwarp();
}

// warp-collective: a user count on round r's table; returns its
// orientation, or 0 (not ready: use the global table)
__device__ __forceinline__ int band_try_acquire(BandTabs &B, long long r,
                                                int lane) {
  const int b = (int)(r & 1);
  const unsigned want = ((unsigned)(r + 1) << 7) | 0x40u;
  int ok = 0;
  if (lane == 0) {
    for (int it = 0; it < 16; ++it) {
      const unsigned w = *(volatile unsigned *)&B.tw[b];
      if ((w & ~0x3Fu) != want) break;
      if (atomicCAS(&B.tw[b], w, w + 1u) == w) {
        ok = 1;
        break;
      }
    }
    if (ok) {
      __threadfence_block();
      ok = *(volatile int *)&B.tb[b];
    }
  }
  return __shfl_sync(kFull, ok, 0);
}

__device__ __forceinline__ void band_release(BandTabs &B, long long r,
                                             int lane) {
  if (lane == 0) atomicSub(&B.tw[(int)(r & 1)], 1u);
}

// Record of one selected trajectory e (warp-collective; lane 0 writes *dst):
// (Fs, Fb) from the phase-1 sums and the solve, recomputed with the search's
// device functions on the epochs at ep_blk (a shared-memory copy) or P.ep,
// so the same bits;
// chi^2 is the search's own phase-2 value, the key e was ranked by.
template <bool H>
__device__ __forceinline__ void fill_one(const SearchParams &P, const Entry e,
                                         const double *t0abs,
                                         const double *tEv, const int lane,
                                         morse_fit *dst,
                                         const float4 *ep_blk = nullptr) {
  morse_fit r;
  const long long total = (long long)P.n_u0 * P.n_alpha * P.n_t0 * P.n_tE;
  if (e.idx < 0 || e.idx >= total) {
    if (lane == 0) {
      r.chi2 = CUDART_INF;
      r.t0 = r.tE = r.u0 = r.alpha = r.Fs = r.Fb = 0.0;
      r.idx = -1;
      r.flags = 0;
      r.reserved = 0;
      *dst = r;
    }
    return;
  }
  const Epochs ep = epochs_at(ep_blk ? ep_blk : P.ep, P.n_ep);
  const TrajC c = traj_consts(P, ep, e.idx);
  const Acc s = phase1<H>(P, ep, c, lane);
  const Solved sol = solve2(P, (double)s.a, (double)s.b, (double)s.d);
  if (lane == 0) {
    long long q = e.idx;
    const int itE = (int)(q % P.n_tE);
    q /= P.n_tE;
    const int it0 = (int)(q % P.n_t0);
    q /= P.n_t0;
    const int ia = (int)(q % P.n_alpha);
    const int iu = (int)(q / P.n_alpha);
    r.chi2 = e.chi2;
    r.tE = (P.lu && P.ltE) ? P.ltE[iu] : tEv[itE];
    if (P.lu) {  // line grid: the record in the (u0, alpha) convention
      r.t0 = t0abs[it0] - P.lsh[iu] * r.tE;
      r.u0 = P.lu[iu];
      r.alpha = P.la[iu];
    } else {
      r.t0 = t0abs[it0];
      r.u0 = P.u0v[iu];
      r.alpha = 2.0 * CUDART_PI * (double)ia / (double)P.n_alpha;
    }
    r.Fs = sol.Fs;
    r.Fb = sol.Bc + P.Fref - sol.Fs;
    r.idx = e.idx;
    r.flags = sol.degenerate ? MORSE_FIT_DEGENERATE : 0;
    r.reserved = 0;
    *dst = r;
  }
}

}  // namespace dev
}  // namespace morse
