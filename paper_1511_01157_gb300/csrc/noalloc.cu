// morse_grid_chi2_noalloc: the top-K trajectory search without any device
// allocation.
//
// Some callers cannot let the library call cudaMalloc or cudaFree once
// set-up is over: cudaFree waits for the whole device, which stalls every
// stream of a latency-bound pipeline, and some applications run under a
// fixed, pre-reserved memory budget where a workspace that grows on demand
// is not acceptable.  They create their context, event and map handles at set-up
// (where allocation is fine) and then search with this entry point, which
// keeps its scratch -- the grid tables, two status words, the two
// per-block top-K lists of the merge tree and the fit records -- in one
// file-scope device array of fixed size instead of the context's growable
// workspace.
//
// The array is shared by every call in the process on a given device and
// keeps whatever the last call wrote; each call clears its status words
// and overwrites every other byte it reads before reading it.  Two calls that
// overlap on the same GPU (different streams or host threads) race on it.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "morse_internal.cuh"

namespace {

// Maximum scratch of the allocation-free search (bytes).
constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;

static __device__ __align__(256) unsigned char
    g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices];

// Device address of g_noalloc_scratch on `device` (which must be current).
// Looked up once per device and kept for the life of the process (a
// cudaDeviceReset would invalidate it); the host-side symbol is only a
// stand-in and must never be passed to a kernel.
cudaError_t scratch_address(int device, void **out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

morse_status set_err(morse_ctx *ctx, morse_status st, const char *msg) {
  snprintf(ctx->err, sizeof(ctx->err), "%s", msg);
  return st;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" morse_status morse_grid_chi2_noalloc(morse_ctx *ctx,
                                                const morse_event *ev,
                                                const morse_map *map,
                                                const morse_grid *g,
                                                morse_fit *out) {
  if (!ctx || !out) return MORSE_EINVAL;
  if (!ev || !map || ev->ctx != ctx || map->ctx != ctx)
    return set_err(ctx, MORSE_EINVAL, "event and map must belong to ctx");
  if (!g || g->n_u0 < 1 || g->n_alpha < 1 || g->n_t0 < 1 || g->n_tE < 1 ||
      !std::isfinite(g->u0_lo) || !std::isfinite(g->u0_hi) ||
      !std::isfinite(g->t0_lo) || !std::isfinite(g->t0_hi) ||
      !(g->tE_lo > 0.0) || !(g->tE_hi > 0.0) || !std::isfinite(g->tE_lo) ||
      !std::isfinite(g->tE_hi) ||
      (g->u0_log && (!(g->u0_lo > 0.0) || !(g->u0_hi > 0.0))) ||
      g->top_k < 1 || g->top_k > 4096)
    return set_err(ctx, MORSE_EINVAL, "invalid grid");
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MORSE_ECUDA, "cudaSetDevice failed");
  }
  void *scratch = nullptr;
  cudaError_t e = scratch_address(ctx->device, &scratch);
  if (e != cudaSuccess) {
    snprintf(ctx->err, sizeof(ctx->err),
             "cudaGetSymbolAddress of the no-alloc scratch: %s",
             cudaGetErrorString(e));
    return MORSE_ECUDA;
  }
  if (g->a_min > 0.0f)
    return set_err(ctx, MORSE_EUNSUPPORTED,
                   "the allocation-free search has no minimum-magnification "
                   "cut");
  const int K = g->top_k;
  const long long count =
      (long long)g->n_u0 * g->n_alpha * g->n_t0 * g->n_tE;

  // launch shape: the same rule as the allocating search
  const size_t fixed = morse::search_smem_bytes(0, K);
  const size_t budget = ctx->smem_optin > 4096 ? ctx->smem_optin - 2048 : 0;
  const bool ep_smem =
      budget > fixed && (size_t)ev->n <= (budget - fixed) / sizeof(float4);
  const size_t smem = fixed + (ep_smem ? sizeof(float4) * (size_t)ev->n : 0);
  const bool h16 = morse::map_h16(map);
  const int bps = morse::search_blocks_per_sm(false, ep_smem, h16, smem);
  if (bps < 1)
    return set_err(ctx, MORSE_EUNSUPPORTED, "search kernel does not fit");
  long long groups =
      morse::main_groups((long long)g->n_t0 * g->n_tE, 0, count);
  long long want = (groups + morse::kSearchWarps - 1) / morse::kSearchWarps;
  int grid = (int)std::min<long long>((long long)bps * ctx->sm_count, want);
  if (grid < 1) grid = 1;

  // scratch layout: grid tables (line slabs, then the FP64 values) |
  // status words | list A | list B | fits
  const size_t tab_n = morse::table_values(g);
  const size_t off_w = up256(morse::tables_bytes(g));
  const size_t off_a = off_w + 256;
  const size_t list = sizeof(morse::Entry) * (size_t)grid * K;
  const size_t off_b = up256(off_a + list);
  const size_t off_fit = up256(off_b + list);
  const size_t need = off_fit + sizeof(morse_fit) * (size_t)K;
  if (need > kNoAllocScratchBytes) {
    snprintf(ctx->err, sizeof(ctx->err),
             "morse_grid_chi2_noalloc: this search needs %zu bytes of scratch "
             "(top_k %d, %d blocks, %zu grid-table values) but the "
             "allocation-free path has %zu; lower top_k or use "
             "morse_grid_chi2",
             need, K, grid, tab_n, kNoAllocScratchBytes);
    return MORSE_EINVAL;
  }
  char *base = (char *)scratch;

  // grid tables (the allocating path's values, from the same helper),
  // staged on the stack
  constexpr size_t kMaxTable = 4096;
  if (tab_n > kMaxTable) {
    snprintf(ctx->err, sizeof(ctx->err),
             "morse_grid_chi2_noalloc: the grid needs %zu table values "
             "(n_u0 + 2 n_alpha + 2 n_t0 + 2 n_tE) but at most %zu fit; use "
             "morse_grid_chi2",
             tab_n, kMaxTable);
    return MORSE_EINVAL;
  }
  double h[kMaxTable];
  const double dlt = (2.0 * map->L) / (double)map->npix;
  morse::table_host(g, ev->t_ref, dlt, h);
  morse::Tables T;
  morse::tables_at(g, base, &T);
  e = cudaMemcpyAsync(T.u0v, h, tab_n * sizeof(double),
                      cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    snprintf(ctx->err, sizeof(ctx->err), "table upload: %s",
             cudaGetErrorString(e));
    return MORSE_ECUDA;
  }
  e = morse::launch_slab(T.u0v, T.ca, T.sa, g->n_u0, g->n_alpha, map->L,
                         T.slab, ctx->stream);
  if (e != cudaSuccess) {
    snprintf(ctx->err, sizeof(ctx->err), "line slabs: %s",
             cudaGetErrorString(e));
    return MORSE_ECUDA;
  }

  // search parameters from the same setters as morse_grid_chi2
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  morse::map_params(map, &P);
  P.quadh = h16 ? map->quadh : nullptr;
  morse::event_params(ev, &P);
  morse::grid_params(g, T, &P);
  P.first = 0;
  P.count = count;
  P.stride = 1;
  morse::set_groups(&P);
  P.partial = (morse::Entry *)(base + off_a);
  // status words: the grid-wide pruning threshold (all-ones = +inf) and the
  // error word of the block locks
  unsigned long long *words = (unsigned long long *)(base + off_w);
  P.gthr = &words[0];
  P.err = (unsigned int *)&words[1];
  e = cudaMemsetAsync(&words[0], 0xFF, sizeof(unsigned long long),
                      ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(&words[1], 0, sizeof(unsigned long long),
                        ctx->stream);
  if (e == cudaSuccess)
    e = morse::launch_search(P, false, ep_smem, grid, smem, ctx->stream);
  morse::Entry *sel = nullptr;
  int levels = 0;
  if (e == cudaSuccess)
    e = morse::launch_topk_merge((morse::Entry *)(base + off_a),
                                 (morse::Entry *)(base + off_b), grid, K, &sel,
                                 &levels, ctx->stream);
  morse_fit *fits = (morse_fit *)(base + off_fit);
  if (e == cudaSuccess) {
    morse::FillParams F;
    F.S = P;
    F.sel = sel;
    F.k = K;
    F.t0abs = T.t0abs;
    F.tEv = T.tEv;
    F.out = fits;
    e = morse::launch_fill(F, ctx->stream);
  }
  if (e == cudaSuccess) {
    ctx->launches += 3 + (uint64_t)levels;
    e = cudaMemcpyAsync(out, fits, sizeof(morse_fit) * K,
                        cudaMemcpyDeviceToHost, ctx->stream);
  }
  unsigned int errword = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&errword, &words[1], sizeof(errword),
                        cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    snprintf(ctx->err, sizeof(ctx->err), "no-alloc search: %s",
             cudaGetErrorString(e));
    return MORSE_ECUDA;
  }
  if (errword & 2u)
    return set_err(ctx, MORSE_ECUDA,
                   "bounds check: a texel index fell outside the map");
  if (errword)
    return set_err(ctx, MORSE_ETIMEOUT,
                   "a search block could not take its top-K lock; results "
                   "are incomplete");
  return MORSE_OK;
}
