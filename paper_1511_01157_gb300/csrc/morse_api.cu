// Host runtime of the MORSE GB300 library: contexts, handles, argument
// checks, workspaces, per-call kernel timing and the extern "C" entry
// points declared in morse.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "morse_internal.cuh"

using morse::Entry;

namespace {

morse_status fail(morse_ctx *ctx, morse_status st, const char *fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

morse_status cuda_fail(morse_ctx *ctx, cudaError_t e, const char *where) {
  return fail(ctx, MORSE_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define MORSE_CUDA(ctx, expr)                                     \
  do {                                                            \
    cudaError_t e_ = (expr);                                      \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #expr);    \
  } while (0)

#define MORSE_TRY(expr)                     \
  do {                                      \
    morse_status s_ = (expr);               \
    if (s_ != MORSE_OK) return s_;          \
  } while (0)

// Grow-only device workspace.
morse_status ws_reserve(morse_ctx *ctx, size_t bytes, void **out) {
  if (bytes > ctx->ws_bytes) {
    if (ctx->ws) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->ws);
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
    }
    size_t want = bytes + bytes / 4 + 4096;
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, MORSE_ENOMEM, "workspace of %zu bytes", want);
    }
    ctx->ws_bytes = want;
  }
  *out = ctx->ws;
  return MORSE_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- timing
void call_begin(morse_ctx *ctx) {
  ctx->rec_kind.clear();
  for (int k = 0; k < KT_COUNT; ++k) ctx->kernel_ms[k] = 0.0;
}

int t_begin(morse_ctx *ctx, int kind) {
  size_t r = ctx->rec_kind.size();
  while (ctx->evpool.size() < 2 * (r + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    ctx->evpool.push_back(e);
  }
  ctx->rec_kind.push_back(kind);
  cudaEventRecord(ctx->evpool[2 * r], ctx->stream);
  return (int)r;
}

void t_end(morse_ctx *ctx, int r) {
  if (r >= 0) cudaEventRecord(ctx->evpool[2 * (size_t)r + 1], ctx->stream);
}

// after the stream has synchronised
void call_collect(morse_ctx *ctx) {
  for (size_t r = 0; r < ctx->rec_kind.size(); ++r) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->evpool[2 * r], ctx->evpool[2 * r + 1]) ==
        cudaSuccess)
      ctx->kernel_ms[ctx->rec_kind[r]] += ms;
    else
      cudaGetLastError();
  }
  ctx->rec_kind.clear();
}

morse_status sync_and_collect(morse_ctx *ctx, const char *what) {
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  call_collect(ctx);
  return MORSE_OK;
}

// ---------------------------------------------------------------- checks
bool is_fin(double x) { return std::isfinite(x); }

morse_status check_grid(morse_ctx *ctx, const morse_grid *g) {
  if (!g) return fail(ctx, MORSE_EINVAL, "grid is NULL");
  if (g->n_u0 < 1 || g->n_alpha < 1 || g->n_t0 < 1 || g->n_tE < 1)
    return fail(ctx, MORSE_EINVAL, "grid axes need at least one value");
  if (!is_fin(g->u0_lo) || !is_fin(g->u0_hi) || !is_fin(g->t0_lo) ||
      !is_fin(g->t0_hi) || !is_fin(g->tE_lo) || !is_fin(g->tE_hi))
    return fail(ctx, MORSE_EINVAL, "grid bounds must be finite");
  if (!(g->tE_lo > 0.0) || !(g->tE_hi > 0.0))
    return fail(ctx, MORSE_EINVAL, "tE bounds must be > 0");
  if (g->u0_log && (!(g->u0_lo > 0.0) || !(g->u0_hi > 0.0)))
    return fail(ctx, MORSE_EINVAL, "log-spaced u0 needs positive bounds");
  if (g->top_k < 1 || g->top_k > 4096)
    return fail(ctx, MORSE_EINVAL, "top_k must be in [1, 4096]");
  double total = (double)g->n_u0 * g->n_alpha * g->n_t0 * g->n_tE;
  if (total > 9.0e15)
    return fail(ctx, MORSE_EINVAL, "grid has too many trajectories");
  return MORSE_OK;
}

long long grid_size(const morse_grid *g) {
  return (long long)g->n_u0 * g->n_alpha * g->n_t0 * g->n_tE;
}

struct BuildSpec {
  double s, q, L, X;
  int npix;
  int64_t nray;
  bool fp64;
  bool fp16;  // also write the FP16 log10 table and search through it
};

morse_status check_build(morse_ctx *ctx, double s, double q, double extent,
                         int npix, int64_t rays_per_axis,
                         const morse_map_opts *opts, BuildSpec *b) {
  if (!(s > 0.0) || !is_fin(s) || !(q > 0.0) || !is_fin(q))
    return fail(ctx, MORSE_EINVAL, "s and q must be finite and > 0");
  if (!(extent > 0.0) || !is_fin(extent))
    return fail(ctx, MORSE_EINVAL, "extent must be finite and > 0");
  if (npix < 2 || npix > 16384)
    return fail(ctx, MORSE_EINVAL, "npix must be in [2, 16384]");
  if (rays_per_axis < 1 || rays_per_axis > 2147483647LL)
    return fail(ctx, MORSE_EINVAL, "rays_per_axis must be in [1, 2^31-1]");
  double X = 1.5 * extent;
  int deflect = MORSE_DEFLECT_FP64;
  if (opts) {
    if (opts->image_halfwidth > 0.0) X = opts->image_halfwidth;
    if (!is_fin(X)) return fail(ctx, MORSE_EINVAL, "image_halfwidth");
    deflect = opts->deflect;
    int store = opts->store | MORSE_STORE_FP32;
    if (deflect != MORSE_DEFLECT_FP64 && deflect != MORSE_DEFLECT_FP32)
      return fail(ctx, MORSE_EINVAL, "unknown deflect mode %d", deflect);
    if (store & ~(MORSE_STORE_FP32 | MORSE_STORE_FP16LOG))
      return fail(ctx, MORSE_EINVAL, "unknown store flags %d", store);
    b->fp16 = (store & MORSE_STORE_FP16LOG) != 0;
  } else {
    b->fp16 = false;
  }
  b->s = s;
  b->q = q;
  b->L = extent;
  b->X = X;
  b->npix = npix;
  b->nray = rays_per_axis;
  b->fp64 = deflect == MORSE_DEFLECT_FP64;
  return MORSE_OK;
}

// ---------------------------------------------------------------- maps
morse_map *map_alloc(morse_ctx *ctx, int npix, bool counts) {
  morse_map *m = (morse_map *)calloc(1, sizeof(morse_map));
  if (!m) return nullptr;
  m->ctx = ctx;
  m->npix = npix;
  size_t n = (size_t)npix * npix;
  m->qpitch = morse::quad_pitch(npix);
  bool ok = cudaMalloc(&m->A, n * sizeof(float)) == cudaSuccess &&
            cudaMalloc(&m->quad, (size_t)npix * m->qpitch * sizeof(float4)) ==
                cudaSuccess &&
            cudaMalloc(&m->tot, 2 * sizeof(unsigned long long)) == cudaSuccess;
  if (ok && counts)
    ok = cudaMalloc(&m->counts, n * sizeof(uint32_t)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (m->A) cudaFree(m->A);
    if (m->quad) cudaFree(m->quad);
    if (m->tot) cudaFree(m->tot);
    if (m->counts) cudaFree(m->counts);
    free(m);
    return nullptr;
  }
  m->has_counts = counts;
  return m;
}

// FP16 table storage of a map (allocated on first use)
bool map_ensure_half(morse_map *m) {
  if (m->quadh) return true;
  size_t n = (size_t)m->npix * m->npix;
  if (cudaMalloc(&m->hcodes, n * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&m->quadh, (size_t)m->npix * m->qpitch * sizeof(uint2)) !=
          cudaSuccess) {
    cudaGetLastError();
    if (m->hcodes) cudaFree(m->hcodes);
    m->hcodes = nullptr;
    m->quadh = nullptr;
    return false;
  }
  return true;
}

// Queue the FP16 table of the map's current FP32 values.
morse_status enqueue_half(morse_ctx *ctx, morse_map *m) {
  if (!map_ensure_half(m))
    return fail(ctx, MORSE_ENOMEM, "FP16 table of %d^2 texels", m->npix);
  MORSE_CUDA(ctx, morse::launch_half_from_A(m->A, m->npix, m->a_floor,
                                            m->hcodes, m->quadh, m->qpitch,
                                            ctx->stream));
  ctx->launches += 2;
  m->half_valid = true;
  return MORSE_OK;
}

void map_release(morse_map *m) {
  if (!m) return;
  if (m->hcodes) cudaFree(m->hcodes);
  if (m->quadh) cudaFree(m->quadh);
  if (m->A) cudaFree(m->A);
  if (m->quad) cudaFree(m->quad);
  if (m->tot) cudaFree(m->tot);
  if (m->counts) cudaFree(m->counts);
  free(m);
}

// Queue the ray shooting and the texel conversion into existing storage
// (no host synchronisation).
morse_status enqueue_build(morse_ctx *ctx, morse_map *m, const BuildSpec &b) {
  m->L = b.L;
  m->s = b.s;
  m->q = b.q;
  m->X = b.X;
  m->nray = b.nray;
  morse::RayParams P;
  memset(&P, 0, sizeof(P));
  P.e1 = 1.0 / (1.0 + b.q);
  P.e2 = b.q / (1.0 + b.q);
  P.xa = -(b.s * P.e2);
  P.xb = b.s * P.e1;
  P.X = b.X;
  P.h = (2.0 * b.X) / (double)b.nray;
  P.L = b.L;
  P.dlt = (2.0 * b.L) / (double)b.npix;
  P.e1f = (float)P.e1;
  P.e2f = (float)P.e2;
  P.xaf = (float)P.xa;
  P.xbf = (float)P.xb;
  P.x0f = (float)(-b.X + 0.5 * P.h);
  P.hf = (float)P.h;
  P.invdf = (float)(1.0 / P.dlt);
  P.offf = (float)(b.L / P.dlt);
  P.npixf = (float)b.npix;
  P.npix = b.npix;
  P.nray = b.nray;
  P.tiles_x = (int)((b.nray + morse::kRayTile - 1) / morse::kRayTile);
  P.tiles_y = P.tiles_x;
  P.counts = m->counts;
  P.tot = m->tot;
  size_t n = (size_t)b.npix * b.npix;
  MORSE_CUDA(ctx, cudaMemsetAsync(m->counts, 0, n * sizeof(uint32_t),
                                  ctx->stream));
  MORSE_CUDA(ctx, cudaMemsetAsync(m->tot, 0, 2 * sizeof(unsigned long long),
                                  ctx->stream));
  long long tiles = (long long)P.tiles_x * P.tiles_y;
  int grid = (int)std::min<long long>(
      tiles, (long long)morse::rayshoot_blocks_per_sm() * ctx->sm_count);
  int r = t_begin(ctx, KT_RAY);
  MORSE_CUDA(ctx, morse::launch_rayshoot(P, b.fp64, grid, ctx->stream));
  t_end(ctx, r);
  ctx->launches += 1;
  const double f = (P.h * P.h) / (P.dlt * P.dlt);
  r = t_begin(ctx, KT_MAP);
  MORSE_CUDA(ctx, morse::launch_counts_to_map(m->counts, b.npix, f, m->A,
                                              m->quad, m->qpitch,
                                              ctx->stream));
  // FP16 floor: half a ray, 0.5 h^2 / Delta^2
  m->a_floor = 0.5 * f;
  m->half_valid = false;
  m->lookup = MORSE_STORE_FP32;
  if (b.fp16) {
    MORSE_TRY(enqueue_half(ctx, m));
    m->lookup = MORSE_STORE_FP16LOG;
  }
  t_end(ctx, r);
  ctx->launches += 1;
  return MORSE_OK;
}

// ---------------------------------------------------------------- search
void axis(double lo, double hi, int n, int logsp, std::vector<double> &out) {
  out.resize(n);
  for (int i = 0; i < n; ++i) {
    double f = (n > 1) ? (double)i / (double)(n - 1) : 0.0;
    out[i] = logsp ? exp(log(lo) + (log(hi) - log(lo)) * f)
                   : lo + (hi - lo) * f;
  }
}

// Device grid tables: u0, cos/sin alpha, t0 - t_ref, 1/(tE Delta), plus the
// absolute t0 and tE for the output records.
struct Tables {
  double *u0v, *ca, *sa, *t0rel, *invtEd, *t0abs, *tEv;
};

size_t tables_bytes(const morse_grid *g) {
  return sizeof(double) *
         (size_t)(g->n_u0 + 2 * g->n_alpha + 2 * g->n_t0 + 2 * g->n_tE);
}

morse_status upload_tables(morse_ctx *ctx, const morse_grid *g, double t_ref,
                           double dlt, void *dev, Tables *T) {
  std::vector<double> u0, t0, tE, h;
  axis(g->u0_lo, g->u0_hi, g->n_u0, g->u0_log, u0);
  axis(g->t0_lo, g->t0_hi, g->n_t0, 0, t0);
  axis(g->tE_lo, g->tE_hi, g->n_tE, g->tE_log, tE);
  h.reserve(tables_bytes(g) / sizeof(double));
  h.insert(h.end(), u0.begin(), u0.end());
  for (int k = 0; k < g->n_alpha; ++k)
    h.push_back(cos(2.0 * M_PI * (double)k / (double)g->n_alpha));
  for (int k = 0; k < g->n_alpha; ++k)
    h.push_back(sin(2.0 * M_PI * (double)k / (double)g->n_alpha));
  for (double v : t0) h.push_back(v - t_ref);
  for (double v : tE) h.push_back(1.0 / (v * dlt));
  h.insert(h.end(), t0.begin(), t0.end());
  h.insert(h.end(), tE.begin(), tE.end());
  double *d = (double *)dev;
  T->u0v = d;
  T->ca = T->u0v + g->n_u0;
  T->sa = T->ca + g->n_alpha;
  T->t0rel = T->sa + g->n_alpha;
  T->invtEd = T->t0rel + g->n_t0;
  T->t0abs = T->invtEd + g->n_tE;
  T->tEv = T->t0abs + g->n_t0;
  // ordered on the context stream, then waited for: the host vector is
  // pageable and dies on return
  MORSE_CUDA(ctx, cudaMemcpyAsync(dev, h.data(), h.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, ctx->stream));
  MORSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return MORSE_OK;
}

void map_params(const morse_map *map, morse::SearchParams *P) {
  const double dlt = (2.0 * map->L) / (double)map->npix;
  P->quad = map->quad;
  P->quadh = morse::map_h16(map) ? map->quadh : nullptr;
  P->qpitch = map->qpitch;
  P->qidx0 = (unsigned)(map->npix / 2 - 0x4B400000) *
             (unsigned)(map->qpitch + 1);
  P->npix = map->npix;
  P->half = map->npix / 2;
  P->vlo = -(float)(map->npix / 2) - 0.5f;
  P->vhi = (float)(map->npix - map->npix / 2) - 0.5f;
  P->vmin = -(float)(map->npix / 2);
  P->vmax = (float)(map->npix - map->npix / 2 - 1);
  P->L = map->L;
  P->dlt = dlt;
  P->coff = 0.5 * map->npix - (double)(map->npix / 2) - 0.5;
  P->voff = (float)(-P->coff);
  P->dltf = (float)dlt;
  P->invDf = (float)(1.0 / dlt);
  P->invD = 1.0 / dlt;
}

void event_params(const morse_event *ev, morse::SearchParams *P) {
  P->ep = ev->ep;
  P->n_ep = (int)ev->n;
  P->S1 = ev->S1;
  P->SF = ev->SF;
  P->SFF = ev->SFF;
  P->Fref = ev->Fref;
  const double m = (double)((ev->n + 31) / 32);
  P->gamma = (m + 10.0) * ldexp(1.0, -24);
}

void grid_params(const morse_grid *g, const Tables &T,
                 morse::SearchParams *P) {
  P->u0v = T.u0v;
  P->ca = T.ca;
  P->sa = T.sa;
  P->t0rel = T.t0rel;
  P->invtEd = T.invtEd;
  P->n_u0 = g->n_u0;
  P->n_alpha = g->n_alpha;
  P->n_t0 = g->n_t0;
  P->n_tE = g->n_tE;
  P->top_k = g->top_k;
}

morse_status check_pair(morse_ctx *ctx, const morse_event *ev,
                        const morse_map *map) {
  if (!ev || !map) return fail(ctx, MORSE_EINVAL, "event or map is NULL");
  if (ev->ctx != ctx || map->ctx != ctx)
    return fail(ctx, MORSE_EINVAL, "event and map must belong to ctx");
  return MORSE_OK;
}

// Launch shape and workspace layout of one search.
struct Plan {
  int K;
  bool dense, ep_smem;
  size_t smem;
  int grid;
  size_t off_tab, off_hdr, off_pa, off_pb, off_out, bytes;
};

// Device words of one search call (in the workspace header): the grid-wide
// pruning threshold, the error word and the exact-sweep counter.
struct Hdr {
  unsigned long long gthr;
  unsigned long long stat_exact;
  unsigned int err;
};

morse_status hdr_init(morse_ctx *ctx, char *base, const Plan &pl,
                      morse::SearchParams *P) {
  Hdr *h = (Hdr *)(base + pl.off_hdr);
  MORSE_CUDA(ctx, cudaMemsetAsync(h, 0, sizeof(Hdr), ctx->stream));
  MORSE_CUDA(ctx, cudaMemsetAsync(&h->gthr, 0xFF, sizeof(h->gthr),
                                  ctx->stream));
  P->gthr = &h->gthr;
  P->err = &h->err;
  P->stat_exact = &h->stat_exact;
  return MORSE_OK;
}

// Reset the pruning threshold between the maps of a sweep (it is per map).
morse_status hdr_reset_threshold(morse_ctx *ctx, char *base, const Plan &pl) {
  Hdr *h = (Hdr *)(base + pl.off_hdr);
  MORSE_CUDA(ctx, cudaMemsetAsync(&h->gthr, 0xFF, sizeof(h->gthr),
                                  ctx->stream));
  return MORSE_OK;
}

// After the stream has synchronised: read the header, report a lock that
// gave up as MORSE_ETIMEOUT.
morse_status hdr_check(morse_ctx *ctx, const Hdr &h) {
  ctx->last_exact = h.stat_exact;
  if (h.err & 2u)
    return fail(ctx, MORSE_ECUDA,
                "bounds check: a texel index fell outside the map (error "
                "0x%x); results are invalid", h.err);
  if (h.err & 1u)
    return fail(ctx, MORSE_ETIMEOUT,
                "a search block could not take its top-K lock (error 0x%x); "
                "results are incomplete", h.err);
  return MORSE_OK;
}

morse_status plan_search(morse_ctx *ctx, const morse_event *ev,
                         const morse_grid *g, long long first,
                         long long count, bool dense, bool h16,
                         long long n_out, Plan *pl) {
  const int K = dense ? 1 : g->top_k;
  const size_t fixed = morse::search_smem_bytes(0, dense ? 0 : K) -
                       (dense ? sizeof(Entry) * morse::kSearchWarps * 32 : 0);
  const size_t budget = ctx->smem_optin > 4096 ? ctx->smem_optin - 2048 : 0;
  const bool ep_smem =
      budget > fixed && (size_t)ev->n <= (budget - fixed) / sizeof(float4);
  const size_t smem = fixed + (ep_smem ? sizeof(float4) * (size_t)ev->n : 0);
  const int bps = morse::search_blocks_per_sm(dense, ep_smem, h16, smem);
  if (bps < 1)
    return fail(ctx, MORSE_EUNSUPPORTED,
                "search kernel does not fit (epochs %lld, top_k %d)",
                (long long)ev->n, K);
  long long groups =
      morse::main_groups((long long)g->n_t0 * g->n_tE, first, count);
  long long want = (groups + morse::kSearchWarps - 1) / morse::kSearchWarps;
  int grid = (int)std::min<long long>((long long)bps * ctx->sm_count, want);
  if (grid < 1) grid = 1;
  pl->K = K;
  pl->dense = dense;
  pl->ep_smem = ep_smem;
  pl->smem = smem;
  pl->grid = grid;
  pl->off_tab = 0;
  pl->off_hdr = align_up(tables_bytes(g), 256);
  pl->off_pa = pl->off_hdr + 256;
  size_t list_bytes = dense ? 0 : sizeof(Entry) * (size_t)grid * K;
  pl->off_pb = align_up(pl->off_pa + list_bytes, 256);
  pl->off_out = align_up(pl->off_pb + list_bytes, 256);
  size_t out_bytes = dense ? sizeof(double) * 3 * (size_t)n_out
                           : sizeof(morse_fit) * (size_t)K * (size_t)n_out;
  pl->bytes = pl->off_out + out_bytes;
  return MORSE_OK;
}

// Queue the top-K search of one map: search kernel, merge tree, fit fill
// into fits_dev[0..K).  No host synchronisation.
morse_status enqueue_topk(morse_ctx *ctx, const Plan &pl,
                          morse::SearchParams P, char *base,
                          const Tables &T, morse_fit *fits_dev) {
  P.partial = (Entry *)(base + pl.off_pa);
  int r;
  // pilot: a strided subset of ~sqrt(K N) trajectories (at least 16 K)
  // seeds the grid-wide pruning threshold
  const double want = std::max(16.0 * pl.K, std::sqrt((double)pl.K * P.count));
  const long long stride = (long long)(P.count / want);
  if (P.gthr && stride >= 4) {
    morse::SearchParams Q = P;
    Q.stride = stride;
    Q.count = (P.count + stride - 1) / stride;
    Q.tpg = morse::kTpgPilot;
    long long groups = (Q.count + Q.tpg - 1) / Q.tpg;
    int grid = (int)std::min<long long>(
        pl.grid, (groups + morse::kSearchWarps - 1) / morse::kSearchWarps);
    if (grid < 1) grid = 1;
    r = t_begin(ctx, KT_SEARCH);
    MORSE_CUDA(ctx, morse::launch_search(Q, false, pl.ep_smem, grid, pl.smem,
                                         ctx->stream));
    t_end(ctx, r);
    Entry *sel = nullptr;
    int levels = 0;
    r = t_begin(ctx, KT_MERGE);
    MORSE_CUDA(ctx, morse::launch_topk_merge((Entry *)(base + pl.off_pa),
                                             (Entry *)(base + pl.off_pb), grid,
                                             pl.K, &sel, &levels,
                                             ctx->stream));
    MORSE_CUDA(ctx, morse::launch_seed_threshold(sel, pl.K, P.gthr,
                                                 ctx->stream));
    t_end(ctx, r);
    ctx->launches += 2 + (uint64_t)levels;
  }
  r = t_begin(ctx, KT_SEARCH);
  MORSE_CUDA(ctx, morse::launch_search(P, false, pl.ep_smem, pl.grid, pl.smem,
                                       ctx->stream));
  t_end(ctx, r);
  ctx->launches += 1;
  Entry *sel = nullptr;
  int levels = 0;
  r = t_begin(ctx, KT_MERGE);
  MORSE_CUDA(ctx, morse::launch_topk_merge((Entry *)(base + pl.off_pa),
                                           (Entry *)(base + pl.off_pb),
                                           pl.grid, pl.K, &sel, &levels,
                                           ctx->stream));
  t_end(ctx, r);
  ctx->launches += (uint64_t)levels;
  morse::FillParams F;
  F.S = P;
  F.sel = sel;
  F.k = pl.K;
  F.t0abs = T.t0abs;
  F.tEv = T.tEv;
  F.out = fits_dev;
  r = t_begin(ctx, KT_FILL);
  MORSE_CUDA(ctx, morse::launch_fill(F, ctx->stream));
  t_end(ctx, r);
  ctx->launches += 1;
  return MORSE_OK;
}

// The (s, q) sweep behind morse_sweep and morse_search_sweep.
morse_status sweep_impl(morse_ctx *ctx, const morse_event *ev,
                        const double *s, const double *q, int n_maps,
                        double extent, int npix, int64_t rays_per_axis,
                        const morse_map_opts *opts, const morse_grid *grid,
                        morse_fit *out) {
  if (n_maps < 1 || !s || !q)
    return fail(ctx, MORSE_EINVAL, "need n_maps >= 1 and (s, q) lists");
  MORSE_TRY(check_grid(ctx, grid));
  std::vector<BuildSpec> specs((size_t)n_maps);
  for (int i = 0; i < n_maps; ++i)
    MORSE_TRY(check_build(ctx, s[i], q[i], extent, npix, rays_per_axis, opts,
                          &specs[(size_t)i]));
  if (ctx->sweep_map && ctx->sweep_map->npix != npix) {
    cudaStreamSynchronize(ctx->stream);
    map_release(ctx->sweep_map);
    ctx->sweep_map = nullptr;
  }
  if (!ctx->sweep_map) {
    ctx->sweep_map = map_alloc(ctx, npix, true);
    if (!ctx->sweep_map)
      return fail(ctx, MORSE_ENOMEM, "sweep map of %d^2 texels", npix);
  }
  morse_map *m = ctx->sweep_map;
  m->L = extent;
  const bool h16 = n_maps > 0 && specs[0].fp16;
  if (h16 && !map_ensure_half(m))
    return fail(ctx, MORSE_ENOMEM, "FP16 table of %d^2 texels", npix);
  Plan pl;
  MORSE_TRY(plan_search(ctx, ev, grid, 0, grid_size(grid), false, h16, n_maps,
                        &pl));
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, pl.bytes, &ws));
  char *base = (char *)ws;
  Tables T;
  const double dlt = (2.0 * extent) / (double)npix;
  MORSE_TRY(upload_tables(ctx, grid, ev->t_ref, dlt, base + pl.off_tab, &T));
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  map_params(m, &P);
  P.quadh = h16 ? m->quadh : nullptr;  // written by each build below
  event_params(ev, &P);
  grid_params(grid, T, &P);
  P.first = 0;
  P.count = grid_size(grid);
  P.stride = 1;
  morse::set_groups(&P);
  morse_fit *fits = (morse_fit *)(base + pl.off_out);
  MORSE_TRY(hdr_init(ctx, base, pl, &P));
  for (int i = 0; i < n_maps; ++i) {
    MORSE_TRY(enqueue_build(ctx, m, specs[(size_t)i]));
    if (i > 0) MORSE_TRY(hdr_reset_threshold(ctx, base, pl));
    MORSE_TRY(enqueue_topk(ctx, pl, P, base, T, fits + (size_t)i * pl.K));
  }
  Hdr h;
  MORSE_CUDA(ctx, cudaMemcpyAsync(&h, base + pl.off_hdr, sizeof(Hdr),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(out, fits,
                                  sizeof(morse_fit) * (size_t)pl.K * n_maps,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "sweep"));
  return hdr_check(ctx, h);
}

}  // namespace

extern "C" {

const char *morse_status_string(morse_status st) {
  switch (st) {
    case MORSE_OK: return "MORSE_OK";
    case MORSE_EINVAL: return "MORSE_EINVAL";
    case MORSE_ENOMEM: return "MORSE_ENOMEM";
    case MORSE_ECUDA: return "MORSE_ECUDA";
    case MORSE_ETIMEOUT: return "MORSE_ETIMEOUT";
    case MORSE_EDEGENERATE: return "MORSE_EDEGENERATE";
    case MORSE_EUNSUPPORTED: return "MORSE_EUNSUPPORTED";
  }
  return "MORSE_UNKNOWN";
}

#ifdef MORSE_CHECK_BOUNDS
const char *morse_version(void) {
  return "morse-gb300 0.1 sm_103a bounds-checked";
}
#else
const char *morse_version(void) { return "morse-gb300 0.1 sm_103a"; }
#endif

morse_status morse_create(morse_ctx **out, int device, void *cuda_stream) {
  if (!out) return MORSE_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return MORSE_ECUDA;
  }
  if (device < 0 || device >= ndev) return MORSE_EINVAL;
  morse_ctx *c = new (std::nothrow) morse_ctx();
  if (!c) return MORSE_ENOMEM;
  c->device = device;
  cudaDeviceProp prop;
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MORSE_ECUDA;
  }
  c->sm_count = prop.multiProcessorCount;
  c->smem_optin = prop.sharedMemPerBlockOptin;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
    c->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) !=
        cudaSuccess) {
      cudaGetLastError();
      delete c;
      return MORSE_ECUDA;
    }
    c->own_stream = true;
  }
  *out = c;
  return MORSE_OK;
}

void morse_destroy(morse_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->sweep_map) map_release(ctx->sweep_map);
  if (ctx->ws) cudaFree(ctx->ws);
  for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char *morse_last_error(const morse_ctx *ctx) {
  return ctx ? ctx->err : "no context";
}

morse_status morse_last_kernel_ms(const morse_ctx *ctx, int which,
                                  double *ms) {
  if (!ctx || !ms || which < 0 || which >= KT_COUNT) return MORSE_EINVAL;
  *ms = ctx->kernel_ms[which];
  return MORSE_OK;
}

morse_status morse_last_search_stats(const morse_ctx *ctx,
                                     uint64_t *exact_sweeps) {
  if (!ctx || !exact_sweeps) return MORSE_EINVAL;
  *exact_sweeps = ctx->last_exact;
  return MORSE_OK;
}

morse_status morse_launch_count(const morse_ctx *ctx, uint64_t *n) {
  if (!ctx || !n) return MORSE_EINVAL;
  *n = ctx->launches;
  return MORSE_OK;
}

// ------------------------------------------------------------------ maps
morse_status morse_build_map(morse_ctx *ctx, double s, double q,
                             double extent, int npix, int64_t rays_per_axis,
                             const morse_map_opts *opts, morse_map **out) {
  if (!ctx || !out) return MORSE_EINVAL;
  *out = nullptr;
  BuildSpec b;
  MORSE_TRY(check_build(ctx, s, q, extent, npix, rays_per_axis, opts, &b));
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  morse_map *m = map_alloc(ctx, npix, true);
  if (!m) return fail(ctx, MORSE_ENOMEM, "map of %d^2 texels", npix);
  morse_status st = enqueue_build(ctx, m, b);
  unsigned long long tot[2] = {0, 0};
  if (st == MORSE_OK) {
    cudaError_t e = cudaMemcpyAsync(tot, m->tot, sizeof(tot),
                                    cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "map totals");
  }
  if (st == MORSE_OK) st = sync_and_collect(ctx, "map build");
  if (st != MORSE_OK) {
    cudaStreamSynchronize(ctx->stream);
    map_release(m);
    return st;
  }
  m->off_map = tot[0];
  m->lost = tot[1];
  *out = m;
  return MORSE_OK;
}

morse_status morse_map_from_host(morse_ctx *ctx, const float *A, int npix,
                                 double extent, morse_map **out) {
  if (!ctx || !out || !A) return MORSE_EINVAL;
  *out = nullptr;
  if (npix < 2 || npix > 16384)
    return fail(ctx, MORSE_EINVAL, "npix must be in [2, 16384]");
  if (!(extent > 0.0) || !is_fin(extent))
    return fail(ctx, MORSE_EINVAL, "extent must be finite and > 0");
  size_t n = (size_t)npix * npix;
  for (size_t k = 0; k < n; ++k)
    if (!(A[k] >= 0.0f) || !std::isfinite(A[k]))
      return fail(ctx, MORSE_EINVAL, "map value %zu is negative or not finite",
                  k);
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  morse_map *m = map_alloc(ctx, npix, false);
  if (!m) return fail(ctx, MORSE_ENOMEM, "map of %d^2 texels", npix);
  m->L = extent;
  m->a_floor = 1e-6;
  m->lookup = MORSE_STORE_FP32;
  cudaError_t e = cudaMemcpyAsync(m->A, A, n * sizeof(float),
                                  cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    e = morse::launch_quads_from_A(m->A, npix, m->quad, m->qpitch,
                                   ctx->stream);
    ctx->launches += 1;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(ctx->stream);
    map_release(m);
    return cuda_fail(ctx, e, "map upload");
  }
  *out = m;
  return MORSE_OK;
}

morse_status morse_map_counts(const morse_map *map, uint32_t *host_counts,
                              uint64_t *off_map, uint64_t *lost) {
  if (!map) return MORSE_EINVAL;
  morse_ctx *ctx = map->ctx;
  if (!map->has_counts)
    return fail(ctx, MORSE_EINVAL, "map was not built by ray shooting");
  if (host_counts) {
    size_t n = (size_t)map->npix * map->npix;
    MORSE_CUDA(ctx, cudaMemcpyAsync(host_counts, map->counts,
                                    n * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, ctx->stream));
    MORSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (off_map) *off_map = map->off_map;
  if (lost) *lost = map->lost;
  return MORSE_OK;
}

morse_status morse_map_values(const morse_map *map, float *host_A) {
  if (!map || !host_A) return MORSE_EINVAL;
  morse_ctx *ctx = map->ctx;
  size_t n = (size_t)map->npix * map->npix;
  MORSE_CUDA(ctx, cudaMemcpyAsync(host_A, map->A, n * sizeof(float),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return MORSE_OK;
}

morse_status morse_map_info(const morse_map *map, int *npix, double *extent,
                            double *s, double *q) {
  if (!map) return MORSE_EINVAL;
  if (npix) *npix = map->npix;
  if (extent) *extent = map->L;
  if (s) *s = map->s;
  if (q) *q = map->q;
  return MORSE_OK;
}

morse_status morse_map_set_lookup(morse_map *map, int store) {
  if (!map) return MORSE_EINVAL;
  morse_ctx *ctx = map->ctx;
  if (store == MORSE_STORE_FP32) {
    map->lookup = MORSE_STORE_FP32;
    return MORSE_OK;
  }
  if (store != MORSE_STORE_FP16LOG)
    return fail(ctx, MORSE_EINVAL, "lookup must be MORSE_STORE_FP32 or "
                "MORSE_STORE_FP16LOG, not %d", store);
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  if (!map->half_valid) {
    call_begin(ctx);
    MORSE_TRY(enqueue_half(ctx, map));
    MORSE_TRY(sync_and_collect(ctx, "FP16 table"));
  }
  map->lookup = MORSE_STORE_FP16LOG;
  return MORSE_OK;
}

morse_status morse_map_half(const morse_map *map, uint16_t *host_codes,
                            double *a_floor) {
  if (!map) return MORSE_EINVAL;
  morse_ctx *ctx = map->ctx;
  if (!map->half_valid)
    return fail(ctx, MORSE_EINVAL, "map has no FP16 table");
  if (a_floor) *a_floor = map->a_floor;
  if (host_codes) {
    size_t n = (size_t)map->npix * map->npix;
    MORSE_CUDA(ctx, cudaMemcpyAsync(host_codes, map->hcodes,
                                    n * sizeof(uint16_t),
                                    cudaMemcpyDeviceToHost, ctx->stream));
    MORSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return MORSE_OK;
}

void morse_map_free(morse_map *map) {
  if (!map) return;
  cudaStreamSynchronize(map->ctx->stream);
  map_release(map);
}

// ------------------------------------------------------------------ events
morse_status morse_event_create(morse_ctx *ctx, const double *t,
                                const double *flux, const double *sigma,
                                int64_t n, double t_ref, morse_event **out) {
  if (!ctx || !out) return MORSE_EINVAL;
  *out = nullptr;
  if (!t || !flux || !sigma) return fail(ctx, MORSE_EINVAL, "NULL array");
  if (n < 3) return fail(ctx, MORSE_EINVAL, "need at least 3 epochs");
  if (n > 0x7fffffffLL) return fail(ctx, MORSE_EINVAL, "too many epochs");
  if (!is_fin(t_ref)) return fail(ctx, MORSE_EINVAL, "t_ref not finite");
  for (int64_t i = 0; i < n; ++i) {
    if (!is_fin(t[i]) || !is_fin(flux[i]) || !is_fin(sigma[i]))
      return fail(ctx, MORSE_EINVAL, "epoch %lld has a non-finite value",
                  (long long)i);
    if (!(sigma[i] > 0.0))
      return fail(ctx, MORSE_EINVAL, "epoch %lld has sigma <= 0",
                  (long long)i);
  }
  // the search needs the epochs in time order (a straight track crosses the
  // map in one time interval): store them sorted, ties in input order
  std::vector<int64_t> order((size_t)n);
  for (int64_t i = 0; i < n; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [t](int64_t a, int64_t b) { return t[a] < t[b]; });
  // weights, weighted mean flux, FP32 storage; the FP64 constants are sums
  // of the stored FP32 values so that the device data is self-consistent
  std::vector<float4> h((size_t)n);
  double sw = 0.0, swf = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double w = 1.0 / (sigma[i] * sigma[i]);
    sw += w;
    swf += w * flux[i];
  }
  const double Fref = swf / sw;
  double S1 = 0.0, SF = 0.0, SFF = 0.0;
  for (int64_t k = 0; k < n; ++k) {
    const int64_t i = order[(size_t)k];
    double w = 1.0 / (sigma[i] * sigma[i]);
    double fc = flux[i] - Fref;
    float4 v;
    v.x = (float)(t[i] - t_ref);
    v.y = (float)w;
    v.z = (float)(w * fc);
    v.w = (float)fc;
    if (!std::isfinite(v.y) || !std::isfinite(v.z) || v.y <= 0.0f)
      return fail(ctx, MORSE_EINVAL,
                  "epoch %lld: weight 1/sigma^2 outside FP32 range",
                  (long long)i);
    h[(size_t)k] = v;
    // constants of the quadratic the exact sweep evaluates: sum w Fc and
    // sum w Fc^2 with the stored w and Fc
    S1 += (double)v.y;
    SF += (double)v.y * (double)v.w;
    SFF += (double)v.y * (double)v.w * (double)v.w;
  }
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  morse_event *ev = (morse_event *)calloc(1, sizeof(morse_event));
  if (!ev) return fail(ctx, MORSE_ENOMEM, "event");
  if (cudaMalloc(&ev->ep, sizeof(float4) * (size_t)n) != cudaSuccess) {
    cudaGetLastError();
    free(ev);
    return fail(ctx, MORSE_ENOMEM, "event of %lld epochs", (long long)n);
  }
  cudaError_t e = cudaMemcpyAsync(ev->ep, h.data(), sizeof(float4) * (size_t)n,
                                  cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ev->ep);
    free(ev);
    return cuda_fail(ctx, e, "event upload");
  }
  ev->ctx = ctx;
  ev->n = n;
  ev->t_ref = t_ref;
  ev->S1 = S1;
  ev->SF = SF;
  ev->SFF = SFF;
  ev->Fref = Fref;
  *out = ev;
  return MORSE_OK;
}

void morse_event_free(morse_event *ev) {
  if (!ev) return;
  cudaStreamSynchronize(ev->ctx->stream);
  if (ev->ep) cudaFree(ev->ep);
  free(ev);
}

morse_status morse_event_info(const morse_event *ev, int64_t *n,
                              double *t_ref) {
  if (!ev) return MORSE_EINVAL;
  if (n) *n = ev->n;
  if (t_ref) *t_ref = ev->t_ref;
  return MORSE_OK;
}

// ------------------------------------------------------------------ search
morse_status morse_grid_chi2(morse_ctx *ctx, const morse_event *ev,
                             const morse_map *map, const morse_grid *grid,
                             morse_fit *out) {
  if (!ctx || !out) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  MORSE_TRY(check_grid(ctx, grid));
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  Plan pl;
  MORSE_TRY(plan_search(ctx, ev, grid, 0, grid_size(grid), false,
                        morse::map_h16(map), 1, &pl));
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, pl.bytes, &ws));
  char *base = (char *)ws;
  Tables T;
  const double dlt = (2.0 * map->L) / (double)map->npix;
  MORSE_TRY(upload_tables(ctx, grid, ev->t_ref, dlt, base + pl.off_tab, &T));
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  map_params(map, &P);
  event_params(ev, &P);
  grid_params(grid, T, &P);
  P.first = 0;
  P.count = grid_size(grid);
  P.stride = 1;
  morse::set_groups(&P);
  morse_fit *fits = (morse_fit *)(base + pl.off_out);
  MORSE_TRY(hdr_init(ctx, base, pl, &P));
  MORSE_TRY(enqueue_topk(ctx, pl, P, base, T, fits));
  Hdr h;
  MORSE_CUDA(ctx, cudaMemcpyAsync(&h, base + pl.off_hdr, sizeof(Hdr),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(out, fits, sizeof(morse_fit) * pl.K,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "grid search"));
  return hdr_check(ctx, h);
}

morse_status morse_grid_chi2_dense(morse_ctx *ctx, const morse_event *ev,
                                   const morse_map *map,
                                   const morse_grid *grid, int64_t first,
                                   int64_t count, double *chi2, double *Fs,
                                   double *Fb) {
  if (!ctx || !chi2) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  MORSE_TRY(check_grid(ctx, grid));
  long long total = grid_size(grid);
  if (first < 0 || count < 0 || first + count > total)
    return fail(ctx, MORSE_EINVAL, "range [%lld, %lld) outside the grid",
                (long long)first, (long long)(first + count));
  if (count == 0) return MORSE_OK;
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  Plan pl;
  MORSE_TRY(plan_search(ctx, ev, grid, first, count, true,
                        morse::map_h16(map), count, &pl));
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, pl.bytes, &ws));
  char *base = (char *)ws;
  Tables T;
  const double dlt = (2.0 * map->L) / (double)map->npix;
  MORSE_TRY(upload_tables(ctx, grid, ev->t_ref, dlt, base + pl.off_tab, &T));
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  map_params(map, &P);
  event_params(ev, &P);
  grid_params(grid, T, &P);
  P.first = first;
  P.count = count;
  P.stride = 1;
  morse::set_groups(&P);
  P.top_k = 1;
  P.dchi2 = (double *)(base + pl.off_out);
  P.dFs = P.dchi2 + count;
  P.dFb = P.dFs + count;
  MORSE_TRY(hdr_init(ctx, base, pl, &P));
  int r = t_begin(ctx, KT_SEARCH);
  MORSE_CUDA(ctx, morse::launch_search(P, true, pl.ep_smem, pl.grid, pl.smem,
                                       ctx->stream));
  t_end(ctx, r);
  ctx->launches += 1;
  MORSE_CUDA(ctx, cudaMemcpyAsync(chi2, P.dchi2, sizeof(double) * count,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  if (Fs)
    MORSE_CUDA(ctx, cudaMemcpyAsync(Fs, P.dFs, sizeof(double) * count,
                                    cudaMemcpyDeviceToHost, ctx->stream));
  if (Fb)
    MORSE_CUDA(ctx, cudaMemcpyAsync(Fb, P.dFb, sizeof(double) * count,
                                    cudaMemcpyDeviceToHost, ctx->stream));
  Hdr h;
  MORSE_CUDA(ctx, cudaMemcpyAsync(&h, base + pl.off_hdr, sizeof(Hdr),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "dense search"));
  return hdr_check(ctx, h);
}

morse_status morse_sweep(morse_ctx *ctx, const morse_event *ev,
                         const double *s, const double *q, int n_maps,
                         double extent, int npix, int64_t rays_per_axis,
                         const morse_map_opts *opts, const morse_grid *grid,
                         morse_fit *out) {
  if (!ctx || !out) return MORSE_EINVAL;
  if (!ev || ev->ctx != ctx)
    return fail(ctx, MORSE_EINVAL, "event missing or of another ctx");
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  return sweep_impl(ctx, ev, s, q, n_maps, extent, npix, rays_per_axis, opts,
                    grid, out);
}

morse_status morse_search_sweep(morse_ctx *ctx, const double *t,
                                const double *flux, const double *sigma,
                                int64_t n, double t_ref, const double *s,
                                const double *q, int n_maps, double extent,
                                int npix, int64_t rays_per_axis,
                                const morse_map_opts *opts,
                                const morse_grid *grid, morse_fit *out) {
  if (!ctx || !out) return MORSE_EINVAL;
  MORSE_TRY(check_grid(ctx, grid));
  morse_event *ev = nullptr;
  MORSE_TRY(morse_event_create(ctx, t, flux, sigma, n, t_ref, &ev));
  call_begin(ctx);
  morse_status st = sweep_impl(ctx, ev, s, q, n_maps, extent, npix,
                               rays_per_axis, opts, grid, out);
  morse_event_free(ev);
  return st;
}

morse_status morse_search(morse_ctx *ctx, const double *t, const double *flux,
                          const double *sigma, int64_t n, double t_ref,
                          double s, double q, double extent, int npix,
                          int64_t rays_per_axis, const morse_map_opts *opts,
                          const morse_grid *grid, morse_fit *out) {
  return morse_search_sweep(ctx, t, flux, sigma, n, t_ref, &s, &q, 1, extent,
                            npix, rays_per_axis, opts, grid, out);
}

morse_status morse_lightcurve(morse_ctx *ctx, const morse_map *map,
                              double t0, double tE, double u0, double alpha,
                              const double *t, int64_t n, double *A_out) {
  if (!ctx || !map || !t || !A_out) return MORSE_EINVAL;
  if (map->ctx != ctx) return fail(ctx, MORSE_EINVAL, "map of another ctx");
  if (!is_fin(t0) || !is_fin(tE) || !is_fin(u0) || !is_fin(alpha) ||
      !(tE > 0.0))
    return fail(ctx, MORSE_EINVAL, "trajectory parameters");
  if (n < 0 || n > 0x7fffffffLL) return fail(ctx, MORSE_EINVAL, "n");
  if (n == 0) return MORSE_OK;
  for (int64_t i = 0; i < n; ++i)
    if (!is_fin(t[i])) return fail(ctx, MORSE_EINVAL, "time not finite");
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  std::vector<float> tf((size_t)n);
  for (int64_t i = 0; i < n; ++i) tf[(size_t)i] = (float)(t[i] - t0);
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, 2 * sizeof(float) * (size_t)n, &ws));
  float *dt = (float *)ws, *dA = dt + n;
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  map_params(map, &P);
  const double dlt = (2.0 * map->L) / (double)map->npix;
  const double k = 1.0 / (tE * dlt);
  const double c = cos(alpha), s = sin(alpha);
  const float ax = (float)(c * k), ay = (float)(s * k);
  const float bx = (float)((-u0 * s) / dlt + P.coff);
  const float by = (float)((u0 * c) / dlt + P.coff);
  const float kt = (float)(1.0 / tE), u02 = (float)(u0 * u0);
  std::vector<float> hA((size_t)n);
  MORSE_CUDA(ctx, cudaMemcpyAsync(dt, tf.data(), sizeof(float) * n,
                                  cudaMemcpyHostToDevice, ctx->stream));
  MORSE_CUDA(ctx, morse::launch_lightcurve(P, ax, bx, ay, by, kt, 0.0f, u02,
                                           dt, (int)n, dA, ctx->stream));
  ctx->launches += 1;
  MORSE_CUDA(ctx, cudaMemcpyAsync(hA.data(), dA, sizeof(float) * n,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "light curve"));
  for (int64_t i = 0; i < n; ++i) A_out[i] = hA[(size_t)i];
  return MORSE_OK;
}

// ------------------------------------------------------------------ refine
static morse_status check_theta(morse_ctx *ctx, const double *theta,
                                int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < 4; ++k)
      if (!is_fin(theta[4 * i + k]))
        return fail(ctx, MORSE_EINVAL, "theta[%lld] is not finite",
                    (long long)i);
    if (!(theta[4 * i + 1] > 0.0))
      return fail(ctx, MORSE_EINVAL, "theta[%lld]: tE must be > 0",
                  (long long)i);
  }
  return MORSE_OK;
}

morse_status morse_chi2_grad_dev(morse_ctx *ctx, const morse_event *ev,
                                 const morse_map *map, const double *theta,
                                 int64_t n, double *chi2, double *grad) {
  if (!ctx) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  if (n < 0 || n > 0x7fffffffLL)
    return fail(ctx, MORSE_EINVAL, "n out of range");
  if (n == 0) return MORSE_OK;
  if (!theta || !chi2) return fail(ctx, MORSE_EINVAL, "NULL device array");
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  map_params(map, &P);
  event_params(ev, &P);
  MORSE_CUDA(ctx, morse::launch_theta(P, theta, (int)n, ev->t_ref, chi2,
                                      grad, nullptr, nullptr, nullptr,
                                      nullptr, ctx->stream));
  ctx->launches += 1;
  return MORSE_OK;
}

morse_status morse_chi2_grad(morse_ctx *ctx, const morse_event *ev,
                             const morse_map *map, const double *theta,
                             int64_t n, double *chi2, double *grad,
                             double *Fs, double *Fb) {
  if (!ctx) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  if (n < 0 || n > 0x7fffffffLL)
    return fail(ctx, MORSE_EINVAL, "n out of range");
  if (n == 0) return MORSE_OK;
  if (!theta || !chi2) return fail(ctx, MORSE_EINVAL, "NULL array");
  MORSE_TRY(check_theta(ctx, theta, n));
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  // workspace: theta | chi2 | grad | Fs | Fb
  const size_t nn = (size_t)n;
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, sizeof(double) * nn * 11 + 1024, &ws));
  double *d_th = (double *)ws, *d_c = d_th + 4 * nn, *d_g = d_c + nn;
  double *d_fs = d_g + 4 * nn, *d_fb = d_fs + nn;
  MORSE_CUDA(ctx, cudaMemcpyAsync(d_th, theta, sizeof(double) * 4 * nn,
                                  cudaMemcpyHostToDevice, ctx->stream));
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  map_params(map, &P);
  event_params(ev, &P);
  int r = t_begin(ctx, KT_ADJ);
  MORSE_CUDA(ctx, morse::launch_theta(P, d_th, (int)n, ev->t_ref, d_c, d_g,
                                      nullptr, d_fs, d_fb, nullptr,
                                      ctx->stream));
  t_end(ctx, r);
  ctx->launches += 1;
  MORSE_CUDA(ctx, cudaMemcpyAsync(chi2, d_c, sizeof(double) * nn,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  if (grad)
    MORSE_CUDA(ctx, cudaMemcpyAsync(grad, d_g, sizeof(double) * 4 * nn,
                                    cudaMemcpyDeviceToHost, ctx->stream));
  if (Fs)
    MORSE_CUDA(ctx, cudaMemcpyAsync(Fs, d_fs, sizeof(double) * nn,
                                    cudaMemcpyDeviceToHost, ctx->stream));
  if (Fb)
    MORSE_CUDA(ctx, cudaMemcpyAsync(Fb, d_fb, sizeof(double) * nn,
                                    cudaMemcpyDeviceToHost, ctx->stream));
  return sync_and_collect(ctx, "chi2 gradient");
}

morse_status morse_refine(morse_ctx *ctx, const morse_event *ev,
                          const morse_map *map, const morse_fit *starts,
                          int n, int iters, int method, morse_fit *out) {
  if (!ctx) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  if (method != MORSE_REFINE_LM)
    return fail(ctx, MORSE_EUNSUPPORTED, "refine method %d", method);
  if (n < 0 || iters < 0 || iters > 100000)
    return fail(ctx, MORSE_EINVAL, "n or iters out of range");
  if (n == 0) return MORSE_OK;
  if (!starts || !out) return fail(ctx, MORSE_EINVAL, "NULL array");
  for (int i = 0; i < n; ++i) {
    const double th[4] = {starts[i].t0, starts[i].tE, starts[i].u0,
                          starts[i].alpha};
    MORSE_TRY(check_theta(ctx, th, 1));
  }
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  const size_t nn = (size_t)n;
  // workspace: 36 doubles + 1 int per trajectory, starts, records
  const size_t dbl = nn * 36, bytes = sizeof(double) * dbl + sizeof(int) * nn +
                                      2 * sizeof(morse_fit) * nn + 4096;
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, bytes, &ws));
  double *d = (double *)ws;
  morse::RefineState S;
  S.th_cur = d;
  S.th_best = S.th_cur + 4 * nn;
  S.chi2_cur = S.th_best + 4 * nn;
  S.chi2_best = S.chi2_cur + nn;
  S.lam = S.chi2_best + nn;
  S.g_cur = S.lam + nn;
  S.g_best = S.g_cur + 4 * nn;
  S.H_cur = S.g_best + 4 * nn;
  S.H_best = S.H_cur + 10 * nn;
  S.Fs = S.H_best + 10 * nn;
  S.Fb = S.Fs + nn;
  S.flags = (int *)(S.Fb + nn);
  morse_fit *d_starts = (morse_fit *)align_up(
      (size_t)(S.flags + nn), alignof(morse_fit));
  morse_fit *d_out = d_starts + nn;
  MORSE_CUDA(ctx, cudaMemcpyAsync(d_starts, starts, sizeof(morse_fit) * nn,
                                  cudaMemcpyHostToDevice, ctx->stream));
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  map_params(map, &P);
  event_params(ev, &P);
  MORSE_CUDA(ctx, morse::launch_lm_init(S, d_starts, n, 1e-3, ctx->stream));
  ctx->launches += 1;
  if (iters > 0) {
    // one iteration (evaluate at theta_cur, then step) as a CUDA graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    MORSE_CUDA(ctx, cudaStreamBeginCapture(ctx->stream,
                                           cudaStreamCaptureModeThreadLocal));
    cudaError_t e1 = morse::launch_theta(P, S.th_cur, n, ev->t_ref,
                                         S.chi2_cur, S.g_cur, S.H_cur,
                                         nullptr, nullptr, nullptr,
                                         ctx->stream);
    cudaError_t e2 = morse::launch_lm_step(S, n, ctx->stream);
    cudaError_t e3 = cudaStreamEndCapture(ctx->stream, &graph);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return cuda_fail(ctx, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3),
                       "refine graph capture");
    }
    cudaError_t e4 = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e4 != cudaSuccess) return cuda_fail(ctx, e4, "refine graph");
    int r = t_begin(ctx, KT_LM);
    for (int it = 0; it < iters; ++it) {
      cudaError_t e = cudaGraphLaunch(exec, ctx->stream);
      if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return cuda_fail(ctx, e, "refine graph launch");
      }
    }
    t_end(ctx, r);
    ctx->launches += 2 * (uint64_t)iters;
    MORSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaGraphExecDestroy(exec);
  }
  // evaluate at the best point (the start if no iteration improved on it)
  int r = t_begin(ctx, KT_ADJ);
  MORSE_CUDA(ctx, morse::launch_theta(P, S.th_best, n, ev->t_ref, S.chi2_cur,
                                      nullptr, nullptr, S.Fs, S.Fb, S.flags,
                                      ctx->stream));
  t_end(ctx, r);
  MORSE_CUDA(ctx, morse::launch_lm_finish(S, d_starts, n, d_out, ctx->stream));
  ctx->launches += 2;
  MORSE_CUDA(ctx, cudaMemcpyAsync(out, d_out, sizeof(morse_fit) * nn,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  return sync_and_collect(ctx, "refine");
}

morse_status morse_topk_merge(const morse_fit *const *lists,
                              const int *counts, int n_lists, int k,
                              morse_fit *out) {
  if (!out || k < 1 || n_lists < 0 || (n_lists > 0 && (!lists || !counts)))
    return MORSE_EINVAL;
  std::vector<morse_fit> all;
  for (int i = 0; i < n_lists; ++i) {
    if (counts[i] < 0 || (counts[i] > 0 && !lists[i])) return MORSE_EINVAL;
    for (int j = 0; j < counts[i]; ++j)
      if (lists[i][j].idx >= 0) all.push_back(lists[i][j]);
  }
  std::sort(all.begin(), all.end(), [](const morse_fit &a, const morse_fit &b) {
    return a.chi2 < b.chi2 || (a.chi2 == b.chi2 && a.idx < b.idx);
  });
  for (int j = 0; j < k; ++j) {
    if (j < (int)all.size()) {
      out[j] = all[(size_t)j];
    } else {
      memset(&out[j], 0, sizeof(morse_fit));
      out[j].chi2 = INFINITY;
      out[j].idx = -1;
    }
  }
  return MORSE_OK;
}

}  // extern "C"
