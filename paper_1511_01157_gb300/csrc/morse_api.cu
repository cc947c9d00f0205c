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
#include <array>
#include <cmath>
#include <new>
#include <vector>

#include "morse_internal.cuh"

using morse::Entry;

namespace {

// spins (of ~64 ns) before a block top-K lock wait gives up: ~67 ms
constexpr unsigned kDefaultSpinLimit = 1u << 20;

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
    if (morse::dev_alloc(ctx, &ctx->ws, want) != cudaSuccess) {
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

// Record a timing event on the context stream; while the stream is being
// captured the record becomes an external event node of the graph, which
// still timestamps the event when the graph runs.
void record(morse_ctx *ctx, cudaEvent_t e) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) == cudaSuccess &&
      cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(e, ctx->stream);
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
  record(ctx, ctx->evpool[2 * r]);
  return (int)r;
}

void t_end(morse_ctx *ctx, int r) {
  if (r >= 0) record(ctx, ctx->evpool[2 * (size_t)r + 1]);
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
  if (!(g->a_min >= 0.0f) || !std::isfinite(g->a_min))
    return fail(ctx, MORSE_EINVAL, "a_min must be finite and >= 0");
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
  bool poly;  // the lens polynomial per texel instead of ray shooting
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
    if (opts->generator != MORSE_GEN_RAYS && opts->generator != MORSE_GEN_POLY)
      return fail(ctx, MORSE_EINVAL, "unknown map generator %d",
                  opts->generator);
    b->poly = opts->generator == MORSE_GEN_POLY;
  } else {
    b->fp16 = false;
    b->poly = false;
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
  bool ok =
      morse::dev_alloc(ctx, (void **)&m->A, n * sizeof(float)) ==
          cudaSuccess &&
      morse::dev_alloc(ctx, (void **)&m->quad,
                       morse::quad_count(npix) * sizeof(float4)) ==
          cudaSuccess &&
      morse::dev_alloc(ctx, (void **)&m->tot,
                       4 * sizeof(unsigned long long)) == cudaSuccess;
  if (ok && counts)
    ok = morse::dev_alloc(ctx, (void **)&m->counts,
                          n * sizeof(uint32_t)) == cudaSuccess;
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
  if (morse::dev_alloc(m->ctx, (void **)&m->hcodes, n * sizeof(uint16_t)) !=
          cudaSuccess ||
      morse::dev_alloc(m->ctx, (void **)&m->quadh,
                       morse::quad_count(m->npix) * sizeof(uint2)) !=
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
  if (b.poly) {
    // the lens polynomial at every texel centre: no rays, no counts
    m->X = 0.0;
    m->nray = 0;
    m->has_counts = false;
    m->a_floor = 1e-6;
    m->half_valid = false;
    m->lookup = MORSE_STORE_FP32;
    MORSE_CUDA(ctx, cudaMemsetAsync(m->tot, 0, 2 * sizeof(unsigned long long),
                                    ctx->stream));
    int r = t_begin(ctx, KT_RAY);
    MORSE_CUDA(ctx, morse::launch_poly_map(b.s, b.q, b.L, b.npix, m->A,
                                           ctx->sm_count, ctx->stream));
    t_end(ctx, r);
    r = t_begin(ctx, KT_MAP);
    MORSE_CUDA(ctx, morse::launch_quads_from_A(m->A, b.npix, m->quad,
                                               m->qpitch, ctx->stream));
    if (b.fp16) {
      MORSE_TRY(enqueue_half(ctx, m));
      m->lookup = MORSE_STORE_FP16LOG;
    }
    t_end(ctx, r);
    ctx->launches += 2;
    return MORSE_OK;
  }
  m->has_counts = m->counts != nullptr;
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
  P.tiles_x = (int)((b.nray + morse::kRayTileX - 1) / morse::kRayTileX);
  // Tile height: the persistent blocks take tiles from a counter, and a
  // last round with few tiles leaves SMs idle, so pick the sub-block rows r
  // (tile height 16 r) that minimise rounds x (tile rays + a per-tile cost
  // of about 2000 rays: window placement, flush, barriers).
  const long long blocks =
      (long long)morse::rayshoot_blocks_per_sm() * ctx->sm_count;
  {
    double best = 0.0;
    P.sub_rows = morse::kRaySubRowsMax;
    for (int r = morse::kRaySubRowsMax; r >= morse::kRaySubRowsMax * 5 / 8;
         --r) {
      const long long th = (long long)morse::kRayWarps * r;
      const long long tiles =
          (long long)P.tiles_x * ((b.nray + th - 1) / th);
      const long long rounds = (tiles + blocks - 1) / blocks;
      const double cost =
          (double)rounds * ((double)morse::kRayTileX * th + 2000.0);
      if (best == 0.0 || cost < best * 0.995) {
        best = cost;
        P.sub_rows = r;
      }
    }
  }
  const long long th = (long long)morse::kRayWarps * P.sub_rows;
  P.tiles_y = (int)((b.nray + th - 1) / th);
  P.counts = m->counts;
  P.tot = m->tot;
  size_t n = (size_t)b.npix * b.npix;
  MORSE_CUDA(ctx, cudaMemsetAsync(m->counts, 0, n * sizeof(uint32_t),
                                  ctx->stream));
  MORSE_CUDA(ctx, cudaMemsetAsync(m->tot, 0, 3 * sizeof(unsigned long long),
                                  ctx->stream));
  long long tiles = (long long)P.tiles_x * P.tiles_y;
  int grid = (int)std::min<long long>(tiles, blocks);
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
  ctx->launches += 2;  // counts -> A, A -> cells
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

using morse::Tables;
using morse::tables_bytes;

// Grid tables at dev (16-byte aligned): the lines' tau intervals inside
// the map of half-width L (computed on the device), then u0, cos and sin
// alpha, t0 - t_ref, 1/(tE Delta), t0, tE.
morse_status upload_tables(morse_ctx *ctx, const morse_grid *g, double t_ref,
                           double L, double dlt, void *dev, Tables *T) {
  std::vector<double> h(morse::table_values(g));
  morse::table_host(g, t_ref, dlt, h.data());
  morse::tables_at(g, dev, T);
  // ordered on the context stream, then waited for: the host vector is
  // pageable and dies on return
  MORSE_CUDA(ctx, cudaMemcpyAsync(T->u0v, h.data(), h.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, ctx->stream));
  MORSE_CUDA(ctx, morse::launch_slab(T->u0v, T->ca, T->sa, g->n_u0,
                                     g->n_alpha, L, T->slab, ctx->stream));
  ctx->launches += 1;
  MORSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return MORSE_OK;
}

}  // namespace

namespace morse {

size_t table_values(const morse_grid *g) {
  return (size_t)(g->n_u0 + 2 * g->n_alpha + 2 * g->n_t0 + 2 * g->n_tE);
}

size_t tables_bytes(const morse_grid *g) {
  return sizeof(double2) * (size_t)g->n_u0 * g->n_alpha +
         sizeof(double) * table_values(g);
}

void table_host(const morse_grid *g, double t_ref, double dlt, double *h) {
  std::vector<double> u0, t0, tE;
  axis(g->u0_lo, g->u0_hi, g->n_u0, g->u0_log, u0);
  axis(g->t0_lo, g->t0_hi, g->n_t0, 0, t0);
  axis(g->tE_lo, g->tE_hi, g->n_tE, g->tE_log, tE);
  size_t k = 0;
  for (double v : u0) h[k++] = v;
  for (int i = 0; i < g->n_alpha; ++i)
    h[k++] = cos(2.0 * M_PI * (double)i / (double)g->n_alpha);
  for (int i = 0; i < g->n_alpha; ++i)
    h[k++] = sin(2.0 * M_PI * (double)i / (double)g->n_alpha);
  for (double v : t0) h[k++] = v - t_ref;
  for (double v : tE) h[k++] = 1.0 / (v * dlt);
  for (double v : t0) h[k++] = v;
  for (double v : tE) h[k++] = v;
}

void tables_at(const morse_grid *g, void *dev, Tables *T) {
  T->slab = (double2 *)dev;
  double *d = (double *)(T->slab + (size_t)g->n_u0 * g->n_alpha);
  T->u0v = d;
  T->ca = T->u0v + g->n_u0;
  T->sa = T->ca + g->n_alpha;
  T->t0rel = T->sa + g->n_alpha;
  T->invtEd = T->t0rel + g->n_t0;
  T->t0abs = T->invtEd + g->n_tE;
  T->tEv = T->t0abs + g->n_t0;
}

cudaError_t dev_alloc(morse_ctx *ctx, void **p, size_t bytes) {
  *p = nullptr;
  if (ctx && ctx->fault_alloc > 0 && --ctx->fault_alloc == 0)
    return cudaErrorMemoryAllocation;  // injected: nothing allocated
  return cudaMalloc(p, bytes);
}

void map_params(const morse_map *map, SearchParams *P) {
  const double dlt = (2.0 * map->L) / (double)map->npix;
  P->quad = map->quad;
  P->quadh = morse::map_h16(map) ? map->quadh : nullptr;
  P->qpitch = map->qpitch;
  P->qidx0 = morse::quad_idx0(map->npix);
  P->npix = map->npix;
  P->half = map->npix / 2;
  P->vlo = -(float)(map->npix / 2) - 0.5f;
  P->vhi = (float)(map->npix - map->npix / 2) - 0.5f;
  P->L = map->L;
  P->dlt = dlt;
  P->coff = 0.5 * map->npix - (double)(map->npix / 2) - 0.5;
  P->voff = (float)(-P->coff);
  P->dltf = (float)dlt;
  P->invDf = (float)(1.0 / dlt);
  P->invD = 1.0 / dlt;
  ctx_params(map->ctx, P);
}

void ctx_params(const morse_ctx *ctx, SearchParams *P) {
  P->spin_limit = ctx ? ctx->spin_limit : 0u;
  P->lock0 = ctx ? ctx->fault_lock_held : 0;
}

void event_params(const morse_event *ev, SearchParams *P) {
  P->ep = ev->ep;
  P->n_ep = (int)ev->n;
  P->S1 = ev->S1;
  P->SF = ev->SF;
  P->SFF = ev->SFF;
  P->Fref = ev->Fref;
  P->invS1 = ev->invS1;
  P->CFF = ev->CFF;
  const double m = (double)((ev->n + 31) / 32);
  P->gamma = (m + 10.0) * ldexp(1.0, -24);
}

void grid_params(const morse_grid *g, const Tables &T, SearchParams *P) {
  P->u0v = T.u0v;
  P->ca = T.ca;
  P->sa = T.sa;
  P->t0rel = T.t0rel;
  P->invtEd = T.invtEd;
  P->tEv = T.tEv;
  P->slab = T.slab;
  P->n_u0 = g->n_u0;
  P->n_alpha = g->n_alpha;
  P->n_t0 = g->n_t0;
  P->n_tE = g->n_tE;
  P->top_k = g->top_k;
}

}  // namespace morse

namespace {

using morse::ctx_params;
using morse::dev_alloc;
using morse::event_params;
using morse::grid_params;
using morse::map_params;

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
  size_t off_tab, off_lmax, off_hdr, off_pub, off_pa, off_pb, off_out, bytes;
  int tab_n;  // band-table entries (0: the search reads the global table)
};

// What the line-aligned pass needs to read its map cells from shared-memory
// band tables: the map size and a bound on the trajectories' pixel
// coordinates' terms, B = (max|t - t_ref| + max|t0 - t_ref|) / (min tE
// Delta) + (max|u| + max|shift|) / Delta.  FP32 rounding moves a position
// by at most 2^-24 (3 B), and the band keeps 1/4 texel to spare, so the
// tables are used only while B <= 1e5 (0.018 texel).
struct BandSpec {
  int npix = 0;  // 0: no band tables
  double L = 0.0, u_max = 0.0, shift_max = 0.0;
};

double grid_umax(const morse_grid *g) {
  return std::max(std::fabs(g->u0_lo), std::fabs(g->u0_hi));
}

BandSpec band_spec(int npix, double L, double u_max, double shift_max) {
  BandSpec b;
  b.npix = npix;
  b.L = L;
  b.u_max = u_max;
  b.shift_max = shift_max;
  return b;
}

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
  // the header and the published block quantiles (tag 0: none)
  MORSE_CUDA(ctx, cudaMemsetAsync(h, 0, pl.off_pa - pl.off_hdr, ctx->stream));
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
  if (h.err & 4u)
    return fail(ctx, MORSE_ECUDA,
                "bounds check: a band-table lookup read another cell than "
                "the map's (error 0x%x); results are invalid", h.err);

  if (h.err & 1u)
    return fail(ctx, MORSE_ETIMEOUT,
                "a search block could not take its top-K lock (error 0x%x); "
                "results are incomplete", h.err);
  return MORSE_OK;
}

morse_status plan_search(morse_ctx *ctx, const morse_event *ev,
                         const morse_grid *g, long long first,
                         long long count, bool dense, bool h16,
                         long long n_out, Plan *pl,
                         const BandSpec &band = BandSpec()) {
  const int K = dense ? 1 : g->top_k;
  const size_t fixed = morse::search_smem_bytes(0, dense ? 0 : K) -
                       (dense ? sizeof(Entry) * morse::kSearchWarps * 32 : 0);
  const size_t budget = ctx->smem_optin > 4096 ? ctx->smem_optin - 2048 : 0;
  const bool ep_smem =
      budget > fixed && (size_t)ev->n <= (budget - fixed) / sizeof(float4);
  size_t smem = fixed + (ep_smem ? sizeof(float4) * (size_t)ev->n : 0);
  // band tables: FP32 cells (decoded from the FP16 table when the search
  // reads that one), one line per block round (kSearchWarps groups per
  // line), two tables in the remaining shared memory, bounded motion
  pl->tab_n = 0;
  if (band.npix >= 2) {
    const long long line = (long long)g->n_t0 * g->n_tE;
    const int tpg = morse::line_tpg(line);
    const double dlt = 2.0 * band.L / band.npix;
    const double tE_min = std::min(g->tE_lo, g->tE_hi);
    const double t0_max = std::max(std::fabs(g->t0_lo - ev->t_ref),
                                   std::fabs(g->t0_hi - ev->t_ref));
    const double B = (ev->t_span + t0_max) / (tE_min * dlt) +
                     (band.u_max + band.shift_max) / dlt + 1.0;
    const int n = 4 * morse::band_stride(band.npix);
    const size_t tb = 2 * sizeof(float4) * (size_t)n;
    // a band costs one warp about the time of 4 (npix + 1) L2 reads (some
    // ten microseconds); a round must be long enough to hide it: at least
    // 4e5 trajectory-epochs per line (a group of config 1 is 1.5e5)
    const bool worth = (double)line * (double)ev->n >= 4e5;
    if ((line + tpg - 1) / tpg == morse::kSearchWarps && tE_min > 0.0 &&
        B <= 1e5 && smem + tb <= budget && worth) {
      pl->tab_n = n;
      smem += tb;
    }
  }
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
  pl->off_lmax = align_up(tables_bytes(g), 256);
  pl->off_hdr = align_up(
      pl->off_lmax + sizeof(double) * (size_t)g->n_u0 * g->n_alpha, 256);
  pl->off_pub = pl->off_hdr + 256;
  pl->off_pa = align_up(
      pl->off_pub + (dense ? 0
                           : sizeof(unsigned long long) * morse::kPubLevels *
                                 (size_t)grid),
      256);
  size_t list_bytes = dense ? 0 : sizeof(Entry) * (size_t)grid * K;
  pl->off_pb = align_up(pl->off_pa + list_bytes, 256);
  pl->off_out = align_up(pl->off_pb + list_bytes, 256);
  size_t out_bytes = dense ? sizeof(double) * 3 * (size_t)n_out
                           : sizeof(morse_fit) * (size_t)K * (size_t)n_out;
  pl->bytes = pl->off_out + out_bytes;
  return MORSE_OK;
}

// The minimum-magnification cut of a grid on a map: queue the line maxima
// into the plan's table and point the search at them (no-op for a_min 0).
morse_status enqueue_cut(morse_ctx *ctx, const morse_map *map,
                         const morse_grid *g, const Tables &T, const Plan &pl,
                         char *base, morse::SearchParams *P) {
  if (!(g->a_min > 0.0f)) {
    P->linemax = nullptr;
    P->a_min = 0.0;
    return MORSE_OK;
  }
  double *lm = (double *)(base + pl.off_lmax);
  MORSE_CUDA(ctx, morse::launch_line_max(map->A, map->npix, map->L, T.u0v,
                                         T.ca, T.sa, g->n_u0, g->n_alpha, lm,
                                         ctx->stream));
  ctx->launches += 1;
  P->linemax = lm;
  P->a_min = (double)g->a_min;
  return MORSE_OK;
}

#ifndef MORSE_PILOT_UB
#define MORSE_PILOT_UB 1  // the pilot keys its samples by chi2_upper
#endif

// A fresh tag for a search launch's published block quantiles (never 0,
// the value of a cleared word).
unsigned next_pub_tag(morse_ctx *ctx) {
  if (++ctx->pub_tag == 0) ctx->pub_tag = 1;
  return ctx->pub_tag;
}

// Queue the top-K search of one map: search kernel, merge tree, fit fill
// into fits_dev[0..K).  No host synchronisation.
morse_status enqueue_topk(morse_ctx *ctx, const Plan &pl,
                          morse::SearchParams P, char *base,
                          const Tables &T, morse_fit *fits_dev) {
  P.partial = (Entry *)(base + pl.off_pa);
  P.pub = (unsigned long long *)(base + pl.off_pub);
  P.tab_n = pl.tab_n;
  P.tab_c = (unsigned)(P.half + 1) - 0x4B400000u;
  int r;
  // pilot: a strided subset of ~sqrt(K N) trajectories (at least 16 K)
  // seeds the grid-wide pruning threshold
  const double want =
      std::max(morse::kPilotMinK * pl.K,
               morse::kPilotSqrt * std::sqrt((double)pl.K * P.count));
  // (no pilot when the sample would be under one trajectory)
  const long long stride = want >= 1.0 ? (long long)(P.count / want) : 0;
  if (P.gthr && stride >= 4) {
    morse::SearchParams Q = P;
    Q.stride = stride;
    Q.count = (P.count + stride - 1) / stride;
    Q.tpg = morse::kTpgPilot;
    long long groups = (Q.count + Q.tpg - 1) / Q.tpg;
    int grid = (int)std::min<long long>(
        pl.grid, (groups + morse::kSearchWarps - 1) / morse::kSearchWarps);
    if (grid < 1) grid = 1;
    Q.pilot_ub = MORSE_PILOT_UB;
    Q.pub_tag = next_pub_tag(ctx);
    Q.pub_nb = grid;
    Q.pub_me = -1;
    Q.pub_stride = grid;
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
                                             ctx->stream, P.gthr));
    t_end(ctx, r);
    ctx->launches += 1 + (uint64_t)levels;
  }
  P.pub_tag = next_pub_tag(ctx);
  P.pub_nb = pl.grid;
  P.pub_me = -1;
  P.pub_stride = pl.grid;
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
#ifndef MORSE_SWEEP_OVERLAP
#define MORSE_SWEEP_OVERLAP 1
#endif
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
  // Two map buffers: map i + 1 is built on a second stream while map i is
  // searched, so the ray shooting fills the SMs that the merges, the fill
  // and the search's last blocks leave idle.  The results do not depend on
  // the overlap (each search waits for its map; each build for the search
  // that last read its buffer).
  const bool two = MORSE_SWEEP_OVERLAP && n_maps > 1;
  morse_map **bufs[2] = {&ctx->sweep_map, &ctx->sweep_map2};
  for (int b = 0; b < (two ? 2 : 1); ++b) {
    morse_map *&mb = *bufs[b];
    if (mb && mb->npix != npix) {
      cudaStreamSynchronize(ctx->stream);
      map_release(mb);
      mb = nullptr;
    }
    if (!mb) {
      mb = map_alloc(ctx, npix, true);
      if (!mb)
        return fail(ctx, MORSE_ENOMEM, "sweep map of %d^2 texels", npix);
    }
    mb->L = extent;
  }
  const bool h16 = n_maps > 0 && specs[0].fp16;
  for (int b = 0; b < (two ? 2 : 1); ++b)
    if (h16 && !map_ensure_half(*bufs[b]))
      return fail(ctx, MORSE_ENOMEM, "FP16 table of %d^2 texels", npix);
  if (two && !ctx->build_stream) {
    MORSE_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->build_stream,
                                              cudaStreamNonBlocking));
    for (int k = 0; k < 4; ++k)
      MORSE_CUDA(ctx, cudaEventCreateWithFlags(&ctx->sweep_ev[k],
                                               cudaEventDisableTiming));
  }
  morse_map *m = ctx->sweep_map;
  Plan pl;
  MORSE_TRY(plan_search(ctx, ev, grid, 0, grid_size(grid), false, h16, n_maps,
                        &pl, band_spec(npix, extent, grid_umax(grid), 0.0)));
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, pl.bytes, &ws));
  char *base = (char *)ws;
  Tables T;
  const double dlt = (2.0 * extent) / (double)npix;
  MORSE_TRY(upload_tables(ctx, grid, ev->t_ref, extent,
                          dlt, base + pl.off_tab, &T));
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
  cudaStream_t s0 = ctx->stream;
  cudaEvent_t *built = ctx->sweep_ev, *freed = ctx->sweep_ev + 2;
  if (two) {  // the builds follow everything queued so far
    MORSE_CUDA(ctx, cudaEventRecord(built[0], s0));
    MORSE_CUDA(ctx, cudaStreamWaitEvent(ctx->build_stream, built[0], 0));
  }
  for (int i = 0; i < n_maps; ++i) {
    const int b = two ? (i & 1) : 0;
    m = *bufs[b];
    if (two) {
      if (i >= 2)  // the search of map i - 2 has read this buffer
        MORSE_CUDA(ctx, cudaStreamWaitEvent(ctx->build_stream, freed[b], 0));
      ctx->stream = ctx->build_stream;
      const morse_status bs = enqueue_build(ctx, m, specs[(size_t)i]);
      ctx->stream = s0;
      MORSE_TRY(bs);
      MORSE_CUDA(ctx, cudaEventRecord(built[b], ctx->build_stream));
      MORSE_CUDA(ctx, cudaStreamWaitEvent(s0, built[b], 0));
    } else {
      MORSE_TRY(enqueue_build(ctx, m, specs[(size_t)i]));
    }
    P.quad = m->quad;
    P.quadh = h16 ? m->quadh : nullptr;
    if (i > 0) MORSE_TRY(hdr_reset_threshold(ctx, base, pl));
    MORSE_TRY(enqueue_cut(ctx, m, grid, T, pl, base, &P));
    MORSE_TRY(enqueue_topk(ctx, pl, P, base, T, fits + (size_t)i * pl.K));
    if (two) MORSE_CUDA(ctx, cudaEventRecord(freed[b], s0));
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

// ---------------------------------------------------------------- batch
// Epoch-count bucket: floor(log2 n_ep).
int ep_bucket(int64_t n) {
  int b = 0;
  while ((int64_t(2) << b) <= n) ++b;
  return b;
}

std::string tune_key(int bucket, const morse_grid *g, const morse_map *m) {
  char buf[128];
  snprintf(buf, sizeof(buf), "%d|%d|%lld|%lld|%d|%d", bucket, g->top_k,
           (long long)g->n_t0 * g->n_tE, grid_size(g), m->npix,
           morse::map_h16(m) ? 1 : 0);
  return std::string(buf);
}

// Staging is decided per bucket, so that one shape holds for every light
// curve of the bucket: buckets of fewer than 4096 epochs (64 KB) may be
// staged.  Staging larger ones looks faster when a bucket is timed alone,
// but the batch's one launch then reserves that shared memory on every
// SM, and the long light curves, which stream their epochs through L1 and
// carry most of the evaluations, lose the L1 (tuned with up to 8191
// staged: 9.1e11 evaluations/s against 9.75e11).
constexpr int kBatchStageDefault = 4095;
constexpr int kBatchStageMax = 4095;

int64_t bucket_top(int64_t n_ep) {
  return (int64_t(2) << ep_bucket(n_ep)) - 1;
}

morse_batch_shape default_shape(int64_t n_ep, long long line) {
  morse_batch_shape s;
  s.tpg = morse::line_tpg(line);
  s.rounds = 4;
  s.stage = bucket_top(n_ep) <= kBatchStageDefault ? 1 : 0;
  s.tuned = 0;
  s.ns_per_eval = 0.0;
  return s;
}

// Host copy of everything a batch launch reads besides the epochs and maps.
struct BatchHost {
  std::vector<morse::BatchEvent> ev;
  std::vector<const void *> tab;
  std::vector<morse::BatchUnit> pilot, main;
  std::vector<int> pilot_list0, main_list0;
  std::vector<double> tables;  // u0 | cos | sin | 1/(tE D) | t0 | tE | t0rel
  long long pilot_count = 0, pilot_stride = 0;
  int ep_cap = 0;
  int main_global = 0;  // the main pass's units of unstaged light curves,
                        // first in `main` (a launch of their own)
};

// Units of one pass over `pairs` pairs: groups [0, groups(p)) of each pair
// cut into units of kSearchWarps * rounds groups.
void batch_units(const std::vector<int> &pair_ids,
                 const std::vector<morse_batch_shape> &shape_of_pair,
                 const std::vector<long long> &groups_of_pair, int pairs,
                 std::vector<morse::BatchUnit> &units,
                 std::vector<int> &list0) {
  list0.assign((size_t)pairs + 1, 0);
  std::vector<long long> per(pairs, 0);
  for (int p : pair_ids) {
    const long long ug = (long long)morse::kSearchWarps *
                         shape_of_pair[(size_t)p].rounds;
    per[(size_t)p] = (groups_of_pair[(size_t)p] + ug - 1) / ug;
  }
  for (int p = 0; p < pairs; ++p)
    list0[(size_t)p + 1] = list0[(size_t)p] + (int)per[(size_t)p];
  units.clear();
  for (int p : pair_ids) {
    const morse_batch_shape &s = shape_of_pair[(size_t)p];
    const long long ug = (long long)morse::kSearchWarps * s.rounds;
    for (long long u = 0; u < per[(size_t)p]; ++u) {
      morse::BatchUnit U;
      U.pair = p;
      U.list = list0[(size_t)p] + (int)u;
      U.g0 = (int)(u * ug);
      U.ng = (int)std::min(ug, groups_of_pair[(size_t)p] - u * ug);
      U.tpg = s.tpg;
      U.stage = s.stage;
      units.push_back(U);
    }
  }
}

// Grid tables shared by the pairs, plus each event's t0 - t_ref (after
// the slab table, which the device fills).
void batch_tables(const morse_grid *g, const morse_event *const *evs, int n_ev,
                  double dlt, std::vector<double> &h) {
  std::vector<double> u0, t0, tE;
  axis(g->u0_lo, g->u0_hi, g->n_u0, g->u0_log, u0);
  axis(g->t0_lo, g->t0_hi, g->n_t0, 0, t0);
  axis(g->tE_lo, g->tE_hi, g->n_tE, g->tE_log, tE);
  h.assign((size_t)2 * g->n_u0 * g->n_alpha, 0.0);  // slab (device)
  h.insert(h.end(), u0.begin(), u0.end());
  for (int k = 0; k < g->n_alpha; ++k)
    h.push_back(cos(2.0 * M_PI * (double)k / (double)g->n_alpha));
  for (int k = 0; k < g->n_alpha; ++k)
    h.push_back(sin(2.0 * M_PI * (double)k / (double)g->n_alpha));
  for (double v : tE) h.push_back(1.0 / (v * dlt));
  h.insert(h.end(), t0.begin(), t0.end());
  h.insert(h.end(), tE.begin(), tE.end());
  for (int e = 0; e < n_ev; ++e)
    for (double v : t0) h.push_back(v - evs[e]->t_ref);
}

// Device layout of a batch call.
struct BatchLayout {
  size_t off_tab, off_ev, off_ptr, off_up, off_um, off_lp, off_lm, off_gthr,
      off_hdr, off_pub, off_pa, off_pb, off_res, off_fit, bytes;
  size_t lists;  // top-K lists of the larger pass
};

struct BatchHdr {
  unsigned counter[3];  // pilot, main (unstaged units), main (staged)
  unsigned err;
  unsigned long long stat_exact;
};

BatchLayout batch_layout(const BatchHost &H, int pairs, int K) {
  BatchLayout L;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  L.off_tab = take(sizeof(double) * H.tables.size());
  L.off_ev = take(sizeof(morse::BatchEvent) * H.ev.size());
  L.off_ptr = take(sizeof(void *) * H.tab.size());
  L.off_up = take(sizeof(morse::BatchUnit) * H.pilot.size());
  L.off_um = take(sizeof(morse::BatchUnit) * H.main.size());
  L.off_lp = take(sizeof(int) * H.pilot_list0.size());
  L.off_lm = take(sizeof(int) * H.main_list0.size());
  L.off_gthr = take(sizeof(unsigned long long) * (size_t)pairs);
  L.off_hdr = take(sizeof(BatchHdr));
  const size_t lists = (size_t)std::max(
      H.pilot_list0.empty() ? 0 : H.pilot_list0.back(), H.main_list0.back());
  L.lists = lists;
  L.off_pub = take(sizeof(unsigned long long) * morse::kPubLevels * lists);
  L.off_pa = take(sizeof(Entry) * lists * (size_t)K);
  L.off_pb = take(sizeof(Entry) * lists * (size_t)K);
  L.off_res = take(sizeof(Entry) * (size_t)pairs * K);
  L.off_fit = take(sizeof(morse_fit) * (size_t)pairs * K);
  L.bytes = o;
  return L;
}

// Fill the per-pair arrays of a batch over the given events and maps.
// shape_of_event: the launch shape of each event.
morse_status batch_prepare(morse_ctx *ctx, const morse_event *const *evs,
                           int n_ev, const morse_map *const *maps, int n_maps,
                           const morse_grid *g,
                           const std::vector<morse_batch_shape> &shape_ev,
                           bool with_pilot, BatchHost &H) {
  const int K = g->top_k;
  const long long N = grid_size(g);
  const long long line = (long long)g->n_t0 * g->n_tE;
  const int pairs = n_ev * n_maps;
  const double dlt = (2.0 * maps[0]->L) / (double)maps[0]->npix;
  batch_tables(g, evs, n_ev, dlt, H.tables);
  H.tab.resize((size_t)n_maps);
  const bool h16 = morse::map_h16(maps[0]);
  for (int m = 0; m < n_maps; ++m)
    H.tab[(size_t)m] = h16 ? (const void *)maps[m]->quadh
                           : (const void *)maps[m]->quad;
  H.ev.resize((size_t)n_ev);
  H.ep_cap = 0;
  // staged light curves must fit next to the block's top-K lists
  const size_t lists = morse::batch_smem_bytes(0, K);
  const long long cap_max =
      ctx->smem_optin > lists + 2048
          ? (long long)((ctx->smem_optin - lists - 2048) / sizeof(float4))
          : 0;
  for (int e = 0; e < n_ev; ++e) {
    morse::BatchEvent &E = H.ev[(size_t)e];
    E.ep = evs[e]->ep;
    E.n_ep = (int)evs[e]->n;
    E.S1 = evs[e]->S1;
    E.SF = evs[e]->SF;
    E.SFF = evs[e]->SFF;
    E.Fref = evs[e]->Fref;
    E.invS1 = evs[e]->invS1;
    E.CFF = evs[e]->CFF;
    E.gamma = ((double)((evs[e]->n + 31) / 32) + 10.0) * ldexp(1.0, -24);
    E.t0rel = nullptr;  // set once the table offset is known
  }
  std::vector<morse_batch_shape> shape_fit = shape_ev;
  for (int e = 0; e < n_ev; ++e) {
    morse_batch_shape &s = shape_fit[(size_t)e];
    if (s.stage && evs[e]->n > cap_max) s.stage = 0;
    if (s.stage) H.ep_cap = std::max(H.ep_cap, (int)evs[e]->n);
  }
  // pairs map by map (one map at a time streams from HBM into L2), within
  // a map longest light curve first (they start early; short ones fill
  // the tail)
  std::vector<int> order((size_t)pairs);
  for (int p = 0; p < pairs; ++p) order[(size_t)p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const int ma = a % n_maps, mb = b % n_maps;
    if (ma != mb) return ma < mb;
    return evs[a / n_maps]->n > evs[b / n_maps]->n;
  });
  std::vector<morse_batch_shape> shape_pair((size_t)pairs);
  for (int p = 0; p < pairs; ++p)
    shape_pair[(size_t)p] = shape_fit[(size_t)(p / n_maps)];
  // pilot: a strided sample of ~sqrt(K N) trajectories per pair
  const double want = std::max(morse::kBatchPilotMinK * K,
                               morse::kBatchPilotSqrt * std::sqrt((double)K * N));
  const long long stride = want >= 1.0 ? (long long)(N / want) : 0;
  H.pilot.clear();
  H.pilot_list0.clear();
  H.pilot_count = 0;
  H.pilot_stride = 0;
  if (with_pilot && stride >= 4) {
    H.pilot_stride = stride;
    H.pilot_count = (N + stride - 1) / stride;
    std::vector<morse_batch_shape> sp = shape_pair;
    std::vector<long long> gp((size_t)pairs);
    for (int p = 0; p < pairs; ++p) {
      sp[(size_t)p].tpg = 16;
      sp[(size_t)p].rounds = 2;
      gp[(size_t)p] = (H.pilot_count + 15) / 16;
    }
    batch_units(order, sp, gp, pairs, H.pilot, H.pilot_list0);
  }
  std::vector<long long> gm((size_t)pairs);
  for (int p = 0; p < pairs; ++p) {
    const int t = shape_pair[(size_t)p].tpg;
    gm[(size_t)p] = (N / line) * ((line + t - 1) / t);
  }
  batch_units(order, shape_pair, gm, pairs, H.main, H.main_list0);
  if ((long long)H.main_list0.back() >= 0x7fffffffLL / std::max(K, 1))
    return fail(ctx, MORSE_EINVAL, "batch needs too many partial lists");
  // units of light curves that are not staged run first, in a launch with
  // no staging space (the shared memory it leaves serves as L1 for their
  // epochs); each part keeps the map-major order
  std::stable_partition(H.main.begin(), H.main.end(),
                        [&](const morse::BatchUnit &u) {
                          return !(u.stage && H.ev[(size_t)(u.pair / n_maps)]
                                                      .n_ep <= H.ep_cap);
                        });
  H.main_global = 0;
  for (const morse::BatchUnit &u : H.main)
    if (!(u.stage && H.ev[(size_t)(u.pair / n_maps)].n_ep <= H.ep_cap))
      ++H.main_global;
  return MORSE_OK;
}

// Upload a prepared batch; returns the kernel parameters of its passes.
morse_status batch_upload(morse_ctx *ctx, BatchHost &H, const BatchLayout &L,
                          char *base, const morse_grid *g,
                          const morse_map *map0, int n_ev,
                          morse::BatchParams *Bp, morse::BatchParams *Bm,
                          double **t0abs, double **tEv) {
  double *tab = (double *)(base + L.off_tab);
  const size_t o_u0 = (size_t)2 * g->n_u0 * g->n_alpha,
               o_ca = o_u0 + g->n_u0, o_sa = o_ca + g->n_alpha,
               o_k = o_sa + g->n_alpha, o_t0 = o_k + g->n_tE,
               o_tE = o_t0 + g->n_t0, o_rel = o_tE + g->n_tE;
  for (int e = 0; e < n_ev; ++e)
    H.ev[(size_t)e].t0rel = tab + o_rel + (size_t)e * g->n_t0;
  // one staging buffer, one copy, one wait (the host vectors are pageable)
  std::vector<char> h(L.off_gthr);
  memcpy(h.data() + L.off_tab, H.tables.data(),
         sizeof(double) * H.tables.size());
  memcpy(h.data() + L.off_ev, H.ev.data(),
         sizeof(morse::BatchEvent) * H.ev.size());
  memcpy(h.data() + L.off_ptr, H.tab.data(), sizeof(void *) * H.tab.size());
  if (!H.pilot.empty()) {
    memcpy(h.data() + L.off_up, H.pilot.data(),
           sizeof(morse::BatchUnit) * H.pilot.size());
    memcpy(h.data() + L.off_lp, H.pilot_list0.data(),
           sizeof(int) * H.pilot_list0.size());
  }
  memcpy(h.data() + L.off_um, H.main.data(),
         sizeof(morse::BatchUnit) * H.main.size());
  memcpy(h.data() + L.off_lm, H.main_list0.data(),
         sizeof(int) * H.main_list0.size());
  MORSE_CUDA(ctx, cudaMemcpyAsync(base, h.data(), h.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
  MORSE_CUDA(ctx, morse::launch_slab(tab + o_u0, tab + o_ca, tab + o_sa,
                                     g->n_u0, g->n_alpha, map0->L,
                                     (double2 *)tab, ctx->stream));
  ctx->launches += 1;
  MORSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  BatchHdr *hd = (BatchHdr *)(base + L.off_hdr);
  morse::BatchParams B;
  memset(&B, 0, sizeof(B));
  map_params(map0, &B.S);
  B.S.quad = nullptr;  // per pair, from B.tab
  B.S.quadh = nullptr;
  B.S.u0v = tab + o_u0;
  B.S.ca = tab + o_ca;
  B.S.sa = tab + o_sa;
  B.S.invtEd = tab + o_k;
  B.S.tEv = tab + o_tE;
  B.S.slab = (const double2 *)tab;
  B.S.n_u0 = g->n_u0;
  B.S.n_alpha = g->n_alpha;
  B.S.n_t0 = g->n_t0;
  B.S.n_tE = g->n_tE;
  B.S.top_k = g->top_k;
  B.S.err = &hd->err;
  B.S.stat_exact = &hd->stat_exact;
  B.S.first = 0;
  B.ev = (const morse::BatchEvent *)(base + L.off_ev);
  B.tab = (const void *const *)(base + L.off_ptr);
  B.n_maps = (int)H.tab.size();
  B.gthr = (unsigned long long *)(base + L.off_gthr);
  B.partial = (Entry *)(base + L.off_pa);
  B.ep_cap = H.ep_cap;
  // published list quantiles: rows of the larger pass's list count, cleared
  // by every call (a graph replay reuses the tags); tags 1 and 2
  B.S.pub = MORSE_BATCH_PUB ? (unsigned long long *)(base + L.off_pub)
                            : nullptr;
  B.S.pub_stride = (int)L.lists;
  B.n_lists = (int)L.lists;
  *Bp = B;
  Bp->S.pub_tag = 1;
  Bp->S.pilot_ub = MORSE_PILOT_UB;  // the pilot keys samples by chi2_upper
  Bp->list0 = (const int *)(base + L.off_lp);
  Bp->S.count = H.pilot_count;
  Bp->S.stride = H.pilot_stride;
  Bp->S.line = 0;
  Bp->units = (const morse::BatchUnit *)(base + L.off_up);
  Bp->n_units = (int)H.pilot.size();
  Bp->counter = &hd->counter[0];
  *Bm = B;
  Bm->S.pub_tag = 2;
  Bm->list0 = (const int *)(base + L.off_lm);
  Bm->S.count = grid_size(g);
  Bm->S.stride = 1;
  Bm->S.line = (long long)g->n_t0 * g->n_tE;
  Bm->units = (const morse::BatchUnit *)(base + L.off_um);
  Bm->n_units = (int)H.main.size();
  Bm->counter = &hd->counter[1];
  *t0abs = tab + o_t0;
  *tEv = tab + o_tE;
  return MORSE_OK;
}

// Queue a batch: reset words, pilot pass and seeding, main pass, merges,
// fill.  No host synchronisation.
morse_status batch_enqueue(morse_ctx *ctx, const BatchLayout &L, char *base,
                           const morse::BatchParams &Bp,
                           const morse::BatchParams &Bm, bool h16, int pairs,
                           const double *t0abs, const double *tEv,
                           int grid, size_t smem, int main_global,
                           int grid_g, size_t smem_g) {
  const int K = Bm.S.top_k;
  MORSE_CUDA(ctx, cudaMemsetAsync(base + L.off_gthr, 0xFF,
                                  sizeof(unsigned long long) * pairs,
                                  ctx->stream));
  MORSE_CUDA(ctx, cudaMemsetAsync(base + L.off_hdr, 0, sizeof(BatchHdr),
                                  ctx->stream));
  MORSE_CUDA(ctx, cudaMemsetAsync(
                      base + L.off_pub, 0,
                      sizeof(unsigned long long) * morse::kPubLevels * L.lists,
                      ctx->stream));
  Entry *pa = (Entry *)(base + L.off_pa), *pb = (Entry *)(base + L.off_pb);
  Entry *res = (Entry *)(base + L.off_res);
  int r;
  if (Bp.n_units > 0) {
    r = t_begin(ctx, KT_SEARCH);
    MORSE_CUDA(ctx, morse::launch_batch(
                        Bp, h16, std::min(grid, Bp.n_units), smem,
                        ctx->stream));
    t_end(ctx, r);
    r = t_begin(ctx, KT_MERGE);
    MORSE_CUDA(ctx, morse::launch_batch_merge(
                        pa, pb, (const int *)(base + L.off_lp), pairs, K, res,
                        Bm.gthr, ctx->stream));
    t_end(ctx, r);
    ctx->launches += 2;
  }
  // main pass: the unstaged light curves' units in a launch without
  // staging space, then the staged ones
  morse::BatchParams Bg = Bm, Bs = Bm;
  Bg.n_units = main_global;
  Bg.ep_cap = 0;
  Bs.units = Bm.units + main_global;
  Bs.n_units = Bm.n_units - main_global;
  Bs.counter = &((BatchHdr *)(base + L.off_hdr))->counter[2];
  r = t_begin(ctx, KT_SEARCH);
  if (Bg.n_units > 0) {
    MORSE_CUDA(ctx, morse::launch_batch(Bg, h16, std::min(grid_g, Bg.n_units),
                                        smem_g, ctx->stream, 1));
    ctx->launches += 1;
  }
  if (Bs.n_units > 0) {
    MORSE_CUDA(ctx, morse::launch_batch(Bs, h16, std::min(grid, Bs.n_units),
                                        smem, ctx->stream));
    ctx->launches += 1;
  }
  t_end(ctx, r);
  r = t_begin(ctx, KT_MERGE);
  MORSE_CUDA(ctx, morse::launch_batch_merge(pa, pb,
                                            (const int *)(base + L.off_lm),
                                            pairs, K, res, nullptr,
                                            ctx->stream));
  t_end(ctx, r);
  ctx->launches += 1;
  r = t_begin(ctx, KT_FILL);
  MORSE_CUDA(ctx, morse::launch_batch_fill(Bm, h16, res, pairs, t0abs, tEv,
                                           (morse_fit *)(base + L.off_fit),
                                           ctx->stream));
  t_end(ctx, r);
  ctx->launches += 1;
  return MORSE_OK;
}

morse_status batch_hdr_check(morse_ctx *ctx, const BatchHdr &h) {
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

// Autotune the launch shape of one bucket on event e (a representative of
// the bucket) against map 0: after one pilot pass (untimed, shared by the
// candidates) the main pass runs on a sample of units of that pair for each
// candidate shape; the fastest per trajectory-epoch wins.
morse_status batch_tune(morse_ctx *ctx, const morse_event *ev,
                        const morse_map *map0, const morse_grid *g,
                        morse_batch_shape *best) {
  const long long line = (long long)g->n_t0 * g->n_tE;
  *best = default_shape(ev->n, line);
  // the default rule's shape is a candidate too, and another shape must
  // beat it by 5 % (the samples are short and their timing noisy)
  std::vector<morse_batch_shape> cands(1, *best);
  cands[0].tuned = 1;
  for (int tpg : {8, 16, 32})
    for (int stage : {1, 0})
      for (int rounds : {2, 8}) {
        if (stage && bucket_top(ev->n) > kBatchStageMax) continue;
        morse_batch_shape s;
        s.tpg = tpg;
        s.stage = stage;
        s.rounds = rounds;
        s.tuned = 1;
        s.ns_per_eval = 0.0;
        cands.push_back(s);
      }
  const bool h16 = morse::map_h16(map0);
  const morse_event *evs[1] = {ev};
  const morse_map *maps[1] = {map0};
  // a sample of about 2e8 trajectory-epochs (a few hundred microseconds,
  // long enough to time), the whole pair if it has fewer; each candidate
  // timed three times, the fastest run counting
  const long long kTuneTrajs =
      std::max(300000LL, (long long)(2e8 / (double)std::max<int64_t>(
                                              ev->n, 1)));
  double best_ns = 0.0;
  cudaEvent_t e0, e1;
  MORSE_CUDA(ctx, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ctx, ce, "tuner event");
  }
  morse_status st = MORSE_OK;
  for (size_t c = 0; c < cands.size() && st == MORSE_OK; ++c) {
    std::vector<morse_batch_shape> sh(1, cands[c]);
    BatchHost H;
    st = batch_prepare(ctx, evs, 1, maps, 1, g, sh, true, H);
    if (st != MORSE_OK) break;
    // time an evenly spaced sample of the pair's units, about
    // kTuneTrajs trajectories
    const long long tpg = cands[c].tpg, ngl = (line + tpg - 1) / tpg;
    auto unit_trajs = [&](const morse::BatchUnit &U) {
      long long n = 0;
      for (long long gi = U.g0; gi < (long long)U.g0 + U.ng; ++gi) {
        const long long j = gi % ngl;
        n += std::min((j + 1) * tpg, line) - j * tpg;
      }
      return n;
    };
    const long long per_unit = std::max(1LL, unit_trajs(H.main[0]));
    const long long want_units = std::max(1LL, kTuneTrajs / per_unit);
    const size_t step = std::max<size_t>(
        1, H.main.size() / (size_t)want_units);
    std::vector<morse::BatchUnit> pick;
    long long trajs = 0;
    for (size_t i = 0; i < H.main.size(); i += step) {
      pick.push_back(H.main[i]);
      trajs += unit_trajs(H.main[i]);
    }
    H.main.swap(pick);
    BatchLayout L = batch_layout(H, 1, g->top_k);
    void *ws = nullptr;
    st = ws_reserve(ctx, L.bytes, &ws);
    if (st != MORSE_OK) break;
    char *base = (char *)ws;
    morse::BatchParams Bp, Bm;
    double *t0abs, *tEv;
    st = batch_upload(ctx, H, L, base, g, map0, 1, &Bp, &Bm, &t0abs, &tEv);
    if (st != MORSE_OK) break;
    // the pilot pass and its merge, then the timed main pass
    const size_t smem = morse::batch_smem_bytes(H.ep_cap, g->top_k);
    const int bps = morse::batch_blocks_per_sm(h16, smem);
    if (bps < 1) continue;
    const int grid = bps * ctx->sm_count;
    cands[c].stage = H.ep_cap > 0 ? 1 : 0;  // as the preparation fitted it
    Entry *pa = (Entry *)(base + L.off_pa), *pb = (Entry *)(base + L.off_pb);
    float ms = 0.f;
    ce = cudaSuccess;
    for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep) {
      // every run starts from the pilot's threshold (the main pass lowers
      // it), so the candidates are timed on the same pruning
      cudaMemsetAsync(base + L.off_gthr, 0xFF, sizeof(unsigned long long),
                      ctx->stream);
      cudaMemsetAsync(base + L.off_hdr, 0, sizeof(BatchHdr), ctx->stream);
      cudaMemsetAsync(base + L.off_pub, 0,
                      sizeof(unsigned long long) * morse::kPubLevels * L.lists,
                      ctx->stream);
      if (Bp.n_units > 0) {
        morse::launch_batch(Bp, h16, std::min(grid, Bp.n_units), smem,
                            ctx->stream);
        morse::launch_batch_merge(pa, pb, (const int *)(base + L.off_lp), 1,
                                  g->top_k, (Entry *)(base + L.off_res),
                                  Bm.gthr, ctx->stream);
        ctx->launches += 2;
      }
      cudaEventRecord(e0, ctx->stream);
      morse::launch_batch(Bm, h16, std::min(grid, Bm.n_units), smem,
                          ctx->stream);
      cudaEventRecord(e1, ctx->stream);
      ctx->launches += 1;
      ce = cudaStreamSynchronize(ctx->stream);
      float r = 0.f;
      if (ce == cudaSuccess) cudaEventElapsedTime(&r, e0, e1);
      if (rep == 0 || r < ms) ms = r;
    }
    if (ce != cudaSuccess) {
      st = cuda_fail(ctx, ce, "tuning run");
      break;
    }
    BatchHdr hh;
    ce = cudaMemcpy(&hh, base + L.off_hdr, sizeof(hh), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) {
      st = cuda_fail(ctx, ce, "tuning run");
      break;
    }
    st = batch_hdr_check(ctx, hh);
    if (st != MORSE_OK) break;
    const double ns = 1e6 * (double)ms / ((double)trajs * (double)ev->n) *
                      (c == 0 ? 0.95 : 1.0);
    if (best_ns == 0.0 || ns < best_ns) {
      best_ns = ns;
      *best = cands[c];
      best->ns_per_eval = ns;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
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
  if (morse::adjoint_setup() != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MORSE_ECUDA;
  }
  c->tune_mode = MORSE_TUNE_ON;
  c->spin_limit = kDefaultSpinLimit;
  c->fault_lock_held = 0;
  c->fault_alloc = 0;
  c->batch_exec = nullptr;
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
  if (ctx->build_stream) {
    cudaStreamSynchronize(ctx->build_stream);
    cudaStreamDestroy(ctx->build_stream);
    for (cudaEvent_t e : ctx->sweep_ev) cudaEventDestroy(e);
  }
  if (ctx->sweep_map) map_release(ctx->sweep_map);
  if (ctx->sweep_map2) map_release(ctx->sweep_map2);
  if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
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

morse_status morse_inject_fault(morse_ctx *ctx, int fault, int64_t arg) {
  if (!ctx) return MORSE_EINVAL;
  switch (fault) {
    case MORSE_FAULT_NONE:
      ctx->spin_limit = kDefaultSpinLimit;
      ctx->fault_lock_held = 0;
      ctx->fault_alloc = 0;
      return MORSE_OK;
    case MORSE_FAULT_LOCK_HELD:
      if (arg < 1 || arg > (int64_t)kDefaultSpinLimit)
        return fail(ctx, MORSE_EINVAL, "spin limit %lld outside 1..%u",
                    (long long)arg, kDefaultSpinLimit);
      ctx->spin_limit = (unsigned)arg;
      ctx->fault_lock_held = 1;
      return MORSE_OK;
    case MORSE_FAULT_ALLOC:
      if (arg < 1)
        return fail(ctx, MORSE_EINVAL, "allocation index %lld < 1",
                    (long long)arg);
      ctx->fault_alloc = arg;
      return MORSE_OK;
    default:
      return fail(ctx, MORSE_EINVAL, "unknown fault %d", fault);
  }
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

morse_status morse_line_max(morse_ctx *ctx, const morse_map *map,
                            const morse_grid *grid, double *out) {
  if (!ctx || !map || !out) return MORSE_EINVAL;
  if (map->ctx != ctx) return fail(ctx, MORSE_EINVAL, "map of another ctx");
  MORSE_TRY(check_grid(ctx, grid));
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  const size_t n = (size_t)grid->n_u0 * grid->n_alpha;
  const size_t off = align_up(tables_bytes(grid), 256);
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, off + sizeof(double) * n, &ws));
  Tables T;
  const double dlt = (2.0 * map->L) / (double)map->npix;
  MORSE_TRY(upload_tables(ctx, grid, 0.0, map->L, dlt, ws, &T));
  double *lm = (double *)((char *)ws + off);
  MORSE_CUDA(ctx, morse::launch_line_max(map->A, map->npix, map->L, T.u0v,
                                         T.ca, T.sa, grid->n_u0,
                                         grid->n_alpha, lm, ctx->stream));
  ctx->launches += 1;
  MORSE_CUDA(ctx, cudaMemcpyAsync(out, lm, sizeof(double) * n,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  return sync_and_collect(ctx, "line maxima");
}

morse_status morse_map_finite_source(morse_ctx *ctx, const morse_map *src,
                                     double rho, double gamma,
                                     morse_map **out) {
  if (!ctx || !src || !out) return MORSE_EINVAL;
  *out = nullptr;
  if (src->ctx != ctx) return fail(ctx, MORSE_EINVAL, "map of another ctx");
  if (!(rho > 0.0) || !is_fin(rho))
    return fail(ctx, MORSE_EINVAL, "rho must be finite and > 0");
  if (!(gamma >= 0.0 && gamma <= 1.0))
    return fail(ctx, MORSE_EINVAL, "gamma must be in [0, 1]");
  const int npix = src->npix;
  const double dlt = (2.0 * src->L) / (double)npix;
  const double rpx = rho / dlt;
  if (!(rpx + 0.5 <= 1600.0))
    return fail(ctx, MORSE_EINVAL,
                "source radius of %.1f texels exceeds the 1600 supported",
                rpx);
  const int R = (int)ceil(rpx + 0.5);
  const int side = 2 * R + 1;
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  // the profile integrated over each texel on 8 x 8 midpoint points, on the
  // device; normalised and rounded to FP32 here
  std::vector<double> w((size_t)side * side, 0.0);
  {
    void *ws0 = nullptr;
    MORSE_TRY(ws_reserve(ctx, sizeof(double) * w.size(), &ws0));
    MORSE_CUDA(ctx, morse::launch_fs_weights(rpx, gamma, R, (double *)ws0,
                                             ctx->stream));
    ctx->launches += 1;
    MORSE_CUDA(ctx, cudaMemcpyAsync(w.data(), ws0, sizeof(double) * w.size(),
                                    cudaMemcpyDeviceToHost, ctx->stream));
    MORSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  double tot = 0.0;
  for (double v : w) tot += v;
  if (!(tot > 0.0)) {  // sub-texel source: the centre texel alone
    std::fill(w.begin(), w.end(), 0.0);
    w[(size_t)R * side + R] = 1.0;
    tot = 1.0;
  }
  std::vector<float> wf(w.size());
  std::vector<int> hw((size_t)side, -1);
  for (int dy = 0; dy < side; ++dy)
    for (int dx = 0; dx < side; ++dx) {
      const double v = w[(size_t)dy * side + dx] / tot;
      wf[(size_t)dy * side + dx] = (float)v;
      if (v != 0.0) hw[(size_t)dy] = std::max(hw[(size_t)dy], std::abs(dx - R));
    }
  call_begin(ctx);
  const size_t wbytes = align_up(sizeof(float) * wf.size(), 256);
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, wbytes + sizeof(int) * hw.size(), &ws));
  float *dW = (float *)ws;
  int *dhw = (int *)((char *)ws + wbytes);
  MORSE_CUDA(ctx, cudaMemcpyAsync(dW, wf.data(), sizeof(float) * wf.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(dhw, hw.data(), sizeof(int) * hw.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
  morse_map *m = map_alloc(ctx, npix, false);
  if (!m) return fail(ctx, MORSE_ENOMEM, "map of %d^2 texels", npix);
  m->L = src->L;
  m->s = src->s;
  m->q = src->q;
  m->a_floor = src->a_floor;
  m->lookup = MORSE_STORE_FP32;
  int r = t_begin(ctx, KT_MAP);
  cudaError_t e = morse::launch_fs_conv(src->A, npix, src->L, R, dW, dhw,
                                        m->A, ctx->stream);
  if (e == cudaSuccess)
    e = morse::launch_quads_from_A(m->A, npix, m->quad, m->qpitch,
                                   ctx->stream);
  t_end(ctx, r);
  ctx->launches += 2;
  morse_status st = e == cudaSuccess ? sync_and_collect(ctx, "finite source")
                                     : cuda_fail(ctx, e, "finite source");
  if (st != MORSE_OK) {
    cudaStreamSynchronize(ctx->stream);
    map_release(m);
    return st;
  }
  *out = m;
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
  // Times are stored as FP32 offsets from t_ref: at |t - t_ref| = 1e5 d
  // they resolve 0.004 d, beyond that the offsets no longer locate a data
  // point on a trajectory (JD-scale times with t_ref = 0 would resolve
  // 0.25 d), so such a t_ref is rejected.
  double t_span = 0.0;
  for (int64_t i = 0; i < n; ++i)
    t_span = std::max(t_span, std::fabs(t[i] - t_ref));
  if (t_span > 1e5)
    return fail(ctx, MORSE_EINVAL,
                "times lie up to %.6g d from t_ref: their FP32 offsets would "
                "resolve only %.3g d; pass a t_ref within the data",
                t_span, t_span * 5.9604644775390625e-8);
  // the search needs the epochs in time order (a straight track crosses the
  // map in one time interval): store them sorted, ties in input order
  std::vector<int64_t> order((size_t)n);
  for (int64_t i = 0; i < n; ++i) order[(size_t)i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [t](int64_t a, int64_t b) { return t[a] < t[b]; });
  // weights, weighted mean flux, FP32 storage; the FP64 constants are sums
  // of the stored FP32 values so that the device data is self-consistent
  // device layout: n float4 slots holding the arrays (t - t_ref, w)[n],
  // w Fc[n] and Fc[n] (structure of arrays, read as such by the sweeps)
  std::vector<float4> h((size_t)n);
  float2 *h_tw = reinterpret_cast<float2 *>(h.data());
  float *h_wf = reinterpret_cast<float *>(h_tw + n);
  float *h_fc = h_wf + n;
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
    h_tw[k] = make_float2(v.x, v.y);
    h_wf[k] = v.z;
    h_fc[k] = v.w;
    // constants of the quadratic the exact sweep evaluates: sum w Fc and
    // sum w Fc^2 with the stored w and Fc
    S1 += (double)v.y;
    SF += (double)v.y * (double)v.w;
    SFF += (double)v.y * (double)v.w * (double)v.w;
  }
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  morse_event *ev = (morse_event *)calloc(1, sizeof(morse_event));
  if (!ev) return fail(ctx, MORSE_ENOMEM, "event");
  if (morse::dev_alloc(ctx, (void **)&ev->ep, sizeof(float4) * (size_t)n) !=
      cudaSuccess) {
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
  ev->invS1 = 1.0 / S1;
  ev->CFF = SFF - SF * SF / S1;
  ev->t_span = t_span;
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
// The top-K of trajectories [first, first + count) of the grid.
static morse_status grid_chi2_impl(morse_ctx *ctx, const morse_event *ev,
                                   const morse_map *map,
                                   const morse_grid *grid, long long first,
                                   long long count, morse_fit *out) {
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  Plan pl;
  MORSE_TRY(plan_search(ctx, ev, grid, first, count, false,
                        morse::map_h16(map), 1, &pl,
                        band_spec(map->npix, map->L, grid_umax(grid), 0.0)));
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, pl.bytes, &ws));
  char *base = (char *)ws;
  Tables T;
  const double dlt = (2.0 * map->L) / (double)map->npix;
  MORSE_TRY(upload_tables(ctx, grid, ev->t_ref, map->L,
                          dlt, base + pl.off_tab, &T));
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  map_params(map, &P);
  event_params(ev, &P);
  grid_params(grid, T, &P);
  P.first = first;
  P.count = count;
  P.stride = 1;
  morse::set_groups(&P);
  morse_fit *fits = (morse_fit *)(base + pl.off_out);
  MORSE_TRY(hdr_init(ctx, base, pl, &P));
  MORSE_TRY(enqueue_cut(ctx, map, grid, T, pl, base, &P));
  MORSE_TRY(enqueue_topk(ctx, pl, P, base, T, fits));
  Hdr h;
  MORSE_CUDA(ctx, cudaMemcpyAsync(&h, base + pl.off_hdr, sizeof(Hdr),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(out, fits, sizeof(morse_fit) * pl.K,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "grid search"));
  return hdr_check(ctx, h);
}

morse_status morse_grid_chi2(morse_ctx *ctx, const morse_event *ev,
                             const morse_map *map, const morse_grid *grid,
                             morse_fit *out) {
  if (!ctx || !out) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  MORSE_TRY(check_grid(ctx, grid));
  return grid_chi2_impl(ctx, ev, map, grid, 0, grid_size(grid), out);
}

morse_status morse_grid_chi2_range(morse_ctx *ctx, const morse_event *ev,
                                   const morse_map *map,
                                   const morse_grid *grid, int64_t first,
                                   int64_t count, morse_fit *out) {
  if (!ctx || !out) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  MORSE_TRY(check_grid(ctx, grid));
  const long long n = grid_size(grid);
  if (first < 0 || count < 1 || first > n || count > n - first)
    return fail(ctx, MORSE_EINVAL,
                "trajectory range [%lld, %lld + %lld) outside the grid of "
                "%lld", (long long)first, (long long)first, (long long)count,
                n);
  return grid_chi2_impl(ctx, ev, map, grid, first, count, out);
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
                        morse::map_h16(map), count, &pl,
                        band_spec(map->npix, map->L, grid_umax(grid), 0.0)));
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, pl.bytes, &ws));
  char *base = (char *)ws;
  Tables T;
  const double dlt = (2.0 * map->L) / (double)map->npix;
  MORSE_TRY(upload_tables(ctx, grid, ev->t_ref, map->L,
                          dlt, base + pl.off_tab, &T));
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
  P.tab_n = pl.tab_n;
  P.tab_c = (unsigned)(P.half + 1) - 0x4B400000u;
  MORSE_TRY(hdr_init(ctx, base, pl, &P));
  MORSE_TRY(enqueue_cut(ctx, map, grid, T, pl, base, &P));
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

// Levenberg-Marquardt refinement of n starts, start i on map maps[0] or,
// with map_of set, on maps[map_of[i]] (maps of one geometry).
static morse_status refine_impl(morse_ctx *ctx, const morse_event *ev,
                                const morse_map *const *maps, int n_maps,
                                const int *map_of, const morse_fit *starts,
                                int n, int iters, int method,
                                morse_fit *out) {
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
    if (map_of && (map_of[i] < 0 || map_of[i] >= n_maps))
      return fail(ctx, MORSE_EINVAL, "start %d: map index %d outside 0..%d",
                  i, map_of[i], n_maps - 1);
  }
  const morse_map *map = maps[0];
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  const size_t nn = (size_t)n;
  // workspace: 36 doubles + 1 int per trajectory, starts, records, and the
  // trajectories' map tables
  const size_t dbl = nn * 36, bytes = sizeof(double) * dbl + sizeof(int) * nn +
                                      2 * sizeof(morse_fit) * nn +
                                      sizeof(void *) * nn + 4096;
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
  const float4 **d_tq = nullptr;
  std::vector<const float4 *> tq;
  if (map_of) {
    d_tq = (const float4 **)align_up((size_t)(d_out + nn), 16);
    tq.resize(nn);
    for (size_t i = 0; i < nn; ++i) tq[i] = maps[map_of[i]]->quad;
    MORSE_CUDA(ctx, cudaMemcpyAsync(d_tq, tq.data(), sizeof(void *) * nn,
                                    cudaMemcpyHostToDevice, ctx->stream));
  }
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
                                         ctx->stream, d_tq);
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
                                      ctx->stream, d_tq));
  t_end(ctx, r);
  MORSE_CUDA(ctx, morse::launch_lm_finish(S, d_starts, n, d_out, ctx->stream));
  ctx->launches += 2;
  MORSE_CUDA(ctx, cudaMemcpyAsync(out, d_out, sizeof(morse_fit) * nn,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  return sync_and_collect(ctx, "refine");
}

morse_status morse_refine(morse_ctx *ctx, const morse_event *ev,
                          const morse_map *map, const morse_fit *starts,
                          int n, int iters, int method, morse_fit *out) {
  if (!ctx) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  return refine_impl(ctx, ev, &map, 1, nullptr, starts, n, iters, method,
                     out);
}

morse_status morse_refine_batch(morse_ctx *ctx, const morse_event *ev,
                                const morse_map *const *maps, int n_maps,
                                const int *map_of, const morse_fit *starts,
                                int n, int iters, int method,
                                morse_fit *out) {
  if (!ctx) return MORSE_EINVAL;
  if (!maps || !map_of || n_maps < 1)
    return fail(ctx, MORSE_EINVAL, "maps, map_of and n_maps >= 1 needed");
  for (int j = 0; j < n_maps; ++j) {
    MORSE_TRY(check_pair(ctx, ev, maps[j]));
    if (maps[j]->npix != maps[0]->npix || maps[j]->L != maps[0]->L)
      return fail(ctx, MORSE_EINVAL,
                  "map %d: every map needs the geometry of map 0 (npix %d, "
                  "extent %g)", j, maps[0]->npix, maps[0]->L);
  }
  return refine_impl(ctx, ev, maps, n_maps, map_of, starts, n, iters, method,
                     out);
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

// ------------------------------------------------------------------ batch
morse_status morse_grid_chi2_batch(morse_ctx *ctx,
                                   const morse_event *const *evs, int n_ev,
                                   const morse_map *const *maps, int n_maps,
                                   const morse_grid *grid, morse_fit *out) {
  if (!ctx || !out || !evs || !maps) return MORSE_EINVAL;
  if (n_ev < 1 || n_maps < 1)
    return fail(ctx, MORSE_EINVAL, "need at least one event and one map");
  if ((long long)n_ev * n_maps > 0x7fffffffLL)
    return fail(ctx, MORSE_EINVAL, "too many (event, map) pairs");
  MORSE_TRY(check_grid(ctx, grid));
  if (grid->a_min > 0.0f)
    return fail(ctx, MORSE_EUNSUPPORTED,
                "the batched search has no minimum-magnification cut");
  for (int e = 0; e < n_ev; ++e)
    if (!evs[e] || evs[e]->ctx != ctx)
      return fail(ctx, MORSE_EINVAL, "event %d is NULL or of another ctx", e);
  for (int m = 0; m < n_maps; ++m) {
    if (!maps[m] || maps[m]->ctx != ctx)
      return fail(ctx, MORSE_EINVAL, "map %d is NULL or of another ctx", m);
    if (maps[m]->npix != maps[0]->npix || maps[m]->L != maps[0]->L ||
        morse::map_h16(maps[m]) != morse::map_h16(maps[0]))
      return fail(ctx, MORSE_EINVAL,
                  "map %d differs from map 0 in npix, extent or lookup "
                  "table; batch maps must share them", m);
  }
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  const int K = grid->top_k;
  const int pairs = n_ev * n_maps;
  const bool h16 = morse::map_h16(maps[0]);
  // launch shapes per light curve, tuned once per bucket and signature
  std::vector<morse_batch_shape> shape_ev((size_t)n_ev);
  for (int e = 0; e < n_ev; ++e) {
    const std::string key = tune_key(ep_bucket(evs[e]->n), grid, maps[0]);
    auto it = ctx->tune.find(key);
    if (it == ctx->tune.end()) {
      morse_batch_shape s =
          default_shape(evs[e]->n, (long long)grid->n_t0 * grid->n_tE);
      if (ctx->tune_mode == MORSE_TUNE_ON) {
        call_begin(ctx);
        MORSE_TRY(batch_tune(ctx, evs[e], maps[0], grid, &s));
      }
      it = ctx->tune.emplace(key, s).first;
    }
    shape_ev[(size_t)e] = it->second;
  }
  call_begin(ctx);
  BatchHost H;
  MORSE_TRY(batch_prepare(ctx, evs, n_ev, maps, n_maps, grid, shape_ev, true,
                          H));
  const BatchLayout L = batch_layout(H, pairs, K);
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, L.bytes, &ws));
  char *base = (char *)ws;
  morse::BatchParams Bp, Bm;
  double *t0abs, *tEv;
  MORSE_TRY(batch_upload(ctx, H, L, base, grid, maps[0], n_ev, &Bp, &Bm,
                         &t0abs, &tEv));
  const size_t smem = morse::batch_smem_bytes(H.ep_cap, K);
  const int bps = morse::batch_blocks_per_sm(h16, smem);
  const size_t smem_g = morse::batch_smem_bytes(0, K);
  const int bps_g = morse::batch_blocks_per_sm(h16, smem_g, 1);
  if (bps < 1 || bps_g < 1)
    return fail(ctx, MORSE_EUNSUPPORTED,
                "batched search kernel does not fit (%d staged epochs, "
                "top_k %d)", H.ep_cap, K);
  // timing events exist before the capture records them
  for (int k = 0; k < 8; ++k) t_end(ctx, t_begin(ctx, KT_SEARCH));
  call_begin(ctx);
  // capture the sequence; update the context's executable graph in place
  // when the shape allows, else instantiate it anew
  MORSE_CUDA(ctx, cudaStreamBeginCapture(ctx->stream,
                                         cudaStreamCaptureModeThreadLocal));
  morse_status st = batch_enqueue(ctx, L, base, Bp, Bm, h16, pairs, t0abs,
                                  tEv, bps * ctx->sm_count, smem, H.main_global,
                                  bps_g * ctx->sm_count, smem_g);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
  if (st != MORSE_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    ctx->rec_kind.clear();
    if (st != MORSE_OK) return st;
    return cuda_fail(ctx, ce, "batch graph capture");
  }
  if (ctx->batch_exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ctx->batch_exec, graph, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(ctx->batch_exec);
      ctx->batch_exec = nullptr;
    }
  }
  if (!ctx->batch_exec) {
    ce = cudaGraphInstantiate(&ctx->batch_exec, graph, 0);
    if (ce != cudaSuccess) {
      cudaGraphDestroy(graph);
      ctx->batch_exec = nullptr;
      ctx->rec_kind.clear();
      return cuda_fail(ctx, ce, "batch graph instantiate");
    }
  }
  cudaGraphDestroy(graph);
  MORSE_CUDA(ctx, cudaGraphLaunch(ctx->batch_exec, ctx->stream));
  BatchHdr h;
  MORSE_CUDA(ctx, cudaMemcpyAsync(&h, base + L.off_hdr, sizeof(h),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(out, base + L.off_fit,
                                  sizeof(morse_fit) * (size_t)pairs * K,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "batched search"));
  return batch_hdr_check(ctx, h);
}

morse_status morse_batch_tuning(morse_ctx *ctx, int mode) {
  if (!ctx) return MORSE_EINVAL;
  if (mode != MORSE_TUNE_OFF && mode != MORSE_TUNE_ON)
    return fail(ctx, MORSE_EINVAL, "unknown tuning mode %d", mode);
  ctx->tune_mode = mode;
  ctx->tune.clear();
  return MORSE_OK;
}

morse_status morse_batch_shape_of(morse_ctx *ctx, int64_t n_ep,
                                  const morse_grid *grid,
                                  const morse_map *map,
                                  morse_batch_shape *out) {
  if (!ctx || !out || !map || n_ep < 1) return MORSE_EINVAL;
  MORSE_TRY(check_grid(ctx, grid));
  auto it = ctx->tune.find(tune_key(ep_bucket(n_ep), grid, map));
  if (it == ctx->tune.end())
    return fail(ctx, MORSE_EINVAL, "no batch shape chosen for this bucket");
  *out = it->second;
  return MORSE_OK;
}

// ------------------------------------------------------------------ probes
morse_status morse_measure_peaks(morse_ctx *ctx, morse_peaks *out) {
  if (!ctx || !out) return MORSE_EINVAL;
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  const size_t win_bytes = (size_t)16 << 20;  // 16 MB gather window
  const int threads = morse::probe_threads();
  const int blocks = 8 * ctx->sm_count;
  const size_t sink_bytes = sizeof(double) * (size_t)blocks * threads;
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, win_bytes + sink_bytes, &ws));
  char *base = (char *)ws;
  MORSE_CUDA(ctx, cudaMemsetAsync(base, 0, win_bytes, ctx->stream));
  void *sink = base + win_bytes;
  cudaEvent_t e0, e1;
  MORSE_CUDA(ctx, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ctx, ce, "probe events");
  }
  // run(n) launches one probe with n iterations per thread; returns ms of
  // the second of two runs, n grown until that takes about 10 ms
  auto timed = [&](auto launch, int &n, double *ms_out) -> cudaError_t {
    for (int round = 0; round < 6; ++round) {
      cudaError_t e = launch(n);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
      if (e == cudaSuccess) e = launch(n);
      if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) return e;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      *ms_out = ms;
      ctx->launches += 2;
      if (ms >= 5.0f || n >= (1 << 24)) break;
      const double grow = ms > 0.01f ? 10.0 / ms : 64.0;
      n = (int)std::min<double>((double)(1 << 24), n * grow);
    }
    return cudaSuccess;
  };
  const double nthr = (double)blocks * threads;
  double ms = 0.0;
  int n = 1024;
  ce = timed([&](int k) { return morse::probe_fma32(blocks, k, (float *)sink,
                                                    ctx->stream); },
             n, &ms);
  if (ce == cudaSuccess)
    out->fp32_fma_per_s = nthr * n * morse::probe_chains() / (ms * 1e-3);
  n = 64;
  if (ce == cudaSuccess)
    ce = timed([&](int k) { return morse::probe_fma64(blocks, k,
                                                      (double *)sink,
                                                      ctx->stream); },
               n, &ms);
  if (ce == cudaSuccess)
    out->fp64_fma_per_s = nthr * n * morse::probe_chains() / (ms * 1e-3);
  n = 256;
  if (ce == cudaSuccess)
    ce = timed([&](int k) { return morse::probe_smem_atomic(
                                blocks, k, (unsigned *)sink, ctx->stream); },
               n, &ms);
  if (ce == cudaSuccess) out->smem_atomics_per_s = nthr * n / (ms * 1e-3);
  const float4 *win = (const float4 *)base;
  n = 256;
  if (ce == cudaSuccess)
    ce = timed([&](int k) { return morse::probe_gather(
                                win, (64u << 10) / 16 - 1, blocks, k,
                                (float *)sink, ctx->stream); },
               n, &ms);
  if (ce == cudaSuccess) out->l1_gather_bytes_per_s = nthr * n * 16.0 / (ms * 1e-3);
  n = 256;
  if (ce == cudaSuccess)
    ce = timed([&](int k) { return morse::probe_gather(
                                win, (unsigned)(win_bytes / 16 - 1), blocks,
                                k, (float *)sink, ctx->stream); },
               n, &ms);
  if (ce == cudaSuccess) out->l2_gather_bytes_per_s = nthr * n * 16.0 / (ms * 1e-3);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return cuda_fail(ctx, ce, "throughput probe");
  return MORSE_OK;
}

// ------------------------------------------------------------------ lines
morse_status morse_caustics(morse_ctx *ctx, double s, double q, int n_psi,
                            morse_caustic out[3], int *n_out) {
  if (!ctx || !out || !n_out) return MORSE_EINVAL;
  if (!(s > 0.0) || !is_fin(s) || !(q > 0.0) || !is_fin(q))
    return fail(ctx, MORSE_EINVAL, "s and q must be finite and > 0");
  if (n_psi < 16 || n_psi > (1 << 20))
    return fail(ctx, MORSE_EINVAL, "n_psi must be in [16, 2^20]");
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  const size_t n = (size_t)4 * n_psi;
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, 2 * n * sizeof(double2), &ws));
  double2 *dz = (double2 *)ws, *dzeta = dz + n;
  MORSE_CUDA(ctx, morse::launch_critical(s, q, n_psi, dz, dzeta,
                                         ctx->stream));
  ctx->launches += 1;
  std::vector<double2> z(n), zeta(n);
  MORSE_CUDA(ctx, cudaMemcpyAsync(z.data(), dz, n * sizeof(double2),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(zeta.data(), dzeta, n * sizeof(double2),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "critical curves"));
  // the 24 orderings of four roots
  std::vector<std::array<int, 4>> perms;
  {
    std::array<int, 4> p = {0, 1, 2, 3};
    do perms.push_back(p);
    while (std::next_permutation(p.begin(), p.end()));
  }
  auto dist = [](double2 a, double2 b) { return hypot(a.x - b.x, a.y - b.y); };
  // the ordering of set b that best continues set a
  auto best_perm = [&](const double2 *a, const double2 *b) {
    int bi = 0;
    double bd = INFINITY;
    for (int i = 0; i < (int)perms.size(); ++i) {
      double d = 0.0;
      for (int t = 0; t < 4; ++t) d += dist(b[perms[i][t]], a[t]);
      if (d < bd) {
        bd = d;
        bi = i;
      }
    }
    return perms[bi];
  };
  for (int k = 1; k < n_psi; ++k) {
    const std::array<int, 4> p = best_perm(&z[4 * (k - 1)], &z[4 * k]);
    double2 tz[4], tc[4];
    for (int t = 0; t < 4; ++t) {
      tz[t] = z[4 * k + p[t]];
      tc[t] = zeta[4 * k + p[t]];
    }
    for (int t = 0; t < 4; ++t) {
      z[4 * k + t] = tz[t];
      zeta[4 * k + t] = tc[t];
    }
  }
  // after a full turn branch t continues as branch wrap[t]: its cycles are
  // the closed critical curves
  const std::array<int, 4> wrap = best_perm(&z[4 * (n_psi - 1)], &z[0]);
  bool seen[4] = {false, false, false, false};
  int nc = 0;
  morse_caustic res[4];
  for (int t = 0; t < 4; ++t) {
    if (seen[t]) continue;
    std::vector<int> cyc;
    for (int j = t; !seen[j]; j = wrap[j]) {
      seen[j] = true;
      cyc.push_back(j);
    }
    double sx = 0.0, sy = 0.0;
    long np = 0;
    for (int k = 0; k < n_psi; ++k)
      for (int j : cyc) {
        sx += zeta[4 * k + j].x;
        sy += zeta[4 * k + j].y;
        ++np;
      }
    const double cx = sx / np, cy = sy / np;
    double size = 0.0;
    for (int k = 0; k < n_psi; ++k)
      for (int j : cyc)
        size = fmax(size, hypot(zeta[4 * k + j].x - cx,
                                zeta[4 * k + j].y - cy));
    res[nc].c1 = cx;
    res[nc].c2 = cy;
    res[nc].size = size;
    res[nc].n_points = (int32_t)np;
    res[nc].reserved = 0;
    ++nc;
  }
  if (nc > 3) return fail(ctx, MORSE_ECUDA, "%d critical curves", nc);
  std::sort(res, res + nc, [](const morse_caustic &a, const morse_caustic &b) {
    const double ax = std::round(a.c1 * 1e9), bx = std::round(b.c1 * 1e9);
    if (ax != bx) return ax < bx;
    return std::round(a.c2 * 1e9) < std::round(b.c2 * 1e9);
  });
  for (int i = 0; i < nc; ++i) out[i] = res[i];
  *n_out = nc;
  return MORSE_OK;
}

morse_status morse_rphi_lines(const morse_caustic *cs, int n_caustics,
                              int n_r, double r_lo, double r_hi, int n_phi,
                              double *lines) {
  if (!cs || !lines || n_caustics < 1 || n_r < 1 || n_phi < 1 ||
      !is_fin(r_lo) || !is_fin(r_hi))
    return MORSE_EINVAL;
  size_t j = 0;
  for (int c = 0; c < n_caustics; ++c)
    for (int i = 0; i < n_r; ++i) {
      const double f = n_r > 1 ? (double)i / (double)(n_r - 1) : 0.0;
      const double r = (r_lo + (r_hi - r_lo) * f) * cs[c].size;
      for (int k = 0; k < n_phi; ++k) {
        const double phi = 2.0 * M_PI * (double)k / (double)n_phi;
        const double dc = cos(phi), ds = sin(phi);
        lines[3 * j + 0] = r + cs[c].c1 * -ds + cs[c].c2 * dc;
        lines[3 * j + 1] = phi;
        lines[3 * j + 2] = cs[c].c1 * dc + cs[c].c2 * ds;
        ++j;
      }
    }
  return MORSE_OK;
}

morse_status morse_grid_chi2_lines(morse_ctx *ctx, const morse_event *ev,
                                   const morse_map *map,
                                   const morse_grid *grid,
                                   const double *lines, morse_fit *out) {
  if (!ctx || !out || !lines || !grid) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  if (grid->n_alpha != 1)
    return fail(ctx, MORSE_EINVAL, "a line grid has n_alpha = 1");
  if (grid->a_min > 0.0f)
    return fail(ctx, MORSE_EUNSUPPORTED,
                "line grids have no minimum-magnification cut");
  // the u0 axis is replaced by the lines: give it valid placeholder bounds
  morse_grid g = *grid;
  g.u0_lo = 1.0;
  g.u0_hi = 1.0;
  g.u0_log = 0;
  MORSE_TRY(check_grid(ctx, &g));
  const int nl = g.n_u0;
  for (int j = 0; j < 3 * nl; ++j)
    if (!is_fin(lines[j])) return fail(ctx, MORSE_EINVAL, "line %d", j / 3);
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  double l_umax = 0.0, l_smax = 0.0;
  for (int j = 0; j < nl; ++j) {
    l_umax = std::max(l_umax, std::fabs(lines[3 * j]));
    l_smax = std::max(l_smax, std::fabs(lines[3 * j + 2]));
  }
  Plan pl;
  MORSE_TRY(plan_search(ctx, ev, &g, 0, grid_size(&g), false,
                        morse::map_h16(map), 1, &pl,
                        band_spec(map->npix, map->L, l_umax, l_smax)));
  const size_t off_lines = align_up(pl.bytes, 256);
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, off_lines + 5 * sizeof(double) * (size_t)nl, &ws));
  char *base = (char *)ws;
  Tables T;
  const double dlt = (2.0 * map->L) / (double)map->npix;
  MORSE_TRY(upload_tables(ctx, &g, ev->t_ref, map->L, dlt, base + pl.off_tab,
                          &T));
  // per line: u, cos, sin, shift, alpha
  std::vector<double> h((size_t)5 * nl);
  for (int j = 0; j < nl; ++j) {
    h[(size_t)j] = lines[3 * j];
    h[(size_t)nl + j] = cos(lines[3 * j + 1]);
    h[(size_t)2 * nl + j] = sin(lines[3 * j + 1]);
    h[(size_t)3 * nl + j] = lines[3 * j + 2];
    h[(size_t)4 * nl + j] = lines[3 * j + 1];
  }
  double *dl = (double *)(base + off_lines);
  MORSE_CUDA(ctx, cudaMemcpyAsync(dl, h.data(), h.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, ctx->stream));
  MORSE_CUDA(ctx, morse::launch_slab_lines(dl, dl + nl, dl + 2 * nl, nl,
                                           map->L, T.slab, ctx->stream));
  ctx->launches += 1;
  morse::SearchParams P;
  memset(&P, 0, sizeof(P));
  map_params(map, &P);
  event_params(ev, &P);
  grid_params(&g, T, &P);
  P.lu = dl;
  P.lc = dl + nl;
  P.ls = dl + 2 * nl;
  P.lsh = dl + 3 * nl;
  P.la = dl + 4 * nl;
  P.first = 0;
  P.count = grid_size(&g);
  P.stride = 1;
  morse::set_groups(&P);
  morse_fit *fits = (morse_fit *)(base + pl.off_out);
  MORSE_TRY(hdr_init(ctx, base, pl, &P));
  MORSE_TRY(enqueue_topk(ctx, pl, P, base, T, fits));
  Hdr hd;
  MORSE_CUDA(ctx, cudaMemcpyAsync(&hd, base + pl.off_hdr, sizeof(Hdr),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(out, fits, sizeof(morse_fit) * pl.K,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "line-grid search"));
  return hdr_check(ctx, hd);
}

}  // extern "C"

namespace {

morse_status check_peak_opts(morse_ctx *ctx, const morse_peak_opts *o) {
  if (!o) return fail(ctx, MORSE_EINVAL, "peak options");
  if (o->sub < 1 || o->sub > 16)
    return fail(ctx, MORSE_EINVAL, "sub %d outside 1..16", o->sub);
  if (o->max_peaks < 1 || o->max_peaks > morse::kPeakMax)
    return fail(ctx, MORSE_EINVAL, "max_peaks %d outside 1..%d", o->max_peaks,
                morse::kPeakMax);
  if (!(o->delta >= 0.0) || !is_fin(o->delta))
    return fail(ctx, MORSE_EINVAL, "delta must be finite and >= 0");
  return MORSE_OK;
}

// lines[3 j ..] = (u, alpha, shift) -> device arrays u, cos, sin, shift,
// alpha of n doubles each at d (cos and sin taken here, in FP64)
morse_status upload_lines(morse_ctx *ctx, const double *lines, int n,
                          double *d) {
  for (int j = 0; j < 3 * n; ++j)
    if (!is_fin(lines[j])) return fail(ctx, MORSE_EINVAL, "line %d", j / 3);
  std::vector<double> h((size_t)5 * n);
  for (int j = 0; j < n; ++j) {
    h[(size_t)j] = lines[3 * j];
    h[(size_t)n + j] = cos(lines[3 * j + 1]);
    h[(size_t)2 * n + j] = sin(lines[3 * j + 1]);
    h[(size_t)3 * n + j] = lines[3 * j + 2];
    h[(size_t)4 * n + j] = lines[3 * j + 1];
  }
  MORSE_CUDA(ctx, cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double),
                                  cudaMemcpyHostToDevice, ctx->stream));
  // the staging vector must outlive the copy
  MORSE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return MORSE_OK;
}

// Device layout of a peak library of n lines, P peaks each, at base + off.
struct PeakLib {
  double *lines;  // 5 n: u, cos, sin, shift, alpha
  int *count;     // n (per map)
  double *pos, *height;  // n P each (per map)
  unsigned *err;
  const float **maps;    // the maps' values (batched library)
  size_t bytes;
};

// (n_maps > 1: counts and peaks of every map, map-major; then the maps'
// value pointers)
PeakLib peak_lib_layout(char *base, size_t off, int n, int P,
                        int n_maps = 1) {
  PeakLib L;
  const size_t nm = (size_t)n * (size_t)n_maps;
  size_t o = align_up(off, 256);
  L.lines = (double *)(base + o);
  o = align_up(o + sizeof(double) * 5 * (size_t)n, 256);
  L.count = (int *)(base + o);
  o = align_up(o + sizeof(int) * nm, 256);
  L.pos = (double *)(base + o);
  o = align_up(o + sizeof(double) * nm * P, 256);
  L.height = (double *)(base + o);
  o = align_up(o + sizeof(double) * nm * P, 256);
  L.err = (unsigned *)(base + o);
  o += 256;
  L.maps = (const float **)(base + o);
  o = align_up(o + sizeof(void *) * (size_t)n_maps, 256);
  L.bytes = o - off;
  return L;
}

morse_status enqueue_peak_lib(morse_ctx *ctx, const morse_map *map,
                              const PeakLib &L, int n,
                              const morse_peak_opts *o) {
  MORSE_CUDA(ctx, cudaMemsetAsync(L.err, 0, sizeof(unsigned), ctx->stream));
  const float r = (float)(1.0 + o->delta);
  const int tr = t_begin(ctx, KT_PEAKS);
  MORSE_CUDA(ctx, morse::launch_line_peaks(
                      map->A, nullptr, 1, map->npix, map->L, L.lines,
                      L.lines + n, L.lines + 2 * (size_t)n,
                      L.lines + 3 * (size_t)n, n, o->sub, r, o->max_peaks,
                      L.count, L.pos, L.height, L.err, ctx->stream));
  t_end(ctx, tr);
  ctx->launches += 1;
  return MORSE_OK;
}

}  // namespace

extern "C" {

morse_status morse_line_peaks(morse_ctx *ctx, const morse_map *map,
                              const double *lines, int n_lines,
                              const morse_peak_opts *opts, int32_t *count,
                              double *pos, double *height) {
  if (!ctx || !map || !lines || !count || !pos || !height || n_lines < 1)
    return MORSE_EINVAL;
  if (map->ctx != ctx) return fail(ctx, MORSE_EINVAL, "map of another ctx");
  MORSE_TRY(check_peak_opts(ctx, opts));
  if (map->npix < 2) return fail(ctx, MORSE_EINVAL, "map of one texel");
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  const int P = opts->max_peaks;
  const size_t bytes = peak_lib_layout(nullptr, 0, n_lines, P).bytes;
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, bytes, &ws));
  const PeakLib L = peak_lib_layout((char *)ws, 0, n_lines, P);
  MORSE_TRY(upload_lines(ctx, lines, n_lines, L.lines));
  MORSE_TRY(enqueue_peak_lib(ctx, map, L, n_lines, opts));
  unsigned err = 0;
  MORSE_CUDA(ctx, cudaMemcpyAsync(count, L.count, sizeof(int) * n_lines,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(pos, L.pos,
                                  sizeof(double) * (size_t)n_lines * P,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(height, L.height,
                                  sizeof(double) * (size_t)n_lines * P,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(&err, L.err, sizeof(unsigned),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "peak library"));
  if (err) return fail(ctx, MORSE_ECUDA, "peak library: sample run clipped");
  return MORSE_OK;
}

morse_status morse_line_peaks_batch(morse_ctx *ctx,
                                    const morse_map *const *maps, int n_maps,
                                    const double *lines, int n_lines,
                                    const morse_peak_opts *opts,
                                    int32_t *count, double *pos,
                                    double *height) {
  if (!ctx || !maps || !lines || !count || !pos || !height || n_lines < 1 ||
      n_maps < 1)
    return MORSE_EINVAL;
  if ((long long)n_lines * n_maps > 0x7fffffffLL)
    return fail(ctx, MORSE_EINVAL, "too many (map, line) pairs");
  for (int m = 0; m < n_maps; ++m) {
    if (!maps[m] || maps[m]->ctx != ctx)
      return fail(ctx, MORSE_EINVAL, "map %d is NULL or of another ctx", m);
    if (maps[m]->npix != maps[0]->npix || maps[m]->L != maps[0]->L)
      return fail(ctx, MORSE_EINVAL,
                  "map %d differs from map 0 in npix or extent", m);
  }
  MORSE_TRY(check_peak_opts(ctx, opts));
  if (maps[0]->npix < 2) return fail(ctx, MORSE_EINVAL, "map of one texel");
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  const int P = opts->max_peaks;
  const size_t nm = (size_t)n_lines * (size_t)n_maps;
  const size_t bytes = peak_lib_layout(nullptr, 0, n_lines, P, n_maps).bytes;
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, bytes, &ws));
  const PeakLib L = peak_lib_layout((char *)ws, 0, n_lines, P, n_maps);
  std::vector<const float *> ptr((size_t)n_maps);
  for (int m = 0; m < n_maps; ++m) ptr[(size_t)m] = maps[m]->A;
  MORSE_CUDA(ctx, cudaMemcpyAsync(L.maps, ptr.data(),
                                  sizeof(void *) * (size_t)n_maps,
                                  cudaMemcpyHostToDevice, ctx->stream));
  MORSE_TRY(upload_lines(ctx, lines, n_lines, L.lines));  // synchronises
  MORSE_CUDA(ctx, cudaMemsetAsync(L.err, 0, sizeof(unsigned), ctx->stream));
  const float r = (float)(1.0 + opts->delta);
  const int n = n_lines;
  const int tr = t_begin(ctx, KT_PEAKS);
  MORSE_CUDA(ctx, morse::launch_line_peaks(
                      nullptr, L.maps, n_maps, maps[0]->npix, maps[0]->L,
                      L.lines, L.lines + n, L.lines + 2 * (size_t)n,
                      L.lines + 3 * (size_t)n, n, opts->sub, r, P, L.count,
                      L.pos, L.height, L.err, ctx->stream));
  t_end(ctx, tr);
  ctx->launches += 1;
  unsigned err = 0;
  MORSE_CUDA(ctx, cudaMemcpyAsync(count, L.count, sizeof(int) * nm,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(pos, L.pos, sizeof(double) * nm * P,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(height, L.height, sizeof(double) * nm * P,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(&err, L.err, sizeof(unsigned),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "peak library"));
  if (err) return fail(ctx, MORSE_ECUDA, "peak library: sample run clipped");
  return MORSE_OK;
}

morse_status morse_peak_search(morse_ctx *ctx, const morse_event *ev,
                               const morse_map *map, const morse_grid *grid,
                               const double *lines, int n_lines,
                               const morse_peak_opts *opts, int min_peaks,
                               const double *tp, int n_tp, morse_fit *out) {
  if (!ctx || !out || !lines || !grid || n_lines < 1) return MORSE_EINVAL;
  MORSE_TRY(check_pair(ctx, ev, map));
  MORSE_TRY(check_peak_opts(ctx, opts));
  if (map->npix < 2) return fail(ctx, MORSE_EINVAL, "map of one texel");
  if (n_tp < 0 || n_tp > 2 || (n_tp > 0 && !tp))
    return fail(ctx, MORSE_EINVAL, "n_tp must be 0, 1 or 2");
  for (int i = 0; i < n_tp; ++i)
    if (!is_fin(tp[i])) return fail(ctx, MORSE_EINVAL, "peak time %d", i);
  if (n_tp == 2 && !(tp[1] > tp[0]))
    return fail(ctx, MORSE_EINVAL, "peak times must increase");
  if (min_peaks < 0) return fail(ctx, MORSE_EINVAL, "min_peaks < 0");
  if (grid->n_alpha != 1)
    return fail(ctx, MORSE_EINVAL, "a line grid has n_alpha = 1");
  if (n_tp == 2 && grid->n_tE != 1)
    return fail(ctx, MORSE_EINVAL, "two peak times fix tE: n_tE = 1");
  const int P = opts->max_peaks;
  const int mode = n_tp;
  const int S = mode == 0 ? 1 : mode == 1 ? P : P * (P - 1) / 2;
  if (S < 1)
    return fail(ctx, MORSE_EINVAL, "two peak times need max_peaks >= 2");
  const long long ne = (long long)n_lines * S;
  if (ne > (1LL << 30)) return fail(ctx, MORSE_EINVAL, "too many entries");
  const int E = (int)ne;
  // the entries replace the u0 axis; the t0 axis runs about t_p1
  morse_grid g = *grid;
  g.n_u0 = E;
  g.u0_lo = 1.0;
  g.u0_hi = 1.0;
  g.u0_log = 0;
  g.a_min = 0.0f;
  if (n_tp >= 1) {
    g.t0_lo += tp[0];
    g.t0_hi += tp[0];
  }
  if (n_tp == 2) {  // tE per entry; the axis is a placeholder
    g.tE_lo = 1.0;
    g.tE_hi = 1.0;
    g.tE_log = 0;
  }
  MORSE_TRY(check_grid(ctx, &g));
  MORSE_CUDA(ctx, cudaSetDevice(ctx->device));
  call_begin(ctx);
  // band tables unless tE varies per entry (two peak times); positions
  // along a line lie within 2 sqrt(2) L of its reference point
  BandSpec band;
  if (n_tp < 2) {
    double umax = 0.0, smax = 0.0;
    for (int j = 0; j < n_lines; ++j) {
      umax = std::max(umax, std::fabs(lines[3 * j]));
      smax = std::max(smax, std::fabs(lines[3 * j + 2]));
    }
    band = band_spec(map->npix, map->L, umax, smax + 3.0 * map->L);
  }
  Plan pl;
  MORSE_TRY(plan_search(ctx, ev, &g, 0, grid_size(&g), false,
                        morse::map_h16(map), 1, &pl, band));
  const size_t off_lib = align_up(pl.bytes, 256);
  const size_t lib_bytes = peak_lib_layout(nullptr, off_lib, n_lines, P).bytes;
  const size_t off_ent = align_up(off_lib + lib_bytes, 256);
  const size_t ent_bytes = sizeof(double) * 7 * (size_t)E;
  void *ws = nullptr;
  MORSE_TRY(ws_reserve(ctx, off_ent + ent_bytes, &ws));
  char *base = (char *)ws;
  Tables T;
  const double dlt = (2.0 * map->L) / (double)map->npix;
  MORSE_TRY(upload_tables(ctx, &g, ev->t_ref, map->L, dlt, base + pl.off_tab,
                          &T));
  const PeakLib L = peak_lib_layout(base, off_lib, n_lines, P);
  MORSE_TRY(upload_lines(ctx, lines, n_lines, L.lines));
  MORSE_TRY(enqueue_peak_lib(ctx, map, L, n_lines, opts));
  double *de = (double *)(base + off_ent);
  morse::PeakEntries PE;
  PE.u = de;
  PE.c = de + (size_t)E;
  PE.s = de + 2 * (size_t)E;
  PE.shift = de + 3 * (size_t)E;
  PE.alpha = de + 4 * (size_t)E;
  PE.keep = de + 5 * (size_t)E;
  PE.tE = mode == 2 ? de + 6 * (size_t)E : nullptr;
  const int need = std::max(min_peaks, n_tp);
  const size_t n = (size_t)n_lines;
  MORSE_CUDA(ctx, morse::launch_peak_entries(
                      n_lines, L.lines, L.lines + n, L.lines + 2 * n,
                      L.lines + 3 * n, L.lines + 4 * n, L.count, L.pos, P,
                      mode, need, n_tp >= 1 ? tp[0] : 0.0,
                      n_tp == 2 ? tp[1] : 0.0, PE, ctx->stream));
  MORSE_CUDA(ctx, morse::launch_slab_lines(PE.u, PE.c, PE.s, E, map->L,
                                           T.slab, ctx->stream));
  ctx->launches += 2;
  morse::SearchParams Q;
  memset(&Q, 0, sizeof(Q));
  map_params(map, &Q);
  event_params(ev, &Q);
  grid_params(&g, T, &Q);
  Q.lu = PE.u;
  Q.lc = PE.c;
  Q.ls = PE.s;
  Q.lsh = PE.shift;
  Q.la = PE.alpha;
  Q.ltE = PE.tE;
  Q.linemax = PE.keep;  // the peak-count cut: entries not in use
  Q.a_min = 0.5f;
  Q.first = 0;
  Q.count = grid_size(&g);
  Q.stride = 1;
  morse::set_groups(&Q);
  morse_fit *fits = (morse_fit *)(base + pl.off_out);
  MORSE_TRY(hdr_init(ctx, base, pl, &Q));
  MORSE_TRY(enqueue_topk(ctx, pl, Q, base, T, fits));
  Hdr hd;
  unsigned err = 0;
  MORSE_CUDA(ctx, cudaMemcpyAsync(&hd, base + pl.off_hdr, sizeof(Hdr),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(&err, L.err, sizeof(unsigned),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_CUDA(ctx, cudaMemcpyAsync(out, fits, sizeof(morse_fit) * pl.K,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  MORSE_TRY(sync_and_collect(ctx, "peak-aligned search"));
  if (err) return fail(ctx, MORSE_ECUDA, "peak library: sample run clipped");
  return hdr_check(ctx, hd);
}

}  // extern "C"
