// Internal declarations of the MORSE GB300 library: handle layouts, kernel
// parameter blocks and launchers.  Not part of the public ABI (morse.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "morse.h"

// kernel kinds timed per call (morse_last_kernel_ms)
enum { KT_RAY = 0, KT_MAP = 1, KT_SEARCH = 2, KT_MERGE = 3, KT_FILL = 4,
       KT_ADJ = 5, KT_LM = 6, KT_PEAKS = 7, KT_COUNT = 8 };

struct morse_ctx {
  int device;
  cudaStream_t stream;
  bool own_stream;
  int sm_count;
  size_t smem_optin;        // max dynamic shared memory per block
  char err[512];
  void *ws;                 // device workspace (grow-only)
  size_t ws_bytes;
  // per-call kernel timing: event pairs recorded around each launch, summed
  // by kind once the call has synchronised
  std::vector<cudaEvent_t> evpool;
  std::vector<int> rec_kind;   // kind of record r (events 2r, 2r+1)
  double kernel_ms[KT_COUNT];
  uint64_t launches;        // kernels launched by this context
  morse_map *sweep_map;     // map storage reused by sweeps
  morse_map *sweep_map2;    // the second buffer: map i + 1 is built (on
                            // build_stream) while map i is searched
  cudaStream_t build_stream;  // created on a sweep's first use
  cudaEvent_t sweep_ev[4];    // built[2], free[2] of the two buffers
  unsigned long long last_exact;  // exact sweeps in the last search call
  // batched search: autotuned launch shapes per epoch-count bucket (key:
  // bucket and the search signature) and the reusable graph
  std::map<std::string, morse_batch_shape> tune;
  int tune_mode;            // MORSE_TUNE_*
  cudaGraphExec_t batch_exec;
  // injected faults (morse_inject_fault; tests of the error paths)
  unsigned spin_limit;      // spins before a block top-K lock wait gives up
  int fault_lock_held;      // searches start with every block lock taken
  long long fault_alloc;    // > 0: the fault_alloc-th device allocation
                            // from now fails (then the count is spent)
  unsigned pub_tag;         // tag of the last top-K search launch
};

struct morse_map {
  morse_ctx *ctx;
  int npix;
  double L, s, q, X;
  int64_t nray;
  bool has_counts;
  uint32_t *counts;         // [npix*npix] ray counts (device)
  float *A;                 // [npix*npix] FP32 magnification (device)
  float4 *quad;             // [npix + 1 rows x qpitch] bilinear cells of
                            // A - 1 (edge rows/columns repeated below and
                            // above the map), pre-differenced along x
  int qpitch;               // quads per row: npix + pad (spreads the rows of
                            // a steep track over cache sets)
  unsigned long long *tot;  // [2] off-map, lost (device)
  uint64_t off_map, lost;
  // FP16 storage form (present when built with MORSE_STORE_FP16LOG or
  // selected later): half(log10(max(A, a_floor))) per texel, and the same
  // 2x2 neighbourhoods as quad packed as four halves (8 bytes)
  uint16_t *hcodes;         // [npix*npix]
  uint2 *quadh;             // [npix + 1 rows x qpitch], cells as quad
  double a_floor;           // half a ray (ray-shot maps), else 1e-6
  bool half_valid;          // the FP16 table holds the current values
  int lookup;               // MORSE_STORE_FP32 or MORSE_STORE_FP16LOG
};

struct morse_event {
  morse_ctx *ctx;
  int64_t n;
  double t_ref;
  float4 *ep;               // n float4 slots holding, as arrays,
                            // (t - t_ref, w)[n], w (F - F_ref)[n],
                            // (F - F_ref)[n]
  double S1, SF, SFF, Fref; // FP64 sums of the stored FP32 values
  double invS1, CFF;        // 1/S_1, S_FF - S_F^2/S_1
  double t_span;            // max |t - t_ref| over the epochs
};

namespace morse {

// ---------------------------------------------------------------- maps
// searches read the FP16 log10 table
inline bool map_h16(const morse_map *m) {
  return m->lookup == MORSE_STORE_FP16LOG && m->quadh != nullptr &&
         m->half_valid;
}

struct RayParams {
  double e1, e2, xa, xb;    // lens mass fractions and positions
  double X, h, L, dlt;      // image half-width, ray spacing, map half-width,
                            // texel size
  float e1f, e2f, xaf, xbf; // FP32 copies
  float x0f, hf;            // first ray centre, ray spacing
  float invdf, offf;        // v = y / Delta + L / Delta
  float npixf;
  int npix;
  int64_t nray;
  int tiles_x, tiles_y;
  int sub_rows;             // rays per thread sub-block along y (tile
                            // height kRayWarps * sub_rows)
  uint32_t *counts;
  unsigned long long *tot;  // [0] off-map rays, [1] lost rays, [2] next
                            // tile (all zero before the launch)
};

constexpr int kRayTileX = 256;    // rays per tile along x
constexpr int kRayWarps = 16;     // sub-block rows per tile (warps per block)
constexpr int kRaySubRowsMax = 16;  // tile height at most 256 rays (512:
                                    // 10 % slower, more rays land outside
                                    // the window)
constexpr int kRayWin = 128;      // shared-memory window side (bins)
constexpr int kRayThreads = 512;  // threads per ray-shooting block

cudaError_t launch_rayshoot(const RayParams &P, bool fp64, int grid,
                            cudaStream_t st);
// Cell tables: (npix + 1)^2 bilinear cells, stored either row-major with a
// row pitch of quad_pitch cells (MORSE_TILE_W = 1), or in tiles of
// MORSE_TILE_W x MORSE_TILE_H cells (powers of two) laid out row-major, so
// that the cells a warp gathers along a track of any direction share fewer
// cache lines.
#ifndef MORSE_QPITCH_PAD
#define MORSE_QPITCH_PAD 8
#endif
#ifndef MORSE_TILE_W
#define MORSE_TILE_W 1
#endif
#ifndef MORSE_TILE_H
#define MORSE_TILE_H 1
#endif
constexpr int kTileW = MORSE_TILE_W, kTileH = MORSE_TILE_H;
constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }
constexpr int kTileLW = ilog2c(kTileW), kTileLH = ilog2c(kTileH);
static_assert((1 << kTileLW) == kTileW && (1 << kTileLH) == kTileH,
              "tile sides are powers of two");
// cells per stored row (a multiple of the tile width)
inline int quad_pitch(int npix) {
  const int p = npix + MORSE_QPITCH_PAD;
  return (p + kTileW - 1) / kTileW * kTileW;
}
// stored rows (a multiple of the tile height)
inline int quad_rows(int npix) {
  return (npix + 1 + kTileH - 1) / kTileH * kTileH;
}
inline size_t quad_count(int npix) {
  return (size_t)quad_rows(npix) * (size_t)quad_pitch(npix);
}
// storage index of cell (c, r)
__host__ __device__ __forceinline__ size_t cell_index(int c, int r,
                                                      int qpitch) {
  if (kTileW == 1 && kTileH == 1) return (size_t)r * qpitch + c;
  const size_t tile = (size_t)(r >> kTileLH) * (size_t)(qpitch >> kTileLW) +
                      (size_t)(c >> kTileLW);
  return (tile << (kTileLW + kTileLH)) |
         (size_t)(((r & (kTileH - 1)) << kTileLW) | (c & (kTileW - 1)));
}
// Row stride of a band table (entries): npix + 1 cells rounded up to 4 mod 8.
// A warp's 16-byte loads are served eight lanes at a time, one bank group
// (of eight) per entry; with a stride of 4 mod 8 the cells one row and up
// to three columns apart, which neighbouring epochs read where the line
// crosses a row, fall in distinct bank groups.
__host__ __device__ __forceinline__ int band_stride(int npix) {
  return (npix + 1) + ((4 - (npix + 1)) & 7);
}
// quad index offset of the folded floor-bit index (see SearchParams)
inline unsigned quad_idx0(int npix) {
  return (unsigned)(npix / 2 + 1 - 0x4B400000) *
         (unsigned)(quad_pitch(npix) + 1);
}

cudaError_t launch_counts_to_map(const uint32_t *counts, int npix, double f,
                                 float *A, float4 *quad, int qpitch,
                                 cudaStream_t st);
cudaError_t launch_quads_from_A(const float *A, int npix, float4 *quad,
                                int qpitch, cudaStream_t st);
// FP16 form from the FP32 values: codes, then their 2x2 quads
cudaError_t launch_half_from_A(const float *A, int npix, double a_floor,
                               uint16_t *codes, uint2 *quadh, int qpitch,
                               cudaStream_t st);
int rayshoot_blocks_per_sm();
// finite-source map: A convolved with the (2R+1)^2 weights W (rows dy),
// rowhw[dy + R] = largest |dx| of a nonzero weight in row dy (-1: none)
size_t fs_smem_bytes(int R);
// unnormalised texel weights of a source of radius rho_px texels, limb
// darkening gamma: w[(dy + R)(2R + 1) + dx + R]
cudaError_t launch_fs_weights(double rho_px, double gamma, int R, double *w,
                              cudaStream_t st);
cudaError_t launch_fs_conv(const float *A, int npix, double L, int R,
                           const float *W, const int *rowhw, float *out,
                           cudaStream_t st);
// point-source A at the npix^2 texel centres by the lens polynomial (FP64)
cudaError_t launch_poly_map(double s, double q, double L, int npix, float *A,
                            int sm_count, cudaStream_t st);

// ---------------------------------------------------------------- search
struct Entry {
  double chi2;
  long long idx;
};

// levels of published block quantiles (search_group.cuh: pub_update)
constexpr int kPubLevels = 3;

struct SearchParams {
  // map: the lookup reads quadh (FP16 log10 quads) when it is set, else
  // quad (FP32 A - 1 quads); both share qpitch and the index folding
  const float4 *quad;
  const uint2 *quadh;
  int npix, half;           // npix, npix/2
  int qpitch;               // quad row pitch (quads)
  unsigned qidx0;           // quad index offset for the raw floor bits:
                            // (half + 1 - 0x4B400000) (qpitch + 1) mod 2^32
  float vlo, vhi;           // inside iff vlo < v < vhi (centred coords)
  float voff;               // -coff: y = (v + voff) Delta
  float dltf;               // Delta
  float invDf;              // 1/Delta
  double invD;              // 1/Delta
  double coff;              // v = y/Delta + coff
  double L, dlt;            // map half-width, Delta (FP64)
  // event
  const float4 *ep;
  int n_ep;
  double S1, SF, SFF, Fref;
  double invS1, CFF;        // 1/S_1 and S_FF - S_F^2/S_1 (pruning bound)
  double gamma;             // relative bound of the FP32 phase-1 sums
  // grid tables (device, FP64)
  const double *u0v, *ca, *sa, *t0rel, *invtEd, *tEv;
  const double2 *slab;      // [n_u0 n_alpha] tau interval of each line
                            // inside the map (k_slab)
  // line grids (n_alpha = 1, line = i_u0), else nullptr: per line the
  // impact u about the origin, cos and sin of the direction, the tau of the
  // closest approach to the line's reference point past that to the origin
  // (grid t0 is the time of the former), and the direction alpha
  const double *lu, *lc, *ls, *lsh, *la;
  const double *ltE;        // line grid: tE per line (Eq. 8), else null
  int n_u0, n_alpha, n_t0, n_tE;
  long long first, count;   // trajectories first + i * stride, i < count
  long long stride;
  int tpg;                  // trajectories per warp group (1..32)
  long long line;           // trajectories per (u0, alpha) line
  long long ng_line;        // warp groups per line (main pass)
  const double *linemax;    // [n_u0 n_alpha] largest A of each line, or
                            // nullptr: no minimum-magnification cut
  double a_min;             // the cut (with linemax)
  int top_k;
  // outputs
  Entry *partial;           // [gridDim.x][top_k] (top-K mode)
  double *dchi2, *dFs, *dFb;  // [count] (dense mode)
  // optional device words (nullptr: unused)
  unsigned long long *gthr; // grid-wide pruning threshold (chi^2 bits),
                            // all-ones = +inf
  unsigned int *err;        // bit 0: a block lock spin gave up;
                            // bit 1: texel index out of range, bit 2: a
                            // band-table cell differs from the map's
                            // (checked build only)
  unsigned long long *stat_exact;  // trajectories given the exact sweep
  int pilot_ub;             // 1: key the candidates by chi2_upper instead
                            // of the exact sweep (the pilot pass)
  unsigned spin_limit;      // block top-K lock: spins before giving up
  int lock0;                // initial lock word (1: held, an injected fault)
  // Published block quantiles (nullptr: off): kPubLevels rows, pub_stride
  // words apart, of pub_nb words (launch tag << 32 | FP32 bits of a list's
  // j-th chi^2, rounded up), one per top-K list of the search; this list's
  // word is pub_me (-1: blockIdx.x).  Words of another tag are ignored.
  unsigned long long *pub;
  unsigned pub_tag;
  int pub_nb, pub_me, pub_stride;
  // Shared-memory band tables of the line-aligned pass (k_search only;
  // 0 = off): entries per table, 4 band_stride(npix), two tables after the
  // lists.
  int tab_n;
  unsigned tab_c;           // half + 1 - 0x4B400000: floor bits -> cell
};

// ------------------------------------------- host set-up of a search
// Grid tables in device memory: the lines' tau intervals inside the map,
// then u0, cos and sin alpha, t0 - t_ref, 1/(tE Delta), and the absolute t0
// and tE of the output records.
struct Tables {
  double2 *slab;
  double *u0v, *ca, *sa, *t0rel, *invtEd, *t0abs, *tEv;
};
// bytes of the tables of grid g (slabs first, 16-byte aligned)
size_t tables_bytes(const morse_grid *g);
// number of FP64 table values after the slabs
size_t table_values(const morse_grid *g);
// the table values of g in device order, written to h[table_values(g)]
void table_host(const morse_grid *g, double t_ref, double dlt, double *h);
// the table pointers of g laid out at dev
void tables_at(const morse_grid *g, void *dev, Tables *T);
// search parameters from the handles (every search path sets them alike)
void map_params(const morse_map *map, SearchParams *P);
void event_params(const morse_event *ev, SearchParams *P);
void grid_params(const morse_grid *g, const Tables &T, SearchParams *P);
void ctx_params(const morse_ctx *ctx, SearchParams *P);
// device allocation through the context: cudaMalloc, or the injected
// failure of morse_inject_fault (cudaErrorMemoryAllocation, nothing made)
cudaError_t dev_alloc(morse_ctx *ctx, void **p, size_t bytes);

struct FillParams {
  SearchParams S;
  const Entry *sel;         // [k] selected (chi2, idx)
  int k;
  const double *t0abs, *tEv;  // absolute t0 and tE tables
  morse_fit *out;           // [k]
};

#ifndef MORSE_SEARCH_WARPS
#define MORSE_SEARCH_WARPS 16
#endif
constexpr int kSearchWarps = MORSE_SEARCH_WARPS;  // one block per SM
#ifndef MORSE_TPG
#define MORSE_TPG 32
#endif
constexpr int kTpgMain = MORSE_TPG;  // main pass, at most
#ifndef MORSE_TPG_PILOT
#define MORSE_TPG_PILOT 2  // (4: 0.7 % slower step, 8: 2.6 %, 1: 0.6 %)
#endif
constexpr int kTpgPilot = MORSE_TPG_PILOT;  // pilot: spread a small sample
                                            // over every SM
// pilot sample: max(kPilotMinK K, kPilotSqrt sqrt(K N)) trajectories
#ifndef MORSE_PILOT_SQRT
#define MORSE_PILOT_SQRT 0.25
#endif
#ifndef MORSE_PILOT_MIN_K
#define MORSE_PILOT_MIN_K 4.0
#endif
constexpr double kPilotSqrt = MORSE_PILOT_SQRT, kPilotMinK = MORSE_PILOT_MIN_K;
// the batched search's pilot (its own launch shapes and merge)
#ifndef MORSE_BATCH_PILOT_SQRT
#define MORSE_BATCH_PILOT_SQRT 1.0
#endif
#ifndef MORSE_BATCH_PILOT_MIN_K
#define MORSE_BATCH_PILOT_MIN_K 16.0
#endif
constexpr double kBatchPilotSqrt = MORSE_BATCH_PILOT_SQRT,
                 kBatchPilotMinK = MORSE_BATCH_PILOT_MIN_K;
// published list quantiles in the batched search (1: on)
#ifndef MORSE_BATCH_PUB
#define MORSE_BATCH_PUB 1
#endif

// Line-aligned warp groups for the main pass: about one line per block
// round (line = n_t0 n_tE trajectories share a track's line).
inline int line_tpg(long long line) {
  long long t = (line + kSearchWarps - 1) / kSearchWarps;
  if (t > kTpgMain) t = kTpgMain;
  if (t < 8) t = 8 < kTpgMain ? 8 : kTpgMain;
  return (int)t;
}
inline void set_groups(SearchParams *P) {
  P->line = (long long)P->n_t0 * P->n_tE;
  P->tpg = line_tpg(P->line);
  P->ng_line = (P->line + P->tpg - 1) / P->tpg;
}
// number of warp groups of the main pass over [first, first + count)
inline long long main_groups(long long line, long long first,
                             long long count) {
  const int t = line_tpg(line);
  const long long ng = (line + t - 1) / t;
  return ((first + count - 1) / line - first / line + 1) * ng;
}

size_t search_smem_bytes(int n_ep_smem, int top_k);
int search_blocks_per_sm(bool dense, bool ep_smem, bool h16, size_t smem);
// (the FP16 kernels are chosen when P.quadh is set)
cudaError_t launch_search(const SearchParams &P, bool dense, bool ep_smem,
                          int grid, size_t smem, cudaStream_t st);
// Merge `lists` sorted lists of `k` entries (ping-pong between a and b) into
// one; returns the buffer that holds the result and the launches queued.
// With `seed`, also seed *seed from the result as launch_seed_threshold.
cudaError_t launch_topk_merge(Entry *a, Entry *b, int lists, int k,
                              Entry **result, int *levels, cudaStream_t st,
                              unsigned long long *seed = nullptr);
cudaError_t launch_fill(const FillParams &F, cudaStream_t st);
// gthr <- min(gthr, chi^2 bits of sel[k-1]) when that entry is real
cudaError_t launch_seed_threshold(const Entry *sel, int k,
                                  unsigned long long *gthr, cudaStream_t st);
// out[iu n_alpha + ia] = largest magnification on line (u0v[iu], alpha_ia)
cudaError_t launch_line_max(const float *A, int npix, double L,
                            const double *u0v, const double *ca,
                            const double *sa, int n_u0, int n_alpha,
                            double *out, cudaStream_t st);
// slab[i] = tau interval of line i of a line grid (u[i], c[i], s[i])
cudaError_t launch_slab_lines(const double *u, const double *c,
                              const double *s, int n, double L, double2 *slab,
                              cudaStream_t st);
// ---------------------------------------------------------------- peaks
constexpr int kPeakMax = 16;  // peaks kept per line, at most
// Peak library of lines (lu, lc, ls) with reference shifts lsh (§4.3
// (iii)): count[j], and the max_peaks highest peaks as pos[j max_peaks + m]
// (tau from the reference point) and height[...], NaN in unused slots;
// err |= 1 if the sample run was clipped (never expected)
// (of the map A, or with As set of the n_maps maps As[m] of one geometry:
// outputs of map m, line j at index m n_lines + j)
cudaError_t launch_line_peaks(const float *A, const float *const *As,
                              int n_maps, int npix, double L,
                              const double *lu, const double *lc,
                              const double *ls, const double *lsh,
                              int n_lines, int sub, float r, int max_peaks,
                              int *count, double *pos, double *height,
                              unsigned *err, cudaStream_t st);
// Peak-aligned line-grid entries (§4.3 (iv)-(v)), n_lines x slots
struct PeakEntries {
  double *u, *c, *s, *shift, *alpha;
  double *tE;    // mode 2 only (else null)
  double *keep;  // 1 in use, 0 not
};
cudaError_t launch_peak_entries(int n_lines, const double *lu,
                                const double *lc, const double *ls,
                                const double *lsh, const double *la,
                                const int *count, const double *pos, int P,
                                int mode, int need, double tp0, double tp1,
                                const PeakEntries &E, cudaStream_t st);
// critical points of the binary lens (s, q): z[k][4] for psi_k = 2 pi k/n
// (unordered within k), as (re, im) pairs, and their caustic points zeta
cudaError_t launch_critical(double s, double q, int n_psi, double2 *z,
                            double2 *zeta, cudaStream_t st);
// slab[iu n_alpha + ia] = tau interval of line (u0v[iu], alpha_ia) inside
// the map of half-width L
cudaError_t launch_slab(const double *u0v, const double *ca, const double *sa,
                        int n_u0, int n_alpha, double L, double2 *slab,
                        cudaStream_t st);
// ---------------------------------------------------------------- batch
// One light curve of a batch, as the batched search reads it.
struct BatchEvent {
  const float4 *ep;         // time-sorted epochs (device)
  int n_ep;
  double S1, SF, SFF, Fref, invS1, CFF, gamma;
  const double *t0rel;      // [n_t0] grid t0 - t_ref of this event
};

// A unit of work: warp groups [g0, g0 + ng) of one (event, map) pair, run
// by one block, whose top-K goes to partial list `list`.
struct BatchUnit {
  int pair;                 // event * n_maps + map
  int list;
  int g0, ng;
  int tpg;                  // trajectories per warp group
  int stage;                // 1: the event's epochs are staged in shared
                            // memory, 0: read from global memory
};

struct BatchParams {
  SearchParams S;           // map geometry, grid tables, top_k, pass mode
                            // (strided sample or line-aligned), err/stats
  const BatchEvent *ev;     // [n_ev]
  const void *const *tab;   // [n_maps] lookup tables (float4 or uint2 quads)
  int n_maps;
  const BatchUnit *units;   // [n_units] in processing order
  int n_units;
  unsigned *counter;        // next unit (zero before the launch)
  unsigned long long *gthr; // [pairs] pruning thresholds (chi^2 bits)
  const int *list0;         // [pairs + 1] first list of each pair (this
                            // pass); S.pub: kPubLevels rows of n_lists
  int n_lists;
  Entry *partial;           // [lists][top_k]
  int ep_cap;               // staged-epoch capacity of shared memory
};

size_t batch_smem_bytes(int ep_cap, int top_k);
// variant 1: the copy of the kernel for the launch of unstaged light
// curves (its own shared-memory carveout)
int batch_blocks_per_sm(bool h16, size_t smem, int variant = 0);
cudaError_t launch_batch(const BatchParams &B, bool h16, int grid,
                         size_t smem, cudaStream_t st, int variant = 0);
// per pair: merge lists [list0[p], list0[p+1]) of a and b (ping-pong) into
// result[p]; with gthr set, also lower gthr[p] to the merged K-th chi^2
cudaError_t launch_batch_merge(Entry *a, Entry *b, const int *list0,
                               int pairs, int k, Entry *result,
                               unsigned long long *gthr, cudaStream_t st);
// records of result[pairs][k] into out[pairs][k]
cudaError_t launch_batch_fill(const BatchParams &B, bool h16,
                              const Entry *result, int pairs,
                              const double *t0abs, const double *tEv,
                              morse_fit *out, cudaStream_t st);

// ---------------------------------------------------------------- probes
cudaError_t probe_fma32(int blocks, int n, float *sink, cudaStream_t st);
cudaError_t probe_fma64(int blocks, int n, double *sink, cudaStream_t st);
cudaError_t probe_smem_atomic(int blocks, int n, unsigned *sink,
                              cudaStream_t st);
cudaError_t probe_gather(const float4 *win, unsigned mask, int blocks, int n,
                         float *sink, cudaStream_t st);
int probe_threads();
int probe_chains();

// ---------------------------------------------------------------- refine
struct RefineState {
  double *th_cur, *th_best;        // [4 n] (t0, tE, u0, alpha)
  double *chi2_cur, *chi2_best;    // [n]
  double *lam;                     // [n] damping
  double *g_cur, *g_best;          // [4 n]
  double *H_cur, *H_best;          // [10 n] upper triangles
  double *Fs, *Fb;                 // [n]
  int *flags;                      // [n]
};

// once per device (morse_create): shared-memory limits of the adjoint
cudaError_t adjoint_setup();
// chi^2 (and gradient, Gauss-Newton matrix) of n trajectories on the map
// P.quad, or with tq set on the map tq[i] of trajectory i (one geometry)
cudaError_t launch_theta(const SearchParams &P, const double *theta, int n,
                         double t_ref, double *chi2, double *grad, double *H,
                         double *Fs, double *Fb, int *flags, cudaStream_t st,
                         const float4 *const *tq = nullptr);
cudaError_t launch_lm_init(const RefineState &S, const morse_fit *starts,
                           int n, double lam0, cudaStream_t st);
cudaError_t launch_lm_step(const RefineState &S, int n, cudaStream_t st);
cudaError_t launch_lm_finish(const RefineState &S, const morse_fit *starts,
                             int n, morse_fit *out, cudaStream_t st);

cudaError_t launch_lightcurve(const SearchParams &P, float ax, float bx,
                              float ay, float by, float kt, float bt,
                              float u02, const float *t, int n, float *A,
                              cudaStream_t st);

}  // namespace morse
