/*
 * morse.h -- C ABI of the GB300 (sm_103a) MORSE hot path.
 *
 * The method is McDougall & Albrow, "Microlensing Observations Rapid Search
 * for Exoplanets: MORSE code for GPUs" (MNRAS 2015): for each binary-lens
 * (s, q) a source-plane magnification map is built (§4.1), and a grid of
 * straight source trajectories is searched through it (§4.2), each data
 * point's magnification read from the map by bilinear interpolation, the
 * flux F = Fs A + Fb fitted linearly (Eq. 5-6) and chi^2 summed over the
 * data points; the best trajectories seed the refinement (§4.4, §5).
 *
 * Conventions shared by every call:
 *  - Units: angles on the sky in Einstein radii; times in days.
 *  - Lens: masses on the first axis, origin at the centre of mass (§4.1).
 *    q = m2/m1; eps1 = 1/(1+q), eps2 = q/(1+q); primary at -s*eps2,
 *    secondary at +s*eps1.
 *  - Trajectory (§4.1 parameters u0, phi = alpha, t0, tE): at time t the
 *    source is at tau = (t - t0)/tE,
 *        y1 = tau cos(alpha) - u0 sin(alpha),
 *        y2 = tau sin(alpha) + u0 cos(alpha).
 *  - Map: npix x npix texels over [-L, L)^2 (L = "extent"), row-major with
 *    the second coordinate major: A[iy*npix + ix]; texel (ix, iy) is centred
 *    at (-L + (ix+1/2) Delta, -L + (iy+1/2) Delta), Delta = 2L/npix.  A
 *    texel holds the magnification averaged over its area (ray count times
 *    h^2/Delta^2, h the image-plane ray spacing).
 *  - Lookup: bilinear between texel centres, coordinates clamped to the
 *    outermost centres; outside the map (|y1| >= L or |y2| >= L) the
 *    single-lens magnification A(u) = (u^2+2)/(u sqrt(u^2+4)), u = |y|.
 *  - Errors: every call returns a morse_status; morse_last_error() gives a
 *    message for the context's most recent failure.  No call aborts, traps
 *    or throws.  Invalid arguments return MORSE_EINVAL before any GPU work.
 *  - Memory: handles own their device memory; input arrays are copied and
 *    stay owned by the caller; output arrays are caller-allocated HOST
 *    memory unless the name ends in _dev.  Calls are synchronous on the
 *    context's stream unless noted.
 *  - Threads: a context may be used by one host thread at a time.
 */
#ifndef MORSE_H
#define MORSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MORSE_OK = 0,
  MORSE_EINVAL = 1,       /* bad argument (NaN, sigma <= 0, sizes ...)   */
  MORSE_ENOMEM = 2,       /* device or host allocation failed            */
  MORSE_ECUDA = 3,        /* a CUDA runtime call or launch failed        */
  MORSE_ETIMEOUT = 4,     /* a bounded device loop gave up               */
  MORSE_EDEGENERATE = 5,  /* linear system singular where not allowed    */
  MORSE_EUNSUPPORTED = 6  /* valid request this build does not handle    */
} morse_status;

typedef struct morse_ctx morse_ctx;     /* device, stream, workspaces     */
typedef struct morse_map morse_map;     /* one (s, q) magnification map   */
typedef struct morse_event morse_event; /* one light curve on the device  */

/* Human-readable name of a status code (static string). */
const char *morse_status_string(morse_status st);

/* Library version string, e.g. "morse-gb300 0.1 sm_103a". */
const char *morse_version(void);

/* Create a context on CUDA device `device`.  cuda_stream is a cudaStream_t
 * cast to void* on which all work is queued; NULL creates a private
 * stream.  The context does not own a caller-provided stream. */
morse_status morse_create(morse_ctx **out, int device, void *cuda_stream);
void morse_destroy(morse_ctx *ctx);
const char *morse_last_error(const morse_ctx *ctx);

/* ------------------------------------------------------------------ */
/* Magnification maps (§3 ray-shooting maps, §4.1)                      */
/* ------------------------------------------------------------------ */

enum {
  MORSE_DEFLECT_FP64 = 0, /* FP64 deflection, IEEE division, no FMA
                             contraction: counts equal those of the plain
                             FP64 definition ray for ray                  */
  MORSE_DEFLECT_FP32 = 1  /* FP32 deflection (fast path)                  */
};
enum {
  MORSE_STORE_FP32 = 1,    /* FP32 A (always kept)                        */
  MORSE_STORE_FP16LOG = 2  /* plus FP16 log10(max(A, A_floor)) texels,
                              which searches then read                    */
};

enum {
  MORSE_GEN_RAYS = 0, /* inverse ray shooting: texel = area-averaged A    */
  MORSE_GEN_POLY = 1  /* the lens polynomial per texel (§4.1): texel = the
                         point-source A at its centre, FP64; no counts     */
};

typedef struct {
  double image_halfwidth; /* X: rays cover [-X, X]^2; <= 0 means 1.5 L    */
  int deflect;            /* MORSE_DEFLECT_FP64 or MORSE_DEFLECT_FP32     */
  int store;              /* OR of MORSE_STORE_* (FP32 is always kept)     */
  int generator;          /* MORSE_GEN_RAYS (default) or MORSE_GEN_POLY   */
} morse_map_opts;

/* Build the magnification map of the binary lens (s, q) by inverse ray
 * shooting (§3 ray-shooting maps; §5 inverse ray shooting) on the source
 * grid of §4.1, or, with opts->generator = MORSE_GEN_POLY, by solving the
 * fifth-order lens polynomial at every texel centre (§4.1; one thread per
 * texel, FP64 roots polished on Eq. 2, images by Eq. 2 residual; such a map
 * has no ray counts and ignores rays_per_axis, image_halfwidth and
 * deflect).  rays_per_axis^2 image-plane rays on the cell-centred grid
 * x = -X + (i+1/2) h, h = 2X/rays_per_axis, are deflected through the real
 * form of Eq. 2,
 *     y = x - eps1 (x - x1)/|x - x1|^2 - eps2 (x - x2)/|x - x2|^2,
 * and counted in half-open source bins [-L, L)^2; rays leaving the map are
 * counted as off-map, rays exactly on a lens as lost.
 * Arguments: s > 0, q > 0 finite; extent L > 0; 2 <= npix <= 16384;
 * 1 <= rays_per_axis <= 2^31 - 1; opts may be NULL (X = 1.5 L, FP64,
 * FP32 store).  *out receives a new map owned by the caller
 * (morse_map_free).  Errors: EINVAL, ENOMEM, ECUDA. */
morse_status morse_build_map(morse_ctx *ctx, double s, double q,
                             double extent, int npix, int64_t rays_per_axis,
                             const morse_map_opts *opts, morse_map **out);

/* Wrap a caller-supplied FP32 map (npix x npix, layout as above, values
 * copied) so that it can be searched.  A must be finite and >= 0.  The map
 * has no counts.  Errors: EINVAL, ENOMEM, ECUDA. */
morse_status morse_map_from_host(morse_ctx *ctx, const float *A, int npix,
                                 double extent, morse_map **out);

/* Copy the ray counts (npix*npix uint32, host) and the off-map and lost
 * ray totals of a ray-shot map.  Any output pointer may be NULL.
 * Errors: EINVAL (map has no counts), ECUDA. */
morse_status morse_map_counts(const morse_map *map, uint32_t *host_counts,
                              uint64_t *off_map, uint64_t *lost);

/* Copy the FP32 magnifications (npix*npix floats, host). */
morse_status morse_map_values(const morse_map *map, float *host_A);

/* Map geometry.  Any output pointer may be NULL. */
morse_status morse_map_info(const morse_map *map, int *npix, double *extent,
                            double *s, double *q);
void morse_map_free(morse_map *map);

/* Finite-source map (§4.1: maps convolved with radially symmetric,
 * limb-darkened source profiles of fixed radii).  A new map whose texel
 * (i, j) is sum W(dx, dy) A(i + dx, j + dy) over |dx|, |dy| <= R =
 * ceil(rho/Delta + 1/2): W is the surface brightness of a source of radius
 * rho (Einstein radii) with linear limb darkening,
 *     I(r) = 1 - gamma (1 - 3/2 sqrt(1 - r^2/rho^2)),
 * integrated over each texel (8 x 8 midpoint points) and normalised, and a
 * texel outside the map takes the Paczynski magnification of its centre
 * (the lookup's outside rule).  The paper uses gamma = 0.53 and seven rho
 * log-spaced in (0.001, 1).  A source smaller than a texel leaves the map
 * unchanged.  The new map has the source map's geometry, FP32 values and
 * no ray counts; it is owned by the caller (morse_map_free).
 * Arguments: rho > 0 with R <= 1600 texels, 0 <= gamma <= 1.
 * Errors: EINVAL, ENOMEM, ECUDA. */
morse_status morse_map_finite_source(morse_ctx *ctx, const morse_map *src,
                                     double rho, double gamma,
                                     morse_map **out);

/* FP16 storage form.  Next to the FP32 values a map can hold the table
 * x = half(log10(max(A, A_floor))) per texel (IEEE binary16, round to
 * nearest even; A_floor = half a ray, 0.5 h^2/Delta^2, for ray-shot maps
 * and 1e-6 for maps from host values), packed as 2x2 neighbourhoods of
 * 8 bytes per texel instead of 16.  A search through it decodes the four
 * texels around each position to A = 10^x in FP32 and interpolates
 * bilinearly in A, as on the FP32 map; sums and the solve are unchanged.
 * The paper stores maps in single precision; this is a storage option of
 * the GPU design, its error is the half quantisation of log10 A (relative
 * error of A at most ln(10) 2^-11 |log10 A|).
 *
 * morse_map_set_lookup selects the table that morse_grid_chi2,
 * morse_grid_chi2_dense, morse_grid_chi2_noalloc and morse_lightcurve read:
 * MORSE_STORE_FP32 or MORSE_STORE_FP16LOG (computing the FP16 table from
 * the current FP32 values if the map has none).  morse_build_map with
 * opts->store including MORSE_STORE_FP16LOG builds both and selects FP16;
 * morse_sweep and morse_search_sweep then search every map through its
 * FP16 table.  The gradient and refine calls always read the FP32 values.
 * Errors: EINVAL (unknown store value), ENOMEM, ECUDA. */
morse_status morse_map_set_lookup(morse_map *map, int store);

/* Copy the FP16 table (npix*npix uint16 codes, host, row-major like A) and
 * A_floor.  Either pointer may be NULL.  Errors: EINVAL (no FP16 table). */
morse_status morse_map_half(const morse_map *map, uint16_t *host_codes,
                            double *a_floor);

/* ------------------------------------------------------------------ */
/* Light curves (§4.1 Eq. 5)                                            */
/* ------------------------------------------------------------------ */

/* Copy a light curve to the device: n epochs with times t (days), fluxes
 * and 1-sigma errors (w = 1/sigma^2), in any order (stored sorted by time,
 * which the search relies on).  Times are stored as FP32 offsets
 * t - t_ref, computed in FP64 on the host, so t_ref should lie within the
 * data (resolution ~4e-6 d for offsets up to 40 d; real data in HJD go
 * through the same path); grid t0 values are absolute times in the same
 * frame as t.  Requires n >= 3, every value finite, sigma > 0, and
 * |t - t_ref| <= 1e5 d for every epoch (FP32 offsets resolve 0.004 d there).
 * Errors: EINVAL, ENOMEM, ECUDA. */
morse_status morse_event_create(morse_ctx *ctx, const double *t,
                                const double *flux, const double *sigma,
                                int64_t n, double t_ref, morse_event **out);
void morse_event_free(morse_event *ev);
morse_status morse_event_info(const morse_event *ev, int64_t *n,
                              double *t_ref);

/* ------------------------------------------------------------------ */
/* Trajectory grid search (§4.2 chi^2 over data points; §4.4 seeds)      */
/* ------------------------------------------------------------------ */

/* The grid: u0 (log or linear in [u0_lo, u0_hi]), alpha_k = 2 pi k /
 * n_alpha, t0 linear in [t0_lo, t0_hi], tE (log or linear in [tE_lo,
 * tE_hi]); an axis with n = 1 takes its lo value.  Trajectory index
 *     idx = ((i_u0 * n_alpha + i_alpha) * n_t0 + i_t0) * n_tE + i_tE.
 * top_k: number of best trajectories kept (1 <= top_k <= 4096). */
typedef struct {
  int n_u0, n_alpha, n_t0, n_tE;
  double u0_lo, u0_hi, t0_lo, t0_hi, tE_lo, tE_hi;
  int u0_log, tE_log;
  int top_k;
  /* minimum-magnification cut (§4.3 (i)); 0: off.  Trajectories whose
   * (u0, alpha) line never reaches a_min (the largest magnification on the
   * whole line: the map's bilinear lookup inside, Paczynski outside; see
   * morse_line_max) cannot fit a light curve that needs a_min and are not
   * searched: top-K results are those of the other trajectories, dense
   * results give them chi2 = +inf and Fs = Fb = 0.  Supported by
   * morse_grid_chi2, morse_grid_chi2_dense, morse_sweep and
   * morse_search_sweep; the batched and allocation-free searches return
   * EUNSUPPORTED for a_min > 0. */
  float a_min;
} morse_grid;

/* Largest magnification on each (u0, alpha) line of the grid (§4.3 (i)):
 * out[i_u0 * n_alpha + i_alpha] (host, n_u0 * n_alpha doubles) = the
 * maximum over the whole straight line of the map's bilinear lookup inside
 * the map (exactly: the lookup is quadratic between texel-centre
 * crossings) and of the Paczynski curve outside it.
 * Errors: EINVAL, ENOMEM, ECUDA. */
morse_status morse_line_max(morse_ctx *ctx, const morse_map *map,
                            const morse_grid *grid, double *out);

/* Caustics of the binary lens (s, q) (§4.2: trajectory grids about the
 * central regions of the caustics, scaled by their sizes).  The critical
 * points solve, for psi_k = 2 pi k / n_psi, the quartic in w = conj(z)
 *     eps1 (w - x2)^2 + eps2 (w - x1)^2 = exp(-i psi) (w - x1)^2 (w - x2)^2
 * (det J = 0, Eq. 4), on the device; their images by Eq. 2 are the caustic
 * points.  The four branches are followed across psi by the pairing of
 * least total distance and a full turn's permutation groups them into
 * closed critical curves, one caustic each (1, 2 or 3 by topology).  A
 * caustic's centre is the mean of its points and its size the largest
 * distance from the centre to one of them.  out receives up to 3 records,
 * sorted by (c1, c2); *n_out their number.  Arguments: s, q > 0,
 * 16 <= n_psi <= 1 << 20.  Errors: EINVAL, ENOMEM, ECUDA. */
typedef struct {
  double c1, c2;    /* centre (Einstein radii, centre-of-mass origin)     */
  double size;      /* largest distance from the centre to the caustic    */
  int32_t n_points; /* caustic points of the caustic                      */
  int32_t reserved;
} morse_caustic;
morse_status morse_caustics(morse_ctx *ctx, double s, double q, int n_psi,
                            morse_caustic out[3], int *n_out);

/* The lines of an (r, phi) grid about caustics: for caustic c (centre C,
 * size R), impact r = (r_lo + (r_hi - r_lo) i / (n_r - 1)) R from C
 * (i < n_r), direction phi_k = 2 pi k / n_phi, in the order (c, i, k).
 * lines[3 j + 0 .. 2] = (u, alpha, shift): the same line about the origin
 * has impact u = r + C.n and direction alpha = phi, and its closest
 * approach to C comes tau = shift = C.d after its closest approach to the
 * origin (d = (cos phi, sin phi), n = (-sin phi, cos phi)).  Host only.
 * Errors: EINVAL. */
morse_status morse_rphi_lines(const morse_caustic *caustics, int n_caustics,
                              int n_r, double r_lo, double r_hi, int n_phi,
                              double *lines);

enum {
  MORSE_FIT_DEGENERATE = 1, /* A constant along the track: Fs = 0          */
  MORSE_FIT_REFINED = 2     /* parameters from morse_refine, off the grid   */
};

/* One fitted trajectory.  chi2 = sum_i w_i (F_i - Fs A_i - Fb)^2 with
 * (Fs, Fb) the weighted least-squares solution of Eq. 6. */
typedef struct {
  double chi2, t0, tE, u0, alpha, Fs, Fb;
  int64_t idx;
  int32_t flags;
  int32_t reserved;
} morse_fit;

/* Search every trajectory of the grid through the map and return the
 * top_k smallest chi^2, ordered by (chi2, idx) ascending, in out[top_k]
 * (host).  If the grid has fewer than top_k trajectories the tail has
 * idx = -1 and chi2 = +inf.  Each trajectory's Fs, Fb come from the
 * closed-form 2x2 solve of the normal equations (Eq. 6) and its chi^2 from
 * the per-point residuals (§4.2).  Errors: EINVAL, ENOMEM, ECUDA. */
morse_status morse_grid_chi2(morse_ctx *ctx, const morse_event *ev,
                             const morse_map *map, const morse_grid *grid,
                             morse_fit *out);

/* morse_grid_chi2 restricted to the trajectories with index in
 * [first, first + count): the top_k smallest chi^2 among them, ordered by
 * (chi2, idx), idx the index in the whole grid (tail idx = -1, chi2 = +inf
 * if the range has fewer than top_k).  Each trajectory's chi^2 does not
 * depend on the range, so the top-K lists of ranges that partition the grid,
 * merged by morse_topk_merge, equal the whole grid's list bit for bit: the
 * shard of one map's search that a GPU (or a call) takes when the grid is
 * split across several.  Errors: EINVAL (range outside the grid), ENOMEM,
 * ECUDA, ETIMEOUT. */
morse_status morse_grid_chi2_range(morse_ctx *ctx, const morse_event *ev,
                                   const morse_map *map,
                                   const morse_grid *grid, int64_t first,
                                   int64_t count, morse_fit *out);

/* morse_grid_chi2 over a grid of arbitrary lines: trajectory
 * (j, i_t0, i_tE), index (j n_t0 + i_t0) n_tE + i_tE, follows line j of
 * lines[3 j .. 3 j + 2] = (u, alpha, shift) (morse_rphi_lines) with t0 the
 * time of its closest approach to the line's reference point, i.e. the
 * (u0, alpha, t0, tE) trajectory (u, alpha, t0 - shift tE, tE).  grid gives
 * n_u0 = the number of lines, n_alpha = 1, the t0 and tE axes and top_k
 * (its u0 range is not used).  The records are in the (u0, alpha, t0, tE)
 * convention of morse_grid_chi2, so they seed morse_refine directly.
 * Errors: EINVAL (n_alpha != 1, non-finite lines), EUNSUPPORTED
 * (a_min > 0), ENOMEM, ECUDA, ETIMEOUT. */
morse_status morse_grid_chi2_lines(morse_ctx *ctx, const morse_event *ev,
                                   const morse_map *map,
                                   const morse_grid *grid,
                                   const double *lines, morse_fit *out);

/* Peak library (§4.3 (iii)): the peaks of the map along each line, a peak
 * being where the magnification turns from rising to falling.
 * lines[3 j .. 3 j + 2] = (u, alpha, shift) as in morse_grid_chi2_lines
 * (a (u0, alpha) grid line has shift 0).  The profile: samples every
 * h = Delta / sub along the part of the line inside the map, tau_k = k h
 * from the closest approach to the origin, each the bilinear lookup
 * between texel centres (clamped to the outermost centres) in FP32.  With
 * r = 1 + delta, a rise counts once a value exceeds r times the lowest
 * value since the last peak, and the highest value after it is a peak once
 * a later value is below it by the factor r (delta = 0: every turn; on a
 * ray-shot map that includes the Poisson noise, which delta > 0 ignores).
 * The profile's first sample is never a peak.
 * Outputs (host): count[j] = the number of peaks; pos[j max_peaks + m] and
 * height[...] = the max_peaks highest peaks (ties: the earlier) in
 * increasing tau, as (tau_k - shift, value); NaN in unused slots.
 * Errors: EINVAL (sub outside 1..16, max_peaks outside 1..16, delta < 0,
 * non-finite lines), ENOMEM, ECUDA. */
typedef struct {
  int sub;        /* samples per texel width along the line (2)           */
  int max_peaks;  /* peaks kept per line, the highest (8)                  */
  double delta;   /* relative threshold of a rise or fall, >= 0           */
} morse_peak_opts;
morse_status morse_line_peaks(morse_ctx *ctx, const morse_map *map,
                              const double *lines, int n_lines,
                              const morse_peak_opts *opts, int32_t *count,
                              double *pos, double *height);

/* morse_line_peaks of the same lines on n_maps maps of one geometry in one
 * launch (the libraries of a whole (s, q) grid: enough lines to fill the
 * GPU, where one map's few thousand lines leave it latency-bound).  Map m's
 * results are those morse_line_peaks gives for it, bit for bit, at
 * count[m n_lines + j], pos[(m n_lines + j) max_peaks + k] and height[...].
 * Errors: EINVAL (as morse_line_peaks; maps of another npix or extent),
 * ENOMEM, ECUDA. */
morse_status morse_line_peaks_batch(morse_ctx *ctx,
                                    const morse_map *const *maps, int n_maps,
                                    const double *lines, int n_lines,
                                    const morse_peak_opts *opts,
                                    int32_t *count, double *pos,
                                    double *height);

/* Search of the trajectories the peak library allows (§4.3 (iii)-(v)).
 * Lines with fewer than max(min_peaks, n_tp) peaks are not searched.
 *  n_tp = 0: the line grid of morse_grid_chi2_lines over lines[n_lines];
 *  n_tp = 1: for each kept peak m of each line (tau_m from the origin's
 *    closest approach), the trajectories whose peak m comes at t_p + dt0:
 *    t0 = t_p + dt0 - tau_m tE (Eq. 7), dt0 on the grid's t0 axis (an
 *    offset: n_t0 = 1, t0_lo = 0 gives Eq. 7 itself), tE on its tE axis;
 *  n_tp = 2 (t_p1 < t_p2): for each pair of kept peaks a < b, tE =
 *    (t_p2 - t_p1) / (tau_b - tau_a) (Eq. 8) and peak a at t_p1 + dt0; the
 *    grid must have n_tE = 1 (its tE values are not used).
 * Index of a trajectory: ((j S + slot) n_t0 + i_t0) n_tE + i_tE, S = 1,
 * max_peaks or max_peaks (max_peaks - 1) / 2 slots per line (slot m, or
 * the pairs (a, b) in the order (0,1), (0,2) .. (1,2) ..); slots a line
 * does not use are skipped like cut lines.  grid: n_alpha = 1, the t0 and
 * tE axes and top_k are used (n_u0, the u0 range and a_min are not).
 * Records (top_k, host) are in the (u0, alpha, t0, tE) convention.
 * Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT. */
morse_status morse_peak_search(morse_ctx *ctx, const morse_event *ev,
                               const morse_map *map, const morse_grid *grid,
                               const double *lines, int n_lines,
                               const morse_peak_opts *opts, int min_peaks,
                               const double *tp, int n_tp, morse_fit *out);

/* morse_grid_chi2 without any device allocation.  The paper has no
 * counterpart: this is a deployment variant of the same search.
 *
 * For callers that must not let the library call cudaMalloc or cudaFree
 * once set-up is over: cudaFree waits for the whole device and so stalls
 * every other stream of a latency-bound pipeline, and some applications run
 * under a fixed memory budget reserved at start-up, where a workspace that
 * grows on demand is not acceptable.  Such callers create the context,
 * event and map at set-up and then call this function, which keeps its
 * scratch (grid tables, per-block top-K lists, fit records) in one static
 * device array of 4 MiB that every GPU loading the library holds until the
 * process exits, instead of the context's growable workspace.  Inputs,
 * output and results are exactly those of morse_grid_chi2 (same kernels,
 * same arithmetic, same parameter set-up); out is caller-allocated host
 * memory of top_k records.  Like morse_grid_chi2 the call is synchronous:
 * it returns once the records are on the host.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and keeps it for the
 * life of the process, so the library must not be used across a
 * cudaDeviceReset of that device.  Every call in the process shares the
 * array: calls that overlap on the same GPU (other streams, other host
 * threads) race on it; each call rewrites every byte it reads, so nothing
 * carries over.  Returns
 * MORSE_EINVAL, with a message naming the sizes, when the search needs
 * more than 4 MiB of scratch (top_k above about 850 on a 152-SM GPU) or
 * more than 4096 grid-table values (n_u0 + 2 n_alpha + 2 n_t0 + 2 n_tE).
 * Errors otherwise as morse_grid_chi2. */
morse_status morse_grid_chi2_noalloc(morse_ctx *ctx, const morse_event *ev,
                                     const morse_map *map,
                                     const morse_grid *grid, morse_fit *out);

/* Batched search: n_ev light curves (any lengths) against n_maps maps,
 * every (event, map) pair searched over the same grid, in one persistent
 * kernel launch.  The pair (e, m) gets the top_k fits of
 * morse_grid_chi2(ev[e], maps[m], grid), bit for bit, in
 * out[(e * n_maps + m) * top_k + r] (host, caller-allocated).  The maps
 * must share npix, extent and lookup table (FP32 or FP16); grid t0 values
 * are absolute times, each event's relative to its own t_ref.  The whole
 * sequence (a strided pilot pass per pair that seeds the pair's pruning
 * threshold, the main pass, the per-pair merges and the record fill) is
 * captured in a CUDA graph, which later calls of the same shape update and
 * replay.  Launch shapes per epoch-count bucket (trajectories per warp
 * group, groups per work unit, shared-memory staging of the epochs) come
 * from the autotuner (morse_batch_tuning) or from the default rule.
 * Errors: EINVAL (mismatched maps, foreign handles, n_ev or n_maps < 1,
 * more than 2^31 partial lists), ENOMEM, ECUDA, ETIMEOUT. */
morse_status morse_grid_chi2_batch(morse_ctx *ctx,
                                   const morse_event *const *ev, int n_ev,
                                   const morse_map *const *maps, int n_maps,
                                   const morse_grid *grid, morse_fit *out);

/* Launch shape of the batched search for light curves of one epoch-count
 * bucket (2^b <= n_ep < 2^(b+1)). */
typedef struct {
  int tpg;             /* trajectories per warp group (8, 16 or 32)        */
  int rounds;          /* warp groups per warp in one work unit             */
  int stage;           /* 1: epochs staged in shared memory                 */
  int tuned;           /* 1: picked by timing candidates, 0: default rule   */
  double ns_per_eval;  /* tuned: time per trajectory-epoch of the winner    */
} morse_batch_shape;

enum {
  MORSE_TUNE_OFF = 0, /* default rule (no timing runs)                     */
  MORSE_TUNE_ON = 1   /* time the candidate shapes of each new bucket once
                         per context on a sample of the batch (default)    */
};

/* Select the autotuner mode and forget the shapes tuned so far. */
morse_status morse_batch_tuning(morse_ctx *ctx, int mode);

/* The shape used for light curves of n_ep epochs with this grid and map
 * geometry, if a batch call has chosen one (else EINVAL). */
morse_status morse_batch_shape_of(morse_ctx *ctx, int64_t n_ep,
                                  const morse_grid *grid,
                                  const morse_map *map,
                                  morse_batch_shape *out);

/* chi^2, Fs and Fb of every trajectory with index in [first, first+count)
 * (host arrays of count doubles; Fs/Fb may be NULL).  Same arithmetic as
 * morse_grid_chi2.  Errors: EINVAL, ENOMEM, ECUDA. */
morse_status morse_grid_chi2_dense(morse_ctx *ctx, const morse_event *ev,
                                   const morse_map *map,
                                   const morse_grid *grid, int64_t first,
                                   int64_t count, double *chi2, double *Fs,
                                   double *Fb);

/* End-to-end search from host buffers: copies the light curve in, builds
 * the (s, q) map, searches the grid and returns the top_k fits to out
 * (host), freeing everything it made.  Equivalent to morse_event_create +
 * morse_build_map + morse_grid_chi2 + frees.  Errors as those calls. */
morse_status morse_search(morse_ctx *ctx, const double *t, const double *flux,
                          const double *sigma, int64_t n, double t_ref,
                          double s, double q, double extent, int npix,
                          int64_t rays_per_axis, const morse_map_opts *opts,
                          const morse_grid *grid, morse_fit *out);

/* The full (s, q) search of one light curve (§4.1: a grid of maps in
 * (log d, log q), each searched over trajectories, §4.2): for each of the
 * n_maps lenses (s[i], q[i]) build the map (as morse_build_map, same
 * extent, npix, rays and opts for all) and search the grid (as
 * morse_grid_chi2).  out (host) receives n_maps * top_k fits, map i's list
 * at out[i*top_k].  The event stays on the device; maps are built one at a
 * time into storage the context reuses, so memory does not grow with
 * n_maps.  Errors: EINVAL, ENOMEM, ECUDA. */
morse_status morse_sweep(morse_ctx *ctx, const morse_event *ev,
                         const double *s, const double *q, int n_maps,
                         double extent, int npix, int64_t rays_per_axis,
                         const morse_map_opts *opts, const morse_grid *grid,
                         morse_fit *out);

/* morse_sweep from host buffers: copies the light curve to the device
 * (as morse_event_create), runs the sweep and frees the event.  This is the
 * end-to-end call of the plain method.  Errors as the calls it combines. */
morse_status morse_search_sweep(morse_ctx *ctx, const double *t,
                                const double *flux, const double *sigma,
                                int64_t n, double t_ref, const double *s,
                                const double *q, int n_maps, double extent,
                                int npix, int64_t rays_per_axis,
                                const morse_map_opts *opts,
                                const morse_grid *grid, morse_fit *out);

/* Map magnification A(t_i) along one trajectory at n host times t (same
 * lookup as the search), written to A_out (host, n doubles).
 * Errors: EINVAL, ENOMEM, ECUDA. */
morse_status morse_lightcurve(morse_ctx *ctx, const morse_map *map,
                              double t0, double tE, double u0, double alpha,
                              const double *t, int64_t n, double *A_out);

/* ------------------------------------------------------------------ */
/* Gradient and refinement of trajectories (seeds of §4.4 refined as §5  */
/* does, here on the same point-source map)                             */
/* ------------------------------------------------------------------ */

/* chi^2 of n trajectories theta[4 i + (0..3)] = (t0, tE, u0, alpha) (t0
 * absolute, tE > 0) on the map, with (Fs, Fb) profiled out by the 2x2 solve
 * of Eq. 6, and its gradient with respect to theta.  Because (Fs, Fb)
 * minimise chi^2 at every theta, d chi^2/d theta_k = sum_i -2 w_i r_i Fs
 * dA_i/d theta_k, with dA/d theta through the bilinear lookup (inside the
 * map) or the single-lens formula (outside).  The bilinear gradient is
 * piecewise: it jumps where a data point crosses a texel edge.  Host
 * arrays: chi2[n]; grad[4 n], Fs[n], Fb[n] may be NULL.
 * Errors: EINVAL (n < 0, non-finite theta, tE <= 0), ENOMEM, ECUDA. */
morse_status morse_chi2_grad(morse_ctx *ctx, const morse_event *ev,
                             const morse_map *map, const double *theta,
                             int64_t n, double *chi2, double *grad,
                             double *Fs, double *Fb);

/* morse_chi2_grad on DEVICE arrays (theta [4 n], chi2 [n], grad [4 n] or
 * NULL), queued on the context stream without host synchronisation (for
 * autograd and other device-side drivers).  theta is not validated on the
 * host: tE is floored at 1e-6 in the kernel.  Errors: EINVAL, ECUDA. */
morse_status morse_chi2_grad_dev(morse_ctx *ctx, const morse_event *ev,
                                 const morse_map *map, const double *theta,
                                 int64_t n, double *chi2, double *grad);

enum { MORSE_REFINE_LM = 0 };

/* Refine n starting trajectories (e.g. grid top-K records) by batched
 * Levenberg-Marquardt on chi^2(theta): each iteration evaluates chi^2, its
 * gradient and the Gauss-Newton matrix sum w Fs^2 dA/dtheta dA/dtheta^T,
 * accepts the point if chi^2 fell, and steps by (H + lam diag H)^-1 g.
 * One iteration is captured as a CUDA graph and replayed iters times.
 * out[n] (host) receives the best point of each, its chi^2, Fs, Fb, the
 * start's idx and MORSE_FIT_REFINED.  chi^2 never increases from the start.
 * method: MORSE_REFINE_LM.  Errors: EINVAL, EUNSUPPORTED, ENOMEM, ECUDA. */
morse_status morse_refine(morse_ctx *ctx, const morse_event *ev,
                          const morse_map *map, const morse_fit *starts,
                          int n, int iters, int method, morse_fit *out);

/* morse_refine of starts on several maps in one call: start i is refined
 * on maps[map_of[i]] (0 <= map_of[i] < n_maps), every start in the same
 * batched launches and the same CUDA graph, so that the grid minima of a
 * whole (s, q) sweep (config 2: the K best over all maps) refine together
 * with every map they need resident on the device.  The maps must share
 * npix and extent; each start's result is the one morse_refine gives on its
 * own map, bit for bit.  Errors: EINVAL (mismatched maps, map index out of
 * range), EUNSUPPORTED, ENOMEM, ECUDA. */
morse_status morse_refine_batch(morse_ctx *ctx, const morse_event *ev,
                                const morse_map *const *maps, int n_maps,
                                const int *map_of, const morse_fit *starts,
                                int n, int iters, int method,
                                morse_fit *out);

/* Merge n_lists top-K lists (each ascending by (chi2, idx), counts[i]
 * entries, entries with idx < 0 ignored) into the k best, ascending, in
 * out[k] (tail padded with idx = -1, chi2 = +inf).  Host-only; used to
 * combine shards of a search run on several GPUs or several calls.
 * Errors: EINVAL. */
morse_status morse_topk_merge(const morse_fit *const *lists,
                              const int *counts, int n_lists, int k,
                              morse_fit *out);

/* Measured throughput of this GPU for the rooflines of the hot path (not
 * part of the paper's method): FP32 and FP64 fused multiply-adds (thread
 * instructions per second, 8 independent chains per thread), shared-memory
 * atomic adds to pseudo-random bins of a 128 x 128 window (the ray-shooting
 * histogram), and 16-byte loads from pseudo-random cells of a 64 KB window
 * (served by L1) and of a 16 MB window (served by L2), in bytes per second.
 * Each probe runs about 10 ms after one warm-up run.  Uses the context's
 * workspace.  Errors: EINVAL, ENOMEM, ECUDA. */
typedef struct {
  double fp32_fma_per_s;
  double fp64_fma_per_s;
  double smem_atomics_per_s;
  double l1_gather_bytes_per_s;
  double l2_gather_bytes_per_s;
} morse_peaks;
morse_status morse_measure_peaks(morse_ctx *ctx, morse_peaks *out);

/* Device time of the kernels of the most recent call on this context, in
 * milliseconds (CUDA events on the context stream), summed over every
 * launch of that kind in the call: which = 0 ray shooting, 1 counts-to-map,
 * 2 grid search, 3 top-K merge, 4 fit fill, 5 adjoint evaluations, 6
 * refine steps, 7 peak-library lines (morse_line_peaks and its batch). */
morse_status morse_last_kernel_ms(const morse_ctx *ctx, int which,
                                  double *ms);

/* Pruning statistics of the most recent search call on this context: the
 * number of trajectories that received the exact residual sweep (the rest
 * were discarded by the error-bounded closed form).  Summed over the maps
 * of a sweep. */
morse_status morse_last_search_stats(const morse_ctx *ctx,
                                     uint64_t *exact_sweeps);

/* Number of CUDA kernels this context has launched since morse_create. */
morse_status morse_launch_count(const morse_ctx *ctx, uint64_t *n);

/* Fault injection for tests of the error paths (not part of the paper's
 * method).  Each fault makes a bounded failure happen on purpose, on the
 * host or as a device wait that gives up; none faults or hangs the GPU, and
 * the context stays usable afterwards.
 *  MORSE_FAULT_NONE: clear every injected fault (arg ignored).
 *  MORSE_FAULT_LOCK_HELD: until cleared, the top-K searches of this context
 *    (morse_grid_chi2 and the calls built on it, the batched and the
 *    allocation-free search) start with every block's top-K lock taken, and
 *    a wait for it gives up after arg spins of ~64 ns (1 <= arg <= 2^20;
 *    the default limit is 2^20): the call returns MORSE_ETIMEOUT.
 *  MORSE_FAULT_ALLOC: the arg-th device allocation from now (arg >= 1)
 *    fails as cudaMalloc would when out of memory, without allocating; the
 *    call that makes it returns MORSE_ENOMEM.  One shot.
 * Errors: EINVAL (unknown fault, arg out of range). */
enum {
  MORSE_FAULT_NONE = 0,
  MORSE_FAULT_LOCK_HELD = 1,
  MORSE_FAULT_ALLOC = 2
};
morse_status morse_inject_fault(morse_ctx *ctx, int fault, int64_t arg);

#ifdef __cplusplus
}
#endif
#endif /* MORSE_H */
