"""Plain FP64 CPU oracle for the MORSE hot path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_1511_01157_gb300``) and neither imports the other.

The arithmetic lives in ``morse_oracle.c`` (plain C, FP64, FMA contraction
off); this module only compiles it and marshals numpy arrays.  Each wrapper
names the passage of McDougall & Albrow (2015) it follows:

* ``lens``            -- §4.1 / §3 Eq. 2 lens geometry (centre-of-mass origin)
* ``rayshoot``        -- §3 / §5 inverse ray shooting into a source-plane map
* ``counts_to_mag``   -- map value = ray count x h^2 / Delta^2
* ``quintic``/``roots5``/``images``/``mag_point`` -- §3 fifth-order lens
  polynomial, 3 or 5 images, A = sum 1/|det J| (Eq. 3-4)
* ``mag_point_grad``  -- Eq. 2, 4 differentiated implicitly: dA/dy
* ``chi2_grad_poly``  -- chi^2 gradient in (t0, tE, u0, alpha) of the
  polynomial light curve, Fs and Fb profiled (Eq. 5-6, §4.2)
* ``poly_map``        -- §4.1 point-source map from the polynomial per texel
* ``fs_weights``/``fs_convolve`` -- §4.1 finite-source maps: the map
  convolved with a limb-darkened source profile
* ``half_bits``/``half_value``/``log10_half``/``half_decode`` -- the FP16
  log10 storage form of a map (IEEE binary16, round to nearest even)
* ``pspl``            -- §4.3 (ii) Paczynski single-lens curve
* ``traj_point``/``map_A`` -- §4.2 straight trajectory, bilinear map lookup
* ``line_max``        -- §4.3 (i) largest magnification along a line
* ``line_peaks``      -- §4.3 (iii) peak library: peaks of the map along a
  line (count, positions, heights)
* ``peak_trajectories`` -- §4.3 (iv)-(v) Eq. 7-8: the trajectories aligned
  with one or two given peak times
* ``fit_A``           -- §4.1 Eq. 5-6 linear flux fit, chi^2 as a sum of
  per-point contributions (§4.2)
* ``grid_chi2``/``topk`` -- brute-force grid and the K best seeds (§4.4)
* ``chi2_theta``      -- chi^2 at an arbitrary trajectory (map or polynomial)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "morse_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``morse_oracle.c`` into ``liborc.so`` (gcc, -O2, no FMA
    contraction, OpenMP when available)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_D = ctypes.c_double
_I = ctypes.c_int
_LL = ctypes.c_longlong
_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    sig = {
        "orc_lens": (None, [_D, _D, _P, _P, _P, _P]),
        "orc_rayshoot": (_I, [_D, _D, _D, _I, _LL, _D, _P, _P, _P, _I]),
        "orc_counts_to_mag": (None, [_P, _I, _D, _LL, _D, _P]),
        "orc_quintic": (_I, [_D, _D, _D, _D, _P, _P]),
        "orc_roots5": (_I, [_P, _P, _P, _P]),
        "orc_images": (_I, [_D, _D, _D, _D, _D, _P, _P, _P, _P]),
        "orc_mag_point": (_D, [_D, _D, _D, _D, _P]),
        "orc_pspl": (_D, [_D]),
        "orc_poly_map": (None, [_D, _D, _D, _I, _P, _I]),
        "orc_mag_point_grad": (_D, [_D, _D, _D, _D, _P]),
        "orc_half_bits": (ctypes.c_uint16, [_D]),
        "orc_fs_weights": (None, [_D, _D, _I, _I, _P]),
        "orc_line_max": (_D, [_P, _I, _D, _D, _D]),
        "orc_line_peaks": (_I, [_P, _I, _D, _D, _D, _D, _D, _I, _D, _I, _P,
                                _P, _P, _P]),
        "orc_fs_convolve": (None, [_P, _I, _D, _P, _I, _P, _I]),
        "orc_half_value": (_D, [ctypes.c_uint16]),
        "orc_log10_half": (None, [_P, ctypes.c_longlong, _D, _P]),
        "orc_half_decode": (None, [_P, ctypes.c_longlong, _P]),
        "orc_chi2_grad_poly": (_D, [_D, _D, _P, _P, _P, ctypes.c_long, _D, _D,
                                    _D, _D, _P, _P, _P]),
        "orc_traj_point": (None, [_D, _D, _D, _D, _D, _P, _P]),
        "orc_map_A": (_D, [_P, _I, _D, _D, _D]),
        "orc_fit_A": (_D, [_P, _P, _P, ctypes.c_long, _P, _P, _P]),
        "orc_axis": (None, [_D, _D, _I, _I, _P]),
        "orc_grid_chi2": (_I, [_P, _I, _D, _D, _D, _I, _P, _P, _P,
                               ctypes.c_long, _P, _I, _I, _P, _I, _P, _I,
                               _LL, _LL, _P, _P, _P, _P, _I]),
        "orc_topk": (_I, [_P, _LL, _LL, _I, _P, _P]),
        "orc_chi2_theta": (_D, [_P, _I, _D, _D, _D, _I, _P, _P, _P,
                                ctypes.c_long, _D, _D, _D, _D, _P, _P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def threads_default() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------- geometry
def lens(s: float, q: float):
    """(eps1, eps2, x_primary, x_secondary): §4.1 centre-of-mass origin."""
    out = [ctypes.c_double() for _ in range(4)]
    _load().orc_lens(s, q, *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


# ---------------------------------------------------------------- ray shooting
def rayshoot(s, q, L, npix, nray, X, nthreads=1):
    """Inverse ray shooting (§3, §5): returns (counts[npix, npix] uint32 with
    counts[iy, ix], off_map, lost)."""
    counts = np.zeros((npix, npix), dtype=np.uint32)
    off = ctypes.c_uint64()
    lost = ctypes.c_uint64()
    rc = _load().orc_rayshoot(float(s), float(q), float(L), int(npix),
                              int(nray), float(X), _ptr(counts),
                              ctypes.byref(off), ctypes.byref(lost),
                              int(nthreads))
    if rc != 0:
        raise ValueError("orc_rayshoot rejected its arguments")
    return counts, int(off.value), int(lost.value)


def counts_to_mag(counts, L, nray, X):
    """A = count * h^2 / Delta^2 in FP64, rounded to FP32."""
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    npix = counts.shape[0]
    A = np.zeros((npix, npix), dtype=np.float32)
    _load().orc_counts_to_mag(_ptr(counts), npix, float(L), int(nray),
                              float(X), _ptr(A))
    return A


def build_map(s, q, L, npix, nray, X, nthreads=1):
    """Oracle magnification map (float32 [npix, npix]) plus the raw counts."""
    c, off, lost = rayshoot(s, q, L, npix, nray, X, nthreads)
    return counts_to_mag(c, L, nray, X), c, off, lost


# ---------------------------------------------------------------- polynomial
def quintic(s, q, y1, y2):
    """Coefficients c[0..5] (c[k] multiplies z^k) of the §3 lens quintic."""
    cre = np.zeros(6)
    cim = np.zeros(6)
    rc = _load().orc_quintic(s, q, y1, y2, _ptr(cre), _ptr(cim))
    if rc != 0:
        raise ValueError("degenerate quintic (source on a lens)")
    return cre + 1j * cim


def roots5(c):
    """All five roots of the quintic by Laguerre + deflation + polishing."""
    c = np.asarray(c, dtype=np.complex128)
    cre = _f64(c.real)
    cim = _f64(c.imag)
    rre = np.zeros(5)
    rim = np.zeros(5)
    _load().orc_roots5(_ptr(cre), _ptr(cim), _ptr(rre), _ptr(rim))
    return rre + 1j * rim


def images(s, q, y1, y2, tol=1e-6):
    """(n_images, z[5], detJ[5], residual[5]) ordered by Eq. 2 residual; the
    first n_images are the images."""
    zre = np.zeros(5)
    zim = np.zeros(5)
    dj = np.zeros(5)
    res = np.zeros(5)
    n = _load().orc_images(s, q, y1, y2, tol, _ptr(zre), _ptr(zim), _ptr(dj),
                           _ptr(res))
    return n, zre + 1j * zim, dj, res


def mag_point(s, q, y1, y2):
    """Point-source magnification sum_j 1/|det J_j| (§3 Eq. 3)."""
    n = ctypes.c_int()
    return _load().orc_mag_point(s, q, y1, y2, ctypes.byref(n))


def mag_point_grad(s, q, y1, y2):
    """(A, dA/dy1, dA/dy2) of the point source, by implicit differentiation
    of the lens equation (Eq. 2, 4)."""
    g = np.zeros(2)
    a = _load().orc_mag_point_grad(float(s), float(q), float(y1), float(y2),
                                   _ptr(g))
    return a, g[0], g[1]


def chi2_grad_poly(t, F, w, theta, s, q):
    """(chi2, grad[4], Fs, Fb) of the polynomial point-source light curve of
    theta = (t0, tE, u0, alpha), the flux fit profiled out (Eq. 5-6)."""
    t = _f64(t)
    F = _f64(F)
    w = _f64(w)
    g = np.zeros(4)
    fs = ctypes.c_double()
    fb = ctypes.c_double()
    c = _load().orc_chi2_grad_poly(float(s), float(q), _ptr(t), _ptr(F),
                                   _ptr(w), len(t), *[float(x) for x in theta],
                                   _ptr(g), ctypes.byref(fs), ctypes.byref(fb))
    return c, g, fs.value, fb.value


def fs_radius(rho_px):
    """Half-width R (texels) of the finite-source kernel of radius rho_px."""
    return int(math.ceil(rho_px + 0.5))


def fs_weights(rho_px, gamma, sub=8):
    """Limb-darkened source profile (§4.1) integrated over the texels
    within R = fs_radius(rho_px), normalised; [2R+1, 2R+1] (dy, dx)."""
    R = fs_radius(rho_px)
    W = np.zeros((2 * R + 1, 2 * R + 1))
    _load().orc_fs_weights(float(rho_px), float(gamma), R, int(sub), _ptr(W))
    return W


def fs_convolve(A, L, W, nthreads=1):
    """Finite-source map: A convolved with W, the Paczynski curve standing
    in for the texels outside the map; FP64 [npix, npix]."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    W = np.ascontiguousarray(W, dtype=np.float64)
    R = (W.shape[0] - 1) // 2
    out = np.zeros(A.shape)
    _load().orc_fs_convolve(_ptr(A), A.shape[0], float(L), _ptr(W), R,
                            _ptr(out), int(nthreads))
    return out


def half_bits(x):
    """IEEE binary16 bit pattern of x (round to nearest even)."""
    return int(_load().orc_half_bits(float(x)))


def half_value(h):
    """Value of a binary16 bit pattern."""
    return _load().orc_half_value(int(h))


def log10_half(A, a_floor):
    """FP16 storage codes of an FP32 map: half(log10(max(A, a_floor)))."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    codes = np.zeros(A.shape, dtype=np.uint16)
    _load().orc_log10_half(_ptr(A), A.size, float(a_floor), _ptr(codes))
    return codes


def half_decode(codes):
    """Decoded FP16 map: 10^x per code, rounded to FP32."""
    codes = np.ascontiguousarray(codes, dtype=np.uint16)
    A = np.zeros(codes.shape, dtype=np.float32)
    _load().orc_half_decode(_ptr(codes), codes.size, _ptr(A))
    return A


def half_floor(L, npix, nray, X):
    """A_floor of a ray-shot map: half a ray, 0.5 h^2 / Delta^2."""
    h = 2.0 * X / nray
    d = 2.0 * L / npix
    return 0.5 * h * h / (d * d)


def poly_map(s, q, L, npix, nthreads=1):
    """Point-source map: the polynomial magnification at texel centres
    (§4.1), FP32 [npix, npix]."""
    A = np.zeros((npix, npix), dtype=np.float32)
    _load().orc_poly_map(float(s), float(q), float(L), int(npix), _ptr(A),
                         int(nthreads))
    return A


def pspl(u):
    """Paczynski A(u) = (u^2+2)/(u sqrt(u^2+4))."""
    return _load().orc_pspl(float(u))


# ---------------------------------------------------------------- lookup
def traj_point(t, t0, tE, u0, alpha):
    a = ctypes.c_double()
    b = ctypes.c_double()
    _load().orc_traj_point(t, t0, tE, u0, alpha, ctypes.byref(a),
                           ctypes.byref(b))
    return a.value, b.value


def map_A(A, L, y1, y2):
    """Bilinear lookup between texel centres; Paczynski outside the map."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    return _load().orc_map_A(_ptr(A), A.shape[0], float(L), float(y1),
                             float(y2))


def line_max(A, L, u0, alpha):
    """Largest magnification on the straight line (u0, alpha): exact for the
    bilinear lookup inside the map and the Paczynski curve outside (§4.3)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    return _load().orc_line_max(_ptr(A), A.shape[0], float(L), float(u0),
                                float(alpha))


def line_peaks(A, L, lines, sub=2, delta=0.0, max_peaks=8, bounds=False):
    """§4.3 (iii): the peak library of the map A along lines[j] = (u,
    alpha, shift) (shift: the line's reference point lies tau = shift past
    its closest approach to the origin), in FP64 from the definition (a
    turn of the sampled bilinear profile from rising to falling, rise and
    fall confirmed by the factor 1 + delta).  Returns (count[n] int32,
    pos[n, max_peaks], height[n, max_peaks]); pos in Einstein radii from the
    reference point, the max_peaks highest peaks in increasing tau, NaN in
    unused slots.  With bounds=True also (herr[n, max_peaks], uncertain[n]
    bool): the height bounds of an FP32 evaluation of the same profile and
    the lines where some decision lies within those bounds (see
    orc_line_peaks)."""
    lib = _load()
    A = np.ascontiguousarray(A, dtype=np.float32)
    lines = np.asarray(lines, dtype=np.float64).reshape(-1, 3)
    n = len(lines)
    count = np.zeros(n, dtype=np.int32)
    pos = np.zeros((n, max_peaks))
    height = np.zeros((n, max_peaks))
    herr = np.zeros((n, max_peaks))
    unsure = np.zeros(n, dtype=bool)
    pb = np.zeros(max_peaks)
    hb = np.zeros(max_peaks)
    eb = np.zeros(max_peaks)
    flag = ctypes.c_int()
    for j, (u, al, sh) in enumerate(lines):
        count[j] = lib.orc_line_peaks(_ptr(A), A.shape[0], L, float(u),
                                      math.cos(al), math.sin(al), float(sh),
                                      sub, delta, max_peaks, _ptr(pb),
                                      _ptr(hb), _ptr(eb), ctypes.byref(flag))
        pos[j] = pb
        height[j] = hb
        herr[j] = eb
        unsure[j] = bool(flag.value)
    if bounds:
        return count, pos, height, herr, unsure
    return count, pos, height


def peak_trajectories(lines, count, pos, tp, t0_offsets, tE_axis,
                      min_peaks=0):
    """§4.3 (iv)-(v), Eq. 7-8: the set of trajectories the peak library
    allows, as rows (line j, u0, alpha, t0, tE).

    A line takes part when it has at least max(min_peaks, len(tp)) peaks;
    its peaks are its kept ones (pos[j], finite entries), tau_m measured
    from the line's closest approach to the origin, M_m = pos + shift.
      * no peak time: every (t0, tE) of the axes, t0 = t0_offsets
        (absolute times) about the line's reference point, i.e. the
        trajectory (u, alpha, t0 - shift tE, tE);
      * one peak time t_p: for every peak m, every dt0 in t0_offsets and
        tE in tE_axis, the trajectory whose peak m comes at t_p + dt0:
        t0 = t_p + dt0 - M_m tE (Eq. 7);
      * two peak times t_p1 < t_p2: for every pair of peaks a before b,
        tE = (t_p2 - t_p1) / (M_b - M_a) (Eq. 8) and peak a at t_p1 + dt0.
    The order of the rows carries no meaning: callers compare sets."""
    lines = np.asarray(lines, dtype=np.float64).reshape(-1, 3)
    need = max(min_peaks, len(tp))
    out = []
    for j, (u, al, sh) in enumerate(lines):
        if count[j] < need:
            continue
        M = sorted(float(p) + sh for p in pos[j] if np.isfinite(p))
        if len(tp) == 0:
            for t0 in t0_offsets:
                for tE in tE_axis:
                    out.append((j, u, al, t0 - sh * tE, tE))
        elif len(tp) == 1:
            for Mm in M:
                for dt in t0_offsets:
                    for tE in tE_axis:
                        out.append((j, u, al, tp[0] + dt - Mm * tE, tE))
        else:
            for a in range(len(M)):
                for b in range(a + 1, len(M)):
                    tE = (tp[1] - tp[0]) / (M[b] - M[a])
                    for dt in t0_offsets:
                        out.append((j, u, al, tp[0] + dt - M[a] * tE, tE))
    return np.array(out, dtype=np.float64).reshape(-1, 5)


def lightcurve_map(A, L, t, t0, tE, u0, alpha):
    """A(t_i) along a straight trajectory from the map (§4.2)."""
    out = np.empty(len(t))
    for i, ti in enumerate(np.asarray(t, dtype=np.float64)):
        y1, y2 = traj_point(float(ti), t0, tE, u0, alpha)
        out[i] = map_A(A, L, y1, y2)
    return out


def lightcurve_point(s, q, t, t0, tE, u0, alpha):
    """A(t_i) along a straight trajectory from the lens polynomial."""
    out = np.empty(len(t))
    for i, ti in enumerate(np.asarray(t, dtype=np.float64)):
        y1, y2 = traj_point(float(ti), t0, tE, u0, alpha)
        out[i] = mag_point(s, q, y1, y2)
    return out


# ---------------------------------------------------------------- fit
def fit_A(A, F, w):
    """(chi2, Fs, Fb, flag) of F = Fs A + Fb by weighted least squares."""
    A = _f64(A)
    F = _f64(F)
    w = _f64(w)
    fs = ctypes.c_double()
    fb = ctypes.c_double()
    fl = ctypes.c_int()
    c = _load().orc_fit_A(_ptr(A), _ptr(F), _ptr(w), len(A), ctypes.byref(fs),
                          ctypes.byref(fb), ctypes.byref(fl))
    return c, fs.value, fb.value, fl.value


def axis(lo, hi, n, logsp):
    out = np.zeros(n)
    _load().orc_axis(float(lo), float(hi), int(n), int(bool(logsp)),
                     _ptr(out))
    return out


class Grid:
    """Trajectory grid (u0, alpha, t0, tE); alpha_k = 2 pi k / n_alpha.
    Trajectory index = ((i_u0 n_alpha + i_alpha) n_t0 + i_t0) n_tE + i_tE."""

    def __init__(self, n_u0, n_alpha, n_t0, n_tE, u0_lo, u0_hi, t0_lo, t0_hi,
                 tE_lo, tE_hi, u0_log=True, tE_log=True):
        self.n_u0, self.n_alpha, self.n_t0, self.n_tE = (n_u0, n_alpha, n_t0,
                                                         n_tE)
        self.u0 = axis(u0_lo, u0_hi, n_u0, u0_log)
        self.t0 = axis(t0_lo, t0_hi, n_t0, False)
        self.tE = axis(tE_lo, tE_hi, n_tE, tE_log)

    @property
    def size(self):
        return self.n_u0 * self.n_alpha * self.n_t0 * self.n_tE

    def params(self, idx):
        itE = idx % self.n_tE
        r = idx // self.n_tE
        it0 = r % self.n_t0
        r //= self.n_t0
        ia = r % self.n_alpha
        iu = r // self.n_alpha
        return (self.t0[it0], self.tE[itE], self.u0[iu],
                2.0 * np.pi * ia / self.n_alpha)


def grid_chi2(grid: Grid, t, F, w, A=None, L=None, s=None, q=None, first=0,
              count=None, nthreads=1):
    """Dense chi^2 for trajectory indices [first, first+count): on the map A
    (half-width L) or, when A is None, on the point-source polynomial
    magnification of (s, q).  Returns (chi2, Fs, Fb, flag) arrays."""
    t = _f64(t)
    F = _f64(F)
    w = _f64(w)
    if count is None:
        count = grid.size - first
    chi2 = np.zeros(count)
    fs = np.zeros(count)
    fb = np.zeros(count)
    fl = np.zeros(count, dtype=np.int32)
    if A is not None:
        A = np.ascontiguousarray(A, dtype=np.float32)
        mode, npix, Lv, sv, qv = 0, A.shape[0], float(L), 0.0, 0.0
        Ap = _ptr(A)
    else:
        mode, npix, Lv, sv, qv = 1, 0, 0.0, float(s), float(q)
        Ap = None
    rc = _load().orc_grid_chi2(
        Ap, npix, Lv, sv, qv, mode, _ptr(t), _ptr(F), _ptr(w), len(t),
        _ptr(grid.u0), grid.n_u0, grid.n_alpha, _ptr(grid.t0), grid.n_t0,
        _ptr(grid.tE), grid.n_tE, int(first), int(count), _ptr(chi2),
        _ptr(fs), _ptr(fb), _ptr(fl), int(nthreads))
    if rc < 0:
        raise ValueError("orc_grid_chi2 rejected its arguments")
    return chi2, fs, fb, fl


def chi2_theta(t, F, w, theta, A=None, L=None, s=None, q=None):
    """chi^2 of one trajectory theta = (t0, tE, u0, alpha) on the map A
    (half-width L) or, when A is None, on the polynomial magnification of
    (s, q); returns (chi2, Fs, Fb)."""
    t = _f64(t)
    F = _f64(F)
    w = _f64(w)
    fs = ctypes.c_double()
    fb = ctypes.c_double()
    if A is not None:
        A = np.ascontiguousarray(A, dtype=np.float32)
        c = _load().orc_chi2_theta(_ptr(A), A.shape[0], float(L), 0.0, 0.0,
                                   0, _ptr(t), _ptr(F), _ptr(w), len(t),
                                   *[float(x) for x in theta],
                                   ctypes.byref(fs), ctypes.byref(fb))
    else:
        c = _load().orc_chi2_theta(None, 0, 0.0, float(s), float(q), 1,
                                   _ptr(t), _ptr(F), _ptr(w), len(t),
                                   *[float(x) for x in theta],
                                   ctypes.byref(fs), ctypes.byref(fb))
    return c, fs.value, fb.value


def topk(chi2, k, first=0):
    """The k smallest (chi2, idx) by a full sort, ties by index."""
    chi2 = _f64(chi2)
    idx = np.zeros(k, dtype=np.int64)
    val = np.zeros(k)
    m = _load().orc_topk(_ptr(chi2), len(chi2), int(first), int(k), _ptr(idx),
                         _ptr(val))
    return idx[:m], val[:m]


__all__ = [n for n in dir() if not n.startswith("_")]
if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
