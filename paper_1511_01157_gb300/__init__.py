"""Python binding of the MORSE GB300 library (libmorse.so, C ABI in
include/morse.h).

Argument marshalling only: every step of the hot path (ray shooting, map
texels, trajectory search, top-K, fits) runs in the library's CUDA kernels.
The library must have been built (``__graft_entry__.build()`` or
``python paper_1511_01157_gb300/build.py``); importing this module without
it raises ``ImportError`` -- there is no CPU fallback.

Method: McDougall & Albrow (2015) MORSE -- a binary-lens magnification map
per (s, q) built by inverse ray shooting (§3, §4.1), a grid of straight
trajectories searched through it with a linear flux fit and chi^2 (§4.2),
and the best trajectories kept as seeds (§4.4).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MORSE_LIB=checked selects the bounds-checked build (tests); a path to a
# .so selects another build of the same library (tuning experiments)
_sel = os.environ.get("MORSE_LIB", "")
if _sel == "checked":
    LIB_PATH = os.path.join(_HERE, "libmorse_checked.so")
elif _sel.endswith(".so") and os.path.exists(_sel):
    LIB_PATH = os.path.abspath(_sel)
else:
    LIB_PATH = os.path.join(_HERE, "libmorse.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libmorse.so is not built; run `python -c 'import __graft_entry__ as "
        "g; g.build()'` (needs nvcc for sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EDEGENERATE, EUNSUPPORTED = range(7)
# morse_inject_fault kinds (tests of the error paths)
FAULT_NONE, FAULT_LOCK_HELD, FAULT_ALLOC = range(3)
DEFLECT_FP64, DEFLECT_FP32 = 0, 1
STORE_FP32, STORE_FP16LOG = 1, 2
GEN_RAYS, GEN_POLY = 0, 1
FIT_DEGENERATE, FIT_REFINED = 1, 2
REFINE_LM = 0


class MorseError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{_status_name(status)}: {msg}")


class Grid(ctypes.Structure):
    """morse_grid: trajectory grid over (u0, alpha, t0, tE)."""
    _fields_ = [("n_u0", ctypes.c_int), ("n_alpha", ctypes.c_int),
                ("n_t0", ctypes.c_int), ("n_tE", ctypes.c_int),
                ("u0_lo", ctypes.c_double), ("u0_hi", ctypes.c_double),
                ("t0_lo", ctypes.c_double), ("t0_hi", ctypes.c_double),
                ("tE_lo", ctypes.c_double), ("tE_hi", ctypes.c_double),
                ("u0_log", ctypes.c_int), ("tE_log", ctypes.c_int),
                ("top_k", ctypes.c_int), ("a_min", ctypes.c_float)]

    @classmethod
    def make(cls, n_u0, n_alpha, n_t0, n_tE, u0_lo, u0_hi, t0_lo, t0_hi,
             tE_lo, tE_hi, u0_log=True, tE_log=True, top_k=16, a_min=0.0):
        return cls(n_u0, n_alpha, n_t0, n_tE, u0_lo, u0_hi, t0_lo, t0_hi,
                   tE_lo, tE_hi, int(bool(u0_log)), int(bool(tE_log)), top_k,
                   float(a_min))

    @property
    def size(self):
        return self.n_u0 * self.n_alpha * self.n_t0 * self.n_tE


class Fit(ctypes.Structure):
    _fields_ = [("chi2", ctypes.c_double), ("t0", ctypes.c_double),
                ("tE", ctypes.c_double), ("u0", ctypes.c_double),
                ("alpha", ctypes.c_double), ("Fs", ctypes.c_double),
                ("Fb", ctypes.c_double), ("idx", ctypes.c_int64),
                ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32)]


FIT_DTYPE = np.dtype([("chi2", "f8"), ("t0", "f8"), ("tE", "f8"),
                      ("u0", "f8"), ("alpha", "f8"), ("Fs", "f8"),
                      ("Fb", "f8"), ("idx", "i8"), ("flags", "i4"),
                      ("reserved", "i4")])
assert FIT_DTYPE.itemsize == ctypes.sizeof(Fit)


class MapOpts(ctypes.Structure):
    _fields_ = [("image_halfwidth", ctypes.c_double),
                ("deflect", ctypes.c_int), ("store", ctypes.c_int),
                ("generator", ctypes.c_int)]


class Caustic(ctypes.Structure):
    """morse_caustic: centre, size and point count of one caustic."""
    _fields_ = [("c1", ctypes.c_double), ("c2", ctypes.c_double),
                ("size", ctypes.c_double), ("n_points", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class PeakOpts(ctypes.Structure):
    """morse_peak_opts: samples per texel, peaks kept per line, threshold."""
    _fields_ = [("sub", ctypes.c_int), ("max_peaks", ctypes.c_int),
                ("delta", ctypes.c_double)]


def rphi_lines(caustics, n_r, r_lo, r_hi, n_phi) -> np.ndarray:
    """Lines (u, alpha, shift) of an (r, phi) grid about the caustics
    (morse_rphi_lines): [n_caustics * n_r * n_phi, 3]."""
    arr = (Caustic * len(caustics))(*caustics)
    out = np.zeros((len(caustics) * n_r * n_phi, 3))
    st = _lib.morse_rphi_lines(arr, len(caustics), int(n_r), float(r_lo),
                               float(r_hi), int(n_phi), _ptr(out))
    if st != OK:
        raise MorseError(st, "morse_rphi_lines")
    return out


class Peaks(ctypes.Structure):
    """morse_peaks: measured throughput of the GPU for the rooflines."""
    _fields_ = [("fp32_fma_per_s", ctypes.c_double),
                ("fp64_fma_per_s", ctypes.c_double),
                ("smem_atomics_per_s", ctypes.c_double),
                ("l1_gather_bytes_per_s", ctypes.c_double),
                ("l2_gather_bytes_per_s", ctypes.c_double)]


class BatchShape(ctypes.Structure):
    """morse_batch_shape: launch shape of one epoch-count bucket."""
    _fields_ = [("tpg", ctypes.c_int), ("rounds", ctypes.c_int),
                ("stage", ctypes.c_int), ("tuned", ctypes.c_int),
                ("ns_per_eval", ctypes.c_double)]


TUNE_OFF, TUNE_ON = 0, 1

_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64
_S = ctypes.c_int  # morse_status

_SIGS = {
    "morse_status_string": (ctypes.c_char_p, [_I]),
    "morse_version": (ctypes.c_char_p, []),
    "morse_create": (_S, [_P, _I, _P]),
    "morse_destroy": (None, [_P]),
    "morse_last_error": (ctypes.c_char_p, [_P]),
    "morse_build_map": (_S, [_P, _D, _D, _D, _I, _I64, _P, _P]),
    "morse_map_from_host": (_S, [_P, _P, _I, _D, _P]),
    "morse_map_counts": (_S, [_P, _P, _P, _P]),
    "morse_map_values": (_S, [_P, _P]),
    "morse_map_info": (_S, [_P, _P, _P, _P, _P]),
    "morse_map_free": (None, [_P]),
    "morse_map_set_lookup": (_S, [_P, _I]),
    "morse_map_finite_source": (_S, [_P, _P, _D, _D, _P]),
    "morse_line_max": (_S, [_P, _P, _P, _P]),
    "morse_caustics": (_S, [_P, _D, _D, _I, _P, _P]),
    "morse_rphi_lines": (_S, [_P, _I, _I, _D, _D, _I, _P]),
    "morse_grid_chi2_lines": (_S, [_P, _P, _P, _P, _P, _P]),
    "morse_line_peaks": (_S, [_P, _P, _P, _I, _P, _P, _P, _P]),
    "morse_peak_search": (_S, [_P, _P, _P, _P, _P, _I, _P, _I, _P, _I, _P]),
    "morse_grid_chi2_batch": (_S, [_P, _P, _I, _P, _I, _P, _P]),
    "morse_measure_peaks": (_S, [_P, _P]),
    "morse_batch_tuning": (_S, [_P, _I]),
    "morse_batch_shape_of": (_S, [_P, _I64, _P, _P, _P]),
    "morse_map_half": (_S, [_P, _P, _P]),
    "morse_event_create": (_S, [_P, _P, _P, _P, _I64, _D, _P]),
    "morse_event_free": (None, [_P]),
    "morse_event_info": (_S, [_P, _P, _P]),
    "morse_grid_chi2": (_S, [_P, _P, _P, _P, _P]),
    "morse_grid_chi2_noalloc": (_S, [_P, _P, _P, _P, _P]),
    "morse_grid_chi2_dense": (_S, [_P, _P, _P, _P, _I64, _I64, _P, _P, _P]),
    "morse_search": (_S, [_P, _P, _P, _P, _I64, _D, _D, _D, _D, _I, _I64, _P,
                          _P, _P]),
    "morse_sweep": (_S, [_P, _P, _P, _P, _I, _D, _I, _I64, _P, _P, _P]),
    "morse_search_sweep": (_S, [_P, _P, _P, _P, _I64, _D, _P, _P, _I, _D, _I,
                                _I64, _P, _P, _P]),
    "morse_lightcurve": (_S, [_P, _P, _D, _D, _D, _D, _P, _I64, _P]),
    "morse_topk_merge": (_S, [_P, _P, _I, _I, _P]),
    "morse_chi2_grad": (_S, [_P, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "morse_chi2_grad_dev": (_S, [_P, _P, _P, _P, _I64, _P, _P]),
    "morse_refine": (_S, [_P, _P, _P, _P, _I, _I, _I, _P]),
    "morse_last_kernel_ms": (_S, [_P, _I, _P]),
    "morse_launch_count": (_S, [_P, _P]),
    "morse_last_search_stats": (_S, [_P, _P]),
    "morse_inject_fault": (_S, [_P, _I, _I64]),
    "morse_grid_chi2_range": (_S, [_P, _P, _P, _P, _I64, _I64, _P]),
    "morse_refine_batch": (_S, [_P, _P, _P, _I, _P, _P, _I, _I, _I, _P]),
    "morse_line_peaks_batch": (_S, [_P, _P, _I, _P, _I, _P, _P, _P, _P]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _status_name(st):
    return _lib.morse_status_string(int(st)).decode()


def version() -> str:
    return _lib.morse_version().decode()


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    h = getattr(stream, "cuda_stream", None)  # torch.cuda.Stream
    if h is None:
        raise TypeError("stream must be a torch.cuda.Stream or an int handle")
    return ctypes.c_void_p(int(h))


class Context:
    """A device, a CUDA stream and the library's workspaces (morse_create)."""

    def __init__(self, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        self._stream_ref = stream  # keep a torch stream alive
        st = _lib.morse_create(ctypes.byref(self._h), int(device),
                               _stream_handle(stream))
        if st != OK:
            raise MorseError(st, f"morse_create(device={device}) failed")
        self.device = device

    def _check(self, st, what):
        if st != OK:
            msg = _lib.morse_last_error(self._h).decode(errors="replace")
            raise MorseError(st, f"{what}: {msg}")

    def close(self):
        if self._h:
            _lib.morse_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ maps
    def build_map(self, s, q, extent, npix, rays_per_axis,
                  image_halfwidth=None, deflect="fp64", fp16log=False,
                  generator="rays"):
        """Magnification map of the binary lens (s, q) by inverse ray
        shooting, or by the lens polynomial per texel with generator="poly"
        (morse_build_map)."""
        opts = MapOpts(float(image_halfwidth or 0.0),
                       DEFLECT_FP64 if deflect == "fp64" else DEFLECT_FP32,
                       STORE_FP32 | (STORE_FP16LOG if fp16log else 0),
                       GEN_POLY if generator == "poly" else GEN_RAYS)
        h = ctypes.c_void_p()
        st = _lib.morse_build_map(self._h, float(s), float(q), float(extent),
                                  int(npix), int(rays_per_axis),
                                  ctypes.byref(opts), ctypes.byref(h))
        self._check(st, "morse_build_map")
        return Map(self, h)

    def map_from_host(self, A, extent):
        A = np.ascontiguousarray(A, dtype=np.float32)
        if A.ndim != 2 or A.shape[0] != A.shape[1]:
            raise ValueError("map must be square [npix, npix]")
        h = ctypes.c_void_p()
        st = _lib.morse_map_from_host(self._h, _ptr(A), A.shape[0],
                                      float(extent), ctypes.byref(h))
        self._check(st, "morse_map_from_host")
        return Map(self, h)

    # ------------------------------------------------------------ events
    def event(self, t, flux, sigma, t_ref=0.0):
        t, flux, sigma = _f64(t), _f64(flux), _f64(sigma)
        if not (len(t) == len(flux) == len(sigma)):
            raise ValueError("t, flux and sigma must have equal length")
        h = ctypes.c_void_p()
        st = _lib.morse_event_create(self._h, _ptr(t), _ptr(flux),
                                     _ptr(sigma), len(t), float(t_ref),
                                     ctypes.byref(h))
        self._check(st, "morse_event_create")
        return Event(self, h, len(t))

    # ------------------------------------------------------------ search
    def grid_chi2(self, event, map_, grid: Grid) -> np.ndarray:
        """Top-K trajectories (structured array, FIT_DTYPE)."""
        out = np.zeros(grid.top_k, dtype=FIT_DTYPE)
        st = _lib.morse_grid_chi2(self._h, event._h, map_._h,
                                  ctypes.byref(grid), _ptr(out))
        self._check(st, "morse_grid_chi2")
        return out

    def grid_chi2_range(self, event, map_, grid: Grid, first, count):
        """Top-K of trajectories [first, first + count) of the grid
        (morse_grid_chi2_range): one shard of a split search."""
        out = np.zeros(grid.top_k, dtype=FIT_DTYPE)
        st = _lib.morse_grid_chi2_range(self._h, event._h, map_._h,
                                        ctypes.byref(grid), int(first),
                                        int(count), _ptr(out))
        self._check(st, "morse_grid_chi2_range")
        return out

    def grid_chi2_batch(self, events, maps, grid: Grid) -> np.ndarray:
        """Batched search of every (event, map) pair in one persistent launch
        (morse_grid_chi2_batch): fits[n_events, n_maps, top_k]."""
        ev = (ctypes.c_void_p * len(events))(*[e._h for e in events])
        mp = (ctypes.c_void_p * len(maps))(*[m._h for m in maps])
        out = np.zeros((len(events), len(maps), grid.top_k), dtype=FIT_DTYPE)
        st = _lib.morse_grid_chi2_batch(self._h, ev, len(events), mp,
                                        len(maps), ctypes.byref(grid),
                                        _ptr(out))
        self._check(st, "morse_grid_chi2_batch")
        return out

    def caustics(self, s, q, n_psi=720):
        """Caustics of the lens (s, q) (morse_caustics): list of Caustic."""
        out = (Caustic * 3)()
        n = ctypes.c_int()
        self._check(_lib.morse_caustics(self._h, float(s), float(q),
                                        int(n_psi), out, ctypes.byref(n)),
                    "morse_caustics")
        return [out[i] for i in range(n.value)]

    def grid_chi2_lines(self, event, map_, grid: Grid, lines) -> np.ndarray:
        """Top-K over a grid of lines (morse_grid_chi2_lines): grid.n_u0 =
        len(lines), grid.n_alpha = 1."""
        lines = np.ascontiguousarray(lines, dtype=np.float64)
        out = np.zeros(grid.top_k, dtype=FIT_DTYPE)
        st = _lib.morse_grid_chi2_lines(self._h, event._h, map_._h,
                                        ctypes.byref(grid), _ptr(lines),
                                        _ptr(out))
        self._check(st, "morse_grid_chi2_lines")
        return out

    def line_peaks(self, map_, lines, sub=2, max_peaks=8, delta=0.0):
        """Peak library of the map along lines (u, alpha, shift)
        (morse_line_peaks): (count[n], pos[n, max_peaks],
        height[n, max_peaks])."""
        lines = np.ascontiguousarray(lines, dtype=np.float64).reshape(-1, 3)
        n = len(lines)
        count = np.zeros(n, dtype=np.int32)
        pos = np.zeros((n, max_peaks))
        height = np.zeros((n, max_peaks))
        o = PeakOpts(int(sub), int(max_peaks), float(delta))
        self._check(_lib.morse_line_peaks(self._h, map_._h, _ptr(lines), n,
                                          ctypes.byref(o), _ptr(count),
                                          _ptr(pos), _ptr(height)),
                    "morse_line_peaks")
        return count, pos, height

    def line_peaks_batch(self, maps, lines, sub=2, max_peaks=8, delta=0.0):
        """Peak libraries of several maps along the same lines in one
        launch (morse_line_peaks_batch): (count[n_maps, n],
        pos[n_maps, n, max_peaks], height[n_maps, n, max_peaks])."""
        lines = np.ascontiguousarray(lines, dtype=np.float64).reshape(-1, 3)
        n, nm = len(lines), len(maps)
        count = np.zeros((nm, n), dtype=np.int32)
        pos = np.zeros((nm, n, max_peaks))
        height = np.zeros((nm, n, max_peaks))
        o = PeakOpts(int(sub), int(max_peaks), float(delta))
        mp = (ctypes.c_void_p * nm)(*[m._h for m in maps])
        self._check(_lib.morse_line_peaks_batch(
            self._h, mp, nm, _ptr(lines), n, ctypes.byref(o), _ptr(count),
            _ptr(pos), _ptr(height)), "morse_line_peaks_batch")
        return count, pos, height

    def peak_search(self, event, map_, grid: Grid, lines, tp=(),
                    min_peaks=0, sub=2, max_peaks=8, delta=0.0) -> np.ndarray:
        """Top-K over the trajectories the peak library allows, aligned
        with the peak times tp (0, 1 or 2 of them) (morse_peak_search)."""
        lines = np.ascontiguousarray(lines, dtype=np.float64).reshape(-1, 3)
        tpa = np.ascontiguousarray(tp, dtype=np.float64)
        out = np.zeros(grid.top_k, dtype=FIT_DTYPE)
        o = PeakOpts(int(sub), int(max_peaks), float(delta))
        st = _lib.morse_peak_search(self._h, event._h, map_._h,
                                    ctypes.byref(grid), _ptr(lines),
                                    len(lines), ctypes.byref(o),
                                    int(min_peaks),
                                    _ptr(tpa) if len(tpa) else None,
                                    len(tpa), _ptr(out))
        self._check(st, "morse_peak_search")
        return out

    def line_max(self, map_, grid: Grid) -> np.ndarray:
        """Largest magnification on every (u0, alpha) line of the grid
        (morse_line_max): [n_u0, n_alpha]."""
        out = np.zeros((grid.n_u0, grid.n_alpha))
        self._check(_lib.morse_line_max(self._h, map_._h, ctypes.byref(grid),
                                        _ptr(out)), "morse_line_max")
        return out

    def measure_peaks(self) -> dict:
        """FP32/FP64 FMA, shared-atomic and L1/L2 gather throughput of this
        GPU (morse_measure_peaks)."""
        pk = Peaks()
        self._check(_lib.morse_measure_peaks(self._h, ctypes.byref(pk)),
                    "morse_measure_peaks")
        return {f: getattr(pk, f) for f, _ in Peaks._fields_}

    def batch_tuning(self, on: bool):
        """Autotune batched launch shapes (default) or use the default rule;
        forgets the shapes chosen so far (morse_batch_tuning)."""
        self._check(_lib.morse_batch_tuning(self._h,
                                            TUNE_ON if on else TUNE_OFF),
                    "morse_batch_tuning")

    def batch_shape(self, n_ep, grid: Grid, map_) -> dict:
        """The batched launch shape chosen for light curves of n_ep epochs."""
        sh = BatchShape()
        self._check(_lib.morse_batch_shape_of(self._h, int(n_ep),
                                              ctypes.byref(grid), map_._h,
                                              ctypes.byref(sh)),
                    "morse_batch_shape_of")
        return {f: getattr(sh, f) for f, _ in BatchShape._fields_}

    def grid_chi2_noalloc(self, event, map_, grid: Grid) -> np.ndarray:
        """Top-K search that allocates no device memory
        (morse_grid_chi2_noalloc): for callers that cannot have cudaMalloc
        or cudaFree run inside their loop.  Same results as grid_chi2."""
        out = np.zeros(grid.top_k, dtype=FIT_DTYPE)
        st = _lib.morse_grid_chi2_noalloc(self._h, event._h, map_._h,
                                          ctypes.byref(grid), _ptr(out))
        self._check(st, "morse_grid_chi2_noalloc")
        return out

    def grid_chi2_dense(self, event, map_, grid: Grid, first=0, count=None):
        if count is None:
            count = grid.size - first
        chi2 = np.zeros(count)
        fs = np.zeros(count)
        fb = np.zeros(count)
        st = _lib.morse_grid_chi2_dense(self._h, event._h, map_._h,
                                        ctypes.byref(grid), int(first),
                                        int(count), _ptr(chi2), _ptr(fs),
                                        _ptr(fb))
        self._check(st, "morse_grid_chi2_dense")
        return chi2, fs, fb

    def search(self, t, flux, sigma, t_ref, s, q, extent, npix,
               rays_per_axis, grid: Grid, image_halfwidth=None,
               deflect="fp32"):
        """End-to-end from host buffers (morse_search)."""
        t, flux, sigma = _f64(t), _f64(flux), _f64(sigma)
        opts = MapOpts(float(image_halfwidth or 0.0),
                       DEFLECT_FP64 if deflect == "fp64" else DEFLECT_FP32,
                       STORE_FP32)
        out = np.zeros(grid.top_k, dtype=FIT_DTYPE)
        st = _lib.morse_search(self._h, _ptr(t), _ptr(flux), _ptr(sigma),
                               len(t), float(t_ref), float(s), float(q),
                               float(extent), int(npix), int(rays_per_axis),
                               ctypes.byref(opts), ctypes.byref(grid),
                               _ptr(out))
        self._check(st, "morse_search")
        return out

    def sweep(self, event, s, q, extent, npix, rays_per_axis, grid: Grid,
              image_halfwidth=None, deflect="fp32", fp16log=False,
              generator="rays"):
        """Full (s, q) search of a device-resident event (morse_sweep):
        returns fits[n_maps, top_k].  fp16log: search each map through its
        FP16 log10 table; generator="poly": maps from the lens polynomial."""
        s, q = _f64(s), _f64(q)
        if len(s) != len(q):
            raise ValueError("s and q lists differ in length")
        opts = MapOpts(float(image_halfwidth or 0.0),
                       DEFLECT_FP64 if deflect == "fp64" else DEFLECT_FP32,
                       STORE_FP32 | (STORE_FP16LOG if fp16log else 0),
                       GEN_POLY if generator == "poly" else GEN_RAYS)
        out = np.zeros((len(s), grid.top_k), dtype=FIT_DTYPE)
        st = _lib.morse_sweep(self._h, event._h, _ptr(s), _ptr(q), len(s),
                              float(extent), int(npix), int(rays_per_axis),
                              ctypes.byref(opts), ctypes.byref(grid),
                              _ptr(out))
        self._check(st, "morse_sweep")
        return out

    def search_sweep(self, t, flux, sigma, t_ref, s, q, extent, npix,
                     rays_per_axis, grid: Grid, image_halfwidth=None,
                     deflect="fp32", fp16log=False, generator="rays"):
        """morse_search_sweep: the full (s, q) search from host buffers."""
        t, flux, sigma = _f64(t), _f64(flux), _f64(sigma)
        s, q = _f64(s), _f64(q)
        if len(s) != len(q):
            raise ValueError("s and q lists differ in length")
        opts = MapOpts(float(image_halfwidth or 0.0),
                       DEFLECT_FP64 if deflect == "fp64" else DEFLECT_FP32,
                       STORE_FP32 | (STORE_FP16LOG if fp16log else 0),
                       GEN_POLY if generator == "poly" else GEN_RAYS)
        out = np.zeros((len(s), grid.top_k), dtype=FIT_DTYPE)
        st = _lib.morse_search_sweep(self._h, _ptr(t), _ptr(flux),
                                     _ptr(sigma), len(t), float(t_ref),
                                     _ptr(s), _ptr(q), len(s), float(extent),
                                     int(npix), int(rays_per_axis),
                                     ctypes.byref(opts), ctypes.byref(grid),
                                     _ptr(out))
        self._check(st, "morse_search_sweep")
        return out

    # ------------------------------------------------------------ gradient
    def chi2_grad(self, event, map_, theta):
        """chi^2, d chi^2/d(t0, tE, u0, alpha), Fs, Fb of trajectories
        theta[n, 4] (morse_chi2_grad)."""
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, 4)
        n = th.shape[0]
        chi2 = np.zeros(n)
        grad = np.zeros((n, 4))
        fs = np.zeros(n)
        fb = np.zeros(n)
        st = _lib.morse_chi2_grad(self._h, event._h, map_._h, _ptr(th), n,
                                  _ptr(chi2), _ptr(grad), _ptr(fs), _ptr(fb))
        self._check(st, "morse_chi2_grad")
        return chi2, grad, fs, fb

    def chi2_grad_dev(self, event, map_, theta, chi2, grad=None):
        """Device version on torch float64 CUDA tensors (theta [n, 4],
        chi2 [n], grad [n, 4] or None), queued on the context's stream."""
        for x in (theta, chi2) + ((grad,) if grad is not None else ()):
            if not (x.is_cuda and x.is_contiguous()) or str(x.dtype) != \
                    "torch.float64":
                raise ValueError("contiguous float64 CUDA tensors expected")
        n = theta.shape[0]
        st = _lib.morse_chi2_grad_dev(
            self._h, event._h, map_._h, ctypes.c_void_p(theta.data_ptr()), n,
            ctypes.c_void_p(chi2.data_ptr()),
            ctypes.c_void_p(grad.data_ptr()) if grad is not None else None)
        self._check(st, "morse_chi2_grad_dev")

    def refine(self, event, map_, starts, iters=50, method=REFINE_LM):
        """Batched Levenberg-Marquardt refinement of fit records
        (morse_refine)."""
        st_ = np.ascontiguousarray(starts, dtype=FIT_DTYPE)
        out = np.zeros(len(st_), dtype=FIT_DTYPE)
        st = _lib.morse_refine(self._h, event._h, map_._h, _ptr(st_),
                               len(st_), int(iters), int(method), _ptr(out))
        self._check(st, "morse_refine")
        return out

    def refine_batch(self, event, maps, map_of, starts, iters=50,
                     method=REFINE_LM):
        """morse_refine of starts on several maps at once
        (morse_refine_batch): start i on maps[map_of[i]]."""
        st_ = np.ascontiguousarray(starts, dtype=FIT_DTYPE)
        mo = np.ascontiguousarray(map_of, dtype=np.int32)
        mp = (ctypes.c_void_p * len(maps))(*[m._h for m in maps])
        out = np.zeros(len(st_), dtype=FIT_DTYPE)
        st = _lib.morse_refine_batch(self._h, event._h, mp, len(maps),
                                     _ptr(mo), _ptr(st_), len(st_),
                                     int(iters), int(method), _ptr(out))
        self._check(st, "morse_refine_batch")
        return out

    def lightcurve(self, map_, t0, tE, u0, alpha, t):
        t = _f64(t)
        out = np.zeros(len(t))
        st = _lib.morse_lightcurve(self._h, map_._h, float(t0), float(tE),
                                   float(u0), float(alpha), _ptr(t), len(t),
                                   _ptr(out))
        self._check(st, "morse_lightcurve")
        return out

    def exact_sweeps(self) -> int:
        """Trajectories given the exact residual sweep in the last search
        call (morse_last_search_stats)."""
        v = ctypes.c_uint64()
        self._check(_lib.morse_last_search_stats(self._h, ctypes.byref(v)),
                    "morse_last_search_stats")
        return int(v.value)

    def inject_fault(self, kind: int, arg: int = 0):
        """Make a bounded failure happen on purpose (morse_inject_fault):
        FAULT_LOCK_HELD (arg: spin limit) makes top-K searches give up their
        lock waits (ETIMEOUT); FAULT_ALLOC (arg: n) fails the n-th device
        allocation from now (ENOMEM); FAULT_NONE clears."""
        self._check(_lib.morse_inject_fault(self._h, int(kind), int(arg)),
                    "morse_inject_fault")

    def launch_count(self) -> int:
        v = ctypes.c_uint64()
        self._check(_lib.morse_launch_count(self._h, ctypes.byref(v)),
                    "morse_launch_count")
        return int(v.value)

    def kernel_ms(self, which: int) -> float:
        v = ctypes.c_double()
        self._check(_lib.morse_last_kernel_ms(self._h, int(which),
                                              ctypes.byref(v)),
                    "morse_last_kernel_ms")
        return v.value


class Map:
    def __init__(self, ctx: Context, h):
        self.ctx, self._h = ctx, h
        n = ctypes.c_int()
        L = ctypes.c_double()
        s = ctypes.c_double()
        q = ctypes.c_double()
        ctx._check(_lib.morse_map_info(h, ctypes.byref(n), ctypes.byref(L),
                                       ctypes.byref(s), ctypes.byref(q)),
                   "morse_map_info")
        self.npix, self.extent, self.s, self.q = n.value, L.value, s.value, \
            q.value

    def counts(self):
        c = np.zeros((self.npix, self.npix), dtype=np.uint32)
        off = ctypes.c_uint64()
        lost = ctypes.c_uint64()
        self.ctx._check(_lib.morse_map_counts(self._h, _ptr(c),
                                              ctypes.byref(off),
                                              ctypes.byref(lost)),
                        "morse_map_counts")
        return c, int(off.value), int(lost.value)

    def values(self):
        A = np.zeros((self.npix, self.npix), dtype=np.float32)
        self.ctx._check(_lib.morse_map_values(self._h, _ptr(A)),
                        "morse_map_values")
        return A

    def finite_source(self, rho, gamma=0.53):
        """New map: this one convolved with a limb-darkened source of radius
        rho (Einstein radii), morse_map_finite_source."""
        h = ctypes.c_void_p()
        self.ctx._check(_lib.morse_map_finite_source(
            self.ctx._h, self._h, float(rho), float(gamma), ctypes.byref(h)),
            "morse_map_finite_source")
        return Map(self.ctx, h)

    def set_lookup(self, fp16log: bool):
        """Search through the FP16 log10 table (built on demand) or the
        FP32 values."""
        self.ctx._check(_lib.morse_map_set_lookup(
            self._h, STORE_FP16LOG if fp16log else STORE_FP32),
            "morse_map_set_lookup")

    def half(self):
        """(FP16 codes [npix, npix] uint16, A_floor)."""
        c = np.zeros((self.npix, self.npix), dtype=np.uint16)
        f = ctypes.c_double()
        self.ctx._check(_lib.morse_map_half(self._h, _ptr(c),
                                            ctypes.byref(f)),
                        "morse_map_half")
        return c, f.value

    def free(self):
        if self._h:
            _lib.morse_map_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self.ctx._h:
                self.free()
        except Exception:
            pass


class Event:
    def __init__(self, ctx: Context, h, n):
        self.ctx, self._h, self.n = ctx, h, n

    def free(self):
        if self._h:
            _lib.morse_event_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            if self.ctx._h:
                self.free()
        except Exception:
            pass


def chi2_function():
    """torch.autograd.Function computing chi^2(theta) per trajectory with
    the adjoint gradient (morse_chi2_grad_dev).  Usage:
        Chi2 = chi2_function(); chi2 = Chi2.apply(theta, ctx, event, map)
    theta: float64 CUDA tensor [n, 4] (t0, tE, u0, alpha)."""
    import torch

    class Chi2(torch.autograd.Function):
        @staticmethod
        def forward(fctx, theta, mctx, event, map_):
            theta = theta.detach().contiguous()
            chi2 = torch.empty(theta.shape[0], dtype=torch.float64,
                               device=theta.device)
            grad = torch.empty_like(theta)
            # order the library's stream after the producer of theta
            cur = torch.cuda.current_stream(theta.device)
            lib_stream = getattr(mctx, "_stream_ref", None)
            if lib_stream is not None:
                lib_stream.wait_stream(cur)
            mctx.chi2_grad_dev(event, map_, theta, chi2, grad)
            if lib_stream is not None:
                cur.wait_stream(lib_stream)
            else:
                torch.cuda.synchronize(theta.device)
            fctx.save_for_backward(grad)
            return chi2

        @staticmethod
        def backward(fctx, gout):
            (grad,) = fctx.saved_tensors
            return gout[:, None] * grad, None, None, None

    return Chi2


def topk_merge(lists, k):
    """Merge sorted top-K lists (FIT_DTYPE arrays) on the host."""
    arrs = [np.ascontiguousarray(a, dtype=FIT_DTYPE) for a in lists]
    ptrs = (ctypes.c_void_p * max(1, len(arrs)))(
        *[a.ctypes.data for a in arrs])
    counts = (ctypes.c_int * max(1, len(arrs)))(*[len(a) for a in arrs])
    out = np.zeros(k, dtype=FIT_DTYPE)
    st = _lib.morse_topk_merge(ptrs, counts, len(arrs), int(k), _ptr(out))
    if st != OK:
        raise MorseError(st, "morse_topk_merge")
    return out


__all__ = ["Context", "Map", "Event", "Grid", "Fit", "FIT_DTYPE", "MapOpts",
           "Caustic", "rphi_lines",
           "MorseError", "topk_merge", "chi2_function", "version",
           "LIB_PATH", "EXPORTED"]
