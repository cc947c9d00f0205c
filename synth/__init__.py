"""Seeded synthetic inputs shaped like survey-plus-follow-up microlensing data.

This module is shared by the oracle tests, the CUDA-path tests and the
benchmark.  It holds none of the method's arithmetic: no lens equation, no
magnification, no flux model, no fit.  Callers pass in the noise-free flux
they computed themselves (oracle or library); this module only draws the
observing times, the photometric noise and the outliers.

Recipe (stand-in for the OGLE/MOA/follow-up light curves of the paper's
examples, which are not available here):

* times: nightly 8-h observing windows every 24 h over [-40, 40] d, 15-min
  slots jittered by U(-2, 2) min; N epochs drawn without replacement, slots
  with |t - t_peak| < 2 d weighted 5x ("denser around the peak").  When N
  exceeds the slots of one site, further sites (windows offset by 8 h and
  16 h: 24-h coverage) are added and the slot length shrinks to
  15 * 7680 / N min until N fits.  Times are rounded to FP32-representable
  values (resolution ~4e-6 d at 40 d) unless the caller asks for raw FP64
  times (raw=True: real data carry times at full precision, e.g. HJD).
* noise: sigma = 0.01 sqrt(F_true) + 0.002, F = F_true + N(0, sigma^2).
* outliers: a seeded fraction of epochs shifted by +-5 sigma.

All draws use numpy's PCG64 generator seeded by the caller.
"""
from __future__ import annotations

import numpy as np

DAY_MIN = 1440.0


def _slots(n_sites: int, slot_min: float, span=(-40.0, 40.0),
           window_h: float = 8.0):
    lo, hi = span
    starts = []
    per_window = int(round(window_h * 60.0 / slot_min))
    for site in range(n_sites):
        off = site * window_h / 24.0
        day = lo
        while day + off < hi:
            w0 = day + off
            for m in range(per_window):
                tt = w0 + (m + 0.5) * slot_min / DAY_MIN
                if lo <= tt < hi:
                    starts.append(tt)
            day += 1.0
    return np.asarray(starts, dtype=np.float64)


def epoch_times(n: int, seed: int, t_peak: float = 0.0,
                span=(-40.0, 40.0), raw: bool = False) -> np.ndarray:
    """Sorted observing times (days) for an n-epoch light curve; rounded to
    FP32-representable values unless raw."""
    if n <= 0:
        return np.zeros(0)
    rng = np.random.Generator(np.random.PCG64(seed))
    n_sites, slot_min = 1, 15.0
    base = _slots(1, slot_min, span)
    if n > base.size:
        n_sites = 3
        base = _slots(3, slot_min, span)
        while n > base.size:
            slot_min = min(slot_min, 15.0 * base.size / n) * 0.98
            base = _slots(3, slot_min, span)
    jit = rng.uniform(-2.0, 2.0, size=base.size) / DAY_MIN
    cand = base + jit
    wgt = np.where(np.abs(cand - t_peak) < 2.0, 5.0, 1.0)
    pick = rng.choice(cand.size, size=n, replace=False, p=wgt / wgt.sum())
    t = np.sort(cand[pick])
    if raw:
        return t
    return t.astype(np.float32).astype(np.float64)


def photometry(f_true: np.ndarray, seed: int, outlier_frac: float = 0.0):
    """(flux, sigma) from noise-free flux: sigma = 0.01 sqrt(F) + 0.002,
    Gaussian noise, and a seeded fraction of +-5 sigma outliers."""
    f_true = np.asarray(f_true, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    sigma = 0.01 * np.sqrt(np.maximum(f_true, 0.0)) + 0.002
    flux = f_true + sigma * rng.standard_normal(f_true.size)
    n_out = int(round(outlier_frac * f_true.size))
    if n_out > 0:
        idx = rng.choice(f_true.size, size=n_out, replace=False)
        sign = rng.choice(np.array([-1.0, 1.0]), size=n_out)
        flux[idx] += 5.0 * sign * sigma[idx]
    return flux, sigma


def event_lengths(n_events: int, seed: int, lo: int = 200,
                  hi: int = 20000) -> np.ndarray:
    """Epoch counts log-uniform in [lo, hi] (uneven batched events)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n_events)).astype(
        np.int64)


def truth_draws(n_events: int, seed: int) -> list[dict]:
    """Per-event truth parameters for the uneven batch: s~logU[0.3,3],
    q~logU[1e-5,1e-1], u0~logU[1e-3,0.5], alpha~U[0,2pi), tE~logU[5,80] d,
    Fb/Fs~U[0,2], Fs = 1, t0 = 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_events):
        out.append(dict(
            s=float(np.exp(rng.uniform(np.log(0.3), np.log(3.0)))),
            q=float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-1)))),
            u0=float(np.exp(rng.uniform(np.log(1e-3), np.log(0.5)))),
            alpha=float(rng.uniform(0.0, 2.0 * np.pi)),
            tE=float(np.exp(rng.uniform(np.log(5.0), np.log(80.0)))),
            t0=0.0, Fs=1.0, Fb=float(rng.uniform(0.0, 2.0))))
    return out


# Workload shapes (sizes of the configurations measured and tested).
CFG0 = dict(s=1.0, q=1e-3, L=2.0, npix=512, nray=4000, X=3.0, fp64=True,
            t0=0.0, tE=20.0, u0=0.05, alpha=0.7, Fs=1.0, Fb=0.3, n=500,
            seed=0, outliers=0.0,
            grid=dict(n_u0=20, n_alpha=36, n_t0=10, n_tE=10, u0_lo=1e-3,
                      u0_hi=0.5, t0_lo=-2.0, t0_hi=2.0, tE_lo=5.0,
                      tE_hi=80.0, u0_log=True, tE_log=True),
            top_k=16)

CFG1 = dict(s_lo=0.3, s_hi=3.0, n_s=31, q_lo=1e-5, q_hi=1e-1, n_q=21, L=2.0,
            npix=1024, nray=10000, X=3.0, fp64=False, s=0.9, q=5e-4, t0=0.0,
            tE=20.0, u0=0.05, alpha=0.7, Fs=1.0, Fb=0.3, n=3000, seed=1,
            outliers=0.01,
            grid=dict(n_u0=40, n_alpha=72, n_t0=25, n_tE=20, u0_lo=1e-3,
                      u0_hi=0.5, t0_lo=-2.0, t0_hi=2.0, tE_lo=5.0,
                      tE_hi=80.0, u0_log=True, tE_log=True),
            top_k=256)


def sq_axes(cfg=CFG1):
    """The (s, q) outer grid: log-spaced s and q values."""
    s = np.exp(np.linspace(np.log(cfg["s_lo"]), np.log(cfg["s_hi"]),
                           cfg["n_s"]))
    q = np.exp(np.linspace(np.log(cfg["q_lo"]), np.log(cfg["q_hi"]),
                           cfg["n_q"]))
    return s, q


# Batched workload: 256 events of log-uniform length in [200, 20000] epochs
# (truths from truth_draws, light curves from the point-source polynomial
# by the caller), against a bank of 64 maps of 1024^2 texels over [-2, 2]^2
# with (s, q) log-uniform in [0.3, 3] x [1e-5, 1e-1], 200,000 trajectories
# per (event, map) pair: 25 u0 x 40 alpha x 20 t0 x 10 tE.
CFG3 = dict(n_events=256, len_lo=200, len_hi=20000, n_maps=64, L=2.0,
            npix=1024, nray=10000, X=3.0, seed=3,
            grid=dict(n_u0=25, n_alpha=40, n_t0=20, n_tE=10, u0_lo=1e-3,
                      u0_hi=0.5, t0_lo=-2.0, t0_hi=2.0, tE_lo=5.0,
                      tE_hi=80.0, u0_log=True, tE_log=True),
            top_k=16)


def bank_sq(n_maps: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """(s, q) of a map bank: log-uniform in [0.3, 3] x [1e-5, 1e-1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = np.exp(rng.uniform(np.log(0.3), np.log(3.0), n_maps))
    q = np.exp(rng.uniform(np.log(1e-5), np.log(1e-1), n_maps))
    return s, q
