"""Benchmark of the MORSE hot path on GB300.

Workload: the full (s, q) search of one event -- s 31 log-spaced in
[0.3, 3], q 21 log-spaced in [1e-5, 1e-1] (651 maps), each map 1024 x 1024
texels over [-2, 2]^2 from 10^4 x 10^4 FP32-deflected rays, a 3000-epoch
light curve, 40 u0 x 72 alpha x 25 t0 x 20 tE = 1.44 M trajectories per
map, top-K = 256.  One step = that whole search (morse_sweep): for each of
the 651 maps, ray shooting, counts -> texels, the trajectory chi^2 search,
the top-K merge and the fit records.  Under torchrun every rank searches
its own event (seeded by rank) over all 651 maps: no collective on the data
path, weak scaling.

Metric: trajectory-epoch chi^2 evaluations per second (whole job).  Also
reported: rays/s of the map build, the dominant kernel's roofline, the CPU
oracle on a bounded sample, and the end-to-end rate through
morse_search_sweep from host buffers.

`--impl reference` times the CPU oracle (the plain FP64 definition) on the
host cores, each step a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = ("trajectory-epoch chi^2 evals/s and rays/s (% of roofline); "
          "time-to-best-fit vs plain")
UNIT = "traj-epoch evals/s"
# FP32 instructions one trajectory-epoch evaluation needs by its definition:
# tau 1, y 2, pixel coords 2, floor/frac/convert 6, bilinear 6, normal-
# equation sums 3, residual sweep 2.  The residual sweep runs only for the
# trajectories the error-bounded closed form cannot discard, so the work the
# search does is 20 instructions per evaluation plus 2 for the exact-sweep
# fraction; the headline roofline counts that, and the 22-instruction
# figure is reported beside it.
ALG_INSTR_PER_EVAL = 22
ALG_INSTR_PRUNED = 20
# one bilinear gather of a 2x2 FP32 cell per trajectory-epoch
GATHER_BYTES_PER_EVAL = 16
# bytes per trajectory-epoch through the shared-memory data pipe as the
# search is built: the 16-byte cell from the band table and half of the
# 12-byte epoch record (one load serves a trajectory pair); the pipe moves
# 128 bytes per clock per SM
SMEM_BYTES_PER_EVAL = 22
SMEM_BYTES_PER_CLK_SM = 128
# adjoint, per trajectory-epoch: the chi^2 of the two sweeps (22, as the
# search) and 14 more for the gradient through the lookup (four FP32 sums
# in the map's pixel axes); the kernel recomputes the lookup in its second
# sweep instead of storing A, and takes the gradient in the map's pixel
# axes, about 37 FP32 instructions in all
ADJ_INSTR_PER_EVAL = 36
# ray shooting, per ray: ray coordinates 2, deflection of Eq. 2 through two
# lenses 12 (+ 2 reciprocals), binning 6; plus one shared-memory atomic
ALG_INSTR_PER_RAY = 22
FP32_LANES_PER_SM = 128
# the search kernel's sources: its traffic record holds while they match
KERNEL_SRC = [os.path.join(ROOT, "paper_1511_01157_gb300", "csrc", f)
              for f in ("k_search.cu", "search_common.cuh",
                        "search_group.cuh", "morse_internal.cuh")]
PROFILE = os.path.join(ROOT, "profiles", "k_search_cfg1.md")


def workload_config(cfg):
    g = cfg["grid"]
    return {
        "workload": "full (s,q) search of one 3000-epoch event: 31 s x 21 q "
                    "= 651 maps per step",
        "maps_per_step": cfg["n_s"] * cfg["n_q"],
        "npix": cfg["npix"], "extent": cfg["L"],
        "rays_per_map": cfg["nray"] ** 2, "deflect": "fp32",
        "epochs": cfg["n"],
        "trajectories_per_map": g["n_u0"] * g["n_alpha"] * g["n_t0"] *
        g["n_tE"], "top_k": cfg["top_k"],
        "grid": f'{g["n_u0"]}u0 x {g["n_alpha"]}alpha x {g["n_t0"]}t0 x '
                f'{g["n_tE"]}tE',
        "l2": "flushed between steps (256 MB write); each 16 MB map is "
              "built inside the step and read from L2 by design",
    }


def sq_lists(cfg):
    s_ax, q_ax = synth.sq_axes(cfg)
    S, Q = np.meshgrid(s_ax, q_ax, indexing="ij")
    return S.ravel().copy(), Q.ravel().copy()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200",
                 "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                rows.append((float(p[0]), float(p[1]), p[4], p[5], p[6],
                             p[7]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown",
                                "sw_thermal_slowdown", "sw_power_cap"),
                               r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(
            r[1] for r in rows), "samples": len(rows),
            "reasons": sorted(reasons)}


# ---------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for f in KERNEL_SRC:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of the search kernel from the committed ncu
    summary, valid only while the kernel source is unchanged."""
    if not os.path.exists(PROFILE):
        return None
    src_hash = kernel_source_hash()
    bytes_, h = None, None
    for line in open(PROFILE):
        if line.startswith("traffic_bytes_per_launch:"):
            try:
                bytes_ = float(line.split(":", 1)[1])
            except ValueError:
                bytes_ = None
        if line.startswith("kernel_source_sha256_16:"):
            h = line.split(":", 1)[1].strip()
    if h != src_hash:
        return None
    return bytes_


def make_event(ctx, m, cfg, seed):
    """Synthetic 3000-epoch light curve: the truth magnification is read
    through the library from a map of the truth lens (self-consistent
    injection), then noise and outliers are drawn by ``synth``."""
    truth = ctx.build_map(cfg["s"], cfg["q"], cfg["L"], cfg["npix"],
                          cfg["nray"], image_halfwidth=cfg["X"],
                          deflect="fp32")
    t = synth.epoch_times(cfg["n"], seed, cfg["t0"])
    A = ctx.lightcurve(truth, cfg["t0"], cfg["tE"], cfg["u0"], cfg["alpha"],
                       t)
    F, sig = synth.photometry(cfg["Fs"] * A + cfg["Fb"], seed,
                              cfg["outliers"])
    truth.free()
    return t, F, sig


def grid_of(m, cfg, top_k=None):
    g = cfg["grid"]
    return m.Grid.make(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"],
                       g["u0_lo"], g["u0_hi"], g["t0_lo"], g["t0_hi"],
                       g["tE_lo"], g["tE_hi"], g["u0_log"], g["tE_log"],
                       cfg["top_k"] if top_k is None else top_k)


def grid_lines(cfg):
    """The (u0, alpha) lines of the config-1 grid as (u, alpha, shift)."""
    g = cfg["grid"]
    u0v = np.exp(np.linspace(np.log(g["u0_lo"]), np.log(g["u0_hi"]),
                             g["n_u0"]))
    return np.array([(u, 2 * np.pi * k / g["n_alpha"], 0.0) for u in u0v
                     for k in range(g["n_alpha"])])


def inside_samples(lines, L, h):
    """Samples every h of each line's part inside the map |y1|, |y2| < L
    (the peak library's work), from the slab geometry."""
    tot = 0.0
    for u, al, _ in lines:
        c, s = math.cos(al), math.sin(al)
        lo, hi = -math.inf, math.inf
        for a, b in ((c, -u * s), (s, u * c)):  # |a tau + b| < L
            if abs(a) > 1e-15:
                t0, t1 = (-L - b) / a, (L - b) / a
                lo, hi = max(lo, min(t0, t1)), min(hi, max(t0, t1))
            elif abs(b) >= L:
                hi = lo
        tot += max(0.0, hi - lo) / h
    return tot


def peak_library(ctx, m, cfg, delta=0.1, max_peaks=8):
    """§4.3 (iii) peak library of one config-1 map over the grid's 2880
    (u0, alpha) lines, two samples per texel: time per library (the C-ABI
    call, device synchronised) and samples per second."""
    import torch
    mp = ctx.build_map(cfg["s"], cfg["q"], cfg["L"], cfg["npix"], cfg["nray"],
                       image_halfwidth=cfg["X"], deflect="fp32")
    lines = grid_lines(cfg)
    times, kt = [], []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        count, _, _ = ctx.line_peaks(mp, lines, sub=2, max_peaks=max_peaks,
                                     delta=delta)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        kt.append(ctx.kernel_ms(7))  # the launch alone (CUDA events)
    mp.free()
    h = 2.0 * cfg["L"] / cfg["npix"] / 2
    n = inside_samples(lines, cfg["L"], h)
    t = min(times)
    # the libraries of 64 maps of the (s, q) grid in one launch
    S, Q = sq_lists(cfg)
    pick = np.linspace(0, len(S) - 1, 64).round().astype(int)
    maps = [ctx.build_map(S[j], Q[j], cfg["L"], cfg["npix"], cfg["nray"],
                          image_halfwidth=cfg["X"], deflect="fp32")
            for j in pick]
    tb, ktb = [], []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cb, _, _ = ctx.line_peaks_batch(maps, lines, sub=2,
                                        max_peaks=max_peaks, delta=delta)
        torch.cuda.synchronize()
        tb.append(time.perf_counter() - t0)
        ktb.append(ctx.kernel_ms(7))
    for mp in maps:
        mp.free()
    # ALU roofline of a sample: about 20 FP32 instructions (its position,
    # the clamps, the bilinear lookup and the comparisons) on every lane
    # of every SM at the maximum clock
    pk, pk_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = float(pk.get("sm_max_mhz", 2070.0))
    roof = sms * 128 * mhz * 1e6 / 20.0
    bk = 64 * n / min(ktb) * 1e3
    return {"lines": len(lines), "ms": 1e3 * t, "samples": n,
            "samples_per_s": n / t, "delta": delta,
            "kernel_ms": min(kt), "kernel_samples_per_s": n / min(kt) * 1e3,
            "median_peaks_per_line": float(np.median(count)),
            "mean_peaks_per_line": float(np.mean(count)),
            "max_peaks_per_line": int(count.max()),
            "batch_mean_peaks_per_line": float(np.mean(cb)),
            "batch_64_maps_ms": 1e3 * min(tb),
            "batch_samples_per_s": 64 * n / min(tb),
            "batch_kernel_ms": min(ktb),
            "batch_kernel_samples_per_s": bk,
            "roofline": {"bound": "alu", "achieved": bk, "peak": roof,
                         "unit": "samples/s", "frac": bk / roof,
                         "peak_source": f"{sms} SMs x 128 FP32 lanes x "
                                        f"{mhz} MHz ({pk_kind} sm_max_mhz)"
                                        " / 20 instructions per sample",
                         "kernel": "k_line_peaks, the 64-map launch"},
            "note": "samples of the lines inside the map, every half "
                    "texel; the batch is one launch over 64 maps' lines; "
                    "ms: the C-ABI call, device synchronised (host copies "
                    "of the results included); kernel_ms: the launch "
                    "alone, CUDA events"}


def adjoint_section(ctx, m, cfg, ev, n_ep, stream, probes, peak_instr_s,
                    n=4096, iters=50):
    """Adjoint gradient and refinement on the truth map of the config-1
    event: n = 4096 trajectories scattered about the truth (the refinement
    workload's start count).  chi^2 and its gradient by morse_chi2_grad_dev
    (device buffers, CUDA events on the context's stream), evals/s against
    the FP32-issue roofline and the L1 gather roofline.  The adjoint sweeps
    the epochs twice (the sums of the 2x2 solve, then the residuals and the
    gradient: the residual form keeps the gradient exact near the minimum,
    where sums of large terms would cancel), so an evaluation is 22 + 36
    FP32 instructions and two 16-byte gathers.  Then `iters`
    Levenberg-Marquardt iterations of all n (morse_refine, a CUDA graph per
    iteration) timed end to end.  The roofline counts 36 FP32 instructions
    per evaluation (chi^2 22 + gradient 14); the earlier accounting of two
    full sweeps (22 + 36) is reported beside it."""
    import torch
    mp = ctx.build_map(cfg["s"], cfg["q"], cfg["L"], cfg["npix"], cfg["nray"],
                       image_halfwidth=cfg["X"], deflect="fp32")
    rng = np.random.default_rng(5)
    th = np.stack([cfg["t0"] + rng.uniform(-1.0, 1.0, n),
                   cfg["tE"] * np.exp(rng.uniform(-0.3, 0.3, n)),
                   cfg["u0"] * np.exp(rng.uniform(-0.5, 0.5, n)),
                   cfg["alpha"] + rng.uniform(-0.2, 0.2, n)], axis=1)
    def grad_ms(th_):
        theta = torch.tensor(th_, dtype=torch.float64, device="cuda")
        nn = theta.shape[0]
        chi2 = torch.empty(nn, dtype=torch.float64, device="cuda")
        grad = torch.empty((nn, 4), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(3):
                ctx.chi2_grad_dev(ev, mp, theta, chi2, grad)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            reps = 10
            e0.record(stream)
            for _ in range(reps):
                ctx.chi2_grad_dev(ev, mp, theta, chi2, grad)
            e1.record(stream)
            e1.synchronize()
        return e0.elapsed_time(e1) / reps
    ms = grad_ms(th)
    evals = n * n_ep / (ms * 1e-3)
    # the same trajectories 32 times over: enough warps to fill the GPU
    ms_big = grad_ms(np.tile(th, (32, 1)))
    evals_big = 32 * n * n_ep / (ms_big * 1e-3)
    peak_instr = peak_instr_s / ADJ_INSTR_PER_EVAL
    peak_instr_58 = peak_instr_s / 58.0
    peak_gather = probes["l1_gather_bytes_per_s"] / 32.0
    starts = np.zeros(n, dtype=m.FIT_DTYPE)
    starts["t0"], starts["tE"], starts["u0"], starts["alpha"] = th.T
    starts["chi2"] = np.inf
    ctx.refine(ev, mp, starts[:64], iters=2)  # warm (graph capture)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = ctx.refine(ev, mp, starts, iters=iters)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t0
    mp.free()
    return {"trajectories": n, "epochs": n_ep, "grad_ms": ms,
            "grad_evals_per_s": evals,
            "frac_fp32_issue": evals / peak_instr,
            "frac_fp32_issue_58": evals / peak_instr_58,
            "frac_l1_gather": evals / peak_gather,
            "grad_evals_per_s_131072": evals_big,
            "frac_fp32_issue_131072": evals_big / peak_instr,
            "frac_fp32_issue_58_131072": evals_big / peak_instr_58,
            "roofline_note": f"{ADJ_INSTR_PER_EVAL} FP32 instr per "
                             "evaluation (chi^2 22 + gradient 14) against "
                             "152 x 128 lanes x max clock; _58: two full "
                             "sweeps counted (22 + 36); gather: 2 x 16 B "
                             "against the measured L1 random gather",
            "refine_iters": iters, "refine_s": t_ref,
            "refine_iters_per_s": n * iters / t_ref,
            "refine_median_chi2": float(np.median(out["chi2"]))}


def fp16_section(ctx, m, cfg, ev, sizes=(1024, 2048, 4096), reps=3):
    """FP16 log10(A) against FP32 A tables: the config-1 search (one map of
    the truth lens, 1.44 M trajectories x 3000 epochs, top-256) at three
    map sizes over [-2, 2]^2, rays scaled with the texel count (10^8 at
    1024^2).  Device time of the search kernels per call (CUDA events on
    the context stream), best of `reps`, and the best chi^2 of each."""
    out = {}
    grid = grid_of(m, cfg)
    for npix in sizes:
        nray = int(cfg["nray"] * npix / 1024)
        mp = ctx.build_map(cfg["s"], cfg["q"], cfg["L"], npix, nray,
                           image_halfwidth=cfg["X"], deflect="fp32",
                           fp16log=True)
        row = {}
        for name, h16 in (("fp32", False), ("fp16", True)):
            mp.set_lookup(h16)
            ctx.grid_chi2(ev, mp, grid)  # warm
            best, chi = None, None
            for _ in range(reps):
                r = ctx.grid_chi2(ev, mp, grid)
                ms = ctx.kernel_ms(2)
                best = ms if best is None else min(best, ms)
                chi = float(r["chi2"][0])
            row[name] = {"search_ms": best, "best_chi2": chi}
        row["fp16_over_fp32_time"] = row["fp16"]["search_ms"] / \
            row["fp32"]["search_ms"]
        row["table_MB"] = {"fp32": 16 * (npix + 1) * (npix + 8) / 1e6,
                           "fp16": 8 * (npix + 1) * (npix + 8) / 1e6}
        out[f"{npix}^2"] = row
        mp.free()
    return out


def config2_section(ctx, m, cfg, ev, S, Q, fits, n_starts=4096, iters=50):
    """Configuration 2: Levenberg-Marquardt refinement (adjoint gradient,
    Gauss-Newton matrix, one CUDA graph per iteration) of the n_starts
    lowest-chi^2 grid minima of the 651-map config-1 sweep (the top-256
    lists of every map), 50 iterations.  The maps those minima lie on are
    built and kept resident together (17 MB each), and every start refines
    in one morse_refine_batch call on its own map.  Reported: wall time
    with the map builds, the refine call alone, and the chi^2 reached."""
    import torch
    flat = fits.reshape(-1)
    mi = np.repeat(np.arange(fits.shape[0]), fits.shape[1])
    ok = np.flatnonzero(flat["idx"] >= 0)
    pick = ok[np.argsort(flat["chi2"][ok], kind="stable")[:n_starts]]
    maps = np.unique(mi[pick])
    slot = {int(j): k for k, j in enumerate(maps)}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    built = [ctx.build_map(S[j], Q[j], cfg["L"], cfg["npix"], cfg["nray"],
                           image_halfwidth=cfg["X"], deflect="fp32")
             for j in maps]
    seeds = flat[pick]
    map_of = np.array([slot[int(j)] for j in mi[pick]], dtype=np.int32)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    out = ctx.refine_batch(ev, built, map_of, seeds, iters=iters)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t1
    wall = time.perf_counter() - t0
    for mp in built:
        mp.free()
    gain = 1.0 - out["chi2"] / seeds["chi2"]
    return {"starts": int(len(pick)), "maps": int(len(maps)),
            "iterations": iters, "wall_s": wall, "refine_s": t_ref,
            "trajectory_iterations_per_s": len(pick) * iters / t_ref,
            "best_grid_chi2": float(seeds["chi2"].min()),
            "best_refined_chi2": float(out["chi2"].min()),
            "median_relative_chi2_drop": float(np.median(gain)),
            "never_increased": bool(np.all(out["chi2"] <= seeds["chi2"] *
                                           (1 + 1e-12)))}


def batch_events(ctx, m, cfg, n_events):
    """Light curves of the batched workload: lengths log-uniform in
    [200, 20000], truths from synth.truth_draws, magnification read through
    the library from a map of each truth lens (self-consistent injection),
    noise as config 0."""
    lens = synth.event_lengths(n_events, cfg["seed"], cfg["len_lo"],
                               cfg["len_hi"])
    truths = synth.truth_draws(n_events, cfg["seed"])
    evs = []
    for i, (n, tr) in enumerate(zip(lens, truths)):
        mp = ctx.build_map(tr["s"], tr["q"], cfg["L"], cfg["npix"],
                           cfg["nray"], image_halfwidth=cfg["X"],
                           deflect="fp32")
        t = synth.epoch_times(int(n), cfg["seed"] * 1000 + i, tr["t0"])
        A = ctx.lightcurve(mp, tr["t0"], tr["tE"], tr["u0"], tr["alpha"], t)
        mp.free()
        F, sig = synth.photometry(tr["Fs"] * A + tr["Fb"],
                                  cfg["seed"] * 1000 + i)
        evs.append(ctx.event(t, F, sig, t_ref=0.0))
    return evs, lens


def run_batched(ctx, m, n_events, n_maps, tune=True):
    """The batched search (one persistent launch per call, CUDA graph) on a
    subset of the 256-event x 64-map workload, against one morse_grid_chi2
    call per (event, map) pair on the same inputs."""
    import torch
    cfg = synth.CFG3
    evs, lens = batch_events(ctx, m, cfg, n_events)
    S, Q = synth.bank_sq(n_maps, cfg["seed"])
    maps = [ctx.build_map(S[j], Q[j], cfg["L"], cfg["npix"], cfg["nray"],
                          image_halfwidth=cfg["X"], deflect="fp32")
            for j in range(n_maps)]
    g = cfg["grid"]
    grid = m.Grid.make(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"],
                       g["u0_lo"], g["u0_hi"], g["t0_lo"], g["t0_hi"],
                       g["tE_lo"], g["tE_hi"], g["u0_log"], g["tE_log"],
                       cfg["top_k"])
    evals = float(grid.size) * float(np.sum(lens)) * n_maps
    ctx.batch_tuning(tune)
    t0 = time.perf_counter()
    out = ctx.grid_chi2_batch(evs, maps, grid)  # first call tunes
    first = time.perf_counter() - t0
    walls, search = [], []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.grid_chi2_batch(evs, maps, grid)
        walls.append(time.perf_counter() - t0)
        search.append(ctx.kernel_ms(2))
    exact = ctx.exact_sweeps()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    same = True
    for e, ev in enumerate(evs):
        for j, mp in enumerate(maps):
            one = ctx.grid_chi2(ev, mp, grid)
            same &= bool(np.array_equal(one["idx"], out[e, j]["idx"]) and
                         np.array_equal(one["chi2"], out[e, j]["chi2"]))
    plain = time.perf_counter() - t0
    shapes = {}
    for b in sorted({int(np.log2(n)) for n in lens}):
        sh = ctx.batch_shape(2 ** b, grid, maps[0])
        shapes[f"2^{b}"] = f"tpg {sh['tpg']} rounds {sh['rounds']} " \
                           f"stage {sh['stage']}"
    for mp in maps:
        mp.free()
    for ev in evs:
        ev.free()
    return {
        "workload": f"{n_events} events (lengths log-uniform in [200, 20000]"
                    f", {int(np.sum(lens))} epochs) x {n_maps} maps of "
                    f"1024^2 x {grid.size} trajectories per pair, top-K "
                    f"{cfg['top_k']} (subset of 256 x 64)",
        "evals_per_call": evals,
        "batch_s": min(walls), "batch_evals_per_s": evals / min(walls),
        "batch_search_ms": float(min(search)),
        "first_call_s_with_tuning": first,
        "per_pair_calls_s": plain, "per_pair_evals_per_s": evals / plain,
        "identical_to_per_pair": same,
        "exact_sweep_fraction": exact / (grid.size * n_events * n_maps),
        "tuned_shapes": shapes,
    }


def refine_best(ctx, m, cfg, ev, S, Q, fits, n_maps=8, iters=40):
    """Levenberg-Marquardt refinement (adjoint gradient) of the top seeds
    of the n_maps maps with the lowest grid chi^2; returns the best chi^2."""
    best = np.inf
    for j in np.argsort(fits["chi2"][:, 0])[:n_maps]:
        mp = ctx.build_map(S[j], Q[j], cfg["L"], cfg["npix"], cfg["nray"],
                           image_halfwidth=cfg["X"], deflect="fp32")
        seeds = fits[j][:16]
        r = ctx.refine(ev, mp, seeds[np.isfinite(seeds["chi2"])], iters=iters)
        best = min(best, float(r["chi2"].min()))
        mp.free()
    return best


def standalone_rays(ctx, cfg, S, Q, n_maps=16):
    """Ray-shooting kernel time with nothing else on the GPU: n_maps of the
    sweep's maps built one at a time (the sweep builds map i + 1 while map
    i is searched, so its per-kernel times include waits for SMs).  Returns
    rays/s over the kernels' CUDA-event time."""
    import torch
    pick = np.linspace(0, len(S) - 1, n_maps).round().astype(int)
    ms = 0.0
    for j in pick:
        mp = ctx.build_map(S[j], Q[j], cfg["L"], cfg["npix"], cfg["nray"],
                           image_halfwidth=cfg["X"], deflect="fp32")
        ms += ctx.kernel_ms(0)
        mp.free()
    torch.cuda.synchronize()
    return n_maps * float(cfg["nray"]) ** 2 / (ms * 1e-3), n_maps


def map_generators(ctx, m, cfg, n_maps=4):
    """The two map generators on config-1 maps (1024^2 over [-2, 2]^2):
    inverse ray shooting of 10^8 FP32 rays and the lens polynomial solved
    in FP64 at every texel centre (the paper's generator), wall time per
    map with the device synchronised."""
    import torch
    S, Q = sq_lists(cfg)
    pick = np.linspace(0, len(S) - 1, n_maps).round().astype(int)
    out = {}
    for gen in ("rays", "poly"):
        times = []
        for j in pick:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            mp = ctx.build_map(S[j], Q[j], cfg["L"], cfg["npix"], cfg["nray"],
                               image_halfwidth=cfg["X"], deflect="fp32",
                               generator=gen)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            mp.free()
        ms = 1e3 * float(np.median(times[1:] if len(times) > 1 else times))
        out[gen] = {"ms_per_map": ms,
                    "texels_per_s": cfg["npix"] ** 2 / (ms * 1e-3)}
    out["rays"]["rays_per_s"] = cfg["nray"] ** 2 / (out["rays"]["ms_per_map"]
                                                   * 1e-3)
    out["maps"] = f"{n_maps} (s, q) of the 651, {cfg['npix']}^2 texels"
    return out


def finite_source_maps(ctx, m, cfg, gamma=0.53):
    """The paper's finite-source set on one config-1 map: seven source
    radii log-spaced over (0.001, 1) Einstein radii, limb darkening 0.53;
    wall time per convolution and multiply-adds per second."""
    import torch
    mp = ctx.build_map(cfg["s"], cfg["q"], cfg["L"], cfg["npix"], cfg["nray"],
                       image_halfwidth=cfg["X"], deflect="fp32")
    dlt = 2.0 * cfg["L"] / cfg["npix"]
    rows = []
    for rho in np.exp(np.linspace(np.log(1e-3), np.log(1.0), 7)):
        times = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fs = mp.finite_source(rho, gamma)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            fs.free()
        R = int(math.ceil(rho / dlt + 0.5))
        taps = math.pi * (rho / dlt) ** 2 if rho / dlt > 0.5 else 1.0
        t = min(times)
        rows.append({"rho": float(rho), "R_texels": R, "ms": 1e3 * t,
                     "fma_per_s": taps * cfg["npix"] ** 2 / t})
    mp.free()
    return {"map": f"{cfg['npix']}^2 texels, (s, q) = ({cfg['s']}, "
                   f"{cfg['q']})", "gamma": gamma, "radii": rows}


def peak_time(t, F):
    """The peak time read off a light curve: the largest running median of
    7 epochs."""
    order = np.argsort(np.asarray(t))
    tt, ff = np.asarray(t)[order], np.asarray(F)[order]
    med = np.array([np.median(ff[max(0, i - 3): i + 4])
                    for i in range(len(tt))])
    return float(tt[np.argmax(med)])


def peak_grid(m, cfg, n_lines):
    g = cfg["grid"]
    return m.Grid.make(2 * n_lines, 1, 3, g["n_tE"], 1.0, 1.0, -0.05, 0.05,
                       g["tE_lo"], g["tE_hi"], False, g["tE_log"], 16)


def peak_aligned_fits(ctx, m, cfg, ev, S, Q, t_peak):
    """§4.3 (iii)-(iv): on every (u0, alpha) line of the grid the
    trajectories whose two highest map peaks (threshold 10%) come at t_peak
    (Eq. 7), 3 t0 offsets within +-0.05 d and the grid's 20 tE, on each
    map; [n_maps, 16] records."""
    lines = grid_lines(cfg)
    pgrid = peak_grid(m, cfg, len(lines))
    fits = []
    for j in range(len(S)):
        mp = ctx.build_map(S[j], Q[j], cfg["L"], cfg["npix"], cfg["nray"],
                           image_halfwidth=cfg["X"], deflect="fp32")
        fits.append(ctx.peak_search(ev, mp, pgrid, lines, tp=[t_peak],
                                    min_peaks=1, sub=2, max_peaks=2,
                                    delta=0.1))
        mp.free()
    return np.stack(fits)


def time_to_best_fit(ctx, m, cfg, ev, S, Q, plain_s, plain_fits, ev_t,
                     ev_flux, ev_sigma):
    """Wall time of each form of the (s, q) search and its best chi^2; a
    form reaches the best fit when its chi^2 is within 1e-3 of the lowest
    chi^2 any form found.  Forms: the plain FP32 grid (timed above), the
    same grid on FP16 log10 tables, the plain grid followed by adjoint
    (Levenberg-Marquardt) refinement of its best seeds, a coarse screen of
    the maps, the grid under the minimum-magnification cut, trajectories
    aligned with the light curve's peak by the peak library, and grids 3.8x
    and 15x coarser, each followed by the same refinement."""
    import torch
    g = cfg["grid"]

    def sweep(grid, fp16=False):
        return ctx.sweep(ev, S, Q, cfg["L"], cfg["npix"], cfg["nray"], grid,
                         image_halfwidth=cfg["X"], deflect="fp32",
                         fp16log=fp16)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v = fn()
        torch.cuda.synchronize()
        return v, time.perf_counter() - t0

    forms = {"plain_fp32_grid": (plain_s, float(plain_fits["chi2"].min()),
                                 "40x72x25x20 grid, 651 maps")}
    f16, t = timed(lambda: sweep(grid_of(m, cfg), True))
    forms["fp16_grid"] = (t, float(f16["chi2"].min()),
                          "same grid on FP16 log10 tables")
    b, t = timed(lambda: refine_best(ctx, m, cfg, ev, S, Q, plain_fits))
    forms["plain_grid_plus_refine"] = (
        plain_s + t, b, "plain grid, then 40 LM iterations on the 16 best "
        "seeds of the 8 best maps")
    coarse = m.Grid.make(20, 36, 13, 10, g["u0_lo"], g["u0_hi"], g["t0_lo"],
                         g["t0_hi"], g["tE_lo"], g["tE_hi"], True, True, 16)

    def screened():
        # coarse screen of all maps, the full grid on the 256 best (of 64,
        # 128, 192 and 256 kept, the smallest that keeps the best map of
        # this event), refine
        first = sweep(coarse)
        best = np.sort(np.argsort(first["chi2"][:, 0])[:256])
        fine = ctx.sweep(ev, S[best].copy(), Q[best].copy(), cfg["L"],
                         cfg["npix"], cfg["nray"], grid_of(m, cfg),
                         image_halfwidth=cfg["X"], deflect="fp32")
        return refine_best(ctx, m, cfg, ev, S[best].copy(), Q[best].copy(),
                           fine)
    b, t = timed(screened)
    forms["screen_then_grid_plus_refine"] = (
        t, b, "20x36x13x10 grid on all 651 maps, the 40x72x25x20 grid on "
        "the 256 best maps, then 40 LM iterations on the 16 best seeds of "
        "the 8 best of those")
    def resident_batched():
        # every map built once and kept resident (about 25 MB each, 16 GB
        # for the 651), the coarse screen of all of them and the full grid
        # on the 256 best each as one batched launch, then the 16 best
        # seeds of the 8 best maps refined in one call
        built = [ctx.build_map(S[j], Q[j], cfg["L"], cfg["npix"],
                               cfg["nray"], image_halfwidth=cfg["X"],
                               deflect="fp32") for j in range(len(S))]
        first = ctx.grid_chi2_batch([ev], built, coarse)[0]
        best = np.sort(np.argsort(first["chi2"][:, 0])[:256])
        sub = [built[j] for j in best]
        fine = ctx.grid_chi2_batch([ev], sub, grid_of(m, cfg, top_k=16))[0]
        top = np.argsort(fine["chi2"][:, 0])[:8]
        seeds = np.concatenate([fine[j][:16] for j in top])
        map_of = np.repeat(np.arange(len(top)), 16).astype(np.int32)
        keep = np.isfinite(seeds["chi2"])
        r = ctx.refine_batch(ev, [sub[j] for j in top], map_of[keep],
                             seeds[keep], iters=40)
        for mp in built:
            mp.free()
        return float(r["chi2"].min())
    b, t = timed(resident_batched)
    forms["resident_batched_screen_grid_refine"] = (
        t, b, "all 651 maps built and kept resident; the 20x36x13x10 "
        "screen of all of them in one batched launch, the 40x72x25x20 grid "
        "on the 256 best in one batched launch, then 40 LM iterations of "
        "the 16 best seeds of the 8 best maps in one batched refine")
    # §4.3 (i): the smallest peak magnification the data allow when the
    # blend flux is not negative, F_peak / F_base with F_peak the largest
    # flux less 3 sigma and F_base the median of the faintest fifth
    Fs_, sg_ = np.asarray(ev_flux), np.asarray(ev_sigma)
    f_base = float(np.median(np.sort(Fs_)[: max(1, len(Fs_) // 5)]))
    a_min = float(np.max(Fs_ - 3.0 * sg_) / f_base)
    cut = m.Grid.make(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"],
                      g["u0_lo"], g["u0_hi"], g["t0_lo"], g["t0_hi"],
                      g["tE_lo"], g["tE_hi"], g["u0_log"], g["tE_log"],
                      cfg["top_k"], a_min)
    b, t = timed(lambda: refine_best(ctx, m, cfg, ev, S, Q, sweep(cut)))
    # share of lines the cut removes, on 8 evenly spaced maps
    shares = []
    for j in np.linspace(0, len(S) - 1, 8).round().astype(int):
        mp = ctx.build_map(S[j], Q[j], cfg["L"], cfg["npix"], cfg["nray"],
                           image_halfwidth=cfg["X"], deflect="fp32")
        shares.append(float(np.mean(ctx.line_max(mp, cut) < a_min)))
        mp.free()
    forms["cut_grid_plus_refine"] = (
        t, b, f"the 40x72x25x20 grid without the lines whose largest "
        f"magnification is below {a_min:.2f} (peak over baseline flux; "
        f"{100 * np.mean(shares):.1f}% of the lines on 8 sample maps), then "
        "the same refinement")
    # §4.3 (iii)-(iv): the peak time read off the light curve (the largest
    # running median of 7 epochs), and on every (u0, alpha) line of the grid
    # the trajectories whose two highest peaks come at it (Eq. 7), 3 t0
    # offsets within +-0.05 d and the grid's 20 tE
    t_peak = peak_time(ev_t, Fs_)
    lines = grid_lines(cfg)
    pgrid = peak_grid(m, cfg, len(lines))
    b, t = timed(lambda: refine_best(
        ctx, m, cfg, ev, S, Q,
        peak_aligned_fits(ctx, m, cfg, ev, S, Q, t_peak)))
    forms["peak_aligned_plus_refine"] = (
        t, b, f"peak time {t_peak:.3f} d from the light curve; on each of "
        f"the 2880 (u0, alpha) lines the trajectories whose two highest "
        f"map peaks (threshold 10%) come at it (Eq. 7), 3 t0 offsets x 20 "
        f"tE ({pgrid.size} trajectories per map, "
        f"{pgrid.size / grid_of(m, cfg).size:.0%} of the grid), then the "
        f"same refinement")
    for name, dims in (("half_grid_plus_refine", (40, 72, 13, 10)),
                       ("coarse_grid_plus_refine", (20, 36, 13, 10))):
        grid = m.Grid.make(*dims, g["u0_lo"], g["u0_hi"], g["t0_lo"],
                           g["t0_hi"], g["tE_lo"], g["tE_hi"], True, True, 16)
        b, t = timed(lambda: refine_best(ctx, m, cfg, ev, S, Q,
                                         sweep(grid)))
        forms[name] = (t, b, "x".join(map(str, dims)) + " grid, then the "
                       "same refinement")
    target = min(v[1] for v in forms.values())
    return {"target_chi2": target,
            "rule": "reached: best chi^2 <= target x (1 + 1e-3)",
            **{k: {"s": v[0], "best_chi2": v[1], "form": v[2],
                   "reached": v[1] <= target * (1 + 1e-3)}
               for k, v in forms.items()}}


# ---------------------------------------------------------------- dist
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- oracle
def oracle_sample(cfg, frac, seed, nthreads, sq=None):
    """Time the oracle on a bounded, proportional sample of one map's share
    of the step: an FP64 map from `frac` of the rays (round(sqrt(frac)
    nray) per axis) and a seeded contiguous slice of `frac` of the
    trajectories.  Map build and search keep the proportions of the full
    step, so the sample's own rate (trajectory-epoch evals per second of
    wall time, map build included) is the whole job's rate, with no
    extrapolation.  Returns the rate, the sample's wall time and its
    description."""
    import oracle as orc
    g = cfg["grid"]
    og = orc.Grid(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"], g["u0_lo"],
                  g["u0_hi"], g["t0_lo"], g["t0_hi"], g["tE_lo"], g["tE_hi"],
                  g["u0_log"], g["tE_log"])
    s, q = sq if sq else (cfg["s"], cfg["q"])
    nray = max(1, int(round(cfg["nray"] * math.sqrt(frac))))
    t0 = time.perf_counter()
    A, c, off, lost = orc.build_map(s, q, cfg["L"], cfg["npix"], nray,
                                    cfg["X"], nthreads=nthreads)
    t_map = time.perf_counter() - t0
    t = synth.epoch_times(cfg["n"], cfg["seed"], cfg["t0"])
    At = orc.lightcurve_map(A, cfg["L"], t, cfg["t0"], cfg["tE"], cfg["u0"],
                            cfg["alpha"])
    F, sig = synth.photometry(cfg["Fs"] * At + cfg["Fb"], cfg["seed"],
                              cfg["outliers"])
    count = max(1, int(og.size * frac))
    first = int(np.random.default_rng(seed).integers(0, og.size - count + 1))
    t0 = time.perf_counter()
    orc.grid_chi2(og, t, F, 1.0 / sig ** 2, A=A, L=cfg["L"], first=first,
                  count=count, nthreads=nthreads)
    t_search = time.perf_counter() - t0
    wall = t_map + t_search
    return {
        "value": count * len(t) / wall, "wall_s": wall,
        "rays_per_s": nray ** 2 / t_map,
        "t_map_s": t_map, "t_search_s": t_search,
        "sample": (f"1 FP64 map of {nray}^2 rays ({100 * nray ** 2 / cfg['nray'] ** 2:.2f}% of "
                   f"{cfg['nray']}^2) + {count} trajectories "
                   f"({100 * count / og.size:.2f}% of {og.size}) x "
                   f"{len(t)} epochs: one map's share of the step in "
                   f"proportion, rate measured on the sample"),
    }


def run_reference(args, cfg):
    world, rank, local = dist_setup()
    if rank != 0:
        return 0
    import oracle as orc
    orc.build()
    nth = os.cpu_count() or 1
    frac = args.ref_frac
    S, Q = sq_lists(cfg)
    for w in range(args.warmup):
        oracle_sample(cfg, frac * 0.1, 100 + w, nth)
    evals, walls = 0.0, []
    for k in range(args.steps):
        sq = (float(S[k % len(S)]), float(Q[k % len(Q)]))
        r = oracle_sample(cfg, frac, 1000 + k, nth, sq=sq)
        walls.append(r["wall_s"])
        evals += r["value"] * r["wall_s"]
    value = evals / float(np.sum(walls))
    cfg_line = workload_config(cfg)
    cfg_line["lookup"] = "FP32 A table"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(walls)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": cfg_line,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nth,
                         "kind": "oracle",
                         "sample": r["sample"] + "; each step one (s,q) "
                         "map of the 651 (cycling), ms_per_step is the "
                         "sample's wall time"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, cfg):
    import torch
    world, rank, local = dist_setup()
    import paper_1511_01157_gb300 as m
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    ctx = m.Context(dev, stream=stream)
    grid = grid_of(m, cfg)
    S, Q = sq_lists(cfg)
    if args.maps and args.maps < len(S):  # evenly spaced subset (profiling)
        pick = np.linspace(0, len(S) - 1, args.maps).round().astype(int)
        S, Q = S[pick].copy(), Q[pick].copy()
    n_maps = len(S)
    fp16 = args.lookup == "fp16log"
    # weak scaling: every rank searches its own event over all 651 maps
    t, F, sig = make_event(ctx, m, cfg, cfg["seed"] + rank)
    ev = ctx.event(t, F, sig)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32,
                        device=f"cuda:{dev}")
    if args.only:  # one section alone (profiling)
        out = {"profiling": args.only}
        if args.only == "adjoint":
            probes = ctx.measure_peaks()
            props = torch.cuda.get_device_properties(dev)
            peaks, _ = measured_peaks()
            peak_instr = props.multi_processor_count * FP32_LANES_PER_SM * \
                float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
            out["adjoint"] = adjoint_section(ctx, m, cfg, ev, len(t), stream,
                                             probes, peak_instr)
            fits = ctx.sweep(ev, S, Q, cfg["L"], cfg["npix"], cfg["nray"],
                             grid, image_halfwidth=cfg["X"], deflect="fp32")
            out["config2_refine"] = config2_section(ctx, m, cfg, ev, S, Q,
                                                    fits)
        elif args.only == "batched":
            out["batched"] = run_batched(ctx, m, args.batch_events,
                                         args.batch_maps,
                                         not args.no_batch_tune)
        elif args.only == "fp16":
            out["fp16_vs_fp32"] = fp16_section(ctx, m, cfg, ev)
        elif args.only == "peaks":
            out["peak_library"] = peak_library(ctx, m, cfg)
        else:
            out["map_generators"] = map_generators(ctx, m, cfg)
        print(json.dumps(out))
        ctx.close()
        return 0
    if args.peak_only:  # profiling of the peak-aligned form alone
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fits = peak_aligned_fits(ctx, m, cfg, ev, S, Q, peak_time(t, F))
        torch.cuda.synchronize()
        print(json.dumps({"profiling": "peak-aligned form", "maps": len(S),
                          "s": time.perf_counter() - t0,
                          "best_chi2": float(fits["chi2"][:, 0].min()),
                          "peak_library": peak_library(ctx, m, cfg)}))
        return 0
    probes = ctx.measure_peaks()  # measured denominators (before timing)
    evals_step = grid.size * len(t) * n_maps
    rays_step = cfg["nray"] ** 2 * n_maps

    exact = []

    def step():
        fits = ctx.sweep(ev, S, Q, cfg["L"], cfg["npix"], cfg["nray"], grid,
                         image_halfwidth=cfg["X"], deflect="fp32",
                         fp16log=fp16)
        exact.append(ctx.exact_sweeps())
        return fits, [ctx.kernel_ms(i) for i in range(5)]

    with torch.cuda.stream(stream):
        for w in range(args.warmup):
            step()
            flush.fill_(float(w))
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        launches0 = ctx.launch_count()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        kernel_ms = []
        best = None
        with ClockSampler(dev) as clk:
            ev0.record(stream)
            for k in range(args.steps):
                fits, ms = step()
                kernel_ms.append(ms)
                b = float(fits["chi2"].min())
                best = b if best is None else min(best, b)
                flush.fill_(float(k))
            ev1.record(stream)
            torch.cuda.synchronize()
        elapsed = ev0.elapsed_time(ev1) / 1e3
        launches = ctx.launch_count() - launches0
        barrier(world)
        torch.cuda.synchronize()
        elapsed = max_over_ranks(elapsed, world)

        # end to end through morse_search_sweep from pinned host buffers
        tp = torch.from_numpy(np.ascontiguousarray(t)).pin_memory().numpy()
        Fp = torch.from_numpy(np.ascontiguousarray(F)).pin_memory().numpy()
        sp = torch.from_numpy(np.ascontiguousarray(sig)).pin_memory().numpy()
        e2e_steps = max(1, args.steps // 2)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            ctx.search_sweep(tp, Fp, sp, 0.0, S, Q, cfg["L"], cfg["npix"],
                             cfg["nray"], grid, image_halfwidth=cfg["X"],
                             deflect="fp32", fp16log=fp16)
        torch.cuda.synchronize()
        e2e_elapsed = max_over_ranks(time.perf_counter() - t0, world)

    km = np.array(kernel_ms)  # [steps, 5], each summed over the 651 maps
    search_ms = float(km[:, 2].mean())
    ray_ms = float(km[:, 0].mean())
    rays_alone, rays_alone_maps = standalone_rays(ctx, cfg, S, Q)
    value = evals_step * args.steps * world / elapsed
    e2e_value = evals_step * e2e_steps * world / e2e_elapsed

    peaks, peak_kind = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_instr = props.multi_processor_count * FP32_LANES_PER_SM * \
        sm_max * 1e6 / 1e12
    exact_frac = float(np.mean(exact[-args.steps:])) / (grid.size * n_maps)
    instr_done = ALG_INSTR_PRUNED + (ALG_INSTR_PER_EVAL -
                                     ALG_INSTR_PRUNED) * exact_frac
    achieved = evals_step * instr_done / (search_ms * 1e-3) / 1e12
    achieved_22 = evals_step * ALG_INSTR_PER_EVAL / (search_ms * 1e-3) / 1e12
    evals_per_s_kernel = evals_step / (search_ms * 1e-3)
    gather_gbs = evals_per_s_kernel * GATHER_BYTES_PER_EVAL / 1e9
    smem_gbs = evals_per_s_kernel * SMEM_BYTES_PER_EVAL / 1e9
    smem_peak = props.multi_processor_count * SMEM_BYTES_PER_CLK_SM * \
        sm_max * 1e6 / 1e9
    rays_kernel = rays_alone
    ray_alu = probes["fp32_fma_per_s"] / ALG_INSTR_PER_RAY
    ray_atom = probes["smem_atomics_per_s"]
    ray_peak = min(ray_alu, ray_atom)
    traffic = recorded_traffic()
    clocks = clk.summary()
    per_launch = evals_step // n_maps

    cfg_line = workload_config(cfg)
    if n_maps != cfg["n_s"] * cfg["n_q"]:
        cfg_line["maps_per_step"] = n_maps
        cfg_line["workload"] += f" (SUBSET: {n_maps} maps, profiling only)"
    cfg_line["lookup"] = "FP16 log10 A table" if fp16 else "FP32 A table"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (FP64 solve and cross-lane sums)", "data": "synthetic",
        "config": cfg_line,
        "rays_per_s": rays_step * args.steps * world / elapsed,
        "rays_per_s_kernel": rays_alone,
        "rays_per_s_kernel_note": f"ray-shooting kernel time of "
                                  f"{rays_alone_maps} of the maps built "
                                  "alone; in the sweep each build overlaps "
                                  "the previous map's search, and its "
                                  "kernel time there "
                                  f"({rays_step / (ray_ms * 1e-3):.3e} "
                                  "rays/s) includes waits for SMs",
        "kernel_ms_per_step": {
            "rayshoot": ray_ms, "counts_to_map": float(km[:, 1].mean()),
            "search": search_ms, "topk_merge": float(km[:, 3].mean()),
            "fill": float(km[:, 4].mean())},
        "roofline": {
            "kernel": "k_search", "bound": "alu", "achieved": achieved,
            "peak": peak_instr, "unit": "T FP32-instr/s",
            "frac": achieved / peak_instr, "traffic": traffic,
            "algorithmic": f"{instr_done:.3f} FP32 instr per "
                           f"trajectory-epoch ({ALG_INSTR_PRUNED} + 2 x the "
                           f"exact-sweep fraction {exact_frac:.4f}) x "
                           f"{per_launch} per launch",
            "frac_22_instr": achieved_22 / peak_instr,
            "peak_source": f"{props.multi_processor_count} SMs x "
                           f"{FP32_LANES_PER_SM} FP32 lanes x {sm_max} MHz "
                           f"({peak_kind} sm_max_mhz)",
            "measured_fp32_fma_per_s": probes["fp32_fma_per_s"],
            "frac_of_measured_fma": achieved * 1e12 /
            probes["fp32_fma_per_s"],
            "gather": {
                "achieved_GBps": gather_gbs,
                "note": "not binding: 99 % of the cells come from the "
                        "shared-memory band tables, not from L1 or L2 "
                        "gathers, so the measured random-gather rates "
                        "are not a ceiling of this kernel",
                "l1_random_gather_GBps": probes["l1_gather_bytes_per_s"] /
                1e9,
                "l2_random_gather_GBps": probes["l2_gather_bytes_per_s"] /
                1e9,
                "algorithmic": f"{GATHER_BYTES_PER_EVAL} B per "
                               "trajectory-epoch (one 2x2 FP32 cell)"},
            "smem_pipe": {
                "achieved_GBps": smem_gbs, "peak_GBps": smem_peak,
                "frac": smem_gbs / smem_peak,
                "bytes": f"{SMEM_BYTES_PER_EVAL} B per trajectory-epoch "
                         "(16 B cell + half of a 12 B epoch record), "
                         "excluding bank conflicts",
                "peak_source": f"{props.multi_processor_count} SMs x "
                               f"{SMEM_BYTES_PER_CLK_SM} B per clock x "
                               f"{sm_max} MHz"}},
        "rayshoot_roofline": {
            "kernel": "k_rayshoot<FP32>", "rays_per_s": rays_kernel,
            "bound": "alu" if ray_alu <= ray_atom else "smem_atomic",
            "peak_rays_per_s": ray_peak, "frac": rays_kernel / ray_peak,
            "algorithmic": f"{ALG_INSTR_PER_RAY} FP32 instr + 1 shared "
                           "atomic per ray",
            "peak_source": "min(measured FP32 FMA/s / instr, measured "
                           "shared atomics/s)"},
        "probes": probes,
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(tp.nbytes + Fp.nbytes + sp.nbytes),
                "d2h_bytes_per_step": int(grid.top_k * n_maps *
                                          m.FIT_DTYPE.itemsize),
                "steps": e2e_steps,
                "path": "morse_search_sweep (event upload, 651 map builds "
                        "and searches, fits to host)"},
        "gpu_launches": int(launches),
        "exact_sweep_fraction": exact_frac,
        "best_chi2": best,
        "clocks": clocks,
    }
    if rank == 0 and not args.no_extras:
        line["time_to_best_fit"] = time_to_best_fit(
            ctx, m, cfg, ev, S, Q, elapsed / args.steps, fits, t, F, sig)
        line["map_generators"] = map_generators(ctx, m, cfg)
        line["finite_source"] = finite_source_maps(ctx, m, cfg)
        line["peak_library"] = peak_library(ctx, m, cfg)
        line["adjoint"] = adjoint_section(ctx, m, cfg, ev, len(t), stream,
                                          probes, peak_instr * 1e12)
        line["config2_refine"] = config2_section(ctx, m, cfg, ev, S, Q, fits)
        line["fp16_vs_fp32"] = fp16_section(ctx, m, cfg, ev)
        line["batched"] = run_batched(ctx, m, args.batch_events,
                                      args.batch_maps, not args.no_batch_tune)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nth = os.cpu_count() or 1
        r = oracle_sample(cfg, args.cpu_frac, 7, nth)
        r1 = oracle_sample(cfg, args.cpu_frac / 16, 7, 1)
        line["cpu_baseline"] = {
            "value": r["value"], "unit": UNIT, "cores": nth, "kind": "oracle",
            "sample": r["sample"],
            "rays_per_s": r["rays_per_s"],
            "single_thread": {"value": r1["value"], "cores": 1,
                              "rays_per_s": r1["rays_per_s"],
                              "sample": r1["sample"]}}
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="morse",
                    choices=["morse", "reference"])
    ap.add_argument("--cpu-frac", type=float, default=0.02,
                    help="trajectory fraction of the CPU-oracle sample")
    ap.add_argument("--ref-frac", type=float, default=0.05,
                    help="trajectory fraction per reference-arm step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the time-to-best-fit and batched sections")
    ap.add_argument("--no-batch-tune", action="store_true",
                    help="batched section with the default launch shapes")
    ap.add_argument("--batch-events", type=int, default=32,
                    help="events of the batched section (of 256)")
    ap.add_argument("--batch-maps", type=int, default=8,
                    help="maps of the batched section (of 64)")
    ap.add_argument("--lookup", default="fp32", choices=["fp32", "fp16log"],
                    help="map table the search reads (the headline is fp32)")
    ap.add_argument("--peak-only", action="store_true",
                    help="run only the peak-aligned search over the maps "
                    "and the peak library section (profiling)")
    ap.add_argument("--only", default="",
                    choices=["", "adjoint", "batched", "rayshoot", "fp16",
                             "peaks"],
                    help="run one section alone on its own workload "
                    "(profiling): the adjoint on the config-1 event, the "
                    "batched search subset, or the config-1 map builds")
    ap.add_argument("--maps", type=int, default=0,
                    help="search an evenly spaced subset of the 651 (s,q) "
                    "maps per step (profiling of small cases only)")
    args = ap.parse_args()
    cfg = dict(synth.CFG1)
    if args.impl == "reference":
        return run_reference(args, cfg)
    return run_gpu(args, cfg)


if __name__ == "__main__":
    sys.exit(main())
