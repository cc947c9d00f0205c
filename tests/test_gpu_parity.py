"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars (written in each test):
* FP64 ray shooting: counts, off-map and lost totals bit-exact; FP32 map
  values bit-exact (same FP64 product, same rounding).
* FP32 ray shooting: relative L1 <= 1e-3 over pixels with >= 100 rays.
* chi^2 on the same FP32 map: relative error <= 1e-5 per trajectory; the
  top-K set identical (pairs whose chi^2 differ by less than the tolerance
  may swap across rank K, and are counted).
Inputs are seeded synthetic light curves (``synth``) with the oracle's
polynomial point-source magnification as the truth.
"""
import math

import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu

CHI2_RTOL = 1e-5


@pytest.fixture(scope="module")
def m():
    import paper_1511_01157_gb300 as lib
    return lib


@pytest.fixture(scope="module")
def ctx(m):
    c = m.Context(0)
    yield c
    c.close()


def _grid(m, g, top_k):
    return m.Grid.make(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"],
                       g["u0_lo"], g["u0_hi"], g["t0_lo"], g["t0_hi"],
                       g["tE_lo"], g["tE_hi"], g["u0_log"], g["tE_log"],
                       top_k)


def _ogrid(g):
    return orc.Grid(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"],
                    g["u0_lo"], g["u0_hi"], g["t0_lo"], g["t0_hi"],
                    g["tE_lo"], g["tE_hi"], g["u0_log"], g["tE_log"])


def _event(cfg, n=None, seed=None):
    n = cfg["n"] if n is None else n
    seed = cfg["seed"] if seed is None else seed
    t = synth.epoch_times(n, seed, cfg["t0"])
    A = orc.lightcurve_point(cfg["s"], cfg["q"], t, cfg["t0"], cfg["tE"],
                             cfg["u0"], cfg["alpha"])
    F, sig = synth.photometry(cfg["Fs"] * A + cfg["Fb"], seed,
                              cfg.get("outliers", 0.0))
    return t, F, sig


NT = orc.threads_default()


# ------------------------------------------------------------------ maps
@pytest.mark.parametrize("s,q,L,npix,nray,X", [
    (1.0, 1e-3, 2.0, 8, 37, 3.0),
    (0.7, 0.3, 1.5, 32, 300, 2.5),
    (1.3, 1e-2, 1.0, 64, 512, 3.0),
    (2.5, 5e-4, 2.0, 33, 257, 3.0),     # ragged tiles, odd sizes
    (1.0, 1.0, 2.0, 8, 3, 0.75),        # two rays exactly on the lenses
])
def test_fp64_counts_bit_exact_small(ctx, s, q, L, npix, nray, X):
    mp = ctx.build_map(s, q, L, npix, nray, image_halfwidth=X,
                       deflect="fp64")
    c, off, lost = mp.counts()
    co, offo, losto = orc.rayshoot(s, q, L, npix, nray, X, nthreads=NT)
    assert np.array_equal(c, co)
    assert (off, lost) == (offo, losto)
    assert int(c.sum(dtype=np.uint64)) + off + lost == nray * nray
    assert np.array_equal(mp.values(), orc.counts_to_mag(co, L, nray, X))


@pytest.fixture(scope="module")
def cfg0_maps(ctx):
    c = synth.CFG0
    mp = ctx.build_map(c["s"], c["q"], c["L"], c["npix"], c["nray"],
                       image_halfwidth=c["X"], deflect="fp64")
    A_o, co, offo, losto = orc.build_map(c["s"], c["q"], c["L"], c["npix"],
                                         c["nray"], c["X"], nthreads=NT)
    return mp, A_o, co, offo, losto


def test_cfg0_counts_bit_exact(cfg0_maps):
    mp, A_o, co, offo, losto = cfg0_maps
    c, off, lost = mp.counts()
    assert np.array_equal(c, co), f"{np.sum(c != co)} bins differ"
    assert (off, lost) == (offo, losto)
    assert np.array_equal(mp.values(), A_o)


def test_fp32_map_relative_l1(ctx):
    s, q, L, npix, nray, X = 0.9, 5e-4, 2.0, 256, 4000, 3.0
    mp = ctx.build_map(s, q, L, npix, nray, image_halfwidth=X,
                       deflect="fp32")
    A_o, co, offo, losto = orc.build_map(s, q, L, npix, nray, X, nthreads=NT)
    A = mp.values()
    sel = co >= 100
    assert sel.sum() > 1000
    rel_l1 = np.abs(A[sel] - A_o[sel]).sum() / np.abs(A_o[sel]).sum()
    assert rel_l1 <= 1e-3, rel_l1
    c, off, lost = mp.counts()
    assert int(c.sum(dtype=np.uint64)) + off + lost == nray * nray


@pytest.mark.parametrize("nray,npix", [(2003, 128), (1029, 64)])
def test_fp32_map_ragged_ray_grid(ctx, nray, npix):
    """FP32 ray shooting with a ray grid that is not a multiple of a
    thread's 8 columns or a tile's 256: the last sub-blocks are partial.
    Every ray is counted once, and the map matches the FP64 oracle."""
    s, q, L, X = 1.1, 3e-3, 2.0, 3.0
    mp = ctx.build_map(s, q, L, npix, nray, image_halfwidth=X,
                       deflect="fp32")
    A_o, co, offo, losto = orc.build_map(s, q, L, npix, nray, X, nthreads=NT)
    c, off, lost = mp.counts()
    assert int(c.sum(dtype=np.uint64)) + off + lost == nray * nray
    assert abs(int(off) - int(offo)) <= 1e-4 * nray * nray
    A = mp.values()
    sel = co >= 100
    assert sel.sum() > 500
    rel_l1 = np.abs(A[sel] - A_o[sel]).sum() / np.abs(A_o[sel]).sum()
    assert rel_l1 <= 1e-3, rel_l1


# ------------------------------------------------------------------ search
@pytest.fixture(scope="module")
def cfg0_event(ctx):
    t, F, sig = _event(synth.CFG0)
    return t, F, sig, ctx.event(t, F, sig, t_ref=0.0)


def _rel(a, b):
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def test_cfg0_dense_chi2(ctx, m, cfg0_maps, cfg0_event):
    mp, A_o, *_ = cfg0_maps
    t, F, sig, ev = cfg0_event
    c = synth.CFG0
    g = _grid(m, c["grid"], c["top_k"])
    og = _ogrid(c["grid"])
    chi2, fs, fb = ctx.grid_chi2_dense(ev, mp, g)
    o_chi2, o_fs, o_fb, o_fl = orc.grid_chi2(og, t, F, 1.0 / sig ** 2,
                                             A=A_o, L=c["L"], nthreads=NT)
    rel = _rel(chi2, o_chi2)
    assert np.all(np.isfinite(chi2))
    assert np.max(rel) <= CHI2_RTOL, (np.max(rel), int(np.argmax(rel)))
    good = o_fl == 0
    # Fs, Fb: chi^2 is stationary in them, so they carry the FP32 sums'
    # first-order error; compare in units of the flux scale
    assert np.max(np.abs(fs - o_fs)[good]) <= 1e-3 * max(1.0, np.max(np.abs(o_fs[good])))


def _check_topk(got, o_chi2, k, tol=CHI2_RTOL):
    idx_o, val_o = orc.topk(o_chi2, k)
    gi = got["idx"]
    assert np.all(np.diff(got["chi2"]) >= 0), "not sorted"
    assert len(set(gi.tolist())) == len(gi), "duplicate indices"
    swaps = 0
    missing = set(idx_o.tolist()) - set(gi.tolist())
    extra = set(gi.tolist()) - set(idx_o.tolist())
    kth = val_o[-1]
    for j in missing | extra:
        # allowed only for ties within tolerance straddling rank K
        assert abs(o_chi2[j] - kth) <= 2 * tol * kth, (j, o_chi2[j], kth)
        swaps += 1
    for r, i in enumerate(gi):
        assert got["chi2"][r] == pytest.approx(o_chi2[i], rel=tol)
    return swaps


def test_cfg0_topk(ctx, m, cfg0_maps, cfg0_event):
    mp, A_o, *_ = cfg0_maps
    t, F, sig, ev = cfg0_event
    c = synth.CFG0
    og = _ogrid(c["grid"])
    o_chi2, o_fs, o_fb, o_fl = orc.grid_chi2(og, t, F, 1.0 / sig ** 2,
                                             A=A_o, L=c["L"], nthreads=NT)
    for k in (1, 16, 300):
        g = _grid(m, c["grid"], k)
        got = ctx.grid_chi2(ev, mp, g)
        swaps = _check_topk(got, o_chi2, k)
        assert swaps == 0
        # parameters and fluxes of the reported fits
        for rec in got[:5]:
            t0, tE, u0, al = og.params(int(rec["idx"]))
            assert (rec["t0"], rec["tE"], rec["u0"]) == pytest.approx(
                (t0, tE, u0), rel=1e-12)
            assert rec["alpha"] == pytest.approx(al, rel=1e-12, abs=1e-15)
            assert rec["Fs"] == pytest.approx(o_fs[rec["idx"]], rel=1e-3,
                                              abs=1e-3)


@pytest.mark.parametrize("dims,k", [((1, 1, 1, 1), 3), ((3, 5, 2, 3), 7),
                                    ((2, 7, 3, 1), 42), ((5, 3, 3, 3), 135)])
def test_ragged_grids_and_k_beyond_size(ctx, m, dims, k):
    c = synth.CFG0
    A_o, *_ = orc.build_map(0.8, 0.05, 2.0, 48, 700, 3.0, nthreads=NT)
    mp = ctx.map_from_host(A_o, 2.0)
    t, F, sig = _event(c, n=97, seed=3)
    ev = ctx.event(t, F, sig)
    n_u0, n_a, n_t0, n_tE = dims
    g = m.Grid.make(n_u0, n_a, n_t0, n_tE, 0.01, 0.4, -1.5, 1.5, 6.0, 50.0,
                    True, True, k)
    og = orc.Grid(n_u0, n_a, n_t0, n_tE, 0.01, 0.4, -1.5, 1.5, 6.0, 50.0)
    got = ctx.grid_chi2(ev, mp, g)
    o_chi2, *_ = orc.grid_chi2(og, t, F, 1.0 / sig ** 2, A=A_o, L=2.0)
    n = og.size
    kk = min(k, n)
    assert _check_topk(got[:kk], o_chi2, kk) == 0
    assert np.all(got["idx"][kk:] == -1) and np.all(np.isinf(got["chi2"][kk:]))
    chi2, fs, fb = ctx.grid_chi2_dense(ev, mp, g)
    assert np.max(_rel(chi2, o_chi2)) <= CHI2_RTOL


@pytest.mark.parametrize("k", [1, 5, 256, 640, 641, 2048, 4096])
def test_topk_merge_equals_dense_order(ctx, m, k):
    """The top-K of a 152-block search (merged 16 or 4 lists at a time in
    shared memory, or in global memory when k > 3632) is, record for
    record, the k smallest (chi^2, idx) of the dense chi^2 of the same
    grid: the same phase-2 value, so bit for bit, and the fill's chi^2 is
    that key."""
    c = synth.CFG0
    A_o, *_ = orc.build_map(0.9, 0.01, 2.0, 128, 900, 3.0, nthreads=NT)
    mp = ctx.map_from_host(A_o, 2.0)
    t, F, sig = _event(c, n=300, seed=5)
    ev = ctx.event(t, F, sig)
    g = m.Grid.make(20, 36, 13, 10, 0.01, 0.5, -2.0, 2.0, 5.0, 80.0, True,
                    True, k)
    got = ctx.grid_chi2(ev, mp, g)
    chi2, fs, fb = ctx.grid_chi2_dense(ev, mp, g)
    order = np.lexsort((np.arange(chi2.size), chi2))[:k]
    np.testing.assert_array_equal(got["idx"], order)
    np.testing.assert_array_equal(got["chi2"], chi2[order])
    np.testing.assert_array_equal(got["Fs"], fs[order])
    np.testing.assert_array_equal(got["Fb"], fb[order])


@pytest.mark.parametrize("case", ["outside", "inside", "mixed", "band"])
def test_paired_and_single_sweeps_identical(ctx, m, case):
    """The search sweeps trajectories two at a time in packed FP32 and the
    fit fill one at a time; both must give the same bits (the records' Fs
    and Fb come from the single sweep, their chi^2 from the paired one).
    A trajectory searched alone (a range of one) is compared with the same
    trajectory searched among its grid neighbours: tracks that never enter
    the map, tracks inside it at every epoch, mixed, and a grid that reads
    the cells from the shared-memory band tables."""
    A_o, *_ = orc.build_map(0.9, 0.01, 2.0, 128, 900, 3.0, nthreads=NT)
    mp = ctx.map_from_host(A_o, 2.0)
    n = 2000 if case == "band" else 300
    t = synth.epoch_times(n, 5, 0.0)
    F, sig = synth.photometry(1.0 + 0.3 / np.sqrt(0.05 + (t / 20.0) ** 2), 5)
    ev = ctx.event(t, F, sig)
    g = {"outside": m.Grid.make(4, 8, 6, 10, 3.0, 3.5, -5.0, 5.0, 5.0, 80.0,
                                False, True, 4),
         "inside": m.Grid.make(4, 8, 6, 10, 0.01, 0.5, -5.0, 5.0, 4000.0,
                               8000.0, True, True, 4),
         "mixed": m.Grid.make(4, 8, 6, 10, 0.01, 0.5, -5.0, 5.0, 5.0, 80.0,
                              True, True, 4),
         "band": m.Grid.make(3, 8, 20, 10, 0.02, 0.6, -1.5, 1.5, 6.0, 50.0,
                             True, True, 4)}[case]
    chi2, fs, fb = ctx.grid_chi2_dense(ev, mp, g)
    rng = np.random.default_rng(7)
    for j in rng.choice(chi2.size, 120, replace=False):
        c1, f1, b1 = ctx.grid_chi2_dense(ev, mp, g, int(j), 1)
        assert (c1[0], f1[0], b1[0]) == (chi2[j], fs[j], fb[j]), (case, j)


def test_band_tables_equal_global_lookups(ctx, m):
    """A grid with 16 warp groups per line (20 t0 x 10 tE) reads its cells
    from the shared-memory band tables: dense chi^2 and top-K equal the
    oracle's, and the top-K records equal, bit for bit, those of the batched
    search of the same pair, which reads the global table.  The lines
    include the axis-parallel and diagonal directions (alpha = k pi / 4) and
    an odd map size."""
    c = synth.CFG0
    for npix, L in ((96, 2.0), (127, 1.5)):
        A_o, *_ = orc.build_map(0.9, 0.02, L, npix, 900, 3.0, nthreads=NT)
        mp = ctx.map_from_host(A_o, L)
        t, F, sig = _event(c, n=2000, seed=11)  # 4e5 per line: tables on
        ev = ctx.event(t, F, sig)
        g = m.Grid.make(3, 8, 20, 10, 0.02, 0.6, -1.5, 1.5, 6.0, 50.0, True,
                        True, 24)
        og = orc.Grid(3, 8, 20, 10, 0.02, 0.6, -1.5, 1.5, 6.0, 50.0)
        o_chi2, *_ = orc.grid_chi2(og, t, F, 1.0 / sig ** 2, A=A_o, L=L,
                                   nthreads=NT)
        chi2, fs, fb = ctx.grid_chi2_dense(ev, mp, g)
        assert np.max(_rel(chi2, o_chi2)) <= CHI2_RTOL
        got = ctx.grid_chi2(ev, mp, g)
        assert _check_topk(got, o_chi2, 24) == 0
        bat = ctx.grid_chi2_batch([ev], [mp], g)[0, 0]
        for f in ("chi2", "t0", "tE", "u0", "alpha", "Fs", "Fb", "idx"):
            np.testing.assert_array_equal(got[f], bat[f])


def test_dense_subrange(ctx, m, cfg0_maps, cfg0_event):
    mp, A_o, *_ = cfg0_maps
    t, F, sig, ev = cfg0_event
    c = synth.CFG0
    g = _grid(m, c["grid"], 4)
    og = _ogrid(c["grid"])
    first, count = 12345, 1003
    chi2, fs, fb = ctx.grid_chi2_dense(ev, mp, g, first, count)
    o_chi2, *_ = orc.grid_chi2(og, t, F, 1.0 / sig ** 2, A=A_o, L=c["L"],
                               first=first, count=count)
    assert np.max(_rel(chi2, o_chi2)) <= CHI2_RTOL


def test_self_consistent_injection_recovers_index(ctx, m):
    """Noiseless light curve made from the map at a grid trajectory: the
    search puts that index first with chi^2 ~ 0."""
    L = 2.0
    A_o, *_ = orc.build_map(1.1, 3e-3, L, 128, 1500, 3.0, nthreads=NT)
    mp = ctx.map_from_host(A_o, L)
    g = m.Grid.make(6, 12, 5, 4, 0.02, 0.5, -2.0, 2.0, 8.0, 40.0, True, True,
                    5)
    og = orc.Grid(6, 12, 5, 4, 0.02, 0.5, -2.0, 2.0, 8.0, 40.0)
    t = synth.epoch_times(400, 11)
    for kstar in (0, 777, og.size - 1):
        p = og.params(kstar)
        At = orc.lightcurve_map(A_o, L, t, *p)
        F = 1.2 * At + 0.1
        sig = np.full(len(t), 0.01)
        ev = ctx.event(t, F, sig)
        got = ctx.grid_chi2(ev, mp, g)
        assert got["idx"][0] == kstar
        assert got["Fs"][0] == pytest.approx(1.2, rel=1e-4)
        assert got["Fb"][0] == pytest.approx(0.1, rel=2e-3, abs=2e-4)
        # the minimum is zero up to FP32 interpolation of the track
        assert got["chi2"][0] < 1e-3 * got["chi2"][1]


def test_lightcurve_matches_oracle(ctx, cfg0_maps):
    mp, A_o, *_ = cfg0_maps
    c = synth.CFG0
    t = synth.epoch_times(300, 2)
    for p in [(0.0, 20.0, 0.05, 0.7), (1.3, 7.0, 0.3, 4.0),
              (-2.0, 60.0, 1e-3, 2.2)]:
        A = ctx.lightcurve(mp, *p, t)
        Ao = orc.lightcurve_map(A_o, c["L"], t, *p)
        assert np.max(np.abs(A - Ao) / Ao) < 2e-5


def test_search_end_to_end_equals_separate_calls(ctx, m, cfg0_event):
    t, F, sig, ev = cfg0_event
    c = synth.CFG0
    g = _grid(m, c["grid"], 8)
    got = ctx.search(t, F, sig, 0.0, c["s"], c["q"], c["L"], c["npix"],
                     c["nray"], g, image_halfwidth=c["X"], deflect="fp64")
    mp = ctx.build_map(c["s"], c["q"], c["L"], c["npix"], c["nray"],
                       image_halfwidth=c["X"], deflect="fp64")
    ref = ctx.grid_chi2(ev, mp, g)
    assert np.array_equal(got["idx"], ref["idx"])
    assert np.array_equal(got["chi2"], ref["chi2"])


def test_invalid_arguments_are_rejected(ctx, m):
    t = np.linspace(-5, 5, 10)
    F = np.ones(10)
    s = np.full(10, 0.01)
    bad = [
        lambda: ctx.event(t[:2], F[:2], s[:2]),
        lambda: ctx.event(t, F, np.where(np.arange(10) == 3, 0.0, s)),
        lambda: ctx.event(t, np.where(np.arange(10) == 1, np.nan, F), s),
        lambda: ctx.build_map(1.0, 0.0, 2.0, 64, 100),
        lambda: ctx.build_map(-1.0, 0.1, 2.0, 64, 100),
        lambda: ctx.build_map(1.0, 0.1, 2.0, 1, 100),
        lambda: ctx.build_map(1.0, 0.1, float("nan"), 64, 100),
        lambda: ctx.build_map(1.0, 0.1, 2.0, 64, 0),
    ]
    for f in bad:
        with pytest.raises(m.MorseError) as e:
            f()
        assert e.value.status == m.EINVAL
    ev = ctx.event(t, F, s)
    mp = ctx.build_map(1.0, 0.1, 2.0, 16, 64)
    for gb in [m.Grid.make(0, 1, 1, 1, .1, .2, 0, 1, 5, 10, True, True, 1),
               m.Grid.make(1, 1, 1, 1, .1, .2, 0, 1, 0, 10, True, True, 1),
               m.Grid.make(1, 1, 1, 1, .1, .2, 0, 1, 5, 10, True, True, 0),
               m.Grid.make(1, 1, 1, 1, .1, .2, 0, 1, 5, 10, True, True,
                           5000)]:
        with pytest.raises(m.MorseError) as e:
            ctx.grid_chi2(ev, mp, gb)
        assert e.value.status == m.EINVAL
    # the context is still usable after every rejection
    g = m.Grid.make(2, 2, 2, 2, .1, .2, -1, 1, 5, 10, True, True, 3)
    assert np.isfinite(ctx.grid_chi2(ev, mp, g)["chi2"][0])


# ------------------------------------------------------------------ full size
@pytest.fixture(scope="module")
def cfg1_setup(ctx, m):
    c = synth.CFG1
    A_o, co, offo, losto = orc.build_map(c["s"], c["q"], c["L"], c["npix"],
                                         c["nray"], c["X"], nthreads=NT)
    t, F, sig = _event(c)
    return c, A_o, co, t, F, sig


def test_cfg1_full_size_fp32_map(ctx, cfg1_setup):
    c, A_o, co, *_ = cfg1_setup
    mp = ctx.build_map(c["s"], c["q"], c["L"], c["npix"], c["nray"],
                       image_halfwidth=c["X"], deflect="fp32")
    A = mp.values()
    sel = co >= 100
    rel_l1 = np.abs(A[sel] - A_o[sel]).sum() / np.abs(A_o[sel]).sum()
    assert rel_l1 <= 1e-3, rel_l1
    cg, off, lost = mp.counts()
    assert int(cg.sum(dtype=np.uint64)) + off + lost == c["nray"] ** 2


@pytest.mark.parametrize("s,q", [(0.9, 5e-4), (1.0, 1e-2)])
def test_cfg1_full_size_search_dense_oracle(ctx, m, cfg1_setup, s, q):
    """Config 1 at full size, in the launch configuration the benchmark
    times: the map of 10^8 FP32-deflected rays built on the GPU, 1.44 M
    trajectories x 3000 epochs, top-K = 256.  The oracle computes the dense
    chi^2 of every trajectory on the same FP32 map values (the event's truth
    map and a resonant-caustic map); bars: every trajectory's chi^2 within
    1e-5 (GPU dense sweep), the top-256 set identical to the oracle's full
    sort (pairs within the tolerance straddling rank K may swap; counted),
    and every record's chi^2 within 1e-5."""
    c, A_o, co, t, F, sig = cfg1_setup
    mp = ctx.build_map(s, q, c["L"], c["npix"], c["nray"],
                       image_halfwidth=c["X"], deflect="fp32")
    A = mp.values()
    ev = ctx.event(t, F, sig)
    g = _grid(m, c["grid"], c["top_k"])
    og = _ogrid(c["grid"])
    w = 1.0 / sig ** 2
    o_chi2, *_ = orc.grid_chi2(og, t, F, w, A=A, L=c["L"], nthreads=NT)
    got = ctx.grid_chi2(ev, mp, g)
    swaps = _check_topk(got, o_chi2, c["top_k"])
    d, _, _ = ctx.grid_chi2_dense(ev, mp, g)
    rel = _rel(d, o_chi2)
    assert np.max(rel) <= CHI2_RTOL, (np.max(rel), int(np.argmax(rel)))
    print(f"(s, q) = ({s}, {q}): {og.size} trajectories, max chi^2 relative "
          f"error {np.max(rel):.2e}, top-{c['top_k']} swaps at rank K: "
          f"{swaps}")
    assert swaps <= 2


def test_sweep_equals_per_map_searches(ctx, m):
    """morse_sweep (one reused map buffer, no host syncs between maps) gives
    the same fits as building and searching each map separately, and
    morse_search_sweep from host buffers gives the same again."""
    c = synth.CFG0
    t, F, sig = _event(c, n=300, seed=5)
    ev = ctx.event(t, F, sig)
    g = m.Grid.make(4, 9, 3, 4, 0.01, 0.4, -1.0, 1.0, 8.0, 40.0, True, True,
                    6)
    S = np.array([0.7, 1.0, 1.4])
    Q = np.array([1e-3, 1e-2, 3e-4])
    fits = ctx.sweep(ev, S, Q, 2.0, 96, 700, g, image_halfwidth=3.0,
                     deflect="fp32")
    assert fits.shape == (3, 6)
    for i in range(3):
        mp = ctx.build_map(S[i], Q[i], 2.0, 96, 700, image_halfwidth=3.0,
                           deflect="fp32")
        ref = ctx.grid_chi2(ev, mp, g)
        assert np.array_equal(fits[i]["idx"], ref["idx"])
        assert np.array_equal(fits[i]["chi2"], ref["chi2"])
    fits2 = ctx.search_sweep(t, F, sig, 0.0, S, Q, 2.0, 96, 700, g,
                             image_halfwidth=3.0, deflect="fp32")
    assert np.array_equal(fits2["chi2"], fits["chi2"])
    assert ctx.kernel_ms(2) > 0.0


def test_sweep_buffers_across_map_sizes(ctx, m):
    """A sweep builds map i + 1 (second buffer, second stream) while map i
    is searched.  Sweeps of one, two and five maps, at two map sizes in
    turn on the same context (both buffers reallocated), each equal to one
    build and search per map."""
    c = synth.CFG0
    t, F, sig = _event(c, n=250, seed=9)
    ev = ctx.event(t, F, sig)
    g = m.Grid.make(3, 8, 3, 3, 0.01, 0.4, -1.0, 1.0, 8.0, 40.0, True, True,
                    5)
    S = np.array([0.7, 1.0, 1.4, 0.9, 1.2])
    Q = np.array([1e-3, 1e-2, 3e-4, 3e-3, 1e-4])
    for npix, n in ((64, 5), (96, 2), (64, 1), (96, 5)):
        fits = ctx.sweep(ev, S[:n], Q[:n], 2.0, npix, 500, g,
                         image_halfwidth=3.0, deflect="fp32")
        for i in range(n):
            mp = ctx.build_map(S[i], Q[i], 2.0, npix, 500,
                               image_halfwidth=3.0, deflect="fp32")
            ref = ctx.grid_chi2(ev, mp, g)
            mp.free()
            assert np.array_equal(fits[i]["idx"], ref["idx"]), (npix, n, i)
            assert np.array_equal(fits[i]["chi2"], ref["chi2"]), (npix, n, i)


def test_epoch_order_does_not_matter(ctx, m, cfg0_maps):
    """Events are stored time-sorted; a shuffled copy searches the same."""
    mp, A_o, *_ = cfg0_maps
    c = synth.CFG0
    t, F, sig = _event(c, n=400, seed=8)
    perm = np.random.default_rng(1).permutation(len(t))
    g = _grid(m, c["grid"], 12)
    a = ctx.grid_chi2(ctx.event(t, F, sig), mp, g)
    b = ctx.grid_chi2(ctx.event(t[perm], F[perm], sig[perm]), mp, g)
    assert np.array_equal(a["idx"], b["idx"])
    np.testing.assert_allclose(a["chi2"], b["chi2"], rtol=1e-12)


def test_pruning_is_exact_and_effective(ctx, m, cfg0_maps, cfg0_event):
    """The bounded closed form discards most trajectories, and the top-K
    with pruning equals the dense (unpruned) ranking."""
    mp, A_o, *_ = cfg0_maps
    t, F, sig, ev = cfg0_event
    c = synth.CFG0
    g = _grid(m, c["grid"], 32)
    got = ctx.grid_chi2(ev, mp, g)
    n_exact = ctx.exact_sweeps()
    chi2, _, _ = ctx.grid_chi2_dense(ev, mp, g)
    order = np.lexsort((np.arange(len(chi2)), chi2))[:32]
    assert np.array_equal(got["idx"], order)
    assert np.array_equal(got["chi2"], chi2[order])
    assert n_exact < 0.5 * g.size
