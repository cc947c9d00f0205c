"""GPU parity of the FP16 log10 map form against the CPU oracle.

* The FP16 table: codes equal the oracle's binary16 rounding of
  log10(max(A, A_floor)) of the same FP32 values (both round an FP64
  log10 once; a one-ulp difference is allowed where the two FP64 log10
  values straddle a rounding midpoint, at most 1e-5 of the texels), and
  A_floor is half a ray.
* Lookups through the FP16 table equal the FP32 lookup of the decoded map
  (10^x per texel) to FP32 decoding accuracy (1e-6 relative), and the
  oracle's lookup of it within the FP32 lookup's bar (2e-5).
* chi^2 through the FP16 table: against the oracle on the decoded map
  within 1e-4 relative (FP32 decoding error only), top-K identical; against
  the oracle on the FP32 map within 5e-3 relative (the half quantisation;
  distribution printed).
"""
import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu

NT = orc.threads_default()
SAME_MAP_RTOL = 1e-4
FP16_RTOL = 5e-3


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


@pytest.fixture(scope="module")
def cfg0(ctx):
    c = synth.CFG0
    mp = ctx.build_map(c["s"], c["q"], c["L"], c["npix"], c["nray"],
                       image_halfwidth=c["X"], deflect="fp64", fp16log=True)
    A = mp.values()
    codes, floor = mp.half()
    t = synth.epoch_times(c["n"], c["seed"], c["t0"])
    At = orc.lightcurve_point(c["s"], c["q"], t, c["t0"], c["tE"], c["u0"],
                              c["alpha"])
    F, sig = synth.photometry(c["Fs"] * At + c["Fb"], c["seed"])
    ev = ctx.event(t, F, sig, t_ref=0.0)
    return c, mp, A, codes, floor, t, F, sig, ev


def _code_diff(codes, ocodes):
    d = np.abs(codes.astype(np.int32) - ocodes.astype(np.int32))
    return d


def test_half_table_matches_oracle(cfg0):
    c, mp, A, codes, floor, *_ = cfg0
    assert floor == pytest.approx(orc.half_floor(c["L"], c["npix"],
                                                 c["nray"], c["X"]),
                                  rel=1e-15)
    ocodes = orc.log10_half(A, floor)
    d = _code_diff(codes, ocodes)
    assert d.max() <= 1 and (d > 0).mean() <= 1e-5, (d.max(), (d > 0).sum())


@pytest.mark.parametrize("npix", [7, 64, 130])
def test_half_table_from_host_and_switch(ctx, m, npix):
    rng = np.random.default_rng(npix)
    A = (10.0 ** rng.uniform(-0.2, 2.0, (npix, npix))).astype(np.float32)
    A[0, :3] = 0.0  # empty texels take the floor
    mp = ctx.map_from_host(A, 1.5)
    with pytest.raises(m.MorseError):
        mp.half()  # no FP16 table yet
    t = synth.epoch_times(200, 5)
    p = (0.5, 25.0, 0.1, 0.8)
    a32 = ctx.lightcurve(mp, *p, t)
    mp.set_lookup(True)
    codes, floor = mp.half()
    assert floor == 1e-6
    assert _code_diff(codes, orc.log10_half(A, floor)).max() <= 1
    a16 = ctx.lightcurve(mp, *p, t)
    mp.set_lookup(False)
    assert np.array_equal(ctx.lightcurve(mp, *p, t), a32)
    # the FP16 lookup is the FP32 lookup of the decoded map, up to the FP32
    # decoding of 10^x (same track coordinates on both sides; a random map
    # amplifies coordinate rounding, so the decoding is isolated here)
    dec = ctx.map_from_host(orc.half_decode(codes), 1.5)
    ad = ctx.lightcurve(dec, *p, t)
    assert np.max(np.abs(a16 - ad) / ad) <= 1e-6
    assert m._lib.morse_map_set_lookup(mp._h, 7) == m.EINVAL


def test_lightcurve_fp16_matches_decoded_oracle(ctx, cfg0):
    c, mp, A, codes, floor, *_ = cfg0
    dec = orc.half_decode(codes)
    t = synth.epoch_times(400, 2)
    for p in [(0.0, 20.0, 0.05, 0.7), (1.3, 7.0, 0.3, 4.0),
              (-2.0, 60.0, 1e-3, 2.2), (0.4, 12.0, 0.01, 3.1)]:
        a16 = ctx.lightcurve(mp, *p, t)
        ao = orc.lightcurve_map(dec, c["L"], t, *p)
        # the FP32 lookup's bar (FP32 track coordinates)
        assert np.max(np.abs(a16 - ao) / ao) <= 2e-5


def test_dense_chi2_fp16(ctx, m, cfg0):
    c, mp, A, codes, floor, t, F, sig, ev = cfg0
    g = _grid(m, c["grid"], c["top_k"])
    og = _ogrid(c["grid"])
    w = 1.0 / sig ** 2
    chi2, fs, fb = ctx.grid_chi2_dense(ev, mp, g)
    o_dec, *_ = orc.grid_chi2(og, t, F, w, A=orc.half_decode(codes),
                              L=c["L"], nthreads=NT)
    rel = np.abs(chi2 - o_dec) / o_dec
    print(f"FP16 vs oracle on the decoded map: max rel {rel.max():.2e}")
    assert rel.max() <= SAME_MAP_RTOL
    o32, *_ = orc.grid_chi2(og, t, F, w, A=A, L=c["L"], nthreads=NT)
    rel32 = np.abs(chi2 - o32) / o32
    print(f"FP16 vs oracle on the FP32 map: median {np.median(rel32):.2e} "
          f"p99 {np.quantile(rel32, 0.99):.2e} max {rel32.max():.2e}")
    assert rel32.max() <= FP16_RTOL


def test_topk_fp16_and_noalloc(ctx, m, cfg0):
    c, mp, A, codes, floor, t, F, sig, ev = cfg0
    og = _ogrid(c["grid"])
    o_dec, *_ = orc.grid_chi2(og, t, F, 1.0 / sig ** 2,
                              A=orc.half_decode(codes), L=c["L"],
                              nthreads=NT)
    for k in (1, 16, 300):
        g = _grid(m, c["grid"], k)
        got = ctx.grid_chi2(ev, mp, g)
        idx_o, val_o = orc.topk(o_dec, k)
        kth = val_o[-1]
        diff = set(idx_o.tolist()) ^ set(got["idx"].tolist())
        for j in diff:  # only near-ties straddling rank K may swap
            assert abs(o_dec[j] - kth) <= 2 * SAME_MAP_RTOL * kth
        np.testing.assert_allclose(got["chi2"], o_dec[got["idx"]],
                                   rtol=SAME_MAP_RTOL)
        if k <= 16:
            na = ctx.grid_chi2_noalloc(ev, mp, g)
            assert np.array_equal(na["idx"], got["idx"])
            assert np.array_equal(na["chi2"], got["chi2"])


def test_sweep_fp16_equals_per_map(ctx, m):
    c = synth.CFG0
    t = synth.epoch_times(300, 8, 0.0)
    At = orc.lightcurve_point(1.0, 1e-3, t, 0.0, 20.0, 0.05, 0.7)
    F, sig = synth.photometry(At + 0.3, 8)
    ev = ctx.event(t, F, sig)
    g = m.Grid.make(8, 12, 5, 5, 1e-3, 0.5, -2.0, 2.0, 5.0, 80.0, True, True,
                    8)
    s = [0.8, 1.0, 1.25]
    q = [1e-3, 3e-3, 1e-2]
    sw = ctx.sweep(ev, s, q, 2.0, 128, 600, g, image_halfwidth=3.0,
                   fp16log=True)
    for i in range(3):
        mp = ctx.build_map(s[i], q[i], 2.0, 128, 600, image_halfwidth=3.0,
                           deflect="fp32", fp16log=True)
        one = ctx.grid_chi2(ev, mp, g)
        assert np.array_equal(sw[i]["idx"], one["idx"])
        assert np.array_equal(sw[i]["chi2"], one["chi2"])
