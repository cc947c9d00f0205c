"""Real-data times: light curves at Julian-date scale (the paper's events
are dated in HJD ~ 2452847, §6) through the library's time handling.

The library stores each epoch as the FP32 offset t - t_ref, subtracted in
FP64 on the host, and takes grid t0 values as absolute times in the frame
of t.  Here the times are raw FP64 values (not rounded to anything FP32
can hold), t_ref and the grid t0 axis sit at JD scale, and the grid is
shaped so that the search reads its map cells from the shared-memory band
tables (16 t0 x 10 tE = 160 trajectories per (u0, alpha) line, 16 warp
groups a line, 4.8e5 trajectory-epochs a line, position bound B ~ 1e3).
The oracle is fed the unshifted FP64 times.  Bars: chi^2 within 1e-5 of
the oracle for every trajectory and the top-K identical.  The FP32 offsets
resolve 2^-24 x 40 d ~ 2.4e-6 d, which moved chi^2 by at most 5.5e-7
relative (measured with the oracle itself, exact against rounded times).
"""
import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu

NT = orc.threads_default()
JD = 2452847.0
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


@pytest.fixture(scope="module")
def setup(ctx):
    c = synth.CFG0
    A_o, *_ = orc.build_map(c["s"], c["q"], c["L"], c["npix"], c["nray"],
                            c["X"], nthreads=NT)
    t_off = synth.epoch_times(3000, 21, 0.0, raw=True)
    assert np.any(t_off.astype(np.float32).astype(np.float64) != t_off)
    T = JD + t_off
    At = orc.lightcurve_point(c["s"], c["q"], t_off, 0.0, c["tE"], c["u0"],
                              c["alpha"])
    F, sig = synth.photometry(c["Fs"] * At + c["Fb"], 21)
    return c, A_o, T, F, sig


def _grids(m, top_k):
    lo, hi = JD - 2.0, JD + 2.0
    g = m.Grid.make(12, 24, 16, 10, 1e-3, 0.5, lo, hi, 5.0, 80.0, True,
                    True, top_k)
    og = orc.Grid(12, 24, 16, 10, 1e-3, 0.5, lo, hi, 5.0, 80.0, True, True)
    return g, og


@pytest.mark.parametrize("t_ref", [JD + 0.37, JD - 12.5])
def test_jd_times_match_fp64_oracle(ctx, m, setup, t_ref):
    c, A_o, T, F, sig = setup
    mp = ctx.map_from_host(A_o, c["L"])
    ev = ctx.event(T, F, sig, t_ref=t_ref)
    g, og = _grids(m, 16)
    o_chi2, *_ = orc.grid_chi2(og, T, F, 1.0 / sig ** 2, A=A_o, L=c["L"],
                               nthreads=NT)
    d, _, _ = ctx.grid_chi2_dense(ev, mp, g)
    rel = np.abs(d - o_chi2) / o_chi2
    assert rel.max() <= CHI2_RTOL, rel.max()
    got = ctx.grid_chi2(ev, mp, g)
    idx_o, val_o = orc.topk(o_chi2, 16)
    assert set(got["idx"].tolist()) == set(idx_o.tolist())
    np.testing.assert_allclose(got["chi2"], o_chi2[got["idx"]],
                               rtol=CHI2_RTOL)
    # records carry absolute t0 in the frame of the data
    for r in got[:4]:
        t0, tE, u0, al = og.params(int(r["idx"]))
        assert r["t0"] == pytest.approx(t0, abs=1e-7)
    print(f"t_ref = {t_ref}: max chi^2 relative error {rel.max():.2e}")


def test_t_ref_far_from_the_data_is_rejected(ctx, m, setup):
    c, A_o, T, F, sig = setup
    with pytest.raises(m.MorseError) as e:
        ctx.event(T, F, sig, t_ref=0.0)  # offsets of 2.45e6 d
    assert e.value.status == m.EINVAL
    ev = ctx.event(T, F, sig, t_ref=JD)  # the context stays usable
    mp = ctx.map_from_host(A_o, c["L"])
    g, _ = _grids(m, 4)
    assert np.isfinite(ctx.grid_chi2(ev, mp, g)["chi2"][0])
