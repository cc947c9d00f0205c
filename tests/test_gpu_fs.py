"""GPU parity of finite-source maps (§4.1: maps convolved with limb-
darkened source profiles) against the oracle's direct convolution.

Bar: relative error <= 2e-6 per texel.  The two compute the same texel
weights (FP64, 8 x 8 points per texel) and sum the same terms; the GPU
rounds the weights and each row's sum to FP32 (at most 2R + 1 terms of
relative rounding 2^-24) and adds the rows in FP64.
"""
import numpy as np
import pytest

import oracle as orc
import synth

pytestmark = pytest.mark.gpu

NT = orc.threads_default()


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
def base_map():
    s, q, L, npix = 1.0, 1e-2, 1.5, 96
    A, c, off, lost = orc.build_map(s, q, L, npix, 1500, 2.5, nthreads=NT)
    return A, L, npix


@pytest.mark.parametrize("rho_px,gamma", [(0.3, 0.53), (2.7, 0.53),
                                          (9.5, 0.0), (30.0, 0.53),
                                          (61.0, 1.0)])
def test_finite_source_matches_oracle(ctx, base_map, rho_px, gamma):
    A, L, npix = base_map
    mp = ctx.map_from_host(A, L)
    dlt = 2 * L / npix
    fs = mp.finite_source(rho_px * dlt, gamma)
    got = fs.values().astype(np.float64)
    ref = orc.fs_convolve(A, L, orc.fs_weights(rho_px, gamma), nthreads=NT)
    rel = np.abs(got - ref) / ref
    print(f"rho {rho_px} texels, gamma {gamma}: max rel {rel.max():.2e}")
    assert rel.max() <= 2e-6
    if rho_px < 0.5:  # a sub-texel source leaves the map unchanged
        assert np.array_equal(fs.values(), A)


def test_finite_source_map_is_searchable(ctx, m, base_map):
    A, L, npix = base_map
    mp = ctx.map_from_host(A, L)
    fs = mp.finite_source(0.1, 0.53)
    V = fs.values()
    t = synth.epoch_times(150, 3, 0.0)
    At = orc.lightcurve_map(V, L, t, 0.0, 15.0, 0.1, 0.8)
    F = 1.1 * At + 0.2
    sig = np.full(len(t), 0.01)
    ev = ctx.event(t, F, sig)
    g = m.Grid.make(5, 8, 4, 4, 1e-2, 0.5, -1.0, 1.0, 8.0, 30.0, True, True,
                    4)
    og = orc.Grid(5, 8, 4, 4, 1e-2, 0.5, -1.0, 1.0, 8.0, 30.0)
    chi2, *_ = ctx.grid_chi2_dense(ev, fs, g)
    o, *_ = orc.grid_chi2(og, t, F, 1.0 / sig ** 2, A=V, L=L)
    assert np.max(np.abs(chi2 - o) / np.maximum(o, 1e-300)) <= 1e-5


def test_finite_source_rejects_bad_arguments(ctx, m, base_map):
    A, L, npix = base_map
    mp = ctx.map_from_host(A, L)
    for rho, gamma in ((0.0, 0.5), (-1.0, 0.5), (0.1, 1.5), (0.1, -0.1),
                       (1e6, 0.5)):
        with pytest.raises(m.MorseError) as e:
            mp.finite_source(rho, gamma)
        assert e.value.status == m.EINVAL
