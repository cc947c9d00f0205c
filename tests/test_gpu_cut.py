"""GPU parity of the minimum-magnification cut (§4.3 (i)).

* Line maxima equal the oracle's exact line_max within 1e-12 relative.
* A search with a_min returns the oracle top-K of the trajectories whose
  line reaches a_min (chi^2 within 1e-5, identical set); dense results are
  +inf on cut lines and unchanged elsewhere; a sweep equals per-map
  searches; the batched and allocation-free searches refuse the cut.
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


DIMS = (12, 16, 5, 4)
RANGES = (1e-3, 0.8, -2.0, 2.0, 5.0, 60.0)


@pytest.fixture(scope="module")
def setup(ctx, m):
    s, q, L = 1.0, 5e-3, 2.0
    A, *_ = orc.build_map(s, q, L, 128, 1500, 3.0, nthreads=NT)
    mp = ctx.map_from_host(A, L)
    t = synth.epoch_times(300, 12, 0.0)
    At = orc.lightcurve_point(s, q, t, 0.0, 20.0, 0.05, 0.7)
    F, sig = synth.photometry(At + 0.3, 12)
    ev = ctx.event(t, F, sig)
    og = orc.Grid(*DIMS, *RANGES)
    return A, L, mp, t, F, sig, ev, og


def _grid(m, k, a_min):
    return m.Grid.make(*DIMS, *RANGES, True, True, k, a_min)


def test_line_max_matches_oracle(ctx, m, setup):
    A, L, mp, t, F, sig, ev, og = setup
    lm = ctx.line_max(mp, _grid(m, 4, 0.0))
    u0 = np.exp(np.linspace(np.log(RANGES[0]), np.log(RANGES[1]), DIMS[0]))
    for iu in range(DIMS[0]):
        for ia in range(DIMS[1]):
            o = orc.line_max(A, L, u0[iu], 2 * np.pi * ia / DIMS[1])
            assert lm[iu, ia] == pytest.approx(o, rel=1e-12), (iu, ia)


def test_search_with_cut_is_the_search_of_the_kept_lines(ctx, m, setup):
    A, L, mp, t, F, sig, ev, og = setup
    lm = ctx.line_max(mp, _grid(m, 4, 0.0)).ravel()
    # a cut between two line maxima, far from both
    v = np.sort(lm)
    k = len(v) // 2
    a_min = float(np.sqrt(v[k - 1] * v[k]))
    assert v[k] > v[k - 1] * (1 + 1e-4)
    per_line = DIMS[2] * DIMS[3]
    kept = np.repeat(lm >= a_min, per_line)
    o_chi2, *_ = orc.grid_chi2(og, t, F, 1.0 / sig ** 2, A=A, L=L,
                               nthreads=NT)
    o_cut = np.where(kept, o_chi2, np.inf)
    for K in (1, 16):
        got = ctx.grid_chi2(ev, mp, _grid(m, K, a_min))
        idx_o, val_o = orc.topk(o_cut, K)
        assert set(got["idx"].tolist()) == set(idx_o.tolist())
        np.testing.assert_allclose(got["chi2"], o_chi2[got["idx"]],
                                   rtol=1e-5)
    dense, fs, fb = ctx.grid_chi2_dense(ev, mp, _grid(m, 1, a_min))
    plain, *_ = ctx.grid_chi2_dense(ev, mp, _grid(m, 1, 0.0))
    assert np.all(np.isinf(dense[~kept])) and np.all(fs[~kept] == 0)
    assert np.array_equal(dense[kept], plain[kept])
    # a_min 0 is no cut
    assert np.array_equal(ctx.grid_chi2(ev, mp, _grid(m, 16, 0.0))["chi2"],
                          ctx.grid_chi2(ev, mp, _grid(m, 16, 0.0))["chi2"])


def test_sweep_with_cut_and_refusals(ctx, m, setup):
    A, L, mp, t, F, sig, ev, og = setup
    g = _grid(m, 8, 3.0)
    S, Q = [0.9, 1.1], [3e-3, 1e-2]
    sw = ctx.sweep(ev, S, Q, 2.0, 128, 600, g, image_halfwidth=3.0)
    for i in range(2):
        one = ctx.grid_chi2(ev, ctx.build_map(S[i], Q[i], 2.0, 128, 600,
                                              image_halfwidth=3.0,
                                              deflect="fp32"), g)
        assert np.array_equal(sw[i]["idx"], one["idx"])
        assert np.array_equal(sw[i]["chi2"], one["chi2"])
    with pytest.raises(m.MorseError) as e:
        ctx.grid_chi2_batch([ev], [mp], g)
    assert e.value.status == m.EUNSUPPORTED
    with pytest.raises(m.MorseError) as e:
        ctx.grid_chi2_noalloc(ev, mp, g)
    assert e.value.status == m.EUNSUPPORTED
