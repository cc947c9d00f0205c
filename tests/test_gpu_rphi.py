"""GPU parity of the (r, phi) trajectory grids about caustics (§4.2).

* Caustics (count, centres, sizes) equal the oracle's for the same psi
  sampling (1e-9), in the close, intermediate and wide topologies.
* Lines equal the oracle's (u, alpha, shift).
* The top-K over a line grid equals the oracle's chi^2 of every
  (line, t0, tE) trajectory (set identical, chi^2 within 1e-5), and the
  records seed the refinement.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import caustics as oc
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


@pytest.mark.parametrize("s,q", [(0.5, 1e-2), (0.8, 0.2), (1.0, 1e-3),
                                 (1.0, 1.0), (1.7, 5e-3), (2.5, 5e-4)])
def test_caustics_match_oracle(ctx, s, q):
    got = ctx.caustics(s, q, 720)
    ref = oc.caustics(s, q, 720)
    assert len(got) == len(ref) == oc.topology_count(s, q)
    for g, r in zip(got, ref):
        assert g.c1 == pytest.approx(r[0], abs=1e-9)
        assert g.c2 == pytest.approx(r[1], abs=1e-9)
        assert g.size == pytest.approx(r[2], rel=1e-9)
        assert g.n_points == r[3]


def test_line_grid_search_matches_oracle_and_refines(ctx, m):
    s, q, L = 1.1, 1e-2, 2.0
    A, *_ = orc.build_map(s, q, L, 256, 2000, 3.0, nthreads=NT)
    mp = ctx.map_from_host(A, L)
    cs = ctx.caustics(s, q, 720)
    lines = m.rphi_lines(cs, 4, 0.0, 1.5, 8)
    ref_lines = oc.rphi_lines([(c.c1, c.c2, c.size, c.n_points) for c in cs],
                              4, 0.0, 1.5, 8)
    np.testing.assert_allclose(lines, ref_lines, rtol=1e-14, atol=1e-14)
    t = synth.epoch_times(300, 9, 0.0)
    At = orc.lightcurve_point(s, q, t, 0.2, 18.0, 0.08, 0.9)
    F, sig = synth.photometry(At + 0.3, 9)
    ev = ctx.event(t, F, sig)
    t0v = np.linspace(-2.0, 2.0, 5)
    tEv = np.exp(np.linspace(np.log(8.0), np.log(40.0), 4))
    g = m.Grid.make(len(lines), 1, 5, 4, 1.0, 1.0, -2.0, 2.0, 8.0, 40.0,
                    False, True, 12)
    got = ctx.grid_chi2_lines(ev, mp, g, lines)
    o = oc.lines_chi2(lines, t0v, tEv, t, F, 1.0 / sig ** 2, A, L)
    idx_o, val_o = orc.topk(o, 12)
    assert set(got["idx"].tolist()) == set(idx_o.tolist())
    np.testing.assert_allclose(got["chi2"], o[got["idx"]], rtol=1e-5)
    # records in the (u0, alpha, t0, tE) convention: the oracle's chi^2 of
    # the record's parameters is the record's chi^2
    for r in got[:4]:
        c = orc.chi2_theta(t, F, 1.0 / sig ** 2,
                           (r["t0"], r["tE"], r["u0"], r["alpha"]), A=A,
                           L=L)[0]
        assert r["chi2"] == pytest.approx(c, rel=1e-5)
    ref = ctx.refine(ev, mp, got, iters=20)
    assert np.all(ref["chi2"] <= got["chi2"] * (1 + 1e-12))
    with pytest.raises(m.MorseError) as e:
        bad = m.Grid.make(len(lines), 2, 5, 4, 1.0, 1.0, -2.0, 2.0, 8.0,
                          40.0, False, True, 12)
        ctx.grid_chi2_lines(ev, mp, bad, lines)
    assert e.value.status == m.EINVAL
