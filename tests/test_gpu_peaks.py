"""GPU parity of the peak library and the peak-aligned searches (§4.3
(iii)-(v), Eq. 7-8).

* The library (count, positions, heights of the kept peaks) equals the
  oracle's bit for bit: the count is an integer decided in FP32 with the
  same operations on both sides.  Ray-shot maps with and without the
  threshold (delta = 0 counts the Poisson noise too, which stresses the
  detector and the choice of the highest peaks), several sampling steps,
  lines of a (u0, alpha) grid and of an (r, phi) grid, axis-parallel lines
  and lines that miss the map.
* The searches' top-K equals the oracle's chi^2 of every allowed trajectory
  (set identical, chi^2 within 1e-5) with no peak time and a peak-count cut,
  with one peak time (Eq. 7) and with two (Eq. 8); each record's chi^2 is
  the oracle's chi^2 of its (t0, tE, u0, alpha).
"""
import math

import numpy as np
import pytest

import oracle as orc
from oracle import caustics as oc
import synth

pytestmark = pytest.mark.gpu

NT = orc.threads_default()
S_, Q_, L_ = 1.1, 1e-2, 2.0


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
def amap():
    A, *_ = orc.build_map(S_, Q_, L_, 256, 2000, 3.0, nthreads=NT)
    return A


def _grid_lines(n_u0, n_alpha, u_lo, u_hi):
    return np.array([(u, 2 * math.pi * k / n_alpha, 0.0)
                     for u in np.linspace(u_lo, u_hi, n_u0)
                     for k in range(n_alpha)])


def _all_lines(m, ctx):
    cs = ctx.caustics(S_, Q_, 720)
    rphi = m.rphi_lines(cs, 3, 0.0, 1.5, 12)
    edge = np.array([(0.3, 0.0, 0.0), (0.3, math.pi / 2, 0.1),
                     (-1.2, math.pi, 0.0), (0.0, 3 * math.pi / 2, -0.2),
                     (2.9, 0.7, 0.0), (-5.0, 2.0, 0.0), (L_, 0.0, 0.0),
                     (1.999, 0.0, 0.0)])
    return np.vstack([_grid_lines(9, 16, -1.2, 1.2), rphi, edge])


@pytest.mark.parametrize("sub,max_peaks,delta",
                         [(2, 8, 0.0), (2, 8, 0.05), (1, 1, 0.02),
                          (3, 16, 0.0), (2, 4, 0.3)])
def test_library_bit_exact(ctx, m, amap, sub, max_peaks, delta):
    lines = _all_lines(m, ctx)
    mp = ctx.map_from_host(amap, L_)
    c, p, h = ctx.line_peaks(mp, lines, sub=sub, max_peaks=max_peaks,
                             delta=delta)
    co, po, ho = orc.line_peaks(amap, L_, lines, sub=sub, delta=delta,
                                max_peaks=max_peaks)
    np.testing.assert_array_equal(c, co)
    np.testing.assert_array_equal(p, po)  # NaN in the same slots
    np.testing.assert_array_equal(h, ho)
    assert c[-4] == 0 and c[-3] == 0  # lines that miss the map
    if delta == 0.0:
        assert c.max() > max_peaks  # noise peaks: the kept ones are chosen


def _event(seed=9):
    t = synth.epoch_times(300, seed, 0.0)
    At = orc.lightcurve_point(S_, Q_, t, 0.2, 18.0, 0.08, 0.9)
    F, sig = synth.photometry(At + 0.3, seed)
    # the two highest maxima of the noise-free curve: the peak times
    mx = [i for i in range(1, len(t) - 1)
          if At[i] > At[i - 1] and At[i] >= At[i + 1]]
    top = sorted(sorted(mx, key=lambda i: -At[i])[:2])
    return t, F, sig, [t[i] for i in top]


def _ref_chi2(rows, t0v, tEv, t, F, w, A):
    out = []
    for u, al, M, tEr, used in rows:
        for t0 in t0v:
            for tE in ([tEr] if not math.isnan(tEr) else tEv):
                if used:
                    out.append(orc.chi2_theta(t, F, w, (t0 - M * tE, tE, u,
                                                        al), A=A, L=L_)[0])
                else:
                    out.append(math.inf)
    return np.array(out)


def _check(got, ref, t, F, w, A, k):
    idx_o, _ = orc.topk(ref, k)
    assert set(got["idx"].tolist()) == set(idx_o.tolist())
    np.testing.assert_allclose(got["chi2"], ref[got["idx"]], rtol=1e-5)
    for r in got[:4]:
        c = orc.chi2_theta(t, F, w, (r["t0"], r["tE"], r["u0"], r["alpha"]),
                           A=A, L=L_)[0]
        assert r["chi2"] == pytest.approx(c, rel=1e-5)


@pytest.mark.parametrize("n_tp", [0, 1, 2])
def test_peak_search_matches_oracle(ctx, m, amap, n_tp):
    t, F, sig, tps = _event()
    w = 1.0 / sig ** 2
    mp = ctx.map_from_host(amap, L_)
    ev = ctx.event(t, F, sig)
    lines = _grid_lines(8, 12, -0.6, 0.6)
    sub, P, delta = 2, 4, 0.3
    tp = tps[:n_tp]
    min_peaks = 2 if n_tp == 0 else n_tp
    co, po, _ = orc.line_peaks(amap, L_, lines, sub=sub, delta=delta,
                               max_peaks=P)
    rows = orc.peak_lines(lines, co, po, tp, min_peaks=min_peaks)
    n_used = int(rows[:, 4].sum())
    assert 0 < n_used < len(rows)  # the cut removes some, keeps some
    if n_tp == 0:
        n_t0, n_tE, t0lo, t0hi = 5, 4, -2.0, 2.0
        t0v = orc.axis(t0lo, t0hi, n_t0, False)
    elif n_tp == 1:
        n_t0, n_tE, t0lo, t0hi = 3, 4, -0.4, 0.4
        t0v = orc.axis(t0lo + tp[0], t0hi + tp[0], n_t0, False)
    else:
        n_t0, n_tE, t0lo, t0hi = 2, 1, -0.1, 0.1
        t0v = orc.axis(t0lo + tp[0], t0hi + tp[0], n_t0, False)
    tEv = orc.axis(8.0, 40.0, n_tE, True)
    g = m.Grid.make(len(rows), 1, n_t0, n_tE, 1.0, 1.0, t0lo, t0hi, 8.0,
                    40.0, False, True, 10)
    got = ctx.peak_search(ev, mp, g, lines, tp=tp, min_peaks=min_peaks,
                          sub=sub, max_peaks=P, delta=delta)
    ref = _ref_chi2(rows, t0v, tEv, t, F, w, amap)
    assert len(ref) == len(rows) * n_t0 * n_tE
    _check(got, ref, t, F, w, amap, 10)
    if n_tp == 2:
        # Eq. 8: the record's tE spans the two peaks
        for r in got[:3]:
            assert np.isfinite(r["tE"]) and r["tE"] > 0


def test_peak_search_all_cut_and_errors(ctx, m, amap):
    t, F, sig, tps = _event()
    mp = ctx.map_from_host(amap, L_)
    ev = ctx.event(t, F, sig)
    lines = _grid_lines(2, 4, 1.6, 1.9)
    g = m.Grid.make(4, 1, 3, 3, 1.0, 1.0, -1.0, 1.0, 8.0, 40.0, False,
                    True, 5)
    got = ctx.peak_search(ev, mp, g, lines, tp=tps[:1], min_peaks=100000,
                          delta=0.05)
    assert (got["idx"] == -1).all() and np.isinf(got["chi2"]).all()
    for kw in (dict(tp=tps[::-1]), dict(tp=tps[:1], sub=0),
               dict(tp=tps[:1], max_peaks=17), dict(tp=tps[:1], delta=-1.0),
               dict(tp=[0.0, 1.0, 2.0])):
        with pytest.raises(m.MorseError) as e:
            ctx.peak_search(ev, mp, g, lines, **kw)
        assert e.value.status == m.EINVAL
    with pytest.raises(m.MorseError) as e:  # two peak times fix tE
        ctx.peak_search(ev, mp, g, lines, tp=tps)
    assert e.value.status == m.EINVAL
