"""GPU parity of the adjoint gradient, the Levenberg-Marquardt refine and the
torch.autograd.Function, against the CPU oracle.

* chi^2 at grid points equals the grid search's (same device functions).
* The gradient equals FP64 central differences of the oracle's map chi^2
  for every component whose +-h evaluations keep every epoch in the same
  texel and on the same side of the map edge (the bilinear lookup is
  smooth there; its gradient jumps at texel edges).  h = 1e-6 relative:
  the FP64 oracle is exact enough for it, and crossings stay rare.
* Against the FP64 gradient of the point-source polynomial chi^2 (the
  oracle's implicit differentiation of the lens equation) on 1000
  trajectories that stay 8 texels from any caustic, on a map holding the
  polynomial at texel centres: the bilinear discretisation sets the
  tolerance (median relative error <= 1e-2); the distribution is
  printed.
"""
import math

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
def setup(ctx):
    c = synth.CFG0
    A_o, *_ = orc.build_map(c["s"], c["q"], c["L"], c["npix"], c["nray"],
                            c["X"], nthreads=NT)
    t = synth.epoch_times(c["n"], c["seed"], c["t0"])
    At = orc.lightcurve_point(c["s"], c["q"], t, c["t0"], c["tE"], c["u0"],
                              c["alpha"])
    F, sig = synth.photometry(c["Fs"] * At + c["Fb"], c["seed"])
    mp = ctx.map_from_host(A_o, c["L"])
    ev = ctx.event(t, F, sig)
    return c, A_o, t, F, sig, mp, ev


def _ogrid(g):
    return orc.Grid(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"],
                    g["u0_lo"], g["u0_hi"], g["t0_lo"], g["t0_hi"],
                    g["tE_lo"], g["tE_hi"], g["u0_log"], g["tE_log"])


def test_chi2_at_grid_points_equals_search(ctx, m, setup):
    c, A_o, t, F, sig, mp, ev = setup
    g = c["grid"]
    og = _ogrid(g)
    grid = m.Grid.make(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"],
                       g["u0_lo"], g["u0_hi"], g["t0_lo"], g["t0_hi"],
                       g["tE_lo"], g["tE_hi"], True, True, 4)
    idx = np.random.default_rng(0).choice(og.size, 64, replace=False)
    theta = np.array([og.params(int(k)) for k in idx])
    chi2, grad, fs, fb = ctx.chi2_grad(ev, mp, theta)
    dense, dfs, dfb = ctx.grid_chi2_dense(ev, mp, grid)
    np.testing.assert_allclose(chi2, dense[idx], rtol=1e-6)
    w = 1.0 / sig ** 2
    for j, k in enumerate(idx[:16]):
        o, ofs, ofb = orc.chi2_theta(t, F, w, theta[j], A=A_o, L=c["L"])
        assert chi2[j] == pytest.approx(o, rel=1e-5)
        assert fs[j] == pytest.approx(ofs, rel=1e-3, abs=1e-3)


def _pixels(theta, t, L, npix):
    """FP64 pixel coordinates (lookup convention) and inside flags."""
    t0, tE, u0, al = theta
    tau = (t - t0) / tE
    y1 = tau * math.cos(al) - u0 * math.sin(al)
    y2 = tau * math.sin(al) + u0 * math.cos(al)
    d = 2 * L / npix
    px = np.clip((y1 + L) / d - 0.5, 0, npix - 1)
    py = np.clip((y2 + L) / d - 0.5, 0, npix - 1)
    inside = (np.abs(y1) < L) & (np.abs(y2) < L)
    return np.floor(px), np.floor(py), inside


def _steps(theta):
    t0, tE, u0, al = theta
    return np.array([1e-6 * tE, 1e-6 * tE, 1e-6 * max(u0, 1e-3), 1e-6])


def test_gradient_matches_oracle_central_differences(ctx, setup):
    c, A_o, t, F, sig, mp, ev = setup
    w = 1.0 / sig ** 2
    rng = np.random.default_rng(5)
    n = 120
    theta = np.stack([rng.uniform(-1.5, 1.5, n), rng.uniform(8.0, 40.0, n),
                      rng.uniform(0.01, 0.3, n), rng.uniform(0, 2 * np.pi, n)],
                     axis=1)
    chi2, grad, _, _ = ctx.chi2_grad(ev, mp, theta)
    rel, used = [], 0
    for i in range(n):
        h = _steps(theta[i])
        base = _pixels(theta[i], t, c["L"], c["npix"])
        for k in range(4):
            tp = theta[i].copy()
            tm = theta[i].copy()
            tp[k] += h[k]
            tm[k] -= h[k]
            pp, pm = _pixels(tp, t, c["L"], c["npix"]), \
                _pixels(tm, t, c["L"], c["npix"])
            clean = all(np.array_equal(a, b) and np.array_equal(a, cc)
                        for a, b, cc in zip(base, pp, pm))
            if not clean:
                continue
            fp = orc.chi2_theta(t, F, w, tp, A=A_o, L=c["L"])[0]
            fm = orc.chi2_theta(t, F, w, tm, A=A_o, L=c["L"])[0]
            fd = (fp - fm) / (2 * h[k])
            # scale: the largest of this component's FD and the gradient
            # magnitude a 1e-3 relative chi^2 change per unit step implies
            scale = max(abs(fd), 1e-3 * chi2[i] / max(h[k] * 1e6, 1e-12))
            rel.append(abs(grad[i, k] - fd) / scale)
            used += 1
    rel = np.array(rel)
    print(f"components compared: {used}; rel err median {np.median(rel):.2e}"
          f" p95 {np.quantile(rel, 0.95):.2e} max {rel.max():.2e}")
    assert used > 200
    assert np.median(rel) < 1e-4
    assert np.quantile(rel, 0.95) < 1e-3


def test_gradient_vs_polynomial_point_source(ctx, m):
    """Map gradient vs the FP64 gradient of the polynomial point-source
    chi^2 on 1000 smooth-region trajectories.

    The map holds the polynomial magnification at its texel centres
    (§4.1's point-source map), so the comparison measures the bilinear
    lookup's discretisation alone.  A ray-shot map would add the ray
    sampling's texel-to-texel noise, which differentiation amplifies by
    1/Delta: finer ray-shot maps agree worse, not better."""
    s, q, L, npix = 1.0, 1e-3, 1.0, 512
    P = orc.poly_map(s, q, L, npix, nthreads=NT)
    mp = ctx.map_from_host(P, L)
    # caustic texels: the image count changes between neighbours, found on
    # a 4x coarser grid and dilated by 2 coarse (8 fine) texels
    nc = npix // 4
    dc = 2 * L / nc
    cnt = np.array([[orc.images(s, q, -L + (i + 0.5) * dc,
                                -L + (j + 0.5) * dc)[0]
                     for i in range(nc)] for j in range(nc)], dtype=np.int8)
    edge = np.zeros_like(cnt, dtype=bool)
    edge[:, 1:] |= cnt[:, 1:] != cnt[:, :-1]
    edge[:, :-1] |= cnt[:, 1:] != cnt[:, :-1]
    edge[1:, :] |= cnt[1:, :] != cnt[:-1, :]
    edge[:-1, :] |= cnt[1:, :] != cnt[:-1, :]
    from scipy.ndimage import binary_dilation
    bad = binary_dilation(edge, iterations=2)
    t = synth.epoch_times(160, 13)
    t = t[np.abs(t) < 30]
    At = orc.lightcurve_point(s, q, t, 0.0, 20.0, 0.1, 0.6)
    F, sig = synth.photometry(At + 0.2, 13)
    w = 1.0 / sig ** 2
    ev = ctx.event(t, F, sig)
    rng = np.random.default_rng(2)
    thetas = []
    while len(thetas) < 1000:
        th = np.array([rng.uniform(-2, 2), rng.uniform(10, 40),
                       rng.uniform(0.05, 0.6), rng.uniform(0, 2 * np.pi)])
        px, py, inside = _pixels(th, t, L, nc)
        if inside.sum() < 10:
            continue
        if bad[py[inside].astype(int), px[inside].astype(int)].any():
            continue
        thetas.append(th)
    theta = np.array(thetas)
    chi2, grad, _, _ = ctx.chi2_grad(ev, mp, theta)
    rel = []
    for i in range(len(theta)):
        g = orc.chi2_grad_poly(t, F, w, theta[i], s, q)[1]
        # components in natural units: t0, tE per tE; u0 per u0; alpha
        sc = np.array([theta[i, 1], theta[i, 1], theta[i, 2], 1.0])
        rel.append(np.linalg.norm((grad[i] - g) * sc) /
                   np.linalg.norm(g * sc))
    rel = np.array(rel)
    print(f"map vs polynomial gradient: median rel {np.median(rel):.2e}, "
          f"p90 {np.quantile(rel, 0.9):.2e}, max {rel.max():.2e}")
    assert np.median(rel) < 1e-2
    assert np.quantile(rel, 0.9) < 1e-1


def test_refine_lowers_chi2_and_matches_oracle(ctx, m, setup):
    c, A_o, t, F, sig, mp, ev = setup
    g = c["grid"]
    grid = m.Grid.make(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"],
                       g["u0_lo"], g["u0_hi"], g["t0_lo"], g["t0_hi"],
                       g["tE_lo"], g["tE_hi"], True, True, 16)
    seeds = ctx.grid_chi2(ev, mp, grid)
    out = ctx.refine(ev, mp, seeds, iters=40)
    assert np.all(out["chi2"] <= seeds["chi2"] * (1 + 1e-12))
    assert out["chi2"].min() < seeds["chi2"].min()
    assert np.all(out["flags"] & m.FIT_REFINED)
    assert np.array_equal(out["idx"], seeds["idx"])
    w = 1.0 / sig ** 2
    for r in out[:6]:
        o = orc.chi2_theta(t, F, w, (r["t0"], r["tE"], r["u0"], r["alpha"]),
                           A=A_o, L=c["L"])[0]
        assert r["chi2"] == pytest.approx(o, rel=1e-5)
    # zero iterations return the starts unchanged
    same = ctx.refine(ev, mp, seeds[:4], iters=0)
    np.testing.assert_allclose(same["chi2"], seeds["chi2"][:4], rtol=1e-6)


def test_refine_from_grid_minima_across_maps(ctx, m):
    """Configuration 2's workload in small: the grid minima of several
    config-1-sized maps (1024^2, 10^8 FP32 rays) of one 3000-epoch event
    (truth s = 0.9, q = 5e-4), the best of them refined for 50
    iterations, each on its own map.  Checked: chi^2 never increases, the
    best refined chi^2 beats the best grid chi^2, and the records' chi^2
    equal the oracle's chi^2 at the refined (t0, tE, u0, alpha) on the same
    FP32 map values (1e-5)."""
    c = synth.CFG1
    t = synth.epoch_times(c["n"], c["seed"], c["t0"])
    At = orc.lightcurve_point(c["s"], c["q"], t, c["t0"], c["tE"], c["u0"],
                              c["alpha"])
    F, sig = synth.photometry(c["Fs"] * At + c["Fb"], c["seed"],
                              c["outliers"])
    w = 1.0 / sig ** 2
    ev = ctx.event(t, F, sig)
    g = c["grid"]
    grid = m.Grid.make(g["n_u0"], g["n_alpha"], g["n_t0"], g["n_tE"],
                       g["u0_lo"], g["u0_hi"], g["t0_lo"], g["t0_hi"],
                       g["tE_lo"], g["tE_hi"], True, True, 64)
    pairs = [(0.9, 5e-4), (0.85, 1e-3), (1.0, 2e-4)]
    maps = [ctx.build_map(s, q, c["L"], c["npix"], c["nray"],
                          image_halfwidth=c["X"], deflect="fp32")
            for s, q in pairs]
    fits = np.stack([ctx.grid_chi2(ev, mp, grid) for mp in maps])
    flat = fits.reshape(-1)
    mi = np.repeat(np.arange(len(maps)), grid.top_k)
    pick = np.argsort(flat["chi2"], kind="stable")[:96]
    best_grid = flat["chi2"][pick].min()
    best = np.inf
    for j, mp in enumerate(maps):
        st = flat[pick[mi[pick] == j]]
        if len(st) == 0:
            continue
        out = ctx.refine(ev, mp, st, iters=50)
        assert np.all(out["chi2"] <= st["chi2"] * (1 + 1e-12))
        best = min(best, out["chi2"].min())
        A = mp.values()
        for r in out[:: max(1, len(out) // 6)]:
            o = orc.chi2_theta(t, F, w, (r["t0"], r["tE"], r["u0"],
                                         r["alpha"]), A=A, L=c["L"])[0]
            assert r["chi2"] == pytest.approx(o, rel=1e-5)
    print(f"best grid chi^2 {best_grid:.2f}, refined {best:.2f}")
    assert best < best_grid
    # all maps in one call: each start's result equals its own map's call
    per_map = {}
    for j, mp in enumerate(maps):
        st = flat[pick[mi[pick] == j]]
        if len(st):
            per_map[j] = ctx.refine(ev, mp, st, iters=50)
    order = np.argsort(mi[pick], kind="stable")
    allst = flat[pick][order]
    got = ctx.refine_batch(ev, maps, mi[pick][order], allst, iters=50)
    want = np.concatenate([per_map[j] for j in sorted(per_map)])
    for f in ("chi2", "t0", "tE", "u0", "alpha", "Fs", "Fb", "idx", "flags"):
        assert np.array_equal(got[f], want[f]), f
    for mp in maps:
        mp.free()
    ev.free()


def test_autograd_function_and_lbfgs(ctx, m, setup):
    torch = pytest.importorskip("torch")
    c, A_o, t, F, sig, mp, ev = setup
    Chi2 = m.chi2_function()
    theta0 = np.array([[0.3, 18.0, 0.08, 0.6], [-0.5, 25.0, 0.04, 0.8]])
    th = torch.tensor(theta0, dtype=torch.float64, device="cuda",
                      requires_grad=True)
    y = Chi2.apply(th, ctx, ev, mp)
    y.sum().backward()
    chi2, grad, _, _ = ctx.chi2_grad(ev, mp, theta0)
    np.testing.assert_allclose(y.detach().cpu().numpy(), chi2, rtol=1e-12)
    np.testing.assert_allclose(th.grad.cpu().numpy(), grad, rtol=1e-12)
    # L-BFGS through the autograd function lowers chi^2
    p = torch.tensor(theta0[:1], dtype=torch.float64, device="cuda",
                     requires_grad=True)
    opt = torch.optim.LBFGS([p], lr=0.5, max_iter=20,
                            line_search_fn="strong_wolfe")

    def closure():
        opt.zero_grad()
        v = Chi2.apply(p, ctx, ev, mp).sum()
        v.backward()
        return v

    before = closure().item()
    opt.step(closure)
    after = Chi2.apply(p.detach(), ctx, ev, mp).sum().item()
    assert after < before


def test_gradient_rejects_bad_theta(ctx, m, setup):
    c, A_o, t, F, sig, mp, ev = setup
    for bad in ([0.0, -1.0, 0.1, 0.0], [np.nan, 10.0, 0.1, 0.0]):
        with pytest.raises(m.MorseError) as e:
            ctx.chi2_grad(ev, mp, np.array([bad]))
        assert e.value.status == m.EINVAL
