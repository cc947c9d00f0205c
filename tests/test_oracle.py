"""Pins for the CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself or with the CUDA path.
Each one checks a closed form, an invariant, a special case that reduces to
a textbook routine, or brute force, chosen so that a plausible slip in the
oracle (a dropped term, a wrong sign or index, a transposed operand) fails:

* equal-mass lens, source at the origin: images and magnification in closed
  form (derived below from Eq. 2 with z on the real / imaginary axis);
* every returned image satisfies Eq. 2; the count is 3 or 5 (§3);
* five-image sources: signed magnifications sum to 1 (Witt & Mao 1995);
* q -> 0: the Paczynski curve (§4.3 (ii));
* ray shooting: ray conservation, mirror symmetry about the lens axis,
  thread-count invariance, and agreement with the pixel-averaged polynomial
  magnification and (q = 0) with the pixel-averaged Paczynski curve;
* bilinear lookup: reproduces a plane exactly (pins orientation and the
  half-texel offset), texel-centre values, the outside rule;
* trajectory geometry: closest approach u0 at t0, direction alpha;
* linear fit: equals weighted least squares by QR; chi^2 is a minimum;
* grid search: self-consistent injection recovers the injected index.
"""
import math

import numpy as np
import pytest

import oracle as orc
import synth


# ------------------------------------------------------------ lens polynomial
def equal_mass_origin(s):
    """Closed form for q = 1, source at the origin (lenses at +-s/2, eps=1/2).

    z = x real:  x - x/(x^2 - s^2/4) = 0  ->  x = 0 or x^2 = 1 + s^2/4.
    z = i y:     y - y/(y^2 + s^2/4) = 0  ->  y = 0 or y^2 = 1 - s^2/4.
    d = sum eps_k/(conj z - z_k)^2 is 4/s^2 at 0, 1 + s^2/2 on the real
    pair and s^2/2 - 1 on the imaginary pair; det J = 1 - |d|^2.
    """
    imgs = [(0.0, 1.0 - 16.0 / s ** 4)]
    x = math.sqrt(1.0 + s * s / 4.0)
    imgs += [(x, 1.0 - (1.0 + s * s / 2.0) ** 2),
             (-x, 1.0 - (1.0 + s * s / 2.0) ** 2)]
    if s < 2.0:
        y = math.sqrt(1.0 - s * s / 4.0)
        imgs += [(1j * y, 1.0 - (s * s / 2.0 - 1.0) ** 2),
                 (-1j * y, 1.0 - (s * s / 2.0 - 1.0) ** 2)]
    return imgs


@pytest.mark.parametrize("s", [0.5, 0.8, 1.0, 1.5, 1.9, 2.5, 4.0])
def test_equal_mass_closed_form(s):
    ref = equal_mass_origin(s)
    n, z, dj, res = orc.images(s, 1.0, 0.0, 0.0)
    assert n == len(ref)
    A_ref = sum(1.0 / abs(d) for _, d in ref)
    assert orc.mag_point(s, 1.0, 0.0, 0.0) == pytest.approx(A_ref, rel=1e-12)
    for zr, dr in ref:
        k = int(np.argmin(np.abs(z[:n] - zr)))
        assert abs(z[k] - zr) < 1e-12
        assert dj[k] == pytest.approx(dr, rel=1e-10, abs=1e-12)


def _lens_residual(s, q, z, zeta):
    e1, e2, xa, xb = orc.lens(s, q)
    zc = np.conj(z)
    return abs(z - e1 / (zc - xa) - e2 / (zc - xb) - zeta)


def test_lens_geometry():
    e1, e2, xa, xb = orc.lens(1.2, 0.25)
    assert e1 + e2 == pytest.approx(1.0)
    assert e2 / e1 == pytest.approx(0.25)
    assert xb - xa == pytest.approx(1.2)          # separation s
    assert e1 * xa + e2 * xb == pytest.approx(0.0, abs=1e-15)  # CoM origin
    assert xa < 0 < xb                            # primary on -x


@pytest.mark.parametrize("q", [1.0, 0.1, 1e-3, 1e-5])
@pytest.mark.parametrize("s", [0.3, 0.7, 1.0, 1.6, 3.0])
def test_images_solve_lens_equation(s, q):
    rng = np.random.default_rng(12345)
    for _ in range(40):
        y1, y2 = rng.uniform(-1.5, 1.5, 2)
        n, z, dj, res = orc.images(s, q, y1, y2)
        assert n in (3, 5)
        for k in range(n):
            r = _lens_residual(s, q, z[k], y1 + 1j * y2)
            scale = abs(z[k]) + math.hypot(y1, y2) + 1.0 / min(
                abs(z[k] - orc.lens(s, q)[2]), abs(z[k] - orc.lens(s, q)[3]))
            assert r <= 1e-10 * scale
        # quintic vanishes at every image
        c = orc.quintic(s, q, y1, y2)
        for k in range(n):
            pz = np.polyval(c[::-1], z[k])
            mag = np.polyval(np.abs(c[::-1]), abs(z[k]))
            assert abs(pz) <= 1e-9 * mag


def test_witt_mao_five_images():
    """Inside the caustic (5 images) the signed magnifications sum to 1."""
    rng = np.random.default_rng(7)
    seen = 0
    for q in (1.0, 0.3, 1e-2, 1e-3):
        for s in (0.6, 0.9, 1.0, 1.2):
            for _ in range(200):
                y1, y2 = rng.uniform(-0.3, 0.3, 2)
                n, z, dj, res = orc.images(s, q, y1, y2)
                if n == 5:
                    seen += 1
                    assert np.sum(1.0 / dj[:5]) == pytest.approx(1.0,
                                                                 abs=1e-8)
    assert seen > 50


@pytest.mark.parametrize("u", [0.05, 0.2, 0.7, 1.0, 1.8])
@pytest.mark.parametrize("s,q", [(1.0, 1e-10), (10.0, 1e-8)])
def test_q_to_zero_is_paczynski(u, s, q):
    """A planet of mass ratio q perturbs the single-lens curve by O(q); at
    q = 1e-10 on the Einstein ring, or 1e-8 far away, the Paczynski curve
    about the primary holds to 1e-6."""
    e1, e2, xa, xb = orc.lens(s, q)
    for ang in (0.3, 1.9, 4.0):
        y1 = xa + u * math.cos(ang)
        y2 = u * math.sin(ang)
        A = orc.mag_point(s, q, y1, y2)
        assert A == pytest.approx(orc.pspl(u), rel=1e-6)


def test_paczynski_closed_forms():
    assert orc.pspl(1.0) == pytest.approx(3.0 / math.sqrt(5.0), rel=1e-15)
    assert orc.pspl(1e-4) * 1e-4 == pytest.approx(1.0, rel=1e-7)
    u = 30.0
    assert orc.pspl(u) - 1.0 == pytest.approx(2.0 / u ** 4, rel=1e-2)


# ------------------------------------------------------------ ray shooting
def test_rayshoot_conservation_and_threads():
    c1, off1, lost1 = orc.rayshoot(0.9, 5e-3, 1.5, 64, 1500, 3.0, nthreads=1)
    c4, off4, lost4 = orc.rayshoot(0.9, 5e-3, 1.5, 64, 1500, 3.0, nthreads=4)
    assert int(c1.sum(dtype=np.uint64)) + off1 + lost1 == 1500 * 1500
    assert np.array_equal(c1, c4) and off1 == off4 and lost1 == lost4


def test_rayshoot_lost_ray_on_lens():
    # X = 0.75 with 3 rays per axis puts ray centres at -0.5, 0, 0.5;
    # s = 1, q = 1 puts the lenses at (-0.5, 0) and (0.5, 0): exactly two
    # rays sit on a lens and are counted as lost.
    c, off, lost = orc.rayshoot(1.0, 1.0, 2.0, 8, 3, 0.75, nthreads=1)
    assert lost == 2
    assert int(c.sum()) + off + lost == 9


def test_rayshoot_mirror_symmetry():
    npix = 64
    c, off, lost = orc.rayshoot(1.1, 0.02, 1.5, npix, 2000, 3.0, nthreads=4)
    flip = c[::-1, :]
    diff = np.abs(c.astype(np.int64) - flip.astype(np.int64)).sum()
    # only rays whose y2 sits on a bin edge (to rounding) may differ
    assert diff <= 1e-4 * c.sum()
    # but the map is not symmetric in y1 (q != 1): pins the axis order
    diffx = np.abs(c.astype(np.int64) - c[:, ::-1].astype(np.int64)).sum()
    assert diffx > 0.01 * c.sum()


def test_counts_to_mag_scale():
    c = np.full((8, 8), 7, dtype=np.uint32)
    A = orc.counts_to_mag(c, 1.0, 100, 2.0)
    h = 4.0 / 100
    d = 2.0 / 8
    assert np.all(A == np.float32(7 * (h * h) / (d * d)))


def _pixel_average(f, L, npix, sub):
    dl = 2 * L / npix
    P = np.zeros((npix, npix))
    G = np.zeros((npix, npix))
    for j in range(npix):
        for i in range(npix):
            v = np.array([f(-L + (i + (a + 0.5) / sub) * dl,
                            -L + (j + (b + 0.5) / sub) * dl)
                          for b in range(sub) for a in range(sub)])
            P[j, i] = v.mean()
            G[j, i] = v.max() / v.min()
    return P, G


def _smooth_mask(G, lim=1.3):
    from scipy.ndimage import binary_erosion
    return binary_erosion(G < lim, iterations=1)


def test_map_matches_polynomial_away_from_caustics():
    s, q, L, npix, nray, X = 1.0, 1e-2, 1.0, 32, 6000, 3.0
    A, c, off, lost = orc.build_map(s, q, L, npix, nray, X, nthreads=8)
    P, G = _pixel_average(lambda a, b: orc.mag_point(s, q, a, b), L, npix, 6)
    m = _smooth_mask(G)
    assert m.mean() > 0.5
    rel = (A - P) / P
    assert np.all(np.abs(rel[m]) <= 3.0 / np.sqrt(c[m]))
    assert abs(np.sum((A - P)[m]) / np.sum(P[m])) < 1e-3
    # the caustic region is where the two disagree most: the map is not
    # simply the polynomial at pixel centres
    assert np.max(np.abs(rel[~m])) > np.max(np.abs(rel[m]))


def test_map_single_lens_is_paczynski():
    L, npix, nray, X = 1.0, 24, 5000, 3.0
    A, c, off, lost = orc.build_map(1.0, 0.0, L, npix, nray, X, nthreads=8)
    P, G = _pixel_average(lambda a, b: orc.pspl(math.hypot(a, b)), L, npix, 8)
    m = _smooth_mask(G, 1.2)
    rel = (A - P) / P
    assert np.all(np.abs(rel[m]) <= 3.0 / np.sqrt(c[m]))
    assert abs(np.sum((A - P)[m]) / np.sum(P[m])) < 1e-3


def test_poly_map_texel_centres():
    # q -> 0: every texel centre carries the Paczynski closed form of its
    # distance from the lens (§4.3 (ii)); index order is [row j, column i]
    L, npix = 1.5, 12
    P = orc.poly_map(1.0, 1e-12, L, npix, nthreads=4)
    d = 2 * L / npix
    for j in range(npix):
        for i in range(npix):
            r = math.hypot(-L + (i + 0.5) * d - 0.0, -L + (j + 0.5) * d)
            assert P[j, i] == pytest.approx(orc.pspl(r), rel=1e-6)
    # binary lens: agrees with the independent ray-shot map in smooth
    # texels, to the pixel-averaging and shot-noise level
    s, q, L, npix = 1.0, 1e-2, 1.0, 32
    A, c, off, lost = orc.build_map(s, q, L, npix, 6000, 3.0, nthreads=8)
    Pm = orc.poly_map(s, q, L, npix, nthreads=4)
    Pa, G = _pixel_average(lambda a, b: orc.mag_point(s, q, a, b), L, npix, 6)
    m = _smooth_mask(G, 1.1)
    assert m.mean() > 0.5
    # centre value vs texel average differ by < 1e-2 where max/min < 1.1
    assert np.max(np.abs((Pa - Pm) / Pm)[m]) < 1e-2
    rel = (A - Pm) / Pm
    assert np.all(np.abs(rel[m]) <= 3.0 / np.sqrt(c[m]) + 1e-2)
    # transposing the map (rows <-> columns) breaks it: the lens axis is y1
    assert np.max(np.abs(Pm.T - A)[m]) > 5 * np.max(np.abs(Pm - A)[m])


# ------------------------------------------------------------ lookup
def test_lookup_reproduces_plane():
    npix, L = 16, 2.0
    jj, ii = np.meshgrid(np.arange(npix), np.arange(npix), indexing="ij")
    A = (1.0 + 2.0 * ii + 3.0 * jj).astype(np.float32)   # A[j, i]
    dl = 2 * L / npix
    rng = np.random.default_rng(3)
    for _ in range(200):
        y1, y2 = rng.uniform(-L + dl / 2, L - dl / 2, 2)
        px = (y1 + L) / dl - 0.5
        py = (y2 + L) / dl - 0.5
        assert orc.map_A(A, L, y1, y2) == pytest.approx(
            1.0 + 2.0 * px + 3.0 * py, rel=1e-12)


def test_lookup_texel_centres_edges_and_outside():
    npix, L = 8, 1.0
    rng = np.random.default_rng(4)
    A = rng.uniform(0.5, 3.0, (npix, npix)).astype(np.float32)
    dl = 2 * L / npix
    for j in range(npix):
        for i in range(npix):
            y1 = -L + (i + 0.5) * dl
            y2 = -L + (j + 0.5) * dl
            assert orc.map_A(A, L, y1, y2) == pytest.approx(float(A[j, i]),
                                                            rel=1e-12)
    # within half a texel of the edge: clamped to the edge texel centre
    assert orc.map_A(A, L, -L + 0.1 * dl, -L + 0.5 * dl) == pytest.approx(
        float(A[0, 0]), rel=1e-12)
    assert orc.map_A(A, L, L - 0.1 * dl, L - 0.2 * dl) == pytest.approx(
        float(A[-1, -1]), rel=1e-12)
    # outside: Paczynski about the centre of mass
    for y in [(L, 0.0), (-L - 0.3, 0.2), (0.1, 1.5 * L)]:
        assert orc.map_A(A, L, *y) == pytest.approx(
            orc.pspl(math.hypot(*y)), rel=1e-14)


def test_trajectory_geometry():
    t0, tE, u0, al = 3.0, 12.0, 0.2, 0.9
    y1, y2 = orc.traj_point(t0, t0, tE, u0, al)
    assert math.hypot(y1, y2) == pytest.approx(u0, rel=1e-14)
    # closest approach: position is perpendicular to the motion
    assert y1 * math.cos(al) + y2 * math.sin(al) == pytest.approx(0, abs=1e-15)
    # motion: one tE later the source moved by one unit along alpha
    z1, z2 = orc.traj_point(t0 + tE, t0, tE, u0, al)
    assert z1 - y1 == pytest.approx(math.cos(al), rel=1e-12)
    assert z2 - y2 == pytest.approx(math.sin(al), rel=1e-12)
    # counter-clockwise: the closest-approach point is alpha + 90 degrees
    assert math.atan2(y2, y1) == pytest.approx(al + math.pi / 2, rel=1e-12)


# ------------------------------------------------------------ linear fit
def test_fit_equals_weighted_lstsq():
    rng = np.random.default_rng(11)
    n = 37
    A = rng.uniform(1.0, 8.0, n)
    w = rng.uniform(100.0, 1e4, n)
    F = 0.7 * A + 0.4 + rng.normal(0, 1, n) / np.sqrt(w)
    chi2, fs, fb, flag = orc.fit_A(A, F, w)
    sw = np.sqrt(w)
    M = np.stack([A * sw, sw], axis=1)
    sol, *_ = np.linalg.lstsq(M, F * sw, rcond=None)
    assert flag == 0
    assert fs == pytest.approx(sol[0], rel=1e-10)
    assert fb == pytest.approx(sol[1], rel=1e-10)
    r = F - sol[0] * A - sol[1]
    assert chi2 == pytest.approx(float(np.sum(w * r * r)), rel=1e-10)
    for dfs, dfb in [(1e-4, 0), (-1e-4, 0), (0, 1e-4), (0, -1e-4)]:
        rr = F - (fs + dfs) * A - (fb + dfb)
        assert np.sum(w * rr * rr) > chi2


def test_fit_degenerate_constant_magnification():
    A = np.full(10, 2.5)
    F = np.linspace(1.0, 2.0, 10)
    w = np.arange(1, 11, dtype=float)
    chi2, fs, fb, flag = orc.fit_A(A, F, w)
    assert flag == 1 and fs == 0.0
    assert fb == pytest.approx(np.sum(w * F) / np.sum(w), rel=1e-14)
    assert chi2 == pytest.approx(float(np.sum(w * (F - fb) ** 2)), rel=1e-12)


# ------------------------------------------------------------ grid search
def test_axes():
    a = orc.axis(1e-3, 0.5, 20, True)
    assert a[0] == pytest.approx(1e-3) and a[-1] == pytest.approx(0.5)
    assert np.allclose(np.diff(np.log(a)), np.log(500.0) / 19)
    b = orc.axis(-2.0, 2.0, 10, False)
    assert np.allclose(np.diff(b), 4.0 / 9)


def test_grid_self_consistent_injection_recovers_index():
    """A noiseless light curve made by map lookup at grid trajectory k*
    gives chi^2 ~ 0 at k* and nowhere else (pins the index order)."""
    L, npix = 2.0, 64
    A, c, off, lost = orc.build_map(0.8, 0.05, L, npix, 1200, 3.0,
                                    nthreads=4)
    g = orc.Grid(3, 4, 3, 3, 0.05, 0.4, -1.0, 1.0, 8.0, 30.0)
    t = synth.epoch_times(50, 5)
    t = t[np.abs(t) < 25]
    for kstar in (0, 17, g.size - 1, 58):
        t0, tE, u0, al = g.params(kstar)
        At = orc.lightcurve_map(A, L, t, t0, tE, u0, al)
        F = 0.9 * At + 0.25
        w = np.full(len(t), 1e4)
        chi2, fs, fb, fl = orc.grid_chi2(g, t, F, w, A=A, L=L)
        assert int(np.argmin(chi2)) == kstar
        assert chi2[kstar] < 1e-12 * np.sum(w * F * F)
        assert fs[kstar] == pytest.approx(0.9, rel=1e-9)
        assert fb[kstar] == pytest.approx(0.25, rel=1e-8)
        idx, val = orc.topk(chi2, 5)
        assert idx[0] == kstar
        # brute force: every listed chi^2 is the plain definition
        for k in idx:
            p = g.params(int(k))
            Ak = orc.lightcurve_map(A, L, t, *p)
            assert orc.fit_A(Ak, F, w)[0] == pytest.approx(chi2[k], rel=1e-12)


def test_topk_order_and_ties():
    chi2 = np.array([5.0, 1.0, 3.0, 1.0, 2.0, 3.0])
    idx, val = orc.topk(chi2, 4, first=100)
    assert list(idx) == [101, 103, 104, 102]
    assert list(val) == [1.0, 1.0, 2.0, 3.0]


def test_grid_polynomial_mode_matches_lightcurve():
    g = orc.Grid(2, 3, 2, 2, 0.05, 0.3, -1.0, 1.0, 10.0, 20.0)
    t = synth.epoch_times(40, 9)
    F = 1.0 + 0.1 * np.cos(t)
    w = np.full(len(t), 100.0)
    chi2, fs, fb, fl = orc.grid_chi2(g, t, F, w, s=1.1, q=0.01)
    for k in (0, 5, g.size - 1):
        Ak = orc.lightcurve_point(1.1, 0.01, t, *g.params(k))
        assert orc.fit_A(Ak, F, w)[0] == pytest.approx(chi2[k], rel=1e-12)


# ------------------------------------------------------------ gradients
@pytest.mark.parametrize("u", [0.05, 0.3, 1.0, 2.5])
def test_mag_point_grad_single_lens_closed_form(u):
    # q -> 0: grad A = A'(u) y/u with A'(u) = -8 / (u^2 (u^2 + 4)^(3/2))
    y1, y2 = 0.6 * u, -0.8 * u
    a, g1, g2 = orc.mag_point_grad(1.0, 1e-12, y1, y2)
    d = -8.0 / (u * u * (u * u + 4.0) ** 1.5)
    assert a == pytest.approx(orc.pspl(u), rel=1e-9)
    assert g1 == pytest.approx(d * 0.6, rel=1e-7)
    assert g2 == pytest.approx(-d * 0.8, rel=1e-7)


@pytest.mark.parametrize("s,q", [(1.0, 1e-3), (0.7, 0.1), (1.3, 1.0)])
def test_mag_point_grad_matches_differences(s, q):
    rng = np.random.default_rng(11)
    n = 0
    for _ in range(120):
        y1, y2 = rng.uniform(-1.5, 1.5, 2)
        h = 1e-6
        n_img = [orc.images(s, q, y1 + a, y2 + b)[0]
                 for a, b in ((h, 0), (-h, 0), (0, h), (0, -h))]
        if len(set(n_img)) != 1:
            continue  # a caustic between the difference points
        a, g1, g2 = orc.mag_point_grad(s, q, y1, y2)
        f1 = (orc.mag_point(s, q, y1 + h, y2) -
              orc.mag_point(s, q, y1 - h, y2)) / (2 * h)
        f2 = (orc.mag_point(s, q, y1, y2 + h) -
              orc.mag_point(s, q, y1, y2 - h)) / (2 * h)
        assert math.hypot(g1 - f1, g2 - f2) <= 1e-6 * max(
            math.hypot(f1, f2), 1.0) + 1e-7 * a / h
        n += 1
    assert n > 100


def test_chi2_grad_poly_matches_differences_and_vanishes_at_truth():
    s, q = 1.0, 5e-3
    t = synth.epoch_times(120, 21)
    t = t[np.abs(t) < 30]
    truth = np.array([0.3, 18.0, 0.12, 0.9])
    At = orc.lightcurve_point(s, q, t, *truth)
    F = 1.3 * At + 0.4
    w = np.full(len(t), 1e4)
    c, g, fs, fb = orc.chi2_grad_poly(t, F, w, truth, s, q)
    # noiseless: chi^2 = 0 and the gradient vanishes at the truth
    assert c < 1e-16 and fs == pytest.approx(1.3) and fb == pytest.approx(0.4)
    assert np.all(np.abs(g) < 1e-5)
    rng = np.random.default_rng(4)
    for _ in range(6):
        th = truth * (1 + rng.uniform(-0.05, 0.05, 4))
        c, g, fs, fb = orc.chi2_grad_poly(t, F, w, th, s, q)
        assert c == pytest.approx(orc.chi2_theta(t, F, w, th, s=s, q=q)[0],
                                  rel=1e-12)
        for k in range(4):
            h = 1e-6 * abs(th[k])
            tp, tm = th.copy(), th.copy()
            tp[k] += h
            tm[k] -= h
            fd = (orc.chi2_theta(t, F, w, tp, s=s, q=q)[0] -
                  orc.chi2_theta(t, F, w, tm, s=s, q=q)[0]) / (2 * h)
            assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-6 * c / h)
        # a small step down the gradient lowers chi^2
        sc = np.array([th[1], th[1], th[2], 1.0]) ** 2
        step = 1e-4 * c / np.dot(g, g * sc) * g * sc
        assert orc.chi2_theta(t, F, w, th - step, s=s, q=q)[0] < c


# ------------------------------------------------------------ FP16 storage
def test_half_bits_definition_points_and_ties():
    cases = {0.0: 0x0000, 1.0: 0x3C00, -2.0: 0xC000, 65504.0: 0x7BFF,
             65519.99: 0x7BFF, 65520.0: 0x7C00, 2.0 ** -14: 0x0400,
             2.0 ** -24: 0x0001, 2.0 ** -25: 0x0000,   # tie -> even (0)
             1.5 * 2.0 ** -24: 0x0002,                 # tie -> even (2)
             1.0 + 2.0 ** -11: 0x3C00,                 # tie -> even
             1.0 + 3 * 2.0 ** -11: 0x3C02,             # tie -> even
             1.0 + 2.0 ** -11 + 2.0 ** -30: 0x3C01,    # above the tie
             0.1: 0x2E66, 1.0 / 3.0: 0x3555}
    for x, b in cases.items():
        assert orc.half_bits(x) == b, (x, hex(orc.half_bits(x)))
    for b in (0x0001, 0x03FF, 0x0400, 0x3C00, 0x3C01, 0x7BFF, 0xBC00):
        assert orc.half_bits(orc.half_value(b)) == b


def test_half_bits_match_numpy_float16():
    # an independent implementation of the same IEEE rounding
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.normal(0, 3, 20000),
                         rng.uniform(-1e-5, 1e-5, 5000),
                         10.0 ** rng.uniform(-9, 4.8, 5000)])
    ours = np.array([orc.half_bits(x) for x in xs], dtype=np.uint16)
    np.testing.assert_array_equal(ours, xs.astype(np.float16).view(np.uint16))


def test_log10_half_quantisation_bound():
    rng = np.random.default_rng(1)
    A = (10.0 ** rng.uniform(-0.3, 3.0, 50000)).astype(np.float32)
    A[:10] = 0.0   # empty texels take the floor
    codes = orc.log10_half(A, 1e-3)
    assert np.all(codes[:10] == orc.half_bits(-3.0))
    dec = orc.half_decode(codes)
    x = np.log10(A[10:].astype(np.float64))
    # half rounding moves x by at most half an ulp of x: 2^-11 |x| relative
    # for normal halves, so A moves by a factor 10^(2^-11 |x|) at most
    # (plus the FP32 rounding of the decoded value)
    bound = np.log(10) * np.maximum(2.0 ** -11 * np.abs(x), 2.0 ** -25) + 2e-7
    rel = np.abs(dec[10:] / A[10:] - 1.0)
    assert np.all(rel <= bound * 1.0001)
    assert rel.max() > 0.5 * bound.max() * 0.5  # the bound is not vacuous
    # A = 10^k for small k is exact in both directions
    assert orc.half_decode(orc.log10_half(np.array([1.0, 10.0, 100.0],
                                                   dtype=np.float32),
                                          1e-3)).tolist() == [1.0, 10.0, 100.0]


# ------------------------------------------------------------ finite source
@pytest.mark.parametrize("gamma", [0.0, 0.53, 1.0])
def test_fs_weights_second_moment_closed_form(gamma):
    # linear limb darkening in the Gamma form: <r^2> = rho^2 (1/2 - Gamma/10)
    # for the continuous profile; texel integration adds 1/6 (texel units)
    rho = 40.0
    W = orc.fs_weights(rho, gamma)
    R = (W.shape[0] - 1) // 2
    d = np.arange(-R, R + 1)
    assert W.sum() == pytest.approx(1.0, abs=1e-12)
    assert np.allclose(W, W[::-1, :]) and np.allclose(W, W.T)
    m2 = (W * (d[None, :] ** 2 + d[:, None] ** 2)).sum()
    closed = rho ** 2 * (0.5 - gamma / 10.0) + 1.0 / 6.0
    assert m2 == pytest.approx(closed, rel=1e-4)
    # the centre of the disc is brighter than its edge for Gamma > 0
    if gamma > 0:
        assert W[R, R] > W[R, R + int(rho) - 1]


def test_fs_convolve_identity_constant_plane_and_paraboloid():
    L, npix = 2.0, 96
    jj, ii = np.meshgrid(np.arange(npix), np.arange(npix), indexing="ij")
    # a source smaller than a texel: identity
    A = (2.0 + np.sin(ii * 0.3) * np.cos(jj * 0.2)).astype(np.float32)
    W0 = orc.fs_weights(0.3, 0.53)
    assert W0.shape == (3, 3)
    out = orc.fs_convolve(A, L, W0)
    np.testing.assert_array_equal(out, A.astype(np.float64))
    rho = 12.0
    W = orc.fs_weights(rho, 0.53)
    R = (W.shape[0] - 1) // 2
    inner = (slice(R, npix - R), slice(R, npix - R))
    # constant and plane: reproduced exactly away from the edge (symmetric
    # kernel, centred on the output texel)
    Pexact = 1.5 + 0.01 * ii + 0.02 * jj
    outP = orc.fs_convolve(Pexact.astype(np.float32), L, W)
    # up to the FP32 rounding of the input texels
    np.testing.assert_allclose(outP[inner], Pexact[inner], rtol=2e-7)
    # paraboloid: the second moment is added
    Q = (1.0 + 1e-3 * ((ii - 40.0) ** 2 + (jj - 50.0) ** 2)).astype(np.float32)
    outQ = orc.fs_convolve(Q, L, W)
    d = np.arange(-R, R + 1)
    m2 = (W * (d[None, :] ** 2 + d[:, None] ** 2)).sum()
    np.testing.assert_allclose(outQ[inner] - Q[inner], 1e-3 * m2, rtol=1e-6,
                               atol=1e-6)
    # outside the map the Paczynski curve stands in
    out_edge = orc.fs_convolve(np.ones((npix, npix), np.float32), L, W)
    assert out_edge[0, 0] > 1.0 and out_edge[npix // 2, npix // 2] == \
        pytest.approx(1.0, abs=1e-12)


def test_fs_uniform_disc_on_a_point_lens_centre():
    # uniform disc centred on a single lens: A = sqrt(1 + 4 / rho^2); the
    # area-averaged (ray-shot) map resolves the 1/u cusp
    L, npix, nray = 1.0, 64, 4000
    A, c, off, lost = orc.build_map(1.0, 1e-12, L, npix, nray, 3.0,
                                    nthreads=8)
    dlt = 2 * L / npix
    rho = 0.4  # Einstein radii
    W = orc.fs_weights(rho / dlt, 0.0)
    out = orc.fs_convolve(A, L, W, nthreads=4)
    # the lens sits on the corner of the four central texels
    centre = out[npix // 2 - 1:npix // 2 + 1, npix // 2 - 1:npix // 2 + 1]
    exact = np.sqrt(1 + 4 / rho ** 2)
    assert centre.mean() == pytest.approx(exact, rel=2e-3)


# ------------------------------------------------------------ line maxima
def _line_samples(A, L, u, al, n=60001, span=6.0):
    tau = np.linspace(-span, span, n)
    return np.array([orc.map_A(A, L, t * math.cos(al) - u * math.sin(al),
                               t * math.sin(al) + u * math.cos(al))
                     for t in tau])


def test_line_max_bounds_dense_samples():
    # brute force: no sample along the line exceeds the exact maximum, and
    # dense samples come close to it
    A, *_ = orc.build_map(1.0, 1e-2, 2.0, 48, 600, 3.0, nthreads=8)
    rng = np.random.default_rng(3)
    for _ in range(12):
        u = rng.uniform(-0.9, 0.9)
        al = rng.uniform(0, 2 * np.pi)
        mx = orc.line_max(A, 2.0, u, al)
        v = _line_samples(A, 2.0, u, al)
        assert v.max() <= mx * (1 + 1e-12)
        assert v.max() >= mx * (1 - 2e-3)


def test_line_max_plane_bump_and_outside():
    L, npix = 1.0, 32
    jj, ii = np.meshgrid(np.arange(npix), np.arange(npix), indexing="ij")
    # plane increasing in the first coordinate: a horizontal line peaks at
    # the last texel centre (the lookup is clamped beyond it)
    P = (10.0 + 0.5 * ii).astype(np.float32)
    assert orc.line_max(P, L, 0.3, 0.0) == pytest.approx(10.0 + 0.5 * 31,
                                                          rel=1e-13)
    # and transposed: a vertical line sees the constant of its column
    assert orc.line_max(P.T.copy(), L, 0.3, 0.0) < 10.0 + 0.5 * 31
    # one bright texel: a line through its centre meets it exactly
    B = np.ones((npix, npix), np.float32)
    B[20, 11] = 5.0
    d = 2 * L / npix
    y1, y2 = -L + 11.5 * d, -L + 20.5 * d
    al = 0.3
    u = -y1 * math.sin(al) + y2 * math.cos(al)  # the line through (y1, y2)
    assert orc.line_max(B, L, u, al) == pytest.approx(5.0, rel=1e-12)
    # a line that misses the map sees only the Paczynski curve, at its
    # closest approach
    assert orc.line_max(B, L, 3.0, 0.7) == pytest.approx(orc.pspl(3.0),
                                                         rel=1e-14)


# ------------------------------------------------------------ peak library
def _interior_maxima(v):
    """Brute force: indices i (0 < i < n - 1) with v[i] above both
    neighbours, for values with no two neighbours equal."""
    return [i for i in range(1, len(v) - 1) if v[i] > v[i - 1] and v[i] > v[i + 1]]


@pytest.mark.parametrize("axis", [0, 1])
def test_line_peaks_profile_maxima_brute_force(axis):
    # A map constant across the line: along a horizontal (vertical) line the
    # profile interpolates the column (row) values, sampled at every texel
    # centre and midpoint (sub = 2), so with delta = 0 its peaks are the
    # interior strict maxima of those values, at the centres' tau.
    L, npix = 2.0, 96
    rng = np.random.default_rng(11 + axis)
    col = rng.permutation(np.linspace(1.0, 9.0, npix)).astype(np.float32)
    A = np.tile(col, (npix, 1)) if axis == 0 else np.tile(col[:, None], (1, npix))
    A = np.ascontiguousarray(A)
    al = 0.0 if axis == 0 else math.pi / 2
    d = 2 * L / npix
    idx = _interior_maxima(col)
    count, pos, height = orc.line_peaks(A, L, [(0.3, al, 0.0)], sub=2,
                                        max_peaks=npix)
    assert count[0] == len(idx)
    got = pos[0][~np.isnan(pos[0])]
    want = np.array([-L + (i + 0.5) * d for i in idx])
    assert np.allclose(got, want, rtol=0, atol=1e-12)
    assert np.allclose(height[0][: len(idx)], col[idx], rtol=1e-4)
    # the three highest, in increasing tau; a shift moves every position
    top = sorted(sorted(idx, key=lambda i: -col[i])[:3])
    count, pos, height = orc.line_peaks(A, L, [(0.3, al, 0.25)], sub=2,
                                        max_peaks=3)
    assert count[0] == len(idx)
    assert np.allclose(pos[0], [-L + (i + 0.5) * d - 0.25 for i in top],
                       atol=1e-12)
    # the reversed direction sees the same peaks at -tau
    count, pos, _ = orc.line_peaks(A, L, [(-0.3, al + math.pi, 0.0)], sub=2,
                                   max_peaks=npix)
    assert count[0] == len(idx)
    assert np.allclose(np.sort(pos[0][~np.isnan(pos[0])]), np.sort(-want),
                       atol=1e-6)


def _bumps(L, npix, centres, heights, sigma):
    d = 2 * L / npix
    c = -L + (np.arange(npix) + 0.5) * d
    Y1, Y2 = np.meshgrid(c, c)  # Y1 varies along a row (first coordinate)
    A = np.ones((npix, npix))
    for (x, y), h in zip(centres, heights):
        A += h * np.exp(-((Y1 - x) ** 2 + (Y2 - y) ** 2) / (2 * sigma ** 2))
    return A.astype(np.float32)


def test_line_peaks_bumps_positions_heights_and_threshold():
    L, npix = 2.0, 256
    h = 2 * L / npix / 2
    # one round bump at the origin: every line through the map has one peak,
    # at its closest approach to the origin (tau = 0)
    A = _bumps(L, npix, [(0.0, 0.0)], [5.0], 0.3)
    lines = [(u, al, sh) for u in (-0.7, 0.0, 0.45) for al in (0.0, 0.9, 2.5)
             for sh in (0.0, 0.3)]
    count, pos, height = orc.line_peaks(A, L, lines, max_peaks=2)
    for j, (u, al, sh) in enumerate(lines):
        assert count[j] == 1
        assert abs(pos[j, 0] + sh) <= h
        assert height[j, 0] == pytest.approx(1 + 5 * math.exp(-u * u / 0.18),
                                             rel=2e-3)
        assert np.isnan(pos[j, 1])
    # a line that misses the map has no peak
    count, pos, _ = orc.line_peaks(A, L, [(3.0, 0.4, 0.0)])
    assert count[0] == 0 and np.isnan(pos[0]).all()
    # three bumps on the line y2 = 0.2 (alpha = 0: tau = y1)
    A = _bumps(L, npix, [(-1.0, 0.2), (0.0, 0.2), (0.8, 0.2)],
               [3.0, 6.0, 4.0], 0.12)
    count, pos, height = orc.line_peaks(A, L, [(0.2, 0.0, 0.0)], max_peaks=8)
    assert count[0] == 3
    assert np.allclose(pos[0, :3], [-1.0, 0.0, 0.8], atol=h)
    assert np.allclose(height[0, :3], [4.0, 7.0, 5.0], rtol=5e-3)
    # the two highest, in increasing tau
    count, pos, _ = orc.line_peaks(A, L, [(0.2, 0.0, 0.0)], max_peaks=2)
    assert np.allclose(pos[0], [0.0, 0.8], atol=h)
    # threshold: two close bumps with a shallow dip count once when the dip
    # is within the factor 1 + delta, twice with delta = 0
    A = _bumps(L, npix, [(-0.15, 0.0), (0.15, 0.0)], [5.0, 4.8], 0.1)
    prof = [orc.map_A(A, L, t, 0.0) for t in np.linspace(-0.3, 0.3, 601)]
    dip = min(prof[150:451])
    assert 1.3 < max(prof) / dip < 1.6  # the dip lies within the factor 1.6
    assert orc.line_peaks(A, L, [(0.0, 0.0, 0.0)], delta=0.0)[0][0] == 2
    assert orc.line_peaks(A, L, [(0.0, 0.0, 0.0)], delta=0.3)[0][0] == 2
    c1, p1, h1 = orc.line_peaks(A, L, [(0.0, 0.0, 0.0)], delta=0.6)
    assert c1[0] == 1
    assert abs(p1[0, 0] + 0.15) <= 2 * h and h1[0, 0] > 5.5


def test_peak_alignment_eq7_eq8_puts_model_peaks_at_the_given_times():
    # Eq. 7: the trajectory t0 = t_p - M_p tE peaks at t_p; Eq. 8: with two
    # peaks, tE = (t_p2 - t_p1)/(M_b - M_a) puts them at t_p1 and t_p2.
    L, npix = 2.0, 256
    # (bump centres off the midpoints between texel centres, so that each
    # top is one texel centre, not a flat stretch between two)
    A = _bumps(L, npix, [(-0.905, 0.2), (0.53, 0.2)], [4.0, 6.0], 0.1)
    line = [(0.2, 0.0, 0.1)]
    count, pos, _ = orc.line_peaks(A, L, line, max_peaks=4)
    assert count[0] == 2
    t = np.linspace(50.0, 200.0, 30001)

    def peaks_of(row):
        _, u, al, t0, tE = row
        lc = np.array(orc.lightcurve_map(A, L, t, t0, tE, u, al))
        # maxima of the sampled light curve (a top may be two equal samples)
        return [t[i] for i in range(1, len(lc) - 1)
                if lc[i] >= lc[i - 1] and lc[i] > lc[i + 1] and lc[i] > 2.0]

    tp0 = 120.0
    # Eq. 7: one family per peak, every tE of the axis (t0 offset 0)
    rows = orc.peak_trajectories(line, count, pos, [tp0], [0.0], [25.0])
    assert rows.shape == (2, 5)
    for r in rows:
        pk = peaks_of(r)
        assert min(abs(p - tp0) for p in pk) < 0.2 * 25.0 * 2 * L / npix
    # the t0 offsets shift the aligned peak by the offset
    rows = orc.peak_trajectories(line, count, pos, [tp0], [-3.0, 3.0],
                                 [25.0])
    assert rows.shape == (4, 5)
    assert sorted(rows[:, 3] - rows[0, 3])[-1] == pytest.approx(6.0, abs=1e-9)
    # Eq. 8: the one pair (a, b) of the two peaks fixes tE and t0
    rows = orc.peak_trajectories(line, count, pos, [tp0, 160.0], [0.0],
                                 [25.0], min_peaks=2)
    assert rows.shape == (1, 5)
    r = rows[0]
    assert r[4] == pytest.approx(40.0 / 1.435, rel=2e-2)
    pk = peaks_of(r)
    assert len(pk) == 2
    assert abs(pk[0] - 120.0) < 0.2 and abs(pk[1] - 160.0) < 0.2
    # a line with fewer peaks than required contributes no trajectory
    rows = orc.peak_trajectories(line, count, pos, [tp0], [0.0], [25.0],
                                 min_peaks=3)
    assert rows.shape == (0, 5)
    # no peak time: the line grid itself, t0 about the reference point
    rows = orc.peak_trajectories(line, count, pos, [], [1.0, 2.0],
                                 [10.0, 20.0], min_peaks=2)
    assert rows.shape == (4, 5)
    assert rows[0, 3] == pytest.approx(1.0 - 0.1 * 10.0)


def test_peak_library_fp32_bounds_cover_a_rounded_profile():
    # The FP64 library's error bounds: a profile evaluated with the sample
    # positions and values perturbed within the stated FP32 bounds (here:
    # the texels rounded to FP32 twice over and the positions shifted by a
    # tenth of a texel's FP32 resolution) gives the same count and
    # positions on every line the library does not flag, and heights
    # within herr.
    L, npix = 2.0, 128
    rng = np.random.default_rng(5)
    A = (1.0 + rng.gamma(4.0, 0.25, size=(npix, npix))).astype(np.float32)
    lines = [(u, al, 0.0) for u in np.linspace(-1.5, 1.5, 13)
             for al in np.linspace(0.0, 3.0, 11)]
    c, p, h, e, uns = orc.line_peaks(A, L, lines, sub=2, delta=0.05,
                                     max_peaks=6, bounds=True)
    # a one-ulp change of every texel moves each value by far less than
    # its bound: unflagged lines keep their library
    A2 = np.nextafter(A, np.float32(np.inf))
    c2, p2, h2 = orc.line_peaks(A2, L, lines, sub=2, delta=0.05,
                                max_peaks=6)
    ok = ~uns
    assert ok.sum() > 0.8 * len(lines)
    assert np.array_equal(c[ok], c2[ok])
    assert np.array_equal(p[ok], p2[ok])
    fin = np.isfinite(h[ok])
    assert (np.abs(h[ok][fin] - h2[ok][fin]) <= e[ok][fin]).all()
    # a plateau (four equal texels) puts two samples at one value: a
    # near-tie of the running maximum, which the library flags
    B = np.ones((npix, npix), dtype=np.float32)
    B[60:62, 60:62] = 5.0
    d = 2 * L / npix
    y = -L + 60.5 * d
    cb, pb, hb, eb, ub = orc.line_peaks(B, L, [(y, 0.0, 0.0)], sub=2,
                                        delta=0.1, max_peaks=2, bounds=True)
    assert cb[0] == 1 and ub[0]


# ------------------------------------------------------------ caustics
def test_critical_points_and_caustic_count_by_topology():
    from oracle import caustics as oc
    for s, q in [(0.5, 1e-2), (0.7, 0.3), (1.0, 1.0), (1.0, 1e-3),
                 (1.6, 1e-3), (2.5, 5e-4), (0.9, 0.1)]:
        z = oc.critical_points(s, q, 360)
        e1, e2, x1, x2 = orc.lens(s, q)
        D = e1 / (np.conj(z) - x1) ** 2 + e2 / (np.conj(z) - x2) ** 2
        assert np.allclose(np.abs(D), 1.0, atol=1e-9)
        cs = oc.caustics(s, q, 720)
        assert len(cs) == oc.topology_count(s, q), (s, q, cs)
        # mirror symmetry about the lens axis
        ys = sorted(round(c[1], 6) for c in cs)
        assert np.allclose(ys, sorted(-y for y in ys), atol=1e-6)


def test_caustic_positions_and_image_count_change():
    from oracle import caustics as oc
    # equal masses, s = 1: one caustic centred on the origin
    (c,) = oc.caustics(1.0, 1.0, 720)
    assert abs(c[0]) < 1e-9 and abs(c[1]) < 1e-9
    # wide, small q: the planetary caustic near s - 1/s from the primary
    s, q = 2.5, 5e-4
    e1, e2, x1, x2 = orc.lens(s, q)
    cs = oc.caustics(s, q, 720)
    planet = max(cs, key=lambda t: t[0])
    assert planet[0] - x1 == pytest.approx(s - 1.0 / s, rel=0.02)
    assert planet[2] < 0.05
    # across a caustic the number of images changes by two
    z = oc.critical_points(1.2, 0.05, 720)
    zeta = oc.caustic_of(1.2, 0.05, z[:, 0])
    changed = 0
    for k in range(10, 720, 37):
        tang = zeta[k + 1] - zeta[k - 1]
        nrm = 1j * tang / abs(tang)
        eps = 1e-4 * abs(tang)
        a = orc.images(1.2, 0.05, (zeta[k] + eps * nrm).real,
                       (zeta[k] + eps * nrm).imag, 1e-9)[0]
        b = orc.images(1.2, 0.05, (zeta[k] - eps * nrm).real,
                       (zeta[k] - eps * nrm).imag, 1e-9)[0]
        changed += {a, b} == {3, 5}
    assert changed >= 17  # of 20 (cusps excepted)
