"""Plain numpy statement of the caustic geometry behind the (r, phi)
trajectory grid of McDougall & Albrow (2015) §4.2 (searching lines at fixed
distances from the centres of caustics, scaled by the caustic sizes), and a
plain reference search over such lines.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

* Critical curves (Eq. 4: det J = 0): with D = sum_k eps_k/(conj(z) - x_k)^2
  the critical points satisfy D = exp(-i psi) for some psi; for each psi
  that is a quartic in w = conj(z),
      eps1 (w - x2)^2 + eps2 (w - x1)^2 - exp(-i psi) (w - x1)^2 (w - x2)^2
      = 0,
  solved here by numpy's companion-matrix roots.  Caustic points are the
  critical points mapped by Eq. 2.
* The four roots are followed from one psi to the next by the pairing of
  least total distance; after a full turn the branches are permuted, and
  each cycle of that permutation is one closed critical curve, whose image
  is one caustic.
* A caustic's centre is the mean of its points (psi sampled uniformly) and
  its size the largest distance from the centre to one of them.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import lens, chi2_theta


def critical_points(s: float, q: float, n_psi: int) -> np.ndarray:
    """z[n_psi, 4] (complex): the critical points for psi_k = 2 pi k/n_psi,
    the branches of consecutive psi paired by least total distance."""
    e1, e2, x1, x2 = lens(s, q)
    out = np.zeros((n_psi, 4), dtype=complex)
    prev = None
    for k in range(n_psi):
        ph = np.exp(-1j * 2.0 * math.pi * k / n_psi)
        a = np.poly1d([1.0, -x1]) ** 2   # (w - x1)^2
        b = np.poly1d([1.0, -x2]) ** 2   # (w - x2)^2
        poly = e1 * b + e2 * a - ph * (a * b)
        w = np.roots(poly.coeffs)
        z = np.conj(w)
        if prev is not None:
            best = min(itertools.permutations(range(4)),
                       key=lambda p: sum(abs(z[p[i]] - prev[i])
                                         for i in range(4)))
            z = z[list(best)]
        out[k] = z
        prev = z
    return out


def caustic_of(s: float, q: float, z: np.ndarray) -> np.ndarray:
    """Caustic points zeta(z) by Eq. 2."""
    e1, e2, x1, x2 = lens(s, q)
    zc = np.conj(z)
    return z - e1 / (zc - x1) - e2 / (zc - x2)


def caustics(s: float, q: float, n_psi: int = 720):
    """[(c1, c2, size, n_points)] of the separate caustics, sorted by
    (c1, c2)."""
    z = critical_points(s, q, n_psi)
    # after a full turn, branch i continues as the branch nearest to it
    last, first = z[-1], z[0]
    perm = min(itertools.permutations(range(4)),
               key=lambda p: sum(abs(first[p[i]] - last[i])
                                 for i in range(4)))
    seen, cycles = set(), []
    for i in range(4):
        if i in seen:
            continue
        cyc, j = [], i
        while j not in seen:
            seen.add(j)
            cyc.append(j)
            j = perm[j]
        cycles.append(cyc)
    out = []
    for cyc in cycles:
        zeta = caustic_of(s, q, z[:, cyc].ravel())
        c = zeta.mean()
        out.append((c.real, c.imag, float(np.max(np.abs(zeta - c))),
                    len(zeta)))
    return sorted(out, key=lambda t: (round(t[0], 9), round(t[1], 9)))


def topology_count(s: float, q: float) -> int:
    """Number of caustics of a binary lens from the topology boundaries
    (Erdl & Schneider 1993): wide if s > ((1 + q^(1/3))^3/(1 + q))^(1/2),
    close if s^8 < (1 + q)^2 (1 - s^4)^3 / (27 q), else intermediate."""
    sw = math.sqrt((1.0 + q ** (1.0 / 3.0)) ** 3 / (1.0 + q))
    if s > sw:
        return 2
    if s < 1.0 and s ** 8 < (1.0 + q) ** 2 * (1.0 - s ** 4) ** 3 / (27.0 * q):
        return 3
    return 1


def rphi_lines(cs, n_r: int, r_lo: float, r_hi: float, n_phi: int):
    """(u, alpha, shift) of the lines of an (r, phi) grid about the
    caustics cs: impact r (linear in [r_lo, r_hi] times the caustic size)
    from the caustic centre C, direction phi_k = 2 pi k/n_phi; about the
    origin the line has impact u = r + C.n and its closest approach to C is
    at tau = shift = C.d past its closest approach to the origin
    (d = (cos phi, sin phi), n = (-sin phi, cos phi))."""
    out = []
    for c1, c2, size, _ in cs:
        for i in range(n_r):
            f = i / (n_r - 1) if n_r > 1 else 0.0
            r = (r_lo + (r_hi - r_lo) * f) * size
            for k in range(n_phi):
                phi = 2.0 * math.pi * k / n_phi
                d = (math.cos(phi), math.sin(phi))
                nrm = (-math.sin(phi), math.cos(phi))
                out.append((r + c1 * nrm[0] + c2 * nrm[1], phi,
                            c1 * d[0] + c2 * d[1]))
    return np.array(out)


def lines_chi2(lines, t0v, tEv, t, F, w, A, L):
    """chi^2 of every trajectory (line, t0, tE), index
    (line * n_t0 + i_t0) * n_tE + i_tE, t0 measured at the closest approach
    to the line's caustic centre."""
    out = []
    for u, phi, shift in lines:
        for t0 in t0v:
            for tE in tEv:
                th = (t0 - shift * tE, tE, u, phi)
                out.append(chi2_theta(t, F, w, th, A=A, L=L)[0])
    return np.array(out)
