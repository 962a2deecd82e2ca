"""Oracle: conversion of a physical problem to the canonical form.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything under ``oracle/``.

Paper Sec. 2.2 (canonical form) and Sec. 3.1 (Helmholtz):
  A0 = L0 + V0;  A = A0/c, L = L0/c, y = y0/c, V = A - L,  ||V|| = 0.95.
Helmholtz  laplacian(psi) + k^2 psi = -S:
  L0 = laplacian + kbar2 with kbar2 the centre of the smallest circle that
  encloses the values k^2(r) (the smallest-circle problem), radius rho;
  c = -rho / (0.95 i) = i rho / 0.95, so that max |V| = 0.95 and A is
  accretive.  V = (k^2 - kbar2)/c, y = -S/c, L^(p) = (-|p|^2 + kbar2)/c.
Diffusion  -D laplacian(u) + eta u = S  (scalar constant D, steady state):
  the values eta(r) are real, their smallest circle is the interval's
  midpoint etabar and half-range rho; c = rho/0.95 (real, positive so that
  A stays accretive).  V = (eta - etabar)/c, y = S/c,
  L^(p) = (D |p|^2 + etabar)/c.
"""

import numpy as np


def _circle_two(a, b):
    c = 0.5 * (a + b)
    return c, abs(a - c)


def _circle_three(a, b, c):
    """Circumcircle of three points (complex numbers); None if collinear."""
    ax, ay, bx, by, cx, cy = a.real, a.imag, b.real, b.imag, c.real, c.imag
    d = 2.0 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
    if d == 0.0:
        return None
    a2, b2, c2 = ax * ax + ay * ay, bx * bx + by * by, cx * cx + cy * cy
    ux = (a2 * (by - cy) + b2 * (cy - ay) + c2 * (ay - by)) / d
    uy = (a2 * (cx - bx) + b2 * (ax - cx) + c2 * (bx - ax)) / d
    centre = complex(ux, uy)
    return centre, abs(a - centre)


def _inside(p, circ, eps=1e-12):
    c, r = circ
    return abs(p - c) <= r * (1.0 + eps) + eps


def _hull_points(pts):
    """The smallest enclosing circle is fixed by points on the convex hull,
    so large sets are first reduced to their hull vertices (library convex
    hull).  Collinear sets reduce to their two extreme points."""
    from scipy.spatial import ConvexHull, QhullError
    xy = np.stack([pts.real, pts.imag], axis=1)
    try:
        hull = ConvexHull(xy)
        return pts[hull.vertices]
    except QhullError:
        d = pts - pts[0]
        k = int(np.argmax(np.abs(d)))
        u = d[k] / abs(d[k])
        s = np.real(d * np.conj(u))
        return pts[[int(np.argmin(s)), int(np.argmax(s))]]


def min_enclosing_circle(points, seed=12345):
    """Smallest circle enclosing complex ``points`` (Welzl's randomised
    incremental algorithm, expected linear time).  Returns (centre, radius)."""
    pts = np.unique(np.asarray(points, np.complex128).ravel())
    if pts.size == 0:
        raise ValueError("no points")
    if pts.size > 4096:
        pts = _hull_points(pts)
    rng = np.random.default_rng(seed)
    pts = pts[rng.permutation(pts.size)]
    P = [complex(p) for p in pts]
    circ = (P[0], 0.0)
    for i in range(1, len(P)):
        if _inside(P[i], circ):
            continue
        circ = (P[i], 0.0)
        for j in range(i):
            if _inside(P[j], circ):
                continue
            circ = _circle_two(P[i], P[j])
            for k in range(j):
                if _inside(P[k], circ):
                    continue
                c3 = _circle_three(P[i], P[j], P[k])
                if c3 is None:   # collinear: the two farthest points span it
                    cands = [_circle_two(P[i], P[j]), _circle_two(P[i], P[k]),
                             _circle_two(P[j], P[k])]
                    c3 = max(cands, key=lambda t: t[1])
                circ = c3
    return circ


def helmholtz(k2, S, dx, norm_v=0.95):
    """Canonical form of laplacian(psi) + k^2 psi = -S.  Returns a dict with
    V, y (complex128), the symbol coefficients a, b of L^ = a|p|^2 + b, the
    scale c and the bias kbar2."""
    kbar2, rho = min_enclosing_circle(k2)
    if rho <= 0.0:
        raise ValueError("homogeneous medium: the scale c is undefined")
    c = -rho / (norm_v * 1j)
    V = (np.asarray(k2, np.complex128) - kbar2) / c
    y = -np.asarray(S, np.complex128) / c
    return dict(V=V, y=y, a=-1.0 / c, b=kbar2 / c, c=c, bias=kbar2, dx=dx)


def diffusion(eta, D, S, dx, norm_v=0.95):
    """Canonical form of -D laplacian(u) + eta u = S."""
    eta = np.asarray(eta, np.float64)
    lo, hi = float(eta.min()), float(eta.max())
    etabar, rho = 0.5 * (lo + hi), 0.5 * (hi - lo)
    if rho <= 0.0:
        raise ValueError("homogeneous medium: the scale c is undefined")
    c = rho / norm_v
    V = (eta - etabar) / c
    y = np.asarray(S, np.complex128) / c
    return dict(V=V.astype(np.complex128), y=y, a=D / c, b=etabar / c,
                c=c, bias=etabar, dx=dx)


def canonical(problem, norm_v=0.95):
    """Canonical form of a problem dict from the seeded generators."""
    if problem["kind"] == "helmholtz":
        return helmholtz(problem["k2"], problem["S"], problem["dx"], norm_v)
    return diffusion(problem["eta"], problem["D"], problem["S"], problem["dx"],
                     norm_v)
