"""Elliptical concentration windows (Sec. III-D of the paper).

The window is an INPUT of the transform: the band-limited function of maximal
energy concentration in the elliptical region R_(theta_c, a) around the north
pole (Eq. region_def), i.e. the top eigenvector of the concentration matrix
  D_{(l m),(l' m')} = int_R conj(Y_l^m) Y_l'^m' ds,
normalised to unit energy, made real-valued (the region is symmetric under
phi -> -phi) and signed so that h_0^0 > 0 (needed by the inverse).

The integral over R is done ring by ring: for each longitude phi the region
is 0 <= theta <= theta_b(phi), with theta_b found by bisection on the
focal-distance sum; theta is integrated by Gauss-Legendre on [0, theta_b(phi)]
and phi by the trapezoid rule (spectrally accurate: theta_b is smooth and
periodic).  Band limit L is exclusive (l < L).
"""

from math import pi, sqrt

import numpy as np


def _plm_block(L, x):
    """Orthonormal associated Legendre Ptilde_l^m(x) (Condon-Shortley phase)
    for 0 <= m <= l < L, as [L, L, nx] indexed [l, m]."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    out = np.zeros((L, L) + x.shape)
    pmm = np.full(x.shape, 1.0 / sqrt(4.0 * pi))
    for m in range(L):
        if m > 0:
            pmm = -sqrt((2.0 * m + 1.0) / (2.0 * m)) * s * pmm
        out[m, m] = pmm
        if m + 1 < L:
            out[m + 1, m] = sqrt(2.0 * m + 3.0) * x * pmm
        for l in range(m + 2, L):
            a = sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            out[l, m] = a * (x * out[l - 1, m] - b * out[l - 2, m])
    return out


def ellipse_from_axes(a_deg, b_deg):
    """(theta_c, a) in radians from the semi-major and semi-minor arcs.

    The foci lie on the major axis at colatitude theta_c; for a spherical
    ellipse centred on the pole, cos(a) = cos(theta_c) cos(b)."""
    a = np.deg2rad(a_deg)
    b = np.deg2rad(b_deg)
    return float(np.arccos(np.cos(a) / np.cos(b))), float(a)


def _angdist(t1, p1, t2, p2):
    """Angular distance on the unit sphere (the Delta_s of Eq. region_def)."""
    c = np.sin(t1) * np.sin(t2) * np.cos(p1 - p2) + np.cos(t1) * np.cos(t2)
    return np.arccos(np.clip(c, -1.0, 1.0))


def boundary(theta_c, a, phi, iters=80):
    """theta_b(phi): largest colatitude on meridian phi inside R_(theta_c, a)."""
    phi = np.asarray(phi, dtype=np.float64)
    lo = np.zeros_like(phi)
    hi = np.full_like(phi, a)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        s = _angdist(mid, phi, theta_c, 0.0) + _angdist(mid, phi, theta_c, pi)
        inside = s <= 2.0 * a
        lo = np.where(inside, mid, lo)
        hi = np.where(inside, hi, mid)
    return 0.5 * (lo + hi)


def region_rule(theta_c, a, L, nphi=None, ntheta=None):
    """Quadrature nodes (theta, phi) and weights for integrals over R_(theta_c, a)
    of band-limited integrands (degree <= 2L)."""
    nphi = nphi or (8 * L + 64)
    ntheta = ntheta or (2 * L + 24)
    phi = 2.0 * pi * np.arange(nphi) / nphi
    tb = boundary(theta_c, a, phi)
    t, wt = np.polynomial.legendre.leggauss(ntheta)
    th = 0.5 * (t[None, :] + 1.0) * tb[:, None]                      # [nphi, nt]
    w = (0.5 * tb[:, None] * wt[None, :]) * np.sin(th) * (2.0 * pi / nphi)
    ph = np.broadcast_to(phi[:, None], th.shape)
    return th.ravel(), np.ascontiguousarray(ph).ravel(), w.ravel()


def concentration_matrix(theta_c, a, L, **kw):
    """D_{(l m),(l' m')} = int_R conj(Y_l^m) Y_l'^m' ds for l, l' < L (flat index l*l+l+m)."""
    th, ph, w = region_rule(theta_c, a, L, **kw)
    P = _plm_block(L, np.cos(th))                                     # [l, m>=0, n]
    Y = np.zeros((L * L, th.size), dtype=np.complex128)
    for m in range(L):
        e = np.exp(1j * m * ph)
        for l in range(m, L):
            Y[l * l + l + m] = P[l, m] * e
            if m > 0:
                Y[l * l + l - m] = (-1) ** m * P[l, m] * np.conj(e)
    B = np.conj(Y) * np.sqrt(w)[None, :]
    return B @ B.conj().T


def window_ellipse(L, theta_c, a, **kw):
    """Top eigenfunction of the concentration problem: returns (h, lambda).

    h: complex128 [L*L], unit energy, real-valued function
    (h_{l,-m} = (-1)^m conj(h_lm)), h_00 > 0.  lambda: its concentration
    (fraction of energy inside R)."""
    D = concentration_matrix(theta_c, a, L, **kw)
    lam, vec = np.linalg.eigh(D)
    v = vec[:, -1]
    # S v = (-1)^m conj(v_{l,-m}); for the (non-degenerate) top eigenvector
    # S v = e^{i psi} v, and e^{i psi/2} v is a fixed point of S.
    Sv = np.zeros_like(v)
    for l in range(L):
        for m in range(-l, l + 1):
            Sv[l * l + l + m] = (-1) ** (m % 2) * np.conj(v[l * l + l - m])
    ph = np.vdot(v, Sv)
    h = v * np.exp(0.5j * np.angle(ph))
    if h[0].real < 0:
        h = -h
    h = h / np.linalg.norm(h)
    return h, float(lam[-1])
