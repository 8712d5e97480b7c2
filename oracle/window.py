"""The elliptical concentration window of Sec. III-D, in FP64 on the CPU.

Test infrastructure only (see the package docstring).  It is the reference the
device generator (slsht_window_ellipse) is checked against, and the script
``tests/golden/make_windows.py`` stores its windows of workloads 2 and 5 as
test inputs.

The window is the band-limited function of largest energy fraction inside the
elliptical region R(theta_c, a) around the north pole (Eq. region_def): the
points x whose great-circle distances to the two foci (theta_c, 0) and
(theta_c, pi) add up to at most 2a.  Its coefficients are the top eigenvector
of the concentration matrix of Sec. III-D,
    D_{(l m),(l' m')} = int_R conj(Y_l^m(x)) Y_l'^m'(x) ds(x),   l, l' < L,
and its eigenvalue is the concentration.  The eigenvector is made real-valued
(h_{l,-m} = (-1)^m conj(h_lm): the region is symmetric under phi -> -phi),
normalised to unit energy and signed so that h_0^0 > 0, which the inverse of
Eq. inversion_2 needs.

Quadrature of the integral over R, ring by ring: for each longitude phi the
region is 0 <= theta <= theta_b(phi), theta_b found by bisection on the
focal-distance sum; theta by Gauss-Legendre on [0, theta_b(phi)] (the
integrand is smooth there), phi by the trapezoid rule (theta_b is smooth and
periodic, so the rule converges spectrally).  Band limits are exclusive.

Parity: pinned by tests/test_window.py against the paper's printed 90 %
concentration (Sec. V-B), the Shannon number trace D = L^2 Area(R) / 4 pi
(addition theorem), the polar-cap limits theta_c = 0 and a = pi/2 where D
decouples the orders, the eigenvalue range [0, 1] and the symmetries above.
"""

from math import pi

import numpy as np

from . import special


def angular_distance(t1, p1, t2, p2):
    """Great-circle distance between (t1, p1) and (t2, p2) (the Delta_s of
    Eq. region_def)."""
    c = np.sin(t1) * np.sin(t2) * np.cos(p1 - p2) + np.cos(t1) * np.cos(t2)
    return np.arccos(np.clip(c, -1.0, 1.0))


def boundary(theta_c, a, phi, iters=80):
    """theta_b(phi): the largest colatitude on meridian phi inside
    R(theta_c, a), by bisection on the focal-distance sum (monotone in theta
    along a meridian through the pole for theta_c <= a < pi/2)."""
    phi = np.asarray(phi, dtype=np.float64)
    lo = np.zeros_like(phi)
    hi = np.full_like(phi, a)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        s = angular_distance(mid, phi, theta_c, 0.0) + angular_distance(mid, phi, theta_c, pi)
        inside = s <= 2.0 * a
        lo = np.where(inside, mid, lo)
        hi = np.where(inside, hi, mid)
    return 0.5 * (lo + hi)


def region_rule(theta_c, a, L, nphi=None, ntheta=None):
    """Nodes (theta, phi) and weights of a rule for int_R F ds, F band-limited
    of degree <= 2(L-1): nphi longitudes (default 8L+64), ntheta Gauss-Legendre
    nodes per ring (default 2L+24), weight sin(theta) dtheta dphi."""
    nphi = nphi or (8 * L + 64)
    ntheta = ntheta or (2 * L + 24)
    phi = 2.0 * pi * np.arange(nphi) / nphi
    tb = boundary(theta_c, a, phi)
    t, wt = special.gauss_legendre(ntheta)
    th = 0.5 * (t[None, :] + 1.0) * tb[:, None]                  # [nphi, ntheta]
    w = (0.5 * tb[:, None] * wt[None, :]) * np.sin(th) * (2.0 * pi / nphi)
    ph = np.broadcast_to(phi[:, None], th.shape)
    return th.ravel(), np.ascontiguousarray(ph).ravel(), w.ravel()


def concentration_matrix(theta_c, a, L, nodes_per_block=4096, **kw):
    """D_{(l m),(l' m')} = int_R conj(Y_l^m) Y_l'^m' ds for l, l' < L (flat
    index l*l + l + m), summed over the nodes of region_rule in blocks (the
    sum is the quadrature itself; blocking only bounds the memory)."""
    th, ph, w = region_rule(theta_c, a, L, **kw)
    n = L * L
    D = np.zeros((n, n), dtype=np.complex128)
    for s in range(0, th.size, nodes_per_block):
        e = slice(s, s + nodes_per_block)
        Y = special.sph_harm_all(L, th[e], ph[e])                 # [L*L, nodes]
        B = Y * np.sqrt(w[e])[None, :]
        D += np.conj(B) @ B.T
    return D


def mirror(v, L):
    """(S v)_lm = (-1)^m conj(v_{l,-m}): the coefficients of conj of the
    function, so S v = v exactly when the function is real-valued."""
    out = np.zeros_like(v)
    for l in range(L):
        for m in range(-l, l + 1):
            out[l * l + l + m] = (-1) ** (m % 2) * np.conj(v[l * l + l - m])
    return out


def window_ellipse(L, theta_c, a, **kw):
    """Top eigenfunction of the concentration problem of Sec. III-D.

    Returns (h, lambda): h complex128 [L*L], unit energy, real-valued function
    (h_{l,-m} = (-1)^m conj(h_lm)), h_0^0 > 0; lambda its concentration (the
    fraction of its energy inside R).  D is Hermitian and commutes with S (the
    region is symmetric under phi -> -phi), so the non-degenerate top
    eigenvector satisfies S v = e^{i psi} v and e^{i psi / 2} v is real."""
    D = concentration_matrix(theta_c, a, L, **kw)
    lam, vec = np.linalg.eigh(D)
    v = vec[:, -1]
    psi = np.angle(np.vdot(v, mirror(v, L)))
    h = v * np.exp(0.5j * psi)
    if h[0].real < 0:
        h = -h
    h = h / np.linalg.norm(h)
    return h, float(lam[-1])
