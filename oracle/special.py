"""Special functions for the oracle (FP64 numpy, exact rationals where noted).

Test infrastructure only (see the package docstring).

Conventions, Sec. II of the paper:
  * Y_l^m(theta, phi) = N_l^m P_l^m(cos theta) e^{i m phi},
    N_l^m = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!)                 (Eq. Sph_harmonics)
    with the Condon-Shortley phase (-1)^m inside P_l^m, so that
    Y_l^{-m} = (-1)^m conj(Y_l^m).
  * Wigner d^l_{m,m'}(beta) = <l m| exp(-i beta J_y) |l m'> (Sakurai), and
    D^l_{m,m'}(alpha, beta, gamma) = e^{-i m alpha} d^l_{m,m'}(beta) e^{-i m' gamma}
                                                                  (Eq. Dlm)
  * Triple product T(l',m'; p,q; l,m) = int Y_l'^m' Y_p^q conj(Y_l^m) ds
                                                        (Sec. III-B, after
                                                         Eq. harmonic_formulation)
"""

from fractions import Fraction
from math import factorial, isqrt, pi, sqrt

import numpy as np


# --------------------------------------------------------------------------
# Normalised associated Legendre functions and spherical harmonics
# --------------------------------------------------------------------------

def plm(lmax, m, x):
    """Ptilde_l^m(x) = N_l^m P_l^m(x) for l = 0..lmax, as an array [lmax+1, len(x)].

    Rows l < |m| are zero.  For m < 0, Ptilde_l^{m} = (-1)^m Ptilde_l^{|m|}
    (the Condon-Shortley relation behind Y_l^{-m} = (-1)^m conj Y_l^m).
    The recurrences are the standard ones for the orthonormal functions:
      Ptilde_0^0 = 1/sqrt(4 pi)
      Ptilde_m^m = -sqrt((2m+1)/(2m)) sqrt(1-x^2) Ptilde_{m-1}^{m-1}
      Ptilde_{m+1}^m = sqrt(2m+3) x Ptilde_m^m
      Ptilde_l^m = a_lm (x Ptilde_{l-1}^m - b_lm Ptilde_{l-2}^m),
        a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)).
    Pinned in tests against scipy.special.sph_harm_y and by orthonormality.
    """
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((lmax + 1,) + x.shape, dtype=np.float64)
    am = abs(m)
    if am > lmax:
        return out
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.full(x.shape, 1.0 / sqrt(4.0 * pi))
    for k in range(1, am + 1):
        pmm = -sqrt((2.0 * k + 1.0) / (2.0 * k)) * s * pmm
    out[am] = pmm
    if am + 1 <= lmax:
        out[am + 1] = sqrt(2.0 * am + 3.0) * x * pmm
    for l in range(am + 2, lmax + 1):
        a = sqrt((4.0 * l * l - 1.0) / (l * l - am * am))
        b = sqrt(((l - 1.0) ** 2 - am * am) / (4.0 * (l - 1.0) ** 2 - 1.0))
        out[l] = a * (x * out[l - 1] - b * out[l - 2])
    if m < 0 and (am % 2 == 1):
        out = -out
    return out


def sph_harm(l, m, theta, phi):
    """Y_l^m(theta, phi), Eq. Sph_harmonics (CS phase)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    p = plm(l, m, np.cos(theta))[l]
    return p * np.exp(1j * m * phi)


def sph_harm_all(L, theta, phi):
    """All Y_l^m for l < L at the given points; returns [L*L, npts] with the
    flat index l*l + l + m (the coefficient layout used everywhere)."""
    theta = np.asarray(theta, dtype=np.float64).ravel()
    phi = np.asarray(phi, dtype=np.float64).ravel()
    x = np.cos(theta)
    out = np.zeros((L * L, theta.size), dtype=np.complex128)
    for m in range(-(L - 1), L):
        p = plm(L - 1, m, x)
        e = np.exp(1j * m * phi)
        for l in range(abs(m), L):
            out[l * l + l + m] = p[l] * e
    return out


def gauss_legendre(n):
    """Gauss-Legendre nodes/weights on [-1, 1] (exact for degree <= 2n-1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return x.astype(np.float64), w.astype(np.float64)


# --------------------------------------------------------------------------
# Wigner d by the three-term recurrence in the degree
# --------------------------------------------------------------------------

def _d_start(l0, m, mp, c, s):
    """d^{l0}_{m,m'}(beta) for l0 = max(|m|,|m'|): the single surviving term of
    Wigner's explicit sum (c = cos(beta/2), s = sin(beta/2))."""
    if m == l0:        # d_{l,m'} = (-1)^{l-m'} sqrt(C(2l, l+m')) c^{l+m'} s^{l-m'}
        sign = -1.0 if (l0 - mp) % 2 else 1.0
        return sign * sqrt(_binom(2 * l0, l0 + mp)) * c ** (l0 + mp) * s ** (l0 - mp)
    if m == -l0:       # d_{-l,m'} = sqrt(C(2l, l-m')) c^{l-m'} s^{l+m'}
        return sqrt(_binom(2 * l0, l0 - mp)) * c ** (l0 - mp) * s ** (l0 + mp)
    if mp == l0:       # d_{m,l} = sqrt(C(2l, l+m)) c^{l+m} s^{l-m}
        return sqrt(_binom(2 * l0, l0 + m)) * c ** (l0 + m) * s ** (l0 - m)
    # mp == -l0:       d_{m,-l} = (-1)^{l+m} sqrt(C(2l, l-m)) c^{l-m} s^{l+m}
    sign = -1.0 if (l0 + m) % 2 else 1.0
    return sign * sqrt(_binom(2 * l0, l0 - m)) * c ** (l0 - m) * s ** (l0 + m)


def _binom(n, k):
    return float(factorial(n) // (factorial(k) * factorial(n - k)))


def wigner_d_table(Lh, betas):
    """d^p_{q,q'}(beta_n) for p < Lh, |q|,|q'| <= p, at every beta in ``betas``.

    Returns an array [Lh, 2Lh-1, 2Lh-1, nbeta]; entry [p, q+Lh-1, q'+Lh-1, n]
    (zero where |q| > p or |q'| > p).  Computed for each (q, q') by the
    textbook recurrence in the degree,
      l sqrt(((l+1)^2-m^2)((l+1)^2-m'^2)) d^{l+1}
        = (2l+1) (l(l+1) cos(beta) - m m') d^l - (l+1) sqrt((l^2-m^2)(l^2-m'^2)) d^{l-1},
    started from the closed form at l0 = max(|q|,|q'|).  This route uses no
    d(pi/2) table, so it checks the factorisation of Eq. WignerD_expansion_new
    independently.  Pinned in tests against Wigner's explicit sum, Legendre /
    spherical-harmonic special cases, the composition law d(b1+b2)=d(b1)d(b2)
    and unitarity.
    """
    betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
    K = 2 * Lh - 1
    out = np.zeros((Lh, K, K, betas.size), dtype=np.float64)
    cb = np.cos(betas)
    c = np.cos(betas / 2.0)
    s = np.sin(betas / 2.0)
    for m in range(-(Lh - 1), Lh):
        for mp in range(-(Lh - 1), Lh):
            l0 = max(abs(m), abs(mp))
            prev = np.zeros_like(betas)
            cur = _d_start(l0, m, mp, c, s)
            out[l0, m + Lh - 1, mp + Lh - 1] = cur
            for l in range(l0, Lh - 1):
                if l == 0:        # only m = m' = 0: d^1_00 = cos(beta)
                    nxt = cb.copy()
                else:
                    den = l * sqrt(((l + 1.0) ** 2 - m * m) * ((l + 1.0) ** 2 - mp * mp))
                    t1 = (2.0 * l + 1.0) * (l * (l + 1.0) * cb - m * mp)
                    t2 = (l + 1.0) * sqrt((l * l - m * m) * (l * l - mp * mp))
                    nxt = (t1 * cur - t2 * prev) / den
                prev, cur = cur, nxt
                out[l + 1, m + Lh - 1, mp + Lh - 1] = cur
    return out


def wigner_d_explicit(l, m, mp, beta):
    """Wigner's explicit finite sum for d^l_{m,m'}(beta) (Sakurai), FP64.

    Used only as a pin for the recurrence at small degree, where the
    alternating sum loses nothing significant.
      d^l_{m,m'} = sum_k (-1)^{k-m'+m} sqrt((l+m')!(l-m')!(l+m)!(l-m)!)
                   / ((l+m'-k)! k! (l-k-m)! (k-m'+m)!)
                   c^{2l-2k+m'-m} s^{2k-m'+m}
    """
    c = np.cos(np.asarray(beta, dtype=np.float64) / 2.0)
    s = np.sin(np.asarray(beta, dtype=np.float64) / 2.0)
    pref = sqrt(factorial(l + mp) * factorial(l - mp) * factorial(l + m) * factorial(l - m))
    tot = np.zeros_like(c)
    for k in range(0, 2 * l + 1):
        a, b, e, f = l + mp - k, k, l - k - m, k - mp + m
        if min(a, b, e, f) < 0:
            continue
        sign = -1.0 if (k - mp + m) % 2 else 1.0
        coef = pref / (factorial(a) * factorial(b) * factorial(e) * factorial(f))
        tot = tot + sign * coef * c ** (2 * l - 2 * k + mp - m) * s ** (2 * k - mp + m)
    return tot


# --------------------------------------------------------------------------
# Exact Wigner-3j (Racah's formula in rational arithmetic) and Gaunt
# --------------------------------------------------------------------------

def _sqrt_fraction(fr):
    """Correctly-rounded-ish float sqrt of a non-negative Fraction (error
    below 2^-60 relative before the final rounding)."""
    n, d = fr.numerator, fr.denominator
    if n == 0:
        return 0.0
    e = n.bit_length() - d.bit_length()
    k = 64 - e // 2
    if k >= 0:
        q = isqrt((n << (2 * k)) // d)
        return float(Fraction(q, 1 << k))
    q = isqrt(n // (d << (-2 * k)))
    return float(q << (-k))


def wigner3j_exact(j1, j2, j3, m1, m2, m3):
    """(j1 j2 j3; m1 m2 m3) by Racah's closed formula, evaluated exactly.

    value = (-1)^{j1-j2-m3} sqrt(Delta(j1 j2 j3) prod (j_i +- m_i)!)
            * sum_k (-1)^k / (k! (j3-j2+k+m1)! (j3-j1+k-m2)! (j1+j2-j3-k)!
                              (j1-k-m1)! (j2-k+m2)!)
    with Delta(abc) = (a+b-c)!(a-b+c)!(-a+b+c)!/(a+b+c+1)!.  The rational sum
    and the rational square of the prefactor are exact; only the final square
    root is rounded.  Integer arguments only (the transform needs no half
    integers).
    """
    if m1 + m2 + m3 != 0:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    if j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    f = factorial
    pre2 = Fraction(f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3), f(j1 + j2 + j3 + 1))
    pre2 *= f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3)
    kmin = max(0, j2 - j3 - m1, j1 - j3 + m2)
    kmax = min(j1 + j2 - j3, j1 - m1, j2 + m2)
    tot = Fraction(0)
    for k in range(kmin, kmax + 1):
        den = (f(k) * f(j3 - j2 + k + m1) * f(j3 - j1 + k - m2) * f(j1 + j2 - j3 - k)
               * f(j1 - k - m1) * f(j2 - k + m2))
        tot += Fraction(-1 if k % 2 else 1, den)
    if tot == 0:
        return 0.0
    mag = _sqrt_fraction(tot * tot * pre2)
    sign = -1.0 if (j1 - j2 - m3) % 2 else 1.0
    return sign * (1.0 if tot > 0 else -1.0) * mag


def wigner3j_m_family(j1, j2, j3, M, digits=100):
    """(j1 j2 j3; mu, M-mu, -M) for every order mu in
    [max(-j1, M-j2), min(j1, M+j2)], as (mu_min, list of floats).

    A second, independent route to large-degree 3j symbols (Racah's rational
    sum costs milliseconds a symbol at j ~ 2000).  The Clebsch-Gordan
    coefficients c(mu) = <j1 mu j2 q | j3 M>, q = M - mu, are the components
    of an eigenvector of J^2 = J1^2 + J2^2 + 2 J1z J2z + J1+ J2- + J1- J2+ with
    eigenvalue j3(j3+1); the component on |mu>|q> reads
      [j3(j3+1) - j1(j1+1) - j2(j2+1) - 2 mu q] c(mu) = a(mu) c(mu-1) + b(mu) c(mu+1),
      a(mu) = sqrt((j1-mu+1)(j1+mu)(j2+q+1)(j2-q)),  b(mu) = sqrt((j1+mu+1)(j1-mu)(j2-q+1)(j2+q)),
    and a vanishes at the lower end of the range.  The recursion runs upward
    from the lower end in decimal arithmetic with `digits` significant digits,
    then the family is normalised by sum_mu c(mu)^2 = 1 (orthonormality of
    the coupled basis).  Its sign is fixed at the lower end, where the
    recursion starts exactly: there the 3j symbol is, by the sign reversal
    of all orders, (-1)^(j1+j2+j3) times the upper end of the family of -M,
    whose Racah sum has a single positive term (m1 = j1 or m2 = -j2), so
    c(mu_min) has the sign (-1)^(j1-j2+j3).  (Near the upper end of a family
    that ends in a classically forbidden tail, upward recursion keeps only an
    absolute accuracy of about 10^-digits times the tail's decay ratio; with
    100 digits that is far below double precision of the family's norm.)
    Finally
      (j1 j2 j3; mu q -M) = (-1)^(j1-j2+M) c(mu) / sqrt(2 j3 + 1).
    """
    from decimal import Decimal, localcontext
    lo, hi = max(-j1, M - j2), min(j1, M + j2)
    if hi < lo or j3 < abs(j1 - j2) or j3 > j1 + j2 or abs(M) > j3:
        return lo, []
    with localcontext() as ctx:
        ctx.prec = digits
        lam = j3 * (j3 + 1) - j1 * (j1 + 1) - j2 * (j2 + 1)
        c = [Decimal(1)]
        prev = Decimal(0)
        for mu in range(lo, hi):
            q = M - mu
            d = Decimal(lam - 2 * mu * q)
            a = Decimal((j1 - mu + 1) * (j1 + mu) * (j2 + q + 1) * (j2 - q)).sqrt()
            b = Decimal((j1 + mu + 1) * (j1 - mu) * (j2 - q + 1) * (j2 + q)).sqrt()
            nxt = (d * c[-1] - a * prev) / b
            prev = c[-1]
            c.append(nxt)
            if abs(nxt) > Decimal(10) ** 200:       # rescale a long growing run
                c = [v / Decimal(10) ** 200 for v in c]
                prev = c[-2]
        norm = sum(v * v for v in c).sqrt()
        if (c[0] < 0) != ((j1 - j2 + j3) % 2 == 1):
            norm = -norm
        sign = -1 if (j1 - j2 + M) % 2 else 1
        fac = Decimal(sign) / (Decimal(2 * j3 + 1).sqrt() * norm)
        return lo, [float(v * fac) for v in c]


def gaunt_exact(lp, mp, p, q, l, m):
    """T(l',m'; p,q; l,m) = int Y_l'^m' Y_p^q conj(Y_l^m) ds via the 3j route
    (Sec. III-B writes this triple integral through Wigner-3j symbols):
      T = (-1)^m sqrt((2l'+1)(2p+1)(2l+1)/(4 pi)) (l' p l; 0 0 0)(l' p l; m' q -m).
    """
    if mp + q != m:
        return 0.0
    w0 = wigner3j_exact(lp, p, l, 0, 0, 0)
    if w0 == 0.0:
        return 0.0
    w1 = wigner3j_exact(lp, p, l, mp, q, -m)
    sign = -1.0 if m % 2 else 1.0
    return sign * sqrt((2 * lp + 1) * (2 * p + 1) * (2 * l + 1) / (4.0 * pi)) * w0 * w1


def gaunt_quadrature(lp, mp, p, q, l, m):
    """The same triple product by exact quadrature of its definition: the phi
    integral is 2 pi delta_{m'+q, m}, the theta integral a polynomial in
    cos(theta) of degree l'+p+l, done by Gauss-Legendre."""
    if mp + q != m:
        return 0.0
    n = (lp + p + l) // 2 + 1
    x, w = gauss_legendre(n)
    lmax = max(lp, p, l)
    a = plm(lmax, mp, x)[lp]
    b = plm(lmax, q, x)[p]
    c = plm(lmax, m, x)[l]
    return 2.0 * pi * float(np.sum(w * a * b * c))
