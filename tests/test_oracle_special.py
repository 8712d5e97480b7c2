"""Pins for the oracle's special functions (CPU only).

Each check compares against something other than the function itself:
library routines (scipy), exact rational arithmetic, closed forms and the
identities Sec. II and IV of the paper state.
"""
from fractions import Fraction
from math import factorial, pi, sqrt

import numpy as np
import pytest

from oracle import special as S
from oracle import slsht as O


# ---------------------------------------------------------------- Y_l^m

def _scipy_Y(l, m, theta, phi):
    sp = pytest.importorskip("scipy.special")
    if hasattr(sp, "sph_harm_y"):
        return sp.sph_harm_y(l, m, theta, phi)
    return sp.sph_harm(m, l, phi, theta)      # older scipy: (m, n, azimuth, polar)


def test_sph_harm_matches_scipy():
    rng = np.random.default_rng(0)
    th = rng.uniform(0, pi, 50)
    ph = rng.uniform(0, 2 * pi, 50)
    for l in range(0, 25):
        for m in range(-l, l + 1):
            ours = S.sph_harm(l, m, th, ph)
            ref = _scipy_Y(l, m, th, ph)
            assert np.max(np.abs(ours - ref)) < 1e-12, (l, m)


def test_sph_harm_orthonormal():
    L = 12
    th, ph, w = O.sphere_rule(2 * (L - 1))
    Y = S.sph_harm_all(L, th, ph)
    G = (Y * w) @ Y.conj().T
    assert np.max(np.abs(G - np.eye(L * L))) < 1e-13


def test_conjugation_symmetry():
    th = np.linspace(0.1, 3.0, 7)
    ph = np.linspace(0.2, 6.0, 7)
    for l in range(6):
        for m in range(1, l + 1):
            a = S.sph_harm(l, -m, th, ph)
            b = (-1) ** m * np.conj(S.sph_harm(l, m, th, ph))
            assert np.max(np.abs(a - b)) < 1e-15


# ---------------------------------------------------------------- Wigner d

BETAS = np.array([0.0, 0.3, 1.1, pi / 2, 2.2, 3.0, pi])


def test_d_recurrence_vs_explicit_sum():
    Lh = 9
    d = S.wigner_d_table(Lh, BETAS)
    for p in range(Lh):
        for q in range(-p, p + 1):
            for qp in range(-p, p + 1):
                e = S.wigner_d_explicit(p, q, qp, BETAS)
                assert np.max(np.abs(d[p, q + Lh - 1, qp + Lh - 1] - e)) < 5e-15


def test_d_low_order_closed_forms():
    d = S.wigner_d_table(3, BETAS)
    c = np.cos(BETAS)
    o = 2
    assert np.allclose(d[1, 1 + o, 0 + o], -np.sin(BETAS) / sqrt(2), atol=1e-15)
    assert np.allclose(d[1, 1 + o, 1 + o], (1 + c) / 2, atol=1e-15)
    assert np.allclose(d[1, 1 + o, -1 + o], (1 - c) / 2, atol=1e-15)
    assert np.allclose(d[2, 1 + o, 1 + o], (1 + c) * (2 * c - 1) / 2, atol=1e-15)
    assert np.allclose(d[2, 0 + o, 0 + o], (3 * c * c - 1) / 2, atol=1e-15)


def test_d_m0_is_spherical_harmonic():
    """d^l_{m,0}(beta) = sqrt(4 pi/(2l+1)) Y_l^m(beta, 0) and d^l_00 = P_l(cos beta)."""
    sp = pytest.importorskip("scipy.special")
    Lh = 20
    b = np.linspace(0.05, 3.1, 11)
    d = S.wigner_d_table(Lh, b)
    for l in range(Lh):
        assert np.max(np.abs(d[l, Lh - 1, Lh - 1] - sp.eval_legendre(l, np.cos(b)))) < 1e-13
        for m in range(-l, l + 1):
            ref = sqrt(4 * pi / (2 * l + 1)) * _scipy_Y(l, m, b, 0.0 * b).real
            assert np.max(np.abs(d[l, m + Lh - 1, Lh - 1] - ref)) < 1e-13, (l, m)


def test_d_composition_and_unitarity():
    """d(b1 + b2) = d(b1) d(b2) (rotations about one axis compose) and d d^T = 1."""
    Lh = 24
    b1, b2 = 0.7, 1.9
    d = S.wigner_d_table(Lh, [b1, b2, b1 + b2])
    for p in range(Lh):
        sl = slice(Lh - 1 - p, Lh + p)
        A, B, C = d[p, sl, sl, 0], d[p, sl, sl, 1], d[p, sl, sl, 2]
        assert np.max(np.abs(A @ B - C)) < 1e-13
        assert np.max(np.abs(A @ A.T - np.eye(2 * p + 1))) < 1e-13


def test_d_symmetries_printed_in_paper():
    """d_{q,q'}(b) = (-1)^{q-q'} d_{q,q'}(-b) = (-1)^{q-q'} d_{-q,-q'}(b)
       = (-1)^{q-q'} d_{q',q}(b) = d_{-q',-q}(b)   (Sec. IV-B)."""
    Lh = 10
    b = np.array([0.4, 1.3, 2.7])
    d = S.wigner_d_table(Lh, np.concatenate([b, -b]))
    o = Lh - 1
    for p in range(Lh):
        for q in range(-p, p + 1):
            for qp in range(-p, p + 1):
                s = (-1) ** ((q - qp) % 2)
                v = d[p, q + o, qp + o, :3]
                assert np.allclose(v, s * d[p, q + o, qp + o, 3:], atol=1e-14)
                assert np.allclose(v, s * d[p, -q + o, -qp + o, :3], atol=1e-14)
                assert np.allclose(v, s * d[p, qp + o, q + o, :3], atol=1e-14)
                assert np.allclose(v, d[p, -qp + o, -q + o, :3], atol=1e-14)


def _delta_exact(p, m, mp):
    """d^p_{m,m'}(pi/2) exactly: with c = s = 2^{-1/2} every term of Wigner's
    sum carries 2^{-p}, so Delta = 2^{-p} sqrt((p+m)!(p-m)!(p+m')!(p-m')!) * R
    with R a rational sum; evaluated in exact arithmetic."""
    R = Fraction(0)
    for k in range(0, 2 * p + 1):
        a, b, e, f = p + mp - k, k, p - k - m, k - mp + m
        if min(a, b, e, f) < 0:
            continue
        sign = -1 if (k - mp + m) % 2 else 1
        R += Fraction(sign, factorial(a) * factorial(b) * factorial(e) * factorial(f))
    pre = factorial(p + m) * factorial(p - m) * factorial(p + mp) * factorial(p - mp)
    if R == 0:
        return 0.0
    mag = S._sqrt_fraction(R * R * pre / Fraction(4 ** p))
    return mag if R > 0 else -mag


def test_delta_pi_half_exact():
    """The Delta = d(pi/2) matrices the fast algorithm uses (Sec. IV-B), against
    exact rational evaluation, up to degree 40."""
    Lh = 41
    d = S.wigner_d_table(Lh, [pi / 2])[..., 0]
    rng = np.random.default_rng(1)
    for p in [0, 1, 2, 5, 11, 17, 26, 33, 40]:
        idx = [(m, mp) for m in range(-p, p + 1) for mp in range(-p, p + 1)]
        if len(idx) > 60:
            idx = [idx[i] for i in rng.choice(len(idx), 60, replace=False)]
        for m, mp in idx:
            assert abs(d[p, m + Lh - 1, mp + Lh - 1] - _delta_exact(p, m, mp)) < 2e-14, (p, m, mp)


def test_delta_factorisation_of_D():
    """Eq. WignerD_expansion_new: D^p_{q,q'}(a,b,g) =
    i^{q-q'} sum_{q''} Delta^p_{q''q} Delta^p_{q''q'} e^{-i q a - i q'' b - i q' g},
    with the sign of the beta exponent as printed."""
    Lh = 12
    a, b, g = 0.37, 1.21, 2.9
    d = S.wigner_d_table(Lh, [b, pi / 2])
    o = Lh - 1
    for p in range(Lh):
        for q in range(-p, p + 1):
            for qp in range(-p, p + 1):
                lhs = np.exp(-1j * q * a) * d[p, q + o, qp + o, 0] * np.exp(-1j * qp * g)
                acc = 0.0j
                for qpp in range(-p, p + 1):
                    acc += d[p, qpp + o, q + o, 1] * d[p, qpp + o, qp + o, 1] * np.exp(-1j * qpp * b)
                rhs = (1j) ** ((q - qp) % 4) * acc * np.exp(-1j * q * a - 1j * qp * g)
                assert abs(lhs - rhs) < 1e-14, (p, q, qp)


# ---------------------------------------------------------------- 3j / Gaunt

def test_3j_known_values():
    assert abs(S.wigner3j_exact(1, 1, 0, 0, 0, 0) + 1 / sqrt(3)) < 3e-16
    assert abs(S.wigner3j_exact(1, 1, 2, 0, 0, 0) - sqrt(2 / 15)) < 3e-16
    assert abs(S.wigner3j_exact(1, 1, 0, 1, -1, 0) - 1 / sqrt(3)) < 3e-16
    assert abs(S.wigner3j_exact(2, 2, 2, 0, 0, 0) + sqrt(2 / 35)) < 3e-16
    assert S.wigner3j_exact(1, 1, 1, 0, 0, 0) == 0.0
    # (j1 j2 j3; 000) closed form, J even, g = J/2
    for j1, j2, j3 in [(3, 4, 5), (10, 7, 5), (20, 12, 14)]:
        J = j1 + j2 + j3
        gg = J // 2
        cf = (-1) ** gg * sqrt(factorial(J - 2 * j1) * factorial(J - 2 * j2) * factorial(J - 2 * j3)
                               / factorial(J + 1)) * factorial(gg) / (
            factorial(gg - j1) * factorial(gg - j2) * factorial(gg - j3))
        assert abs(S.wigner3j_exact(j1, j2, j3, 0, 0, 0) - cf) < 1e-15


def test_3j_symmetries_and_sum_rules():
    rng = np.random.default_rng(2)
    for _ in range(25):
        j1, j2 = int(rng.integers(0, 9)), int(rng.integers(0, 9))
        j3 = int(rng.integers(abs(j1 - j2), j1 + j2 + 1))
        m1 = int(rng.integers(-j1, j1 + 1))
        m2 = int(rng.integers(-j2, j2 + 1))
        m3 = -m1 - m2
        if abs(m3) > j3:
            continue
        v = S.wigner3j_exact(j1, j2, j3, m1, m2, m3)
        ph = (-1) ** (j1 + j2 + j3)
        assert abs(S.wigner3j_exact(j2, j3, j1, m2, m3, m1) - v) < 1e-15      # cyclic
        assert abs(S.wigner3j_exact(j2, j1, j3, m2, m1, m3) - ph * v) < 1e-15  # odd perm
        assert abs(S.wigner3j_exact(j1, j2, j3, -m1, -m2, -m3) - ph * v) < 1e-15
    # sum_{m1,m2} (3j)^2 = 1/(2 j3 + 1); orthogonality over j3
    j1, j2, j3, m3 = 4, 3, 5, 2
    tot = sum(S.wigner3j_exact(j1, j2, j3, m1, -m3 - m1, m3) ** 2
              for m1 in range(-j1, j1 + 1) if abs(m3 + m1) <= j2)
    assert abs(tot - 1 / (2 * j3 + 1)) < 1e-15
    for m1 in range(-j1, j1 + 1):
        m2 = 1 - m1
        if abs(m2) > j2:
            continue
        tot = sum((2 * J + 1) * S.wigner3j_exact(j1, j2, J, m1, m2, -1) ** 2
                  for J in range(abs(j1 - j2), j1 + j2 + 1))
        assert abs(tot - 1.0) < 1e-14


def test_gaunt_quadrature_vs_3j():
    rng = np.random.default_rng(3)
    n = 0
    while n < 40:
        lp, p, l = (int(v) for v in rng.integers(0, 14, 3))
        q = int(rng.integers(-p, p + 1))
        mp = int(rng.integers(-lp, lp + 1))
        m = mp + q
        if abs(m) > l:
            continue
        n += 1
        assert abs(S.gaunt_exact(lp, mp, p, q, l, m) - S.gaunt_quadrature(lp, mp, p, q, l, m)) < 1e-14


def test_wigner3j_order_family_matches_racah():
    """The order-recursion families agree with Racah's exact sum, at small
    degrees for every order and at l ~ 2000 (workload 5) at both ends and in
    the middle of a 127-term family."""
    import random
    rng = random.Random(7)
    for _ in range(150):
        j1, j2 = rng.randint(0, 22), rng.randint(0, 22)
        j3 = rng.randint(abs(j1 - j2), j1 + j2)
        M = rng.randint(-j3, j3)
        lo, fam = S.wigner3j_m_family(j1, j2, j3, M)
        for i, v in enumerate(fam):
            mu = lo + i
            assert abs(v - S.wigner3j_exact(j1, j2, j3, mu, M - mu, -M)) <= 1e-15 * max(1.0, abs(v))
    lo, fam = S.wigner3j_m_family(1999, 63, 2022, 1202)
    assert len(fam) == 127
    for mu in (lo, lo + 1, lo + 63, lo + 126):
        e = S.wigner3j_exact(1999, 63, 2022, mu, 1202 - mu, -1202)
        assert abs(fam[mu - lo] - e) <= 1e-14 * abs(e)
