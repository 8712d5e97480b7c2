"""Pins for the oracle's forward and inverse transform (CPU only).

The two forward routes share nothing but the spherical harmonics: the
quadrature route never uses a Wigner function (the window is rotated
geometrically), the coefficient route never evaluates f or h on the sphere.
On top of their mutual agreement, each special case the paper states
(Sec. III) or that follows from its definitions is checked.
"""
import json
import os
from math import floor, pi, sqrt

import numpy as np
import pytest

import synth
from oracle import slsht as O
from oracle import special as S

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _all_pairs(lmax):
    return [(l, m) for l in range(lmax + 1) for m in range(-l, l + 1)]


# ------------------------------------------------------ forward: two routes

def test_quadrature_and_coefficient_routes_agree_config1():
    """Workload 1 (L_f=16, L_h=4, all l<16, grid 31x16x7), both routes in full."""
    c = synth.CONFIGS[1]
    f, h, pairs = synth.config_inputs(1)
    g_q = O.forward_quadrature(f, h, c["Lf"], c["Lh"], pairs, c["grid"])
    g_c = O.forward_coeff(f, h, c["Lf"], c["Lh"], pairs, c["grid"])
    assert _rel(g_q, g_c) < 1e-13


def test_routes_agree_above_Lf_and_odd_grids():
    Lf, Lh = 6, 3
    f = synth.signal_cn_real(Lf, 11)
    h = synth.window_cn(Lh, 12)
    pairs = _all_pairs(Lf + Lh - 2)
    for grid in [(5, 3, 1), (9, 5, 4), (2, 7, 3)]:
        g_q = O.forward_quadrature(f, h, Lf, Lh, pairs, grid)
        g_c = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
        assert _rel(g_q, g_c) < 1e-13, grid


def test_modulated_sht_vs_exact_gaunt():
    """Appendix A's separated form (Gauss-Legendre, exact) against the
    triple-product sum with exact 3j symbols (Eq. harmonic_formulation)."""
    Lf, Lh = 9, 4
    f = synth.signal_powerlaw(Lf, 5)
    ms = O.ModulatedSHT(f, Lf, Lh, Lf + Lh - 2)
    for l, m in [(0, 0), (3, -2), (8, 8), (8, -5), (10, 3), (11, -11)]:
        k1 = ms.coeffs(l, m)
        k2 = O.modulated_coeffs_gaunt(f, Lf, Lh, l, m)
        assert np.max(np.abs(k1 - k2)) < 1e-14, (l, m)


def test_modulated_sht_accuracy_at_high_degree():
    """At l = 255 (workload 3) the quadrature route of Appendix A stays within
    its documented ~1e-11 of the exact-3j route the oracle uses by default."""
    Lf, Lh = 256, 16
    f = synth.signal_powerlaw(Lf, 3001)
    ms = O.ModulatedSHT(f, Lf, Lh, 255)
    for l, m in [(255, -1), (255, 255), (128, 3)]:
        ke = O.modulated_coeffs_gaunt(f, Lf, Lh, l, m)
        kq = ms.coeffs(l, m)
        assert np.linalg.norm(kq - ke) / np.linalg.norm(ke) < 5e-11


# ------------------------------------------------------ conventions

def test_rotation_geometric_equals_wigner_D():
    """(D_rho h)(x) = h(R^{-1} x) has coefficients sum_m' D^l_{m m'} h_l^m'
    (Eq. rotation_non_symm, Eq. Dlm)."""
    L = 6
    h = synth.window_cn(L, 3)
    th, ph, w = O.sphere_rule(2 * (L - 1))
    pts = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    Yc = np.conj(S.sph_harm_all(L, th, ph))
    for rho in [(0.3, 1.0, 2.0), (4.0, 2.5, 0.7), (0.0, np.pi / 2, 0.0)]:
        R = O.rotation_matrix(*rho)
        y = R.T @ pts
        vals = O.eval_signal(h, L, np.arccos(np.clip(y[2], -1, 1)), np.arctan2(y[1], y[0]))
        coef = Yc @ (w * vals)
        assert np.max(np.abs(coef - O.rotate_coeffs(h, L, *rho))) < 1e-13


# ------------------------------------------------------ special cases

def test_constant_signal_gives_rotated_window():
    """f = f00 Y_0^0 (a constant): g(rho; l, m) = (f00/sqrt(4 pi)) (D_rho h)_l^m."""
    Lf, Lh = 3, 4
    f = np.zeros(Lf * Lf, complex)
    f[0] = 0.7 - 0.2j
    h = synth.window_cn(Lh, 8)
    grid = (5, 4, 3)
    pairs = _all_pairs(Lh - 1)
    g = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    a, b, c = O.grid_angles(*grid)
    for i, j, k in [(0, 0, 0), (1, 2, 1), (4, 3, 2)]:
        rh = O.rotate_coeffs(h, Lh, a[i], b[j], c[k])
        ref = f[0] / sqrt(4 * pi) * np.array([rh[l * l + l + m] for l, m in pairs])
        assert np.max(np.abs(g[:, i, j, k] - ref)) < 1e-14


def test_window_Y00_gives_signal_coefficients():
    """h = Y_0^0: g(rho; l, m) = f_lm / sqrt(4 pi) for every rho."""
    Lf, Lh = 7, 1
    f = synth.signal_cn_real(Lf, 4)
    h = np.ones(1, complex)
    g = O.forward_coeff(f, h, Lf, Lh, _all_pairs(Lf - 1), (3, 2, 1))
    ref = f / sqrt(4 * pi)
    assert np.max(np.abs(g - ref[:, None, None, None])) < 1e-15


def test_azimuthally_symmetric_window_is_gamma_independent():
    """h_p^{q'} = 0 for q' != 0: g does not depend on gamma (remark after
    Definition 1; the ordinary SLSHT)."""
    Lf, Lh = 8, 5
    f = synth.signal_cn_real(Lf, 6)
    h = synth.window_cn(Lh, 7)
    for p in range(Lh):
        for q in range(-p, p + 1):
            if q != 0:
                h[p * p + p + q] = 0
    g = O.forward_coeff(f, h, Lf, Lh, _all_pairs(Lf + Lh - 2), (9, 5, 6))
    assert np.max(np.abs(g - g[..., :1])) < 1e-14


def test_real_signal_and_window_conjugate_symmetry():
    """Real f and h: g(rho; l, -m) = (-1)^m conj g(rho; l, m) (Sec. IV-B)."""
    Lf, Lh = 8, 4
    f = synth.signal_cn_real(Lf, 9)
    h = synth.signal_cn_real(Lh, 10)
    pairs = _all_pairs(Lf + Lh - 2)
    g = O.forward_coeff(f, h, Lf, Lh, pairs, (7, 4, 5))
    idx = {pr: i for i, pr in enumerate(pairs)}
    for (l, m), i in idx.items():
        j = idx[(l, -m)]
        assert np.max(np.abs(g[j] - (-1) ** (m % 2) * np.conj(g[i]))) < 1e-14


def test_vanishes_above_Lf_plus_Lh():
    """g = 0 for l > L_f + L_h (inclusive), i.e. l >= Lf + Lh - 1 here
    (remark after Eq. harmonic_formulation)."""
    Lf, Lh = 6, 4
    f = synth.signal_cn_real(Lf, 1)
    h = synth.window_cn(Lh, 2)
    g_top = O.forward_coeff(f, h, Lf, Lh, [(Lf + Lh - 2, 1)], (5, 3, 5))
    g_out = O.forward_coeff(f, h, Lf, Lh, [(Lf + Lh - 1, 1), (Lf + Lh + 3, -2)], (5, 3, 5))
    assert np.max(np.abs(g_top)) > 1e-3
    assert np.max(np.abs(g_out)) < 1e-15


def test_D_projection_identity():
    """int g conj(D^p_{q q'}) d rho = 8 pi^2/(2p+1) k_lm(p,q) h_p^{q'}
    (remark after Eq. inversion_2, with Eq. WignerD_ortho).  The grid rule is
    exact here because the product has degree <= 2 Lh - 2 in each angle."""
    Lf, Lh = 7, 4
    f = synth.signal_cn_real(Lf, 13)
    h = synth.window_cn(Lh, 14)
    grid = (2 * Lh - 1, 2 * Lh - 1, 2 * Lh - 1)
    pairs = [(3, 1), (6, -4), (9, 2)]
    g = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    a, b, c = O.grid_angles(*grid)
    d = S.wigner_d_table(Lh, b)
    ms = O.ModulatedSHT(f, Lf, Lh, 9)
    o = Lh - 1
    for i, (l, m) in enumerate(pairs):
        k = ms.coeffs(l, m)
        for p in range(Lh):
            for q in range(-p, p + 1):
                for qp in range(-p, p + 1):
                    D = (np.exp(-1j * q * a)[:, None, None] * d[p, q + o, qp + o][None, :, None]
                         * np.exp(-1j * qp * c)[None, None, :])
                    lhs = O.so3_integral(g[i] * np.conj(D), grid)
                    rhs = 8 * pi ** 2 / (2 * p + 1) * k[p, q + o] * h[p * p + p + qp]
                    assert abs(lhs - rhs) < 1e-13, (l, m, p, q, qp)


def test_parseval_over_all_degrees():
    """sum_{l,m} |g(rho; l, m)|^2 = int |f (D_rho h)|^2 ds: the g(rho; .) are
    the coefficients of f D_rho h (Definition 1)."""
    Lf, Lh = 6, 3
    f = synth.signal_cn_real(Lf, 21)
    h = synth.window_cn(Lh, 22)
    pairs = _all_pairs(Lf + Lh - 2)
    grid = (4, 3, 3)
    g = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    th, ph, w = O.sphere_rule(2 * (Lf + Lh - 2))
    pts = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
    fx = O.eval_signal(f, Lf, th, ph)
    a, b, c = O.grid_angles(*grid)
    for i, j, k in [(0, 0, 0), (3, 2, 1), (1, 1, 2)]:
        y = O.rotation_matrix(a[i], b[j], c[k]).T @ pts
        hx = O.eval_signal(h, Lh, np.arccos(np.clip(y[2], -1, 1)), np.arctan2(y[1], y[0]))
        rhs = np.sum(w * np.abs(fx * hx) ** 2)
        lhs = np.sum(np.abs(g[:, i, j, k]) ** 2)
        assert abs(lhs - rhs) / rhs < 1e-13


# ------------------------------------------------------ inverse

def test_beta_weights_integrate_legendre():
    sp = pytest.importorskip("scipy.special")
    for Nb in [1, 2, 5, 16, 64]:
        q = O.beta_weights(Nb)
        b = 2 * pi * np.arange(Nb) / (2 * Nb - 1)
        for p in range(Nb):
            val = np.sum(q * sp.eval_legendre(p, np.cos(b)))
            assert abs(val - (2.0 if p == 0 else 0.0)) < 1e-13, (Nb, p)


def test_weights_equal_printed_formula():
    """For Na = Ng = Nb*2-1 = 2L+1 our (2pi/M)^2 q_b equals the printed
    q(beta)/(2L+1)^3 of Eq. sig_reconstruction_discrete, including the
    beta = 0 closed form 4 pi^2 (floor(L/2)+1/2)^{-1}."""
    assert "floor(L/2)" in GOLDEN["q_beta"]["beta_zero"]
    for L in [1, 2, 3, 7, 18, 31]:
        M = 2 * L + 1
        ours = (2 * pi / M) ** 2 * O.beta_weights(L + 1)
        b = 2 * pi * np.arange(L + 1) / M

        def w(m):
            if m == 1:
                return 1j * pi / 2
            if m == -1:
                return -1j * pi / 2
            if m % 2:
                return 0.0
            return 2.0 / (1.0 - m * m)
        printed = np.empty(L + 1)
        printed[0] = 4 * pi ** 2 / (floor(L / 2) + 0.5)
        for n in range(1, L + 1):
            printed[n] = (8 * pi ** 2 * sum(w(-m) * np.cos(m * b[n]) for m in range(-L, L + 1))).real
        assert np.max(np.abs(ours - printed / M ** 3)) < 1e-13, L


def test_inverse_recovers_signal():
    """Eq. inversion_1 / inversion_2 on the sampled distribution, including
    oversampled and minimal grids (Na, Ng, Nb >= Lh)."""
    Lf, Lh = 10, 4
    f = synth.signal_powerlaw(Lf, 31)
    h = synth.window_cn(Lh, 32)
    pairs = _all_pairs(Lf - 1)
    for grid in [(Lh, Lh, Lh), (2 * Lh - 1, Lh, 2 * Lh - 1), (19, 10, 7)]:
        g = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
        fr = O.inverse(g, h[0], grid)
        assert np.max(np.abs(fr - f)) < 1e-14 * max(1.0, np.abs(f).max()) * 10, grid


def test_inversion_constant_printed():
    """int_SO(3) g d rho = sqrt(16 pi^3) h00 f_lm (the constant of Eq. inversion_1)."""
    assert GOLDEN["inversion_constant"]["value"] == "sqrt(16*pi^3)"
    Lf, Lh = 5, 2
    f = synth.signal_cn_real(Lf, 41)
    h = synth.window_cn(Lh, 42)
    g = O.forward_coeff(f, h, Lf, Lh, _all_pairs(Lf - 1), (3, 2, 3))
    fhat = O.so3_integral(g, (3, 2, 3))
    assert np.max(np.abs(fhat - sqrt(16 * pi ** 3) * h[0] * f)) < 1e-13


def test_inverse_rejects_zero_dc():
    with pytest.raises(ValueError):
        O.inverse(np.zeros((1, 2, 2, 2)), 0.0, (2, 2, 2))


def test_modulated_sht_accuracy_at_large_band_limit():
    """The quadrature route of Appendix A at l ~ 1800 with a short window
    band, against exact 3j symbols (Racah, rationals), where every T needs
    only a few exact symbols.  (With a 64-degree band at l ~ 2000 the route
    loses accuracy to cancellation; workload 5 uses GauntRecurrence.)"""
    Lf, Lh = 1900, 3
    f = synth.signal_powerlaw(Lf, 3002)
    ms = O.ModulatedSHT(f, Lf, Lh, 1899)
    for l, m in [(1800, 1200), (1899, -1899), (1850, 7)]:
        ke = O.modulated_coeffs_gaunt(f, Lf, Lh, l, m)
        kq = ms.coeffs(l, m)
        assert np.linalg.norm(kq - ke) / np.linalg.norm(ke) < 1e-9, (l, m)


def test_gaunt_recurrence_route_matches_exact():
    """k from the order-recursion 3j families equals k from Racah's exact
    3j symbols: every pair of a small case, and large-degree pairs."""
    Lf, Lh = 20, 6
    f = synth.signal_powerlaw(Lf, 3003)
    gr = O.GauntRecurrence(f, Lf, Lh)
    for l, m in [(0, 0), (3, -2), (12, 12), (19, 5), (24, -20)]:
        ke = O.modulated_coeffs_gaunt(f, Lf, Lh, l, m)
        assert np.abs(gr.coeffs(l, m) - ke).max() <= 1e-14 * max(np.abs(ke).max(), 1e-300)
    Lf, Lh = 1900, 3
    f = synth.signal_powerlaw(Lf, 3002)
    gr = O.GauntRecurrence(f, Lf, Lh)
    for l, m in [(1800, 1200), (1850, 7)]:
        ke = O.modulated_coeffs_gaunt(f, Lf, Lh, l, m)
        assert np.linalg.norm(gr.coeffs(l, m) - ke) / np.linalg.norm(ke) < 1e-13


def test_d_projection_equals_coupling_times_window():
    """d_projection against the identity of the remark after Eq. inversion_2,
    its right side from the Appendix A route to k (independent of the 3j
    symbols and of the projection's own code): the grid here is the smallest
    the oracle's docstring allows (every size Lh + p)."""
    Lf, Lh, p = 7, 4, 2
    f = synth.signal_cn_real(Lf, 23)
    h = synth.window_cn(Lh, 24)
    grid = (Lh + p, Lh + p, Lh + p)
    pairs = [(3, 1), (6, -4), (8, 2)]
    g = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    P = O.d_projection(g, grid, p)
    ms = O.ModulatedSHT(f, Lf, Lh, 8)
    for i, (l, m) in enumerate(pairs):
        k = ms.coeffs(l, m)
        for q in range(-p, p + 1):
            for qp in range(-p, p + 1):
                rhs = 8 * pi ** 2 / (2 * p + 1) * k[p, q + Lh - 1] * h[p * p + p + qp]
                assert abs(P[i, q + p, qp + p] - rhs) < 1e-13


def test_threej_orthogonality_over_the_window_order():
    """The 3j orthogonality the alternative inversion rests on, in exact
    rationals: for fixed (p, l) and M, sum over q of (L p l; M q -(M+q))
    (L' p l; M q -(M+q)) = delta_{L L'} / (2L+1)."""
    from fractions import Fraction
    p, l = 2, 5
    for M in (-3, 0, 2):
        for L in range(abs(l - p), l + p + 1):
            for L2 in range(abs(l - p), l + p + 1):
                if abs(M) > min(L, L2):
                    continue
                s = Fraction(0)
                for q in range(-p, p + 1):
                    if abs(M + q) > l:
                        continue
                    a = S.wigner3j_exact(L, p, l, M, q, -(M + q))
                    b = S.wigner3j_exact(L2, p, l, M, q, -(M + q))
                    s += Fraction(a) * Fraction(b)
                want = Fraction(1, 2 * L + 1) if L == L2 else Fraction(0)
                assert abs(float(s - want)) < 1e-15, (M, L, L2)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_inverse_alt_recovers_signal_without_dc(p):
    """The inverse of the remark after Eq. inversion_2 on a window with
    h_0^0 = 0 (where Eq. inversion_2 cannot be used): f recovered to rounding
    from the distribution at degrees L + p, for each degree p of the window,
    on the smallest grid its quadrature allows; one size smaller in beta the
    rule is no longer exact and the recovery fails."""
    Lf, Lh = 8, 4
    f = synth.signal_cn_real(Lf, 3)
    h = synth.window_cn(Lh, 4)
    h[0] = 0.0
    outs = synth.pairs_all(Lf)
    pairs = sorted({(L + p, M + q) for L, M in outs for q in range(-p, p + 1)})
    ft = f[outs[:, 0] ** 2 + outs[:, 0] + outs[:, 1]]
    grid = (Lh + p, Lh + p, Lh + p)
    g = O.forward_coeff(f, h, Lf, Lh, pairs, grid)
    fr = O.inverse_alt(g, h, Lh, pairs, grid, p, outs)
    assert np.max(np.abs(fr - ft)) < 1e-13 * np.max(np.abs(ft))
    with pytest.raises(ValueError):
        O.inverse(g[:1], h[0], grid)
    small = (Lh + p, Lh + p - 1, Lh + p)
    gs = O.forward_coeff(f, h, Lf, Lh, pairs, small)
    fs = O.inverse_alt(gs, h, Lh, pairs, small, p, outs)
    assert np.max(np.abs(fs - ft)) > 1e-6 * np.max(np.abs(ft))
