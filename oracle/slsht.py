"""The directional SLSHT in FP64 on the CPU: forward by two independent routes,
and the inverse.

Test infrastructure only (see the package docstring).

Band limits are EXCLUSIVE throughout (f_lm = 0 for l >= Lf, h_pq = 0 for
p >= Lh); the paper's inclusive band limit is this Lf - 1.  Coefficient
vectors are complex128 with the flat index l*l + l + m.

SO(3) grid (Sec. II-D, the tessellation E_L generalised to independent sizes):
  alpha_a = 2 pi a / Na,  beta_b = 2 pi b / (2 Nb - 1),  gamma_c = 2 pi c / Ng,
  0 <= a < Na, 0 <= b < Nb, 0 <= c < Ng.
For Na = Ng = 2L+1 and Nb = L+1 this is exactly E_L of the paper.
g is returned as [npairs, Na, Nb, Ng] (gamma fastest).

Rotation convention (Sec. II-B): (D_rho h)(x) = h(R^{-1} x) with
R = R_z(alpha) R_y(beta) R_z(gamma); on coefficients this is
(D_rho h)_l^m = sum_m' D^l_{m,m'}(rho) h_l^m' (Eq. rotation_non_symm).
"""

from math import pi, sqrt

import numpy as np

from . import special


# --------------------------------------------------------------------------
# grid
# --------------------------------------------------------------------------

def grid_angles(Na, Nb, Ng):
    """(alpha, beta, gamma) sample angles of the equiangular SO(3) grid."""
    a = 2.0 * pi * np.arange(Na) / Na
    b = 2.0 * pi * np.arange(Nb) / (2 * Nb - 1)
    c = 2.0 * pi * np.arange(Ng) / Ng
    return a, b, c


# --------------------------------------------------------------------------
# modulated-signal coefficients  (Appendix A)
# --------------------------------------------------------------------------

class ModulatedSHT:
    """k_{l m}(p, q) = conj((conj(f) Y_l^m)_p^q), p < Lh, |q| <= p, by the
    separation of variables of Appendix A (Eq. sht_sep_variable):
      (conj(f) Y_l^m)_p^q = N_l^m N_p^q int_0^pi P_l^m P_p^q I(theta, m-q) sin(theta) dtheta,
      I(theta, m-q) = int_0^{2pi} conj(f(theta, phi)) e^{i(m-q)phi} dphi.
    For a band-limited f given by its coefficients, I(theta, mu) is exactly
    2 pi conj(F_mu(cos theta)) with F_mu(x) = sum_l' f_{l' mu} Ptilde_l'^mu(x) (the
    mu-th azimuthal Fourier mode of f on the ring), and the theta integrand is
    a polynomial in x = cos(theta) of degree l' + p + l, so Gauss-Legendre
    quadrature with enough nodes is exact.  Hence
      k_{lm}(p, q) = 2 pi sum_i w_i F_{m-q}(x_i) Ptilde_p^q(x_i) Ptilde_l^m(x_i).
    Only degrees with |l-p| <= l' <= l+p can contribute (the triangle rule of
    the triple product), so F is summed over l' in [l-Lh+1, l+Lh-1]: the
    exact value is unchanged and the cancellation of the rest of f's energy is
    avoided.  Rounding of the oscillatory integrand still limits this route to
    about 1e-11 relative at l ~ 255 (pinned in the tests); at l ~ 2000 with a
    64-degree window band the degrees of F that T removes cancel badly (errors
    near 1e-2 were seen), so workload 5 uses GauntRecurrence.
    GauntCoefficients is the exact route used by default.
    """

    def __init__(self, f, Lf, Lh, lmax_out):
        self.f = np.asarray(f, dtype=np.complex128)
        assert self.f.shape == (Lf * Lf,)
        self.Lf, self.Lh = Lf, Lh
        deg = (Lf - 1) + (Lh - 1) + lmax_out
        self.x, self.w = special.gauss_legendre(deg // 2 + 1)
        # Ptilde_p^q at the nodes, [Lh, 2Lh-1, nx]
        self.Pw = np.zeros((Lh, 2 * Lh - 1, self.x.size))
        for q in range(-(Lh - 1), Lh):
            self.Pw[:, q + Lh - 1] = special.plm(Lh - 1, q, self.x)

    def coeffs(self, l, m):
        """k_{lm}(p, q) as an array [Lh, 2Lh-1] (entry [p, q+Lh-1], zero for |q|>p)."""
        Lf, Lh, f = self.Lf, self.Lh, self.f
        plm_l = special.plm(l, m, self.x)[l]
        lo, hi = max(0, l - (Lh - 1)), min(Lf - 1, l + Lh - 1)
        k = np.zeros((Lh, 2 * Lh - 1), dtype=np.complex128)
        for q in range(-(Lh - 1), Lh):
            mu = m - q
            if abs(mu) > Lf - 1 or hi < max(abs(mu), lo):
                continue
            ls = np.arange(max(abs(mu), lo), hi + 1)
            F = f[ls * ls + ls + mu] @ special.plm(hi, mu, self.x)[ls]     # F_mu, band only
            k[:, q + Lh - 1] = 2.0 * pi * (self.Pw[:, q + Lh - 1] @ (self.w * F * plm_l))
        return k


class GauntCoefficients:
    """k_{lm}(p, q) = sum_l' f_{l', m-q} T(l', m-q; p, q; l, m) (Eq. harmonic_formulation,
    the triple product T 'evaluated using Wigner-3j symbols', Sec. III-B), with
    every T from exact rational 3j symbols (special.gaunt_exact); only the
    final sum over at most Lh degrees l' is rounded.  The default source of
    k in forward_coeff."""

    def __init__(self, f, Lf, Lh, lmax_out=None):
        self.f = np.asarray(f, dtype=np.complex128)
        self.Lf, self.Lh = Lf, Lh

    def coeffs(self, l, m):
        return modulated_coeffs_gaunt(self.f, self.Lf, self.Lh, l, m)


class GauntRecurrence:
    """The same k_{lm}(p, q) as GauntCoefficients, with the 3j symbols of T
    from their order families (special.wigner3j_m_family: the J^2
    eigen-equation in the coupled basis, run in 100-digit decimal arithmetic)
    instead of Racah's rational sum, which costs milliseconds a symbol at the
    degrees of workload 5 (l ~ 2000).  Pinned against GauntCoefficients at
    small and at large degree."""

    def __init__(self, f, Lf, Lh, lmax_out=None):
        self.f = np.asarray(f, dtype=np.complex128)
        self.Lf, self.Lh = Lf, Lh

    def coeffs(self, l, m):
        Lf, Lh, f = self.Lf, self.Lh, self.f
        k = np.zeros((Lh, 2 * Lh - 1), dtype=np.complex128)
        for p in range(Lh):
            for lp in range(abs(l - p), min(Lf - 1, l + p) + 1):
                if (lp + p + l) % 2:
                    continue                          # (l' p l; 0 0 0) = 0
                lo0, fam0 = special.wigner3j_m_family(lp, p, l, 0)
                w0 = fam0[-lo0]                       # the order mu = 0
                if w0 == 0.0:
                    continue
                lo, fam = special.wigner3j_m_family(lp, p, l, m)
                t0 = sqrt((2 * lp + 1) * (2 * p + 1) * (2 * l + 1) / (4.0 * pi)) * w0
                for i, w1 in enumerate(fam):
                    mu = lo + i                       # order of l'; q = m - mu
                    k[p, m - mu + Lh - 1] += f[lp * lp + lp + mu] * (t0 * w1)
        return (-1) ** (m % 2) * k


def modulated_coeffs_gaunt(f, Lf, Lh, l, m):
    """k_{lm}(p,q) = sum_l' f_{l',m-q} T(l',m-q; p,q; l,m) with T from exact
    3j symbols (Eq. harmonic_formulation and the Gaunt form of T):
      T = (-1)^m sqrt((2l'+1)(2p+1)(2l+1)/(4 pi)) (l' p l; 0 0 0)(l' p l; m' q -m)."""
    k = np.zeros((Lh, 2 * Lh - 1), dtype=np.complex128)
    w0 = {}
    for p in range(Lh):
        for q in range(-p, p + 1):
            mu = m - q
            acc = 0.0j
            for lp in range(max(abs(mu), abs(l - p)), min(Lf - 1, l + p) + 1):
                if (lp + p + l) % 2:
                    continue                      # (l' p l; 0 0 0) = 0
                if (lp, p) not in w0:
                    w0[(lp, p)] = special.wigner3j_exact(lp, p, l, 0, 0, 0)
                w1 = special.wigner3j_exact(lp, p, l, mu, q, -m)
                if w1 == 0.0:
                    continue
                t = sqrt((2 * lp + 1) * (2 * p + 1) * (2 * l + 1) / (4.0 * pi)) * w0[(lp, p)] * w1
                acc += f[lp * lp + lp + mu] * t
            k[p, q + Lh - 1] = (-1) ** (m % 2) * acc
    return k


# --------------------------------------------------------------------------
# forward, coefficient domain (Eq. alternative_harmonic_formulation_wigner)
# --------------------------------------------------------------------------

def h_table(h, Lh):
    """h_p^{q'} as [Lh, 2Lh-1] (entry [p, q'+Lh-1])."""
    out = np.zeros((Lh, 2 * Lh - 1), dtype=np.complex128)
    for p in range(Lh):
        for q in range(-p, p + 1):
            out[p, q + Lh - 1] = h[p * p + p + q]
    return out


def forward_coeff(f, h, Lf, Lh, pairs, grid, beta_rows=None, msht=None, dtab=None,
                  kroute="exact"):
    """g(rho; l, m) on the grid via the convolution form
      g = sum_p sum_q sum_q' k_{lm}(p,q) h_p^{q'} d^p_{q,q'}(beta) e^{-i q' gamma} e^{-i q alpha}
    (Eq. alternative_harmonic_formulation and ..._wigner, with
    D^p_{q,q'} from Eq. Dlm), k from exact 3j symbols (GauntCoefficients,
    kroute="exact"), from order-recursion 3j families (GauntRecurrence,
    kroute="recurrence", for large degrees) or from the Appendix A quadrature
    (ModulatedSHT, kroute="quadrature"), d^p from the degree recurrence
    (special.wigner_d_table).  The triple sum is done as three library
    contractions (p, then q', then q); nothing else is reordered.

    pairs: iterable of (l, m).  grid: (Na, Nb, Ng).  beta_rows: optional
    subset of beta indices (returns only those rows).
    Returns complex128 [npairs, Na, nrows, Ng].
    """
    Na, Nb, Ng = grid
    pairs = [tuple(int(v) for v in pr) for pr in pairs]
    a, b, c = grid_angles(Na, Nb, Ng)
    if beta_rows is not None:
        b = b[np.asarray(beta_rows)]
    qs = np.arange(-(Lh - 1), Lh)
    Ea = np.exp(-1j * np.outer(qs, a))            # [K, Na]
    Eg = np.exp(-1j * np.outer(qs, c))            # [K, Ng]
    if dtab is None:
        dtab = special.wigner_d_table(Lh, b)      # [Lh, K, K, nb]
    ht = h_table(h, Lh)
    if msht is None:
        lmax = max(l for l, _ in pairs)
        msht = {"exact": GauntCoefficients, "quadrature": ModulatedSHT,
                "recurrence": GauntRecurrence}[kroute](f, Lf, Lh, lmax)
    K = 2 * Lh - 1
    nb = b.size
    out = np.zeros((len(pairs), Na, nb, Ng), dtype=np.complex128)
    for i, (l, m) in enumerate(pairs):
        k = msht.coeffs(l, m)                                   # [Lh, K]
        kh = k[:, :, None] * ht[:, None, :]                      # [Lh, K(q), K(q')]
        G = np.einsum('pij,pijn->ijn', kh, dtab)                 # sum over p
        X = np.matmul(G.transpose(0, 2, 1), Eg)                  # sum over q': [q, n, c]
        out[i] = (Ea.T @ X.reshape(K, nb * Ng)).reshape(Na, nb, Ng)   # sum over q
    return out


# --------------------------------------------------------------------------
# forward by direct quadrature of the definition (Eq. stft_spatial)
# --------------------------------------------------------------------------

def rotation_matrix(alpha, beta, gamma):
    """R = R_z(alpha) R_y(beta) R_z(gamma) (zyz, Sec. II-B), active, right-handed."""
    def rz(t):
        ct, st = np.cos(t), np.sin(t)
        return np.array([[ct, -st, 0.0], [st, ct, 0.0], [0.0, 0.0, 1.0]])

    def ry(t):
        ct, st = np.cos(t), np.sin(t)
        return np.array([[ct, 0.0, st], [0.0, 1.0, 0.0], [-st, 0.0, ct]])
    return rz(alpha) @ ry(beta) @ rz(gamma)


def sphere_rule(deg):
    """Exact quadrature for band-limited integrands of total degree <= deg:
    Gauss-Legendre in cos(theta) x uniform phi.  Returns theta, phi, weights."""
    x, w = special.gauss_legendre(deg // 2 + 1)
    nphi = deg + 1
    phi = 2.0 * pi * np.arange(nphi) / nphi
    th = np.arccos(x)
    T, P = np.meshgrid(th, phi, indexing='ij')
    W = np.outer(w, np.full(nphi, 2.0 * pi / nphi))
    return T.ravel(), P.ravel(), W.ravel()


def eval_signal(coef, L, theta, phi):
    """sum_{l<L} coef_lm Y_l^m(theta, phi)  (Eq. f_expansion)."""
    return coef @ special.sph_harm_all(L, theta, phi)


def forward_quadrature(f, h, Lf, Lh, pairs, grid, rot_index=None):
    """g(rho; l, m) = int f(x) (D_rho h)(x) conj(Y_l^m(x)) ds  (Eq. stft_spatial).

    The integrand is band-limited (degree <= (Lf-1)+(Lh-1)+l), so the sphere
    rule of sphere_rule is exact.  (D_rho h)(x) is evaluated geometrically as
    h(R^T x), by summing h's expansion at the rotated points: no Wigner
    function appears anywhere on this route.
    rot_index: optional list of (a, b, c) grid indices; default all.
    Returns [npairs, Na, Nb, Ng] (or [npairs, len(rot_index)]).
    """
    Na, Nb, Ng = grid
    pairs = [tuple(int(v) for v in pr) for pr in pairs]
    lmax = max(l for l, _ in pairs)
    deg = (Lf - 1) + (Lh - 1) + lmax
    th, ph, W = sphere_rule(deg)
    pts = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])  # [3, n]
    fx = eval_signal(np.asarray(f, np.complex128), Lf, th, ph)
    Yall = special.sph_harm_all(lmax + 1, th, ph)
    Yc = np.conj(Yall[[l * l + l + m for l, m in pairs]])                  # [npairs, n]
    A = Yc * (W * fx)[None, :]                                             # [npairs, n]
    a, b, c = grid_angles(Na, Nb, Ng)
    if rot_index is None:
        rot_index = [(i, j, k) for i in range(Na) for j in range(Nb) for k in range(Ng)]
    hc = np.asarray(h, np.complex128)
    out = np.zeros((len(pairs), len(rot_index)), dtype=np.complex128)
    for r, (i, j, k) in enumerate(rot_index):
        R = rotation_matrix(a[i], b[j], c[k])
        y = R.T @ pts
        tr = np.arccos(np.clip(y[2], -1.0, 1.0))
        pr = np.arctan2(y[1], y[0])
        hrot = eval_signal(hc, Lh, tr, pr)                                  # [n]
        out[:, r] = A @ hrot
    if len(rot_index) == Na * Nb * Ng:
        return out.reshape(len(pairs), Na, Nb, Ng)
    return out


def rotate_coeffs(coef, L, alpha, beta, gamma):
    """(D_rho f)_l^m = sum_m' D^l_{m,m'}(rho) f_l^{m'}  (Eq. rotation_non_symm, Eq. Dlm)."""
    d = special.wigner_d_table(L, [beta])[..., 0]
    out = np.zeros_like(np.asarray(coef, np.complex128))
    for l in range(L):
        for m in range(-l, l + 1):
            acc = 0.0j
            for mp in range(-l, l + 1):
                D = np.exp(-1j * m * alpha) * d[l, m + L - 1, mp + L - 1] * np.exp(-1j * mp * gamma)
                acc += D * coef[l * l + l + mp]
            out[l * l + l + m] = acc
    return out


# --------------------------------------------------------------------------
# inverse (Eq. inversion_1, inversion_2, sig_reconstruction_discrete)
# --------------------------------------------------------------------------

def beta_weights(Nb):
    """Quadrature weights q_b with sum_b q_b F(beta_b) = int_0^pi F(beta) sin(beta) dbeta
    for every even trigonometric polynomial F of degree <= Nb - 1.

    From w(k) = int_0^pi e^{ik beta} sin(beta) dbeta (the w(m) printed after
    Eq. sig_reconstruction_discrete: +-i pi/2 at k = +-1, 0 for other odd k,
    2/(1-k^2) for even k) and the exact Fourier coefficients of F on the
    M = 2Nb-1 point circle: folding the samples b and M-b together gives
      q_0 = (1/M) sum_{|k|<Nb} W(k),   q_b = (2/M) sum_{|k|<Nb} W(k) cos(k beta_b),
    where W(k) = 2/(1-k^2) for even k and 0 otherwise (the k = +-1 terms cancel
    in the cosine sum).  With Na = Ng = M the paper's printed weights
    q(beta)/(2L+1)^3 equal (2 pi/M)^2 q_b; the tests check this.
    """
    M = 2 * Nb - 1
    ks = np.arange(-(Nb - 1), Nb)
    W = np.zeros(ks.size)
    even = ks % 2 == 0
    W[even] = 2.0 / (1.0 - ks[even].astype(np.float64) ** 2)
    beta = 2.0 * pi * np.arange(Nb) / M
    q = (2.0 / M) * (np.cos(np.outer(beta, ks)) @ W)
    q[0] = W.sum() / M
    return q


def so3_integral(g, grid):
    """int_SO(3) g(rho) d rho on the grid, d rho = d alpha sin(beta) d beta d gamma.
    g: [..., Na, Nb, Ng].  Exact for g band-limited at Lh when Na, Ng, Nb >= Lh."""
    Na, Nb, Ng = grid
    q = beta_weights(Nb)
    return (2.0 * pi / Na) * (2.0 * pi / Ng) * np.einsum('...abc,b->...', g, q)


def inverse(g, h00, grid):
    """f_lm = fhat_lm / (sqrt(16 pi^3) h_0^0), fhat_lm = int g(rho; l, m) d rho
    (Eq. inversion_1, Eq. inversion_2).  g: [npairs, Na, Nb, Ng] -> [npairs]."""
    if h00 == 0:
        raise ValueError("h_0^0 must be non-zero for the inverse (Eq. inversion_2)")
    return so3_integral(g, grid) / (sqrt(16.0 * pi ** 3) * h00)


# --------------------------------------------------------------------------
# inverse without h_0^0 (the remark after Eq. inversion_2)
# --------------------------------------------------------------------------

def d_projection(g, grid, p):
    """P[i, q, q'] = int_SO(3) g(rho; pair i) conj(D^p_{q,q'}(rho)) d rho for
    |q|, |q'| <= p, by the same SO(3) quadrature as the inverse, with
    D^p_{q,q'} = e^{-i q alpha} d^p_{q,q'}(beta) e^{-i q' gamma} (Eq. Dlm).
    Exact when every grid size is at least Lh + p (the integrand is then
    band-limited within the rule's reach in every angle).
    g: [npairs, Na, Nb, Ng] -> [npairs, 2p+1, 2p+1] (index q + p, q' + p)."""
    Na, Nb, Ng = grid
    a, b, c = grid_angles(Na, Nb, Ng)
    qs = np.arange(-p, p + 1)
    Ea = np.exp(1j * np.outer(qs, a))             # conj(e^{-i q alpha})   [2p+1, Na]
    Eg = np.exp(1j * np.outer(qs, c))             # conj(e^{-i q' gamma})  [2p+1, Ng]
    d = special.wigner_d_table(p + 1, b)[p]       # d^p_{q,q'}(beta_b), [K, K, Nb] with K = 2p + 1
    wq = beta_weights(Nb)
    out = np.einsum('iabc,qa,qrb,rc,b->iqr', g, Ea, d, Eg, wq)
    return (2.0 * pi / Na) * (2.0 * pi / Ng) * out


def inverse_alt(g, h, Lh, pairs, grid, p, out_pairs):
    """f_{L,M} from g without the condition h_0^0 != 0, by the reconstruction of
    the remark after Eq. inversion_2, taken in its steps:
      1. project g on conj(D^p_{q,q'}) (d_projection): by the orthogonality of
         the Wigner D functions (Eq. WignerD_ortho) the projection of
         g(.; l, m) is 8 pi^2 / (2p+1) k_lm(p, q) h_p^{q'};
      2. decouple the window with its coefficients at degree p: summing
         conj(h_p^{q'}) times the projection over q' leaves
         8 pi^2 / (2p+1) E_p k_lm(p, q), E_p = sum_q' |h_p^q'|^2 the window's
         energy at degree p (non-zero: the condition that replaces h_0^0 != 0);
      3. decouple the signal with the orthogonality of the Wigner-3j symbols:
         with k_lm(p, q) = sum_l' f_{l', m-q} T(l', m-q; p, q; l, m) and T
         through 3j symbols (Sec. III-B),
           sum_q (L p l; M q -(M+q)) (l' p l; M q -(M+q)) = delta_{L l'} / (2L+1),
         so f_{L,M} = (2L+1) / c^2 sum_q T(L, M; p, q; l, M+q) k_{l, M+q}(p, q),
         c^2 = (2L+1)(2p+1)(2l+1)/(4 pi) (L p l; 0 0 0)^2, for any degree l with
         (L p l; 0 0 0) != 0.  Here l = L + p, which always qualifies.
    pairs: the (l, m) of g's rows; every (L + p, M + q), |q| <= p, of each
    requested (L, M) must be among them.  out_pairs: the (L, M) to recover.
    Returns complex128 [len(out_pairs)]."""
    pairs = [tuple(int(v) for v in pr) for pr in pairs]
    row = {pr: i for i, pr in enumerate(pairs)}
    hp = np.array([h[p * p + p + q] for q in range(-p, p + 1)])
    Ep = float(np.sum(np.abs(hp) ** 2))
    if Ep == 0.0:
        raise ValueError("the window has no energy at degree p")
    out = np.zeros(len(out_pairs), dtype=np.complex128)
    need = sorted({row[(L + p, M + q)] for L, M in out_pairs for q in range(-p, p + 1)})
    proj = d_projection(g[need], grid, p)                       # [n, 2p+1, 2p+1]
    khat = {need[i]: (2 * p + 1) / (8.0 * pi ** 2 * Ep) * (proj[i] @ np.conj(hp)) for i in range(len(need))}
    for o, (L, M) in enumerate(out_pairs):
        l = L + p
        c2 = (2 * L + 1) * (2 * p + 1) * (2 * l + 1) / (4.0 * pi) * special.wigner3j_exact(L, p, l, 0, 0, 0) ** 2
        acc = 0.0
        for q in range(-p, p + 1):
            acc += special.gaunt_exact(L, M, p, q, l, M + q) * khat[row[(l, M + q)]][q + p]
        out[o] = (2 * L + 1) / c2 * acc
    return out
