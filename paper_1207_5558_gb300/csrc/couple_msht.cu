// Coupling by the spherical harmonic transform of the modulated signal
// (Appendix A, Eq. sht_sep_variable), the paper's own route to k:
//   k_lm(p, q) = conj((conj(f) Y_l^m)_p^q)
//             = 2 pi sum_i w_i F_{m-q}(x_i) Ptilde_p^q(x_i) Ptilde_l^m(x_i),
// where F_mu(x) = sum_l' f_{l' mu} Ptilde_l'^mu(x) is the mu-th azimuthal mode
// of f on the ring at colatitude arccos(x) (what the phi-FFT of f sampled on
// the sphere gives), and x_i, w_i is a Gauss-Legendre rule exact for the
// polynomial integrand (degree <= (L_f-1) + (L_h-1) + l_max).  Only the
// degrees l' in [l - L_h + 1, l + L_h - 1] can contribute (triangle rule of
// the triple product), so F is summed over that band (the others would only
// add cancelling rounding).  Three kernels:
//   k_msht_plow   Ptilde_p^q(x_i) for every window degree, once per call;
//   k_msht_g      one CTA per pair, one thread per node: G[q][i] =
//                 w_i Ptilde_l^m(x_i) F_{m-q}(x_i) (FP64 recurrences in l);
//   k_msht_k      one thread per (pair, p, q): k = 2 pi sum_i G[q][i] Ptilde_p^q(x_i)
//                 in a fixed order (bitwise reproducible).
// Cost per pair ~ n (2L_h - 1)(l + L_h) recurrence steps: the route pays off
// against the 3j chains (~L_h^3) when the window band is wide and the signal
// band narrow; rounding in the band sums limits it to ~1e-11 relative near
// l = 255 (the same as the oracle's quadrature route).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

__device__ __forceinline__ double plm_start(int m, double s) {
  double p = 0.28209479177387814;           // 1 / sqrt(4 pi)
  for (int k = 1; k <= m; ++k) p *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * s;
  return p;
}

// Ptilde_p^q(x_i), p < Lh, |q| <= p: tab[(p*p+p+q) * n + i]
__global__ void k_msht_plow(const double* __restrict__ x, int n, int Lh, double* __restrict__ tab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = (int)blockIdx.y - (Lh - 1);
  if (i >= n) return;
  const int aq = q < 0 ? -q : q;
  const double xi = x[i], s = sqrt(fmax(0.0, 1.0 - xi * xi));
  const double sign = (q < 0 && (aq & 1)) ? -1.0 : 1.0;        // Ptilde^{-q} = (-1)^q Ptilde^q
  double p2 = 0.0, p1 = plm_start(aq, s);
  tab[(size_t)(aq * aq + aq + q) * n + i] = sign * p1;
  for (int p = aq + 1; p < Lh; ++p) {
    double v;
    if (p == aq + 1) {
      v = sqrt(2.0 * aq + 3.0) * xi * p1;
    } else {
      const double a = sqrt((4.0 * p * p - 1.0) / ((double)p * p - (double)aq * aq));
      const double b = sqrt((((double)p - 1) * (p - 1) - (double)aq * aq) / (4.0 * ((double)p - 1) * (p - 1) - 1.0));
      v = a * (xi * p1 - b * p2);
    }
    tab[(size_t)(p * p + p + q) * n + i] = sign * v;
    p2 = p1;
    p1 = v;
  }
}

// Ptilde_mu^mu(x) = C_mu (-s)^mu, s = sqrt(1 - x^2), from the table C.
__device__ __forceinline__ double plm_diag(int mu, double s, const double* __restrict__ C) {
  double r = 1.0, b = s;
  for (int e = mu; e > 0; e >>= 1) {
    if (e & 1) r *= b;
    b *= b;
  }
  return ((mu & 1) ? -r : r) * C[mu];
}

// G[pair][q + Lh - 1][i] (complex) = w_i Ptilde_l^m(x_i) F_{m-q}(x_i), the
// degree recurrences driven by the coefficient table ab[mu * Lt + l] =
// (sqrt((4l^2-1)/(l^2-mu^2)), sqrt(((l-1)^2-mu^2)/(4(l-1)^2-1))), l > mu.
__global__ void __launch_bounds__(128) k_msht_g(const double2* __restrict__ f, int Lf, int Lh,
                                                const int2* __restrict__ lm, const double* __restrict__ x,
                                                const double* __restrict__ w, int n, const double2* __restrict__ ab,
                                                const double* __restrict__ C, int Lt, double2* __restrict__ G) {
  const int pair = blockIdx.x;
  const int l = lm[pair].x, m = lm[pair].y;
  const int K = 2 * Lh - 1;
  const int lo = max(0, l - (Lh - 1)), hi = min(Lf - 1, l + Lh - 1);
  double2* Gp = G + (size_t)pair * K * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double xi = x[i], s = sqrt(fmax(0.0, 1.0 - xi * xi));
    // Ptilde_l^m(x_i)
    const int am = m < 0 ? -m : m;
    double plm;
    {
      const double2* abm = ab + (size_t)am * Lt;
      double p2 = 0.0, p1 = plm_diag(am, s, C);
      for (int ll = am + 1; ll <= l; ++ll) {
        const double2 c = abm[ll];
        const double v = c.x * (xi * p1 - c.y * p2);
        p2 = p1;
        p1 = v;
      }
      plm = (m < 0 && (am & 1)) ? -p1 : p1;
    }
    const double wp = w[i] * plm;
    for (int qi = 0; qi < K; ++qi) {
      const int q = qi - (Lh - 1);
      const int mu = m - q, amu = mu < 0 ? -mu : mu;
      double fr = 0.0, fi = 0.0;
      const int l0 = max(amu, lo);
      if (amu <= Lf - 1 && l0 <= hi) {
        const double sg = (mu < 0 && (amu & 1)) ? -1.0 : 1.0;
        const double2* abm = ab + (size_t)amu * Lt;
        double p2 = 0.0, p1 = sg * plm_diag(amu, s, C);
        if (l0 == amu) {
          const double2 fv = f[amu * amu + amu + mu];
          fr = p1 * fv.x;
          fi = p1 * fv.y;
        }
        for (int ll = amu + 1; ll <= hi; ++ll) {
          const double2 c = abm[ll];
          const double v = c.x * (xi * p1 - c.y * p2);
          p2 = p1;
          p1 = v;
          if (ll >= l0) {
            const double2 fv = f[ll * ll + ll + mu];
            fr = fma(v, fv.x, fr);
            fi = fma(v, fv.y, fi);
          }
        }
      }
      Gp[(size_t)qi * n + i] = make_double2(wp * fr, wp * fi);
    }
  }
}

// k[pair][p*p+p+q] = 2 pi sum_i G[pair][q][i] Ptilde_p^q(x_i)
__global__ void k_msht_k(const double2* __restrict__ G, const double* __restrict__ plow, int Lh, int n, int npairs,
                         double2* __restrict__ kc) {
  const int n2 = Lh * Lh, K = 2 * Lh - 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)npairs * n2) return;
  const int pair = (int)(idx / n2), t = (int)(idx % n2);
  int p = (int)sqrtf((float)t);
  while (p * p > t) --p;
  while ((p + 1) * (p + 1) <= t) ++p;
  const int q = t - p * p - p;
  const double2* g = G + ((size_t)pair * K + q + Lh - 1) * n;
  const double* pt = plow + (size_t)t * n;
  double re = 0.0, im = 0.0;
  for (int i = 0; i < n; ++i) {
    re = fma(g[i].x, pt[i], re);
    im = fma(g[i].y, pt[i], im);
  }
  const double tp = 6.283185307179586;
  kc[idx] = make_double2(tp * re, tp * im);
}

int msht_nodes(int Lf, int Lh, int lmax) { return ((Lf - 1) + (Lh - 1) + lmax) / 2 + 1; }

static int msht_lt(int Lf, int Lh, int lmax) { return std::max(std::max(Lf, lmax + 1), Lh) + 1; }

size_t msht_scratch_bytes(int Lf, int Lh, int lmax, int npairs) {
  const size_t n = (size_t)msht_nodes(Lf, Lh, lmax), Lt = (size_t)msht_lt(Lf, Lh, lmax);
  return sizeof(double) * 2 * n + sizeof(double) * n * Lh * Lh + sizeof(double2) * n * (2 * Lh - 1) * npairs +
         sizeof(double2) * Lt * Lt + sizeof(double) * Lt;
}

cudaError_t launch_couple_msht(const double2* f, int Lf, int Lh, const int2* lm, int npairs, int lmax, void* scratch,
                               double2* kc, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  const int n = msht_nodes(Lf, Lh, lmax), Lt = msht_lt(Lf, Lh, lmax);
  std::vector<double> x, w;
  gauss_legendre(n, x, w);
  // degree-recurrence coefficients and the diagonal constants
  //   C_mu = sqrt(1/(4 pi) prod_{k<=mu} (2k+1)/(2k)),  Ptilde_mu^mu = C_mu (-s)^mu
  std::vector<double2> ab((size_t)Lt * Lt, make_double2(0.0, 0.0));
  std::vector<double> C(Lt);
  C[0] = 0.28209479177387814;
  for (int k = 1; k < Lt; ++k) C[k] = C[k - 1] * std::sqrt((2.0 * k + 1.0) / (2.0 * k));
  for (int mu = 0; mu < Lt; ++mu)
    for (int l = mu + 1; l < Lt; ++l)
      ab[(size_t)mu * Lt + l] = make_double2(
          std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)mu * mu)),
          std::sqrt((((double)l - 1) * (l - 1) - (double)mu * mu) / (4.0 * ((double)l - 1) * (l - 1) - 1.0)));
  double* dx = (double*)scratch;
  double* dw = dx + n;
  double* plow = dw + n;
  double2* G = (double2*)(plow + (size_t)n * Lh * Lh);
  double2* dab = G + (size_t)n * (2 * Lh - 1) * npairs;
  double* dC = (double*)(dab + (size_t)Lt * Lt);
  cudaError_t e = cudaMemcpyAsync(dx, x.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dw, w.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dab, ab.data(), sizeof(double2) * ab.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dC, C.data(), sizeof(double) * C.size(), cudaMemcpyHostToDevice, st);
  // the host vectors must outlive the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  dim3 gp((n + 127) / 128, 2 * Lh - 1);
  k_msht_plow<<<gp, 128, 0, st>>>(dx, n, Lh, plow);
  k_msht_g<<<npairs, 128, 0, st>>>(f, Lf, Lh, lm, dx, dw, n, dab, dC, Lt, G);
  const long long tot = (long long)npairs * Lh * Lh;
  k_msht_k<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(G, plow, Lh, n, npairs, kc);
  return cudaGetLastError();
}
