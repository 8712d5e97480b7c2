// Gaunt coupling of the signal and the window (Sec. III-B, Sec. IV-B):
//   k_lm(p, q) = conj((conj(f) Y_l^m)_p^q) = sum_l' f_{l', m-q} T(l', m-q; p, q; l, m),
//   T(l',m';p,q;l,m) = (-1)^m sqrt((2l'+1)(2p+1)(2l+1)/(4 pi))
//                      (l' p l; 0 0 0) (l' p l; m' q -m),
// with both Wigner-3j families generated by recurrences in l' (= j1) in FP64.
#include "common.cuh"

// 3j symbols (j1 j2 j3; m1 m2 m3), m1 = -m2 - m3, for every j1 in
// [j1min, j1max] = [max(|j2-j3|, |m1|), j2 + j3], into f[0 .. n-1].
// Schulten-Gordon recurrence in j1:
//   j1 A(j1+1) f(j1+1) + B(j1) f(j1) + (j1+1) A(j1) f(j1-1) = 0,
//   A(j1) = sqrt((j1^2 - (j2-j3)^2) ((j2+j3+1)^2 - j1^2) (j1^2 - m1^2)),
//   B(j1) = -(2j1+1) (j2(j2+1) m1 - j3(j3+1) m1 - j1(j1+1)(m3-m2)).
// Stability: run forward from j1min while |f| grows, backward from j1max while
// |f| grows, continue forward through the oscillatory middle, match the two
// pieces by least squares on two overlapping points, normalise with
// sum_j1 (2 j1 + 1) f^2 = 1 and fix the sign by sgn f(j1max) = (-1)^{j2-j3-m1}.
// When j1min = 0 (j2 = j3, m1 = 0) the recurrence is silent at j1 = 0 and the
// first step uses f(1)/f(0) = m2 / sqrt(j2 (j2 + 1)).
// Returns n (0 if the chain is empty).
__device__ int threej_chain(int j2, int j3, int m2, int m3, double* f, double* bwd, int* j1min_out) {
  const int m1 = -m2 - m3;
  const int j1min = max(abs(j2 - j3), abs(m1));
  const int j1max = j2 + j3;
  *j1min_out = j1min;
  const int n = j1max - j1min + 1;
  if (n <= 0 || abs(m2) > j2 || abs(m3) > j3) return 0;
  const double dj = (double)(j2 - j3), sj = (double)(j2 + j3 + 1), dm1 = (double)m1;
  const double bj = (double)j2 * (j2 + 1.0) * dm1 - (double)j3 * (j3 + 1.0) * dm1;
  const double dm = (double)(m3 - m2);
  auto A = [&](int j1) -> double {
    const double x = (double)j1;
    const double v = (x * x - dj * dj) * (sj * sj - x * x) * (x * x - dm1 * dm1);
    return v > 0.0 ? sqrt(v) : 0.0;
  };
  auto B = [&](int j1) -> double {
    const double x = (double)j1;
    return -(2.0 * x + 1.0) * (bj - x * (x + 1.0) * dm);
  };
  if (n == 1) {
    f[0] = 1.0;
  } else {
    f[0] = 1.0;
    int kf = 0;
    auto fstep = [&](int i) {
      const int j1 = j1min + i;
      if (j1 == 0) {
        f[1] = (double)m2 / sqrt((double)j2 * (j2 + 1.0));
      } else {
        const double prev = i > 0 ? f[i - 1] : 0.0;
        f[i + 1] = -(B(j1) * f[i] + (j1 + 1.0) * A(j1) * prev) / (j1 * A(j1 + 1));
      }
    };
    while (kf + 1 < n) {
      fstep(kf);
      ++kf;
      if (fabs(f[kf]) < fabs(f[kf - 1])) break;
    }
    bwd[n - 1] = 1.0;
    int kb = n - 1;
    while (kb - 1 >= 0) {
      const int j1 = j1min + kb;
      const double nxt = (kb + 1 < n) ? bwd[kb + 1] : 0.0;
      bwd[kb - 1] = -(B(j1) * bwd[kb] + j1 * A(j1 + 1) * nxt) / ((j1 + 1.0) * A(j1));
      --kb;
      if (fabs(bwd[kb]) < fabs(bwd[kb + 1])) break;
    }
    const int lo = (kb + 1 < n) ? kb : n - 2;
    while (kf < lo + 1) {
      fstep(kf);
      ++kf;
    }
    const double num = f[lo] * bwd[lo] + f[lo + 1] * bwd[lo + 1];
    const double den = f[lo] * f[lo] + f[lo + 1] * f[lo + 1];
    const double s = num / den;
    for (int i = 0; i <= lo; ++i) f[i] *= s;
    for (int i = lo + 1; i < n; ++i) f[i] = bwd[i];
  }
  double norm = 0.0;
  for (int i = 0; i < n; ++i) norm += (2.0 * (j1min + i) + 1.0) * f[i] * f[i];
  double scale = 1.0 / sqrt(norm);
  const double want = ((j2 - j3 - m1) & 1) ? -1.0 : 1.0;
  if (f[n - 1] * want < 0.0) scale = -scale;
  for (int i = 0; i < n; ++i) f[i] *= scale;
  return n;
}

// One CTA per pair; item t = p*p + p + q (the window's flat index) computes
// k_lm(p, q).  The (l' p l; 0 0 0) family obeys the two-term relation
//   f(j1+1) = -sqrt((j1^2-d^2)(S^2-j1^2) / (((j1+1)^2-d^2)(S^2-(j1+1)^2))) f(j1-1),
// d = p - l, S = p + l + 1, non-zero for even j1 + p + l; it is walked twice
// (norm and sign first, values second) so no array is needed for it.
__global__ void __launch_bounds__(256) k_couple(const double2* __restrict__ f, int Lf, int Lh,
                                                const int2* __restrict__ lm, double2* __restrict__ kc) {
  const int pair = blockIdx.x;
  const int l = lm[pair].x, m = lm[pair].y;
  const int nitems = Lh * Lh;
  double fm[SLSHT_CHAIN_MAX], bwd[SLSHT_CHAIN_MAX];
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    int p = (int)sqrt((double)t);
    while (p * p > t) --p;
    while ((p + 1) * (p + 1) <= t) ++p;
    const int q = t - p * p - p;
    double2 acc = make_double2(0.0, 0.0);
    int j1min_m;
    const int nm = threej_chain(p, l, q, -m, fm, bwd, &j1min_m);
    if (nm > 0) {
      // (l' p l; 000): first pass for the normalisation and the sign at l' = p + l
      const int j0 = abs(p - l), j1top = p + l;
      const double dd = (double)(p - l), SS = (double)(p + l + 1);
      auto ratio = [&](int j1) -> double {   // f(j1+1)/f(j1-1)
        const double x = (double)j1, y = x + 1.0;
        return -sqrt(((x * x - dd * dd) * (SS * SS - x * x)) / ((y * y - dd * dd) * (SS * SS - y * y)));
      };
      double w = 1.0, norm = (2.0 * j0 + 1.0);
      for (int j1 = j0 + 2; j1 <= j1top; j1 += 2) {
        w *= ratio(j1 - 1);
        norm += (2.0 * j1 + 1.0) * w * w;
      }
      double s0 = 1.0 / sqrt(norm);
      const double want = ((p - l) & 1) ? -1.0 : 1.0;
      if (w * want < 0.0) s0 = -s0;
      // second pass: accumulate over l' < Lf with l' + p + l even and in the m chain
      const int mu = m - q;
      const int jend = min(j1top, Lf - 1);
      w = s0;
      for (int j1 = j0; j1 <= jend; j1 += 2) {
        if (j1 > j0) w *= ratio(j1 - 1);
        if (j1 >= j1min_m) {
          const double c = sqrt(2.0 * j1 + 1.0) * w * fm[j1 - j1min_m];
          const double2 fv = f[j1 * j1 + j1 + mu];
          acc.x = fma(c, fv.x, acc.x);
          acc.y = fma(c, fv.y, acc.y);
        }
      }
      const double pre = ((m & 1) ? -1.0 : 1.0) *
                         sqrt((2.0 * p + 1.0) * (2.0 * l + 1.0) / (4.0 * 3.14159265358979323846));
      acc.x *= pre;
      acc.y *= pre;
    }
    kc[(size_t)pair * nitems + t] = acc;
  }
}

cudaError_t launch_couple(const double2* f, int Lf, int Lh, const int2* lm, int npairs,
                          double2* kc, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  const int threads = Lh * Lh < 256 ? ((Lh * Lh + 31) / 32) * 32 : 256;
  k_couple<<<npairs, threads, 0, st>>>(f, Lf, Lh, lm, kc);
  return cudaGetLastError();
}
