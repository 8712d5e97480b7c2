// Per-column bodies of the CUDA-core alpha stage, shared by the per-call
// kernels (k_alpha_cc, k_alpha_split) and the persistent batch kernel.
//
// Both evaluate g(alpha_a, j) = sum_{|q| < Lh} X_q(j) e^{-i q alpha_a},
// alpha_a = 2 pi a / Na, for one column j whose coefficients sit in shared
// memory at sx[row * ld] (one column of a [row][ld] tile).
#pragma once

#include "common.cuh"

#define ALPHA_ABLK 4   // alpha rows per pass of the direct sum

// Direct sum with +-q paired:
//   g = X_0 + sum_{r=1}^{Lh-1} ( P_r cos(r alpha) - i M_r sin(r alpha) ),
//   P_r = X_r + X_-r, M_r = X_r - X_-r,
// X_0 in row x0row, P_r in row p0 + r*ps, M_r in row m0 + r*ms_; csa[a*Lh + r] =
// (cos, sin)(2 pi r a / Na).  Rows a0, a0+1, .., a0+ALPHA_ABLK-1 for a0 =
// a_first, a_first + a_step, ...  A coefficient load feeds 4*ALPHA_ABLK fused
// multiply-adds.  mdst (nullable): also stores sgn * conj(g) there.
template <typename T>
__device__ __forceinline__ void alpha_direct_column(const typename vec2<T>::t* __restrict__ sx, int ld, int x0row,
                                                    int p0, int ps, int m0, int ms_, int Lh, int Na, int J,
                                                    const typename vec2<T>::t* __restrict__ csa,
                                                    typename vec2<T>::t* __restrict__ dst,
                                                    typename vec2<T>::t* __restrict__ mdst, T sgn, int a_first,
                                                    int a_step) {
  typedef typename vec2<T>::t T2;
  const T2 x0 = sx[x0row * ld];
  for (int a0 = a_first; a0 < Na; a0 += a_step) {
    T re[ALPHA_ABLK], im[ALPHA_ABLK];
#pragma unroll
    for (int u = 0; u < ALPHA_ABLK; ++u) { re[u] = x0.x; im[u] = x0.y; }
    for (int r = 1; r < Lh; ++r) {
      const T2 P = sx[(p0 + r * ps) * ld];
      const T2 M = sx[(m0 + r * ms_) * ld];
#pragma unroll
      for (int u = 0; u < ALPHA_ABLK; ++u) {
        const int a = min(a0 + u, Na - 1);
        const T2 cs = csa[(size_t)a * Lh + r];
        re[u] = fma(P.x, cs.x, re[u]);
        re[u] = fma(M.y, cs.y, re[u]);
        im[u] = fma(P.y, cs.x, im[u]);
        im[u] = fma(-M.x, cs.y, im[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < ALPHA_ABLK; ++u)
      if (a0 + u < Na) dst[(size_t)(a0 + u) * J] = mk2(re[u], im[u]);
    if (mdst != nullptr) {
#pragma unroll
      for (int u = 0; u < ALPHA_ABLK; ++u)
        if (a0 + u < Na) mdst[(size_t)(a0 + u) * J] = mk2(sgn * re[u], -sgn * im[u]);
    }
  }
}

// cos / sin (2 pi r s / P) for r, s <= (P-1)/2, filled by threads 0 .. ((P+1)/2)^2 - 1.
template <typename T, int P>
__device__ __forceinline__ void alpha_split_consts(T (*cpr)[(P - 1) / 2 + 1], T (*spr)[(P - 1) / 2 + 1], int t) {
  constexpr int H = (P - 1) / 2;
  if (t < (H + 1) * (H + 1)) {
    const int r = t / (H + 1), s = t % (H + 1);
    double sv, cv;
    sincospi(2.0 * r * s / P, &sv, &cv);
    cpr[r][s] = (T)cv;
    spr[r][s] = (T)sv;
  }
}

// The same sum with the grid index split as a = Q s + t (Na = P Q, P a small
// odd factor): since e^{-i q alpha_a} = e^{-2 pi i q s / P} e^{-2 pi i q t / Na},
//   g[Q s + t] = sum_{r < P} e^{-2 pi i r s / P} Z_t(r),
//   Z_t(r)     = sum_{q = r (mod P)} X_q e^{-2 pi i q t / Na}.
// Per t the P sums Z_t (one complex multiply-add per order q) and a P-point
// DFT with its odd symmetry folded,
//   y_0 = sum_r Z_r,  y_s, y_{P-s} = Z_0 + A_s -/+ i B_s,
//   A_s = sum_{r=1}^{(P-1)/2} (Z_r + Z_{P-r}) cos(2 pi r s / P),
//   B_s = sum_{r=1}^{(P-1)/2} (Z_r - Z_{P-r}) sin(2 pi r s / P),
// so a sample costs about 4(2Lh-1)/P + 10 real multiply-adds instead of
// 4(Lh-1)+2 (Lh = 16, P = 7: 28 instead of 62).  X_q sits in row q + Lh - 1;
// tw[t * (2Lh-1) + q + Lh - 1] = (cos, sin)(2 pi q t / Na) for t < Q.
// Residues t = t_first, t_first + t_step, ... < Q.
template <typename T, int P>
__device__ __forceinline__ void alpha_split_column(const typename vec2<T>::t* __restrict__ sx, int ld, int Lh,
                                                   int Na, int J, const typename vec2<T>::t* __restrict__ tw,
                                                   const T (*cpr)[(P - 1) / 2 + 1],
                                                   const T (*spr)[(P - 1) / 2 + 1],
                                                   typename vec2<T>::t* __restrict__ dst,
                                                   typename vec2<T>::t* __restrict__ mdst, T sgn, int t_first,
                                                   int t_step) {
  typedef typename vec2<T>::t T2;
  constexpr int H = (P - 1) / 2;
  const int K = 2 * Lh - 1, Q = Na / P;
  // first order q >= -(Lh-1) of each residue class r (mod P)
  int qfirst[P];
#pragma unroll
  for (int r = 0; r < P; ++r) {
    int q = -(Lh - 1);
    q += (((r - q) % P) + P) % P;
    qfirst[r] = q;
  }
  const int nq = (K + P - 1) / P;          // most orders in one residue class
  for (int tt = t_first; tt < Q; tt += t_step) {
    const T2* w = tw + (size_t)tt * K + (Lh - 1);
    // the P residue classes advance together, one order of each per step:
    // 2P independent multiply-add chains
    T zr[P], zi[P];
#pragma unroll
    for (int r = 0; r < P; ++r) zr[r] = zi[r] = (T)0;
    for (int jj = 0; jj < nq; ++jj) {
#pragma unroll
      for (int r = 0; r < P; ++r) {
        const int q = qfirst[r] + jj * P;
        if (q < Lh) {                                  // X_q e^{-i theta} = X_q (cos - i sin)
          const T2 x = sx[(q + Lh - 1) * ld];
          const T2 e = __ldg(w + q);
          zr[r] = fma(x.x, e.x, zr[r]); zr[r] = fma(x.y, e.y, zr[r]);
          zi[r] = fma(x.y, e.x, zi[r]); zi[r] = fma(-x.x, e.y, zi[r]);
        }
      }
    }
    // folded pairs Z_r +- Z_{P-r}, once per t
    T sr[H + 1], si[H + 1], dr[H + 1], di[H + 1];
    T y0r = zr[0], y0i = zi[0];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      sr[r] = zr[r] + zr[P - r]; si[r] = zi[r] + zi[P - r];
      dr[r] = zr[r] - zr[P - r]; di[r] = zi[r] - zi[P - r];
      y0r += sr[r];
      y0i += si[r];
    }
    T outr[P], outi[P];
    outr[0] = y0r;
    outi[0] = y0i;
#pragma unroll
    for (int s = 1; s <= H; ++s) {
      T Ar = zr[0], Ai = zi[0], Br = 0, Bi = 0;
#pragma unroll
      for (int r = 1; r <= H; ++r) {
        const T c = cpr[r][s], sn = spr[r][s];
        Ar = fma(sr[r], c, Ar); Ai = fma(si[r], c, Ai);
        Br = fma(dr[r], sn, Br); Bi = fma(di[r], sn, Bi);
      }
      outr[s] = Ar + Bi;  outi[s] = Ai - Br;           // A - iB
      outr[P - s] = Ar - Bi;  outi[P - s] = Ai + Br;   // A + iB
    }
#pragma unroll
    for (int s = 0; s < P; ++s) dst[(size_t)(Q * s + tt) * J] = mk2(outr[s], outi[s]);
    if (mdst != nullptr) {
#pragma unroll
      for (int s = 0; s < P; ++s) mdst[(size_t)(Q * s + tt) * J] = mk2(sgn * outr[s], -sgn * outi[s]);
    }
  }
}
