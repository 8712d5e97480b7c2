// The alpha stage of one column in double-float arithmetic (dd.cuh): the same
// two forms as alpha_dev.cuh -- the +-q paired direct sum and the split DFT
// a = Q s + t -- with every coefficient, table entry and partial sum a pair of
// floats, and the output assembled as a double with the column's power-of-two
// scale.  Coefficients sit in shared memory as float4 {re.h, im.h, re.l,
// im.l} at sx[row * ld]; tables are float4 {cos.h, sin.h, cos.l, sin.l}.
#pragma once

#include "alpha_dev.cuh"
#include "dd.cuh"

// A normalised double-float value.
struct ddv {
  float h, l;
};
__device__ __forceinline__ ddv ddv_of(const dd_acc& a) {
  ddv r;
  dd_acc_get(a, &r.h, &r.l);
  return r;
}
__device__ __forceinline__ ddv ddv_add(ddv a, ddv b) {
  float e;
  const float s = two_sum(a.h, b.h, &e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  ddv r;
  r.h = __fadd_rn(s, e);
  r.l = __fadd_rn(e, -__fadd_rn(r.h, -s));          // e - (h - s)
  return r;
}
__device__ __forceinline__ ddv ddv_neg(ddv a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ddv ddv_sub(ddv a, ddv b) { return ddv_add(a, ddv_neg(b)); }
__device__ __forceinline__ void dd_mac(dd_acc& acc, ddv a, ddv b) { dd_mac(acc, a.h, a.l, b.h, b.l); }
__device__ __forceinline__ void dd_add(dd_acc& acc, ddv b) { dd_add(acc, b.h, b.l); }

struct ddc {   // complex
  ddv re, im;
};
__device__ __forceinline__ ddc ddc_load_smem(const float4* p) {
  const float4 v = *p;
  return {{v.x, v.z}, {v.y, v.w}};
}
__device__ __forceinline__ ddc ddc_load_tab(const float4* p) {
  const float4 v = __ldg(p);
  return {{v.x, v.z}, {v.y, v.w}};
}
__device__ __forceinline__ float4 ddc_pack(ddc a) { return make_float4(a.re.h, a.im.h, a.re.l, a.im.l); }

// Output of one column: g at dst and, for a mirrored pair (real fields),
// sgn * conj(g) at mdst (nullable).
struct DdOut {
  double2* dst;
  double2* mdst;
  unsigned long long sgn;   // sign bit of (-1)^m: 0 or 1 << 63
  int sc;
  __device__ __forceinline__ void put(size_t off, ddv re, ddv im) const {
    const double r = dd_to_double(re.h, re.l, sc), i = dd_to_double(im.h, im.l, sc);
    dst[off] = make_double2(r, i);
    if (mdst != nullptr) {   // (-1)^m conj(g): sign flips on the bit patterns, no FP64 multiply
      const unsigned long long br = (unsigned long long)__double_as_longlong(r) ^ sgn;
      const unsigned long long bi = (unsigned long long)__double_as_longlong(i) ^ sgn ^ (1ull << 63);
      mdst[off] = make_double2(__longlong_as_double((long long)br), __longlong_as_double((long long)bi));
    }
  }
};

// Direct sum, +-q paired, rows a0 .. a0 + ALPHA_ABLK - 1 for a0 = a_first,
// a_first + a_step, ...; X_0 in row x0row, P_r in row p0 + r*ps, M_r in row
// m0 + r*ms_; csa[a*Lh + r] = (cos, sin)(2 pi r a / Na).
__device__ __forceinline__ void alpha_direct_column_dd(const float4* __restrict__ sx, int ld, int x0row, int p0,
                                                       int ps, int m0, int ms_, int Lh, int Na, int J,
                                                       const float4* __restrict__ csa, const DdOut& out,
                                                       int a_first, int a_step) {
  const ddc x0 = ddc_load_smem(sx + x0row * ld);
  for (int a0 = a_first; a0 < Na; a0 += a_step) {
    dd_acc re[ALPHA_ABLK], im[ALPHA_ABLK];
#pragma unroll
    for (int u = 0; u < ALPHA_ABLK; ++u) {
      re[u] = dd_acc_of(x0.re.h, x0.re.l);
      im[u] = dd_acc_of(x0.im.h, x0.im.l);
    }
    for (int r = 1; r < Lh; ++r) {
      const ddc P = ddc_load_smem(sx + (p0 + r * ps) * ld);
      const ddc M = ddc_load_smem(sx + (m0 + r * ms_) * ld);
#pragma unroll
      for (int u = 0; u < ALPHA_ABLK; ++u) {
        const int a = min(a0 + u, Na - 1);
        const ddc cs = ddc_load_tab(csa + (size_t)a * Lh + r);   // re: cos, im: sin
        dd_mac(re[u], P.re, cs.re);
        dd_mac(re[u], M.im, cs.im);
        dd_mac(im[u], P.im, cs.re);
        dd_mac(im[u], ddv_neg(M.re), cs.im);
      }
    }
#pragma unroll
    for (int u = 0; u < ALPHA_ABLK; ++u)
      if (a0 + u < Na) out.put((size_t)(a0 + u) * J, ddv_of(re[u]), ddv_of(im[u]));
  }
}

// Split DFT (see alpha_split_column): X_q in row q + Lh - 1; tw[t * (2Lh-1) +
// q + Lh - 1] = (cos, sin)(2 pi q t / Na); cpr / spr[r * (H+1) + s] = cos / sin
// (2 pi r s / P) as double-floats.  Residues t = t_first, t_first + t_step, ...
template <int P>
__device__ __forceinline__ void alpha_split_column_dd(const float4* __restrict__ sx, int ld, int Lh, int Na, int J,
                                                      const float4* __restrict__ tw, const ddv* cpr, const ddv* spr,
                                                      const DdOut& out, int t_first, int t_step) {
  constexpr int H = (P - 1) / 2;
  const int K = 2 * Lh - 1, Q = Na / P;
  int qfirst[P];
#pragma unroll
  for (int r = 0; r < P; ++r) {
    int q = -(Lh - 1);
    q += (((r - q) % P) + P) % P;
    qfirst[r] = q;
  }
  for (int tt = t_first; tt < Q; tt += t_step) {
    const float4* w = tw + (size_t)tt * K + (Lh - 1);
    ddv zr[P], zi[P];
#pragma unroll
    for (int r = 0; r < P; ++r) {
      dd_acc ar = dd_acc_zero(), ai = dd_acc_zero();
      for (int q = qfirst[r]; q < Lh; q += P) {      // X_q (cos - i sin)
        const ddc x = ddc_load_smem(sx + (q + Lh - 1) * ld);
        const ddc e = ddc_load_tab(w + q);
        dd_mac(ar, x.re, e.re);
        dd_mac(ar, x.im, e.im);
        dd_mac(ai, x.im, e.re);
        dd_mac(ai, ddv_neg(x.re), e.im);
      }
      zr[r] = ddv_of(ar);
      zi[r] = ddv_of(ai);
    }
    ddv sr[H + 1], si[H + 1], dr[H + 1], di[H + 1];
    dd_acc y0r = dd_acc_of(zr[0].h, zr[0].l), y0i = dd_acc_of(zi[0].h, zi[0].l);
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      sr[r] = ddv_add(zr[r], zr[P - r]); si[r] = ddv_add(zi[r], zi[P - r]);
      dr[r] = ddv_sub(zr[r], zr[P - r]); di[r] = ddv_sub(zi[r], zi[P - r]);
      dd_add(y0r, sr[r]);
      dd_add(y0i, si[r]);
    }
    out.put((size_t)tt * J, ddv_of(y0r), ddv_of(y0i));
#pragma unroll
    for (int s = 1; s <= H; ++s) {
      dd_acc Ar = dd_acc_of(zr[0].h, zr[0].l), Ai = dd_acc_of(zi[0].h, zi[0].l);
      dd_acc Br = dd_acc_zero(), Bi = dd_acc_zero();
#pragma unroll
      for (int r = 1; r <= H; ++r) {
        const ddv c = cpr[r * (H + 1) + s], sn = spr[r * (H + 1) + s];
        dd_mac(Ar, sr[r], c); dd_mac(Ai, si[r], c);
        dd_mac(Br, dr[r], sn); dd_mac(Bi, di[r], sn);
      }
      const ddv ar = ddv_of(Ar), ai = ddv_of(Ai), br = ddv_of(Br), bi = ddv_of(Bi);
      // y_s = A - iB, y_{P-s} = A + iB
      out.put((size_t)(Q * s + tt) * J, ddv_add(ar, bi), ddv_sub(ai, br));
      out.put((size_t)(Q * (P - s) + tt) * J, ddv_sub(ar, bi), ddv_add(ai, br));
    }
  }
}
