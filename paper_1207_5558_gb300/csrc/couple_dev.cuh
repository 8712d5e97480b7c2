// Gather-sum of the Gaunt coupling from a kept coefficient table, shared by
// the per-call kernel (k_couple_apply) and the batch kernel (k_batch_couple).
#pragma once

#include "common.cuh"

// k_lm(p, q) = sum_i T_i f_{l'_i, m - q} (Sec. III-B) for item t = p*p + p + q
// of one pair: coef = the pair's table rows ([i][t], Lh rows of Lh*Lh), md =
// (first l', count) of item t, the l' advancing by 2 (parity rule).
__device__ __forceinline__ double2 couple_apply_one(const double2* __restrict__ f, int Lh, int m,
                                                    const double* __restrict__ coef, int2 md, int t) {
  const int n2 = Lh * Lh;
  int p = (int)sqrtf((float)t);
  while (p * p > t) --p;
  while ((p + 1) * (p + 1) <= t) ++p;
  const int q = t - p * p - p;
  const int mu = m - q;
  double2 acc = make_double2(0.0, 0.0);
  const double* c = coef + t;
  for (int i = 0; i < md.y; ++i) {
    const int j1 = md.x + 2 * i;
    const double ci = c[(size_t)i * n2];
    const double2 fv = __ldg(f + j1 * j1 + j1 + mu);
    acc.x = fma(ci, fv.x, acc.x);
    acc.y = fma(ci, fv.y, acc.y);
  }
  return acc;
}
