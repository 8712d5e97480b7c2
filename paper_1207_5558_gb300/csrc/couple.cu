// Gaunt coupling of the signal and the window (Sec. III-B, Sec. IV-B):
//   k_lm(p, q) = conj((conj(f) Y_l^m)_p^q) = sum_l' f_{l', m-q} T(l', m-q; p, q; l, m),
//   T(l',m';p,q;l,m) = (-1)^m sqrt((2l'+1)(2p+1)(2l+1)/(4 pi))
//                      (l' p l; 0 0 0) (l' p l; m' q -m),
// with both Wigner-3j families generated by recurrences in l' (= j1) in FP64.
#include "batch.cuh"
#include "couple_dev.cuh"

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
// A(j1) and 1/A(j1) come from one rsqrt of the polynomial A^2 and are carried
// from step to step; the reciprocals 1/j1 come from the table rc (rc[j - rbase]
// = 1/j, correctly rounded, for every j1 + 1 of the chain).  Returns n (0 if
// the chain is empty).
template <int CMAX>
__device__ int threej_chain(int j2, int j3, int m2, int m3, double* f, double* bwd, int* j1min_out,
                            const double* rc, int rbase) {
  const int m1 = -m2 - m3;
  const int j1min = max(abs(j2 - j3), abs(m1));
  const int j1max = j2 + j3;
  *j1min_out = j1min;
  const int n = j1max - j1min + 1;
  if (n <= 0 || n > CMAX || abs(m2) > j2 || abs(m3) > j3) return 0;
  const double dj = (double)(j2 - j3), sj = (double)(j2 + j3 + 1), dm1 = (double)m1;
  const double bj = (double)j2 * (j2 + 1.0) * dm1 - (double)j3 * (j3 + 1.0) * dm1;
  const double dm = (double)(m3 - m2);
  auto A2 = [&](int j1) -> double {
    const double x = (double)j1;
    const double v = (x * x - dj * dj) * (sj * sj - x * x) * (x * x - dm1 * dm1);
    return v > 0.0 ? v : 0.0;
  };
  auto B = [&](int j1) -> double {
    const double x = (double)j1;
    return -(2.0 * x + 1.0) * (bj - x * (x + 1.0) * dm);
  };
  if (n == 1) {
    f[0] = 1.0;
  } else {
    // forward: A(j1) carried in acur (A(j1min) is 0 or irrelevant: f(j1min-1) = 0)
    f[0] = 1.0;
    int kf = 0;
    double acur = sqrt(A2(j1min));
    auto fstep = [&](int i) {
      const int j1 = j1min + i;
      const double p2 = A2(j1 + 1);
      const double rn = rsqrt(p2);
      if (j1 == 0) {
        f[1] = (double)m2 * rsqrt((double)j2 * (j2 + 1.0));
      } else {
        const double prev = i > 0 ? f[i - 1] : 0.0;
        f[i + 1] = -(B(j1) * f[i] + (j1 + 1.0) * acur * prev) * rn * rc[j1 - rbase];
      }
      acur = p2 * rn;
    };
    while (kf + 1 < n) {
      fstep(kf);
      ++kf;
      if (fabs(f[kf]) < fabs(f[kf - 1])) break;
    }
    // backward: A(j1+1) carried in anext (A(j1max+1) = 0)
    bwd[n - 1] = 1.0;
    int kb = n - 1;
    double anext = 0.0;
    while (kb - 1 >= 0) {
      const int j1 = j1min + kb;
      const double p2 = A2(j1);
      const double r = rsqrt(p2);
      const double nxt = (kb + 1 < n) ? bwd[kb + 1] : 0.0;
      bwd[kb - 1] = -(B(j1) * bwd[kb] + j1 * anext * nxt) * r * rc[j1 + 1 - rbase];
      anext = p2 * r;
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
  double scale = rsqrt(norm);
  const double want = ((j2 - j3 - m1) & 1) ? -1.0 : 1.0;
  if (f[n - 1] * want < 0.0) scale = -scale;
  for (int i = 0; i < n; ++i) f[i] *= scale;
  return n;
}

// Shared per-pair tables of a CTA (couple_setup): w0s, the (l' p l; 0 0 0)
// family of every p < Lh by the two-term relation
//   f(j1+1) = -sqrt((j1^2-d^2)(S^2-j1^2) / (((j1+1)^2-d^2)(S^2-(j1+1)^2))) f(j1-1),
// d = p - l, S = p + l + 1, over the even j1 + p + l, normalised by
// sum (2 j1 + 1) f^2 = 1 with sgn f(p + l) = (-1)^{p-l}, stored already
// multiplied by the rest of T that does not depend on q or the chain:
// (-1)^m sqrt((2p+1)(2l+1)/(4 pi)) sqrt(2 l' + 1); and rcs, the reciprocals
// 1/j for j in [rbase, l + Lh] (every j1 + 1 of the pair's chains, rbase =
// max(0, l - Lh + 1)) for threej_chain.  Every thread of the block takes
// part (the block may call it again after it).
#define COUPLE_RCS (2 * SLSHT_MAX_LH + 2)
__device__ __forceinline__ int couple_setup(int Lh, int l, int m, double* w0s, double* rcs) {
  __syncthreads();                              // the tables of a previous call are read
  const int rbase = max(0, l - Lh + 1);
  for (int i = threadIdx.x; i <= l + Lh - rbase; i += blockDim.x) {
    const int j = rbase + i;
    rcs[i] = j > 0 ? 1.0 / (double)j : 0.0;
  }
  for (int p = threadIdx.x; p < Lh; p += blockDim.x) {
    double* w = w0s + p * (p + 1) / 2;
    const int j0 = abs(p - l), cnt = min(p, l) + 1;
    const double dd = (double)(p - l), SS = (double)(p + l + 1);
    double v = 1.0, norm = 2.0 * j0 + 1.0;
    w[0] = 1.0;
    for (int i = 1; i < cnt; ++i) {
      const double x = (double)(j0 + 2 * i - 1), y = x + 1.0;
      v *= -sqrt(((x * x - dd * dd) * (SS * SS - x * x)) / ((y * y - dd * dd) * (SS * SS - y * y)));
      w[i] = v;
      norm += (2.0 * (j0 + 2 * i) + 1.0) * v * v;
    }
    double s0 = rsqrt(norm);
    const double want = ((p - l) & 1) ? -1.0 : 1.0;
    if (v * want < 0.0) s0 = -s0;
    const double pre = ((m & 1) ? -1.0 : 1.0) *
                       sqrt((2.0 * p + 1.0) * (2.0 * l + 1.0) / (4.0 * 3.14159265358979323846));
    for (int i = 0; i < cnt; ++i) w[i] *= s0 * pre * sqrt(2.0 * (j0 + 2 * i) + 1.0);
  }
  __syncthreads();
  return rbase;
}

// (p, q) of item t = p*p + p + q
__device__ __forceinline__ void couple_item(int t, int* p_out, int* q_out) {
  int p = (int)sqrt((double)t);
  while (p * p > t) --p;
  while ((p + 1) * (p + 1) <= t) ++p;
  *p_out = p;
  *q_out = t - p * p - p;
}

// One pair's k_lm(p, q), every item t = p*p + p + q, by one CTA: item (p, q)
// runs the (l' p l; m-q q -m) chain and accumulates
//   k_lm(p, q) = sum_l' f_{l', m-q} T(l', m-q; p, q; l, m).
// Mirror items share their chain: with q -> -q and m -> -m,
//   (l' p l; -m+q, -q, m) = (-1)^{l'+p+l} (l' p l; m-q, q, -m),
// and l'+p+l is even wherever (l' p l; 0 0 0) is non-zero, so item (p, -q)
// of the pair (l, -m) has the same T with f_{l', -(m-q)}: kcm (nullable) is
// that pair's k row, filled from the same chains; for m = 0 the pair is its
// own mirror and only the items q >= 0 run chains (q > 0 also fill (p, -q)).
template <int CMAX>
__device__ __forceinline__ void couple_pair_chains(const double2* __restrict__ f, int Lf, int Lh, int l, int m,
                                                   double2* __restrict__ kc, double2* __restrict__ kcm, double* w0s,
                                                   double* rcs) {
  const int rbase = couple_setup(Lh, l, m, w0s, rcs);
  const int nitems = Lh * Lh;
  const bool self = m == 0;
  double fm[CMAX], bwd[CMAX];
  for (int t = threadIdx.x; t < nitems; t += blockDim.x) {
    int p, q;
    couple_item(t, &p, &q);
    if (self && q < 0) continue;                    // filled by the item (p, -q)
    const bool two = kcm != nullptr || (self && q > 0);
    double2 acc = make_double2(0.0, 0.0), accm = make_double2(0.0, 0.0);
    int j1min_m;
    const int nm = threej_chain<CMAX>(p, l, q, -m, fm, bwd, &j1min_m, rcs, rbase);
    if (nm > 0) {
      const double* w = w0s + p * (p + 1) / 2;
      const int j0 = abs(p - l);
      const int mu = m - q;
      const int jend = min(p + l, Lf - 1);
      // l' = j0 + 2i, l' >= j1min_m
      int i0 = (j1min_m - j0 + 1) / 2;
      if (i0 < 0) i0 = 0;
      for (int j1 = j0 + 2 * i0; j1 <= jend; j1 += 2) {
        const double c = w[(j1 - j0) >> 1] * fm[j1 - j1min_m];
        const double2 fv = f[j1 * j1 + j1 + mu];
        acc.x = fma(c, fv.x, acc.x);
        acc.y = fma(c, fv.y, acc.y);
        if (two) {
          const double2 fw = f[j1 * j1 + j1 - mu];
          accm.x = fma(c, fw.x, accm.x);
          accm.y = fma(c, fw.y, accm.y);
        }
      }
    }
    kc[t] = acc;
    if (kcm != nullptr) kcm[p * p + p - q] = accm;
    else if (self && q > 0) kc[p * p + p - q] = accm;
  }
}

// One CTA per work item: pair work[i].x, and the mirror pair work[i].y
// (l, -m) filled from the same chains (-1: none); without a work list, one
// CTA per pair.
template <int CMAX>
__global__ void __launch_bounds__(256) k_couple(const double2* __restrict__ f, int Lf, int Lh,
                                                const int2* __restrict__ lm, const int2* __restrict__ work,
                                                double2* __restrict__ kc) {
  __shared__ double w0s[SLSHT_MAX_LH * (SLSHT_MAX_LH + 1) / 2];
  __shared__ double rcs[COUPLE_RCS];
  const int2 wk = work != nullptr ? work[blockIdx.x] : make_int2((int)blockIdx.x, -1);
  const size_t n2 = (size_t)Lh * Lh;
  couple_pair_chains<CMAX>(f, Lf, Lh, lm[wk.x].x, lm[wk.x].y, kc + (size_t)wk.x * n2,
                           wk.y >= 0 ? kc + (size_t)wk.y * n2 : nullptr, w0s, rcs);
}

// The same for the pairs of many couplings (serving ticks): blocks stride
// over the list of *n work items {coupling + SERVE_CPL_MAX (mirror + 1), pair}
// (serve_couple_entry), pair and mirror indices within the coupling's list.
template <int CMAX>
__global__ void __launch_bounds__(256) k_serve_couple(const BCouple* __restrict__ cpl, const int2* __restrict__ list,
                                                      const int* __restrict__ n) {
  __shared__ double w0s[SLSHT_MAX_LH * (SLSHT_MAX_LH + 1) / 2];
  __shared__ double rcs[COUPLE_RCS];
  const int cnt = *n;
  for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
    const int2 e = list[i];
    const int ci = e.x % SERVE_CPL_MAX, mir = e.x / SERVE_CPL_MAX - 1;
    const BCouple c = cpl[ci];
    const int2 pr = c.lm[e.y];
    const size_t n2 = (size_t)c.Lh * c.Lh;
    couple_pair_chains<CMAX>(c.f, c.Lf, c.Lh, pr.x, pr.y, c.kc + (size_t)e.y * n2,
                             mir >= 0 ? c.kc + (size_t)mir * n2 : nullptr, w0s, rcs);
  }
}

cudaError_t launch_serve_couple(int cls, const BCouple* cpl, const int2* list, const int* n, int grid,
                                cudaStream_t st) {
  if (cls == 0) k_serve_couple<32><<<grid, 256, 0, st>>>(cpl, list, n);
  else if (cls == 1) k_serve_couple<64><<<grid, 256, 0, st>>>(cpl, list, n);
  else k_serve_couple<128><<<grid, 256, 0, st>>>(cpl, list, n);
  return cudaGetLastError();
}

cudaError_t launch_couple(const double2* f, int Lf, int Lh, const int2* lm, int npairs, double2* kc, cudaStream_t st,
                          const int2* work, int nwork) {
  if (npairs <= 0) return cudaSuccess;
  const int threads = Lh * Lh < 256 ? ((Lh * Lh + 31) / 32) * 32 : 256;
  const int grid = work != nullptr ? nwork : npairs;
  // same carveout as the kernels it runs beside (see the tensor-core alpha stage)
  cudaFuncSetAttribute(k_couple<32>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_couple<64>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_couple<128>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (Lh <= 16) k_couple<32><<<grid, threads, 0, st>>>(f, Lf, Lh, lm, work, kc);
  else if (Lh <= 32) k_couple<64><<<grid, threads, 0, st>>>(f, Lf, Lh, lm, work, kc);
  else k_couple<128><<<grid, threads, 0, st>>>(f, Lf, Lh, lm, work, kc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- cached form
// The coupling splits into a signal-independent table and a gather:
//   k_lm(p, q) = sum_i c_i(l, m; p, q) f_{l'_i, m-q},   l'_i = l'_0 + 2 i,
//   c_i = T(l'_i, m-q; p, q; l, m)   (both 3j families, FP64, as in k_couple).
// k_gaunt_table writes c[pair][i][t] (i < Lh, zero past the item's count;
// t = p*p + p + q fastest) and meta[pair][t] = (l'_0, count); the table
// depends only on (L_f, L_h, the pair list), so a caller that repeats a pair
// list for many signals builds it once, like the Delta and d(beta) tables.
// Mirror pairs share their chains: with q -> -q,
//   (l' p l; -m+q, -q, m) = (-1)^{l'+p+l} (l' p l; m-q, q, -m)
// and l'+p+l is even wherever (l' p l; 0 0 0) is non-zero, so
// T(l', -m+q; p, -q; l, -m) = T(l', m-q; p, q; l, m) with the same l' range:
// work item w = (pair, mirror) fills item (p, q) of `pair` and item (p, -q) of
// `mirror` (when mirror >= 0) from one chain; a pair with m = 0 is its own
// mirror (its items q > 0 also fill (p, -q)).
template <int CMAX>
__global__ void __launch_bounds__(256) k_gaunt_table(int Lf, int Lh, const int2* __restrict__ lm,
                                                     const int2* __restrict__ work, double* __restrict__ coef,
                                                     int2* __restrict__ meta) {
  __shared__ double w0s[SLSHT_MAX_LH * (SLSHT_MAX_LH + 1) / 2];
  __shared__ double rcs[COUPLE_RCS];
  const int pair = work[blockIdx.x].x, mirror = work[blockIdx.x].y;
  const int l = lm[pair].x, m = lm[pair].y;
  const int rbase = couple_setup(Lh, l, m, w0s, rcs);
  const int n2 = Lh * Lh;
  // the item (p, -q) that shares the chain of (p, q): the mirror pair's, or,
  // for m = 0, the pair's own (then only the items q >= 0 run chains)
  const bool self = m == 0;
  double fm[CMAX], bwd[CMAX];
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    int p, q;
    couple_item(t, &p, &q);
    if (self && q < 0) continue;
    const int tm = p * p + p - q;
    const int opair = mirror >= 0 ? mirror : (self && q > 0 ? pair : -1);
    int j1min_m, first = 0, cnt = 0;
    const int nm = threej_chain<CMAX>(p, l, q, -m, fm, bwd, &j1min_m, rcs, rbase);
    if (nm > 0) {
      const double* w = w0s + p * (p + 1) / 2;
      const int j0 = abs(p - l);
      const int jend = min(p + l, Lf - 1);
      int i0 = (j1min_m - j0 + 1) / 2;
      if (i0 < 0) i0 = 0;
      first = j0 + 2 * i0;
      for (int j1 = first; j1 <= jend; j1 += 2, ++cnt) {
        const double c = w[(j1 - j0) >> 1] * fm[j1 - j1min_m];
        coef[((size_t)pair * Lh + cnt) * n2 + t] = c;
        if (opair >= 0) coef[((size_t)opair * Lh + cnt) * n2 + tm] = c;
      }
    }
    for (int i = cnt; i < Lh; ++i) {
      coef[((size_t)pair * Lh + i) * n2 + t] = 0.0;
      if (opair >= 0) coef[((size_t)opair * Lh + i) * n2 + tm] = 0.0;
    }
    meta[(size_t)pair * n2 + t] = make_int2(first, cnt);
    if (opair >= 0) meta[(size_t)opair * n2 + tm] = make_int2(first, cnt);
  }
}

// k_lm(p, q) from the table: one thread per (pair, t), coefficient rows
// read coalesced across t, f gathered (L2 resident); body couple_apply_one
// (couple_dev.cuh).
__global__ void __launch_bounds__(256) k_couple_apply(const double2* __restrict__ f, int Lh, const int2* __restrict__ lm,
                                                      const double* __restrict__ coef, const int2* __restrict__ meta,
                                                      int npairs, double2* __restrict__ kc) {
  const int n2 = Lh * Lh;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)npairs * n2) return;
  const int pair = (int)(idx / n2), t = (int)(idx % n2);
  kc[idx] = couple_apply_one(f, Lh, lm[pair].y, coef + (size_t)pair * Lh * n2, meta[idx], t);
}

size_t gaunt_table_bytes(int Lh, int npairs) {
  const size_t n2 = (size_t)Lh * Lh;
  return (size_t)npairs * (n2 * Lh * sizeof(double) + n2 * sizeof(int2));
}

cudaError_t launch_gaunt_table(int Lf, int Lh, const int2* lm, int npairs, const int2* work, int nwork, void* table,
                               cudaStream_t st) {
  if (npairs <= 0 || nwork <= 0) return cudaSuccess;
  const int threads = Lh * Lh < 256 ? ((Lh * Lh + 31) / 32) * 32 : 256;
  double* coef = (double*)table;
  int2* meta = (int2*)(coef + (size_t)npairs * Lh * Lh * Lh);
  if (Lh <= 16) k_gaunt_table<32><<<nwork, threads, 0, st>>>(Lf, Lh, lm, work, coef, meta);
  else if (Lh <= 32) k_gaunt_table<64><<<nwork, threads, 0, st>>>(Lf, Lh, lm, work, coef, meta);
  else k_gaunt_table<128><<<nwork, threads, 0, st>>>(Lf, Lh, lm, work, coef, meta);
  return cudaGetLastError();
}

cudaError_t launch_couple_apply(const double2* f, int Lh, const int2* lm, int npairs, const void* table, double2* kc,
                                cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  const double* coef = (const double*)table;
  const int2* meta = (const int2*)(coef + (size_t)npairs * Lh * Lh * Lh);
  const long long n = (long long)npairs * Lh * Lh;
  k_couple_apply<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(f, Lh, lm, coef, meta, npairs, kc);
  return cudaGetLastError();
}
