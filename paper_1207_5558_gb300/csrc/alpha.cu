// alpha stage on CUDA cores (FP64 path; also an FP32 variant):
//   g[a][j] = sum_q X_q[j] e^{-i q alpha_a}
//           = X_0[j] + sum_{r=1}^{Lh-1} ( P_r[j] cos(r alpha_a) - i M_r[j] sin(r alpha_a) ),
// with P_r = X_r + X_-r and M_r = X_r - X_-r from the gamma stage: pairing +q
// and -q halves the multiply-adds of the direct sum (4(Lh-1) + 2 per sample).
// One thread per column j = (beta, gamma) sample; its 2Lh-1 coefficients sit
// in shared memory; each thread produces ABLK consecutive alpha rows per pass
// so a coefficient load feeds 4*ABLK fused multiply-adds.  Stores are
// coalesced: for a fixed row a, a warp writes 32 consecutive columns.
#include "common.cuh"

#define ABLK 4

// NT columns per CTA: 128, or 64 when the 2Lh-1 staged coefficients of 128
// columns would not fit in shared memory (FP64 at Lh = 64).
template <typename T, int NT>
__global__ void __launch_bounds__(NT)
k_alpha_cc(const typename vec2<T>::t* __restrict__ Xs, const typename vec2<T>::t* __restrict__ csa,
           int Lh, int Na, int J, typename vec2<T>::t* __restrict__ g, const int2* __restrict__ slots) {
  typedef typename vec2<T>::t T2;
  extern __shared__ unsigned char smem_raw[];
  T2* sx = reinterpret_cast<T2*>(smem_raw);      // [2Lh-1][NT]
  const int K = 2 * Lh - 1;
  const int pair = blockIdx.y;
  const int j0 = blockIdx.x * NT;
  const int t = threadIdx.x;
  const int j = j0 + t;
  const T2* src = Xs + (size_t)pair * K * J;
  for (int c = 0; c < K; ++c)
    sx[c * NT + t] = (j < J) ? src[(size_t)c * J + j] : mk2((T)0, (T)0);
  __syncthreads();
  if (j >= J) return;
  // output slot and, for a mirrored pair, the slot of (l, -m) with (-1)^m
  const int2 sl = slots != nullptr ? slots[pair] : make_int2(pair, -1);
  T2* dst = g + (size_t)sl.x * Na * J + j;
  T2* mdst = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + j : nullptr;
  const T ms = (sl.y & 1) ? (T)-1 : (T)1;
  const T2 x0 = sx[t];
  for (int a0 = 0; a0 < Na; a0 += ABLK) {
    T re[ABLK], im[ABLK];
#pragma unroll
    for (int u = 0; u < ABLK; ++u) { re[u] = x0.x; im[u] = x0.y; }
    for (int r = 1; r < Lh; ++r) {
      const T2 P = sx[(2 * r - 1) * NT + t];
      const T2 M = sx[(2 * r) * NT + t];
#pragma unroll
      for (int u = 0; u < ABLK; ++u) {
        const int a = min(a0 + u, Na - 1);
        const T2 cs = csa[(size_t)a * Lh + r];
        re[u] = fma(P.x, cs.x, re[u]);
        re[u] = fma(M.y, cs.y, re[u]);
        im[u] = fma(P.y, cs.x, im[u]);
        im[u] = fma(-M.x, cs.y, im[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < ABLK; ++u)
      if (a0 + u < Na) dst[(size_t)(a0 + u) * J] = mk2(re[u], im[u]);
    if (mdst != nullptr) {
#pragma unroll
      for (int u = 0; u < ABLK; ++u)
        if (a0 + u < Na) mdst[(size_t)(a0 + u) * J] = mk2(ms * re[u], -ms * im[u]);
    }
  }
}

template <typename T>
static cudaError_t launch_alpha_t(const typename vec2<T>::t* Xs, const typename vec2<T>::t* csa,
                                  int Lh, int Na, int J, int npairs, typename vec2<T>::t* g,
                                  const int2* slots, cudaStream_t st) {
  if (npairs <= 0 || J <= 0) return cudaSuccess;
  typedef typename vec2<T>::t T2;
  const size_t smem128 = sizeof(T2) * (size_t)(2 * Lh - 1) * 128;
  if (smem128 <= 200 * 1024) {
    if (smem128 > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_alpha_cc<T, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem128);
      if (e != cudaSuccess) return e;
    }
    dim3 grid((J + 127) / 128, npairs);
    k_alpha_cc<T, 128><<<grid, 128, smem128, st>>>(Xs, csa, Lh, Na, J, g, slots);
    return cudaGetLastError();
  }
  const size_t smem64 = smem128 / 2;
  if (smem64 > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_alpha_cc<T, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem64);
  if (e != cudaSuccess) return e;
  dim3 grid((J + 63) / 64, npairs);
  k_alpha_cc<T, 64><<<grid, 64, smem64, st>>>(Xs, csa, Lh, Na, J, g, slots);
  return cudaGetLastError();
}

cudaError_t launch_alpha_f64(const double2* Xs, const double2* csa, int Lh, int Na, int J,
                             int npairs, double2* g, const int2* slots, cudaStream_t st) {
  return launch_alpha_t<double>(Xs, csa, Lh, Na, J, npairs, g, slots, st);
}
cudaError_t launch_alpha_f32(const float2* Xs, const float2* csa, int Lh, int Na, int J,
                             int npairs, float2* g, const int2* slots, cudaStream_t st) {
  return launch_alpha_t<float>(Xs, csa, Lh, Na, J, npairs, g, slots, st);
}

// ---------------------------------------------------------------- split DFT
// The same alpha sum with the grid index split as a = Q s + t (Na = P Q, P a
// small odd factor): since e^{-i q alpha_a} = e^{-2 pi i q s / P} e^{-2 pi i q t / Na},
//   g[Q s + t] = sum_{r < P} e^{-2 pi i r s / P} Z_t(r),
//   Z_t(r)     = sum_{q = r (mod P)} X_q e^{-2 pi i q t / Na}.
// Per t a thread forms the P sums Z_t (one complex multiply-add per order q)
// and a P-point DFT with its odd symmetry folded,
//   y_0 = sum_r Z_r,  y_s, y_{P-s} = Z_0 + A_s -/+ i B_s,
//   A_s = sum_{r=1}^{(P-1)/2} (Z_r + Z_{P-r}) cos(2 pi r s / P),
//   B_s = sum_{r=1}^{(P-1)/2} (Z_r - Z_{P-r}) sin(2 pi r s / P),
// so a sample costs about 4(2Lh-1)/P + 10 real multiply-adds instead of
// 4(Lh-1)+2 (Lh = 16, P = 7: 28 instead of 62).  X_{+-r} are rebuilt from the
// paired coefficients, X_{+-r} = (P_r +- M_r) / 2.  tw[t * K + q + Lh - 1] =
// (cos, sin)(2 pi q t / Na) for t < Q.
template <typename T, int P, int NT>
__global__ void __launch_bounds__(NT)
k_alpha_split(const typename vec2<T>::t* __restrict__ Xs, const typename vec2<T>::t* __restrict__ tw, int Lh,
              int Na, int J, typename vec2<T>::t* __restrict__ g, const int2* __restrict__ slots) {
  typedef typename vec2<T>::t T2;
  constexpr int H = (P - 1) / 2;
  extern __shared__ unsigned char smem_raw[];
  T2* sx = reinterpret_cast<T2*>(smem_raw);      // [q + Lh - 1][NT]: X_q
  __shared__ T cpr[H + 1][H + 1], spr[H + 1][H + 1];   // cos / sin(2 pi r s / P), r, s >= 1
  const int K = 2 * Lh - 1, Q = Na / P;
  const int pair = blockIdx.y;
  const int t = threadIdx.x;
  const int j = blockIdx.x * NT + t;
  const T2* src = Xs + (size_t)pair * K * J;
  if (t < (H + 1) * (H + 1)) {
    const int r = t / (H + 1), s = t % (H + 1);
    double sv, cv;
    sincospi(2.0 * r * s / P, &sv, &cv);
    cpr[r][s] = (T)cv;
    spr[r][s] = (T)sv;
  }
  if (j < J) {
    const T2 x0 = src[j];
    sx[(Lh - 1) * NT + t] = x0;
    for (int r = 1; r < Lh; ++r) {
      const T2 pr = src[(size_t)(2 * r - 1) * J + j], mr = src[(size_t)(2 * r) * J + j];
      sx[(Lh - 1 + r) * NT + t] = mk2((T)0.5 * (pr.x + mr.x), (T)0.5 * (pr.y + mr.y));
      sx[(Lh - 1 - r) * NT + t] = mk2((T)0.5 * (pr.x - mr.x), (T)0.5 * (pr.y - mr.y));
    }
  }
  __syncthreads();
  if (j >= J) return;
  const int2 sl = slots != nullptr ? slots[pair] : make_int2(pair, -1);
  T2* dst = g + (size_t)sl.x * Na * J + j;
  T2* mdst = sl.y >= 0 ? g + (size_t)(sl.y >> 1) * Na * J + j : nullptr;
  const T ms = (sl.y & 1) ? (T)-1 : (T)1;
  // first order q >= -(Lh-1) of each residue class r (mod P)
  int qfirst[P];
#pragma unroll
  for (int r = 0; r < P; ++r) {
    int q = -(Lh - 1);
    q += (((r - q) % P) + P) % P;
    qfirst[r] = q;
  }
  for (int tt = 0; tt < Q; ++tt) {
    const T2* w = tw + (size_t)tt * K + (Lh - 1);
    T zr[P], zi[P];
#pragma unroll
    for (int r = 0; r < P; ++r) {
      T ar = 0, ai = 0;
      for (int q = qfirst[r]; q < Lh; q += P) {       // X_q e^{-i theta} = X_q (cos - i sin)
        const T2 x = sx[(q + Lh - 1) * NT + t];
        const T2 e = __ldg(w + q);
        ar = fma(x.x, e.x, ar); ar = fma(x.y, e.y, ar);
        ai = fma(x.y, e.x, ai); ai = fma(-x.x, e.y, ai);
      }
      zr[r] = ar;
      zi[r] = ai;
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
      for (int s = 0; s < P; ++s) mdst[(size_t)(Q * s + tt) * J] = mk2(ms * outr[s], -ms * outi[s]);
    }
  }
}

// The split factor for Na: the odd P in {9, 7, 5, 3} dividing Na with the
// fewest multiply-adds per sample (about 4K/P + P + 3), or 0 (direct sum).
int alpha_split_factor(int Lh, int Na) {
  const int K = 2 * Lh - 1;
  const double direct = 4.0 * (Lh - 1) + 2.0;
  int best = 0;
  double cost = direct;
  const int cand[4] = {9, 7, 5, 3};
  for (int i = 0; i < 4; ++i) {
    const int P = cand[i];
    if (Na % P != 0 || Na / P < 1) continue;
    const double c = 4.0 * K / P + P + 3.0;
    if (c < cost) { cost = c; best = P; }
  }
  return best;
}

template <typename T, int P>
static cudaError_t launch_split_p(const typename vec2<T>::t* Xs, const typename vec2<T>::t* tw, int Lh, int Na,
                                  int J, int npairs, typename vec2<T>::t* g, const int2* slots, cudaStream_t st) {
  typedef typename vec2<T>::t T2;
  const size_t smem128 = sizeof(T2) * (size_t)(2 * Lh - 1) * 128;
  if (smem128 <= 200 * 1024) {
    if (smem128 > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_alpha_split<T, P, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem128);
      if (e != cudaSuccess) return e;
    }
    dim3 grid((J + 127) / 128, npairs);
    k_alpha_split<T, P, 128><<<grid, 128, smem128, st>>>(Xs, tw, Lh, Na, J, g, slots);
    return cudaGetLastError();
  }
  const size_t smem64 = smem128 / 2;
  if (smem64 > 200 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_alpha_split<T, P, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem64);
  if (e != cudaSuccess) return e;
  dim3 grid((J + 63) / 64, npairs);
  k_alpha_split<T, P, 64><<<grid, 64, smem64, st>>>(Xs, tw, Lh, Na, J, g, slots);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_split_t(const typename vec2<T>::t* Xs, const typename vec2<T>::t* tw, int Lh, int Na,
                                  int J, int npairs, typename vec2<T>::t* g, const int2* slots, cudaStream_t st) {
  if (npairs <= 0 || J <= 0) return cudaSuccess;
  switch (alpha_split_factor(Lh, Na)) {
    case 9: return launch_split_p<T, 9>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
    case 7: return launch_split_p<T, 7>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
    case 5: return launch_split_p<T, 5>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
    case 3: return launch_split_p<T, 3>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_alpha_split_f64(const double2* Xs, const double2* tw, int Lh, int Na, int J, int npairs,
                                   double2* g, const int2* slots, cudaStream_t st) {
  return launch_split_t<double>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
}
cudaError_t launch_alpha_split_f32(const float2* Xs, const float2* tw, int Lh, int Na, int J, int npairs,
                                   float2* g, const int2* slots, cudaStream_t st) {
  return launch_split_t<float>(Xs, tw, Lh, Na, J, npairs, g, slots, st);
}
