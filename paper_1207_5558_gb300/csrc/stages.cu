// beta and gamma stages of the forward transform.
//
// The distribution is (Eq. alternative_harmonic_formulation_wigner)
//   g(a, b, c) = sum_q e^{-i q alpha_a} sum_q' e^{-i q' gamma_c}
//                sum_p k(p, q) h_p^{q'} d^p_{q,q'}(beta_b).
// The innermost p sum ("beta stage") is done either
//   * directly with a table of d^p_{q,q'}(beta_b) (separation of variables,
//     the alternative remark of Sec. IV-B), or
//   * by the factoring of rotations: the C tensor of
//     Eq. constant_alternative_formulation followed by a DFT over q''
//     (Eq. alternative_harmonic_formulation_2_2),
// and both feed the same gamma sum, which also forms the +-q pairs the alpha
// stage consumes.
#include <algorithm>

#include "stages_dev.cuh"

// ---------------------------------------------------------------------------
// C_{q,q',q''} = i^{q-q'} sum_{p >= max(|q|,|q'|,|q''|)} Delta^p_{q''q} Delta^p_{q''q'} k(p,q) h_p^{q'}
// One CTA per pair, threads over the K^3 entries; layout [pair][q][q'][q''].
__global__ void k_ctensor(const double2* __restrict__ kc, const double2* __restrict__ h,
                          const double* __restrict__ D, int Lh, double2* __restrict__ C) {
  const int pair = blockIdx.y;
  const int K = 2 * Lh - 1;
  const long long n3 = (long long)K * K * K;
  const double2* kp = kc + (size_t)pair * Lh * Lh;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n3;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / ((long long)K * K)) - (Lh - 1);
    const int qp = (int)((t / K) % K) - (Lh - 1);
    const int qpp = (int)(t % K) - (Lh - 1);
    const int p0 = max(abs(q), max(abs(qp), abs(qpp)));
    double re = 0.0, im = 0.0;
    for (int p = p0; p < Lh; ++p) {
      const int W = 2 * p + 1;
      const double* blk = D + blk_off(p);
      const double dd = blk[(qpp + p) * W + (q + p)] * blk[(qpp + p) * W + (qp + p)];
      const double2 kv = kp[p * p + p + q], hv = h[p * p + p + qp];
      const double khr = kv.x * hv.x - kv.y * hv.y, khi = kv.x * hv.y + kv.y * hv.x;
      re = fma(dd, khr, re);
      im = fma(dd, khi, im);
    }
    double2 v;
    switch ((((q - qp) % 4) + 4) % 4) {        // multiply by i^{q-q'}
      case 0: v = make_double2(re, im); break;
      case 1: v = make_double2(-im, re); break;
      case 2: v = make_double2(-re, -im); break;
      default: v = make_double2(im, -re); break;
    }
    C[(size_t)pair * n3 + t] = v;
  }
}

cudaError_t launch_ctensor(const double2* kc, const double2* h, const double* D, int Lh,
                           int npairs, double2* C, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  const int K = 2 * Lh - 1;
  const long long n3 = (long long)K * K * K;
  dim3 grid((unsigned)((n3 + 255) / 256 < 64 ? (n3 + 255) / 256 : 64), npairs);
  k_ctensor<<<grid, 256, 0, st>>>(kc, h, D, Lh, C);
  return cudaGetLastError();
}

// Y[pair][b][q][q'] = sum_{q''} C[q][q'][q''] e^{-i q'' beta_b}: one CTA per
// (pair, q), the C slice C[q][:][:] staged in shared memory.
__global__ void k_beta_dft(const double2* __restrict__ C, int Lh, int Nb, double2* __restrict__ Y) {
  extern __shared__ double2 sC[];                // [K(q')][K(q'')]
  const int K = 2 * Lh - 1;
  const int qi = blockIdx.x, pair = blockIdx.y;
  const double2* src = C + ((size_t)pair * K + qi) * K * K;
  for (int t = threadIdx.x; t < K * K; t += blockDim.x) sC[t] = src[t];
  __syncthreads();
  const long long M = 2LL * Nb - 1;
  for (int t = threadIdx.x; t < K * Nb; t += blockDim.x) {
    const int b = t / K, qpi = t % K;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < K; ++k) {
      const int qpp = k - (Lh - 1);
      double s, c;
      sincos_2pi_frac((long long)qpp * b, M, &s, &c);
      const double2 v = sC[qpi * K + k];       // v * (c - i s)
      re += v.x * c + v.y * s;
      im += v.y * c - v.x * s;
    }
    Y[(((size_t)pair * Nb + b) * K + qi) * K + qpi] = make_double2(re, im);
  }
}

cudaError_t launch_beta_dft(const double2* C, int Lh, int Nb, int npairs, double2* Y,
                            cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  const int K = 2 * Lh - 1;
  const size_t smem = (size_t)K * K * sizeof(double2);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_beta_dft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(K, npairs);
  k_beta_dft<<<grid, 256, smem, st>>>(C, Lh, Nb, Y);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// beta + gamma for one (pair, beta row):
//   G[q][q'] = sum_p k(p,q) h_p^{q'} d^p_{q,q'}(beta_b)   (or G = Y[pair][b])
//   X_q[c]   = sum_q' G[q][q'] e^{-i q' gamma_c}
//            = G[q][0] + sum_{s>=1} (G[q][s] + G[q][-s]) cos(s gamma_c)
//                      - i (G[q][s] - G[q][-s]) sin(s gamma_c)        (+-q' paired)
// and the +-q pairs for the alpha stage: Xs[c=0] = X_0, Xs[2r-1] = X_r + X_-r,
// Xs[2r] = X_r - X_-r.  T is the arithmetic type of the sums.
template <typename T>
__global__ void k_betagamma(const double2* __restrict__ kc, const double2* __restrict__ h,
                            const T* __restrict__ dt, const double2* __restrict__ Y,
                            const typename vec2<T>::t* __restrict__ eg, int Lh, int Nb, int Ng,
                            typename vec2<T>::t* __restrict__ Xs) {
  typedef typename vec2<T>::t T2;
  extern __shared__ unsigned char smem_raw[];
  const int K = 2 * Lh - 1;
  const int LhP = Lh + 1;                         // padded row: rows q, q+1 on different banks
  const int b = blockIdx.x, pair = blockIdx.y;
  T2* sk = reinterpret_cast<T2*>(smem_raw);      // [Lh*Lh]
  T2* sh = sk + Lh * Lh;                          // [Lh*Lh]
  T2* sGp = sh + Lh * Lh;                         // [K][LhP]  G[q][s] + G[q][-s] (s = 0: G[q][0])
  T2* sGm = sGp + K * LhP;                        // [K][LhP]  G[q][s] - G[q][-s]
  T2* sE = sGm + K * LhP;                         // [Lh][Ng] (cos, sin)(s gamma_c), c fastest
  const int n2 = Lh * Lh;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const double2 kv = kc[(size_t)pair * n2 + t], hv = h[t];
    sk[t] = mk2((T)kv.x, (T)kv.y);
    sh[t] = mk2((T)hv.x, (T)hv.y);
  }
  for (int t = threadIdx.x; t < Ng * Lh; t += blockDim.x) {
    const int sidx = t / Ng, c = t % Ng;
    sE[t] = eg[c * K + sidx + (Lh - 1)];
  }
  __syncthreads();
  const int S = blk_off(Lh);
  const T* drow = dt ? dt + (size_t)b * S : nullptr;
  for (int t = threadIdx.x; t < K * Lh; t += blockDim.x) {
    const int qi = t / Lh, sidx = t % Lh;
    const int q = qi - (Lh - 1);
    T pr = 0, pim = 0, mr = 0, mim = 0;
    if (Y == nullptr) {
      for (int p = max(abs(q), sidx); p < Lh; ++p) {
        const T2 kv = sk[p * p + p + q];
        const int row = blk_off(p) + (q + p) * (2 * p + 1) + p;
        {
          const T2 hv = sh[p * p + p + sidx];
          const T d = drow[row + sidx];
          pr = fma(d, kv.x * hv.x - kv.y * hv.y, pr);
          pim = fma(d, kv.x * hv.y + kv.y * hv.x, pim);
        }
        if (sidx > 0) {
          const T2 hv = sh[p * p + p - sidx];
          const T d = drow[row - sidx];
          mr = fma(d, kv.x * hv.x - kv.y * hv.y, mr);
          mim = fma(d, kv.x * hv.y + kv.y * hv.x, mim);
        }
      }
    } else {
      const double2* src = Y + (((size_t)pair * Nb + b) * K + qi) * K;
      const double2 vp = src[sidx + Lh - 1];
      pr = (T)vp.x; pim = (T)vp.y;
      if (sidx > 0) { const double2 vm = src[-sidx + Lh - 1]; mr = (T)vm.x; mim = (T)vm.y; }
    }
    const int o = qi * LhP + sidx;
    if (sidx == 0) { sGp[o] = mk2(pr, pim); sGm[o] = mk2(pr, pim); }
    else { sGp[o] = mk2(pr + mr, pim + mim); sGm[o] = mk2(pr - mr, pim - mim); }
  }
  __syncthreads();
  const size_t J = (size_t)Nb * Ng;
  T2* out = Xs + (size_t)pair * K * J;
  for (int t = threadIdx.x; t < Lh * Ng; t += blockDim.x) {
    const int r = t / Ng, c = t % Ng;
    const T2* ap = sGp + (r + Lh - 1) * LhP;      // row q = +r
    const T2* am = sGm + (r + Lh - 1) * LhP;
    const T2* bp = sGp + (-r + Lh - 1) * LhP;     // row q = -r
    const T2* bm = sGm + (-r + Lh - 1) * LhP;
    T xr = ap[0].x, xi = ap[0].y, yr = bp[0].x, yi = bp[0].y;
    for (int sidx = 1; sidx < Lh; ++sidx) {       // (Gp cos - i Gm sin)
      const T2 E = sE[sidx * Ng + c];
      const T2 P1 = ap[sidx], M1 = am[sidx], P2 = bp[sidx], M2 = bm[sidx];
      xr = fma(P1.x, E.x, xr); xr = fma(M1.y, E.y, xr);
      xi = fma(P1.y, E.x, xi); xi = fma(-M1.x, E.y, xi);
      yr = fma(P2.x, E.x, yr); yr = fma(M2.y, E.y, yr);
      yi = fma(P2.y, E.x, yi); yi = fma(-M2.x, E.y, yi);
    }
    const size_t j = (size_t)b * Ng + c;
    if (r == 0) {
      out[j] = mk2(xr, xi);
    } else {
      out[(size_t)(2 * r - 1) * J + j] = mk2(xr + yr, xi + yi);
      out[(size_t)(2 * r) * J + j] = mk2(xr - yr, xi - yi);
    }
  }
}

template <typename T>
static cudaError_t launch_betagamma_t(const double2* kc, const double2* h, const T* dt,
                                      const double2* Y, const typename vec2<T>::t* eg, int Lh,
                                      int Nb, int Ng, int npairs, typename vec2<T>::t* Xs,
                                      cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  typedef typename vec2<T>::t T2;
  const int K = 2 * Lh - 1;
  const size_t smem = sizeof(T2) * ((size_t)2 * Lh * Lh + (size_t)2 * K * (Lh + 1) + (size_t)Ng * Lh);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_betagamma<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(Nb, npairs);
  k_betagamma<T><<<grid, 256, smem, st>>>(kc, h, dt, Y, eg, Lh, Nb, Ng, Xs);
  return cudaGetLastError();
}

cudaError_t launch_betagamma_f64(const double2* kc, const double2* h, const double* dt,
                                 const double2* Y, const double2* eg, int Lh, int Nb, int Ng,
                                 int npairs, double2* Xs, cudaStream_t st) {
  return launch_betagamma_t<double>(kc, h, dt, Y, eg, Lh, Nb, Ng, npairs, Xs, st);
}
cudaError_t launch_betagamma_f32(const double2* kc, const double2* h, const float* dt,
                                 const double2* Y, const float2* eg, int Lh, int Nb, int Ng,
                                 int npairs, float2* Xs, cudaStream_t st) {
  return launch_betagamma_t<float>(kc, h, dt, Y, eg, Lh, Nb, Ng, npairs, Xs, st);
}

// ---------------------------------------------------------------------------
// Rotated-window route.  Regrouping the sums of
// Eq. alternative_harmonic_formulation_wigner,
//   g(a, j) = sum_q e^{-i q alpha_a} sum_{p>=|q|} k(p,q) H^p_q(j),
//   H^p_q(j) = sum_{q'} h_p^{q'} d^p_{q,q'}(beta_b) e^{-i q' gamma_c},   j = b*Ng + c,
// H is the window's coefficients rotated by (0, beta_b, gamma_c) (Eq. rotation_non_symm
// with Eq. Dlm): it does not depend on the pair (l, m), so it is built once per call and
// every pair costs only Lh^2 multiply-adds per column.
// H in the tiled layout of h_index.  One CTA per (ROTWIN_NB beta rows,
// degree p, chunk): rotwin_block_smem_to (stages_dev.cuh).
template <typename T>
__global__ void __launch_bounds__(128) k_rotwin_smem(const double2* __restrict__ h, const T* __restrict__ dt,
                                                     const typename vec2<T>::t* __restrict__ eg, int Lh, int Nb,
                                                     int Ng, RotChunks ch, typename vec2<T>::t* __restrict__ H,
                                                     const uint32_t* __restrict__ qmask) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b0 = blockIdx.x * ROTWIN_NB, p = blockIdx.y;
  const int S = blk_off(Lh);
  rotwin_block_smem_to<T>(h, dt + (size_t)b0 * S + blk_off(p), (size_t)S, min(ROTWIN_NB, Nb - b0), eg, Lh, Ng, b0,
                          p, ch, blockIdx.z, RotwinStore<T>{H}, smem_raw, qmask);
}

// Active orders of a window (launch_order_mask): one block of 128 threads.
__global__ void __launch_bounds__(128) k_order_mask(const double2* __restrict__ h, int Lh, int rel_exp,
                                                    uint32_t* __restrict__ mask) {
  __shared__ double red[4];
  __shared__ uint32_t sm[4];
  const int n2 = Lh * Lh;
  double mx = 0.0;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const double2 v = h[t];
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  if (threadIdx.x < 4) sm[threadIdx.x] = 0u;
  __syncthreads();
  mx = fmax(fmax(red[0], red[1]), fmax(red[2], red[3]));
  const double eps = rel_exp > 0 ? ldexp(mx, -rel_exp) : 0.0;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    int p = (int)sqrtf((float)t);
    while (p * p > t) --p;
    while ((p + 1) * (p + 1) <= t) ++p;
    const int q = t - p * p - p;
    const double2 v = h[t];
    if (fabs(v.x) > eps || fabs(v.y) > eps) {
      const int bit = q + 63;
      atomicOr(&sm[bit >> 5], 1u << (bit & 31));
    }
  }
  __syncthreads();
  if (threadIdx.x < 4) mask[threadIdx.x] = sm[threadIdx.x];
}

cudaError_t launch_order_mask(const double2* h, int Lh, int rel_exp, uint32_t* mask, cudaStream_t st) {
  k_order_mask<<<1, 128, 0, st>>>(h, Lh, rel_exp, mask);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_rotwin_t(const double2* h, const T* dt, const typename vec2<T>::t* eg, int Lh,
                                   int Nb, int Ng, typename vec2<T>::t* H, cudaStream_t st, const uint32_t* qmask) {
  typedef typename vec2<T>::t T2;
  const RotChunks ch = rot_chunks(Lh, Ng, sizeof(T2));
  const size_t smem = ch.smem(Lh, sizeof(T2));
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_rotwin_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((Nb + ROTWIN_NB - 1) / ROTWIN_NB, Lh, ch.nq * ch.nc);
  k_rotwin_smem<T><<<grid, 128, smem, st>>>(h, dt, eg, Lh, Nb, Ng, ch, H, qmask);
  return cudaGetLastError();
}

cudaError_t launch_rotwin_f64(const double2* h, const double* dt, const double2* eg, int Lh, int Nb, int Ng,
                              double2* H, cudaStream_t st, const uint32_t* qmask) {
  return launch_rotwin_t<double>(h, dt, eg, Lh, Nb, Ng, H, st, qmask);
}
cudaError_t launch_rotwin_f32(const double2* h, const float* dt, const float2* eg, int Lh, int Nb, int Ng,
                              float2* H, cudaStream_t st, const uint32_t* qmask) {
  return launch_rotwin_t<float>(h, dt, eg, Lh, Nb, Ng, H, st, qmask);
}
