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
#include "common.cuh"

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
  const int b = blockIdx.x, pair = blockIdx.y;
  T2* sk = reinterpret_cast<T2*>(smem_raw);      // [Lh*Lh]
  T2* sh = sk + Lh * Lh;                          // [Lh*Lh]
  T2* sG = sh + Lh * Lh;                          // [K*K]
  T2* sE = sG + K * K;                            // [K][Ng] (cos, sin)(q' gamma_c), c fastest
  const int n2 = Lh * Lh;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) {
    const double2 kv = kc[(size_t)pair * n2 + t], hv = h[t];
    sk[t] = mk2((T)kv.x, (T)kv.y);
    sh[t] = mk2((T)hv.x, (T)hv.y);
  }
  for (int t = threadIdx.x; t < Ng * K; t += blockDim.x) {
    const int k = t / Ng, c = t % Ng;
    sE[t] = eg[c * K + k];
  }
  __syncthreads();
  if (Y == nullptr) {
    const int S = blk_off(Lh);
    const T* drow = dt + (size_t)b * S;
    for (int t = threadIdx.x; t < K * K; t += blockDim.x) {
      const int q = t / K - (Lh - 1), qp = t % K - (Lh - 1);
      const int p0 = max(abs(q), abs(qp));
      T re = 0, im = 0;
      for (int p = p0; p < Lh; ++p) {
        const T2 kv = sk[p * p + p + q], hv = sh[p * p + p + qp];
        const T d = drow[blk_off(p) + (q + p) * (2 * p + 1) + (qp + p)];
        const T khr = kv.x * hv.x - kv.y * hv.y, khi = kv.x * hv.y + kv.y * hv.x;
        re = fma(d, khr, re);
        im = fma(d, khi, im);
      }
      sG[t] = mk2(re, im);
    }
  } else {
    const double2* src = Y + ((size_t)pair * Nb + b) * K * K;
    for (int t = threadIdx.x; t < K * K; t += blockDim.x) {
      const double2 v = src[t];
      sG[t] = mk2((T)v.x, (T)v.y);
    }
  }
  __syncthreads();
  const size_t J = (size_t)Nb * Ng;
  T2* out = Xs + (size_t)pair * K * J;
  for (int t = threadIdx.x; t < Lh * Ng; t += blockDim.x) {
    const int r = t / Ng, c = t % Ng;
    const T2* gp = sG + (r + Lh - 1) * K;          // row q = +r
    const T2* gm = sG + (-r + Lh - 1) * K;         // row q = -r
    const T2* e = sE + c;                          // stride Ng: no bank conflicts across c
    T pr = 0, pi = 0, mr = 0, mi = 0;
    for (int k = 0; k < K; ++k) {                  // multiply by (cos - i sin)
      const T2 E = e[k * Ng], a = gp[k], bb = gm[k];
      pr = fma(a.x, E.x, pr); pr = fma(a.y, E.y, pr);
      pi = fma(a.y, E.x, pi); pi = fma(-a.x, E.y, pi);
      mr = fma(bb.x, E.x, mr); mr = fma(bb.y, E.y, mr);
      mi = fma(bb.y, E.x, mi); mi = fma(-bb.x, E.y, mi);
    }
    const size_t j = (size_t)b * Ng + c;
    if (r == 0) {
      out[j] = mk2(pr, pi);
    } else {
      out[(size_t)(2 * r - 1) * J + j] = mk2(pr + mr, pi + mi);
      out[(size_t)(2 * r) * J + j] = mk2(pr - mr, pi - mi);
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
  const size_t smem = sizeof(T2) * ((size_t)2 * Lh * Lh + (size_t)K * K + (size_t)Ng * K);
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
